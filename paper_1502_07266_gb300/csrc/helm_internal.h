// Internal declarations shared by the CUDA translation units of libhelm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/helm.h"

#define HELM_KMAX 64          // largest quasi-1D block (window lines x layers)
// HELM_MAX_BATCH (problems in one batched sweep launch) comes from helm.h

// One swept-axis block and its auxiliary window (Section 3 / 4.1 readings):
// the window covers nodes [lo, lo+L) and the block's own layers are
// [lo+ia, lo+ib).  One front: block 0 is the boundary PML slab [0, b), block
// M >= 1 starts at m = b + (M-1) d and its window is [m - b_aux, e) with a
// moving PML whose wall is at m - b_aux - 1 (clipped to [0, e) with the real
// profile when m - b_aux < 0).  Two fronts: the upper front's windows mirror
// these ([m, e + b_aux), wall at e + b_aux), the centre block's extends to both
// sides; a side without a moving PML keeps the global profile.
struct AxisWin {
    int lo, L, ia, ib;
    int moving;        // 1: moving PML on the low side, 0: global profile there
    int moving_hi;     // 1: moving PML on the high side, 0: global profile there
};

// One quasi-1D auxiliary problem (slab M, line block M').
struct Prob {
    int k;             // block size Ly * Lz
    int Ly, Lz;
    int ylo;           // first y node of the y-window
    int a0, ni;        // interest entries [a0, a0+ni) of an x-block (z fastest)
    int yb0, yb1;      // the line block's own lines [yb0, yb1) (global y)
    long long off;     // offset of T_0 in stored entries; T_i at off + i*kstride
    int kstride;       // k*ldk (whole 16-byte TMA granules in every format)
    int ldk;           // row stride of T_i in entries: k rounded up to a multiple of 8,
                       // + 2 (8-byte entries) or + 4 (4-byte entries) so that the 8 rows
                       // a quarter-warp reads at one column fall in distinct bank groups;
                       // columns [k, ldk) are zero except the block scale (row 0, last)
    int hp;            // column pairs per row, ceil(k/2)
    int pad_[2];
};

// Dense restricted operators (the alternative of Section 6 to the
// substitution chain): for each quasi-1D problem the map from its input
// entries to its output entries, G = R_out H~^{-1} R_in^T, stored densely.
// An index set is a union of "rects": lines [line0, line0+nl) (global y) x
// window z rows [z0, z0+nz) x every x.  Output entries are numbered rect by
// rect with x fastest (then z row, then line); input entries (one rect) with
// the z row fastest, then the line, x slowest:  j = zr + nz (l + nl x).
struct DRect { int line0, nl, z0, nz; };

struct DProb {
    int n_out, n_in;
    int nrect;          // output rects (1 or 2)
    int fp;             // quasi-1D problem (M*B + M') whose factors define H~
    DRect out[2];
    DRect in;
    int n_mt;           // output tiles of 64 + xr rows
    int KR;             // K-range of each of the 8 ranks of a cluster (multiple of 16)
    int nkc;            // K-chunks of at most 128 per rank
    int xr;             // extra rows per tile (0..2), stored in complex FP32 after the tile
    long long off;      // byte offset of the operator's tiles
    long long soff;     // float offset of its per-row scales (FP16 forms)
};

#define HELM_DENSE_CS 8   // CTAs per cluster in the dense apply (the K split)

struct Geom {
    int n, b, d, N, B, b_aux;
    int cen;           // the centre block: the last block of the forward passes (one front: B-1)
    int sched;         // HELM_ONE_FRONT or HELM_TWO_FRONT
    double h, omega, C;
    int Wmax;          // longest window
};

// Device-resident coefficient tables (all float2 = complex FP32 unless noted).
struct Tables {
    float2* s_node;    // [N]       global s at nodes
    float2* s_half;    // [N+1]     global s at g - 1/2, g = 0..N
    float2* c_dn;      // [N]       s(g) s(g-1/2) / h^2 : A's coupling g -> g-1
    float2* c_up;      // [N]       s(g) s(g+1/2) / h^2 : A's coupling g -> g+1
    float2* w_node;    // [B][Wmax]     window profile at nodes
    float2* w_half;    // [B][Wmax+1]   window profile at half points
    AxisWin* win;      // [B]
    float* kappa;      // [N^3]     omega^2 / c^2
    double* kappa64;   // [N^3]     the same in FP64 (for the FP64 residual)
    double2* c_dn64;   // [N]       c_dn in FP64
    double2* c_up64;   // [N]       c_up in FP64
    Prob* prob;        // [B*B]     problem p = M*B + M'
};

struct helm_ctx {
    Geom g;
    helm_opts opts;
    int device;
    Tables t;
    float2* factors;         // raw storage of the stored factors (format: opts.precision)
    size_t factor_elems;     // storage size in float2 units
    size_t factor_bytes;     // bytes of stored factors
    int esz;                 // bytes per stored entry: 8 (FP32, SPLIT_FP16) or 4 (FP16)
    int kmax;
    int stage_elems;         // largest kstride (stored entries)
    // sweep work space
    float2* slab;            // per CTA slab vectors
    size_t slab_elems;
    int sweep_rc;            // RHS per CTA
    int sweep_stages;
    size_t sweep_smem;
    int* dev_err;            // device error word (bounded waits)
    // adjoint right-hand side D g (grown on demand)
    float2* adj_buf;
    size_t adj_elems;
    // GMRES work space (grown on demand)
    void* gm_buf;
    // GMRES iterations captured as CUDA graphs (one per iteration index j of a
    // cycle), valid for the work space, right-hand-side count and options below
    void* gm_graphs;         // GmGraph[restart], owned by api.cu
    int gm_graph_R, gm_graph_timing;
    double gm_graph_tol;
    void* gm_graph_buf;
    void* gm_cap_stream;     // the stream graphs are captured on (cudaStream_t)
    size_t gm_bytes;
    long long launches;
    // batch handle (helm_setup_batch): owns nsub per-problem handles and no
    // tables of its own; its vectors are the problems' vectors back to back
    int nsub;
    struct helm_ctx* sub[HELM_MAX_BATCH];
    int sub_nrhs[HELM_MAX_BATCH];
    // opt-in kernel timing: pending (start, stop, kind, nrhs) event records
    int timing;
    void* tpending;          // std::vector<TimedLaunch>* (api.cu)
    helm_stats stats;
    // dense restricted-operator form (opts.apply_form == HELM_DENSE)
    int dense;
    DProb* dprob;            // device [B*B + B]: operator (M, M') at M*B+M'; first-block backward at B*B+M
    DProb* dprob_h;          // host copy
    Prob* prob_h;            // host copy of the quasi-1D problem table (B*B)
    unsigned char* dG;       // operator tiles
    size_t dG_bytes;
    float* dscale;           // per-row power-of-two scales (FP16 forms)
    size_t dscale_elems;
    float2* dV;              // apply work space: slab vector [line][z row][x][64 RHS], then the op counter
    size_t dV_elems;
    int dclus;               // clusters of HELM_DENSE_CS CTAs in the apply launch
    size_t dsmem;            // dynamic shared memory of the apply kernel
};

// Records events around a launch when timing is on (api.cu).
void helm_time_begin(helm_ctx* h, cudaStream_t st, void** ev0);
void helm_time_end(helm_ctx* h, cudaStream_t st, void* ev0, int kind, int nrhs);

// ---- error helpers -------------------------------------------------------
#define HELM_CUDA_TRY(expr)                                                  \
    do {                                                                     \
        cudaError_t _e = (expr);                                             \
        if (_e != cudaSuccess) {                                             \
            helm_set_cuda_error(_e);                                         \
            return (_e == cudaErrorMemoryAllocation) ? HELM_ENOMEM : HELM_ECUDA; \
        }                                                                    \
    } while (0)

void helm_set_cuda_error(cudaError_t e);

// Raises the dynamic shared-memory limit of kernel `fn` on the current device
// to at least `bytes`, never lowering it.  The limit is per-function state
// shared by every host thread, so a plain set before each launch would let one
// thread lower it between another thread's set and launch.
cudaError_t ensure_dyn_smem(const void* fn, size_t bytes);

// ---- kernel launchers (each returns a cudaError_t of its launch) --------
cudaError_t launch_coefficients(helm_ctx* h, const float* c, cudaStream_t st);
cudaError_t launch_factor(helm_ctx* h, cudaStream_t st);
// Factorisation of problems [p0, p0+np) into `dst`, whose entry 0 is factor
// entry off0 of the handle's layout (the dense setup works a chunk at a time).
cudaError_t launch_factor_range(helm_ctx* h, int p0, int np, float2* dst, long long off0, int fmt, cudaStream_t st);
// Dense form: setup (after the coefficients), apply, and the operator readback.
int dense_setup(helm_ctx* h, const void* win_host, const void* prob_host, cudaStream_t st);
int dense_rebuild(helm_ctx* h, int Ma, int Mb, int Pa, int Pb, cudaStream_t st);
cudaError_t sweep_prepare(helm_ctx* h, int nrhs, cudaStream_t st);
cudaError_t launch_dense_apply(helm_ctx* h, const float2* r, float2* z, int nrhs, float2* work, cudaStream_t st);
size_t dense_work_elems(const helm_ctx* h, int nrhs);
void dense_free(helm_ctx* h);
cudaError_t launch_stencil_c64(helm_ctx* h, const float2* x, float2* y, int nrhs, cudaStream_t st);
cudaError_t launch_stencil_c128(helm_ctx* h, const double2* x, double2* y, int nrhs, cudaStream_t st);
cudaError_t launch_residual_c128(helm_ctx* h, const float2* f, const double2* u, double2* r,
                                 int nrhs, cudaStream_t st);
cudaError_t launch_sweep(helm_ctx* h, const float2* r, float2* z, int nrhs, int slab_only,
                         int M_only, cudaStream_t st);
int sweep_configure(helm_ctx* h);
int sweep_config_stages(helm_ctx* h, int stages);
cudaError_t launch_sweep_batch(helm_ctx* const* hs, const float2* const* r, float2* const* z,
                               const int* nrhs, int n, cudaStream_t st);
cudaError_t launch_scale_D(helm_ctx* h, const float2* x, float2* y, int nrhs, int divide, cudaStream_t st);
cudaError_t launch_velocity_gradient(helm_ctx* h, const float2* lam, const float2* u, int nrhs, double* grad,
                                     cudaStream_t st);
