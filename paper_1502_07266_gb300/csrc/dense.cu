// Dense restricted-operator form of the recursive sweep.
//
// Section 6 notes that the quasi-1D solves of Algorithm 4 are the sequential
// bottleneck and can be restructured.  Every use of |T~_{M'}| in Algorithms 4
// and 6 maps the values on a few lines of the quasi-1D window to values on a
// few lines: |T~| = R_out H~^{-1} R_in^T.  This form stores that map densely
// (G, about 973 x 973 complex entries per problem at n = 127, b = 6, d = 1) and
// replaces each 2 N-step block substitution by one complex matrix product over
// all right-hand sides: the same preconditioner M up to rounding.
//
// Index sets (in the window of problem (M, M'); see DProb):
//   M' >= 1   in = out = the block's lines x every z row of the window.
//   M' = 0    forward:  in  = lines [0, b) x the slab's own layers [za, zb)
//                       out = lines [0, b-1) x [za, zb)  and  line b-1 x every z row
//             backward: in  = line b-1 x every z row
//                       out = lines [0, b) x [za, zb)
// (the first line block is only ever fed on its own layers, its backward input
// is the coupling into line b-1, and only the slab's own layers and the line
// that couples to M' = 1 are read from it).
//
// Setup: the quasi-1D problems are factored chunk by chunk (the twisted block
// LDU of factor.cu into a temporary buffer), k_dense_G solves with the unit
// columns of R_in^T and keeps the rows of R_out, and k_dense_pack stores G in
// the apply's tiles: complex FP32 for the SIMT form, FP16 hi + lo (or hi only)
// with one power-of-two scale per real row for the tensor-core forms.
//
// Apply: one persistent launch of clusters of 8 CTAs walks the (2B-1)^2 solves
// of Algorithm 6 over Algorithm 4 in order (dense_sched.h: with two fronts a
// step carries a lower-front and an upper-front solve on two groups of
// clusters).  A solve computes Y = G q for up to 64 right-hand sides: cluster c
// of its group takes 64-row output tiles c, c + ncl, ...; rank r of the cluster
// takes input entries [r KR, (r+1) KR).  Each CTA gathers its slice of q
// straight from the slab vector and the outer vectors (the couplings of
// Algorithms 4 and 6), multiplies it by its G tile (streamed by one thread
// through a shared-memory ring with bulk copies), the 8 partial products are
// summed through distributed shared memory, and the owner of each output row
// applies the step's update (store, subtract, restrict to the output).  Step
// s+1 starts when every CTA has arrived on a global counter for step s.  All waits are bounded by a clock limit; on expiry the kernel
// sets the error word, drains its copies, frees its TMEM and returns.
#include "helm_internal.h"
#include "ptx.cuh"

#include <cuda_fp16.h>
#include <string.h>

#include <algorithm>
#include <vector>

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Exponent of the power-of-two scale that puts a largest magnitude f 2^ex
// (f in [0.5, 1)) into [2^14, 2^15), clamped so that both the scale and its
// inverse stay normal FP32 numbers: an almost-zero row or column (below about
// 2^-105) is scaled by 2^120 only, its FP16 parts then losing digits that are
// negligible next to the other rows and columns of the product.
__host__ __device__ __forceinline__ int scale_exp(int ex) {
    const int e = 15 - ex;
    return e < -120 ? -120 : (e > 120 ? 120 : e);
}

// Bytes per K column of the main part of one stored tile: 64 complex rows in
// FP32 (512), or 128 real rows of FP16 hi + lo (512) or hi only (256).  A tile
// also carries xr extra complex rows in FP32 (8 bytes per row and K column).
int tile_unit(int precision) { return precision == HELM_FP16 ? 256 : 512; }

#include "dense_sched.h"

// ============================================================== setup ========

constexpr int GW = 64;      // input columns per setup work item
constexpr int GT = 128;     // threads of k_dense_G
constexpr int TLD = 68;     // row stride (complex) of the transposed factor block in shared memory

struct GItem { int p, j0; };

// T_i of the chunk's factors as a pointer (row-major, row stride ldk, complex FP32).
__device__ __forceinline__ const float2* fac_block(const float2* fac, const Prob& P, long long off0, int i) {
    return fac + (P.off - off0 + (long long)i * P.kstride);
}

// acc[8 rows][4 columns] = T W over the block's k columns; this thread's rows
// are 2 rg + 16 ii + e (ii < 4, e < 2), its columns 4 cg + cc.
__device__ __forceinline__ void setup_product(const float2* __restrict__ Tt, const float2* __restrict__ W, int k,
                                              int rg, int cg, float2 (&acc)[8][4]) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[q][cc] = make_float2(0.f, 0.f);
    for (int kk = 0; kk < k; ++kk) {
        const float4* tr = reinterpret_cast<const float4*>(Tt + kk * TLD + 2 * rg);
        const float4* wr = reinterpret_cast<const float4*>(W + kk * GW + 4 * cg);
        float2 a[8], b[4];
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
            const float4 v = tr[8 * ii];              // rows 2rg + 16 ii, +1
            a[2 * ii] = make_float2(v.x, v.y);
            a[2 * ii + 1] = make_float2(v.z, v.w);
        }
        const float4 w0 = wr[0], w1 = wr[1];
        b[0] = make_float2(w0.x, w0.y);
        b[1] = make_float2(w0.z, w0.w);
        b[2] = make_float2(w1.x, w1.y);
        b[3] = make_float2(w1.z, w1.w);
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) cfma(acc[q][cc], a[q], b[cc]);
    }
}

__device__ __forceinline__ int setup_row(int rg, int q) { return 2 * rg + 16 * (q >> 1) + (q & 1); }

// One work item = operator p, input columns [j0, j0 + GW).  X = H~^{-1} E with
// E the unit columns, by the twisted substitution of the factor layout
// (left chain T_0..T_{m-1}, right chain T_{N-1}..T_{m+1}, middle T_m):
//   left   y_i = T_i (e_i - cdn(i) y_{i-1})       from the first column's x up to m-1
//   right  y_i = T_i (e_i - cup(i) y_{i+1})       from the last column's x down to m+1
//   middle x_m = T_m (e_m - cdn(m) y_{m-1} - cup(m) y_{m+1})
//   back   x_i = y_i - cup(i) T_i x_{i+1}  (i < m),   x_i = y_i - cdn(i) T_i x_{i-1}  (i > m)
// (y is zero below the first column's x on the left and above the last
// column's x on the right).  Row a of x_i is written to G row so[a] + i.
__global__ void __launch_bounds__(GT)
k_dense_G(Geom g, Tables t, const DProb* __restrict__ dp, const GItem* __restrict__ items, int nitems,
          const float2* __restrict__ fac, long long off0, float2* __restrict__ Gt,
          const long long* __restrict__ goff, float2* __restrict__ yscr, size_t yslot) {
    extern __shared__ __align__(16) float2 gsm[];
    float2* Tt = gsm;                      // [64][TLD]: Tt[c][r] = T_i[r][c]
    float2* W = Tt + 64 * TLD;             // [64][GW]   product input
    float2* Xm = W + 64 * GW;              // [64][GW]   x_m for the second back pass
    int* sa = reinterpret_cast<int*>(Xm + 64 * GW);   // [GW] block row of column jj's unit entry
    int* sx = sa + GW;                     // [GW] x of column jj (-1: no column)
    int* so = sx + GW;                     // [64] output row of block row a at x = 0 (-1: not an output)
    const int tid = threadIdx.x;
    const int rg = tid & 7, cg = tid >> 3;
    const int N = g.N, m = (N - 1) / 2;
    float2* Y = yscr + (size_t)blockIdx.x * yslot;    // [N][64][GW] forward values

    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const GItem I = items[it];
        const DProb D = dp[I.p];
        const Prob P = t.prob[D.fp];
        const int k = P.k, Lz = P.Lz;
        float2* Gp = Gt + goff[I.p];
        __syncthreads();                   // previous item done with the shared arrays
        int xa = N, xb = -1;
        for (int jj = tid; jj < GW; jj += GT) {
            const int j = I.j0 + jj;
            int a = -1, x = -1;
            if (j < D.n_in) {
                const int per = D.in.nz * D.in.nl;
                x = j / per;
                const int r = j - x * per, l = r / D.in.nz;
                const int lz = D.in.z0 + (r - l * D.in.nz), line = D.in.line0 + l;
                a = lz + Lz * (line - P.ylo);
            }
            sa[jj] = a;
            sx[jj] = x;
        }
        for (int a = tid; a < 64; a += GT) {
            int o = -1;
            if (a < k) {
                const int lz = a % Lz, line = P.ylo + a / Lz;
                int base = 0;
                for (int q = 0; q < D.nrect; ++q) {
                    const DRect R = D.out[q];
                    if (line >= R.line0 && line < R.line0 + R.nl && lz >= R.z0 && lz < R.z0 + R.nz)
                        o = base + N * ((lz - R.z0) + R.nz * (line - R.line0));
                    base += R.nl * R.nz * N;
                }
            }
            so[a] = o;
        }
        for (int e = tid; e < 64 * TLD; e += GT) Tt[e] = make_float2(0.f, 0.f);
        __syncthreads();
        // first and last x of the item's columns (columns are in x order)
        xa = sx[0];
        {
            int last = GW - 1;
            while (last > 0 && sx[last] < 0) --last;
            xb = sx[last];
        }
        const bool do_left = xa < m, do_right = xb > m;
        const int jn = min(GW, D.n_in - I.j0);
        const int c0 = 4 * cg;

        // the step list: left forward, right forward, middle, back left, back right
        const int nlf = do_left ? m - xa : 0;
        const int nrf = do_right ? xb - m : 0;
        const int nsteps = nlf + nrf + 1 + m + (N - 1 - m);
        auto step_x = [&](int q) -> int {
            if (q < nlf) return xa + q;
            q -= nlf;
            if (q < nrf) return xb - q;
            q -= nrf;
            if (q == 0) return m;
            q -= 1;
            if (q < m) return m - 1 - q;
            return m + 1 + (q - m);
        };
        auto has_y = [&](int i) -> bool {
            return (i < m && do_left && i >= xa) || (i > m && do_right && i <= xb);
        };
        // load T of the first step (transposed)
        {
            const float2* T0 = fac_block(fac, P, off0, step_x(0));
            for (int e = tid; e < k * k; e += GT) {
                const int r = e / k, c = e - r * k;
                Tt[c * TLD + r] = T0[(size_t)r * P.ldk + c];
            }
        }
        // the first step's input: e at block step_x(0)
        {
            const int i0 = step_x(0);
            for (int e = tid; e < 64 * GW; e += GT) {
                const int a = e / GW, jj = e - a * GW;
                W[e] = make_float2((sx[jj] == i0 && sa[jj] == a) ? 1.f : 0.f, 0.f);
            }
        }
        __syncthreads();
        for (int q = 0; q < nsteps; ++q) {
            const int i = step_x(q);
            // prefetch the next step's factor block into registers
            constexpr int PF = (64 * 64 + GT - 1) / GT;
            float2 pf[PF];
            const bool more = q + 1 < nsteps;
            if (more) {
                const float2* Tn = fac_block(fac, P, off0, step_x(q + 1));
#pragma unroll
                for (int u = 0; u < PF; ++u) {
                    const int e = tid + u * GT;
                    pf[u] = make_float2(0.f, 0.f);
                    if (e < k * k) {
                        const int r = e / k, c = e - r * k;
                        pf[u] = Tn[(size_t)r * P.ldk + c];
                    }
                }
            }
            float2 acc[8][4];
            setup_product(Tt, W, k, rg, cg, acc);
            __syncthreads();                                   // Tt and W consumed
            if (more) {
#pragma unroll
                for (int u = 0; u < PF; ++u) {
                    const int e = tid + u * GT;
                    if (e < k * k) {
                        const int r = e / k, c = e - r * k;
                        Tt[c * TLD + r] = pf[u];
                    }
                }
            }
            const int inext = more ? step_x(q + 1) : -1;
            const bool fwd = q < nlf + nrf;                     // this step produced y_i
            const bool mid = q == nlf + nrf;
            // the next step's input, row by row of this thread's tile
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
                const int a = setup_row(rg, qq);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int jj = c0 + cc;
                    float2 val = acc[qq][cc];                   // T_i W
                    float2* ys = Y + ((size_t)i * 64 + a) * GW + jj;
                    if (fwd) {
                        *ys = val;                               // y_i
                    } else if (!mid) {
                        // back substitution: x_i = y_i - coupling * (T_i x_prev)
                        const float2 cp = (i < m) ? t.c_up[i] : t.c_dn[i];
                        const float2 yv = has_y(i) ? *ys : make_float2(0.f, 0.f);
                        val = csub(yv, cmul(cp, val));
                    }
                    if (!fwd) {                                  // val = x_i: output rows
                        if (mid) Xm[a * GW + jj] = val;
                        const int o = so[a];
                        if (o >= 0 && jj < jn) Gp[(size_t)(o + i) * D.n_in + I.j0 + jj] = val;
                    }
                    acc[qq][cc] = val;
                }
            }
            if (more) {
                // W for step q+1
                const bool nfwd = q + 1 < nlf + nrf, nmid = q + 1 == nlf + nrf;
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    const int a = setup_row(rg, qq);
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        const int jj = c0 + cc;
                        const float2 e = make_float2((sx[jj] == inext && sa[jj] == a) ? 1.f : 0.f, 0.f);
                        float2 w;
                        if (nfwd) {
                            const bool first = (q + 1 == 0) || (q + 1 == nlf);   // a chain starts at its end block
                            if (first) {
                                w = e;
                            } else {
                                const float2 cp = (inext < m) ? t.c_dn[inext] : t.c_up[inext];
                                w = csub(e, cmul(cp, acc[qq][cc]));
                            }
                        } else if (nmid) {
                            w = e;
                            if (do_left) w = csub(w, cmul(t.c_dn[m], Y[((size_t)(m - 1) * 64 + a) * GW + jj]));
                            if (do_right) w = csub(w, cmul(t.c_up[m], Y[((size_t)(m + 1) * 64 + a) * GW + jj]));
                        } else if (inext == m + 1) {
                            w = Xm[a * GW + jj];                 // the right back pass starts from x_m
                        } else {
                            w = acc[qq][cc];                     // x of the previous block
                        }
                        W[a * GW + jj] = w;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Real rows of an FP16 tile: the 64 complex rows' real parts and imaginary
// parts, interleaved in groups of 16 so that both parts of a complex row land
// in the same 32-lane quarter of the MMA accumulator (one warp reads both):
// tile row rho = 32 (i / 16) + 16 part + i mod 16 for complex row i.
__host__ __device__ __forceinline__ int tile_row(int i, int part) { return 32 * (i >> 4) + 16 * part + (i & 15); }
__host__ __device__ __forceinline__ int tile_cplx(int rho) { return 16 * (rho >> 5) + (rho & 15); }
__host__ __device__ __forceinline__ int tile_part(int rho) { return (rho >> 4) & 1; }

// Pack one output tile (operator p, 64 complex rows) into the apply's format.
struct PItem { int p, mt; };

template <int FMT>
__global__ void __launch_bounds__(256)
k_dense_pack(const DProb* __restrict__ dp, const PItem* __restrict__ items, const float2* __restrict__ Gt,
             const long long* __restrict__ goff, unsigned char* __restrict__ G, float* __restrict__ scale) {
    __shared__ float s_sc[128];
    __shared__ float2 stage[64][33];
    const PItem I = items[blockIdx.x];
    const DProb D = dp[I.p];
    const float2* src = Gt + goff[I.p];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_in = D.n_in;
    const int row0 = I.mt * (64 + D.xr);             // first output row of the tile
    if (FMT != HELM_FP32) {
        // one power-of-two scale per real row: its largest |part| into [2^14, 2^15)
        for (int rho = warp; rho < 128; rho += 8) {
            const int o = row0 + tile_cplx(rho), part = tile_part(rho);
            float mx = 0.f;
            if (o < D.n_out)
                for (int j = lane; j < n_in; j += 32) {
                    const float2 v = src[(size_t)o * n_in + j];
                    mx = fmaxf(mx, fabsf(part ? v.y : v.x));
                }
            for (int s = 16; s > 0; s >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
            if (lane == 0) {
                float sc = 1.f;
                if (mx > 0.f) {
                    int ex;
                    frexpf(mx, &ex);
                    sc = ldexpf(1.f, scale_exp(ex));
                }
                s_sc[rho] = sc;
                scale[D.soff + (long long)I.mt * 128 + rho] = sc;
            }
        }
        __syncthreads();
    }
    const int unit = (FMT == HELM_FP16) ? 256 : 512;
    const int unit_x = unit + 8 * D.xr;
    for (int r = 0; r < HELM_DENSE_CS; ++r) {
        for (int c = 0; c < D.nkc; ++c) {
            const int kw = min(128, D.KR - 128 * c);
            const int jb = r * D.KR + 128 * c;
            unsigned char* tile = G + D.off + ((long long)(I.mt * HELM_DENSE_CS + r) * D.KR + 128 * c) * unit_x;
            if (FMT == HELM_FP32) {
                // [kw][64] complex: element (kj, row) at kj * 64 + row
                float2* T = reinterpret_cast<float2*>(tile);
                for (int k0 = 0; k0 < kw; k0 += 32) {
                    __syncthreads();
                    for (int e = tid; e < 64 * 32; e += 256) {
                        const int row = e >> 5, kj = e & 31;
                        const int o = row0 + row, j = jb + k0 + kj;
                        stage[row][kj] = (row < 64 && o < D.n_out && j < n_in && k0 + kj < kw)
                                             ? src[(size_t)o * n_in + j] : make_float2(0.f, 0.f);
                    }
                    __syncthreads();
                    for (int e = tid; e < 64 * 32; e += 256) {
                        const int kj = e >> 6, row = e & 63;
                        if (k0 + kj < kw) T[(size_t)(k0 + kj) * 64 + row] = stage[row][kj];
                    }
                }
            } else {
                // 128 real rows (real and imaginary parts in the tile_row order) x kw,
                // FP16, K-major core-matrix layout; the lo tile follows the hi tile
                const int sbo = (kw / 8) * 128;
                for (int e = tid; e < 128 * (kw / 8); e += 256) {
                    const int rho = e / (kw / 8), kg = e - rho * (kw / 8);
                    const int o = row0 + tile_cplx(rho), part = tile_part(rho);
                    const float sc = s_sc[rho];
                    __align__(16) __half hi[8], lo[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = jb + 8 * kg + q;
                        float v = 0.f;
                        if (o < D.n_out && j < n_in) {
                            const float2 z = src[(size_t)o * n_in + j];
                            v = (part ? z.y : z.x) * sc;
                        }
                        hi[q] = __float2half_rn(v);
                        lo[q] = __float2half_rn(v - __half2float(hi[q]));
                    }
                    const size_t pos = (size_t)(rho >> 3) * sbo + (size_t)kg * 128 + (rho & 7) * 16;
                    *reinterpret_cast<uint4*>(tile + pos) = *reinterpret_cast<const uint4*>(hi);
                    if (FMT == HELM_SPLIT_FP16)
                        *reinterpret_cast<uint4*>(tile + (size_t)128 * kw * 2 + pos) = *reinterpret_cast<const uint4*>(lo);
                }
            }
            // extra rows: complex FP32 [xr][kw] after the main part
            float2* X = reinterpret_cast<float2*>(tile + (size_t)unit * kw);
            for (int e = tid; e < D.xr * kw; e += 256) {
                const int x = e / kw, kj = e - x * kw;
                const int o = row0 + 64 + x, j = jb + kj;
                X[e] = (o < D.n_out && j < n_in) ? src[(size_t)o * n_in + j] : make_float2(0.f, 0.f);
            }
        }
    }
}

// Read one stored operator back as complex FP32 [n_out][n_in] (for tests).
template <int FMT>
__global__ void k_dense_unpack(DProb D, const unsigned char* __restrict__ G, const float* __restrict__ scale,
                               float2* __restrict__ out) {
    const long long total = (long long)D.n_out * D.n_in;
    const int unit = (FMT == HELM_FP16) ? 256 : 512;
    const int unit_x = unit + 8 * D.xr, rows = 64 + D.xr;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(e / D.n_in), j = (int)(e - (long long)o * D.n_in);
        const int mt = o / rows, row = o - mt * rows;
        const int r = j / D.KR, jr = j - r * D.KR, c = jr >> 7, kj = jr & 127;
        const int kw = min(128, D.KR - 128 * c);
        const unsigned char* tile = G + D.off + ((long long)(mt * HELM_DENSE_CS + r) * D.KR + 128 * c) * unit_x;
        float2 v;
        if (row >= 64) {
            v = reinterpret_cast<const float2*>(tile + (size_t)unit * kw)[(size_t)(row - 64) * kw + kj];
        } else if (FMT == HELM_FP32) {
            v = reinterpret_cast<const float2*>(tile)[(size_t)kj * 64 + row];
        } else {
            const int sbo = (kw / 8) * 128;
            float part[2];
            for (int q = 0; q < 2; ++q) {
                const int rho = tile_row(row, q);
                const size_t pos = (size_t)(rho >> 3) * sbo + (size_t)(kj >> 3) * 128 + (rho & 7) * 16 + (kj & 7) * 2;
                float x = __half2float(*reinterpret_cast<const __half*>(tile + pos));
                if (FMT == HELM_SPLIT_FP16)
                    x += __half2float(*reinterpret_cast<const __half*>(tile + (size_t)128 * kw * 2 + pos));
                part[q] = x / scale[D.soff + (long long)mt * 128 + rho];
            }
            v = make_float2(part[0], part[1]);
        }
        out[e] = v;
    }
}

// ============================================================== apply ========

constexpr int DT = 256;                 // compute threads (8 warps)
constexpr int PT = 32;                  // the thread that issues the ring's copies (warp 1, lane 0)
constexpr int DSTAGES = 2;              // operator tiles in flight
constexpr int TILE_BYTES = 128 * 528;  // one ring stage: 128 K columns x (512 + 2 extra rows x 8) bytes
constexpr int PSTR = 132;               // partial-sum row stride in floats (re/im interleaved, TC forms;
                                        // 132 = 4 mod 32 banks: 16-byte stores of 8 rows hit distinct banks)
constexpr int BBUF_BYTES = 128 * PSTR * 4;   // B operand, then the partial sums
constexpr int PF_AHEAD = 4;             // tiles prefetched into L2 ahead of the ring
constexpr long long DEFAULT_WAIT = 4000000000ll;   // about 2 s at 2 GHz
// shared memory before the per-slab tables: ring, B / partials, column scales,
// gather plan, column maxima, extra-row partials, update operands, barriers,
// flags and the tile walk
constexpr int DENSE_SMEM_FIXED = DSTAGES * TILE_BYTES + BBUF_BYTES + 128 * 4 + 128 * 4 + 128 * 4 + 2 * 64 * 8 +
                                 3 * 256 * 8 + (DSTAGES + 3) * 8 + 16 + 2 * 48;

enum { FORM_FP32 = 0, FORM_SPLIT = 1, FORM_HI = 2 };

// Work space of one apply launch (R8 right-hand sides, right-hand side fastest):
//   V   [N lines][Wmax z rows][N x][R8]   forward values of the current slab
//   Q   [N lines][Wmax z rows][N x][R8]   inputs of the next solves: the line
//                                         couplings of Algorithm 4, written by
//                                         the solve that produces them
//   Gv  [N lines][DZ layers][N x][R8]     the slab's right-hand side on its own layers
//   Zv  [N lines][DZ layers][N x][R8]     the slab's restricted result
struct DenseArgs {
    Geom g;
    const AxisWin* win;
    const DProb* dp;
    const unsigned char* G;
    const float* scale;
    const float2* c_dn;
    const float2* c_up;
    const float2* rin;
    float2* zout;
    float2* V;
    float2* Q;
    float2* Gv;
    float2* Zv;
    unsigned* ctr;
    int* err;
    int nrhs, R8, nclus, nsteps, DZ;
    long long wait_cycles;
    int unmet;
    int unit;
};



__device__ __forceinline__ int vbase(const DenseArgs& A, int line, int lz, int x) {
    return ((line * A.g.Wmax + lz) * A.g.N + x) * A.R8;
}
__device__ __forceinline__ int zbase(const DenseArgs& A, int line, int zr, int x) {
    return ((line * A.DZ + zr) * A.g.N + x) * A.R8;
}

__device__ __forceinline__ void named_sync_compute() { asm volatile("bar.sync 1, %0;" ::"n"(DT) : "memory"); }

// Bounded wait on an mbarrier phase; gives up after `limit` cycles or when
// *stop is set (stop may be null).
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t ph, long long limit, bool cluster_scope,
                                         volatile int* stop) {
    const long long t0 = clock64();
    for (;;) {
        if (cluster_scope ? ptx::mbar_try_cluster(bar, ph) : ptx::mbar_try(bar, ph)) return true;
        if (clock64() - t0 > limit) return false;
        if (stop && *stop) return false;
    }
}

// The walk over this CTA's operator tiles in consumption order, with the
// fields of the current step's operator cached (one thread of the CTA runs it
// and keeps it in shared memory between calls).  Operator records of the slab
// visit whose table is in shared memory (tab_jo) are read from there, others
// from global memory.
template <int TWO>
struct TileIter {
    int s, mt, c, done;
    int n_mt, nkc, KR, xr;
    int m0, mstride;            // this cluster's first tile of step s and its tile stride
    long long off;
    __device__ void load(const DenseArgs& A, int cid, const DProb* tab, int tab_jo) {
        const StepInfo t = step_info(s, A.g.B, A.g.cen, TWO, cid, A.nclus);
        m0 = t.mcid;
        mstride = t.mncl;
        if (t.phase) {
            n_mt = 0;
            return;
        }
        if (t.jo == tab_jo) {
            const DProb& D = tab[op_slot(t.o.Mp, t.o.id, A.g.B)];
            n_mt = D.n_mt;
            nkc = D.nkc;
            KR = D.KR;
            xr = D.xr;
            off = D.off;
        } else {
            const DProb* D = &A.dp[t.o.p];
            n_mt = __ldg(&D->n_mt);
            nkc = __ldg(&D->nkc);
            KR = __ldg(&D->KR);
            xr = __ldg(&D->xr);
            off = __ldg(&D->off);
        }
    }
    __device__ void fix(const DenseArgs& A, int cid, const DProb* tab, int tab_jo) {
        while (s < A.nsteps) {
            load(A, cid, tab, tab_jo);
            mt = m0;
            c = 0;
            if (mt < n_mt) return;
            ++s;
        }
        done = 1;
    }
    __device__ void start(const DenseArgs& A, int cid) {
        s = 0;
        done = 0;
        fix(A, cid, nullptr, -1);
    }
    __device__ void next(const DenseArgs& A, int cid, const DProb* tab, int tab_jo) {
        if (++c < nkc) return;
        c = 0;
        mt += mstride;
        if (mt < n_mt) return;
        ++s;
        fix(A, cid, tab, tab_jo);
    }
    __device__ const unsigned char* ptr(const DenseArgs& A, int rank, uint32_t* bytes) const {
        const int kw = min(128, KR - 128 * c);
        const int ux = A.unit + 8 * xr;
        *bytes = (uint32_t)(kw * ux);
        return A.G + off + ((long long)(mt * HELM_DENSE_CS + rank) * KR + 128 * c) * ux;
    }
};

// Gather plan of one K-chunk: the single source of each input entry's value,
// encoded as 2 * offset (into Q) or 2 * offset + 1 (into Gv), or -1 for zero.
// Forward solves read the line couplings earlier solves wrote into Q on the
// lines next to the neighbours they come from (the first line for the lower
// front, the last for the upper, both for the centre), and the slab
// right-hand side Gv on its own layers elsewhere; backward solves read the
// coupling on the line next to the block their pass comes from.
__device__ __forceinline__ void gather_plan(const DenseArgs& A, const DProb& D, const OpInfo& o, const AxisWin& wz,
                                            int yb0, int yb1, int k0, int kw, int* s_src, int tid) {
    for (int jj = tid; jj < 128; jj += DT) {
        const int j = k0 + jj;
        int src = -1;
        if (jj < kw && j < D.n_in) {
            const int per = D.in.nz * D.in.nl;
            const int x = j / per;
            const int r = j - x * per, l = r / D.in.nz;
            const int lz = D.in.z0 + (r - l * D.in.nz), line = D.in.line0 + l;
            if (o.id == 0) {
                const bool from_below = o.ry != ROLE_U && o.Mp > 0 && line == yb0;
                const bool from_above = o.ry != ROLE_L && o.Mp < A.g.B - 1 && line == yb1 - 1;
                if (from_below || from_above) src = 2 * vbase(A, line, lz, x);
                else if (lz >= wz.ia && lz < wz.ib) src = 2 * zbase(A, line, lz - wz.ia, x) + 1;
            } else if (o.ry == ROLE_L ? line == yb1 - 1 : line == yb0) {
                src = 2 * vbase(A, line, lz, x);
            }
        }
        s_src[jj] = src;
    }
}

__device__ __forceinline__ float2 gather_val(const DenseArgs& A, const int* s_src, int jj, int rhs) {
    const int src = s_src[jj];
    if (src < 0) return make_float2(0.f, 0.f);     // no load for an absent entry
    const float2* base = (src & 1) ? A.Gv : A.Q;
    return __ldcg(base + (src >> 1) + rhs);
}

// TWO: the sweep schedule (0 one front, 1 two fronts) as a compile-time constant:
// the one-front kernel carries none of the two-front step mapping.
template <int FORM, int TWO>
__global__ void __launch_bounds__(DT, 1) k_dense(const __grid_constant__ DenseArgs A) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int B = A.g.B;
    unsigned char* ring = smem;
    unsigned char* Bbuf = smem + DSTAGES * TILE_BYTES;
    float* colsc = reinterpret_cast<float*>(Bbuf + BBUF_BYTES);      // [128] inverse column scales
    int* s_src = reinterpret_cast<int*>(colsc + 128);                // [128] gather plan
    unsigned* s_cmax = reinterpret_cast<unsigned*>(s_src + 128);     // [128] column maxima (float bits)
    float2* s_xp = reinterpret_cast<float2*>(s_cmax + 128);          // [2][64] extra rows' partial sums
    float2* s_pre = s_xp + 2 * 64;                                   // [3][DT] update operands (cp.async)
    uint64_t* full = reinterpret_cast<uint64_t*>(s_pre + 3 * DT);
    uint64_t* mma_bar = full + DSTAGES;
    uint64_t* ready = mma_bar + 1;         // every rank's partial sums are in place (8 arrivals)
    uint64_t* done = ready + 1;            // every rank has read the partial sums (8 arrivals)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* s_stop = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* s_issued = s_stop + 1;   // tiles issued into the ring
    volatile int* s_pend = s_issued + 1;   // released stages whose refill waits for the next step
    TileIter<TWO>* s_itr = reinterpret_cast<TileIter<TWO>*>(tslot + 4);   // [2] fill, prefetch (8-byte aligned)
    static_assert(sizeof(TileIter<TWO>) <= 48, "the tile walk's shared slot");
    DProb* s_dp = reinterpret_cast<DProb*>(smem + DENSE_SMEM_FIXED);  // [B+1] operators of the current slab
    AxisWin* s_win = reinterpret_cast<AxisWin*>(s_dp + (B + 2));      // [B] windows

    constexpr bool TC = FORM != FORM_FP32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const int cid = blockIdx.x / HELM_DENSE_CS;
    const int R8 = A.R8, N = A.g.N;
    const long long limit = A.wait_cycles > 0 ? A.wait_cycles : DEFAULT_WAIT;

    if (tid == 0) {
        for (int q = 0; q < DSTAGES; ++q) {
            ptx::mbar_init(&full[q], 1);
        }
        ptx::mbar_init(mma_bar, 1);
        ptx::mbar_init(ready, HELM_DENSE_CS);
        ptx::mbar_init(done, HELM_DENSE_CS);
        *s_stop = 0;
        *s_issued = 0;
        *s_pend = 0;
        ptx::fence_mbar_init();
    }
    for (int q = tid; q < B; q += DT) s_win[q] = A.win[q];
    if (TC && warp == 0) {
        ptx::tmem_alloc(tslot, 256);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
    ptx::tc_fence_after();
    const uint32_t tmem = TC ? *tslot : 0u;

    int consumed = 0;                      // ring tiles seen landed by thread 0
    int tab_jo = -1;                       // the slab visit whose operator table is in s_dp
    uint32_t mph = 0;                      // mma_bar phase
    bool mma_pending = false;
    // Thread PT keeps the ring full: tile t goes into stage t mod DSTAGES once the
    // stage's previous tile is released, and one more tile is prefetched into L2
    // PF_AHEAD tiles ahead.  A release whose next tile belongs to a later step is
    // only counted (s_pend); its refill runs at the top of the next step, while
    // thread 0 polls the step counter, instead of on this step's critical path.
    auto refill = [&]() {
        TileIter<TWO> f = s_itr[0], pf = s_itr[1];
        const int stage = *s_issued % DSTAGES;
        if (!f.done) {
            uint32_t bytes;
            const unsigned char* src = f.ptr(A, (int)rank, &bytes);
            ptx::mbar_expect_tx(&full[stage], bytes);
            ptx::bulk_g2s(ring + (size_t)stage * TILE_BYTES, src, bytes, &full[stage]);
            *s_issued = *s_issued + 1;
            f.next(A, cid, s_dp, tab_jo);
        }
        if (!pf.done) {
            uint32_t pb;
            const unsigned char* ps = pf.ptr(A, (int)rank, &pb);
            ptx::prefetch_l2(ps, pb);
            pf.next(A, cid, s_dp, tab_jo);
        }
        s_itr[0] = f;
        s_itr[1] = pf;
    };
    if (tid == PT) {
        TileIter<TWO> f, pf;
        f.start(A, cid);
        pf.start(A, cid);
        for (int q = 0; q < PF_AHEAD && !pf.done; ++q) pf.next(A, cid, nullptr, -1);
        s_itr[0] = f;
        s_itr[1] = pf;
        for (int q = 0; q < DSTAGES; ++q) refill();
    }
    {
        // ---------------- compute warps ----------------
        int stg = 0;
        uint32_t sph = 0, rph = 0, dph = 0;
        const uint32_t idesc_all = ptx::umma_idesc_f16(128, 4 * R8);
        const uint32_t idesc_hi = ptx::umma_idesc_f16(128, 2 * R8);
        const int TPR = DT / R8;           // TC gather: threads per right-hand side (R8 a power of 2)
        const size_t NN = (size_t)N * N;
        for (int s = 0; s < A.nsteps; ++s) {
            const StepInfo si = step_info(s, B, A.g.cen, TWO, cid, A.nclus);
            const int mcid = si.mcid, mncl = si.mncl;   // this cluster among the clusters of its solve
            // ---- the operator of an op step (phase steps: unused placeholders) ----
            const OpInfo o = si.o;
            const DProb& D = s_dp[op_slot(o.Mp, o.id, B)];
            const AxisWin wz = s_win[o.M], wy = s_win[o.Mp];
            const int yb0 = wy.lo + wy.ia, yb1 = wy.lo + wy.ib;
            const int n_mt = D.n_mt, nkc = D.nkc, KR = D.KR, xr = D.xr, rows = 64 + xr;
            const int cen = A.g.cen;
            // Couplings of Algorithm 4 this solve's result feeds (constants of the
            // operator), by the line block's role: a forward solve of the lower front
            // feeds the next block's first line (-c_dn), of the upper front the block
            // below's last line (-c_up); the centre's forward value is final and feeds
            // the backward passes of both neighbours (c_up below, c_dn above, the
            // second target); a backward solve feeds the next block of its pass
            // (c_up below for the lower front, c_dn above for the upper).
            float2 cf = make_float2(0.f, 0.f), cf2 = make_float2(0.f, 0.f);
            if (!si.phase) {
                const float2 dn = A.c_dn[yb1 < N ? yb1 : N - 1], up = A.c_up[yb0 > 0 ? yb0 - 1 : 0];
                if (o.id == 0 && o.ry == ROLE_L) cf = make_float2(-dn.x, -dn.y);
                else if (o.id == 0 && o.ry == ROLE_U) cf = make_float2(-up.x, -up.y);
                else if (o.id == 0) { cf = up; cf2 = dn; }
                else cf = (o.ry == ROLE_L) ? up : dn;
            }
            // the upper front's last forward solve adds its coupling to the centre's
            // line that the lower front already coupled into, when the centre block
            // is a single line (its first line is its last)
            const bool cen_one = s_win[cen].ib - s_win[cen].ia == 1;
            // Plan of one output row (tile-relative index orow): offsets of its forward
            // value (V), restricted result (Zv), coupling target (Q) and the target's
            // update source (>= 0: a slab term in Gv; <= -2: Q itself at -2 - value),
            // -1 where absent; z2 is the centre's second coupling target.
            int z2m = -1, z2x = -1;
            auto row_plan = [&](int orow, int* z2) {
                int4 pl = make_int4(-1, -1, -1, -1);
                *z2 = -1;
                if (orow < D.n_out) {
                    int q = orow;
                    const int s0 = D.out[0].nl * D.out[0].nz * N;
                    const bool r1 = D.nrect > 1 && q >= s0;
                    if (r1) q -= s0;
                    const int l0 = r1 ? D.out[1].line0 : D.out[0].line0;
                    const int z0 = r1 ? D.out[1].z0 : D.out[0].z0;
                    const int nz = r1 ? D.out[1].nz : D.out[0].nz;
                    const int x = q % N, t = q / N;
                    const int lz = z0 + t % nz, line = l0 + t / nz;
                    const bool zint = lz >= wz.ia && lz < wz.ib;
                    pl.x = vbase(A, line, lz, x);
                    if (zint) pl.y = zbase(A, line, lz - wz.ia, x);
                    if (o.id == 0 && o.ry == ROLE_L) {
                        if (line == yb1 - 1) {                      // into the next block's first line
                            pl.z = vbase(A, yb1, lz, x);
                            if (zint) pl.w = zbase(A, yb1, lz - wz.ia, x);
                        }
                    } else if (o.id == 0 && o.ry == ROLE_U) {
                        if (line == yb0) {                          // into the block below's last line
                            pl.z = vbase(A, yb0 - 1, lz, x);
                            if (o.Mp == cen + 1 && cen_one) pl.w = -2 - pl.z;
                            else if (zint) pl.w = zbase(A, yb0 - 1, lz - wz.ia, x);
                        }
                    } else if (o.id == 0) {                         // the centre: final, feeds both backward passes
                        if (o.Mp > 0 && line == yb0) pl.z = vbase(A, yb0 - 1, lz, x);
                        if (o.Mp < B - 1 && line == yb1 - 1) *z2 = vbase(A, yb1, lz, x);
                    } else if (o.ry == ROLE_L) {
                        if (o.Mp > 0 && line == yb0) pl.z = vbase(A, yb0 - 1, lz, x);   // the block below's last line
                    } else {
                        if (o.Mp < B - 1 && line == yb1 - 1) pl.z = vbase(A, yb1, lz, x);   // the block above's first line
                    }
                }
                return pl;
            };
            // Thread tid < 4 R8 owns output row mi of this rank's 8 and the right-hand
            // sides mrhs, mrhs + 1; thread tid < R8 also owns right-hand side tid of the
            // extra row this rank sums (tile row 64 + xown), if the tile has it.
            const int mi = tid / (R8 / 2), mrhs = 2 * (tid - mi * (R8 / 2));
            const int xown = HELM_DENSE_CS - 1 - (int)rank;
            int4 plm = make_int4(-1, -1, -1, -1), plx = make_int4(-1, -1, -1, -1);
            // Row scales (powers of two).  The partial sums of complex row i are kept in
            // units of s_min(i), the smaller scale of its real-part and imaginary-part
            // tile rows: a tile row rho read back from TMEM is multiplied by s_min /
            // s_rho (exact), the summed row by 1 / s_min.  Deferring 1 / s_min to after
            // the sum keeps the partials in the normal FP32 range for tiny right-hand
            // sides.
            float sc_self = 1.f, sc_part = 1.f, sc_y0 = 1.f, sc_y1 = 1.f;
            // This thread's plans and row scales for output tile mt (static data).
            auto tile_plans = [&](int mt) {
                if (tid < 4 * R8) plm = row_plan(rows * mt + 8 * (int)rank + mi, &z2m);
                if (xown < xr && tid < R8) plx = row_plan(rows * mt + 64 + xown, &z2x);
                if (TC) {
                    const float* sc = A.scale + D.soff + (long long)mt * 128;
                    const int rt = 32 * (warp & 3) + lane;
                    sc_self = __ldg(sc + rt);
                    sc_part = __ldg(sc + (rt ^ 16));
                    if (tid < 4 * R8) {
                        const int rr = 8 * (int)rank + mi;
                        sc_y0 = __ldg(sc + tile_row(rr, 0));
                        sc_y1 = __ldg(sc + tile_row(rr, 1));
                    }
                }
            };
            // The update operands of those rows, fetched asynchronously: forward values
            // of the block (a backward solve; written by its forward solve, two or more
            // steps back), the slab terms of the coupling (a forward solve; written by
            // the visit's boundary phase) or the coupled centre line (written by the
            // lower front's last forward solve, two or more steps back).
            auto pre_src = [&](const int4& pl) -> const float2* {
                if (o.id == 1) return pl.x >= 0 ? A.V + pl.x : nullptr;
                if (pl.w >= 0) return A.Gv + pl.w;
                if (pl.w <= -2) return A.Q + (-2 - pl.w);
                return nullptr;
            };
            auto fetch_pre = [&]() {
                if (tid < 4 * R8) {
                    const float2* src = pre_src(plm);
                    if (src) ptx::cp_async16(&s_pre[2 * tid], src + mrhs);
                }
                if (xown < xr && tid < R8) {
                    const float2* src = pre_src(plx);
                    if (src) ptx::cp_async8(&s_pre[2 * DT + tid], src + tid);
                }
                ptx::cp_async_commit();
            };
            // ---- prologue: the first tile's plans and the chunk-0 gather plan are made
            //      while thread 0 waits for step s-1 (single-chunk TC steps and all SIMT
            //      steps; multi-chunk TC steps plan inline).  The update operands are
            //      fetched here too unless step s-1 is the boundary phase that writes
            //      them (then after the wait). ----
            const bool pro = !si.phase && mcid < n_mt && !(TC && nkc > 1);
            // (two fronts: the upper front's last forward solve reads the centre line the
            // lower front wrote one step before)
            const bool pre_early = si.k >= 2 && !(TWO && o.id == 0 && o.ry == ROLE_U && o.Mp == cen + 1 && cen_one);
            if (pro) {
                tile_plans(mcid);
                if (pre_early) fetch_pre();
                if (TC && tid < 2 * R8) s_cmax[tid] = 0u;
                gather_plan(A, D, o, wz, yb0, yb1, (int)rank * KR, min(128, KR), s_src, tid);
            }
            if (tid == PT && *s_pend > 0 && !*s_stop) {
                for (int q = *s_pend; q > 0; --q) refill();
                *s_pend = 0;
            }
            // ---- every CTA has finished step s-1 ----
            if (s > 0 || A.unmet) {
                if (tid == 0) {
                    const unsigned target =
                        A.unmet ? 0xFFFFFFF0u : (unsigned)(HELM_DENSE_CS * A.nclus) * (unsigned)s;
                    const long long t0 = clock64();
                    while (ptx::ld_acquire_gpu(A.ctr) < target) {
                        if (clock64() - t0 > limit) {
                            atomicOr(A.err, 2);
                            *s_stop = 1;
                            break;
                        }
                    }
                }
                named_sync_compute();
                if (*s_stop) break;
            }
            if (si.phase) {
                // ---- boundary of slab visits jo-1 and jo (Algorithm 6) ----
                // The previous visit's result goes to z (a backward visit subtracts its
                // correction); then the new visit's right-hand side on its own layers:
                // forward, f minus the couplings of the neighbours already swept (the
                // block below for the lower front and the centre, the block above for
                // the upper front and the centre); backward, the coupling of the
                // neighbour its pass comes from (above for the lower front, below for
                // the upper).  Neighbour values are read back from z: each thread owns
                // whole (x, y, right-hand side) columns, so it reads what it wrote.
                PassPos vp{0, 0, 0}, vc{0, 0, 0};
                if (si.jo > 0) vp = pass_pos(si.jo - 1, B, A.g.cen);
                const bool cur = si.jo < 2 * B - 1;
                if (cur) {
                    vc = pass_pos(si.jo, B, A.g.cen);
                    // the operators of the new slab (slots of op_slot)
                    for (int q = tid; q <= B + 1; q += DT) s_dp[q] = A.dp[op_index(vc.M, q, B)];
                    tab_jo = si.jo;
                }
                const AxisWin wp = s_win[vp.M], wc = s_win[vc.M];
                const int dzp = wp.ib - wp.ia, dzc = wc.ib - wc.ia;
                const int mc = wc.lo + wc.ia, ec = wc.lo + wc.ib;       // the new slab's own layers [mc, ec)
                const bool cpl_lo = cur && (vc.bwd ? vc.role == ROLE_U : (vc.role != ROLE_U && vc.M > 0));
                const bool cpl_hi = cur && (vc.bwd ? vc.role == ROLE_L : (vc.role != ROLE_L && vc.M < B - 1));
                const float sgn = vc.bwd ? 1.f : -1.f;
                // a neighbour layer the previous visit just wrote is taken from registers
                const int pv0 = wp.lo + wp.ia, pv1 = wp.lo + wp.ib;
                const bool reg_lo = si.jo > 0 && mc - 1 >= pv0 && mc - 1 < pv1;
                const bool reg_hi = si.jo > 0 && ec >= pv0 && ec < pv1;
                const long long total = (long long)NN * R8;
                const long long stride = (long long)gridDim.x * DT;
                constexpr int PP = 4;                           // points per thread and pass
                for (long long p0 = (long long)blockIdx.x * DT + tid; p0 < total; p0 += PP * stride) {
                    int xs[PP], ls[PP], rs[PP];
                    bool ok[PP];
                    float2 nb_lo[PP], nb_hi[PP];
#pragma unroll
                    for (int q = 0; q < PP; ++q) {
                        nb_lo[q] = nb_hi[q] = make_float2(0.f, 0.f);
                        const long long p = min(p0 + q * stride, total - 1);
                        ok[q] = p0 + q * stride < total;
                        xs[q] = (int)(p % N);
                        const long long t = p / N;
                        ls[q] = (int)(t % N);
                        rs[q] = (int)(t / N);
                    }
                    if (si.jo > 0) {
                        for (int zr = 0; zr < dzp; ++zr) {
                            const int layer = wp.lo + wp.ia + zr;
                            float2 v[PP], old[PP];
#pragma unroll
                            for (int q = 0; q < PP; ++q) {
                                const int rr = min(rs[q], A.nrhs - 1);
                                v[q] = __ldcg(A.Zv + zbase(A, ls[q], zr, xs[q]) + rs[q]);
                                old[q] = (vp.bwd && rs[q] < A.nrhs)
                                             ? A.zout[((size_t)rr * N + layer) * NN + (size_t)ls[q] * N + xs[q]]
                                             : make_float2(0.f, 0.f);
                            }
#pragma unroll
                            for (int q = 0; q < PP; ++q) {
                                const float2 nz = vp.bwd ? csub(old[q], v[q]) : v[q];
                                if (ok[q] && rs[q] < A.nrhs)
                                    A.zout[((size_t)rs[q] * N + layer) * NN + (size_t)ls[q] * N + xs[q]] = nz;
                                if (layer == mc - 1) nb_lo[q] = nz;
                                if (layer == ec) nb_hi[q] = nz;
                            }
                        }
                    }
                    if (cur) {
                        // neighbour values (z, after the write above) times the couplings
                        float2 add_lo[PP], add_hi[PP];
#pragma unroll
                        for (int q = 0; q < PP; ++q) {
                            const int rr = min(rs[q], A.nrhs - 1);
                            const size_t col = (size_t)ls[q] * N + xs[q];
                            add_lo[q] = make_float2(0.f, 0.f);
                            add_hi[q] = make_float2(0.f, 0.f);
                            if (cpl_lo && rs[q] < A.nrhs) {
                                const float2 u = reg_lo ? nb_lo[q] : A.zout[((size_t)rr * N + mc - 1) * NN + col];
                                const float2 c = cmul(A.c_dn[mc], u);
                                add_lo[q] = make_float2(sgn * c.x, sgn * c.y);
                            }
                            if (cpl_hi && rs[q] < A.nrhs) {
                                const float2 u = reg_hi ? nb_hi[q] : A.zout[((size_t)rr * N + ec) * NN + col];
                                const float2 c = cmul(A.c_up[ec - 1], u);
                                add_hi[q] = make_float2(sgn * c.x, sgn * c.y);
                            }
                        }
                        for (int zr = 0; zr < dzc; ++zr) {
                            const int layer = mc + zr;
                            float2 rv[PP];
#pragma unroll
                            for (int q = 0; q < PP; ++q) {
                                const int rr = min(rs[q], A.nrhs - 1);
                                rv[q] = vc.bwd ? make_float2(0.f, 0.f)
                                               : A.rin[((size_t)rr * N + layer) * NN + (size_t)ls[q] * N + xs[q]];
                            }
#pragma unroll
                            for (int q = 0; q < PP; ++q) {
                                float2 gv = make_float2(0.f, 0.f);
                                if (rs[q] < A.nrhs) {
                                    gv = rv[q];
                                    if (zr == 0) gv = cadd(gv, add_lo[q]);
                                    if (zr == dzc - 1) gv = cadd(gv, add_hi[q]);
                                }
                                if (ok[q]) A.Gv[zbase(A, ls[q], zr, xs[q]) + rs[q]] = gv;
                            }
                        }
                    }
                }
                named_sync_compute();
                if (tid == 0) ptx::red_release_gpu_add(A.ctr, 1u);
                continue;
            }
            // this CTA's tiles of the step after tile (mt, c)
            auto tiles_left = [&](int mt_, int c_) {
                const int total = ((n_mt - mcid + mncl - 1) / mncl) * nkc;
                return total - (((mt_ - mcid) / mncl) * nkc + c_) - 1;
            };
            for (int mt = mcid; mt < n_mt; mt += mncl) {
                const bool first = (mt == mcid);
                if (!first || !pro) {
                    // a later tile of this step (or a multi-chunk step): plans inline
                    named_sync_compute();
                    tile_plans(mt);
                    fetch_pre();
                } else if (!pre_early) {
                    fetch_pre();
                }
                for (int q = tid; q < 2 * 64; q += DT) s_xp[q] = make_float2(0.f, 0.f);
                float2 acc[4][4];                               // SIMT form: rows 4 rg.., RHS 4 cg..
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
                for (int c = 0; c < nkc; ++c) {
                    const int kw = min(128, KR - 128 * c);
                    const int k0 = (int)rank * KR + 128 * c;
                    const int nkg = kw / 8;
                    const bool planned = first && pro && c == 0;   // the prologue made this chunk's plan
                    if (TC) {
                        // ---- q slice -> FP16 hi + lo B tile, one power-of-two scale per column ----
                        // thread (rhs = tid % R8, sub = tid / R8) takes K groups sub, sub + TPR, ...
                        const int rhs = tid % R8, sub = tid / R8;
                        if (!planned) {
                        if (c == 0) {
                            if (tid < 2 * R8) s_cmax[tid] = 0u;
                            if (nkc > 1) {
                                // several chunks share the accumulator: the column scale spans them all
                                float mre = 0.f, mim = 0.f;
                                for (int cc = 0; cc < nkc; ++cc) {
                                    named_sync_compute();
                                    gather_plan(A, D, o, wz, yb0, yb1, (int)rank * KR + 128 * cc,
                                                min(128, KR - 128 * cc), s_src, tid);
                                    named_sync_compute();
                                    for (int kg = sub; kg < 16; kg += TPR)
#pragma unroll
                                        for (int e = 0; e < 8; ++e) {
                                            const float2 v = gather_val(A, s_src, 8 * kg + e, rhs);
                                            mre = fmaxf(mre, fabsf(v.x));
                                            mim = fmaxf(mim, fabsf(v.y));
                                        }
                                }
                                atomicMax(&s_cmax[rhs], __float_as_uint(mre));
                                atomicMax(&s_cmax[R8 + rhs], __float_as_uint(mim));
                            }
                        }
                        named_sync_compute();
                        gather_plan(A, D, o, wz, yb0, yb1, k0, kw, s_src, tid);
                        named_sync_compute();
                        }
                        float2 qv[4][8];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            // only the K groups of this chunk issue loads (kw = 64: two of the
                            // four), so the ones that count are in flight together
                            const int kg = min(sub + u * TPR, 15);
                            if (sub + u * TPR < nkg) {
#pragma unroll
                                for (int e = 0; e < 8; ++e) qv[u][e] = gather_val(A, s_src, 8 * kg + e, rhs);
                            } else {
#pragma unroll
                                for (int e = 0; e < 8; ++e) qv[u][e] = make_float2(0.f, 0.f);
                            }
                        }
                        if (nkc == 1) {
                            float mre = 0.f, mim = 0.f;
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                if (sub + u * TPR < nkg)
#pragma unroll
                                    for (int e = 0; e < 8; ++e) {
                                        mre = fmaxf(mre, fabsf(qv[u][e].x));
                                        mim = fmaxf(mim, fabsf(qv[u][e].y));
                                    }
                            atomicMax(&s_cmax[rhs], __float_as_uint(mre));
                            atomicMax(&s_cmax[R8 + rhs], __float_as_uint(mim));
                        }
                        named_sync_compute();
                        // each thread forms its own columns' scales from the maxima; colsc (the
                        // inverses, read at the TMEM read-back) is written for later
                        // (the maxima are non-negative floats: their bits order like the values; for
                        // m > 0, frexp's exponent is the biased exponent field - 126, also for
                        // subnormal m, where the clamp of scale_exp decides; 2^e is built from
                        // its exponent field, exact for |e| <= 120)
                        auto col_exp = [](unsigned bits) {
                            return bits == 0u ? 0 : scale_exp((int)((bits >> 23) & 0xFFu) - 126);
                        };
                        const float sre = __int_as_float((col_exp(s_cmax[rhs]) + 127) << 23);
                        const float sim = __int_as_float((col_exp(s_cmax[R8 + rhs]) + 127) << 23);
                        if (c == 0 && tid < 2 * R8) colsc[tid] = __int_as_float((127 - col_exp(s_cmax[tid])) << 23);
                        const int sbo = nkg * 128;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int kg = sub + u * TPR;
                            if (kg < nkg) {
                                __align__(16) __half hr[8], lr[8], hm[8], lm[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) {
                                    const float xr = qv[u][e].x * sre, xi = qv[u][e].y * sim;
                                    hr[e] = __float2half_rn(xr);
                                    lr[e] = __float2half_rn(xr - __half2float(hr[e]));
                                    hm[e] = __float2half_rn(xi);
                                    lm[e] = __float2half_rn(xi - __half2float(hm[e]));
                                }
                                const size_t base = (size_t)kg * 128 + (rhs & 7) * 16;
                                *reinterpret_cast<uint4*>(Bbuf + (size_t)(rhs >> 3) * sbo + base) =
                                    *reinterpret_cast<const uint4*>(hr);
                                *reinterpret_cast<uint4*>(Bbuf + (size_t)((R8 + rhs) >> 3) * sbo + base) =
                                    *reinterpret_cast<const uint4*>(hm);
                                *reinterpret_cast<uint4*>(Bbuf + (size_t)((2 * R8 + rhs) >> 3) * sbo + base) =
                                    *reinterpret_cast<const uint4*>(lr);
                                *reinterpret_cast<uint4*>(Bbuf + (size_t)((3 * R8 + rhs) >> 3) * sbo + base) =
                                    *reinterpret_cast<const uint4*>(lm);
                            }
                        }
                        ptx::fence_proxy_async_smem();
                        // the tile must have landed: the MMA reads it, the extra rows are read below
                        if (!wait_bar(&full[stg], sph, limit, false, nullptr)) {
                            atomicOr(A.err, 2);
                            *s_stop = 1;
                        }
                        named_sync_compute();
                        const bool go = !*s_stop;          // the same value in every thread after the sync
                        if (tid == 0 && go) {
                            ++consumed;
                            ptx::tc_fence_after();
                            const uint32_t a_hi = ptx::smem_u32(ring + (size_t)stg * TILE_BYTES);
                            const uint32_t a_lo = a_hi + (uint32_t)(128 * kw * 2);
                            const uint32_t b0 = ptx::smem_u32(Bbuf);
                            const uint32_t sb = (uint32_t)sbo;
                            for (int ks = 0; ks < kw / 16; ++ks)
                                ptx::umma_f16(tmem, ptx::umma_desc(a_hi + 256u * ks, 128u, sb),
                                              ptx::umma_desc(b0 + 256u * ks, 128u, sb), idesc_all,
                                              (c > 0 || ks > 0) ? 1u : 0u);
                            if (FORM == FORM_SPLIT)
                                for (int ks = 0; ks < kw / 16; ++ks)
                                    ptx::umma_f16(tmem, ptx::umma_desc(a_lo + 256u * ks, 128u, sb),
                                                  ptx::umma_desc(b0 + 256u * ks, 128u, sb), idesc_hi, 1u);
                            ptx::umma_commit(mma_bar);
                        }
                        if (go && xr > 0) {
                            // the FP32 extra rows on the SIMT lanes while the tensor core runs
                            const float2* X = reinterpret_cast<const float2*>(ring + (size_t)stg * TILE_BYTES +
                                                                              (size_t)A.unit * kw);
                            for (int ex = 0; ex < xr; ++ex) {
                                float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    const int kg = sub + u * TPR;
                                    if (kg < nkg)
#pragma unroll
                                        for (int e = 0; e < 8; e += 2) {
                                            cfma(a0, X[ex * kw + 8 * kg + e], qv[u][e]);
                                            cfma(a1, X[ex * kw + 8 * kg + e + 1], qv[u][e + 1]);
                                        }
                                }
                                atomicAdd(&s_xp[ex * 64 + rhs].x, a0.x + a1.x);
                                atomicAdd(&s_xp[ex * 64 + rhs].y, a0.y + a1.y);
                            }
                        }
                        if (++stg == DSTAGES) { stg = 0; sph ^= 1u; }
                        if (!go) break;
                        // B is rewritten by the next chunk and TMEM is read after the last
                        if (wait_bar(mma_bar, mph, limit, false, nullptr)) {
                            mph ^= 1u;
                        } else {
                            atomicOr(A.err, 2);
                            *s_stop = 1;
                            mma_pending = true;            // teardown waits for it again
                        }
                        ptx::tc_fence_after();
                        named_sync_compute();
                        // the MMA and the extra rows are done with the stage: refill it now if
                        // this step still needs the tile that goes there, else at the next step
                        if (tid == PT && !*s_stop) {
                            if (tiles_left(mt, c) >= DSTAGES) refill();
                            else *s_pend = *s_pend + 1;
                        }
                        if (*s_stop) break;
                    } else {
                        // ---- SIMT: q slice as complex FP32 [kw][64], then the tile product ----
                        if (!planned) {
                            named_sync_compute();
                            gather_plan(A, D, o, wz, yb0, yb1, k0, kw, s_src, tid);
                            named_sync_compute();
                        }
                        float2* Bq = reinterpret_cast<float2*>(Bbuf);
                        const int rhs = tid & 63, kq = tid >> 6, rc = min(rhs, R8 - 1);
                        for (int t0 = 0; t0 < 32; t0 += 8) {               // slots kq + 4 t, t < 32
                            float2 vals[8];
#pragma unroll
                            for (int t = 0; t < 8; ++t) vals[t] = gather_val(A, s_src, kq + 4 * (t0 + t), rc);
#pragma unroll
                            for (int t = 0; t < 8; ++t) {
                                const int kj = kq + 4 * (t0 + t);
                                if (kj < kw) Bq[kj * 64 + rhs] = (rhs < R8) ? vals[t] : make_float2(0.f, 0.f);
                            }
                        }
                        if (!wait_bar(&full[stg], sph, limit, false, s_stop)) {
                            atomicOr(A.err, 2);
                            *s_stop = 1;
                        } else if (tid == 0) {
                            ++consumed;
                        }
                        named_sync_compute();
                        if (*s_stop) break;
                        const float2* At = reinterpret_cast<const float2*>(ring + (size_t)stg * TILE_BYTES);
                        const int rg = tid >> 4, cg = tid & 15;
                        if (4 * cg < R8) {
                            for (int kk = 0; kk < kw; ++kk) {
                                const float4* ar = reinterpret_cast<const float4*>(At + kk * 64 + 4 * rg);
                                const float4* br = reinterpret_cast<const float4*>(Bq + kk * 64 + 4 * cg);
                                const float4 a0 = ar[0], a1 = ar[1], b0 = br[0], b1 = br[1];
                                const float2 av[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w),
                                                      make_float2(a1.x, a1.y), make_float2(a1.z, a1.w)};
                                const float2 bv[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                                                      make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
#pragma unroll
                                for (int a = 0; a < 4; ++a)
#pragma unroll
                                    for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
                            }
                        }
                        if (xr > 0) {
                            const float2* X = reinterpret_cast<const float2*>(ring + (size_t)stg * TILE_BYTES +
                                                                              (size_t)A.unit * kw);
                            const int rr = tid & 63, kq2 = tid >> 6;
                            for (int ex = 0; ex < xr; ++ex) {
                                float2 acc2 = make_float2(0.f, 0.f);
                                for (int kj = kq2; kj < kw; kj += 4) cfma(acc2, X[ex * kw + kj], Bq[kj * 64 + rr]);
                                atomicAdd(&s_xp[ex * 64 + rr].x, acc2.x);
                                atomicAdd(&s_xp[ex * 64 + rr].y, acc2.y);
                            }
                        }
                        named_sync_compute();
                        if (tid == PT) {
                            if (tiles_left(mt, c) >= DSTAGES) refill();
                            else *s_pend = *s_pend + 1;
                        }
                        if (++stg == DSTAGES) { stg = 0; sph ^= 1u; }
                    }
                }
                if (*s_stop) break;
                // the update operands fetched asynchronously with the plans
                ptx::cp_async_wait_all();
                // ---- this rank's partial sums into Bbuf ----
                if (TC) {
                    // Warp (qd, hp) reads TMEM lanes 32 qd.. (tile rows) for right-hand sides
                    // hp R8/2 .. (all of them in warps 0-3 when R8 = 8).  Per right-hand side
                    // j: the row times q's real part, hi + lo, in columns j and 2 R8 + j,
                    // times q's imaginary part in R8 + j and 3 R8 + j.  Lane l holds part
                    // (l / 16) of complex row i = 16 qd + l mod 16: the real part contributes
                    // (x, y) to Y_i = G_i q, the imaginary part (-y, x); lanes l and l ^ 16
                    // add their contributions with one shuffle, each keeping half of the
                    // right-hand sides, and store (re, im) pairs.
                    float* Pp = reinterpret_cast<float*>(Bbuf);
                    const int qd = warp & 3, hp = warp >> 2;
                    const bool imp = (lane & 16) != 0;
                    const float tfac = fminf(sc_self, sc_part) / sc_self;
                    const uint32_t tb = tmem + ((uint32_t)(32 * qd) << 16);
                    const int nh = R8 >= 16 ? R8 / 2 : (hp == 0 ? R8 : 0);
                    const int j0 = R8 >= 16 ? hp * (R8 / 2) : 0;
                    float* prow = Pp + (16 * qd + (lane & 15)) * PSTR;
                    if (nh >= 16) {
                        for (int jb = j0; jb < j0 + nh; jb += 16) {
                            float hre[16], him[16], lre[16], lim[16];
                            ptx::tmem_ld16(tb + (uint32_t)jb, hre);
                            ptx::tmem_ld16(tb + (uint32_t)(R8 + jb), him);
                            ptx::tmem_ld16(tb + (uint32_t)(2 * R8 + jb), lre);
                            ptx::tmem_ld16(tb + (uint32_t)(3 * R8 + jb), lim);
                            ptx::tmem_wait_ld();
                            ptx::reg_tie16(hre);
                            ptx::reg_tie16(him);
                            ptx::reg_tie16(lre);
                            ptx::reg_tie16(lim);
                            float tx[16], ty[16];
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                const float x = (hre[e] + lre[e]) * colsc[jb + e] * tfac;
                                const float y = (him[e] + lim[e]) * colsc[R8 + jb + e] * tfac;
                                tx[e] = imp ? -y : x;
                                ty[e] = imp ? x : y;
                            }
                            // lane keeps right-hand sides jb + 8 imp .. + 7
                            float ox[8], oy[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const float sx = imp ? tx[e] : tx[8 + e], sy = imp ? ty[e] : ty[8 + e];
                                const float rx_ = __shfl_xor_sync(0xffffffffu, sx, 16);
                                const float ry_ = __shfl_xor_sync(0xffffffffu, sy, 16);
                                ox[e] = (imp ? tx[8 + e] : tx[e]) + rx_;
                                oy[e] = (imp ? ty[8 + e] : ty[e]) + ry_;
                            }
                            const int jk = jb + (imp ? 8 : 0);
#pragma unroll
                            for (int e = 0; e < 8; e += 2)
                                *reinterpret_cast<float4*>(prow + 2 * (jk + e)) =
                                    make_float4(ox[e], oy[e], ox[e + 1], oy[e + 1]);
                        }
                    } else if (nh == 8) {
                        float hre[8], him[8], lre[8], lim[8];
                        ptx::tmem_ld8(tb + (uint32_t)j0, hre);
                        ptx::tmem_ld8(tb + (uint32_t)(R8 + j0), him);
                        ptx::tmem_ld8(tb + (uint32_t)(2 * R8 + j0), lre);
                        ptx::tmem_ld8(tb + (uint32_t)(3 * R8 + j0), lim);
                        ptx::tmem_wait_ld();
                        ptx::reg_tie8(hre);
                        ptx::reg_tie8(him);
                        ptx::reg_tie8(lre);
                        ptx::reg_tie8(lim);
                        float tx[8], ty[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const float x = (hre[e] + lre[e]) * colsc[j0 + e] * tfac;
                            const float y = (him[e] + lim[e]) * colsc[R8 + j0 + e] * tfac;
                            tx[e] = imp ? -y : x;
                            ty[e] = imp ? x : y;
                        }
                        float ox[4], oy[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float sx = imp ? tx[e] : tx[4 + e], sy = imp ? ty[e] : ty[4 + e];
                            const float rx_ = __shfl_xor_sync(0xffffffffu, sx, 16);
                            const float ry_ = __shfl_xor_sync(0xffffffffu, sy, 16);
                            ox[e] = (imp ? tx[4 + e] : tx[e]) + rx_;
                            oy[e] = (imp ? ty[4 + e] : ty[e]) + ry_;
                        }
                        const int jk = j0 + (imp ? 4 : 0);
#pragma unroll
                        for (int e = 0; e < 4; e += 2)
                            *reinterpret_cast<float4*>(prow + 2 * (jk + e)) =
                                make_float4(ox[e], oy[e], ox[e + 1], oy[e + 1]);
                    }
                    ptx::tc_fence_before();
                } else {
                    float2* Pp = reinterpret_cast<float2*>(Bbuf);
                    const int rg = tid >> 4, cg = tid & 15;
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) Pp[(4 * rg + a) * 64 + 4 * cg + b] = acc[a][b];
                }
                named_sync_compute();
                if (tid < HELM_DENSE_CS) ptx::mbar_arrive_remote(ptx::mapa(ready, (uint32_t)tid));
                if (!wait_bar(ready, rph, limit, true, nullptr)) {
                    atomicOr(A.err, 2);
                    *s_stop = 1;
                }
                rph ^= 1u;
                // ---- sum the 8 partials of this rank's 8 output rows; apply the update ----
                // Thread tid < 4 R8: row i = tid / (R8/2), right-hand sides rhs, rhs + 1; the
                // eight remote loads are issued before the first is used.
                const float2 coef = cf;
                const bool main_ok = tid < 4 * R8;
                float4 rv[HELM_DENSE_CS];
                if (main_ok) {
                    const int row = 8 * (int)rank + mi;
                    const float* src = TC ? reinterpret_cast<const float*>(Bbuf) + row * PSTR + 2 * mrhs
                                          : reinterpret_cast<const float*>(Bbuf) + 2 * (row * 64 + mrhs);
#pragma unroll
                    for (int q = 0; q < HELM_DENSE_CS; ++q) rv[q] = ptx::ld_dsmem_f32x4(ptx::mapa(src, (uint32_t)q));
                }
                float2 rx[HELM_DENSE_CS];
                const bool xown_ok = xown < xr && tid < R8;
                if (xown_ok) {
#pragma unroll
                    for (int q = 0; q < HELM_DENSE_CS; ++q)
                        rx[q] = ptx::ld_dsmem_f32x2(ptx::mapa(s_xp + xown * 64 + tid, (uint32_t)q));
                }
                if (main_ok) {
                    float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < HELM_DENSE_CS; ++q) {
                        y.x += rv[q].x;
                        y.y += rv[q].y;
                        y.z += rv[q].z;
                        y.w += rv[q].w;
                    }
                    const float yinv = 1.f / fminf(sc_y0, sc_y1);
                    y.x *= yinv;
                    y.y *= yinv;
                    y.z *= yinv;
                    y.w *= yinv;
                    const float2 Y0 = make_float2(y.x, y.y), Y1 = make_float2(y.z, y.w);
                    const int4 pl = plm;
                    if (pl.x >= 0) {
                        const float4 pre = *reinterpret_cast<const float4*>(&s_pre[2 * tid]);
                        const float2 p0 = make_float2(pre.x, pre.y), p1 = make_float2(pre.z, pre.w);
                        if (o.id == 0) {
                            *reinterpret_cast<float4*>(A.V + pl.x + mrhs) = y;   // forward values of the line block
                            if (o.ry == ROLE_C && pl.y >= 0)                       // the centre has no backward step
                                *reinterpret_cast<float4*>(A.Zv + pl.y + mrhs) = y;
                            if (pl.z >= 0) {
                                const bool has = pl.w != -1;
                                const float2 g0 = has ? p0 : make_float2(0.f, 0.f);
                                const float2 g1 = has ? p1 : make_float2(0.f, 0.f);
                                const float2 q0 = cadd(g0, cmul(coef, Y0)), q1 = cadd(g1, cmul(coef, Y1));
                                *reinterpret_cast<float4*>(A.Q + pl.z + mrhs) = make_float4(q0.x, q0.y, q1.x, q1.y);
                            }
                            if (z2m >= 0) {
                                const float2 q0 = cmul(cf2, Y0), q1 = cmul(cf2, Y1);
                                *reinterpret_cast<float4*>(A.Q + z2m + mrhs) = make_float4(q0.x, q0.y, q1.x, q1.y);
                            }
                        } else {
                            const float2 v0 = csub(p0, Y0), v1 = csub(p1, Y1);   // backward correction
                            if (pl.y >= 0) *reinterpret_cast<float4*>(A.Zv + pl.y + mrhs) = make_float4(v0.x, v0.y, v1.x, v1.y);
                            if (pl.z >= 0) {
                                const float2 q0 = cmul(coef, v0), q1 = cmul(coef, v1);
                                *reinterpret_cast<float4*>(A.Q + pl.z + mrhs) = make_float4(q0.x, q0.y, q1.x, q1.y);
                            }
                        }
                    }
                }
                if (xown_ok) {
                    float2 Y = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < HELM_DENSE_CS; ++q) Y = cadd(Y, rx[q]);
                    const int4 pl = plx;
                    const int rhs = tid;
                    if (pl.x >= 0) {
                        const float2 pre = s_pre[2 * DT + tid];
                        if (o.id == 0) {
                            A.V[pl.x + rhs] = Y;
                            if (o.ry == ROLE_C && pl.y >= 0) A.Zv[pl.y + rhs] = Y;
                            if (pl.z >= 0) A.Q[pl.z + rhs] = cadd(pl.w != -1 ? pre : make_float2(0.f, 0.f), cmul(coef, Y));
                            if (z2x >= 0) A.Q[z2x + rhs] = cmul(cf2, Y);
                        } else {
                            const float2 v = csub(pre, Y);
                            if (pl.y >= 0) A.Zv[pl.y + rhs] = v;
                            if (pl.z >= 0) A.Q[pl.z + rhs] = cmul(coef, v);
                        }
                    }
                }
                if (mt + mncl < n_mt) {
                    // another tile of this solve reuses Bbuf: wait until every rank has read it
                    named_sync_compute();
                    if (tid < HELM_DENSE_CS) ptx::mbar_arrive_remote(ptx::mapa(done, (uint32_t)tid));
                    if (!wait_bar(done, dph, limit, true, nullptr)) {
                        atomicOr(A.err, 2);
                        *s_stop = 1;
                    }
                    dph ^= 1u;
                }
                named_sync_compute();
                if (*s_stop) break;
            }
            if (*s_stop) break;
            // ---- this CTA's share of step s is written ----
            if (tid == 0) ptx::red_release_gpu_add(A.ctr, 1u);
        }
    }
    named_sync_compute();
    // ---- teardown: let issued copies land, free TMEM, leave with the cluster ----
    if (tid == 0) {
        const int issued = *s_issued;
        int q = consumed % DSTAGES;
        uint32_t ph = (uint32_t)((consumed / DSTAGES) & 1);
        for (int u = consumed; u < issued; ++u) {
            wait_bar(&full[q], ph, limit, false, nullptr);
            if (++q == DSTAGES) { q = 0; ph ^= 1u; }
        }
        if (TC && mma_pending) wait_bar(mma_bar, mph, limit, false, nullptr);
    }
    if (TC) {
        ptx::tc_fence_before();
        named_sync_compute();
        if (warp == 0) ptx::tmem_dealloc(tmem, 256);
    }
    asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

size_t dense_smem_bytes(int B) {
    return (size_t)DENSE_SMEM_FIXED + (size_t)(B + 2) * sizeof(DProb) + (size_t)B * sizeof(AxisWin);
}

template <int FORM>
const void* dense_kernel(int sched) {
    return sched == HELM_TWO_FRONT ? (const void*)k_dense<FORM, 1> : (const void*)k_dense<FORM, 0>;
}

const void* dense_kernel_for(int precision, int sched) {
    switch (precision) {
        case HELM_SPLIT_FP16: return dense_kernel<FORM_SPLIT>(sched);
        case HELM_FP16: return dense_kernel<FORM_HI>(sched);
        default: return dense_kernel<FORM_FP32>(sched);
    }
}

}  // namespace

// ================================================================ host =======

// The operator table: sizes, index sets and storage offsets.
static void build_dense_table(helm_ctx* h, const std::vector<AxisWin>& win, int nclus, std::vector<DProb>& out,
                              size_t* gbytes, size_t* nscale) {
    const int B = h->g.B, N = h->g.N, b = h->g.b;
    const bool two = h->g.sched == HELM_TWO_FRONT;
    const int unit = tile_unit(h->opts.precision);
    out.assign((size_t)dense_nops(B), DProb());
    size_t off = 0, soff = 0;
    for (int p = 0; p < dense_nops(B); ++p) {
        DProb D;
        memset(&D, 0, sizeof(D));
        // slab M, slot q (op_index inverted)
        const int M = p < B * B ? p / B : (p < B * B + B ? p - B * B : p - B * B - B);
        const int q = p < B * B ? p % B : (p < B * B + B ? B : B + 1);
        const int Mp = q < B ? q : (q == B ? 0 : B - 1);
        const AxisWin& wz = win[M];
        const AxisWin& wy = win[Mp];
        const int Lz = wz.L, za = wz.ia, zb = wz.ib;
        D.fp = M * B + Mp;
        if (q == B + 1 && !two) {
            out[p] = D;                                   // no backward map of the last block (one front)
            continue;
        }
        if (q == 0) {
            // the low boundary slab's forward map: its own entries in, the line
            // next to block 1 whole and the others' interest rows out
            D.in = DRect{0, b, za, zb - za};
            D.nrect = 0;
            if (b > 1) D.out[D.nrect++] = DRect{0, b - 1, za, zb - za};
            D.out[D.nrect++] = DRect{b - 1, 1, 0, Lz};
        } else if (q == B) {
            // its backward map: the coupling line in, the interest rows out
            D.in = DRect{b - 1, 1, 0, Lz};
            D.out[0] = DRect{0, b, za, zb - za};
            D.nrect = 1;
        } else if (two && q == B - 1) {
            // the high boundary slab's forward map (mirror of q = 0)
            D.in = DRect{N - b, b, za, zb - za};
            D.nrect = 0;
            D.out[D.nrect++] = DRect{N - b, 1, 0, Lz};
            if (b > 1) D.out[D.nrect++] = DRect{N - b + 1, b - 1, za, zb - za};
        } else if (q == B + 1) {
            D.in = DRect{N - b, 1, 0, Lz};
            D.out[0] = DRect{N - b, b, za, zb - za};
            D.nrect = 1;
        } else {
            D.in = DRect{wy.lo + wy.ia, wy.ib - wy.ia, 0, Lz};
            D.out[0] = D.in;
            D.nrect = 1;
        }
        D.n_in = D.in.nl * D.in.nz * N;
        D.n_out = 0;
        for (int r = 0; r < D.nrect; ++r) D.n_out += D.out[r].nl * D.out[r].nz * N;
        // tiles of 64 + xr rows: up to 2 extra rows let the operator fit the resident clusters in one round
        const int per_cluster = ceil_div(D.n_out, nclus);
        D.xr = (per_cluster > 64 && per_cluster <= 66) ? per_cluster - 64 : 0;
        D.n_mt = ceil_div(D.n_out, 64 + D.xr);
        D.KR = 16 * ceil_div(ceil_div(D.n_in, HELM_DENSE_CS), 16);
        D.nkc = ceil_div(D.KR, 128);
        D.off = (long long)off;
        D.soff = (long long)soff;
        off += (size_t)D.n_mt * HELM_DENSE_CS * D.KR * (unit + 8 * D.xr);
        if (h->opts.precision != HELM_FP32) soff += (size_t)D.n_mt * 128;
        out[p] = D;
    }
    *gbytes = off;
    *nscale = soff;
}

// Factors and restricted operators of slabs Ma..Mb, for the line blocks
// Pa..Pb (and the first block's backward operator when Pa = 0): the build of
// helm_setup (all of them) and of helm_update_velocity (those a box touches).
static int dense_build(helm_ctx* h, const Prob* prob, int Ma, int Mb, int Pa, int Pb, cudaStream_t st) {
    const int B = h->g.B, N = h->g.N;
    const int P = dense_nops(B);
    const DProb* dp = h->dprob_h;
    cudaError_t e;
#define DTRY(x) do { e = (x); if (e != cudaSuccess) { helm_set_cuda_error(e); return e == cudaErrorMemoryAllocation ? HELM_ENOMEM : HELM_ECUDA; } } while (0)
    // ---- chunks of slabs: factors, then the operators of the chunk's problems ----
    // the first-block backward operator of slab M (index B*B+M) uses problem (M, 0)
    const size_t budget = (size_t)6 << 30;            // bytes of temporary factors + G per chunk
    int dev = 0;
    cudaGetDevice(&dev);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int gblocks = 2 * std::max(nsm, 1);
    const size_t yslot = (size_t)N * 64 * GW;           // complex entries per setup CTA
    float2* yscr = nullptr;
    DTRY(cudaMalloc(&yscr, (size_t)gblocks * yslot * sizeof(float2)));
    const size_t gsm = (size_t)(64 * TLD + 2 * 64 * GW) * sizeof(float2) + (2 * GW + 64) * sizeof(int);
    e = ensure_dyn_smem((const void*)k_dense_G, gsm);
    if (e != cudaSuccess) { cudaFree(yscr); helm_set_cuda_error(e); return HELM_ECUDA; }
    float2* fac = nullptr;
    float2* Gt = nullptr;
    size_t fac_cap = 0, gt_cap = 0;
    GItem* d_items = nullptr;
    PItem* d_pitems = nullptr;
    long long* d_goff = nullptr;
    size_t items_cap = 0, pitems_cap = 0;
    int rc = HELM_OK;
    DTRY(cudaMalloc(&d_goff, sizeof(long long) * P));
    std::vector<long long> goff(P, 0);
    int M0 = Ma;
    while (M0 <= Mb && rc == HELM_OK) {
        // grow the chunk while it fits the budget
        int M1 = M0;
        size_t fbytes = 0, gtb = 0;
        for (;;) {
            const int M = M1;
            const long long f0 = prob[(size_t)M0 * B].off;
            const long long f1 = prob[(size_t)M * B + B - 1].off + (long long)N * prob[(size_t)M * B + B - 1].kstride;
            size_t fb = (size_t)(f1 - f0) * sizeof(float2);
            size_t gb = gtb;
            for (int Mp = 0; Mp < B; ++Mp) gb += (size_t)dp[(size_t)M * B + Mp].n_out * dp[(size_t)M * B + Mp].n_in;
            gb += (size_t)dp[(size_t)B * B + M].n_out * dp[(size_t)B * B + M].n_in;
            gb += (size_t)dp[(size_t)B * B + B + M].n_out * dp[(size_t)B * B + B + M].n_in;
            if (M1 > M0 && fb + gb * sizeof(float2) > budget) break;
            fbytes = fb;
            gtb = gb;
            ++M1;
            if (M1 > Mb) break;
        }
        const long long off0 = prob[(size_t)M0 * B].off;
        if (fbytes > fac_cap) {
            if (fac) cudaFree(fac);
            fac = nullptr;
            DTRY(cudaMalloc(&fac, fbytes));
            fac_cap = fbytes;
        }
        if (gtb * sizeof(float2) > gt_cap) {
            if (Gt) cudaFree(Gt);
            Gt = nullptr;
            DTRY(cudaMalloc(&Gt, gtb * sizeof(float2)));
            gt_cap = gtb * sizeof(float2);
        }
        DTRY(launch_factor_range(h, M0 * B, (M1 - M0) * B, fac, off0, HELM_FP32, st));
        // work items and temporary operator offsets of the chunk
        std::vector<GItem> items;
        std::vector<PItem> pitems;
        long long go = 0;
        for (int M = M0; M < M1; ++M) {
            for (int q = 0; q <= B + 1; ++q) {
                // an operator the build leaves as it is (slot B: block 0's backward map, B + 1: block B-1's)
                if (q < B ? (q < Pa || q > Pb) : (q == B ? Pa != 0 : Pb != B - 1)) continue;
                const int p = op_index(M, q, B);
                if (dp[p].n_out == 0) continue;
                goff[p] = go;
                go += (long long)dp[p].n_out * dp[p].n_in;
                for (int j0 = 0; j0 < dp[p].n_in; j0 += GW) items.push_back(GItem{p, j0});
                for (int mt = 0; mt < dp[p].n_mt; ++mt) pitems.push_back(PItem{p, mt});
            }
        }
        if (items.size() > items_cap) {
            if (d_items) cudaFree(d_items);
            d_items = nullptr;
            DTRY(cudaMalloc(&d_items, items.size() * sizeof(GItem)));
            items_cap = items.size();
        }
        if (pitems.size() > pitems_cap) {
            if (d_pitems) cudaFree(d_pitems);
            d_pitems = nullptr;
            DTRY(cudaMalloc(&d_pitems, pitems.size() * sizeof(PItem)));
            pitems_cap = pitems.size();
        }
        DTRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(GItem), cudaMemcpyHostToDevice, st));
        DTRY(cudaMemcpyAsync(d_pitems, pitems.data(), pitems.size() * sizeof(PItem), cudaMemcpyHostToDevice, st));
        DTRY(cudaMemcpyAsync(d_goff, goff.data(), sizeof(long long) * P, cudaMemcpyHostToDevice, st));
        const int nblk = (int)std::min<size_t>(items.size(), (size_t)gblocks);
        k_dense_G<<<nblk, GT, gsm, st>>>(h->g, h->t, h->dprob, d_items, (int)items.size(), fac, off0, Gt, d_goff,
                                         yscr, yslot);
        h->launches++;
        DTRY(cudaGetLastError());
        switch (h->opts.precision) {
            case HELM_SPLIT_FP16:
                k_dense_pack<HELM_SPLIT_FP16><<<(int)pitems.size(), 256, 0, st>>>(h->dprob, d_pitems, Gt, d_goff,
                                                                                h->dG, h->dscale);
                break;
            case HELM_FP16:
                k_dense_pack<HELM_FP16><<<(int)pitems.size(), 256, 0, st>>>(h->dprob, d_pitems, Gt, d_goff, h->dG,
                                                                          h->dscale);
                break;
            default:
                k_dense_pack<HELM_FP32><<<(int)pitems.size(), 256, 0, st>>>(h->dprob, d_pitems, Gt, d_goff, h->dG,
                                                                          h->dscale);
        }
        h->launches++;
        DTRY(cudaGetLastError());
        // the host arrays above must outlive their copies
        DTRY(cudaStreamSynchronize(st));
        M0 = M1;
    }
    cudaFree(yscr);
    cudaFree(fac);
    cudaFree(Gt);
    cudaFree(d_items);
    cudaFree(d_pitems);
    cudaFree(d_goff);
#undef DTRY
    return rc;
}

int dense_setup(helm_ctx* h, const void* win_host, const void* prob_host, cudaStream_t st) {
    const std::vector<AxisWin>& win = *static_cast<const std::vector<AxisWin>*>(win_host);
    const std::vector<Prob>& prob = *static_cast<const std::vector<Prob>*>(prob_host);
    const int B = h->g.B;
    const int P = dense_nops(B);
    cudaError_t e;
    // ---- the apply launch: clusters of 8 CTAs, as many as can be resident (<= 16) ----
    h->dsmem = dense_smem_bytes(B);
    if (h->dsmem > (size_t)227 * 1024) return HELM_ENOTSUP;
    {
        const void* kfn = dense_kernel_for(h->opts.precision, h->g.sched);
        e = ensure_dyn_smem(kfn, h->dsmem);
        if (e != cudaSuccess) { helm_set_cuda_error(e); return HELM_ECUDA; }
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = HELM_DENSE_CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(HELM_DENSE_CS * 16, 1, 1);
        cfg.blockDim = dim3(DT, 1, 1);
        cfg.dynamicSmemBytes = h->dsmem;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        e = cudaOccupancyMaxActiveClusters(&ncl, kfn, &cfg);
        if (e != cudaSuccess) { helm_set_cuda_error(e); return HELM_ECUDA; }
        if (ncl < 1) return HELM_ENOTSUP;
        h->dclus = std::min(ncl, 16);
        if (h->opts.dense_clusters > 0) h->dclus = std::min(h->dclus, h->opts.dense_clusters);
    }
    std::vector<DProb> dp;
    size_t gbytes = 0, nscale = 0;
    build_dense_table(h, win, h->dclus, dp, &gbytes, &nscale);
    h->dprob_h = new DProb[P];
    memcpy(h->dprob_h, dp.data(), sizeof(DProb) * P);
#define DTRY(x) do { e = (x); if (e != cudaSuccess) { helm_set_cuda_error(e); return e == cudaErrorMemoryAllocation ? HELM_ENOMEM : HELM_ECUDA; } } while (0)
    DTRY(cudaMalloc(&h->dprob, sizeof(DProb) * P));
    DTRY(cudaMemcpyAsync(h->dprob, dp.data(), sizeof(DProb) * P, cudaMemcpyHostToDevice, st));
    DTRY(cudaMalloc(&h->dG, gbytes));
    h->dG_bytes = gbytes;
    if (nscale) {
        DTRY(cudaMalloc(&h->dscale, nscale * sizeof(float)));
        h->dscale_elems = nscale;
    }
#undef DTRY
    const int rc = dense_build(h, prob.data(), 0, B - 1, 0, B - 1, st);
    if (rc != HELM_OK) return rc;
    int most = 0;
    for (int p = 0; p < P; ++p) most = std::max(most, dp[p].n_mt);
    // two fronts run two solves side by side: at least two clusters, up to twice the tiles
    const bool two = h->g.sched == HELM_TWO_FRONT;
    h->dclus = std::min(h->dclus, std::max(two ? 2 * most : most, two ? 2 : 1));
    if (two && h->dclus < 2) return HELM_ENOTSUP;
    return HELM_OK;
}

// Right-hand sides of one apply launch padded to a power of two >= 8 (the MMA
// width is 4 x that, the gather maps 256 threads onto the columns).
static int dense_r8(int nr) {
    int r = 8;
    while (r < nr) r <<= 1;
    return r;
}

// Layers of a slab's own block: b for the boundary slabs, at most d otherwise (2d for the two-front centre).
static int dense_dz(const helm_ctx* h) {
    return std::max(h->g.b, h->g.sched == HELM_TWO_FRONT ? 2 * h->g.d : h->g.d);   // two fronts: the centre <= 2d
}

size_t dense_work_elems(const helm_ctx* h, int nrhs) {
    // V, Q, Gv and Zv for one launch group (<= 64 right-hand sides), then the step counter (16 bytes)
    const size_t r8 = (size_t)dense_r8(std::min(nrhs, 64));
    const size_t NN = (size_t)h->g.N * h->g.N;
    return 2 * NN * h->g.Wmax * r8 + 2 * NN * dense_dz(h) * r8 + 2;
}

cudaError_t launch_dense_apply(helm_ctx* h, const float2* r, float2* z, int nrhs, float2* work, cudaStream_t st) {
    const size_t n3 = (size_t)h->g.N * h->g.N * h->g.N;
    const void* kfn = dense_kernel_for(h->opts.precision, h->g.sched);
    const size_t r8max = (size_t)dense_r8(std::min(nrhs, 64));
    const size_t NN = (size_t)h->g.N * h->g.N;
    float2* V = work;
    float2* Qb = V + NN * h->g.Wmax * r8max;
    float2* Gv = Qb + NN * h->g.Wmax * r8max;
    float2* Zv = Gv + NN * dense_dz(h) * r8max;
    unsigned* ctr = reinterpret_cast<unsigned*>(Zv + NN * dense_dz(h) * r8max);
    const int B = h->g.B;
    for (int r0 = 0; r0 < nrhs; r0 += 64) {
        const int nr = std::min(64, nrhs - r0);
        DenseArgs A;
        memset(&A, 0, sizeof(A));
        A.g = h->g;
        A.win = h->t.win;
        A.dp = h->dprob;
        A.G = h->dG;
        A.scale = h->dscale;
        A.c_dn = h->t.c_dn;
        A.c_up = h->t.c_up;
        A.rin = r + (size_t)r0 * n3;
        A.zout = z + (size_t)r0 * n3;
        A.V = V;
        A.Q = Qb;
        A.Gv = Gv;
        A.Zv = Zv;
        A.ctr = ctr;
        A.err = h->dev_err;
        A.nrhs = nr;
        A.R8 = dense_r8(nr);
        A.nclus = h->dclus;
        A.nsteps = (2 * B - 1) * (inner_steps(B, h->g.cen, h->g.sched == HELM_TWO_FRONT) + 1) + 1;
        A.DZ = dense_dz(h);
        A.wait_cycles = h->opts.wait_cycles;
        A.unmet = h->opts.debug_unmet_wait;
        A.unit = tile_unit(h->opts.precision);
        cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = HELM_DENSE_CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(HELM_DENSE_CS * h->dclus, 1, 1);
        cfg.blockDim = dim3(DT, 1, 1);
        cfg.dynamicSmemBytes = h->dsmem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void* args[] = {&A};
        e = cudaLaunchKernelExC(&cfg, kfn, args);
        if (e != cudaSuccess) return e;
        h->launches++;
    }
    return cudaSuccess;
}

int dense_rebuild(helm_ctx* h, int Ma, int Mb, int Pa, int Pb, cudaStream_t st) {
    if (!h->dense || !h->prob_h || !h->dprob_h) return HELM_EINVAL;
    return dense_build(h, h->prob_h, Ma, Mb, Pa, Pb, st);
}

void dense_free(helm_ctx* h) {
    void* ptrs[] = {h->dprob, h->dG, h->dscale, h->dV};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete[] h->dprob_h;
    h->dprob = nullptr;
    h->dprob_h = nullptr;
    h->dG = nullptr;
    h->dscale = nullptr;
    h->dV = nullptr;
}

extern "C" int helm_dense_operator(helm_handle h, int M, int Mp, int dir, int* n_out, int* n_in, int* rects,
                                   void* G, void* stream) {
    if (!h || h->nsub || !h->dense) return HELM_ENOTSUP;
    const int B = h->g.B;
    if (M < 0 || M >= B || Mp < 0 || Mp >= B || dir < 0 || dir > 1) return HELM_EINVAL;
    if (dir == 1 && Mp != 0 && !(h->g.sched == HELM_TWO_FRONT && Mp == B - 1)) return HELM_EINVAL;
    const int p = op_index(M, op_slot(Mp, dir, B), B);
    const DProb& D = h->dprob_h[p];
    if (n_out) *n_out = D.n_out;
    if (n_in) *n_in = D.n_in;
    if (rects) {
        // [nrect, in(4), out0(4), out1(4)]
        rects[0] = D.nrect;
        const DRect rs[3] = {D.in, D.out[0], D.nrect > 1 ? D.out[1] : DRect{0, 0, 0, 0}};
        for (int q = 0; q < 3; ++q) {
            rects[1 + 4 * q] = rs[q].line0;
            rects[2 + 4 * q] = rs[q].nl;
            rects[3 + 4 * q] = rs[q].z0;
            rects[4 + 4 * q] = rs[q].nz;
        }
    }
    if (!G) return HELM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    switch (h->opts.precision) {
        case HELM_SPLIT_FP16: k_dense_unpack<HELM_SPLIT_FP16><<<512, 256, 0, st>>>(D, h->dG, h->dscale, (float2*)G); break;
        case HELM_FP16: k_dense_unpack<HELM_FP16><<<512, 256, 0, st>>>(D, h->dG, h->dscale, (float2*)G); break;
        default: k_dense_unpack<HELM_FP32><<<512, 256, 0, st>>>(D, h->dG, h->dscale, (float2*)G);
    }
    h->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        helm_set_cuda_error(e);
        return HELM_ECUDA;
    }
    return HELM_OK;
}
