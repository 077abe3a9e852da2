// Persistent sweep kernel: the preconditioner apply z = M r.
//
// Algorithm 6 (outer sweep along x3 over slabs M) calls |[T_M]|: embed the
// block's layers into the slab window, run Algorithm 4 (inner sweep along x2
// over line blocks M'), restrict.  Algorithm 4 calls |T~_{M'}|: embed the
// block's lines into the quasi-1D window, solve the block-tridiagonal system
// along x1 with the twisted factors of the setup (left chain T_0..T_{m-1},
// right chain T_{N-1}..T_{m+1}, middle T_m, m = (N-1)/2), restrict:
//   left   y_0 = T_0 q_0,  y_i = T_i (q_i - cdn(i) y_{i-1}),             i < m
//   right  y_{N-1} = T_{N-1} q_{N-1},  y_i = T_i (q_i - cup(i) y_{i+1}),  i > m
//   middle x_m = T_m (q_m - cdn(m) y_{m-1} - cup(m) y_{m+1})
//   back   x_i = y_i - cup(i) T_i x_{i+1} (i < m),  x_i = y_i - cdn(i) T_i x_{i-1} (i > m)
// (the Section 3 solve run from both ends; the x-couplings are scalars).
//
// The apply is a chain of (2B-1)^2 quasi-1D solves.  Right-hand sides are
// independent; a cluster of two CTAs runs the whole chain for one right-hand
// side: CTA 0 owns x in [0, m], CTA 1 owns x in [m+1, N-1].  Everything in
// the sweep except the middle block is local in x, so each CTA gathers,
// eliminates, back-substitutes and scatters its own half; per solve the two
// exchange one k-vector through distributed shared memory (a cluster-scope
// mbarrier), so a solve is N+1 dependent steps instead of 2N-1.  Each CTA
// has a producer warp that walks its static factor stream and fills a TMA
// ring (cp.async.bulk, full/empty mbarriers) with L2 prefetch ahead; eight
// compute warps form each step's row products in 2-row x 8-column tiles
// (128-bit shared loads, row stride with ldk/2 odd) and reduce the chunks in
// shared memory.  Every wait is bounded.
#include "helm_internal.h"

#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <string.h>

namespace cg = cooperative_groups;

namespace {

constexpr int L2_AHEAD = 24;                  // items prefetched into L2 ahead of the ring

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

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void l2_prefetch(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// try_wait with a suspend-time hint: the warp sleeps in hardware until the
// phase completes or the hint (ns) expires, instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns) : "memory");
    return ok != 0;
}
// Bounded wait on a ring barrier: polls without a suspend hint (a released
// stage is seen at once) for at most WAIT_CYCLES SM cycles (about 2 s); false
// if the phase never completed.
constexpr long long WAIT_CYCLES = 4000000000ll;
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < WAIT_CYCLES)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// Soft lockstep of the clusters that sweep one problem.  They read the same
// factor stream; while they stay within a few solves of each other the stream
// is fetched from HBM about once and served to the others from L2, but left
// alone they drift apart over the millions of steps of an apply and each then
// streams the factors from HBM.  After every quasi-1D solve, rank 0 of each
// cluster publishes its solve count; before a solve, a cluster more than
// SOLVES_AHEAD solves ahead of the slowest running one polls until that one
// catches up, for at most THROTTLE_CYCLES.  A counter holds 0 while its cluster
// is not running (zeroed by the host before the launch, reset by the cluster
// when it finishes) and 1 + solves done while it runs, so clusters that wait
// for an SM (more clusters than SMs) or have finished never hold others back.
constexpr int SOLVES_AHEAD = 2;
constexpr long long THROTTLE_CYCLES = 400000;  // about 0.2 ms at 2 GHz

// Kept out of line: inlined, its registers and branches reshape the step
// loop's code and cost about 7 % of the apply.
__device__ __noinline__ void throttle(const int* prog, int n, int mine, int lane) {
    const long long t0 = clock64();
    for (;;) {
        int mn = 0x7fffffff;
        for (int c = lane; c < n; c += 32) {
            const int v = *reinterpret_cast<const volatile int*>(prog + c);
            if (v > 0) mn = min(mn, v - 1);
        }
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        if (mn == 0x7fffffff || mine <= mn + SOLVES_AHEAD || clock64() - t0 > THROTTLE_CYCLES) return;
        __nanosleep(256);
    }
}

struct Ctx {
    Geom g;
    Tables t;
    const unsigned char* factors;   // stored factors (entries of the handle's precision)
    int nsol_in;       // inner solves per slab: 2B-1
    int mode;          // 0: full apply, 1: one slab (M_only)
    int M_only;
    int n_outer;       // slabs visited: 2B-1 (mode 0) or 1 (mode 1)
};

// One problem of a launch: its tables and factors, vectors, work space and ring shape.
struct Item {
    Ctx C;
    const float2* rin;
    float2* zout;
    float2* slab;
    int* err;
    int nrhs, stages, stage_elems, kmax;
};

// A launch covers up to HELM_MAX_BATCH problems; cluster c (two CTAs) serves
// right-hand side c - rhs_begin[p] of the problem p with rhs_begin[p] <= c.
struct SweepArgs {
    int nitems;
    int rhs_begin[HELM_MAX_BATCH + 1];
    Item items[HELM_MAX_BATCH];
};

// Index of stream item t of a solve for cluster rank r (forward, middle, back).
__device__ __forceinline__ int item_x(int r, int t, int N) {
    const int m = (N - 1) / 2, L = N - 1 - m;
    if (r == 0) return (t < m) ? t : ((t == m) ? m : 2 * m - t);
    return (t < L) ? N - 1 - t : ((t == L) ? m : m + (t - L));
}

// Walks this rank's static factor stream in consumption order.
struct StreamIter {
    int jo, ji, t, per;
    long long base;    // factor offset of the current problem (float2 units)
    int kstride;
    bool done;

    __device__ void load(const Ctx& C) {
        const int B = C.g.B;
        int M = (C.mode == 1) ? C.M_only : ((jo < B) ? jo : 2 * B - 2 - jo);
        int Mp = (ji < B) ? ji : 2 * B - 2 - ji;
        const Prob* P = C.t.prob + (M * B + Mp);
        base = P->off;
        kstride = P->kstride;
    }
    __device__ void start(const Ctx& C, int r) {
        const int N = C.g.N, m = (N - 1) / 2;
        per = (r == 0) ? 2 * m + 1 : 2 * (N - 1 - m) + 1;
        jo = ji = t = 0;
        done = false;
        load(C);
    }
    __device__ void next(const Ctx& C) {
        if (++t < per) return;
        t = 0;
        if (++ji == C.nsol_in) {
            ji = 0;
            if (++jo == C.n_outer) { done = true; return; }
        }
        load(C);
    }
    __device__ const unsigned char* ptr(const Ctx& C, int r, int esz) const {
        return C.factors + (size_t)(base + (long long)item_x(r, t, C.g.N) * kstride) * esz;
    }
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Producer warp (one lane): fill the ring in stream order; a stage is refilled
// once the compute warps have released it through its "empty" barrier.
template <int ESZ>
__device__ void produce(const Ctx& C, int r, unsigned char* ring, int stages, int stage_elems, uint64_t* full,
                        uint64_t* empty, int* err, int* s_perr) {
    StreamIter fill, pf;
    fill.start(C, r);
    pf.start(C, r);
    for (int q = 0; q < L2_AHEAD && !pf.done; ++q) pf.next(C);
    int stg = 0;
    uint32_t round = 0;
    while (!fill.done) {
        if (round > 0 && !mbar_wait(&empty[stg], (round - 1) & 1)) {
            atomicOr(err, 2);
            *s_perr = 1;
            return;
        }
        bulk_load(ring + (size_t)stg * stage_elems * ESZ, fill.ptr(C, r, ESZ), (uint32_t)(fill.kstride * ESZ),
                  &full[stg]);
        if (!pf.done) {
            l2_prefetch(pf.ptr(C, r, ESZ), (uint32_t)(pf.kstride * ESZ));
            pf.next(C);
        }
        fill.next(C);
        if (++stg == stages) { stg = 0; ++round; }
    }
}

constexpr int NT = 256;                       // compute threads (8 warps)
// The producer is hardware warp 7: warps share an SM sub-partition by warp
// index mod 4, and sub-partition 3 otherwise hosts a single product warp, while
// sub-partition 0 holds the first reduction warp.  Compute threads are warps
// 0-6 and 8, numbered ct = 0..255 (hardware warp 8 takes column chunk 7).
constexpr int PRODUCER_WARP = 7;

__device__ __forceinline__ void named_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }

__device__ __forceinline__ uint32_t peer_smem(const void* local, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(local)), "r"(rank));
    return out;
}
__device__ __forceinline__ void st_peer(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void arrive_peer(uint32_t bar_addr) {
    asm volatile("fence.acq_rel.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_addr) : "memory");
}
__device__ __forceinline__ bool xbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bytes per stored factor entry of each precision.
template <int FMT> struct StoredEntry { static constexpr int bytes = 8; };
template <> struct StoredEntry<HELM_FP16> { static constexpr int bytes = 4; };

__device__ __forceinline__ float2 h2f(unsigned u) {
    __half2 h;
    memcpy(&h, &u, sizeof(h));
    return __half22float2(h);
}

// Row products of one step: thread (rp, q8) forms partial products of rows rp
// and rp+32 over the 8-column chunk q8 into Pp.  Rows are zero padded to whole
// 8-column chunks and W is zero beyond k, so a chunk needs no bounds test.
// FP32 entries: 4 x 16-byte loads per row.  FP16 entries: 2 loads per row,
// each half pair widened to FP32, the block scale applied to the partial sums.
// SPLIT_FP16 entries: hi + lo widened and added in FP32 (exact: the pair holds
// at most 22 significant bits), 4 loads per row, then the scale.
// The chunk of the step input a thread multiplies, read before its ring stage
// is waited for (it does not depend on the stage).
__device__ __forceinline__ void load_w(const float2* __restrict__ W, int k, int q8, float2 (&w)[8]) {
    const int b0 = q8 * 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = (b0 < k) ? W[b0 + j] : make_float2(0.f, 0.f);
}

template <int FMT>
__device__ __forceinline__ void step_products(const unsigned char* __restrict__ Tb, const float2 (&w)[8],
                                              float2* __restrict__ Pp, int k, int ldk, int rp, int q8) {
    constexpr int ESZ = StoredEntry<FMT>::bytes;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
    const int b0 = q8 * 8;
    if (b0 < k) {
        const bool r0ok = rp < k, r1ok = rp + 32 < k;
        const uint4* T0 = reinterpret_cast<const uint4*>(Tb + ((size_t)rp * ldk + b0) * ESZ);
        const uint4* T1 = reinterpret_cast<const uint4*>(Tb + ((size_t)(rp + 32) * ldk + b0) * ESZ);
        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
        constexpr int NV = 8 * ESZ / 16;          // 16-byte loads per row chunk
        uint4 t0[NV], t1[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            t0[j] = r0ok ? T0[j] : z4;
            t1[j] = r1ok ? T1[j] : z4;
        }
        if (FMT == HELM_FP32) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                cfma(acc0, make_float2(__uint_as_float(t0[j].x), __uint_as_float(t0[j].y)), w[2 * j]);
                cfma(acc0, make_float2(__uint_as_float(t0[j].z), __uint_as_float(t0[j].w)), w[2 * j + 1]);
                cfma(acc1, make_float2(__uint_as_float(t1[j].x), __uint_as_float(t1[j].y)), w[2 * j]);
                cfma(acc1, make_float2(__uint_as_float(t1[j].z), __uint_as_float(t1[j].w)), w[2 * j + 1]);
            }
        } else if (FMT == HELM_FP16) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                cfma(acc0, h2f(t0[j].x), w[4 * j]);
                cfma(acc0, h2f(t0[j].y), w[4 * j + 1]);
                cfma(acc0, h2f(t0[j].z), w[4 * j + 2]);
                cfma(acc0, h2f(t0[j].w), w[4 * j + 3]);
                cfma(acc1, h2f(t1[j].x), w[4 * j]);
                cfma(acc1, h2f(t1[j].y), w[4 * j + 1]);
                cfma(acc1, h2f(t1[j].z), w[4 * j + 2]);
                cfma(acc1, h2f(t1[j].w), w[4 * j + 3]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                cfma(acc0, cadd(h2f(t0[j].x), h2f(t0[j].y)), w[2 * j]);
                cfma(acc0, cadd(h2f(t0[j].z), h2f(t0[j].w)), w[2 * j + 1]);
                cfma(acc1, cadd(h2f(t1[j].x), h2f(t1[j].y)), w[2 * j]);
                cfma(acc1, cadd(h2f(t1[j].z), h2f(t1[j].w)), w[2 * j + 1]);
            }
        }
        if (FMT != HELM_FP32) {
            const float sc = *reinterpret_cast<const float*>(Tb + (size_t)(ldk - 1) * ESZ);   // row 0, last column
            acc0 = make_float2(acc0.x * sc, acc0.y * sc);
            acc1 = make_float2(acc1.x * sc, acc1.y * sc);
        }
    }
    Pp[q8 * 64 + rp] = acc0;
    Pp[q8 * 64 + rp + 32] = acc1;
}

// Sum of the eight chunk partials of row a (chunks past k hold zeros).
__device__ __forceinline__ float2 chunk_sum(const float2* __restrict__ Pp, int a) {
    float2 pq[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) pq[q] = Pp[q * 64 + a];
    return cadd(cadd(cadd(pq[0], pq[1]), cadd(pq[2], pq[3])), cadd(cadd(pq[4], pq[5]), cadd(pq[6], pq[7])));
}

template <int FMT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NT + 32, 1)
k_sweep(const __grid_constant__ SweepArgs A) {
    constexpr int ESZ = StoredEntry<FMT>::bytes;
    extern __shared__ __align__(128) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    // ---- which problem and right-hand side this cluster serves ----
    const int cidx = blockIdx.x / 2;
    int pi = 0;
    while (pi + 1 < A.nitems && cidx >= A.rhs_begin[pi + 1]) ++pi;
    const Item& I = A.items[pi];
    const Ctx& C = I.C;
    const float2* __restrict__ rin = I.rin;
    float2* __restrict__ zout = I.zout;
    float2* __restrict__ slab_all = I.slab;
    int* err = I.err;
    const int nrhs = I.nrhs, stages = I.stages, stage_elems = I.stage_elems, kmax = I.kmax;
    const int N = C.g.N, B = C.g.B, Wmax = C.g.Wmax;
    const int m = (N - 1) / 2, L = N - 1 - m;
    const int tid = threadIdx.x;
    const int r = (int)cluster.block_rank();
    const int col = cidx - A.rhs_begin[pi];               // the right-hand side of this cluster
    const int nf = (r == 0) ? m : L;                      // forward steps of this half
    const int xlo = (r == 0) ? 0 : m + 1;                 // owned x range [xlo, xhi]
    const int xhi = (r == 0) ? m : N - 1;
    const int nslot = (N + 1) / 2;
    // ---- shared memory carve-up (ring first: 16-byte aligned TMA targets) ----
    unsigned char* ring = smem;
    // Y slot x - xlo holds the solve's input q_x on the interest entries until the
    // step before x has consumed it, then y_x (forward), then x_x (backward).
    float2* Y = reinterpret_cast<float2*>(ring + (size_t)stages * stage_elems * ESZ);   // [nslot][kmax]
    float2* W = Y + (((size_t)nslot * kmax + 1) & ~(size_t)1);        // [64] step input
    float2* Pp = W + 64;                                              // [8][64] partial sums
    float2* s_cdn = Pp + 8 * 64;                                      // [N] coupling g -> g-1
    float2* s_cup = s_cdn + N;                                        // [N] coupling g -> g+1
    float2* xbuf = s_cup + N;                                         // [2][64] from the peer
    float2* xown = xbuf + 128;                                        // [64] own half of the middle input
    float2* pre_s = xown + 64;                                        // [64] finish operand per row
    float2* cp_s = pre_s + 64;                                        // [2]  finish coupling
    uint64_t* full = reinterpret_cast<uint64_t*>(cp_s + 2);
    uint64_t* empty = full + stages;
    uint64_t* xbar = empty + stages;
    // s_err: the compute warps' stop flag, written only by compute threads before
    // a barrier that precedes every read of it, so all of them take the same
    // branch; the producer reports through s_perr (a failed producer leaves the
    // compute warps' own waits to expire).
    int* s_err = reinterpret_cast<int*>(xbar + 1);
    int* s_perr = s_err + 1;

    for (int q = tid; q < N; q += blockDim.x) {
        s_cdn[q] = C.t.c_dn[q];
        s_cup[q] = C.t.c_up[q];
    }
    for (int q = tid; q < 64; q += blockDim.x) W[q] = make_float2(0.f, 0.f);
    if (tid == 0) {
        for (int q = 0; q < stages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        mbar_init(xbar, 1);
        *s_err = 0;
        *s_perr = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cluster.sync();                                       // peers see initialised barriers
    const uint32_t peer = (uint32_t)(r ^ 1);
    const uint32_t peer_xbar = peer_smem(xbar, peer);

    const int ct = (tid < PRODUCER_WARP * 32) ? tid : tid - 32;   // compute thread index
    if ((tid >> 5) == PRODUCER_WARP) {                    // producer warp
        if ((tid & 31) == 0 && col < nrhs) produce<ESZ>(C, r, ring, stages, stage_elems, full, empty, err, s_perr);
    } else if (col < nrhs) {
        float2* V = slab_all + (size_t)col * ((size_t)N * N * Wmax);
        // per-cluster solve counters of this problem, after the slab vectors
        int* prog = reinterpret_cast<int*>(slab_all + (size_t)nrhs * ((size_t)N * N * Wmax));
        int done = 0;                                    // inner solves this cluster has finished
        if (r == 0 && ct == 0) atomicExch(prog + col, 1);   // running, no solve done
        const long long NN = (long long)N * N, N3 = NN * N;
        const int rp = ct & 31, q8 = ct >> 5;          // product phase: row pair, column chunk
        const int pa = ct;                              // reduction phase: row
        int stg = 0;
        uint32_t phase = 0, xpar = 0;
        const int xw = xhi - xlo + 1;

        for (int jo = 0; jo < C.n_outer && !*s_err; ++jo) {
            const int M = (C.mode == 1) ? C.M_only : ((jo < B) ? jo : 2 * B - 2 - jo);
            const bool outer_fwd = (C.mode == 1) || (jo < B);
            const AxisWin wz = C.t.win[M];
            const int za = (C.mode == 1) ? 0 : wz.ia, zb = (C.mode == 1) ? wz.L : wz.ib;
            // ---- embed the outer right-hand side into the slab window (owned x) ----
            if (C.mode == 0) {
                const int zb0 = wz.lo + wz.ia, zb1 = wz.lo + wz.ib;
                const long long cnt = (long long)(zb1 - zb0) * N * xw;
                for (long long e = ct; e < cnt; e += NT) {
                    const int x = xlo + (int)(e % xw);
                    const long long rest = e / xw;
                    const int y = (int)(rest % N);
                    const int z = zb0 + (int)(rest / N);
                    const long long gi = (long long)col * N3 + (long long)z * NN + (long long)y * N + x;
                    float2 v = make_float2(0.f, 0.f);
                    if (outer_fwd) {
                        v = rin[gi];
                        if (M > 0 && z == zb0) v = csub(v, cmul(s_cdn[z], zout[gi - NN]));
                    } else if (z == zb1 - 1) {
                        v = cmul(s_cup[z], zout[gi + NN]);
                    }
                    V[((size_t)x * N + y) * Wmax + (z - wz.lo)] = v;
                }
            } else {
                const long long cnt = (long long)wz.L * N * xw;
                for (long long e = ct; e < cnt; e += NT) {
                    const int x = xlo + (int)(e % xw);
                    const long long rest = e / xw;
                    const int y = (int)(rest % N);
                    const int lz = (int)(rest / N);
                    V[((size_t)x * N + y) * Wmax + lz] =
                        rin[(long long)col * wz.L * NN + (long long)lz * NN + (long long)y * N + x];
                }
            }
            named_sync();

            for (int ji = 0; ji < C.nsol_in && !*s_err; ++ji) {
                if (r == 0 && ct < 32) throttle(prog, nrhs, done, ct);
                const int Mp = (ji < B) ? ji : 2 * B - 2 - ji;
                const bool inner_fwd = ji < B;
                const Prob P = C.t.prob[M * B + Mp];
                const int k = P.k, Lz = P.Lz, a0 = P.a0, ni = P.ni, ldk = P.ldk;
                // ---- gather the solve's input on its interest entries (owned x) ----
                for (int e = ct; e < xw * ni; e += NT) {
                    const int ai = e % ni, x = xlo + e / ni;
                    const int a = a0 + ai;
                    const int lz = a % Lz, y = P.ylo + a / Lz;
                    const size_t vrow = ((size_t)x * N + y) * Wmax + lz;
                    float2 v = make_float2(0.f, 0.f);
                    if (inner_fwd) {
                        if (lz >= za && lz < zb) v = V[vrow];
                        if (Mp > 0 && y == P.yb0) v = csub(v, cmul(s_cdn[y], V[vrow - (size_t)Wmax]));
                    } else if (y == P.yb1 - 1) {
                        v = cmul(s_cup[y], V[vrow + (size_t)Wmax]);
                    }
                    Y[(size_t)(x - xlo) * kmax + a] = v;
                }
                named_sync();
                // input of the first step: q at this half's outer end
                {
                    const int x0 = (r == 0) ? 0 : N - 1;
                    if (pa < 64) {
                        float2 w = make_float2(0.f, 0.f);
                        if (pa >= a0 && pa < a0 + ni) w = Y[(size_t)(x0 - xlo) * kmax + pa];
                        W[pa] = w;
                    }
                }
                named_sync();

                for (int t = 0; t < 2 * nf + 1; ++t) {
                    const int i = item_x(r, t, N);
                    // operands of this step's finish, read during the products by the
                    // last two compute warps (their column chunks are the lightest)
                    if (ct >= NT - 64) {
                        const int a = ct - (NT - 64);
                        const bool a_int = a >= a0 && a < a0 + ni;   // row a is an interest entry
                        float2 pv = make_float2(0.f, 0.f), cv = pv;
                        if (t + 1 < nf) {                              // next forward input: q, coupling
                            const int in = (r == 0) ? i + 1 : i - 1;
                            cv = (r == 0) ? s_cdn[in] : s_cup[in];
                            if (a_int) pv = Y[(size_t)(in - xlo) * kmax + a];
                        } else if (t + 1 == nf) {                      // middle-input share
                            cv = (r == 0) ? s_cdn[m] : s_cup[m];
                            if (r == 0 && a_int) pv = Y[(size_t)(m - xlo) * kmax + a];
                        } else if (t > nf && a < k) {                  // back substitution: y_i
                            cv = (r == 0) ? s_cup[i] : s_cdn[i];
                            pv = Y[(size_t)(i - xlo) * kmax + a];
                        }
                        pre_s[a] = pv;
                        if (a == 0) *cp_s = cv;
                    }
                    float2 w[8];
                    load_w(W, k, q8, w);
                    // ---- wait for T_i, partial products ----
                    if (!mbar_wait(&full[stg], phase)) {
                        atomicOr(err, 2);
                        *s_err = 1;
                    }
                    step_products<FMT>(ring + (size_t)stg * stage_elems * ESZ, w, Pp, k, ldk, rp, q8);
                    named_sync();
                    const int stop = *s_err;                           // set before the barrier above, if at all
                    if (ct == NT - 1) mbar_arrive(&empty[stg]);       // stage consumed (a lane outside the reduction)
                    if (++stg == stages) { stg = 0; phase ^= 1u; }
                    // ---- reduce the chunks, finish the step, form the next input ----
                    if (pa < k) {
                        const int a = pa;
                        const float2 pre = pre_s[a], cp = *cp_s;
                        const float2 sum = chunk_sum(Pp, a);
                        float2* Yi = Y + (size_t)(i - xlo) * kmax + a;
                        if (t < nf) {                                  // forward elimination
                            *Yi = sum;                                 // y_i
                            if (t + 1 < nf) {
                                W[a] = csub(pre, cmul(cp, sum));
                            } else {                                   // q_m - cdn(m) y_{m-1}  or  cup(m) y_{m+1}
                                const float2 h = (r == 0) ? csub(pre, cmul(cp, sum)) : cmul(cp, sum);
                                xown[a] = h;
                                st_peer(peer_smem(xbuf + xpar * 64 + a, peer), h);
                            }
                        } else if (t == nf) {                          // middle block: x_m
                            W[a] = sum;
                            if (r == 0) *Yi = sum;
                        } else {                                       // back substitution
                            const float2 x = csub(pre, cmul(cp, sum));
                            W[a] = x;
                            *Yi = x;                                   // slot now holds x_i
                        }
                    }
                    named_sync();
                    if (stop) break;
                    if (t == nf - 1) {
                        // exchange the halves of the middle input through the cluster
                        if (ct == 0) arrive_peer(peer_xbar);
                        bool ok = xbar_try(xbar, xpar);            // polled, bounded like the ring waits
                        for (const long long x0 = clock64(); !ok && clock64() - x0 < WAIT_CYCLES;)
                            ok = xbar_try(xbar, xpar);
                        if (!ok) {
                            atomicOr(err, 2);
                            *s_err = 1;
                        }
                        if (pa < 64) {
                            float2 w = make_float2(0.f, 0.f);
                            if (pa < k) {
                                const float2 mine = xown[pa], theirs = xbuf[xpar * 64 + pa];
                                w = (r == 0) ? csub(mine, theirs) : csub(theirs, mine);
                            }
                            W[pa] = w;
                        }
                        xpar ^= 1u;
                        named_sync();
                        if (*s_err) break;
                    }
                }
                if (*s_err) break;
                // ---- scatter the restricted solution (owned x) into the slab ----
                for (int e = ct; e < xw * ni; e += NT) {
                    const int ai = e % ni, x = xlo + e / ni;
                    const int a = a0 + ai;
                    const int lz = a % Lz, y = P.ylo + a / Lz;
                    const float2 v = Y[(size_t)(x - xlo) * kmax + a];
                    float2* dst = V + ((size_t)x * N + y) * Wmax + lz;
                    if (inner_fwd) *dst = v;
                    else *dst = csub(*dst, v);
                }
                named_sync();
                ++done;
                if (r == 0 && ct == 0) __stcg(prog + col, done + 1);
            }
            if (*s_err) break;
            // ---- restrict the slab to the block's layers (owned x) ----
            if (C.mode == 0) {
                const int zb0 = wz.lo + wz.ia, zb1 = wz.lo + wz.ib;
                const long long cnt = (long long)(zb1 - zb0) * N * xw;
                for (long long e = ct; e < cnt; e += NT) {
                    const int x = xlo + (int)(e % xw);
                    const long long rest = e / xw;
                    const int y = (int)(rest % N);
                    const int z = zb0 + (int)(rest / N);
                    const float2 v = V[((size_t)x * N + y) * Wmax + (z - wz.lo)];
                    const long long gi = (long long)col * N3 + (long long)z * NN + (long long)y * N + x;
                    if (outer_fwd) zout[gi] = v;
                    else zout[gi] = csub(zout[gi], v);
                }
            } else {
                const long long cnt = (long long)wz.L * N * xw;
                for (long long e = ct; e < cnt; e += NT) {
                    const int x = xlo + (int)(e % xw);
                    const long long rest = e / xw;
                    const int y = (int)(rest % N);
                    const int lz = (int)(rest / N);
                    zout[(long long)col * wz.L * NN + (long long)lz * NN + (long long)y * N + x] =
                        V[((size_t)x * N + y) * Wmax + lz];
                }
            }
            named_sync();
        }
        if (r == 0 && ct == 0) __stcg(prog + col, 0);       // no longer running
        if (*s_err && ct == 0) {
            // error path: let the copies already in flight land (bounded)
            int q = stg;
            uint32_t ph = phase;
            for (int d = 0; d < stages; ++d) {
                for (int it = 0; it < (1 << 12) && !mbar_try_sleep(&full[q], ph, 1000u); ++it) {
                }
                if (++q == stages) { q = 0; ph ^= 1u; }
            }
        }
    }
    cluster.sync();                                       // no CTA leaves while its peer may write to it
}

size_t sweep_smem_bytes(const helm_ctx* h, int stages) {
    const int N = h->g.N, kmax = h->kmax;
    const size_t nslot = (size_t)(N + 1) / 2;
    size_t f2 = ((nslot * kmax + 1) & ~(size_t)1) + 64 + 8 * 64 + (size_t)2 * N + 128 + 64 + 66;
    return (size_t)stages * h->stage_elems * h->esz + f2 * sizeof(float2) +
           (size_t)(2 * stages + 1) * sizeof(uint64_t) + 16;
}

}  // namespace

int sweep_config_stages(helm_ctx* h, int stages) {
    const size_t b = sweep_smem_bytes(h, stages);
    if (stages < 2 || b > (size_t)227 * 1024) return HELM_ENOTSUP;
    h->sweep_stages = stages;
    h->sweep_smem = b;
    return HELM_OK;
}

int sweep_configure(helm_ctx* h) {
    const int limit = 227 * 1024;
    if (h->opts.rhs_per_cta > 1) return HELM_ENOTSUP;
    for (int stages = 8; stages >= 2; --stages) {
        size_t b = sweep_smem_bytes(h, stages);
        if (b <= (size_t)limit) {
            h->sweep_rc = 1;
            h->sweep_stages = stages;
            h->sweep_smem = b;
            return HELM_OK;
        }
    }
    return HELM_ENOTSUP;
}

// Work space of one launch for nrhs right-hand sides, in float2 units: the
// slab vectors, then one solve counter (int) per cluster.
static size_t slab_need(const helm_ctx* h, int nrhs) {
    return (size_t)nrhs * h->g.N * h->g.N * h->g.Wmax + ((size_t)nrhs + 1) / 2;
}

// Grows the handle's work space; new counters start at zero.
static cudaError_t ensure_slab(helm_ctx* h, int nrhs, cudaStream_t st) {
    const size_t need = slab_need(h, nrhs);
    if (need <= h->slab_elems) return cudaSuccess;
    if (h->slab) cudaFree(h->slab);
    h->slab = nullptr;
    h->slab_elems = 0;
    cudaError_t e = cudaMalloc(&h->slab, need * sizeof(float2));
    if (e != cudaSuccess) return e;
    h->slab_elems = need;
    return cudaMemsetAsync(h->slab, 0, need * sizeof(float2), st);
}

// Marks every cluster of a launch as not running (its pacing counter = 0).
static cudaError_t clear_counters(const helm_ctx* h, float2* slab, int nrhs, cudaStream_t st) {
    int* prog = reinterpret_cast<int*>(slab + (size_t)nrhs * h->g.N * h->g.N * h->g.Wmax);
    return cudaMemsetAsync(prog, 0, sizeof(int) * (size_t)nrhs, st);
}

static void make_item(helm_ctx* h, const float2* r, float2* z, int nrhs, int slab_only, int M_only,
                      float2* slab, Item* it) {
    it->C.g = h->g;
    it->C.t = h->t;
    it->C.factors = reinterpret_cast<const unsigned char*>(h->factors);
    it->C.nsol_in = 2 * h->g.B - 1;
    it->C.mode = slab_only ? 1 : 0;
    it->C.M_only = M_only;
    it->C.n_outer = slab_only ? 1 : 2 * h->g.B - 1;
    it->rin = r;
    it->zout = z;
    it->slab = slab;
    it->err = h->dev_err;
    it->nrhs = nrhs;
    it->stages = h->sweep_stages;
    it->stage_elems = h->stage_elems;
    it->kmax = h->kmax;
}

template <int FMT>
static cudaError_t launch_fmt(const SweepArgs& A, size_t smem, cudaStream_t st) {
    cudaError_t e = ensure_dyn_smem((const void*)k_sweep<FMT>, smem);
    if (e != cudaSuccess) return e;
    k_sweep<FMT><<<2 * A.rhs_begin[A.nitems], NT + 32, smem, st>>>(A);
    return cudaGetLastError();
}

static cudaError_t launch_args(const SweepArgs& A, int fmt, size_t smem, cudaStream_t st) {
    switch (fmt) {
        case HELM_FP16: return launch_fmt<HELM_FP16>(A, smem, st);
        case HELM_SPLIT_FP16: return launch_fmt<HELM_SPLIT_FP16>(A, smem, st);
        default: return launch_fmt<HELM_FP32>(A, smem, st);
    }
}

static cudaError_t launch_sweep_on(helm_ctx* h, const float2* r, float2* z, int nrhs, int slab_only,
                                   int M_only, float2* slab, cudaStream_t st) {
    SweepArgs A;
    memset(&A, 0, sizeof(A));
    A.nitems = 1;
    A.rhs_begin[0] = 0;
    A.rhs_begin[1] = nrhs;
    make_item(h, r, z, nrhs, slab_only, M_only, slab, &A.items[0]);
    cudaError_t e = clear_counters(h, slab, nrhs, st);
    if (e != cudaSuccess) return e;
    h->launches++;
    return launch_args(A, h->opts.precision, h->sweep_smem, st);
}

// One launch over several problems (each with its own handle, vectors and
// work space); the dynamic shared memory is the largest any problem needs.
cudaError_t launch_sweep_batch(helm_ctx* const* hs, const float2* const* r, float2* const* z,
                               const int* nrhs, int n, cudaStream_t st) {
    if (n < 1 || n > HELM_MAX_BATCH) return cudaErrorInvalidValue;
    for (int p = 1; p < n; ++p)
        if (hs[p]->opts.precision != hs[0]->opts.precision || hs[p]->dense != hs[0]->dense)
            return cudaErrorInvalidValue;
    if (hs[0]->dense) {
        // every dense launch spans the whole GPU: the problems run one after the other
        for (int p = 0; p < n; ++p) {
            cudaError_t e = launch_sweep(hs[p], r[p], z[p], nrhs[p], 0, 0, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    SweepArgs A;
    memset(&A, 0, sizeof(A));
    A.nitems = n;
    size_t smem = 0;
    for (int p = 0; p < n; ++p) {
        helm_ctx* h = hs[p];
        cudaError_t e = ensure_slab(h, nrhs[p], st);
        if (e != cudaSuccess) return e;
        A.rhs_begin[p + 1] = A.rhs_begin[p] + nrhs[p];
        make_item(h, r[p], z[p], nrhs[p], 0, 0, h->slab, &A.items[p]);
        e = clear_counters(h, h->slab, nrhs[p], st);
        if (e != cudaSuccess) return e;
        if (h->sweep_smem > smem) smem = h->sweep_smem;
        h->launches++;
    }
    return launch_args(A, hs[0]->opts.precision, smem, st);
}

// Everything an apply of nrhs right-hand sides needs besides its launches (work
// space, the kernel's shared-memory limit), so that the launches alone can be
// captured into a CUDA graph.
cudaError_t sweep_prepare(helm_ctx* h, int nrhs, cudaStream_t st) {
    if (h->dense) {
        const size_t need = dense_work_elems(h, nrhs);
        if (need > h->dV_elems) {
            if (h->dV) cudaFree(h->dV);
            h->dV = nullptr;
            h->dV_elems = 0;
            cudaError_t e = cudaMalloc(&h->dV, need * sizeof(float2));
            if (e != cudaSuccess) return e;
            h->dV_elems = need;
        }
        return cudaSuccess;
    }
    cudaError_t e = ensure_slab(h, nrhs, st);
    if (e != cudaSuccess) return e;
    switch (h->opts.precision) {
        case HELM_FP16: return ensure_dyn_smem((const void*)k_sweep<HELM_FP16>, h->sweep_smem);
        case HELM_SPLIT_FP16: return ensure_dyn_smem((const void*)k_sweep<HELM_SPLIT_FP16>, h->sweep_smem);
        default: return ensure_dyn_smem((const void*)k_sweep<HELM_FP32>, h->sweep_smem);
    }
}

cudaError_t launch_sweep(helm_ctx* h, const float2* r, float2* z, int nrhs, int slab_only, int M_only,
                         cudaStream_t st) {
    if (h->dense) {
        if (slab_only) return cudaErrorNotSupported;
        const size_t need = dense_work_elems(h, nrhs);
        if (need > h->dV_elems) {
            if (h->dV) cudaFree(h->dV);
            h->dV = nullptr;
            h->dV_elems = 0;
            cudaError_t e = cudaMalloc(&h->dV, need * sizeof(float2));
            if (e != cudaSuccess) return e;
            h->dV_elems = need;
        }
        return launch_dense_apply(h, r, z, nrhs, h->dV, st);
    }
    cudaError_t e = ensure_slab(h, nrhs, st);
    if (e != cudaSuccess) return e;
    return launch_sweep_on(h, r, z, nrhs, slab_only, M_only, h->slab, st);
}

// ---------------------------------------------------------------------------
// Apply without allocation: the slab work space lives in one file-scope device
// array of HELM_NOALLOC_SCRATCH_BYTES.  Host code cannot use the array's name
// as a device address (it is a host-side stand-in), so its address is looked
// up with cudaGetSymbolAddress on every call, with the handle's device
// current.  The lookup allocates nothing and is cheap; not caching it keeps a
// stale address from surviving a context teardown (cudaDeviceReset reloads
// the module, and the array may then sit elsewhere).

static __device__ __align__(256) float2 g_noalloc_scratch[HELM_NOALLOC_SCRATCH_BYTES / sizeof(float2)];

extern "C" int helm_apply_precond_noalloc(helm_handle h, const void* r, void* z, int nrhs, void* stream) {
    if (h && h->nsub) return HELM_ENOTSUP;                 // batch handles: use helm_apply_precond
    if (!h || !r || !z || nrhs < 1 || r == z) return HELM_EINVAL;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        helm_set_cuda_error(e);
        return HELM_ECUDA;
    }
    if (dev != h->device) return HELM_EINVAL;             // the handle's factors live on another GPU
    const size_t need = h->dense ? dense_work_elems(h, nrhs) : slab_need(h, nrhs);
    if (need > HELM_NOALLOC_SCRATCH_BYTES / sizeof(float2)) return HELM_EINVAL;
    void* scratch = nullptr;
    e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
    if (e != cudaSuccess) {
        helm_set_cuda_error(e);
        return HELM_ECUDA;
    }
    e = h->dense ? launch_dense_apply(h, (const float2*)r, (float2*)z, nrhs, static_cast<float2*>(scratch),
                                      (cudaStream_t)stream)
                 : launch_sweep_on(h, (const float2*)r, (float2*)z, nrhs, 0, 0, static_cast<float2*>(scratch),
                                   (cudaStream_t)stream);
    if (e != cudaSuccess) {
        helm_set_cuda_error(e);
        return (e == cudaErrorMemoryAllocation) ? HELM_ENOMEM : HELM_ECUDA;
    }
    return HELM_OK;
}
