// Persistent sweep kernel: the preconditioner apply z = M r.
//
// Algorithm 6 (outer sweep along x3 over slabs M) calls |[T_M]|: embed the
// block's layers into the slab window, run Algorithm 4 (inner sweep along x2
// over line blocks M'), restrict.  Algorithm 4 calls |T~_{M'}|: embed the
// block's lines into the quasi-1D window, solve by the block LDU along x1,
// restrict.  With T_i = S_i^{-1} from the setup:
//     forward   y_0 = T_0 q_0,  y_i = T_i (q_i - cdn(i) y_{i-1})
//     backward  x_{N-1} = y_{N-1},  x_i = y_i - cup(i) T_i x_{i+1}
// (the Section 3 solve, with the x-couplings being scalars).
//
// The whole apply is one dependency chain of (2B-1)^2 quasi-1D solves of
// 2N-1 block steps each, so one CTA runs the entire chain for a group of RC
// right-hand sides; groups are independent (no inter-CTA waits).  All CTAs
// walk the same factor stream, so the factors are read from HBM about once
// per use and shared through L2.  The stream is static: thread 0 issues
// TMA bulk copies (cp.async.bulk) of T_i into a ring of shared-memory
// stages, signalled by mbarriers, and prefetches further ahead into L2.
//
// Per step: every thread (row a, quarter q of the columns) forms a partial
// row-vector product over RC columns; the quarters are summed by the
// threads (a, c) that then form the next step's input.
#include "helm_internal.h"

namespace {

constexpr int NT = 256;
constexpr long long WAIT_LIMIT = 1LL << 26;   // bounded mbarrier spin (seconds)
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
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (it > 256) __nanosleep(64);
    }
    return false;
}

struct Ctx {
    Geom g;
    Tables t;
    const float2* factors;
    int nsol_in;       // inner solves per slab: 2B-1
    int per_solve;     // stream items per solve: 2N-1
    int mode;          // 0: full apply, 1: one slab (M_only)
    int M_only;
};

__device__ __forceinline__ void solve_index(const Ctx& C, long long j, int& M, int& Mp) {
    const int B = C.g.B;
    long long jo = j / C.nsol_in;
    int ji = (int)(j - jo * C.nsol_in);
    if (C.mode == 1) M = C.M_only;
    else M = (jo < B) ? (int)jo : (int)(2 * B - 2 - jo);
    Mp = (ji < B) ? ji : 2 * B - 2 - ji;
}

// Factor block of stream item s (thread 0 only).
__device__ __forceinline__ const float2* item_ptr(const Ctx& C, long long s, uint32_t& bytes) {
    long long j = s / C.per_solve;
    int tt = (int)(s - j * C.per_solve);
    int M, Mp;
    solve_index(C, j, M, Mp);
    const Prob P = C.t.prob[M * C.g.B + Mp];
    int i = (tt < C.g.N) ? tt : 2 * C.g.N - 2 - tt;
    bytes = (uint32_t)P.kstride * 8u;
    return C.factors + P.off + (long long)i * P.kstride;
}

template <int RC>
__global__ void __launch_bounds__(NT, 1)
k_sweep(Ctx C, const float2* __restrict__ rin, float2* __restrict__ zout, float2* __restrict__ slab_all,
        int nrhs, int stages, int stage_elems, int kmax, long long total_items, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int N = C.g.N, B = C.g.B, Wmax = C.g.Wmax;
    const int tid = threadIdx.x;
    // ---- shared memory carve-up (ring first: 16-byte aligned TMA targets) ----
    float2* ring = reinterpret_cast<float2*>(smem);
    // Y slot i holds the solve's input q_i on the interest entries until the
    // step before i has consumed it, then y_i (the forward-substitution result).
    float2* Y = ring + (size_t)stages * stage_elems;      // [N][kmax][RC]
    float2* W = Y + (size_t)N * kmax * RC;                 // [64][RC]
    float2* Pp = W + 64 * RC;                              // [4][64][RC]
    uint64_t* bars = reinterpret_cast<uint64_t*>(Pp + 4 * 64 * RC);
    int* s_err = reinterpret_cast<int*>(bars + stages);

    const int col0 = blockIdx.x * RC;
    float2* V = slab_all + (size_t)blockIdx.x * ((size_t)N * N * Wmax * RC);
    const long long NN = (long long)N * N, N3 = NN * N;

    if (tid == 0) {
        for (int q = 0; q < stages; ++q) mbar_init(&bars[q], 1);
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        for (long long q = 0; q < stages && q < total_items; ++q) {
            uint32_t by;
            const float2* src = item_ptr(C, q, by);
            bulk_load(ring + (size_t)q * stage_elems, src, by, &bars[q]);
        }
        for (long long q = stages; q < stages + L2_AHEAD && q < total_items; ++q) {
            uint32_t by;
            const float2* src = item_ptr(C, q, by);
            l2_prefetch(src, by);
        }
    }

    long long s = 0;     // next stream item to consume
    const int n_outer = (C.mode == 1) ? 1 : 2 * B - 1;
    const int a_row = tid & 63, part = tid >> 6;
    const int pa = tid & 63, pc = tid >> 6;     // reduction-phase mapping (a, column)

    for (int jo = 0; jo < n_outer; ++jo) {
        int M = (C.mode == 1) ? C.M_only : ((jo < B) ? jo : 2 * B - 2 - jo);
        const bool outer_fwd = (C.mode == 1) || (jo < B);
        const AxisWin wz = C.t.win[M];
        const int za = (C.mode == 1) ? 0 : wz.ia, zb = (C.mode == 1) ? wz.L : wz.ib;
        // ---- embed the outer right-hand side into the slab window ----
        if (C.mode == 0) {
            const int zb0 = wz.lo + wz.ia, zb1 = wz.lo + wz.ib;
            const long long cnt = (long long)RC * (zb1 - zb0) * NN;
            for (long long e = tid; e < cnt; e += NT) {
                int x = (int)(e % N);
                long long rest = e / N;
                int y = (int)(rest % N);
                rest /= N;
                int z = zb0 + (int)(rest % (zb1 - zb0));
                int c = (int)(rest / (zb1 - zb0));
                int col = col0 + c;
                float2 v = make_float2(0.f, 0.f);
                if (col < nrhs) {
                    long long gi = (long long)col * N3 + (long long)z * NN + (long long)y * N + x;
                    if (outer_fwd) {
                        v = rin[gi];
                        if (M > 0 && z == zb0) v = csub(v, cmul(C.t.c_dn[z], zout[gi - NN]));
                    } else if (z == zb1 - 1) {
                        v = cmul(C.t.c_up[z], zout[gi + NN]);
                    }
                }
                V[(((size_t)x * N + y) * Wmax + (z - wz.lo)) * RC + c] = v;
            }
        } else {
            const long long cnt = (long long)RC * wz.L * NN;
            for (long long e = tid; e < cnt; e += NT) {
                int x = (int)(e % N);
                long long rest = e / N;
                int y = (int)(rest % N);
                rest /= N;
                int lz = (int)(rest % wz.L);
                int c = (int)(rest / wz.L);
                int col = col0 + c;
                float2 v = make_float2(0.f, 0.f);
                if (col < nrhs) v = rin[(long long)col * wz.L * NN + (long long)lz * NN + (long long)y * N + x];
                V[(((size_t)x * N + y) * Wmax + lz) * RC + c] = v;
            }
        }
        __syncthreads();

        for (int ji = 0; ji < 2 * B - 1; ++ji) {
            const int Mp = (ji < B) ? ji : 2 * B - 2 - ji;
            const bool inner_fwd = ji < B;
            const Prob P = C.t.prob[M * B + Mp];
            const int k = P.k, Lz = P.Lz, a0 = P.a0, ni = P.ni, ldk = P.ldk;
            // ---- gather the solve's input on its interest entries (all x) ----
            for (int e = tid; e < N * ni * RC; e += NT) {
                int c = e % RC;
                int rest = e / RC;
                int ai = rest % ni;
                int x = rest / ni;
                int a = a0 + ai;
                int lz = a % Lz, y = P.ylo + a / Lz;
                size_t vrow = ((size_t)x * N + y) * Wmax + lz;
                float2 v = make_float2(0.f, 0.f);
                if (inner_fwd) {
                    if (lz >= za && lz < zb) v = V[vrow * RC + c];
                    if (Mp > 0 && y == P.yb0)
                        v = csub(v, cmul(C.t.c_dn[y], V[(vrow - (size_t)Wmax) * RC + c]));
                } else if (y == P.yb1 - 1) {
                    v = cmul(C.t.c_up[y], V[(vrow + (size_t)Wmax) * RC + c]);
                }
                Y[((size_t)x * kmax + a) * RC + c] = v;
            }
            __syncthreads();
            // input of step 0: w = q_0
            if (pc < RC && pa < k) {
                float2 w = make_float2(0.f, 0.f);
                if (pa >= a0 && pa < a0 + ni) w = Y[(size_t)pa * RC + pc];
                W[pa * RC + pc] = w;
            }
            __syncthreads();

            for (int t = 0; t < 2 * N - 1; ++t) {
                const bool fwd = t < N;
                const int i = fwd ? t : 2 * N - 2 - t;
                const int stg = (int)(s % stages);
                // ---- wait for T_i, partial products ----
                if (!mbar_wait(&bars[stg], (uint32_t)((s / stages) & 1))) {
                    atomicOr(err, 2);
                    *s_err = 1;
                }
                const float2* T = ring + (size_t)stg * stage_elems;
                float2 acc[RC];
#pragma unroll
                for (int c = 0; c < RC; ++c) acc[c] = make_float2(0.f, 0.f);
                if (a_row < k) {
                    const int b0 = part * 16;
                    const int b1 = min(b0 + 16, k);
                    const float2* Trow = T + a_row * ldk;
                    for (int b = b0; b < b1; ++b) {
                        float2 tv = Trow[b];
#pragma unroll
                        for (int c = 0; c < RC; ++c) cfma(acc[c], tv, W[b * RC + c]);
                    }
                }
#pragma unroll
                for (int c = 0; c < RC; ++c) Pp[(part * 64 + a_row) * RC + c] = acc[c];
                __syncthreads();
                if (*s_err) goto done;
                // ---- the stage is free: refill it, prefetch further ahead ----
                if (tid == 0) {
                    long long nx = s + stages;
                    if (nx < total_items) {
                        uint32_t by;
                        const float2* src = item_ptr(C, nx, by);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        bulk_load(ring + (size_t)stg * stage_elems, src, by, &bars[stg]);
                    }
                    long long pf = s + stages + L2_AHEAD;
                    if (pf < total_items) {
                        uint32_t by;
                        const float2* src = item_ptr(C, pf, by);
                        l2_prefetch(src, by);
                    }
                }
                ++s;
                // ---- reduce quarters, finish the step, form the next input ----
                if (pc < RC && pa < k) {
                    const int c = pc, a = pa;
                    float2 sum = Pp[a * RC + c];
                    sum = cadd(sum, Pp[(64 + a) * RC + c]);
                    sum = cadd(sum, Pp[(128 + a) * RC + c]);
                    sum = cadd(sum, Pp[(192 + a) * RC + c]);
                    float2* Yi = Y + ((size_t)i * kmax + a) * RC + c;
                    if (fwd) {
                        *Yi = sum;                                  // y_i
                        if (i + 1 < N) {                            // w_{i+1} = q_{i+1} - cdn(i+1) y_i
                            float2 w = cmul(C.t.c_dn[i + 1], sum);
                            w = make_float2(-w.x, -w.y);
                            if (a >= a0 && a < a0 + ni)
                                w = cadd(w, Y[((size_t)(i + 1) * kmax + a) * RC + c]);
                            W[a * RC + c] = w;
                        } else {                                     // x_{N-1} = y_{N-1}
                            W[a * RC + c] = sum;
                            if (a >= a0 && a < a0 + ni) {
                                int lz = a % Lz, y = P.ylo + a / Lz;
                                float2* dst = V + (((size_t)i * N + y) * Wmax + lz) * RC + c;
                                if (inner_fwd) *dst = sum;
                                else *dst = csub(*dst, sum);
                            }
                        }
                    } else {                                         // x_i = y_i - cup(i) T_i x_{i+1}
                        float2 x = csub(*Yi, cmul(C.t.c_up[i], sum));
                        W[a * RC + c] = x;
                        if (a >= a0 && a < a0 + ni) {
                            int lz = a % Lz, y = P.ylo + a / Lz;
                            float2* dst = V + (((size_t)i * N + y) * Wmax + lz) * RC + c;
                            if (inner_fwd) *dst = x;
                            else *dst = csub(*dst, x);
                        }
                    }
                }
                __syncthreads();
            }
        }
        // ---- restrict the slab to the block's layers ----
        if (C.mode == 0) {
            const int zb0 = wz.lo + wz.ia, zb1 = wz.lo + wz.ib;
            const long long cnt = (long long)RC * (zb1 - zb0) * NN;
            for (long long e = tid; e < cnt; e += NT) {
                int x = (int)(e % N);
                long long rest = e / N;
                int y = (int)(rest % N);
                rest /= N;
                int z = zb0 + (int)(rest % (zb1 - zb0));
                int c = (int)(rest / (zb1 - zb0));
                int col = col0 + c;
                if (col >= nrhs) continue;
                float2 v = V[(((size_t)x * N + y) * Wmax + (z - wz.lo)) * RC + c];
                long long gi = (long long)col * N3 + (long long)z * NN + (long long)y * N + x;
                if (outer_fwd) zout[gi] = v;
                else zout[gi] = csub(zout[gi], v);
            }
        } else {
            const long long cnt = (long long)RC * wz.L * NN;
            for (long long e = tid; e < cnt; e += NT) {
                int x = (int)(e % N);
                long long rest = e / N;
                int y = (int)(rest % N);
                rest /= N;
                int lz = (int)(rest % wz.L);
                int c = (int)(rest / wz.L);
                int col = col0 + c;
                if (col >= nrhs) continue;
                zout[(long long)col * wz.L * NN + (long long)lz * NN + (long long)y * N + x] =
                    V[(((size_t)x * N + y) * Wmax + lz) * RC + c];
            }
        }
        __syncthreads();
    }
    return;
done:
    // error path: drain the copies still in flight (bounded), then leave
    if (tid == 0) {
        for (long long q = s; q < total_items && q < s + stages; ++q)
            (void)mbar_wait(&bars[q % stages], (uint32_t)((q / stages) & 1));
    }
    __syncthreads();
}

size_t sweep_smem_bytes(const helm_ctx* h, int rc, int stages) {
    const int N = h->g.N, kmax = h->kmax;
    size_t f2 = (size_t)stages * h->stage_elems + (size_t)N * kmax * rc + (size_t)64 * rc +
                (size_t)4 * 64 * rc;
    return f2 * sizeof(float2) + (size_t)stages * sizeof(uint64_t) + 16;
}

}  // namespace

int sweep_configure(helm_ctx* h) {
    const int limit = 227 * 1024;
    int want = h->opts.rhs_per_cta;
    int cands[3] = {2, 1, 4};
    int ncand = 3;
    if (want > 0) { cands[0] = want; ncand = 1; }
    for (int q = 0; q < ncand; ++q) {
        int rc = cands[q];
        if (rc != 1 && rc != 2 && rc != 4) continue;
        for (int stages = 8; stages >= 2; --stages) {
            size_t b = sweep_smem_bytes(h, rc, stages);
            if (b <= (size_t)limit) {
                h->sweep_rc = rc;
                h->sweep_stages = stages;
                h->sweep_smem = b;
                return HELM_OK;
            }
        }
    }
    return HELM_ENOTSUP;
}

template <int RC>
static cudaError_t launch_rc(helm_ctx* h, const Ctx& C, const float2* r, float2* z, int nrhs,
                             long long total, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)h->sweep_smem);
    if (e != cudaSuccess) return e;
    int grid = (nrhs + RC - 1) / RC;
    k_sweep<RC><<<grid, NT, h->sweep_smem, st>>>(C, r, z, h->slab, nrhs, h->sweep_stages,
                                                  h->stage_elems, h->kmax, total, h->dev_err);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t launch_sweep(helm_ctx* h, const float2* r, float2* z, int nrhs, int slab_only, int M_only,
                         cudaStream_t st) {
    const int rc = h->sweep_rc;
    const int grid = (nrhs + rc - 1) / rc;
    size_t need = (size_t)grid * h->g.N * h->g.N * h->g.Wmax * rc;
    if (need > h->slab_elems) {
        if (h->slab) cudaFree(h->slab);
        h->slab = nullptr;
        h->slab_elems = 0;
        cudaError_t e = cudaMalloc(&h->slab, need * sizeof(float2));
        if (e != cudaSuccess) return e;
        h->slab_elems = need;
    }
    Ctx C;
    C.g = h->g;
    C.t = h->t;
    C.factors = h->factors;
    C.nsol_in = 2 * h->g.B - 1;
    C.per_solve = 2 * h->g.N - 1;
    C.mode = slab_only ? 1 : 0;
    C.M_only = M_only;
    long long nsol = slab_only ? (long long)C.nsol_in : (long long)C.nsol_in * C.nsol_in;
    long long total = nsol * C.per_solve;
    if (rc == 1) return launch_rc<1>(h, C, r, z, nrhs, total, st);
    if (rc == 2) return launch_rc<2>(h, C, r, z, nrhs, total, st);
    return launch_rc<4>(h, C, r, z, nrhs, total, st);
}
