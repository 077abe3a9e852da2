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
// 2N-1 block steps each.  Right-hand sides are independent, so each CTA runs
// the entire chain for one right-hand side with a single compute warp: lane l
// owns rows l and l+32 of every T_i, holds both dot products in registers, and
// a step needs only warp-level synchronisation.  All CTAs walk the same
// factor stream, so the factors are read from HBM about once per use and
// shared through L2.  The stream is static: a producer warp issues TMA bulk
// copies (cp.async.bulk) of T_i into a ring of shared-memory stages,
// signalled by full/empty mbarriers, and prefetches further ahead into L2.
#include "helm_internal.h"

#include <mutex>

namespace {

constexpr int WAIT_LIMIT = 1 << 22;           // bounded mbarrier wait (a few seconds)
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

// d += a * b elementwise on float pairs (one packed FP32 FMA)
__device__ __forceinline__ void ffma2(float2& d, float2 a, float2 b) {
    unsigned long long dd = *reinterpret_cast<unsigned long long*>(&d);
    unsigned long long aa = *reinterpret_cast<const unsigned long long*>(&a);
    unsigned long long bb = *reinterpret_cast<const unsigned long long*>(&b);
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(dd) : "l"(aa), "l"(bb));
    d = *reinterpret_cast<float2*>(&dd);
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
// Bounded wait (about WAIT_LIMIT x 1 us at most): false if the phase never completed.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    for (int it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try_sleep(bar, parity, 1000u)) return true;
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
    int n_outer;       // slabs visited: 2B-1 (mode 0) or 1 (mode 1)
};

// Walks the static factor stream in the order the compute warps consume it:
// slabs jo (Algorithm 6: forward then backward), inner solves ji
// (Algorithm 4: forward then backward), steps t (x forward then backward).
struct StreamIter {
    int jo, ji, t;
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
    __device__ void start(const Ctx& C) {
        jo = ji = t = 0;
        done = false;
        load(C);
    }
    __device__ void next(const Ctx& C) {
        if (++t < C.per_solve) return;
        t = 0;
        if (++ji == C.nsol_in) {
            ji = 0;
            if (++jo == C.n_outer) { done = true; return; }
        }
        load(C);
    }
    __device__ const float2* ptr(const Ctx& C) const {
        const int N = C.g.N;
        int i = (t < N) ? t : 2 * N - 2 - t;
        return C.factors + base + (long long)i * kstride;
    }
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Producer warp (one lane): fill the ring in stream order; a stage is refilled
// once the compute warps have released it through its "empty" barrier.
__device__ void produce(const Ctx& C, float2* ring, int stages, int stage_elems, uint64_t* full,
                        uint64_t* empty, int* err) {
    StreamIter fill, pf;
    fill.start(C);
    pf.start(C);
    for (int q = 0; q < L2_AHEAD && !pf.done; ++q) pf.next(C);
    int stg = 0;
    uint32_t round = 0;
    while (!fill.done) {
        if (round > 0 && !mbar_wait(&empty[stg], (round - 1) & 1)) {
            atomicOr(err, 2);
            return;
        }
        bulk_load(ring + (size_t)stg * stage_elems, fill.ptr(C), (uint32_t)fill.kstride * 8u, &full[stg]);
        if (!pf.done) {
            l2_prefetch(pf.ptr(C), (uint32_t)pf.kstride * 8u);
            pf.next(C);
        }
        fill.next(C);
        if (++stg == stages) { stg = 0; ++round; }
    }
}

constexpr int NT = 256;                       // compute threads (8 warps)

__device__ __forceinline__ void named_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }

// Per step: thread (rp, q8) forms partial products of rows rp and rp+32 of T_i
// over the 8-column chunk q8 for RC right-hand sides (128-bit shared loads of
// column pairs; T rows have an even stride with ldk/2 odd so that the eight
// rows read by a quarter-warp hit distinct banks); the chunks are summed by the
// threads (a, c), which also form the next step's input.  Two barriers a step.
template <int RC>
__global__ void __launch_bounds__(NT + 32, 1)
k_sweep(Ctx C, const float2* __restrict__ rin, float2* __restrict__ zout, float2* __restrict__ slab_all,
        int nrhs, int stages, int stage_elems, int kmax, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int N = C.g.N, B = C.g.B, Wmax = C.g.Wmax;
    const int tid = threadIdx.x;
    // ---- shared memory carve-up (ring first: 16-byte aligned TMA targets) ----
    float2* ring = reinterpret_cast<float2*>(smem);
    // Y slot i holds the solve's input q_i on the interest entries until the
    // step before i has consumed it, then y_i (forward), then x_i (backward).
    float2* Y = ring + (size_t)stages * stage_elems;                 // [N][kmax][RC]
    float2* W = Y + (((size_t)N * kmax * RC + 1) & ~(size_t)1);      // [64][RC] step input
    float2* Pp = W + 64 * RC;                                        // [8][RC][64] partial sums
    float2* s_cdn = Pp + 8 * 64 * RC;                                // [N] coupling g -> g-1
    float2* s_cup = s_cdn + N;                                       // [N] coupling g -> g+1
    uint64_t* full = reinterpret_cast<uint64_t*>(s_cup + N);
    uint64_t* empty = full + stages;
    int* s_err = reinterpret_cast<int*>(empty + stages);

    for (int q = tid; q < N; q += blockDim.x) {
        s_cdn[q] = C.t.c_dn[q];
        s_cup[q] = C.t.c_up[q];
    }
    if (tid == 0) {
        for (int q = 0; q < stages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        *s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid >= NT) {                       // producer warp
        if (tid == NT) produce(C, ring, stages, stage_elems, full, empty, err);
        return;
    }

    const int col0 = blockIdx.x * RC;
    float2* V = slab_all + (size_t)blockIdx.x * ((size_t)N * N * Wmax * RC);
    const long long NN = (long long)N * N, N3 = NN * N;
    const int rp = tid & 31, q8 = tid >> 5;     // product phase: row pair, column chunk
    const int pa = tid & 63, pc = tid >> 6;     // reduction phase: row, column
    int stg = 0;
    uint32_t phase = 0;

    for (int jo = 0; jo < C.n_outer; ++jo) {
        const int M = (C.mode == 1) ? C.M_only : ((jo < B) ? jo : 2 * B - 2 - jo);
        const bool outer_fwd = (C.mode == 1) || (jo < B);
        const AxisWin wz = C.t.win[M];
        const int za = (C.mode == 1) ? 0 : wz.ia, zb = (C.mode == 1) ? wz.L : wz.ib;
        // ---- embed the outer right-hand side into the slab window ----
        if (C.mode == 0) {
            const int zb0 = wz.lo + wz.ia, zb1 = wz.lo + wz.ib;
            const long long cnt = (long long)RC * (zb1 - zb0) * NN;
            for (long long e = tid; e < cnt; e += NT) {
                const int x = (int)(e % N);
                long long rest = e / N;
                const int y = (int)(rest % N);
                rest /= N;
                const int z = zb0 + (int)(rest % (zb1 - zb0));
                const int c = (int)(rest / (zb1 - zb0));
                const int col = col0 + c;
                float2 v = make_float2(0.f, 0.f);
                if (col < nrhs) {
                    const long long gi = (long long)col * N3 + (long long)z * NN + (long long)y * N + x;
                    if (outer_fwd) {
                        v = rin[gi];
                        if (M > 0 && z == zb0) v = csub(v, cmul(s_cdn[z], zout[gi - NN]));
                    } else if (z == zb1 - 1) {
                        v = cmul(s_cup[z], zout[gi + NN]);
                    }
                }
                V[(((size_t)x * N + y) * Wmax + (z - wz.lo)) * RC + c] = v;
            }
        } else {
            const long long cnt = (long long)RC * wz.L * NN;
            for (long long e = tid; e < cnt; e += NT) {
                const int x = (int)(e % N);
                long long rest = e / N;
                const int y = (int)(rest % N);
                rest /= N;
                const int lz = (int)(rest % wz.L);
                const int c = (int)(rest / wz.L);
                const int col = col0 + c;
                float2 v = make_float2(0.f, 0.f);
                if (col < nrhs) v = rin[(long long)col * wz.L * NN + (long long)lz * NN + (long long)y * N + x];
                V[(((size_t)x * N + y) * Wmax + lz) * RC + c] = v;
            }
        }
        named_sync();

        for (int ji = 0; ji < C.nsol_in; ++ji) {
            const int Mp = (ji < B) ? ji : 2 * B - 2 - ji;
            const bool inner_fwd = ji < B;
            const Prob P = C.t.prob[M * B + Mp];
            const int k = P.k, Lz = P.Lz, a0 = P.a0, ni = P.ni, ldk = P.ldk;
            const int nchunk = (k + 7) >> 3;
            // ---- gather the solve's input on its interest entries (all x) ----
            for (int e = tid; e < N * ni * RC; e += NT) {
                const int c = e % RC;
                const int rest = e / RC;
                const int ai = rest % ni;
                const int x = rest / ni;
                const int a = a0 + ai;
                const int lz = a % Lz, y = P.ylo + a / Lz;
                const size_t vrow = ((size_t)x * N + y) * Wmax + lz;
                float2 v = make_float2(0.f, 0.f);
                if (inner_fwd) {
                    if (lz >= za && lz < zb) v = V[vrow * RC + c];
                    if (Mp > 0 && y == P.yb0) v = csub(v, cmul(s_cdn[y], V[(vrow - (size_t)Wmax) * RC + c]));
                } else if (y == P.yb1 - 1) {
                    v = cmul(s_cup[y], V[(vrow + (size_t)Wmax) * RC + c]);
                }
                Y[((size_t)x * kmax + a) * RC + c] = v;
            }
            named_sync();
            // input of step 0: w = q_0 (entries k..63 stay zero for the padded pairs)
            if (pc < RC) {
                float2 w = make_float2(0.f, 0.f);
                if (pa >= a0 && pa < a0 + ni) w = Y[(size_t)pa * RC + pc];
                W[pa * RC + pc] = w;
            }
            named_sync();

            for (int t = 0; t < 2 * N - 1; ++t) {
                const bool fwd = t < N;
                const int i = fwd ? t : 2 * N - 2 - t;
                // ---- wait for T_i, partial products ----
                if (!mbar_wait(&full[stg], phase)) {
                    atomicOr(err, 2);
                    *s_err = 1;
                }
                const float2* T = ring + (size_t)stg * stage_elems;
                {
                    // rows rp and rp+32, columns [8 q8, 8 q8 + 8) in pairs
                    float2 acc0[RC], acc1[RC];
#pragma unroll
                    for (int c = 0; c < RC; ++c) acc0[c] = acc1[c] = make_float2(0.f, 0.f);
                    const int b0 = q8 * 8;
                    if (b0 < k) {
                        const bool r0ok = rp < k, r1ok = rp + 32 < k;
                        const float4* T0 = reinterpret_cast<const float4*>(T + rp * ldk + b0);
                        const float4* T1 = reinterpret_cast<const float4*>(T + (rp + 32) * ldk + b0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (b0 + 2 * j < k) {
                                const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                                const float4 t0 = r0ok ? T0[j] : z4;
                                const float4 t1 = r1ok ? T1[j] : z4;
                                const int b = b0 + 2 * j;
#pragma unroll
                                for (int c = 0; c < RC; ++c) {
                                    const float2 w0 = W[b * RC + c], w1 = W[(b + 1) * RC + c];
                                    cfma(acc0[c], make_float2(t0.x, t0.y), w0);
                                    cfma(acc0[c], make_float2(t0.z, t0.w), w1);
                                    cfma(acc1[c], make_float2(t1.x, t1.y), w0);
                                    cfma(acc1[c], make_float2(t1.z, t1.w), w1);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < RC; ++c) {
                        Pp[(q8 * RC + c) * 64 + rp] = acc0[c];
                        Pp[(q8 * RC + c) * 64 + rp + 32] = acc1[c];
                    }
                }
                named_sync();
                if (*s_err) {
                    // error path: let the copies already in flight land (bounded), then leave
                    if (tid == 0) {
                        int q = stg;
                        uint32_t ph = phase;
                        for (int d = 0; d < stages; ++d) {
                            for (int it = 0; it < (1 << 12) && !mbar_try_sleep(&full[q], ph, 1000u); ++it) {
                            }
                            if (++q == stages) { q = 0; ph ^= 1u; }
                        }
                    }
                    return;
                }
                if (tid == 0) mbar_arrive(&empty[stg]);        // stage consumed
                if (++stg == stages) { stg = 0; phase ^= 1u; }
                // ---- reduce the chunks, finish the step, form the next input ----
                if (pc < RC && pa < k) {
                    const int c = pc, a = pa;
                    float2 pq[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        pq[q] = (q < nchunk) ? Pp[(q * RC + c) * 64 + a] : make_float2(0.f, 0.f);
                    const float2 sum = cadd(cadd(cadd(pq[0], pq[1]), cadd(pq[2], pq[3])),
                                            cadd(cadd(pq[4], pq[5]), cadd(pq[6], pq[7])));
                    float2* Yi = Y + ((size_t)i * kmax + a) * RC + c;
                    if (fwd) {
                        *Yi = sum;                                  // y_i
                        if (i + 1 < N) {                            // w_{i+1} = q_{i+1} - cdn(i+1) y_i
                            float2 w = cmul(s_cdn[i + 1], sum);
                            w = make_float2(-w.x, -w.y);
                            if (a >= a0 && a < a0 + ni)
                                w = cadd(w, Y[((size_t)(i + 1) * kmax + a) * RC + c]);
                            W[a * RC + c] = w;
                        } else {                                     // x_{N-1} = y_{N-1} (kept in slot N-1)
                            W[a * RC + c] = sum;
                        }
                    } else {                                         // x_i = y_i - cup(i) T_i x_{i+1}
                        const float2 x = csub(*Yi, cmul(s_cup[i], sum));
                        W[a * RC + c] = x;
                        *Yi = x;                                     // slot i now holds x_i
                    }
                }
                named_sync();
            }
            // ---- scatter the restricted solution (slot x holds x_x) into the slab ----
            for (int e = tid; e < N * ni * RC; e += NT) {
                const int c = e % RC;
                const int rest = e / RC;
                const int ai = rest % ni;
                const int x = rest / ni;
                const int a = a0 + ai;
                const int lz = a % Lz, y = P.ylo + a / Lz;
                const float2 v = Y[((size_t)x * kmax + a) * RC + c];
                float2* dst = V + (((size_t)x * N + y) * Wmax + lz) * RC + c;
                if (inner_fwd) *dst = v;
                else *dst = csub(*dst, v);
            }
            named_sync();
        }
        // ---- restrict the slab to the block's layers ----
        if (C.mode == 0) {
            const int zb0 = wz.lo + wz.ia, zb1 = wz.lo + wz.ib;
            const long long cnt = (long long)RC * (zb1 - zb0) * NN;
            for (long long e = tid; e < cnt; e += NT) {
                const int x = (int)(e % N);
                long long rest = e / N;
                const int y = (int)(rest % N);
                rest /= N;
                const int z = zb0 + (int)(rest % (zb1 - zb0));
                const int c = (int)(rest / (zb1 - zb0));
                const int col = col0 + c;
                if (col >= nrhs) continue;
                const float2 v = V[(((size_t)x * N + y) * Wmax + (z - wz.lo)) * RC + c];
                const long long gi = (long long)col * N3 + (long long)z * NN + (long long)y * N + x;
                if (outer_fwd) zout[gi] = v;
                else zout[gi] = csub(zout[gi], v);
            }
        } else {
            const long long cnt = (long long)RC * wz.L * NN;
            for (long long e = tid; e < cnt; e += NT) {
                const int x = (int)(e % N);
                long long rest = e / N;
                const int y = (int)(rest % N);
                rest /= N;
                const int lz = (int)(rest % wz.L);
                const int c = (int)(rest / wz.L);
                const int col = col0 + c;
                if (col >= nrhs) continue;
                zout[(long long)col * wz.L * NN + (long long)lz * NN + (long long)y * N + x] =
                    V[(((size_t)x * N + y) * Wmax + lz) * RC + c];
            }
        }
        named_sync();
    }
}

size_t sweep_smem_bytes(const helm_ctx* h, int rc, int stages) {
    const int N = h->g.N, kmax = h->kmax;
    size_t f2 = (size_t)stages * h->stage_elems + (((size_t)N * kmax * rc + 1) & ~(size_t)1) +
                (size_t)64 * rc + (size_t)8 * 64 * rc + (size_t)2 * N;
    return f2 * sizeof(float2) + (size_t)2 * stages * sizeof(uint64_t) + 16;
}

}  // namespace

int sweep_configure(helm_ctx* h) {
    const int limit = 227 * 1024;
    int want = h->opts.rhs_per_cta;
    int cands[3] = {1, 2, 4};
    int ncand = 3;
    if (want > 0) { cands[0] = want; ncand = 1; }
    for (int q = 0; q < ncand; ++q) {
        const int rc = cands[q];
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
                             cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)h->sweep_smem);
    if (e != cudaSuccess) return e;
    const int grid = (nrhs + RC - 1) / RC;
    k_sweep<RC><<<grid, NT + 32, h->sweep_smem, st>>>(C, r, z, h->slab, nrhs, h->sweep_stages,
                                                       h->stage_elems, h->kmax, h->dev_err);
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
    C.n_outer = slab_only ? 1 : 2 * h->g.B - 1;
    if (rc == 1) return launch_rc<1>(h, C, r, z, nrhs, st);
    if (rc == 2) return launch_rc<2>(h, C, r, z, nrhs, st);
    return launch_rc<4>(h, C, r, z, nrhs, st);
}

// ---------------------------------------------------------------------------
// Apply without allocation: the slab work space lives in one file-scope device
// array of HELM_NOALLOC_SCRATCH_BYTES.  Host code cannot use the array's name
// as a device address (it is a host-side stand-in), so its address is looked
// up once per device with cudaGetSymbolAddress while that device is current.

static __device__ __align__(256) float2 g_noalloc_scratch[HELM_NOALLOC_SCRATCH_BYTES / sizeof(float2)];

namespace {

std::mutex g_noalloc_mu;
float2* g_noalloc_addr[64] = {nullptr};

cudaError_t noalloc_scratch(float2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<float2*>(p);
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

template <int RC>
cudaError_t launch_rc_noalloc(helm_ctx* h, const Ctx& C, const float2* r, float2* z, int nrhs,
                              float2* scratch, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)h->sweep_smem);
    if (e != cudaSuccess) return e;
    const int grid = (nrhs + RC - 1) / RC;
    k_sweep<RC><<<grid, NT + 32, h->sweep_smem, st>>>(C, r, z, scratch, nrhs, h->sweep_stages,
                                                       h->stage_elems, h->kmax, h->dev_err);
    h->launches++;
    return cudaGetLastError();
}

}  // namespace

extern "C" int helm_apply_precond_noalloc(helm_handle h, const void* r, void* z, int nrhs, void* stream) {
    if (!h || !r || !z || nrhs < 1 || r == z) return HELM_EINVAL;
    const int rc = h->sweep_rc;
    const size_t grid = (size_t)(nrhs + rc - 1) / rc;
    const size_t need = grid * h->g.N * h->g.N * h->g.Wmax * rc;
    if (need > HELM_NOALLOC_SCRATCH_BYTES / sizeof(float2)) return HELM_EINVAL;
    float2* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) {
        helm_set_cuda_error(e);
        return HELM_ECUDA;
    }
    Ctx C;
    C.g = h->g;
    C.t = h->t;
    C.factors = h->factors;
    C.nsol_in = 2 * h->g.B - 1;
    C.per_solve = 2 * h->g.N - 1;
    C.mode = 0;
    C.M_only = 0;
    C.n_outer = 2 * h->g.B - 1;
    cudaStream_t st = (cudaStream_t)stream;
    if (rc == 1) e = launch_rc_noalloc<1>(h, C, (const float2*)r, (float2*)z, nrhs, scratch, st);
    else if (rc == 2) e = launch_rc_noalloc<2>(h, C, (const float2*)r, (float2*)z, nrhs, scratch, st);
    else e = launch_rc_noalloc<4>(h, C, (const float2*)r, (float2*)z, nrhs, scratch, st);
    if (e != cudaSuccess) {
        helm_set_cuda_error(e);
        return (e == cudaErrorMemoryAllocation) ? HELM_ENOMEM : HELM_ECUDA;
    }
    return HELM_OK;
}
