// Batched block-LDU factorisation of every quasi-1D auxiliary problem
// (Algorithm 5 = Algorithm 3 for every slab; the P = B^2 problems are
// independent, Section 6 notes they can be set up in parallel).
//
// Problem (M, M') lives on x in [0, N), y in the window of line block M',
// z in the window of slab M, with the moving-PML profiles of those windows
// (Sections 3 and 4.1).  Ordered with (z, y) inside a block and x last, it
// is block tridiagonal along x with k x k diagonal blocks D_i and scalar
// couplings (s_1 depends on x only):  A_{i,i-1} = cdn(i) I,
// A_{i,i+1} = cup(i) I.  The Section 3 recursion is run from both ends and
// meets at the middle block m = (N-1)/2 (a twisted block factorisation: the
// same inverse, two independent elimination chains):
//     left   S_0 = D_0,  S_i = D_i - cdn(i) cup(i-1) T_{i-1},          i < m
//     right  S_{N-1} = D_{N-1},  S_i = D_i - cup(i) cdn(i+1) T_{i+1},  i > m
//     middle S_m = D_m - cdn(m) cup(m-1) T_{m-1} - cup(m) cdn(m+1) T_{m+1}
// with T_i = S_i^{-1}.  One CTA per problem; S_i is inverted in shared memory
// by Gauss-Jordan elimination with partial (row) pivoting, complex FP32.  T_i
// is stored row-major (row stride ldk, zero padded) at entry off + i*kstride
// in the handle's precision: complex FP32, or with the block scale 2^e (the
// largest scaled part in [2^14, 2^15)) as FP16 pairs or FP16 hi + lo pairs,
// the scale kept as an FP32 value in row 0, column ldk-1.  The chains always
// continue from the unrounded FP32 T_i.
#include "helm_internal.h"

#include <cuda_fp16.h>

namespace {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
// 1/z = conj(z) / |z|^2 (plain formula; |z| is far from the FP32 range limits here)
__device__ __forceinline__ float2 crecipf(float2 z) {
    float d = z.x * z.x + z.y * z.y;
    return make_float2(z.x / d, -z.y / d);
}

constexpr int NT = 256;

__global__ void __launch_bounds__(NT)
k_factor(Geom g, Tables t, float2* __restrict__ factors, int kmax, int fmt, int esz, int p0, long long off0) {
    extern __shared__ float2 sm[];
    const int p = p0 + blockIdx.x;
    const Prob P = t.prob[p];
    const int M = p / g.B, Mp = p % g.B;
    const AxisWin wz = t.win[M], wy = t.win[Mp];
    const int k = P.k, Lz = P.Lz, Ly = P.Ly;
    const int N = g.N;
    const int tid = threadIdx.x;

    float2* S = sm;                       // k x k, row-major
    float2* Tp = S + kmax * kmax;         // previous T of the running chain, row-major
    float2* TL = Tp + kmax * kmax;        // T_{m-1}, kept for the middle block
    float2* colf = TL + kmax * kmax;      // saved pivot column
    float2* zdn = colf + kmax;            // window couplings (per layer / line)
    float2* zup = zdn + kmax;
    float2* ydn = zup + kmax;
    float2* yup = ydn + kmax;
    int* perm = reinterpret_cast<int*>(yup + kmax);
    int* q = perm + kmax;
    int* s_piv = q + kmax;
    unsigned* s_max = reinterpret_cast<unsigned*>(s_piv + 1);   // block max |part| (float bits)

    const float inv_h2 = (float)(1.0 / (g.h * g.h));
    const int per = g.Wmax + 1;
    // couplings inside the windows: node s times the half-point s, over h^2
    for (int l = tid; l < Lz; l += NT) {
        float2 sn = t.w_node[M * g.Wmax + l];
        float2 a = cmulf(sn, t.w_half[M * per + l]), b = cmulf(sn, t.w_half[M * per + l + 1]);
        zdn[l] = make_float2(a.x * inv_h2, a.y * inv_h2);
        zup[l] = make_float2(b.x * inv_h2, b.y * inv_h2);
    }
    for (int l = tid; l < Ly; l += NT) {
        float2 sn = t.w_node[Mp * g.Wmax + l];
        float2 a = cmulf(sn, t.w_half[Mp * per + l]), b = cmulf(sn, t.w_half[Mp * per + l + 1]);
        ydn[l] = make_float2(a.x * inv_h2, a.y * inv_h2);
        yup[l] = make_float2(b.x * inv_h2, b.y * inv_h2);
    }
    __syncthreads();

    const long long NN = (long long)N * N;
    const int mid = (N - 1) / 2;
    for (int step = 0; step < N; ++step) {
        // chain order: left i = 0..m-1, right i = N-1..m+1, then the middle
        const int i = (step < mid) ? step : ((step < N - 1) ? N - 1 - (step - mid) : mid);
        const bool first_right = (step == mid);
        if (tid == 0) *s_max = 0u;
        // ---- D_i, minus the Schur term(s) ----
        const float2 xdiag = caddf(t.c_dn[i], t.c_up[i]);
        float2 beta = make_float2(0.f, 0.f), beta2 = make_float2(0.f, 0.f);
        bool use_tp = false, use_tl = false;
        if (i < mid && i > 0) { beta = cmulf(t.c_dn[i], t.c_up[i - 1]); use_tp = true; }
        if (i > mid && !first_right) { beta = cmulf(t.c_up[i], t.c_dn[i + 1]); use_tp = true; }
        if (i == mid) {
            if (mid + 1 <= N - 1) { beta = cmulf(t.c_up[i], t.c_dn[i + 1]); use_tp = true; }
            if (mid - 1 >= 0) { beta2 = cmulf(t.c_dn[i], t.c_up[i - 1]); use_tl = true; }
        }
        for (int e = tid; e < k * k; e += NT) {
            int a = e / k, b = e - a * k;
            int lz = a % Lz, ly = a / Lz;
            float2 v = make_float2(0.f, 0.f);
            if (a == b) {
                float kap = t.kappa[(long long)(wz.lo + lz) * NN + (long long)(wy.lo + ly) * N + i];
                v = make_float2(kap, 0.f);
                v = csubf(v, xdiag);
                v = csubf(v, caddf(ydn[ly], yup[ly]));
                v = csubf(v, caddf(zdn[lz], zup[lz]));
            } else if (b == a + 1 && lz + 1 < Lz) {
                v = zup[lz];
            } else if (b == a - 1 && lz > 0) {
                v = zdn[lz];
            } else if (b == a + Lz) {
                v = yup[ly];
            } else if (b == a - Lz) {
                v = ydn[ly];
            }
            if (use_tp) v = csubf(v, cmulf(beta, Tp[e]));
            if (use_tl) v = csubf(v, cmulf(beta2, TL[e]));
            S[e] = v;
        }
        __syncthreads();

        // ---- in-place Gauss-Jordan with row pivoting ----
        for (int j = 0; j < k; ++j) {
            if (tid < 32) {
                float best = -1.f;
                int bi = j;
                for (int r = j + tid; r < k; r += 32) {
                    float2 z = S[r * k + j];
                    float m = z.x * z.x + z.y * z.y;
                    if (m > best) { best = m; bi = r; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    float ob = __shfl_xor_sync(0xffffffffu, best, o);
                    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (tid == 0) { *s_piv = bi; perm[j] = bi; }
            }
            __syncthreads();
            const int pr = *s_piv;
            if (pr != j) {
                for (int c = tid; c < k; c += NT) {
                    float2 tmp = S[j * k + c];
                    S[j * k + c] = S[pr * k + c];
                    S[pr * k + c] = tmp;
                }
            }
            __syncthreads();
            const float2 inv = crecipf(S[j * k + j]);
            for (int r = tid; r < k; r += NT) colf[r] = S[r * k + j];
            __syncthreads();
            for (int c = tid; c < k; c += NT)
                S[j * k + c] = (c == j) ? inv : cmulf(S[j * k + c], inv);
            __syncthreads();
            for (int e = tid; e < k * k; e += NT) {
                int r = e / k, c = e - r * k;
                if (r == j) continue;
                float2 base = (c == j) ? make_float2(0.f, 0.f) : S[e];
                S[e] = csubf(base, cmulf(colf[r], S[j * k + c]));
            }
            __syncthreads();
        }
        // column unscrambling: result column c is column q[c] of S
        if (tid == 0) {
            for (int c = 0; c < k; ++c) q[c] = c;
            for (int j = k - 1; j >= 0; --j) {
                int pj = perm[j];
                int tmp = q[j]; q[j] = q[pj]; q[pj] = tmp;
            }
        }
        __syncthreads();
        // ---- the stored copy: block scale of the reduced formats ----
        float inv = 1.f, sc = 1.f;
        if (fmt != HELM_FP32) {
            float mx = 0.f;
            for (int e = tid; e < k * k; e += NT) {
                const float2 v = S[e];
                mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if ((tid & 31) == 0) atomicMax(s_max, __float_as_uint(mx));   // non-negative: bit order = value order
            __syncthreads();
            const float m = __uint_as_float(*s_max);
            if (m > 0.f) {
                int ex;
                frexpf(m, &ex);                   // m = f 2^ex, f in [0.5, 1)
                // both the scale and its inverse stay normal FP32 numbers
                const int e = min(max(15 - ex, -120), 120);
                sc = ldexpf(1.f, -e);
                inv = ldexpf(1.f, e);
            }
        }
        char* outb = reinterpret_cast<char*>(factors) + (size_t)(P.off - off0 + (long long)i * P.kstride) * esz;
        for (int e = tid; e < k * k; e += NT) {
            int a = e / k, b = e - a * k;
            float2 v = S[a * k + q[b]];
            if (i == mid - 1) TL[e] = v;      // the left chain's last factor
            Tp[e] = v;
            const size_t pos = (size_t)a * P.ldk + b;
            if (fmt == HELM_FP32) {
                reinterpret_cast<float2*>(outb)[pos] = v;
            } else if (fmt == HELM_FP16) {
                reinterpret_cast<__half2*>(outb)[pos] = __floats2half2_rn(v.x * inv, v.y * inv);
            } else {
                const float zx = v.x * inv, zy = v.y * inv;
                const __half2 hi = __floats2half2_rn(zx, zy);
                const float2 hf = __half22float2(hi);
                reinterpret_cast<__half2*>(outb)[2 * pos] = hi;
                reinterpret_cast<__half2*>(outb)[2 * pos + 1] = __floats2half2_rn(zx - hf.x, zy - hf.y);
            }
        }
        for (int e = tid; e < k * (P.ldk - k); e += NT) {      // zero row padding
            int a = e / (P.ldk - k), b = k + e % (P.ldk - k);
            if (fmt != HELM_FP32 && a == 0 && b == P.ldk - 1) {
                if (esz == 4) *reinterpret_cast<float*>(outb + (size_t)b * esz) = sc;
                else *reinterpret_cast<float2*>(outb + (size_t)b * esz) = make_float2(sc, 0.f);
            } else if (esz == 4) {
                *reinterpret_cast<unsigned*>(outb + ((size_t)a * P.ldk + b) * esz) = 0u;
            } else {
                *reinterpret_cast<float2*>(outb + ((size_t)a * P.ldk + b) * esz) = make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_factor_range(helm_ctx* h, int p0, int np, float2* dst, long long off0, int fmt,
                                cudaStream_t st) {
    const int kmax = h->kmax;
    size_t smem = (size_t)(3 * kmax * kmax + 5 * kmax) * sizeof(float2) + (2 * kmax + 4) * sizeof(int);
    cudaError_t e = ensure_dyn_smem((const void*)k_factor, smem);
    if (e != cudaSuccess) return e;
    if (np <= 0) return cudaSuccess;
    const int esz = (fmt == HELM_FP16) ? 4 : 8;
    k_factor<<<np, NT, smem, st>>>(h->g, h->t, dst, kmax, fmt, esz, p0, off0);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t launch_factor(helm_ctx* h, cudaStream_t st) {
    return launch_factor_range(h, 0, h->g.B * h->g.B, h->factors, 0, h->opts.precision, st);
}
