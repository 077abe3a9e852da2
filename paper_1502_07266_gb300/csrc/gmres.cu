// Vector kernels of right-preconditioned restarted GMRES (the Section 5
// solver), every right-hand side an independent Krylov space.  Basis vectors
// are complex FP32; norms, the Hessenberg matrix, the Givens rotations and the
// solution accumulate in FP64.  The Gram-Schmidt inner products run per thread
// in compensated FP32 arithmetic (the Dot2 scheme of Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005: error-free products and sums, result
// as accurate as a dot product computed in twice the working precision) and are
// summed across threads in FP64: the FP64 pipe of this GPU is 1/64 of its FP32
// pipe, and FP64 products made that kernel ALU bound at about 10x its memory
// time.
#include "helm_internal.h"
#include "gmres_kernels.h"

namespace {

constexpr int NT = 256;

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV complex values; result valid in thread 0.
template <int NV>
__device__ void block_sum(double2 (&acc)[NV], double2* sbuf /* [NT/32][NV] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double re = warp_sum(acc[v].x), im = warp_sum(acc[v].y);
        if (lane == 0) sbuf[warp * NV + v] = make_double2(re, im);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double2 s = make_double2(0.0, 0.0);
            for (int w = 0; w < NT / 32; ++w) s = dadd(s, sbuf[w * NV + v]);
            acc[v] = s;
        }
    }
}

// One Dot2 step: the value s + c gains x * y.  The product's rounding error
// (exact through the FMA) and the sum's (Knuth's TwoSum) both go to c.  The
// _rn intrinsics keep the compiler from contracting the product into an FMA,
// which would break the error-free transformations.
__device__ __forceinline__ void dot2_step(float& s, float& c, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float ep = fmaf(x, y, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(ep, es));
}

// partial[(r*G + blk)*NV + v] = sum over the block's slice of conj(V_{j0+v}[r]) w[r]
template <int NV>
__global__ void __launch_bounds__(NT)
k_dots(const float2* __restrict__ V, long long vstride, int j0, int nv, const float2* __restrict__ w,
       long long n, int R, double2* __restrict__ partial) {
    __shared__ double2 sbuf[(NT / 32) * NV];
    const int r = blockIdx.y, G = gridDim.x;
    float sre[NV], cre[NV], sim[NV], cim[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) sre[v] = cre[v] = sim[v] = cim[v] = 0.f;
    const float2* wr = w + (long long)r * n;
    const float2* Vr = V + (long long)j0 * vstride + (long long)r * n;
    for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < n; e += (long long)G * NT) {
        const float2 b = wr[e];
        float2 a[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v)
            a[v] = v < nv ? __ldcs(Vr + (long long)v * vstride + e) : make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (v < nv) {
                // conj(a) * b = (a.x b.x + a.y b.y) + i (a.x b.y - a.y b.x)
                dot2_step(sre[v], cre[v], a[v].x, b.x);
                dot2_step(sre[v], cre[v], a[v].y, b.y);
                dot2_step(sim[v], cim[v], a[v].x, b.y);
                dot2_step(sim[v], cim[v], -a[v].y, b.x);
            }
        }
    }
    double2 acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v)
        acc[v] = make_double2((double)sre[v] + (double)cre[v], (double)sim[v] + (double)cim[v]);
    block_sum<NV>(acc, sbuf);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) partial[((long long)r * G + blockIdx.x) * NV + v] = acc[v];
    }
}

// out[r*ostride + j0 + v] (+)= sum over blocks of partial
__global__ void k_reduce(const double2* __restrict__ partial, int G, int NV, int nv, int R,
                         double2* __restrict__ out, int ostride, int j0, int accumulate) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * nv) return;
    int r = t / nv, v = t % nv;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < G; ++b) s = dadd(s, partial[((long long)r * G + b) * NV + v]);
    double2* o = out + (long long)r * ostride + j0 + v;
    if (accumulate) *o = dadd(*o, s);
    else *o = s;
}

// w[r] -= sum_{j < J} V_j[r] h[r][j]
__global__ void __launch_bounds__(NT)
k_axpy_basis(const float2* __restrict__ V, long long vstride, int J, const double2* __restrict__ h,
             int hstride, float2* __restrict__ w, long long n) {
    __shared__ float2 hs[64];
    const int r = blockIdx.y;
    if (threadIdx.x < J) {
        double2 c = h[(long long)r * hstride + threadIdx.x];
        hs[threadIdx.x] = make_float2((float)c.x, (float)c.y);
    }
    __syncthreads();
    float2* wr = w + (long long)r * n;
    for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < n; e += (long long)gridDim.x * NT) {
        float2 acc = wr[e];
        for (int j = 0; j < J; ++j) {
            float2 a = V[(long long)j * vstride + (long long)r * n + e];
            float2 c = hs[j];
            acc.x -= a.x * c.x - a.y * c.y;
            acc.y -= a.x * c.y + a.y * c.x;
        }
        wr[e] = acc;
    }
}

// squared norms of c64 (mode 0) or c128 (mode 1) vectors: partial sums
template <class T2>
__global__ void __launch_bounds__(NT)
k_norm2(const T2* __restrict__ x, long long n, double2* __restrict__ partial) {
    __shared__ double2 sbuf[NT / 32];
    const int r = blockIdx.y, G = gridDim.x;
    double2 acc[1] = {make_double2(0.0, 0.0)};
    const T2* xr = x + (long long)r * n;
    for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < n; e += (long long)G * NT) {
        T2 a = xr[e];
        acc[0].x += (double)a.x * a.x + (double)a.y * a.y;
    }
    block_sum<1>(acc, sbuf);
    if (threadIdx.x == 0) partial[(long long)r * G + blockIdx.x] = acc[0];
}

// dst[r] = src[r] * scale[r] (c128 or c64 source, c64 destination); zero when scale is 0
template <class T2>
__global__ void __launch_bounds__(NT)
k_scale_to_c64(const T2* __restrict__ src, const double* __restrict__ scale, float2* __restrict__ dst,
               long long n) {
    const int r = blockIdx.y;
    const double s = scale[r];
    for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < n; e += (long long)gridDim.x * NT) {
        T2 a = src[(long long)r * n + e];
        dst[(long long)r * n + e] = make_float2((float)(a.x * s), (float)(a.y * s));
    }
}

// u[r] += sum_{j < mlen[r]} Z_j[r] y[r][j]   (c128 accumulation)
__global__ void __launch_bounds__(NT)
k_update(const float2* __restrict__ Z, long long zstride, const double2* __restrict__ y, int ystride,
         const int* __restrict__ mlen, double2* __restrict__ u, long long n) {
    const int r = blockIdx.y;
    const int J = mlen[r];
    if (J <= 0) return;
    for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < n; e += (long long)gridDim.x * NT) {
        double2 acc = u[(long long)r * n + e];
        for (int j = 0; j < J; ++j) {
            float2 a = Z[(long long)j * zstride + (long long)r * n + e];
            double2 c = y[(long long)r * ystride + j];
            acc.x += (double)a.x * c.x - (double)a.y * c.y;
            acc.y += (double)a.x * c.y + (double)a.y * c.x;
        }
        u[(long long)r * n + e] = acc;
    }
}

__global__ void k_c128_to_c64(const double2* __restrict__ src, float2* __restrict__ dst, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = make_float2((float)src[e].x, (float)src[e].y);
}

// The convergence test of iteration j on the device: a right-hand side that is
// not frozen counts the iteration and freezes (its cycle length is j + 1) when
// the Arnoldi residual estimate reaches tol ||f|| or it used maxit iterations;
// *nact counts those still active (zeroed before the launch).
__global__ void k_converge(const double* __restrict__ est, const double* __restrict__ fn2, double tol, int maxit,
                           int* __restrict__ frozen, int* __restrict__ its, int* __restrict__ mlen, int j, int R,
                           int* __restrict__ nact) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || frozen[r]) return;
    const int k = ++its[r];
    if (est[r] <= tol * sqrt(fn2[r]) || k >= maxit) {
        frozen[r] = 1;
        mlen[r] = j + 1;
    } else {
        atomicAdd(nact, 1);
    }
}

// Cycle end: a right-hand side active in the cycle and never frozen ran jend iterations.
__global__ void k_cycle_len(const int* __restrict__ active, int* __restrict__ mlen, int jend, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R && active[r] && mlen[r] == 0) mlen[r] = jend;
}

// ---- per-RHS small FP64 work: one thread per right-hand side ----

__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cabsd(double2 a) { return hypot(a.x, a.y); }

// Column j of the Hessenberg matrix H[r] ((m+1) x m, column-major, ld m+1):
// rotate by the previous Givens rotations, make a new one that zeroes
// H[j+1][j], apply it to g.  est[r] = |g[j+1]| (the Arnoldi residual).
__global__ void k_givens(double2* __restrict__ H, double2* __restrict__ cs, double2* __restrict__ sn,
                         double2* __restrict__ gv, double* __restrict__ est, const int* __restrict__ frozen,
                         int R, int m, int j) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || frozen[r]) return;
    double2* Hc = H + ((long long)r * m + j) * (m + 1);
    double2* c = cs + (long long)r * m;
    double2* s = sn + (long long)r * m;
    double2* g = gv + (long long)r * (m + 1);
    for (int i = 0; i < j; ++i) {
        double2 hi = Hc[i], hi1 = Hc[i + 1];
        // [ c  s ; -conj(s) conj(c) ] applied to (hi, hi1)
        double2 t0 = dadd(cmuld(c[i], hi), cmuld(s[i], hi1));
        double2 t1 = dadd(cmuld(make_double2(-s[i].x, s[i].y), hi), cmuld(conjd(c[i]), hi1));
        Hc[i] = t0;
        Hc[i + 1] = t1;
    }
    double2 a = Hc[j], b = Hc[j + 1];
    double den = hypot(cabsd(a), cabsd(b));
    double2 cj, sj;
    if (den == 0.0) {
        cj = make_double2(1.0, 0.0);
        sj = make_double2(0.0, 0.0);
    } else {
        cj = make_double2(a.x / den, -a.y / den);   // conj(a)/den
        sj = make_double2(b.x / den, -b.y / den);   // conj(b)/den
    }
    c[j] = cj;
    s[j] = sj;
    Hc[j] = make_double2(den, 0.0);
    Hc[j + 1] = make_double2(0.0, 0.0);
    double2 gj = g[j];
    g[j + 1] = cmuld(make_double2(-sj.x, sj.y), gj);   // -conj(s) g_j
    g[j] = cmuld(cj, gj);
    est[r] = cabsd(g[j + 1]);
}

// y = R^{-1} g on the leading mlen x mlen triangle (back substitution)
__global__ void k_backsolve(const double2* __restrict__ H, const double2* __restrict__ gv,
                            double2* __restrict__ y, const int* __restrict__ mlen, int R, int m) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int J = mlen[r];
    const double2* Hr = H + (long long)r * m * (m + 1);
    const double2* g = gv + (long long)r * (m + 1);
    double2* yr = y + (long long)r * m;
    for (int i = J - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int q = i + 1; q < J; ++q) {
            double2 t = cmuld(Hr[(long long)q * (m + 1) + i], yr[q]);
            acc.x -= t.x;
            acc.y -= t.y;
        }
        double2 d = Hr[(long long)i * (m + 1) + i];
        double dd = d.x * d.x + d.y * d.y;
        yr[i] = (dd == 0.0) ? make_double2(0.0, 0.0)
                            : make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
    }
}

// Start of a cycle: beta from the residual norm^2, g = beta e1, 1/beta for V_0.
__global__ void k_cycle_start(const double* __restrict__ rn2, double2* __restrict__ gv,
                              double* __restrict__ inv, const int* __restrict__ active, int R, int m) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double beta = sqrt(rn2[r]);
    double2* g = gv + (long long)r * (m + 1);
    for (int i = 0; i <= m; ++i) g[i] = make_double2(0.0, 0.0);
    g[0] = make_double2(active[r] ? beta : 0.0, 0.0);
    inv[r] = (active[r] && beta > 0.0) ? 1.0 / beta : 0.0;
}

// After the norm of w: H[j+1][j] = ||w||, inverse scale for V_{j+1} (0 when frozen/zero).
__global__ void k_subdiag(const double* __restrict__ wn2, double2* __restrict__ H, double* __restrict__ inv,
                          const int* __restrict__ frozen, int R, int m, int j) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double nrm = sqrt(wn2[r]);
    H[((long long)r * m + j) * (m + 1) + j + 1] = make_double2(nrm, 0.0);
    inv[r] = (!frozen[r] && nrm > 0.0) ? 1.0 / nrm : 0.0;
}

// dst[r][i] += src[r][i], i < J
__global__ void k_addcol(const double2* __restrict__ src, int sstride, double2* __restrict__ dst,
                         int dstride, int J, int R) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= R * J) return;
    int r = t / J, i = t % J;
    dst[(long long)r * dstride + i] = dadd(dst[(long long)r * dstride + i], src[(long long)r * sstride + i]);
}

// partial norm sums (one complex slot, real part used) -> real array
__global__ void k_reduce_real(const double2* __restrict__ partial, int G, int R, double* __restrict__ out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += partial[(long long)r * G + b].x;
    out[r] = s;
}

}  // namespace

// ---------------------------------------------------------------- launchers

static int vec_grid(long long n) {
    long long g = (n + NT - 1) / NT;
    if (g > 304) g = 304;
    return (int)g;
}

cudaError_t gm_dots(helm_ctx* h, const float2* V, long long vstride, int j0, int nv, const float2* w,
                    long long n, int R, double2* partial, double2* out, int ostride, int accumulate,
                    cudaStream_t st) {
    const int G = vec_grid(n) > 64 ? 64 : vec_grid(n);
    for (int b = 0; b < nv; b += 8) {
        int cnt = nv - b < 8 ? nv - b : 8;
        dim3 grid(G, R);
        k_dots<8><<<grid, NT, 0, st>>>(V, vstride, j0 + b, cnt, w, n, R, partial);
        h->launches++;
        k_reduce<<<(R * cnt + 127) / 128, 128, 0, st>>>(partial, G, 8, cnt, R, out, ostride, j0 + b,
                                                         accumulate);
        h->launches++;
    }
    return cudaGetLastError();
}

cudaError_t gm_axpy(helm_ctx* h, const float2* V, long long vstride, int J, const double2* hcoef,
                    int hstride, float2* w, long long n, int R, cudaStream_t st) {
    dim3 grid(vec_grid(n), R);
    k_axpy_basis<<<grid, NT, 0, st>>>(V, vstride, J, hcoef, hstride, w, n);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_norm2_c64(helm_ctx* h, const float2* x, long long n, int R, double2* partial, double* out,
                         cudaStream_t st) {
    const int G = 64;
    k_norm2<float2><<<dim3(G, R), NT, 0, st>>>(x, n, partial);
    k_reduce_real<<<(R + 127) / 128, 128, 0, st>>>(partial, G, R, out);
    h->launches += 2;
    return cudaGetLastError();
}

cudaError_t gm_norm2_c128(helm_ctx* h, const double2* x, long long n, int R, double2* partial,
                          double* out, cudaStream_t st) {
    const int G = 64;
    k_norm2<double2><<<dim3(G, R), NT, 0, st>>>(x, n, partial);
    k_reduce_real<<<(R + 127) / 128, 128, 0, st>>>(partial, G, R, out);
    h->launches += 2;
    return cudaGetLastError();
}

cudaError_t gm_scale_c128(helm_ctx* h, const double2* src, const double* scale, float2* dst, long long n,
                          int R, cudaStream_t st) {
    k_scale_to_c64<double2><<<dim3(vec_grid(n), R), NT, 0, st>>>(src, scale, dst, n);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_scale_c64(helm_ctx* h, const float2* src, const double* scale, float2* dst, long long n,
                         int R, cudaStream_t st) {
    k_scale_to_c64<float2><<<dim3(vec_grid(n), R), NT, 0, st>>>(src, scale, dst, n);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_update(helm_ctx* h, const float2* Z, long long zstride, const double2* y, int ystride,
                      const int* mlen, double2* u, long long n, int R, cudaStream_t st) {
    k_update<<<dim3(vec_grid(n), R), NT, 0, st>>>(Z, zstride, y, ystride, mlen, u, n);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_to_c64(helm_ctx* h, const double2* src, float2* dst, long long n, cudaStream_t st) {
    k_c128_to_c64<<<1216, NT, 0, st>>>(src, dst, n);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_givens(helm_ctx* h, double2* H, double2* cs, double2* sn, double2* g, double* est,
                      const int* frozen, int R, int m, int j, cudaStream_t st) {
    k_givens<<<(R + 63) / 64, 64, 0, st>>>(H, cs, sn, g, est, frozen, R, m, j);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_backsolve(helm_ctx* h, const double2* H, const double2* g, double2* y, const int* mlen,
                         int R, int m, cudaStream_t st) {
    k_backsolve<<<(R + 63) / 64, 64, 0, st>>>(H, g, y, mlen, R, m);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_cycle_start(helm_ctx* h, const double* rn2, double2* g, double* inv, const int* active,
                           int R, int m, cudaStream_t st) {
    k_cycle_start<<<(R + 63) / 64, 64, 0, st>>>(rn2, g, inv, active, R, m);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_subdiag(helm_ctx* h, const double* wn2, double2* H, double* inv, const int* frozen, int R,
                       int m, int j, cudaStream_t st) {
    k_subdiag<<<(R + 63) / 64, 64, 0, st>>>(wn2, H, inv, frozen, R, m, j);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_converge(helm_ctx* h, const double* est, const double* fn2, double tol, int maxit, int* frozen,
                        int* its, int* mlen, int j, int R, int* nact, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(nact, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_converge<<<(R + 127) / 128, 128, 0, st>>>(est, fn2, tol, maxit, frozen, its, mlen, j, R, nact);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_cycle_len(helm_ctx* h, const int* active, int* mlen, int jend, int R, cudaStream_t st) {
    k_cycle_len<<<(R + 127) / 128, 128, 0, st>>>(active, mlen, jend, R);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t gm_addcol(helm_ctx* h, const double2* src, int sstride, double2* dst, int dstride, int J, int R,
                      cudaStream_t st) {
    k_addcol<<<(R * J + 127) / 128, 128, 0, st>>>(src, sstride, dst, dstride, J, R);
    h->launches++;
    return cudaGetLastError();
}
