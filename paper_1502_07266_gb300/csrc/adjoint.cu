// Adjoint solve and velocity gradient.
//
// s_d depends on x_d only, so A = D A_sym with D = diag(s(x) s(y) s(z)) and
// A_sym complex symmetric; hence A^T = D^{-1} A D and the adjoint system
// A^T lambda = g is solved as lambda = D^{-1} A^{-1} (D g) with the forward
// factors.  The velocity gradient of L(c) with A(c) u = f and
// A^T lambda = (dL/du)^* is dL/dc = Re(sum_r lambda_r u_r) 2 omega^2 / c^3,
// from d(kappa)/dc = -2 omega^2 / c^3 (kappa = omega^2/c^2 on the diagonal).
#include "helm_internal.h"

namespace {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// y = D x (divide = 0) or y = D^{-1} x (divide = 1), D = s(x) s(y) s(z)
__global__ void k_scale_D(const float2* __restrict__ x, float2* __restrict__ y, const float2* __restrict__ s,
                          int N, long long n3, int nrhs, int divide) {
    const long long total = n3 * nrhs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long idx = e % n3;
        const int i = (int)(idx % N), j = (int)((idx / N) % N), k = (int)(idx / ((long long)N * N));
        float2 d = cmulf(cmulf(s[i], s[j]), s[k]);
        if (divide) {
            const float m = d.x * d.x + d.y * d.y;     // 1/d = conj(d)/|d|^2 (|d| in [1e-3, 1])
            d = make_float2(d.x / m, -d.y / m);
        }
        y[e] = cmulf(d, x[e]);
    }
}

// grad[idx] = sum_r Re(lam_r[idx] u_r[idx]) * 2 omega^2 / c^3, with
// omega^2 / c^3 = kappa^{3/2} / omega.
__global__ void k_velocity_gradient(const float2* __restrict__ lam, const float2* __restrict__ u,
                                    const double* __restrict__ kappa, double omega, long long n3, int nrhs,
                                    double* __restrict__ grad) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n3;
         idx += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int r = 0; r < nrhs; ++r) {
            const float2 a = lam[(long long)r * n3 + idx], b = u[(long long)r * n3 + idx];
            acc += (double)a.x * b.x - (double)a.y * b.y;
        }
        const double kap = kappa[idx];
        grad[idx] = acc * 2.0 * kap * sqrt(kap) / omega;
    }
}

}  // namespace

cudaError_t launch_scale_D(helm_ctx* h, const float2* x, float2* y, int nrhs, int divide, cudaStream_t st) {
    const long long n3 = (long long)h->g.N * h->g.N * h->g.N;
    k_scale_D<<<152 * 8, 256, 0, st>>>(x, y, h->t.s_node, h->g.N, n3, nrhs, divide);
    h->launches++;
    return cudaGetLastError();
}

cudaError_t launch_velocity_gradient(helm_ctx* h, const float2* lam, const float2* u, int nrhs, double* grad,
                                     cudaStream_t st) {
    const long long n3 = (long long)h->g.N * h->g.N * h->g.N;
    k_velocity_gradient<<<152 * 8, 256, 0, st>>>(lam, u, h->t.kappa64, h->g.omega, n3, nrhs, grad);
    h->launches++;
    return cudaGetLastError();
}
