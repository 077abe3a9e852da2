// Coefficient tables (the PML stretching of Section 2 and kappa = omega^2/c^2).
//
// sigma(t) = (C/eta) ((t - eta)/eta)^2 for 0 <= t <= eta, else 0, with t the
// distance from a Dirichlet wall; s = (1 + i sigma/omega)^{-1}.  The global
// profile has a PML of width b h at both ends of every axis (walls at g = -1
// and g = N).  A moving window side (Section 3: s_3^m(x) = s(x_3 - (m-b)h)) has
// its own wall just outside the window (lo - 1 below, lo + L above) and width
// b_aux h; a side without one keeps the global profile of that face.
// Computed in FP64, stored as complex FP32.
#include "helm_internal.h"

namespace {

__device__ double pml_sigma(double t, double eta, double C) {
    if (t < 0.0 || t > eta) return 0.0;
    double q = (t - eta) / eta;
    return (C / eta) * q * q;
}

// Global sigma at padded position pos (integer or half-integer).
__device__ double sigma_global(double pos, const Geom g) {
    double eta = g.b * g.h;
    return pml_sigma((pos + 1.0) * g.h, eta, g.C) + pml_sigma((g.N - pos) * g.h, eta, g.C);
}

// Each side of a window: a moving PML of width b_aux whose wall is the node
// just outside the window, or the global profile of that side.
__device__ double sigma_window(double pos, const AxisWin w, const Geom g) {
    const double eta = g.b * g.h, eta_aux = g.b_aux * g.h;
    const double s_lo = w.moving ? pml_sigma((pos - (w.lo - 1.0)) * g.h, eta_aux, g.C)
                                 : pml_sigma((pos + 1.0) * g.h, eta, g.C);
    const double s_hi = w.moving_hi ? pml_sigma(((double)(w.lo + w.L) - pos) * g.h, eta_aux, g.C)
                                    : pml_sigma((g.N - pos) * g.h, eta, g.C);
    return s_lo + s_hi;
}

// s = 1 / (1 + i a), a = sigma/omega  ->  (1 - i a) / (1 + a^2)
__device__ double2 stretch(double sigma, double omega) {
    double a = sigma / omega;
    double den = 1.0 + a * a;
    return make_double2(1.0 / den, -a / den);
}

__device__ double2 cmul(double2 x, double2 y) {
    return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}

__global__ void k_axis_tables(Geom g, Tables t) {
    const int N = g.N;
    const double inv_h2 = 1.0 / (g.h * g.h);
    int tid = blockIdx.x * blockDim.x + threadIdx.x;
    // global profile, node and half tables, A's layer couplings
    if (tid <= N) {
        double2 sh = stretch(sigma_global(tid - 0.5, g), g.omega);
        t.s_half[tid] = make_float2((float)sh.x, (float)sh.y);
    }
    if (tid < N) {
        double2 sn = stretch(sigma_global((double)tid, g), g.omega);
        double2 sm = stretch(sigma_global(tid - 0.5, g), g.omega);
        double2 sp = stretch(sigma_global(tid + 0.5, g), g.omega);
        t.s_node[tid] = make_float2((float)sn.x, (float)sn.y);
        double2 dn = cmul(sn, sm), up = cmul(sn, sp);
        t.c_dn[tid] = make_float2((float)(dn.x * inv_h2), (float)(dn.y * inv_h2));
        t.c_up[tid] = make_float2((float)(up.x * inv_h2), (float)(up.y * inv_h2));
        t.c_dn64[tid] = make_double2(dn.x * inv_h2, dn.y * inv_h2);
        t.c_up64[tid] = make_double2(up.x * inv_h2, up.y * inv_h2);
    }
    // window profiles: B windows, Wmax+1 entries each
    int per = g.Wmax + 1;
    if (tid < g.B * per) {
        int M = tid / per, l = tid % per;
        AxisWin w = t.win[M];
        if (l <= w.L) {
            double2 sh = stretch(sigma_window(w.lo + l - 0.5, w, g), g.omega);
            t.w_half[M * per + l] = make_float2((float)sh.x, (float)sh.y);
        }
        if (l < w.L) {
            double2 sn = stretch(sigma_window((double)(w.lo + l), w, g), g.omega);
            t.w_node[M * g.Wmax + l] = make_float2((float)sn.x, (float)sn.y);
        }
    }
}

__global__ void k_kappa(const float* __restrict__ c, float* __restrict__ kappa,
                        double* __restrict__ kappa64, long long n3, double omega, int* err) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; i < n3; i += (long long)gridDim.x * blockDim.x) {
        float ci = c[i];
        if (!(ci > 0.0f) || !isfinite(ci)) atomicOr(err, 1);
        double cd = (double)ci;
        double kd = omega * omega / (cd * cd);
        kappa64[i] = kd;
        kappa[i] = (float)kd;
    }
}

}  // namespace

cudaError_t launch_coefficients(helm_ctx* h, const float* c, cudaStream_t st) {
    const Geom& g = h->g;
    int total = g.B * (g.Wmax + 1);
    if (total < g.N + 1) total = g.N + 1;
    k_axis_tables<<<(total + 255) / 256, 256, 0, st>>>(g, h->t);
    h->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long n3 = (long long)g.N * g.N * g.N;
    int blocks = (int)((n3 + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_kappa<<<blocks, 256, 0, st>>>(c, h->t.kappa, h->t.kappa64, n3, g.omega, h->dev_err);
    h->launches++;
    return cudaGetLastError();
}
