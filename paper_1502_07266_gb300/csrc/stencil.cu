// The 7-point nonsymmetric PML stencil of Eq. (system), batched over RHS.
//
//   (A u)_g = kappa_g u_g + sum_axes [ cup(g) (u_{g+1} - u_g) - cdn(g) (u_g - u_{g-1}) ]
//   cup(g) = s(g) s(g+1/2) / h^2,  cdn(g) = s(g) s(g-1/2) / h^2
// with u = 0 beyond the walls at g = -1 and g = N.  The same global profile
// serves all three axes (cubic grid, PML on every face).  HBM-bound: each
// thread owns one z column and marches along it, keeping the z neighbours in
// registers; x and y neighbours come through L1.
#include "helm_internal.h"

namespace {

template <class T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

template <class T>
__device__ __forceinline__ typename C2<T>::t cmk(T a, T b) { return {a, b}; }

template <class V>
__device__ __forceinline__ V cadd(V a, V b) { return {a.x + b.x, a.y + b.y}; }
template <class V>
__device__ __forceinline__ V csub(V a, V b) { return {a.x - b.x, a.y - b.y}; }
template <class V>
__device__ __forceinline__ V cmul(V a, V b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

// Loads a c64 or c128 value as the compute type.
__device__ __forceinline__ float2 ld(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ld(const double2* p) { return __ldg(p); }

// T: compute type; VI: stored vector type; MODE 0: y = A x, MODE 1: y = f - A x.
// A thread owns one column c = j N + i of the flattened (x, y) plane (so a
// warp's 32 columns are contiguous and no lane idles at the end of an x row)
// and marches along z with a pointer that moves one plane per step.  Software
// pipelined: while plane k is computed, plane k+1's x and y neighbours and
// kappa and the value two planes ahead are in flight.  A missing neighbour
// (a wall) is read at offset 0 and multiplied by 0.
template <class T, class VI, int MODE>
__global__ void __launch_bounds__(256)
k_stencil(const VI* __restrict__ x, VI* __restrict__ y, const float2* __restrict__ f,
          const T* __restrict__ kappa, const typename C2<T>::t* __restrict__ cdn,
          const typename C2<T>::t* __restrict__ cup, int N) {
    using V = typename C2<T>::t;
    extern __shared__ unsigned char smem_raw[];
    V* s_dn = reinterpret_cast<V*>(smem_raw);
    V* s_up = s_dn + N;
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
        s_dn[q] = cdn[q];
        s_up[q] = cup[q];
    }
    __syncthreads();
    const int NN = N * N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (c >= NN) return;
    const int j = c / N, i = c - j * N;
    const long long base = (long long)r * NN * N + c;
    const VI* px = x + base;
    VI* py = y + base;
    const float2* pf = (MODE == 1) ? f + base : nullptr;
    const T* pk = kappa + c;
    const V zero = cmk<T>(0, 0);
    const V dni = s_dn[i], upi = s_up[i], dnj = s_dn[j], upj = s_up[j];
    const int oxm = i > 0 ? -1 : 0, oxp = i + 1 < N ? 1 : 0;
    const int oym = j > 0 ? -N : 0, oyp = j + 1 < N ? N : 0;
    const T mxm = i > 0 ? T(1) : T(0), mxp = i + 1 < N ? T(1) : T(0);
    const T mym = j > 0 ? T(1) : T(0), myp = j + 1 < N ? T(1) : T(0);
    V u_prev = zero;
    V u_cur = ld(px);
    V u_next = (N > 1) ? ld(px + NN) : zero;
    V xm = ld(px + oxm), xp = ld(px + oxp), ym = ld(px + oym), yp = ld(px + oyp);
    T kap = pk[0];
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
        const V u_nn = (k + 2 < N) ? ld(px + 2 * NN) : zero;
        V nxm = zero, nxp = zero, nym = zero, nyp = zero;
        T nkap = 0;
        if (k + 1 < N) {
            const VI* q = px + NN;
            nxm = ld(q + oxm);
            nxp = ld(q + oxp);
            nym = ld(q + oym);
            nyp = ld(q + oyp);
            nkap = pk[NN];
        }
        xm = cmk<T>(xm.x * mxm, xm.y * mxm);
        xp = cmk<T>(xp.x * mxp, xp.y * mxp);
        ym = cmk<T>(ym.x * mym, ym.y * mym);
        yp = cmk<T>(yp.x * myp, yp.y * myp);
        V acc = cmk<T>(kap * u_cur.x, kap * u_cur.y);
        acc = cadd(acc, csub(cmul(upi, csub(xp, u_cur)), cmul(dni, csub(u_cur, xm))));
        acc = cadd(acc, csub(cmul(upj, csub(yp, u_cur)), cmul(dnj, csub(u_cur, ym))));
        acc = cadd(acc, csub(cmul(s_up[k], csub(u_next, u_cur)), cmul(s_dn[k], csub(u_cur, u_prev))));
        if (MODE == 1) {
            const float2 fv = __ldg(pf);
            pf += NN;
            acc = cmk<T>((T)fv.x - acc.x, (T)fv.y - acc.y);
        }
        *py = acc;
        px += NN;
        py += NN;
        pk += NN;
        u_prev = u_cur;
        u_cur = u_next;
        u_next = u_nn;
        xm = nxm; xp = nxp; ym = nym; yp = nyp; kap = nkap;
    }
}

template <class T, class VI, int MODE>
cudaError_t launch(helm_ctx* h, const VI* x, VI* y, const float2* f, const T* kappa,
                   const typename C2<T>::t* cdn, const typename C2<T>::t* cup, int nrhs,
                   cudaStream_t st) {
    const int N = h->g.N;
    dim3 block(256);
    dim3 grid((N * N + 255) / 256, nrhs);
    size_t smem = 2 * sizeof(typename C2<T>::t) * N;
    k_stencil<T, VI, MODE><<<grid, block, smem, st>>>(x, y, f, kappa, cdn, cup, N);
    h->launches++;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stencil_c64(helm_ctx* h, const float2* x, float2* y, int nrhs, cudaStream_t st) {
    return launch<float, float2, 0>(h, x, y, nullptr, h->t.kappa, h->t.c_dn, h->t.c_up, nrhs, st);
}

cudaError_t launch_stencil_c128(helm_ctx* h, const double2* x, double2* y, int nrhs, cudaStream_t st) {
    return launch<double, double2, 0>(h, x, y, nullptr, h->t.kappa64, h->t.c_dn64,
                                      h->t.c_up64, nrhs, st);
}

cudaError_t launch_residual_c128(helm_ctx* h, const float2* f, const double2* u, double2* r,
                                 int nrhs, cudaStream_t st) {
    return launch<double, double2, 1>(h, u, r, f, h->t.kappa64, h->t.c_dn64, h->t.c_up64,
                                      nrhs, st);
}
