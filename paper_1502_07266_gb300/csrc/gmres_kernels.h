// Launchers of the GMRES vector kernels (gmres.cu).
#pragma once
#include "helm_internal.h"

cudaError_t gm_dots(helm_ctx* h, const float2* V, long long vstride, int j0, int nv, const float2* w,
                    long long n, int R, double2* partial, double2* out, int ostride, int accumulate,
                    cudaStream_t st);
cudaError_t gm_axpy(helm_ctx* h, const float2* V, long long vstride, int J, const double2* hcoef,
                    int hstride, float2* w, long long n, int R, cudaStream_t st);
cudaError_t gm_norm2_c64(helm_ctx* h, const float2* x, long long n, int R, double2* partial, double* out,
                         cudaStream_t st);
cudaError_t gm_norm2_c128(helm_ctx* h, const double2* x, long long n, int R, double2* partial,
                          double* out, cudaStream_t st);
cudaError_t gm_scale_c128(helm_ctx* h, const double2* src, const double* scale, float2* dst, long long n,
                          int R, cudaStream_t st);
cudaError_t gm_scale_c64(helm_ctx* h, const float2* src, const double* scale, float2* dst, long long n,
                         int R, cudaStream_t st);
cudaError_t gm_update(helm_ctx* h, const float2* Z, long long zstride, const double2* y, int ystride,
                      const int* mlen, double2* u, long long n, int R, cudaStream_t st);
cudaError_t gm_to_c64(helm_ctx* h, const double2* src, float2* dst, long long n, cudaStream_t st);
cudaError_t gm_givens(helm_ctx* h, double2* H, double2* cs, double2* sn, double2* g, double* est,
                      const int* frozen, int R, int m, int j, cudaStream_t st);
cudaError_t gm_backsolve(helm_ctx* h, const double2* H, const double2* g, double2* y, const int* mlen,
                         int R, int m, cudaStream_t st);
cudaError_t gm_cycle_start(helm_ctx* h, const double* rn2, double2* g, double* inv, const int* active,
                           int R, int m, cudaStream_t st);
cudaError_t gm_subdiag(helm_ctx* h, const double* wn2, double2* H, double* inv, const int* frozen, int R,
                       int m, int j, cudaStream_t st);
cudaError_t gm_addcol(helm_ctx* h, const double2* src, int sstride, double2* dst, int dstride, int J, int R,
                      cudaStream_t st);
cudaError_t gm_converge(helm_ctx* h, const double* est, const double* fn2, double tol, int maxit, int* frozen,
                        int* its, int* mlen, int j, int R, int* nact, cudaStream_t st);
cudaError_t gm_cycle_len(helm_ctx* h, const int* active, int* mlen, int jend, int R, cudaStream_t st);
