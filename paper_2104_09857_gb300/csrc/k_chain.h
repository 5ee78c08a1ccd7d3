// Launchers of the FP64 screening-chain kernels (k_chain.cu).
#pragma once

#include <cuda_runtime.h>

namespace gw {

// out[k][e] = sum_j w[k * nin + j] in[j][e], n elements per matrix
void chain_lincomb(const double* in, int nin, const double* w, int nout, long long n, double* out,
                   cudaStream_t st);
// out[j][e] += w[j * ldw + k] x[e] for j < nout
void chain_axpy_multi(const double* x, const double* w, int ldw, int k, int nout, long long n,
                      double* out, cudaStream_t st);
void chain_set_identity(double* a, int n, cudaStream_t st);
void chain_transpose(const double* a, double* b, int n, cudaStream_t st);
// C = alpha op(A) op(B) + beta C (row-major; op transposes when ta / tb)
void chain_dgemm(bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
                 const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t st);
// in-place lower Cholesky; err[0] |= 1 on a non-positive pivot
void chain_potrf(double* a, int n, int* err, cudaStream_t st);
// B <- R^-1 B with R lower triangular (n x n), B n x m
void chain_trsm_left_lower(const double* r, int n, double* bm, int m, cudaStream_t st);

}  // namespace gw
