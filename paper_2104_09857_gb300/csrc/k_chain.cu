// FP64 kernels of the screening chain between chi(i tau) and W^c(i tau):
// cosine transforms (weighted sums over the time or frequency grid), the
// dielectric matrix eps = 1 - L^T chi L (Eq. 7) with V = L L^T (Eq. 8), its
// Cholesky factorisation, a triangular solve, and W^c = L (eps^-1 - 1) L^T
// (Eq. 9) formed as Z^T Z - V with Z = R^-1 L^T, eps = R R^T.
//
// Everything is FP64: the transform weights are large and of both signs (the
// sums cancel), and the factorisation of eps needs the precision.  Row-major
// n x n matrices throughout.
#include <cuda_runtime.h>
#include <math.h>

#include "k_chain.h"

namespace gw {
namespace chain {

// out[k][e] = sum_j w[k * nin + j] * in[j][e]   (fixed j order)
__global__ void k_lincomb(const double* __restrict__ in, int nin, const double* __restrict__ w,
                          int nout, long long n, double* __restrict__ out) {
  long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (; e < n; e += stride) {
    for (int k = 0; k < nout; ++k) {
      double acc = 0.0;
      for (int j = 0; j < nin; ++j) acc = fma(w[k * nin + j], in[static_cast<long long>(j) * n + e], acc);
      out[static_cast<long long>(k) * n + e] = acc;
    }
  }
}

// out[j][e] += w[j * ldw + k] * x[e] for all j < nout
__global__ void k_axpy_multi(const double* __restrict__ x, const double* __restrict__ w, int ldw,
                             int k, int nout, long long n, double* __restrict__ out) {
  long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (; e < n; e += stride) {
    const double v = x[e];
    for (int j = 0; j < nout; ++j) out[static_cast<long long>(j) * n + e] += w[j * ldw + k] * v;
  }
}

__global__ void k_set_identity(double* __restrict__ a, int n) {
  long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long nn = static_cast<long long>(n) * n;
  if (i < nn) a[i] = (i / n == i % n) ? 1.0 : 0.0;
}

__global__ void k_transpose(const double* __restrict__ a, double* __restrict__ b, int n) {
  __shared__ double t[32][33];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8)
    if (y0 + i < n && x0 + tx < n) t[i][tx] = a[static_cast<long long>(y0 + i) * n + x0 + tx];
  __syncthreads();
  for (int i = ty; i < 32; i += 8)
    if (x0 + i < n && y0 + tx < n) b[static_cast<long long>(x0 + i) * n + y0 + tx] = t[tx][i];
}

__global__ void k_zero_upper(double* __restrict__ a, int n) {
  long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long nn = static_cast<long long>(n) * n;
  if (i < nn && i % n > i / n) a[i] = 0.0;
}

// C = alpha op(A) op(B) + beta C, m x n x k, row-major; op = transpose if TA/TB.
// 64 x 64 tile, 256 threads, thread (tx, ty) owns rows ty + 16 i, cols tx + 16 j.
template <bool TA, bool TB>
__global__ void k_dgemm(int m, int n, int k, double alpha, const double* __restrict__ A, int lda,
                        const double* __restrict__ B, int ldb, double beta, double* __restrict__ C,
                        int ldc) {
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < k; k0 += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + 256 * e;
      // A tile: As[kk][row] = op(A)[m0 + row][k0 + kk]
      if (!TA) {
        const int row = idx >> 4, kk = idx & 15;
        const int gm = m0 + row, gk = k0 + kk;
        As[kk][row] = (gm < m && gk < k) ? A[static_cast<long long>(gm) * lda + gk] : 0.0;
      } else {
        const int kk = idx >> 6, row = idx & 63;
        const int gm = m0 + row, gk = k0 + kk;
        As[kk][row] = (gm < m && gk < k) ? A[static_cast<long long>(gk) * lda + gm] : 0.0;
      }
      // B tile: Bs[kk][col] = op(B)[k0 + kk][n0 + col]
      if (!TB) {
        const int kk = idx >> 6, col = idx & 63;
        const int gk = k0 + kk, gn = n0 + col;
        Bs[kk][col] = (gk < k && gn < n) ? B[static_cast<long long>(gk) * ldb + gn] : 0.0;
      } else {
        const int col = idx >> 4, kk = idx & 15;
        const int gk = k0 + kk, gn = n0 + col;
        Bs[kk][col] = (gk < k && gn < n) ? B[static_cast<long long>(gn) * ldb + gk] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
      if (r < m && c < n) {
        double* p = C + static_cast<long long>(r) * ldc + c;
        *p = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *p);
      }
    }
}

constexpr int kNb = 32;

// Unblocked Cholesky of the b x b diagonal block at (k0, k0), in place
// (lower part); err[0] |= 1 on a non-positive or non-finite pivot.
__global__ void k_potrf_diag(double* __restrict__ a, int n, int k0, int b, int* __restrict__ err) {
  __shared__ double d[kNb][kNb + 1];
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  for (int i = t; i < b * b; i += blockDim.x) d[i / b][i % b] = a[static_cast<long long>(k0 + i / b) * n + k0 + i % b];
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (t == 0) {
      const double p = d[j][j];
      if (!(p > 0.0) || !isfinite(p)) {
        bad = 1;
        d[j][j] = 1.0;
      } else {
        d[j][j] = sqrt(p);
      }
    }
    __syncthreads();
    for (int i = j + 1 + t; i < b; i += blockDim.x) d[i][j] /= d[j][j];
    __syncthreads();
    for (int e = t; e < b * b; e += blockDim.x) {
      const int r = e / b, c = e % b;
      if (c > j && r >= c) d[r][c] -= d[r][j] * d[c][j];
    }
    __syncthreads();
  }
  for (int i = t; i < b * b; i += blockDim.x) {
    const int r = i / b, c = i % b;
    if (r >= c) a[static_cast<long long>(k0 + r) * n + k0 + c] = d[r][c];
  }
  if (t == 0 && bad) atomicOr(err, 1);
}

// Rows i >= k0 + b of the panel: A[i][k0:k0+b] <- A[i][k0:k0+b] D^-T, D the
// factored diagonal block (one thread per row, forward substitution).
__global__ void k_trsm_panel(double* __restrict__ a, int n, int k0, int b) {
  __shared__ double d[kNb][kNb + 1];
  for (int i = threadIdx.x; i < b * b; i += blockDim.x)
    d[i / b][i % b] = a[static_cast<long long>(k0 + i / b) * n + k0 + i % b];
  __syncthreads();
  const int row = k0 + b + blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  double x[kNb];
  double* r = a + static_cast<long long>(row) * n + k0;
#pragma unroll
  for (int c = 0; c < kNb; ++c) {
    if (c < b) {
      double v = r[c];
      for (int t = 0; t < c; ++t) v -= x[t] * d[c][t];
      x[c] = v / d[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < kNb; ++c)
    if (c < b) r[c] = x[c];
}

// Left lower solve on block rows k0..k0+b of B (n x m): B[k0:k0+b][col] <-
// D^-1 B[k0:k0+b][col], D = R[k0:k0+b][k0:k0+b] (one thread per column).
__global__ void k_trsm_rows(const double* __restrict__ r, int n, double* __restrict__ bm, int m,
                            int k0, int b) {
  __shared__ double d[kNb][kNb + 1];
  for (int i = threadIdx.x; i < b * b; i += blockDim.x)
    d[i / b][i % b] = r[static_cast<long long>(k0 + i / b) * n + k0 + i % b];
  __syncthreads();
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= m) return;
  double x[kNb];
#pragma unroll
  for (int i = 0; i < kNb; ++i) {
    if (i < b) {
      double v = bm[static_cast<long long>(k0 + i) * m + col];
      for (int t = 0; t < i; ++t) v -= d[i][t] * x[t];
      x[i] = v / d[i][i];
    }
  }
#pragma unroll
  for (int i = 0; i < kNb; ++i)
    if (i < b) bm[static_cast<long long>(k0 + i) * m + col] = x[i];
}

}  // namespace chain

namespace {
inline unsigned blocks_for(long long n, int threads, long long cap = 152LL * 16) {
  long long b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  return static_cast<unsigned>(b < 1 ? 1 : b);
}
}  // namespace

void chain_lincomb(const double* in, int nin, const double* w, int nout, long long n, double* out,
                   cudaStream_t st) {
  chain::k_lincomb<<<blocks_for(n, 256), 256, 0, st>>>(in, nin, w, nout, n, out);
}

void chain_axpy_multi(const double* x, const double* w, int ldw, int k, int nout, long long n,
                      double* out, cudaStream_t st) {
  chain::k_axpy_multi<<<blocks_for(n, 256), 256, 0, st>>>(x, w, ldw, k, nout, n, out);
}

void chain_set_identity(double* a, int n, cudaStream_t st) {
  const long long nn = static_cast<long long>(n) * n;
  chain::k_set_identity<<<static_cast<unsigned>((nn + 255) / 256), 256, 0, st>>>(a, n);
}

void chain_transpose(const double* a, double* b, int n, cudaStream_t st) {
  dim3 g((n + 31) / 32, (n + 31) / 32);
  chain::k_transpose<<<g, 256, 0, st>>>(a, b, n);
}

void chain_dgemm(bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
                 const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  dim3 g((n + 63) / 64, (m + 63) / 64);
  if (!ta && !tb) chain::k_dgemm<false, false><<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  if (!ta && tb) chain::k_dgemm<false, true><<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  if (ta && !tb) chain::k_dgemm<true, false><<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  if (ta && tb) chain::k_dgemm<true, true><<<g, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

// In-place blocked Cholesky (lower) of the n x n row-major a; strict upper
// triangle zeroed.  err[0] != 0 afterwards means a pivot was not positive.
void chain_potrf(double* a, int n, int* err, cudaStream_t st) {
  for (int k0 = 0; k0 < n; k0 += chain::kNb) {
    const int b = n - k0 < chain::kNb ? n - k0 : chain::kNb;
    chain::k_potrf_diag<<<1, 256, 0, st>>>(a, n, k0, b, err);
    const int rest = n - k0 - b;
    if (rest > 0) {
      chain::k_trsm_panel<<<(rest + 127) / 128, 128, 0, st>>>(a, n, k0, b);
      // trailing update A22 -= P P^T (P = rows k0+b.., columns k0..k0+b)
      const double* p = a + static_cast<long long>(k0 + b) * n + k0;
      double* a22 = a + static_cast<long long>(k0 + b) * n + k0 + b;
      chain_dgemm(false, true, rest, rest, b, -1.0, p, n, p, n, 1.0, a22, n, st);
    }
  }
  const long long nn = static_cast<long long>(n) * n;
  chain::k_zero_upper<<<static_cast<unsigned>((nn + 255) / 256), 256, 0, st>>>(a, n);
}

// B (n x m) <- R^-1 B, R lower triangular n x n (blocked forward substitution).
void chain_trsm_left_lower(const double* r, int n, double* bm, int m, cudaStream_t st) {
  for (int k0 = 0; k0 < n; k0 += chain::kNb) {
    const int b = n - k0 < chain::kNb ? n - k0 : chain::kNb;
    chain::k_trsm_rows<<<(m + 127) / 128, 128, 0, st>>>(r, n, bm, m, k0, b);
    const int rest = n - k0 - b;
    if (rest > 0) {
      // B[k0+b:, :] -= R[k0+b:, k0:k0+b] Z[k0:k0+b, :]
      chain_dgemm(false, false, rest, m, b, -1.0, r + static_cast<long long>(k0 + b) * n + k0, n,
                  bm + static_cast<long long>(k0) * m, m, 1.0, bm + static_cast<long long>(k0 + b) * m, m,
                  st);
    }
  }
}

}  // namespace gw
