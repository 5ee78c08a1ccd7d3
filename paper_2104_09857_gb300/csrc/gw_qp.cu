// Quasiparticle energies from the self-energy on imaginary time, FP64 on the
// device: Sigma^c_n(+-i tau) -> Sigma^c_n(i omega) by a cosine and a sine
// transform, analytic continuation to the real axis with a Pade interpolant
// (Thiele's continued fraction through all frequency points, coefficients by
// the Vidberg-Serene recursion), and the Newton-Raphson solve of the
// quasiparticle equation, Eq. 12.  One thread per orbital.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "gw_internal.h"

namespace {

constexpr int kMaxOmega = 128;
constexpr int kMaxIter = 100;
constexpr double kTol = 1e-12;
constexpr double kH = 1e-6;  // central-difference step of the derivative of Re Sigma^c

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a / b by Smith's method (scaled by the larger component of b)
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.y + b.x * r;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}

// Re C(x) of the continued fraction with coefficients a[0..n) and nodes
// z_p = i omega_p: C(w) = a0 / (1 + a1 (w - z0) / (1 + a2 (w - z1) / ...)).
__device__ double re_pade(double x, const double2* a, const double* omega, int n) {
  const double2 w = make_double2(x, 0.0);
  double2 acc = make_double2(1.0, 0.0);
  for (int p = n - 1; p >= 1; --p)
    acc = cadd(make_double2(1.0, 0.0), cdiv(cmul(a[p], csub(w, make_double2(0.0, omega[p - 1]))), acc));
  return cdiv(a[0], acc).x;
}

__global__ void k_qp(int n_orb, int n_tau, int n_om, const double* __restrict__ sig,
                     const double* __restrict__ omega, const double* __restrict__ gamma,
                     const double* __restrict__ sw, const double* __restrict__ eps,
                     const double* __restrict__ vxc, const double* __restrict__ sx,
                     double* __restrict__ out, int* __restrict__ iters) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_orb) return;
  double2 u[kMaxOmega];
  // Sigma(i omega_k) = sum_j [gamma_kj / 2 (S+ + S-) - i s_kj (S+ - S-)]
  for (int k = 0; k < n_om; ++k) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < n_tau; ++j) {
      const double sp = sig[(static_cast<long long>(a) * n_tau + j) * 2];
      const double sm = sig[(static_cast<long long>(a) * n_tau + j) * 2 + 1];
      re += 0.5 * gamma[k * n_tau + j] * (sp + sm);
      im -= sw[k * n_tau + j] * (sp - sm);
    }
    u[k] = make_double2(re, im);
  }
  // coefficients in place: after step p, u[p] = a_p
  for (int p = 1; p < n_om; ++p) {
    const double2 prev = u[p - 1];
    const double2 zp = make_double2(0.0, omega[p - 1]);
    for (int i = p; i < n_om; ++i)
      u[i] = cdiv(csub(prev, u[i]), cmul(csub(make_double2(0.0, omega[i]), zp), u[i]));
  }
  const double e0 = eps[a] - vxc[a] + sx[a];
  double e = eps[a];
  // iterations to convergence, or -(iterations done) when the solve stopped
  // without converging: a zero or non-finite derivative, a non-finite step,
  // or kMaxIter steps
  int status = -kMaxIter;
  for (int it = 1; it <= kMaxIter; ++it) {
    const double f = e - (e0 + re_pade(e, u, omega, n_om));
    const double d = 1.0 - (re_pade(e + kH, u, omega, n_om) - re_pade(e - kH, u, omega, n_om)) / (2.0 * kH);
    if (!(d != 0.0) || !isfinite(d) || !isfinite(f)) {
      status = -it;
      break;
    }
    const double step = f / d;
    if (!isfinite(step)) {
      status = -it;
      break;
    }
    e -= step;
    if (fabs(step) < kTol * fmax(1.0, fabs(e))) {
      status = it;
      break;
    }
  }
  out[a] = e;
  iters[a] = status;
}

#define QP_TRY(call)                                                               \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ctx->err = std::string("gw_qp_g0w0: ") + #call + ": " + cudaGetErrorString(e_); \
      return e_ == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA;           \
    }                                                                              \
  } while (0)

bool all_finite(const double* p, long long n) {
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

}  // namespace

extern "C" int gw_qp_g0w0(gw_ctx* ctx, int n_orb, int n_tau, int n_omega, const double* sigma_c,
                          const double* omega, const double* gamma, const double* s_weights,
                          const double* eps, const double* vxc, const double* sx, double* qp_out,
                          int* iters_out) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_qp_g0w0");
  ctx->err.clear();
  if (n_orb <= 0 || n_tau <= 0 || n_omega <= 1 || n_omega > kMaxOmega || !sigma_c || !omega ||
      !gamma || !s_weights || !eps || !vxc || !sx || !qp_out) {
    ctx->err = "gw_qp_g0w0: bad arguments (need n_orb, n_tau >= 1, 2 <= n_omega <= 128, non-null arrays)";
    return GW_ERR_INVALID_ARG;
  }
  for (int k = 0; k < n_omega; ++k) {
    bool ok = omega[k] > 0.0;
    for (int l = 0; l < k && ok; ++l) ok = omega[k] != omega[l];
    if (!ok) {
      ctx->err = "gw_qp_g0w0: frequencies must be positive and distinct";
      return GW_ERR_INVALID_ARG;
    }
  }
  if (!all_finite(sigma_c, 2LL * n_orb * n_tau) || !all_finite(omega, n_omega) ||
      !all_finite(gamma, (long long)n_omega * n_tau) || !all_finite(s_weights, (long long)n_omega * n_tau) ||
      !all_finite(eps, n_orb) || !all_finite(vxc, n_orb) || !all_finite(sx, n_orb)) {
    ctx->err = "gw_qp_g0w0: non-finite input";
    return GW_ERR_NONFINITE;
  }
  QP_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DevBuf b_sig, b_om, b_g, b_s, b_e, b_v, b_x, b_out, b_it;
  const size_t nw = (size_t)n_omega * n_tau;
  QP_TRY(cudaMalloc(&b_sig.p, 2 * (size_t)n_orb * n_tau * sizeof(double)));
  QP_TRY(cudaMalloc(&b_om.p, n_omega * sizeof(double)));
  QP_TRY(cudaMalloc(&b_g.p, nw * sizeof(double)));
  QP_TRY(cudaMalloc(&b_s.p, nw * sizeof(double)));
  QP_TRY(cudaMalloc(&b_e.p, n_orb * sizeof(double)));
  QP_TRY(cudaMalloc(&b_v.p, n_orb * sizeof(double)));
  QP_TRY(cudaMalloc(&b_x.p, n_orb * sizeof(double)));
  QP_TRY(cudaMalloc(&b_out.p, n_orb * sizeof(double)));
  QP_TRY(cudaMalloc(&b_it.p, n_orb * sizeof(int)));
  QP_TRY(cudaMemcpyAsync(b_sig.p, sigma_c, 2 * (size_t)n_orb * n_tau * sizeof(double),
                         cudaMemcpyHostToDevice, st));
  QP_TRY(cudaMemcpyAsync(b_om.p, omega, n_omega * sizeof(double), cudaMemcpyHostToDevice, st));
  QP_TRY(cudaMemcpyAsync(b_g.p, gamma, nw * sizeof(double), cudaMemcpyHostToDevice, st));
  QP_TRY(cudaMemcpyAsync(b_s.p, s_weights, nw * sizeof(double), cudaMemcpyHostToDevice, st));
  QP_TRY(cudaMemcpyAsync(b_e.p, eps, n_orb * sizeof(double), cudaMemcpyHostToDevice, st));
  QP_TRY(cudaMemcpyAsync(b_v.p, vxc, n_orb * sizeof(double), cudaMemcpyHostToDevice, st));
  QP_TRY(cudaMemcpyAsync(b_x.p, sx, n_orb * sizeof(double), cudaMemcpyHostToDevice, st));
  k_qp<<<(n_orb + 127) / 128, 128, 0, st>>>(n_orb, n_tau, n_omega, (const double*)b_sig.p,
                                             (const double*)b_om.p, (const double*)b_g.p,
                                             (const double*)b_s.p, (const double*)b_e.p,
                                             (const double*)b_v.p, (const double*)b_x.p,
                                             (double*)b_out.p, (int*)b_it.p);
  QP_TRY(cudaGetLastError());
  QP_TRY(cudaMemcpyAsync(qp_out, b_out.p, n_orb * sizeof(double), cudaMemcpyDeviceToHost, st));
  std::vector<int> it(n_orb);
  QP_TRY(cudaMemcpyAsync(it.data(), b_it.p, n_orb * sizeof(int), cudaMemcpyDeviceToHost, st));
  QP_TRY(cudaStreamSynchronize(st));
  if (iters_out)
    for (int a = 0; a < n_orb; ++a) iters_out[a] = it[a];
  for (int a = 0; a < n_orb; ++a)
    if (it[a] <= 0) {
      ctx->err = "gw_qp_g0w0: the Newton solve of orbital " + std::to_string(a) +
                 " did not converge (" + std::to_string(-it[a]) +
                 " iterations; zero or non-finite derivative, or the iteration limit)";
      return GW_ERR_NOT_CONVERGED;
    }
  return GW_OK;
}
