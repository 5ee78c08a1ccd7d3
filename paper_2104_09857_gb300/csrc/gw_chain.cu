// C ABI of the screening chain: chi(i tau) -> chi(i omega) -> eps(i omega)
// (Eq. 7, with V = L L^T, Eq. 8) -> W^c(i omega) (Eq. 9) -> W^c(i tau).
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "gw_internal.h"
#include "k_chain.h"

namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

#define CH_TRY(call)                                                              \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ctx->err = std::string("chain: ") + #call + ": " + cudaGetErrorString(e_);      \
      return e_ == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA;          \
    }                                                                             \
  } while (0)

}  // namespace

extern "C" int gw_chi_to_w(gw_ctx* ctx, const double* V, int n_omega, const double* gamma,
                           const double* delta, const double* chi_tau, int chi_on_device,
                           double* w_tau_out, int out_on_device) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_chi_to_w");
  ctx->err.clear();
  if (ctx->n_at == 0 || !ctx->have_greens) {
    ctx->err = "gw_chi_to_w: call gw_set_basis and gw_set_greens first (the tau grid)";
    return GW_ERR_ORDER;
  }
  const int n = ctx->nri;
  const int n_tau = (int)ctx->tau.size();
  if (!V || !gamma || !delta || !chi_tau || !w_tau_out || n_omega <= 0 || n_omega > 4096) {
    ctx->err = "gw_chi_to_w: bad arguments";
    return GW_ERR_INVALID_ARG;
  }
  for (long long i = 0; i < (long long)n_omega * n_tau; ++i)
    if (!std::isfinite(gamma[i]) || !std::isfinite(delta[i])) {
      ctx->err = "gw_chi_to_w: non-finite transform weight";
      return GW_ERR_NONFINITE;
    }
  for (long long i = 0; i < (long long)n * n; ++i)
    if (!std::isfinite(V[i])) {
      ctx->err = "gw_chi_to_w: non-finite Coulomb matrix element";
      return GW_ERR_NONFINITE;
    }
  CH_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const size_t nn = (size_t)n * n;
  DevBuf b_low, b_chi, b_w, b_cw, b_t1, b_eps, b_z, b_ww, b_g, b_d, b_err;
  CH_TRY(cudaMalloc(&b_low.p, nn * 8));
  CH_TRY(cudaMalloc(&b_cw.p, nn * 8));
  CH_TRY(cudaMalloc(&b_t1.p, nn * 8));
  CH_TRY(cudaMalloc(&b_eps.p, nn * 8));
  CH_TRY(cudaMalloc(&b_z.p, nn * 8));
  CH_TRY(cudaMalloc(&b_ww.p, nn * 8));
  CH_TRY(cudaMalloc(&b_g.p, (size_t)n_omega * n_tau * 8));
  CH_TRY(cudaMalloc(&b_d.p, (size_t)n_omega * n_tau * 8));
  CH_TRY(cudaMalloc(&b_err.p, sizeof(int)));
  double* low = (double*)b_low.p;
  double* cw = (double*)b_cw.p;
  double* t1 = (double*)b_t1.p;
  double* eps = (double*)b_eps.p;
  double* z = (double*)b_z.p;
  double* ww = (double*)b_ww.p;
  double* g = (double*)b_g.p;
  double* d = (double*)b_d.p;
  int* err = (int*)b_err.p;
  const double* chi;
  if (chi_on_device) {
    chi = chi_tau;
  } else {
    CH_TRY(cudaMalloc(&b_chi.p, (size_t)n_tau * nn * 8));
    CH_TRY(cudaMemcpyAsync(b_chi.p, chi_tau, (size_t)n_tau * nn * 8, cudaMemcpyHostToDevice, st));
    chi = (const double*)b_chi.p;
  }
  double* wout;
  if (out_on_device) {
    wout = w_tau_out;
  } else {
    CH_TRY(cudaMalloc(&b_w.p, (size_t)n_tau * nn * 8));
    wout = (double*)b_w.p;
  }
  CH_TRY(cudaMemsetAsync(wout, 0, (size_t)n_tau * nn * 8, st));
  CH_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  CH_TRY(cudaMemcpyAsync(low, V, nn * 8, cudaMemcpyHostToDevice, st));
  CH_TRY(cudaMemcpyAsync(g, gamma, (size_t)n_omega * n_tau * 8, cudaMemcpyHostToDevice, st));
  CH_TRY(cudaMemcpyAsync(d, delta, (size_t)n_omega * n_tau * 8, cudaMemcpyHostToDevice, st));
  // V = L L^T (Eq. 8)
  gw::chain_potrf(low, n, err, st);
  CH_TRY(cudaGetLastError());
  int h_err = 0;
  CH_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CH_TRY(cudaStreamSynchronize(st));
  if (h_err) {
    ctx->err = "gw_chi_to_w: the Coulomb matrix is not positive definite";
    return GW_ERR_NOT_SPD;
  }
  for (int k = 0; k < n_omega; ++k) {
    // chi(i omega_k) = sum_j gamma_kj chi(i tau_j)
    gw::chain_lincomb(chi, n_tau, g + (size_t)k * n_tau, 1, (long long)nn, cw, st);
    // eps = 1 - L^T (chi L)     (Eq. 7)
    gw::chain_dgemm(false, false, n, n, n, 1.0, cw, n, low, n, 0.0, t1, n, st);
    gw::chain_set_identity(eps, n, st);
    gw::chain_dgemm(true, false, n, n, n, -1.0, low, n, t1, n, 1.0, eps, n, st);
    // eps = R R^T; Z = R^-1 L^T; W^c = Z^T Z - V   (Eq. 9)
    gw::chain_potrf(eps, n, err, st);
    gw::chain_transpose(low, z, n, st);
    gw::chain_trsm_left_lower(eps, n, z, n, st);
    gw::chain_dgemm(false, true, n, n, n, 1.0, low, n, low, n, 0.0, ww, n, st);  // V = L L^T
    gw::chain_dgemm(true, false, n, n, n, 1.0, z, n, z, n, -1.0, ww, n, st);
    // W^c(i tau_j) += delta_jk W^c(i omega_k)
    gw::chain_axpy_multi(ww, d, n_omega, k, n_tau, (long long)nn, wout, st);
    CH_TRY(cudaGetLastError());
  }
  CH_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (!out_on_device)
    CH_TRY(cudaMemcpyAsync(w_tau_out, wout, (size_t)n_tau * nn * 8, cudaMemcpyDeviceToHost, st));
  CH_TRY(cudaStreamSynchronize(st));
  if (h_err) {
    ctx->err = "gw_chi_to_w: eps(i omega) is not positive definite (chi must be negative semidefinite)";
    return GW_ERR_NOT_SPD;
  }
  return GW_OK;
}

// S^-1 M S^-1 for n_mat symmetric matrices M (chi~ of Eq. 5, W~ of Eq. 10,
// V~ of Eq. 11), FP64: S = R R^T (blocked Cholesky), R^-1 by a triangular
// solve on the identity, S^-1 = R^-T R^-1, then two products per matrix.
extern "C" int gw_ri_metric(gw_ctx* ctx, const double* S, int n_mat, const double* M, int m_on_device,
                            double* out, int out_on_device) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_ri_metric");
  ctx->err.clear();
  if (ctx->n_at == 0) {
    ctx->err = "gw_ri_metric: call gw_set_basis first (the RI size)";
    return GW_ERR_ORDER;
  }
  if (!S || !M || !out || n_mat <= 0) {
    ctx->err = "gw_ri_metric: bad arguments";
    return GW_ERR_INVALID_ARG;
  }
  const int n = ctx->nri;
  const size_t nn = (size_t)n * n;
  for (size_t i = 0; i < nn; ++i)
    if (!std::isfinite(S[i])) {
      ctx->err = "gw_ri_metric: non-finite metric element";
      return GW_ERR_NONFINITE;
    }
  CH_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DevBuf b_r, b_ri, b_si, b_t, b_m, b_o, b_err;
  CH_TRY(cudaMalloc(&b_r.p, nn * 8));
  CH_TRY(cudaMalloc(&b_ri.p, nn * 8));
  CH_TRY(cudaMalloc(&b_si.p, nn * 8));
  CH_TRY(cudaMalloc(&b_t.p, nn * 8));
  CH_TRY(cudaMalloc(&b_err.p, sizeof(int)));
  double *r = (double*)b_r.p, *ri = (double*)b_ri.p, *si = (double*)b_si.p, *t = (double*)b_t.p;
  int* err = (int*)b_err.p;
  const double* m = M;
  if (!m_on_device) {
    CH_TRY(cudaMalloc(&b_m.p, (size_t)n_mat * nn * 8));
    CH_TRY(cudaMemcpyAsync(b_m.p, M, (size_t)n_mat * nn * 8, cudaMemcpyHostToDevice, st));
    m = (const double*)b_m.p;
  }
  double* o = out;
  if (!out_on_device) {
    CH_TRY(cudaMalloc(&b_o.p, (size_t)n_mat * nn * 8));
    o = (double*)b_o.p;
  }
  CH_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  CH_TRY(cudaMemcpyAsync(r, S, nn * 8, cudaMemcpyHostToDevice, st));
  gw::chain_potrf(r, n, err, st);
  CH_TRY(cudaGetLastError());
  int h_err = 0;
  CH_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CH_TRY(cudaStreamSynchronize(st));
  if (h_err) {
    ctx->err = "gw_ri_metric: the metric is not positive definite";
    return GW_ERR_NOT_SPD;
  }
  gw::chain_set_identity(ri, n, st);
  gw::chain_trsm_left_lower(r, n, ri, n, st);                                 // R^-1
  gw::chain_dgemm(true, false, n, n, n, 1.0, ri, n, ri, n, 0.0, si, n, st);  // S^-1 = R^-T R^-1
  for (int k = 0; k < n_mat; ++k) {
    gw::chain_dgemm(false, false, n, n, n, 1.0, si, n, m + (size_t)k * nn, n, 0.0, t, n, st);
    gw::chain_dgemm(false, false, n, n, n, 1.0, t, n, si, n, 0.0, o + (size_t)k * nn, n, st);
  }
  CH_TRY(cudaGetLastError());
  if (!out_on_device)
    CH_TRY(cudaMemcpyAsync(out, o, (size_t)n_mat * nn * 8, cudaMemcpyDeviceToHost, st));
  CH_TRY(cudaStreamSynchronize(st));
  return GW_OK;
}
