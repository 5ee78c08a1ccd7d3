// Eigenvalue-self-consistent GW (the paragraph after Eq. 12): host
// orchestration of the library's own steps.  Each cycle builds G (Eq. 2) from
// the current levels and runs chi (Eq. 3), the FP64 chain to W^c (Eqs. 7-9),
// Sigma^c (Eq. 10) and the quasiparticle equation (Eq. 12); the new energies
// then shift the levels of the next cycle.  Every arithmetic step is one of
// the GPU entry points; this file only moves the levels and decides when to
// stop.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gw_internal.h"

namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// Levels of the next cycle: each level moves by the shift e_k - eps_k of the
// nearest listed orbital on its side of the gap (nearest by index; on a tie
// the one nearer the gap); a side with no listed orbital keeps its levels.
void shifted_levels(const std::vector<double>& eps, int n_occ, const int* orbitals, int n_orb,
                    const double* e_qp, std::vector<double>& out) {
  out = eps;
  for (int i = 0; i < static_cast<int>(eps.size()); ++i) {
    const bool occ = i < n_occ;
    int best = -1;
    for (int k = 0; k < n_orb; ++k) {
      const int n = orbitals[k];
      if ((n < n_occ) != occ) continue;
      if (best < 0) {
        best = k;
        continue;
      }
      const int d = std::abs(n - i), db = std::abs(orbitals[best] - i);
      if (d < db || (d == db && (occ ? n > orbitals[best] : n < orbitals[best]))) best = k;
    }
    if (best >= 0) out[i] = eps[i] + (e_qp[best] - eps[orbitals[best]]);
  }
}

// Puts the levels given to gw_set_greens back on the device when the call
// ends, whatever the exit path.
struct RestoreLevels {
  gw_ctx* ctx;
  ~RestoreLevels() {
    cudaMemcpyAsync(ctx->d_eps, ctx->h_eps.data(), ctx->h_eps.size() * sizeof(double),
                    cudaMemcpyHostToDevice, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
  }
};

int ev_fail(gw_ctx* ctx, int code, const std::string& msg) {
  ctx->err = "gw_evgw: " + msg;
  return code;
}

}  // namespace

extern "C" int gw_evgw(gw_ctx* ctx, const double* V, int n_omega, const double* omega,
                       const double* gamma, const double* delta, const double* s_weights,
                       const int* orbitals, int n_orb, const double* vxc, double thr, int precision,
                       int max_cycles, double tol, double* qp_out, int* cycles_out) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_evgw");
  ctx->err.clear();
  if (ctx->n_at == 0 || !ctx->have_greens || ctx->h_eps.empty())
    return ev_fail(ctx, GW_ERR_ORDER, "call gw_set_basis, gw_set_3c_tensor and gw_set_greens first");
  if (!V || !omega || !gamma || !delta || !s_weights || !orbitals || !vxc || !qp_out || n_orb < 1 ||
      n_omega < 2 || max_cycles < 1 || !(tol > 0.0) || !std::isfinite(tol))
    return ev_fail(ctx, GW_ERR_INVALID_ARG, "bad arguments");
  const int nao = ctx->nao;
  for (int k = 0; k < n_orb; ++k)
    if (orbitals[k] < 0 || orbitals[k] >= nao) return ev_fail(ctx, GW_ERR_INVALID_ARG, "orbital index out of range");
  const int n_tau = static_cast<int>(ctx->tau.size());
  const size_t per_tau = static_cast<size_t>(ctx->nri) * ctx->nri;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ev_fail(ctx, GW_ERR_CUDA, "cudaSetDevice");
  DevBuf chi, w;
  if (cudaMalloc(&chi.p, std::max<size_t>(per_tau * n_tau, 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&w.p, std::max<size_t>(per_tau * n_tau, 1) * sizeof(double)) != cudaSuccess)
    return ev_fail(ctx, GW_ERR_OOM, "device buffers for chi and W");

  std::vector<double> sx(n_orb), sig(static_cast<size_t>(n_orb) * n_tau * 2), e(n_orb), prev(n_orb),
      eps_n(n_orb), levels;
  for (int k = 0; k < n_orb; ++k) eps_n[k] = ctx->h_eps[orbitals[k]];
  int rc = gw_sigma_x(ctx, V, 0, orbitals, n_orb, thr, precision, sx.data());
  if (rc) return rc;

  RestoreLevels restore{ctx};
  for (int cycle = 1; cycle <= max_cycles; ++cycle) {
    if ((rc = gw_chi_tau(ctx, 0, n_tau, thr, precision, GW_SCREEN_BOUND, static_cast<double*>(chi.p), 1)))
      return rc;
    if ((rc = gw_chi_to_w(ctx, V, n_omega, gamma, delta, static_cast<double*>(chi.p), 1,
                          static_cast<double*>(w.p), 1)))
      return rc;
    if ((rc = gw_sigma_tau(ctx, static_cast<double*>(w.p), 1, orbitals, n_orb, thr, precision, sig.data())))
      return rc;
    if ((rc = gw_qp_g0w0(ctx, n_orb, n_tau, n_omega, sig.data(), omega, gamma, s_weights, eps_n.data(),
                         vxc, sx.data(), e.data(), nullptr)))
      return rc;
    if (cycle > 1) {
      double change = 0.0;
      for (int k = 0; k < n_orb; ++k) change = std::max(change, std::fabs(e[k] - prev[k]));
      if (change < tol) {
        std::copy(e.begin(), e.end(), qp_out);
        if (cycles_out) *cycles_out = cycle;
        return GW_OK;
      }
    }
    prev = e;
    shifted_levels(ctx->h_eps, ctx->n_occ, orbitals, n_orb, e.data(), levels);
    for (int i = 0; i < nao; ++i)
      if ((i < ctx->n_occ) ? !(levels[i] < ctx->mu) : !(levels[i] > ctx->mu)) {
        std::copy(e.begin(), e.end(), qp_out);
        if (cycles_out) *cycles_out = cycle;
        return ev_fail(ctx, GW_ERR_NOT_CONVERGED, "a shifted level crossed mu_fermi");
      }
    if (cudaMemcpyAsync(ctx->d_eps, levels.data(), nao * sizeof(double), cudaMemcpyHostToDevice,
                        ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
      return ev_fail(ctx, GW_ERR_CUDA, "upload of the shifted levels");
  }
  std::copy(prev.begin(), prev.end(), qp_out);
  if (cycles_out) *cycles_out = max_cycles;
  return ev_fail(ctx, GW_ERR_NOT_CONVERGED, "no convergence within max_cycles");
}
