// The full atomic-orbital matrix of the correlation self-energy, Eq. 10
// before it is projected on an orbital:
//   Sigma_{mu nu}(+i tau) = -sum (mu lam|P) G^occ_{lam sig}(tau) W_PQ(tau) (sig nu|Q)
//   Sigma_{mu nu}(-i tau) = +sum (mu lam|P) G^virt_{lam sig}(tau) W_PQ(tau) (sig nu|Q)
// (the real representation of gw_sigma_tau: C_n^T Sigma C_n is Sigma^c_n).
//
// FP64 dense route for molecules: T[mu][lam][P] is scattered once from the
// stored atom blocks, then per tau point three products on the CUDA cores,
//   Z = T W            (n_AO^2 x n_RI by n_RI x n_RI),
//   U = G Z            (n_AO x n_AO by n_AO x n_AO n_RI),
//   Sigma = -+ sum_lam T[:, lam, :] U[lam]^T   (n_AO products of n_AO x n_RI).
// Memory is 3 n_AO^2 n_RI doubles; the filter drops 3c blocks and G blocks
// with Frobenius norm < thr, like the other contractions.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gw_internal.h"
#include "k_chain.h"
#include "k_simt.h"

namespace gw {
namespace sigma_ao {

// One CTA per stored block (A <= B, P): its [nA][nB][nP] elements go to
// T[a0 + i][b0 + j][p0 + p] and, for A != B, to the mirrored T[b0 + j][a0 + i].
// Blocks with norm < thr stay zero.  Every index is checked against the
// dense size before the store.
__global__ void k_scatter_3c(const double* __restrict__ t3, const int* __restrict__ blk,
                             const long long* __restrict__ blk_off, const double* __restrict__ blk_norm,
                             double thr, const int* __restrict__ ao_off, const int* __restrict__ ri_off,
                             int nao, int nri, long long total, double* __restrict__ T) {
  const long long b = blockIdx.x;
  if (blk_norm[b] < thr) return;
  const int A = blk[3 * b], B = blk[3 * b + 1], P = blk[3 * b + 2];
  const int a0 = ao_off[A], na = ao_off[A + 1] - a0;
  const int b0 = ao_off[B], nb = ao_off[B + 1] - b0;
  const int p0 = ri_off[P], np = ri_off[P + 1] - p0;
  const double* src = t3 + blk_off[b];
  const int cnt = na * nb * np;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int i = e / (nb * np), j = (e / np) % nb, p = e % np;
    const double v = src[e];
    const long long x1 = (static_cast<long long>(a0 + i) * nao + b0 + j) * nri + p0 + p;
    if (x1 < total) T[x1] = v;
    if (A != B) {
      const long long x2 = (static_cast<long long>(b0 + j) * nao + a0 + i) * nri + p0 + p;
      if (x2 < total) T[x2] = v;
    }
  }
}

}  // namespace sigma_ao
}  // namespace gw

namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// n_AO^2 n_RI elements of each of T, Z and U (24 GB each at the limit)
constexpr long long kMaxDense = 3LL << 30;

#define SA_TRY(call)                                                              \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ctx->err = std::string("gw_sigma_ao_tau: ") + #call + ": " + cudaGetErrorString(e_); \
      return e_ == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA;          \
    }                                                                             \
  } while (0)

}  // namespace

extern "C" int gw_sigma_ao_tau(gw_ctx* ctx, const double* W_tau, int w_on_device, double thr,
                               double* sigma_out, int out_on_device) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_sigma_ao_tau");
  ctx->err.clear();
  if (ctx->d_t3f) {
    ctx->err = "gw_sigma_ao_tau: the tensor is kept in FP32 (option tensor_fp32); this route needs it in FP64";
    return GW_ERR_UNSUPPORTED;
  }
  if (!ctx->have_greens || ctx->n_at == 0 || (ctx->n_blocks > 0 && ctx->d_t3 == nullptr)) {
    ctx->err = "gw_sigma_ao_tau: call gw_set_basis, gw_set_3c_tensor and gw_set_greens first";
    return GW_ERR_ORDER;
  }
  if (!W_tau || !sigma_out || !(thr >= 0.0) || !std::isfinite(thr)) {
    ctx->err = "gw_sigma_ao_tau: bad arguments";
    return GW_ERR_INVALID_ARG;
  }
  const int nao = ctx->nao, nri = ctx->nri, n_at = ctx->n_at;
  const int n_tau = static_cast<int>(ctx->tau.size());
  const long long dense = static_cast<long long>(nao) * nao * nri;
  // the products' grids: n_AO^2 rows of 64 (at most 65535 row tiles), n_AO n_RI columns in an int
  if (dense > kMaxDense || ctx->n_blocks > 0x7fffffffLL ||
      static_cast<long long>(nao) * nao > 65535LL * 64 || static_cast<long long>(nao) * nri > 0x7fffffffLL) {
    ctx->err = "gw_sigma_ao_tau: the dense route holds n_AO^2 n_RI <= 3*2^30 elements and n_AO <= 2047";
    return GW_ERR_INVALID_ARG;
  }
  const size_t nn_ao = static_cast<size_t>(nao) * nao, nn_ri = static_cast<size_t>(nri) * nri;
  if (!w_on_device)
    for (size_t i = 0; i < nn_ri * n_tau; ++i)
      if (!std::isfinite(W_tau[i])) {
        ctx->err = "gw_sigma_ao_tau: non-finite W";
        return GW_ERR_NONFINITE;
      }
  SA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DevBuf b_t, b_z, b_u, b_go, b_gv, b_cso, b_csv, b_fl, b_w, b_out;
  SA_TRY(cudaMalloc(&b_t.p, std::max<long long>(dense, 1) * 8));
  SA_TRY(cudaMalloc(&b_z.p, std::max<long long>(dense, 1) * 8));
  SA_TRY(cudaMalloc(&b_u.p, std::max<long long>(dense, 1) * 8));
  SA_TRY(cudaMalloc(&b_go.p, nn_ao * 8));
  SA_TRY(cudaMalloc(&b_gv.p, nn_ao * 8));
  SA_TRY(cudaMalloc(&b_cso.p, static_cast<size_t>(nao) * std::max(ctx->n_occ, 1) * 8));
  SA_TRY(cudaMalloc(&b_csv.p, static_cast<size_t>(nao) * std::max(nao - ctx->n_occ, 1) * 8));
  SA_TRY(cudaMalloc(&b_fl.p, static_cast<size_t>(n_at) * n_at));
  if (!w_on_device) SA_TRY(cudaMalloc(&b_w.p, nn_ri * 8));
  if (!out_on_device) SA_TRY(cudaMalloc(&b_out.p, 2 * nn_ao * 8));
  double* T = static_cast<double*>(b_t.p);
  double* Z = static_cast<double*>(b_z.p);
  double* U = static_cast<double*>(b_u.p);
  double* go = static_cast<double*>(b_go.p);
  double* gv = static_cast<double*>(b_gv.p);

  SA_TRY(cudaMemsetAsync(T, 0, std::max<long long>(dense, 1) * 8, st));
  if (ctx->n_blocks > 0) {
    gw::sigma_ao::k_scatter_3c<<<static_cast<unsigned>(ctx->n_blocks), 128, 0, st>>>(
        ctx->d_t3, ctx->d_blk, ctx->d_blk_off, ctx->d_blk_norm, thr, ctx->d_ao_off, ctx->d_ri_off, nao,
        nri, dense, T);
    SA_TRY(cudaGetLastError());
  }
  const long long row = static_cast<long long>(nao) * nri;  // one lambda (or sigma) slab of T, Z, U
  for (int j = 0; j < n_tau; ++j) {
    gw::launch_greens(ctx->d_C, ctx->d_eps, nao, ctx->n_occ, ctx->mu, ctx->tau[j],
                      static_cast<double*>(b_cso.p), static_cast<double*>(b_csv.p), go, gv, st);
    if (thr > 0.0) {
      gw::launch_sym_block_filter(go, nao, ctx->d_ao_off, n_at, thr, static_cast<unsigned char*>(b_fl.p), st);
      gw::launch_sym_block_filter(gv, nao, ctx->d_ao_off, n_at, thr, static_cast<unsigned char*>(b_fl.p), st);
    }
    const double* wj = W_tau + static_cast<size_t>(j) * nn_ri;
    if (!w_on_device) {
      SA_TRY(cudaMemcpyAsync(b_w.p, wj, nn_ri * 8, cudaMemcpyHostToDevice, st));
      wj = static_cast<const double*>(b_w.p);
    }
    // Z[sig][nu][P] = sum_Q T[sig][nu][Q] W[Q][P]
    gw::chain_dgemm(false, false, nao * nao, nri, nri, 1.0, T, nri, wj, nri, 0.0, Z, nri, st);
    double* dst = out_on_device ? sigma_out + static_cast<size_t>(j) * 2 * nn_ao
                                : static_cast<double*>(b_out.p);
    for (int k = 0; k < 2; ++k) {
      const double* g = k == 0 ? go : gv;
      const double sign = k == 0 ? -1.0 : 1.0;
      // U[lam][nu][P] = sum_sig G[lam][sig] Z[sig][nu][P]
      gw::chain_dgemm(false, false, nao, static_cast<int>(row), nao, 1.0, g, nao, Z, static_cast<int>(row),
                      0.0, U, static_cast<int>(row), st);
      // Sigma[mu][nu] = sign sum_lam sum_P T[mu][lam][P] U[lam][nu][P]
      double* out = dst + static_cast<size_t>(k) * nn_ao;
      for (int lam = 0; lam < nao; ++lam)
        gw::chain_dgemm(false, true, nao, nao, nri, sign, T + static_cast<size_t>(lam) * nri,
                        static_cast<int>(row), U + static_cast<size_t>(lam) * row, nri, lam == 0 ? 0.0 : 1.0,
                        out, nao, st);
    }
    SA_TRY(cudaGetLastError());
    if (!out_on_device)
      SA_TRY(cudaMemcpyAsync(sigma_out + static_cast<size_t>(j) * 2 * nn_ao, b_out.p, 2 * nn_ao * 8,
                             cudaMemcpyDeviceToHost, st));
  }
  SA_TRY(cudaStreamSynchronize(st));
  return GW_OK;
}
