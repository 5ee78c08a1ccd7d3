// Diagonal correlation self-energy of Eq. 10 for selected orbitals n:
//   B^n[mu][P]  = sum_nu C[nu][n] (nu mu | P)          (half transform, Eq. 10 text)
//   S^g_n(tau)  = sum_{mu nu} G^g_{mu nu}(tau) (B^n W(tau) B^nT)_{mu nu},  g = occ, virt
//   Sigma^c_n(i tau) = -S^occ_n(tau),  Sigma^c_n(-i tau) = +S^virt_n(tau)
// FP64 throughout.  B^n is formed from the owner panels of the 3c tensor
// (each (sigma, P) pair belongs to exactly one panel); its (mu-atom, P-atom)
// blocks below the filter threshold are dropped, as are G blocks.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "gw_internal.h"
#include "k_chain.h"
#include "k_simt.h"
#include "k_tc.h"

namespace gw {
namespace sigma {

// Bn[j][ao(s) + s'][p0 + pw] = sum_k Csel[lam[k]][j] panel_s[k][pw * nsig + s']
__global__ void k_bn_panels(const double* __restrict__ pool, const PanelDesc* __restrict__ panels,
                            const int* __restrict__ owners, const int* __restrict__ lam,
                            const int* __restrict__ ao_off, const double* __restrict__ csel,
                            int n_orb, int nao, int nri, double* __restrict__ bn) {
  const PanelDesc d = panels[owners[blockIdx.y]];
  const int N = d.npw * d.nsig;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.z;
  if (n >= N) return;
  const double* p = pool + d.off;
  const int* lk = lam + d.lam_off;
  double acc = 0.0;
  for (int k = 0; k < d.K; ++k) acc = fma(csel[static_cast<long long>(lk[k]) * n_orb + j], p[static_cast<long long>(k) * N + n], acc);
  const int pw = n / d.nsig, sp = n - pw * d.nsig;
  bn[(static_cast<long long>(j) * nao + ao_off[d.owner] + sp) * nri + d.p0 + pw] = acc;
}

// zero the (mu-atom, P-atom) blocks of Bn_j with norm < thr (warp per block)
__global__ void k_bn_filter(double* __restrict__ bn, int n_orb, int n_at, int nao, int nri,
                            const int* __restrict__ ao_off, const int* __restrict__ ri_off, double thr) {
  const long long w = static_cast<long long>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  const long long nblk = static_cast<long long>(n_orb) * n_at * n_at;
  if (w >= nblk) return;
  const int p = static_cast<int>(w % n_at);
  const int m = static_cast<int>((w / n_at) % n_at);
  const int j = static_cast<int>(w / (static_cast<long long>(n_at) * n_at));
  const int r0 = ao_off[m], nr = ao_off[m + 1] - r0, c0 = ri_off[p], nc = ri_off[p + 1] - c0;
  double* base = bn + static_cast<long long>(j) * nao * nri;
  double s = 0.0;
  for (int e = lane; e < nr * nc; e += 32) {
    const double v = base[static_cast<long long>(r0 + e / nc) * nri + c0 + e % nc];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (sqrt(s) < thr)
    for (int e = lane; e < nr * nc; e += 32) base[static_cast<long long>(r0 + e / nc) * nri + c0 + e % nc] = 0.0;
}

// partial[b][0..1] = sum over this block's elements of (go * z, gv * z)
__global__ void k_dot2(const double* __restrict__ go, const double* __restrict__ gv,
                       const double* __restrict__ z, long long n, double* __restrict__ partial) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, b = 0.0;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    a = fma(go[i], z[i], a);
    b = fma(gv[i], z[i], b);
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0[0];
    partial[2 * blockIdx.x + 1] = s1[0];
  }
}

}  // namespace sigma
}  // namespace gw

namespace {
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};
#define SG_TRY(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ctx->err = std::string("gw_sigma_tau: ") + #call + ": " + cudaGetErrorString(e_); \
      return e_ == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA;               \
    }                                                                                  \
  } while (0)
constexpr int kDotBlocks = 256;
}  // namespace

namespace {
// Eq. 10 for the listed orbitals at the imaginary times taus[0..n_tau), with
// W_tau[n_tau][n_ri][n_ri]; sigma_out [n_orb][n_tau][2] = (-S^occ, +S^virt).
int sigma_impl(gw_ctx* ctx, const double* W_tau, int w_on_device, const int* orbitals, int n_orb,
               double thr, int precision, const double* taus, int n_tau, double* sigma_out) {
  if (ctx->n_at == 0 || ctx->blk_off.empty() || !ctx->have_greens) {
    ctx->err = "gw_sigma_tau: call gw_set_basis, gw_set_3c_tensor and gw_set_greens first";
    return GW_ERR_ORDER;
  }
  if (!W_tau || !orbitals || !sigma_out || n_orb <= 0 || n_orb > 1024 || !(thr >= 0.0) ||
      !std::isfinite(thr)) {
    ctx->err = "gw_sigma_tau: bad arguments";
    return GW_ERR_INVALID_ARG;
  }
  if (precision != GW_FP64 && precision != GW_BF16X3 && precision != GW_BF16X6 &&
      precision != GW_FP16X3) {
    ctx->err = "gw_sigma_tau: precision must be GW_FP64, GW_BF16X3, GW_BF16X6 or GW_FP16X3";
    return GW_ERR_UNSUPPORTED;
  }
  const bool mixed = precision != GW_FP64;
  const int slices = precision == GW_BF16X6 ? 3 : 2;
  const int f16 = precision == GW_FP16X3;
  const int nao = ctx->nao, nri = ctx->nri, n_at = ctx->n_at;
  for (int a = 0; a < n_orb; ++a)
    if (orbitals[a] < 0 || orbitals[a] >= nao) {
      ctx->err = "gw_sigma_tau: orbital index out of range";
      return GW_ERR_INVALID_ARG;
    }
  SG_TRY(cudaSetDevice(ctx->device));
  int rc = gw::build_panels_for(ctx, thr);
  if (rc) return rc;
  cudaStream_t st = ctx->stream;
  const size_t nn_ri = (size_t)nri * nri, nn_ao = (size_t)nao * nao;
  DevBuf b_w, b_csel, b_bn, b_y, b_z, b_cso, b_csv, b_go, b_gv, b_fl, b_part, b_own, b_aooff;
  const double* w;
  if (w_on_device) {
    w = W_tau;
  } else {
    SG_TRY(cudaMalloc(&b_w.p, (size_t)n_tau * nn_ri * 8));
    SG_TRY(cudaMemcpyAsync(b_w.p, W_tau, (size_t)n_tau * nn_ri * 8, cudaMemcpyHostToDevice, st));
    w = (const double*)b_w.p;
  }
  // selected orbital columns of C: csel[mu][j] = C[mu][orbitals[j]] (host gather
  // from the device copy would need a kernel; the host keeps no copy of C, so
  // gather on the device by strided copies)
  SG_TRY(cudaMalloc(&b_csel.p, (size_t)nao * n_orb * 8));
  for (int a = 0; a < n_orb; ++a)
    SG_TRY(cudaMemcpy2DAsync((double*)b_csel.p + a, n_orb * 8, ctx->d_C + orbitals[a], nao * 8, 8, nao,
                             cudaMemcpyDeviceToDevice, st));
  SG_TRY(cudaMalloc(&b_bn.p, (size_t)n_orb * nao * nri * 8));
  SG_TRY(cudaMemsetAsync(b_bn.p, 0, (size_t)n_orb * nao * nri * 8, st));
  std::vector<int> owners;
  int maxN = 0;
  for (int s = 0; s < n_at; ++s)
    if (ctx->panels[s].K > 0) {
      owners.push_back(s);
      maxN = std::max(maxN, ctx->panels[s].npw * ctx->panels[s].nsig);
    }
  DevBuf b_pd;
  SG_TRY(cudaMalloc(&b_pd.p, ctx->panels.size() * sizeof(gw::PanelDesc)));
  SG_TRY(cudaMemcpyAsync(b_pd.p, ctx->panels.data(), ctx->panels.size() * sizeof(gw::PanelDesc),
                         cudaMemcpyHostToDevice, st));
  SG_TRY(cudaMalloc(&b_own.p, std::max<size_t>(owners.size(), 1) * sizeof(int)));
  if (!owners.empty())
    SG_TRY(cudaMemcpyAsync(b_own.p, owners.data(), owners.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  double* bn = (double*)b_bn.p;
  if (!owners.empty()) {
    dim3 g((maxN + 127) / 128, (unsigned)owners.size(), n_orb);
    gw::sigma::k_bn_panels<<<g, 128, 0, st>>>(ctx->d_panel64, (const gw::PanelDesc*)b_pd.p,
                                              (const int*)b_own.p, ctx->d_lam, ctx->d_ao_off,
                                              (const double*)b_csel.p, n_orb, nao, nri, bn);
    SG_TRY(cudaGetLastError());
  }
  if (thr > 0.0) {
    const long long nblk = (long long)n_orb * n_at * n_at;
    gw::sigma::k_bn_filter<<<(unsigned)((nblk + 7) / 8), 256, 0, st>>>(bn, n_orb, n_at, nao, nri,
                                                                       ctx->d_ao_off, ctx->d_ri_off, thr);
    SG_TRY(cudaGetLastError());
  }
  SG_TRY(cudaMalloc(&b_y.p, (size_t)nao * nri * 8));
  SG_TRY(cudaMalloc(&b_z.p, nn_ao * 8));
  SG_TRY(cudaMalloc(&b_cso.p, (size_t)nao * std::max(ctx->n_occ, 1) * 8));
  SG_TRY(cudaMalloc(&b_csv.p, (size_t)nao * std::max(nao - ctx->n_occ, 1) * 8));
  SG_TRY(cudaMalloc(&b_go.p, nn_ao * 8));
  SG_TRY(cudaMalloc(&b_gv.p, nn_ao * 8));
  SG_TRY(cudaMalloc(&b_fl.p, (size_t)n_at * n_at));
  SG_TRY(cudaMalloc(&b_part.p, (size_t)kDotBlocks * 2 * 8));
  double *y = (double*)b_y.p, *z = (double*)b_z.p, *go = (double*)b_go.p, *gv = (double*)b_gv.p;
  std::vector<double> part((size_t)kDotBlocks * 2);
  // tensor-core route: both products as step-C style tile jobs on bf16 slices
  //   y = -(B W)     (rows mu, columns Q, K = P)
  //   z = -(y B^T)   (rows mu, columns nu, K = Q)  = B W B^T
  const int tile = gw::tc_tile_rows();
  const int kpad = (nri + 63) / 64 * 64;
  DevBuf b_bs, b_ws, b_ys, b_tl1, b_tk1, b_ct1, b_k01, b_ln1, b_tl2, b_tk2, b_ct2, b_err, b_mx;
  int nslab = 0, n_tiles1 = 0, n_tiles2 = 0, nqt1 = 0, nqt2 = 0;
  CUtensorMap m_b, m_w, m_y, m_bq;
  if (mixed) {
    const int slab = 512;
    nslab = (kpad + slab - 1) / slab;
    std::vector<long long> k0(nslab);
    std::vector<int> len(nslab);
    for (int i = 0; i < nslab; ++i) {
      k0[i] = (long long)i * slab;
      len[i] = std::min(slab, kpad - i * slab);
    }
    const int npt = (nao + tile - 1) / tile;
    nqt1 = (nri + tile - 1) / tile;
    nqt2 = (nao + tile - 1) / tile;
    n_tiles1 = npt * nqt1;
    n_tiles2 = npt * nqt2;
    auto lists = [&](int nt, DevBuf& tl, DevBuf& tk, DevBuf& ct) -> int {
      std::vector<int> h_tl(nt), h_tk((size_t)nt * nslab), h_ct(nt, nslab);
      for (int t = 0; t < nt; ++t) {
        h_tl[t] = t;
        for (int i = 0; i < nslab; ++i) h_tk[(size_t)t * nslab + i] = i;
      }
      SG_TRY(cudaMalloc(&tl.p, nt * sizeof(int)));
      SG_TRY(cudaMalloc(&tk.p, h_tk.size() * sizeof(int)));
      SG_TRY(cudaMalloc(&ct.p, nt * sizeof(int)));
      SG_TRY(cudaMemcpy(tl.p, h_tl.data(), nt * sizeof(int), cudaMemcpyHostToDevice));
      SG_TRY(cudaMemcpy(tk.p, h_tk.data(), h_tk.size() * sizeof(int), cudaMemcpyHostToDevice));
      SG_TRY(cudaMemcpy(ct.p, h_ct.data(), nt * sizeof(int), cudaMemcpyHostToDevice));
      return GW_OK;
    };
    if ((rc = lists(n_tiles1, b_tl1, b_tk1, b_ct1))) return rc;
    if ((rc = lists(n_tiles2, b_tl2, b_tk2, b_ct2))) return rc;
    SG_TRY(cudaMalloc(&b_k01.p, nslab * sizeof(long long)));
    SG_TRY(cudaMalloc(&b_ln1.p, nslab * sizeof(int)));
    SG_TRY(cudaMemcpy(b_k01.p, k0.data(), nslab * sizeof(long long), cudaMemcpyHostToDevice));
    SG_TRY(cudaMemcpy(b_ln1.p, len.data(), nslab * sizeof(int), cudaMemcpyHostToDevice));
    SG_TRY(cudaMalloc(&b_bs.p, (size_t)slices * nao * kpad * 2));
    SG_TRY(cudaMalloc(&b_ws.p, (size_t)slices * nri * kpad * 2));
    SG_TRY(cudaMalloc(&b_ys.p, (size_t)slices * nao * kpad * 2));
    SG_TRY(cudaMalloc(&b_err.p, sizeof(int)));
    SG_TRY(cudaMalloc(&b_mx.p, 4 * sizeof(double)));
    SG_TRY(cudaMemsetAsync(b_err.p, 0, sizeof(int), st));
    if (gw::make_slice_map(&m_b, b_bs.p, kpad, nao, slices, tile, f16) ||
        gw::make_slice_map(&m_w, b_ws.p, kpad, nri, slices, tile, f16) ||
        gw::make_slice_map(&m_y, b_ys.p, kpad, nao, slices, tile, f16)) {
      ctx->err = "gw_sigma_tau: cuTensorMapEncodeTiled failed";
      return GW_ERR_CUDA;
    }
    m_bq = m_b;
  }
  for (int jt = 0; jt < n_tau; ++jt) {
    gw::launch_greens(ctx->d_C, ctx->d_eps, nao, ctx->n_occ, ctx->mu, taus[jt], (double*)b_cso.p,
                      (double*)b_csv.p, go, gv, st);
    if (thr > 0.0) {
      gw::launch_sym_block_filter(go, nao, ctx->d_ao_off, n_at, thr, (unsigned char*)b_fl.p, st);
      gw::launch_sym_block_filter(gv, nao, ctx->d_ao_off, n_at, thr, (unsigned char*)b_fl.p, st);
    }
    const double* wt = w + (size_t)jt * nn_ri;
    for (int a = 0; a < n_orb; ++a) {
      const double* b = bn + (size_t)a * nao * nri;
      if (!mixed) {
        gw::chain_dgemm(false, false, nao, nri, nri, 1.0, b, nri, wt, nri, 0.0, y, nri, st);  // Y = B W
        gw::chain_dgemm(false, true, nao, nao, nri, 1.0, y, nri, b, nri, 0.0, z, nao, st);    // Z = Y B^T
      } else {
        // binary16 scales: max |B|, max |W| and the bound |B W| <= max_mu
        // sum_P |B[mu][P]| * max |W| (all 1 for bf16 slices)
        double s_b = 1.0, s_w = 1.0, s_y = 1.0;
        if (f16) {
          double h[4];
          gw::launch_absmax_rowsum(b, nri, nao, nri, (double*)b_mx.p, st);
          gw::launch_absmax_rowsum(wt, nri, nri, nri, (double*)b_mx.p + 2, st);
          SG_TRY(cudaGetLastError());
          SG_TRY(cudaMemcpyAsync(h, b_mx.p, sizeof(h), cudaMemcpyDeviceToHost, st));
          SG_TRY(cudaStreamSynchronize(st));
          s_b = gw::pow2_scale(h[0]);
          s_w = gw::pow2_scale(h[2]);
          s_y = gw::pow2_scale(h[1] * h[2]);
        }
        gw::launch_split_f64(b, nri, nao, nri, kpad, slices, f16, s_b, b_bs.p, st);
        gw::launch_split_f64(wt, nri, nri, nri, kpad, slices, f16, s_w, b_ws.p, st);
        SG_TRY(cudaMemsetAsync(y, 0, (size_t)nao * nri * 8, st));
        if (gw::launch_chi_tc(slices, f16, (float)(1.0 / (s_b * s_w)), m_b, m_w, (const int*)b_tl1.p,
                              n_tiles1, (const int*)b_tk1.p,
                              (const int*)b_ct1.p, nslab, (const long long*)b_k01.p,
                              (const int*)b_ln1.p, 0, nao, nri, 0, nri, nqt1, y, ctx->flush_k,
                              (int*)b_err.p, st)) {
          ctx->err = "gw_sigma_tau: tensor-core launch setup failed";
          return GW_ERR_CUDA;
        }
        // y holds -(B W); its slices are the row operand of the second product
        gw::launch_split_f64(y, nri, nao, nri, kpad, slices, f16, s_y, b_ys.p, st);
        SG_TRY(cudaMemsetAsync(z, 0, nn_ao * 8, st));
        if (gw::launch_chi_tc(slices, f16, (float)(1.0 / (s_y * s_b)), m_y, m_bq, (const int*)b_tl2.p,
                              n_tiles2, (const int*)b_tk2.p,
                              (const int*)b_ct2.p, nslab, (const long long*)b_k01.p,
                              (const int*)b_ln1.p, 0, nao, nao, 0, nao, nqt2, z, ctx->flush_k,
                              (int*)b_err.p, st)) {
          ctx->err = "gw_sigma_tau: tensor-core launch setup failed";
          return GW_ERR_CUDA;
        }
        SG_TRY(cudaGetLastError());
      }
      gw::sigma::k_dot2<<<kDotBlocks, 256, 0, st>>>(go, gv, z, (long long)nn_ao, (double*)b_part.p);
      SG_TRY(cudaGetLastError());
      SG_TRY(cudaMemcpyAsync(part.data(), b_part.p, part.size() * 8, cudaMemcpyDeviceToHost, st));
      SG_TRY(cudaStreamSynchronize(st));
      double so = 0.0, sv = 0.0;
      for (int bl = 0; bl < kDotBlocks; ++bl) {
        so += part[2 * bl];
        sv += part[2 * bl + 1];
      }
      sigma_out[((size_t)a * n_tau + jt) * 2 + 0] = -so;
      sigma_out[((size_t)a * n_tau + jt) * 2 + 1] = sv;
    }
  }
  if (mixed) {
    int h_err = 0;
    SG_TRY(cudaMemcpy(&h_err, b_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h_err) {
      ctx->err = "gw_sigma_tau: a bounded wait of the tensor-core kernel gave up";
      return GW_ERR_TIMEOUT;
    }
  }
  return GW_OK;
}
}  // namespace

extern "C" int gw_sigma_tau(gw_ctx* ctx, const double* W_tau, int w_on_device, const int* orbitals,
                            int n_orb, double thr, int precision, double* sigma_out) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_sigma_tau");
  ctx->err.clear();
  if (!ctx->have_greens) {
    ctx->err = "gw_sigma_tau: call gw_set_basis, gw_set_3c_tensor and gw_set_greens first";
    return GW_ERR_ORDER;
  }
  return sigma_impl(ctx, W_tau, w_on_device, orbitals, n_orb, thr, precision, ctx->tau.data(),
                    (int)ctx->tau.size(), sigma_out);
}

// Eq. 11 is Eq. 10's contraction with W = V at tau = 0, where G^occ(0) is the
// density matrix D = C_occ C_occ^T: Sigma^x_n = -S^occ_n.
extern "C" int gw_sigma_x(gw_ctx* ctx, const double* V, int v_on_device, const int* orbitals,
                          int n_orb, double thr, int precision, double* sx_out) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_sigma_x");
  ctx->err.clear();
  if (!ctx->have_greens) {
    ctx->err = "gw_sigma_x: call gw_set_basis, gw_set_3c_tensor and gw_set_greens first";
    return GW_ERR_ORDER;
  }
  if (!sx_out || n_orb <= 0 || n_orb > 1024) {
    ctx->err = "gw_sigma_x: bad arguments";
    return GW_ERR_INVALID_ARG;
  }
  const double tau0 = 0.0;
  std::vector<double> tmp((size_t)n_orb * 2);
  const int rc = sigma_impl(ctx, V, v_on_device, orbitals, n_orb, thr, precision, &tau0, 1, tmp.data());
  if (rc) return rc;
  for (int a = 0; a < n_orb; ++a) sx_out[a] = tmp[(size_t)a * 2];
  return GW_OK;
}
