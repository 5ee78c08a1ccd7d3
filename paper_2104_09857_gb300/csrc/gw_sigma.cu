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

// ===========================================================================
// batched self-energy: many molecules, one grouped launch per product
// ===========================================================================
namespace gw {
namespace sigma {

// partial[(p * kDotBlocks + b) * 2 + 0..1] = block b's part of
// (sum G^occ * Z_p, sum G^virt * Z_p) over problem p's n elements
struct DotDesc {
  long long g_off, z_off, n;
};
__global__ void k_dot2_group(const double* __restrict__ go, const double* __restrict__ gv,
                             const double* __restrict__ z, const DotDesc* __restrict__ desc,
                             double* __restrict__ partial) {
  __shared__ double s0[256], s1[256];
  const DotDesc d = desc[blockIdx.y];
  double a = 0.0, b = 0.0;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < d.n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const double zz = z[d.z_off + i];
    a = fma(go[d.g_off + i], zz, a);
    b = fma(gv[d.g_off + i], zz, b);
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
    double* o = partial + (static_cast<long long>(blockIdx.y) * gridDim.x + blockIdx.x) * 2;
    o[0] = s0[0];
    o[1] = s1[0];
  }
}

}  // namespace sigma
}  // namespace gw

namespace {

#define SB_TRY(call)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      c0->err = std::string("gw_sigma_tau_batch: ") + #call + ": " + cudaGetErrorString(e_); \
      return e_ == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA;                     \
    }                                                                                        \
  } while (0)

struct Prob {
  int mol, a, nao, nri;
  long long rowB;  // first slice row of B_p (and of Y_p)
  long long offY, offZ;
};

int sigma_batch_mixed(gw_ctx* const* ctxs, int n_mol, const double* const* W_tau, int w_on_device,
                      const int* const* orbitals, const int* n_orb, double thr, int precision,
                      double* const* sigma_out) {
  gw_ctx* c0 = ctxs[0];
  cudaStream_t st = c0->stream;
  const int slices = precision == GW_BF16X6 ? 3 : 2;
  const int f16 = precision == GW_FP16X3;
  const int n_tau = (int)c0->tau.size();
  const int tile = gw::tc_tile_rows();
  // problems (molecule, orbital) and the buffers' layout
  std::vector<Prob> pr;
  std::vector<long long> offB64(n_mol), offW(n_mol), offG(n_mol), offWrow(n_mol);
  long long nB64 = 0, nW = 0, nG = 0, rowsB = 0, rowsW = 0, nY = 0, nZ = 0;
  int kmax = 64, max_nao = 1, max_nri = 1, max_occ = 1, max_virt = 1;
  for (int i = 0; i < n_mol; ++i) {
    const gw_ctx* c = ctxs[i];
    offB64[i] = nB64;
    offW[i] = nW;
    offG[i] = nG;
    offWrow[i] = rowsW;
    nB64 += (long long)n_orb[i] * c->nao * c->nri;
    nW += (long long)c->nri * c->nri;
    nG += (long long)c->nao * c->nao;
    rowsW += c->nri;
    kmax = std::max(kmax, (c->nri + 63) / 64 * 64);
    max_nao = std::max(max_nao, c->nao);
    max_nri = std::max(max_nri, c->nri);
    max_occ = std::max(max_occ, c->n_occ);
    max_virt = std::max(max_virt, c->nao - c->n_occ);
    for (int a = 0; a < n_orb[i]; ++a) {
      Prob p{i, a, c->nao, c->nri, rowsB, nY, nZ};
      rowsB += c->nao;
      nY += (long long)c->nao * c->nri;
      nZ += (long long)c->nao * c->nao;
      pr.push_back(p);
    }
  }
  const int np = (int)pr.size();
  DevBuf b_bn, b_csel, b_bs, b_ws, b_ys, b_w64, b_y64, b_z64, b_go, b_gv, b_cso, b_csv, b_fl, b_mx,
      b_sd, b_t1, b_t2, b_dd, b_part, b_err, b_pd, b_own;
  SB_TRY(cudaMalloc(&b_bn.p, std::max<long long>(nB64, 1) * 8));
  SB_TRY(cudaMemsetAsync(b_bn.p, 0, std::max<long long>(nB64, 1) * 8, st));
  double* bn = (double*)b_bn.p;
  // B^n of every molecule from its FP64 panels (built and released one
  // molecule at a time, so that one pool is resident at once)
  for (int i = 0; i < n_mol; ++i) {
    gw_ctx* c = ctxs[i];
    int rc = gw::build_panels_for(c, thr);
    if (rc) {
      c0->err = "gw_sigma_tau_batch: molecule " + std::to_string(i) + ": " + c->err;
      return rc;
    }
    DevBuf csel;
    SB_TRY(cudaMalloc(&csel.p, (size_t)c->nao * n_orb[i] * 8));
    for (int a = 0; a < n_orb[i]; ++a)
      SB_TRY(cudaMemcpy2DAsync((double*)csel.p + a, n_orb[i] * 8, c->d_C + orbitals[i][a], c->nao * 8, 8,
                               c->nao, cudaMemcpyDeviceToDevice, st));
    std::vector<int> owners;
    int maxN = 0;
    for (int s = 0; s < c->n_at; ++s)
      if (c->panels[s].K > 0) {
        owners.push_back(s);
        maxN = std::max(maxN, c->panels[s].npw * c->panels[s].nsig);
      }
    DevBuf pd, own;
    SB_TRY(cudaMalloc(&pd.p, c->panels.size() * sizeof(gw::PanelDesc)));
    SB_TRY(cudaMemcpyAsync(pd.p, c->panels.data(), c->panels.size() * sizeof(gw::PanelDesc),
                           cudaMemcpyHostToDevice, st));
    SB_TRY(cudaMalloc(&own.p, std::max<size_t>(owners.size(), 1) * sizeof(int)));
    if (!owners.empty()) {
      SB_TRY(cudaMemcpyAsync(own.p, owners.data(), owners.size() * sizeof(int), cudaMemcpyHostToDevice, st));
      dim3 g((maxN + 127) / 128, (unsigned)owners.size(), n_orb[i]);
      gw::sigma::k_bn_panels<<<g, 128, 0, st>>>(c->d_panel64, (const gw::PanelDesc*)pd.p,
                                                (const int*)own.p, c->d_lam, c->d_ao_off,
                                                (const double*)csel.p, n_orb[i], c->nao, c->nri,
                                                bn + offB64[i]);
      SB_TRY(cudaGetLastError());
    }
    if (thr > 0.0) {
      const long long nblk = (long long)n_orb[i] * c->n_at * c->n_at;
      gw::sigma::k_bn_filter<<<(unsigned)((nblk + 7) / 8), 256, 0, st>>>(bn + offB64[i], n_orb[i], c->n_at,
                                                                         c->nao, c->nri, c->d_ao_off,
                                                                         c->d_ri_off, thr);
      SB_TRY(cudaGetLastError());
    }
    SB_TRY(cudaStreamSynchronize(st));
    // the pool is not needed again here: release it
    cudaFree(c->d_panel64);
    c->d_panel64 = nullptr;
    c->panels_ok = false;
    c->panels_thr = -1.0;
    c->panel32_ok = false;
  }
  // slices of B (tau independent) with per-problem binary16 scales
  std::vector<gw::SplitDesc> sd(np);
  for (int p = 0; p < np; ++p) {
    const Prob& q = pr[p];
    sd[p] = gw::SplitDesc{offB64[q.mol] + (long long)q.a * q.nao * q.nri, q.rowB, q.nao, q.nri, q.nri, 0, 1.0};
  }
  SB_TRY(cudaMalloc(&b_sd.p, std::max(np, n_mol) * sizeof(gw::SplitDesc)));
  SB_TRY(cudaMalloc(&b_mx.p, 2 * std::max(np, n_mol) * sizeof(double)));
  std::vector<double> bmx(2 * np, 1.0);
  if (f16) {
    SB_TRY(cudaMemcpyAsync(b_sd.p, sd.data(), np * sizeof(gw::SplitDesc), cudaMemcpyHostToDevice, st));
    gw::launch_absmax_group(bn, (const gw::SplitDesc*)b_sd.p, np, max_nao, (double*)b_mx.p, st);
    SB_TRY(cudaGetLastError());
    SB_TRY(cudaMemcpyAsync(bmx.data(), b_mx.p, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, st));
    SB_TRY(cudaStreamSynchronize(st));
  }
  std::vector<double> s_b(np, 1.0);
  for (int p = 0; p < np; ++p) {
    if (f16) s_b[p] = gw::pow2_scale(bmx[2 * p]);
    sd[p].scale = s_b[p];
  }
  SB_TRY(cudaMemcpyAsync(b_sd.p, sd.data(), np * sizeof(gw::SplitDesc), cudaMemcpyHostToDevice, st));
  const long long bs_elems = std::max<long long>(rowsB, 1) * kmax;
  SB_TRY(cudaMalloc(&b_bs.p, (size_t)slices * bs_elems * 2));
  SB_TRY(cudaMalloc(&b_ys.p, (size_t)slices * bs_elems * 2));
  gw::launch_split_group(bn, (const gw::SplitDesc*)b_sd.p, np, max_nao, kmax, slices, bs_elems, f16, b_bs.p, st);
  SB_TRY(cudaGetLastError());
  const long long ws_elems = std::max<long long>(rowsW, 1) * kmax;
  SB_TRY(cudaMalloc(&b_ws.p, (size_t)slices * ws_elems * 2));
  SB_TRY(cudaMalloc(&b_y64.p, std::max<long long>(nY, 1) * 8));
  SB_TRY(cudaMalloc(&b_z64.p, std::max<long long>(nZ, 1) * 8));
  SB_TRY(cudaMalloc(&b_go.p, std::max<long long>(nG, 1) * 8));
  SB_TRY(cudaMalloc(&b_gv.p, std::max<long long>(nG, 1) * 8));
  SB_TRY(cudaMalloc(&b_cso.p, (size_t)max_nao * max_occ * 8));
  SB_TRY(cudaMalloc(&b_csv.p, (size_t)max_nao * max_virt * 8));
  SB_TRY(cudaMalloc(&b_err.p, sizeof(int)));
  SB_TRY(cudaMemsetAsync(b_err.p, 0, sizeof(int), st));
  if (!w_on_device) SB_TRY(cudaMalloc(&b_w64.p, std::max<long long>(nW, 1) * 8));
  int max_at = 1;
  for (int i = 0; i < n_mol; ++i) max_at = std::max(max_at, ctxs[i]->n_at);
  SB_TRY(cudaMalloc(&b_fl.p, (size_t)max_at * max_at));
  CUtensorMap m_b, m_w, m_y;
  if (gw::make_slice_map(&m_b, b_bs.p, kmax, std::max<long long>(rowsB, 1), slices, tile, f16) ||
      gw::make_slice_map(&m_w, b_ws.p, kmax, std::max<long long>(rowsW, 1), slices, tile, f16) ||
      gw::make_slice_map(&m_y, b_ys.p, kmax, std::max<long long>(rowsB, 1), slices, tile, f16)) {
    c0->err = "gw_sigma_tau_batch: cuTensorMapEncodeTiled failed";
    return GW_ERR_CUDA;
  }
  // dot descriptors and tiles of the two grouped products
  std::vector<gw::sigma::DotDesc> dd(np);
  for (int p = 0; p < np; ++p)
    dd[p] = gw::sigma::DotDesc{offG[pr[p].mol], pr[p].offZ, (long long)pr[p].nao * pr[p].nao};
  SB_TRY(cudaMalloc(&b_dd.p, np * sizeof(gw::sigma::DotDesc)));
  SB_TRY(cudaMemcpyAsync(b_dd.p, dd.data(), np * sizeof(gw::sigma::DotDesc), cudaMemcpyHostToDevice, st));
  SB_TRY(cudaMalloc(&b_part.p, (size_t)np * kDotBlocks * 2 * 8));
  std::vector<double> part((size_t)np * kDotBlocks * 2);
  std::vector<gw::GroupTile> t1, t2;
  for (const Prob& q : pr) {
    for (int mt = 0; mt * tile < q.nao; ++mt)
      for (int nt = 0; nt * tile < q.nri; ++nt)
        t1.push_back(gw::GroupTile{q.offY + (long long)mt * tile * q.nri + nt * tile, (int)(q.rowB + mt * tile),
                                   (int)(offWrow[q.mol] + nt * tile), (q.nri + 63) / 64,
                                   std::min(tile, q.nao - mt * tile), std::min(tile, q.nri - nt * tile), q.nri,
                                   1.f, 0});
    for (int mt = 0; mt * tile < q.nao; ++mt)
      for (int nt = 0; nt * tile < q.nao; ++nt)
        t2.push_back(gw::GroupTile{q.offZ + (long long)mt * tile * q.nao + nt * tile, (int)(q.rowB + mt * tile),
                                   (int)(q.rowB + nt * tile), (q.nri + 63) / 64,
                                   std::min(tile, q.nao - mt * tile), std::min(tile, q.nao - nt * tile), q.nao,
                                   1.f, 0});
  }
  SB_TRY(cudaMalloc(&b_t1.p, std::max<size_t>(t1.size(), 1) * sizeof(gw::GroupTile)));
  SB_TRY(cudaMalloc(&b_t2.p, std::max<size_t>(t2.size(), 1) * sizeof(gw::GroupTile)));
  std::vector<gw::SplitDesc> wd(n_mol), yd(np);
  for (int j = 0; j < n_tau; ++j) {
    // W(tau_j) of every molecule: magnitudes, then slices
    const double* w64 = nullptr;
    if (w_on_device) {
      // one contiguous view is needed: copy the molecules' matrices together
      if (!b_w64.p) SB_TRY(cudaMalloc(&b_w64.p, std::max<long long>(nW, 1) * 8));
      for (int i = 0; i < n_mol; ++i)
        SB_TRY(cudaMemcpyAsync((double*)b_w64.p + offW[i], W_tau[i] + (size_t)j * ctxs[i]->nri * ctxs[i]->nri,
                               (size_t)ctxs[i]->nri * ctxs[i]->nri * 8, cudaMemcpyDeviceToDevice, st));
    } else {
      for (int i = 0; i < n_mol; ++i)
        SB_TRY(cudaMemcpyAsync((double*)b_w64.p + offW[i], W_tau[i] + (size_t)j * ctxs[i]->nri * ctxs[i]->nri,
                               (size_t)ctxs[i]->nri * ctxs[i]->nri * 8, cudaMemcpyHostToDevice, st));
    }
    w64 = (const double*)b_w64.p;
    for (int i = 0; i < n_mol; ++i)
      wd[i] = gw::SplitDesc{offW[i], offWrow[i], ctxs[i]->nri, ctxs[i]->nri, ctxs[i]->nri, 0, 1.0};
    std::vector<double> wmx(2 * n_mol, 1.0);
    if (f16) {
      SB_TRY(cudaMemcpyAsync(b_sd.p, wd.data(), n_mol * sizeof(gw::SplitDesc), cudaMemcpyHostToDevice, st));
      gw::launch_absmax_group(w64, (const gw::SplitDesc*)b_sd.p, n_mol, max_nri, (double*)b_mx.p, st);
      SB_TRY(cudaGetLastError());
      SB_TRY(cudaMemcpyAsync(wmx.data(), b_mx.p, 2 * n_mol * sizeof(double), cudaMemcpyDeviceToHost, st));
      SB_TRY(cudaStreamSynchronize(st));
    }
    std::vector<double> s_w(n_mol, 1.0);
    for (int i = 0; i < n_mol; ++i) {
      if (f16) s_w[i] = gw::pow2_scale(wmx[2 * i]);
      wd[i].scale = s_w[i];
    }
    SB_TRY(cudaMemcpyAsync(b_sd.p, wd.data(), n_mol * sizeof(gw::SplitDesc), cudaMemcpyHostToDevice, st));
    gw::launch_split_group(w64, (const gw::SplitDesc*)b_sd.p, n_mol, max_nri, kmax, slices, ws_elems, f16,
                           b_ws.p, st);
    SB_TRY(cudaGetLastError());
    // product 1, every problem in one launch: Y_p = -(B_p W)
    size_t k = 0;
    for (int p = 0; p < np; ++p) {
      const Prob& q = pr[p];
      const float sc = (float)(1.0 / (s_b[p] * s_w[q.mol]));
      for (int mt = 0; mt * tile < q.nao; ++mt)
        for (int nt = 0; nt * tile < q.nri; ++nt) t1[k++].scale = sc;
    }
    SB_TRY(cudaMemcpyAsync(b_t1.p, t1.data(), t1.size() * sizeof(gw::GroupTile), cudaMemcpyHostToDevice, st));
    SB_TRY(cudaMemsetAsync(b_y64.p, 0, std::max<long long>(nY, 1) * 8, st));
    if (gw::launch_group_tc(slices, f16, m_b, m_w, (const gw::GroupTile*)b_t1.p, (int)t1.size(),
                            (double*)b_y64.p, c0->flush_k, (int*)b_err.p, st)) {
      c0->err = "gw_sigma_tau_batch: tensor-core launch setup failed";
      return GW_ERR_CUDA;
    }
    SB_TRY(cudaGetLastError());
    // Y slices with the bound |B W| <= max_mu sum_P |B[mu][P]| * max |W|
    std::vector<double> s_y(np, 1.0);
    for (int p = 0; p < np; ++p) {
      if (f16) s_y[p] = gw::pow2_scale(bmx[2 * p + 1] * wmx[2 * pr[p].mol]);
      yd[p] = gw::SplitDesc{pr[p].offY, pr[p].rowB, pr[p].nao, pr[p].nri, pr[p].nri, 0, s_y[p]};
    }
    SB_TRY(cudaMemcpyAsync(b_sd.p, yd.data(), np * sizeof(gw::SplitDesc), cudaMemcpyHostToDevice, st));
    gw::launch_split_group((const double*)b_y64.p, (const gw::SplitDesc*)b_sd.p, np, max_nao, kmax, slices,
                           bs_elems, f16, b_ys.p, st);
    SB_TRY(cudaGetLastError());
    // product 2: Z_p = -(Y_p B_p^T) = B_p W B_p^T
    k = 0;
    for (int p = 0; p < np; ++p) {
      const Prob& q = pr[p];
      const float sc = (float)(1.0 / (s_y[p] * s_b[p]));
      for (int mt = 0; mt * tile < q.nao; ++mt)
        for (int nt = 0; nt * tile < q.nao; ++nt) t2[k++].scale = sc;
    }
    SB_TRY(cudaMemcpyAsync(b_t2.p, t2.data(), t2.size() * sizeof(gw::GroupTile), cudaMemcpyHostToDevice, st));
    SB_TRY(cudaMemsetAsync(b_z64.p, 0, std::max<long long>(nZ, 1) * 8, st));
    if (gw::launch_group_tc(slices, f16, m_y, m_b, (const gw::GroupTile*)b_t2.p, (int)t2.size(),
                            (double*)b_z64.p, c0->flush_k, (int*)b_err.p, st)) {
      c0->err = "gw_sigma_tau_batch: tensor-core launch setup failed";
      return GW_ERR_CUDA;
    }
    SB_TRY(cudaGetLastError());
    // Green's functions of every molecule at its tau_j (FP64, filtered)
    for (int i = 0; i < n_mol; ++i) {
      const gw_ctx* c = ctxs[i];
      gw::launch_greens(c->d_C, c->d_eps, c->nao, c->n_occ, c->mu, c->tau[j], (double*)b_cso.p,
                        (double*)b_csv.p, (double*)b_go.p + offG[i], (double*)b_gv.p + offG[i], st);
      if (thr > 0.0) {
        gw::launch_sym_block_filter((double*)b_go.p + offG[i], c->nao, c->d_ao_off, c->n_at, thr,
                                    (unsigned char*)b_fl.p, st);
        gw::launch_sym_block_filter((double*)b_gv.p + offG[i], c->nao, c->d_ao_off, c->n_at, thr,
                                    (unsigned char*)b_fl.p, st);
      }
    }
    SB_TRY(cudaGetLastError());
    gw::sigma::k_dot2_group<<<dim3(kDotBlocks, np), 256, 0, st>>>((const double*)b_go.p, (const double*)b_gv.p,
                                                                  (const double*)b_z64.p,
                                                                  (const gw::sigma::DotDesc*)b_dd.p,
                                                                  (double*)b_part.p);
    SB_TRY(cudaGetLastError());
    SB_TRY(cudaMemcpyAsync(part.data(), b_part.p, part.size() * 8, cudaMemcpyDeviceToHost, st));
    SB_TRY(cudaStreamSynchronize(st));
    for (int p = 0; p < np; ++p) {
      double so = 0.0, sv = 0.0;
      for (int bl = 0; bl < kDotBlocks; ++bl) {
        so += part[((size_t)p * kDotBlocks + bl) * 2];
        sv += part[((size_t)p * kDotBlocks + bl) * 2 + 1];
      }
      double* o = sigma_out[pr[p].mol] + ((size_t)pr[p].a * n_tau + j) * 2;
      o[0] = -so;
      o[1] = sv;
    }
  }
  int h_err = 0;
  SB_TRY(cudaMemcpy(&h_err, b_err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h_err) {
    c0->err = "gw_sigma_tau_batch: a bounded wait of the tensor-core kernel gave up";
    return GW_ERR_TIMEOUT;
  }
  return GW_OK;
}
#undef SB_TRY

}  // namespace

extern "C" int gw_sigma_tau_batch(gw_ctx* const* ctxs, int n_mol, const double* const* W_tau, int w_on_device,
                                  const int* const* orbitals, const int* n_orb, double thr, int precision,
                                  double* const* sigma_out) {
  if (!ctxs || n_mol <= 0 || !ctxs[0]) return GW_ERR_INVALID_ARG;
  gw_ctx* c0 = ctxs[0];
  gw::TraceRange trace("gw_sigma_tau_batch");
  c0->err.clear();
  if (!W_tau || !orbitals || !n_orb || !sigma_out || !(thr >= 0.0) || !std::isfinite(thr)) {
    c0->err = "gw_sigma_tau_batch: bad arguments";
    return GW_ERR_INVALID_ARG;
  }
  if (precision != GW_FP64 && precision != GW_BF16X3 && precision != GW_BF16X6 && precision != GW_FP16X3) {
    c0->err = "gw_sigma_tau_batch: precision must be GW_FP64, GW_BF16X3, GW_BF16X6 or GW_FP16X3";
    return GW_ERR_UNSUPPORTED;
  }
  for (int i = 0; i < n_mol; ++i) {
    const gw_ctx* c = ctxs[i];
    if (!c || !W_tau[i] || !orbitals[i] || !sigma_out[i] || n_orb[i] <= 0 || n_orb[i] > 1024) {
      c0->err = "gw_sigma_tau_batch: bad arguments for molecule " + std::to_string(i);
      return GW_ERR_INVALID_ARG;
    }
    if (c->n_at == 0 || c->blk_off.empty() || !c->have_greens) {
      c0->err = "gw_sigma_tau_batch: molecule " + std::to_string(i) +
                ": call gw_set_basis, gw_set_3c_tensor and gw_set_greens first";
      return GW_ERR_ORDER;
    }
    if (c->device != c0->device || c->tau.size() != c0->tau.size()) {
      c0->err = "gw_sigma_tau_batch: every context must be on the same device and have as many tau points";
      return GW_ERR_INVALID_ARG;
    }
    for (int a = 0; a < n_orb[i]; ++a)
      if (orbitals[i][a] < 0 || orbitals[i][a] >= c->nao) {
        c0->err = "gw_sigma_tau_batch: orbital index out of range (molecule " + std::to_string(i) + ")";
        return GW_ERR_INVALID_ARG;
      }
  }
  if (cudaSetDevice(c0->device) != cudaSuccess) return GW_ERR_CUDA;
  if (precision == GW_FP64) {
    // the plain FP64 form, one molecule at a time
    for (int i = 0; i < n_mol; ++i) {
      gw_ctx* c = ctxs[i];
      c->err.clear();
      const int rc = sigma_impl(c, W_tau[i], w_on_device, orbitals[i], n_orb[i], thr, precision,
                                c->tau.data(), (int)c->tau.size(), sigma_out[i]);
      if (rc) {
        c0->err = "gw_sigma_tau_batch: molecule " + std::to_string(i) + ": " + c->err;
        return rc;
      }
    }
    return GW_OK;
  }
  return sigma_batch_mixed(ctxs, n_mol, W_tau, w_on_device, orbitals, n_orb, thr, precision, sigma_out);
}
