// C ABI of libgwchi and the host-side orchestration of the chi(i tau) path.
//
// Per tau point (Eq. 2, Eq. 3):
//   1. G^occ(tau), G^virt(tau) = scaled orbital products (FP64), block filter.
//   2. For each batch of sigma-atoms (owners of 3c panels):
//        step A  X[P][(s, mu, s')] = sum_l G^occ[mu][l] T[l, s', P]    (M of Eq. 3)
//        step B  Y[Q][(s, mu, s')] = sum_l G^virt[s'][l] T[l, mu, Q]   (N of Eq. 3)
//        block filter of X and Y, slab/tile occupancy, per-tile task lists
//        step C  chi[P][Q] -= sum_k X[P][k] Y[Q][k]   over surviving slabs
//   3. mirror the atom-block upper triangle, write chi(tau).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "gw_internal.h"
#include "k_simt.h"
#include "k_tc.h"
#include "k_mlp.h"

using gw::Batch;
using gw::kSlabAO;
using gw::PanelDesc;
using gw::PanelTask;

namespace {


#define GW_TRY(call)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
      return e_ == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA;              \
    }                                                                                 \
  } while (0)

#define GW_CHECK_LAUNCH()                                                             \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess) {                                                          \
      ctx->err = std::string("kernel launch: ") + cudaGetErrorString(e_);             \
      return GW_ERR_CUDA;                                                             \
    }                                                                                 \
  } while (0)

int fail(gw_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

// named device scratch buffer, grown on demand
int ws(gw_ctx* ctx, const char* name, size_t bytes, void** out) {
  auto& wb = ctx->work;
  auto it = wb.find(name);
  if (it != wb.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return GW_OK;
  }
  if (it != wb.end()) {
    cudaFree(it->second.first);
    wb.erase(it);
  }
  void* p = nullptr;
  if (bytes > 0 && ctx->test_fail_alloc) {
    ctx->test_fail_alloc = 0;
    ctx->err = std::string("cudaMalloc of work buffer '") + name + "' (" + std::to_string(bytes) +
               " bytes): injected failure (option test_fail_alloc)";
    return GW_ERR_OOM;
  }
  if (bytes > 0) {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->err = std::string("cudaMalloc of work buffer '") + name + "' (" +
                 std::to_string(bytes) + " bytes): " + cudaGetErrorString(e);
      return GW_ERR_OOM;
    }
  }
  wb[name] = {p, bytes};
  *out = p;
  return GW_OK;
}

// release every scratch buffer of a context (before a route with different
// buffer sizes, so that two routes' operands are never resident together)
void ws_release_all(gw_ctx* ctx) {
  auto& wb = ctx->work;
  ctx->ptB_m0 = ctx->ptB_m1 = -1;  // a streamed panel region lives in a work buffer
  if (wb.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : wb) cudaFree(kv.second.first);
  wb.clear();
}

template <typename T>
int wsT(gw_ctx* ctx, const char* name, size_t count, T** out) {
  void* p = nullptr;
  int rc = ws(ctx, name, count * sizeof(T), &p);
  *out = static_cast<T*>(p);
  return rc;
}

template <typename T>
int upload(gw_ctx* ctx, const char* name, const std::vector<T>& v, T** out) {
  int rc = wsT<T>(ctx, name, std::max<size_t>(v.size(), 1), out);
  if (rc) return rc;
  if (!v.empty())
    GW_TRY(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                           ctx->stream));
  return GW_OK;
}

void free_dev(void* p) {
  if (p) cudaFree(p);
}

void reset_tensor(gw_ctx* ctx) {
  free_dev(ctx->d_t3);
  free_dev(ctx->d_t3f);
  ctx->d_t3f = nullptr;
  free_dev(ctx->d_blk);
  free_dev(ctx->d_blk_off);
  free_dev(ctx->d_blk_norm);
  free_dev(ctx->d_panel64);
  free_dev(ctx->d_panel32);
  free_dev(ctx->d_lam);
  ctx->d_t3 = nullptr;
  ctx->d_blk = nullptr;
  ctx->d_blk_off = nullptr;
  ctx->d_blk_norm = nullptr;
  ctx->d_panel64 = nullptr;
  ctx->d_panel32 = nullptr;
  ctx->d_lam = nullptr;
  ctx->n_blocks = ctx->n_elems = 0;
  ctx->blk.clear();
  ctx->blk_off.clear();
  ctx->blk_norm.clear();
  ctx->plan_ok = false;
  ctx->panels_ok = false;
  ctx->panel32_ok = false;
  free_dev(ctx->d_pt);
  ctx->d_pt = nullptr;
  ctx->pt_ok = false;
  ctx->ycov_valid = false;
}

void reset_greens(gw_ctx* ctx) {
  free_dev(ctx->d_C);
  free_dev(ctx->d_eps);
  ctx->d_C = ctx->d_eps = nullptr;
  ctx->have_greens = false;
  ctx->tau.clear();
  ctx->h_eps.clear();
}

struct Timer {
  cudaEvent_t a, b;
};

// ---------------------------------------------------------------------------
// panels
// ---------------------------------------------------------------------------
// Host plan of the owner panels for threshold thr: which 3c blocks survive
// the filter, each owner's lambda atoms and RI window, and where each kept
// block lands in the two panels it belongs to.  Uploads the lambda lists.
int plan_panels(gw_ctx* ctx, double thr) {
  if (ctx->plan_ok && ctx->plan_thr == thr) return GW_OK;
  // everything derived from an earlier plan stops being valid here: an
  // allocation or copy below may fail and leave it half built
  ctx->plan_ok = false;
  ctx->plan_thr = -1.0;
  ctx->panels_ok = false;
  ctx->panels_thr = -1.0;
  ctx->pt_ok = false;
  ctx->panel32_ok = false;
  ctx->ycov_valid = false;
  const int n = ctx->n_at;
  std::vector<int>& kept = ctx->plan_kept;
  kept.clear();
  kept.reserve(ctx->n_blocks);
  for (long long b = 0; b < ctx->n_blocks; ++b)
    if (!(ctx->blk_norm[b] < thr)) kept.push_back((int)b);
  // per owner: lambda atoms and RI window
  std::vector<std::vector<int>> lam_atoms(n);
  std::vector<int> p0(n, INT32_MAX), p1(n, -1);
  for (int b : kept) {
    int A = ctx->blk[3 * b], B = ctx->blk[3 * b + 1], p = ctx->blk[3 * b + 2];
    lam_atoms[B].push_back(A);
    p0[B] = std::min(p0[B], ctx->ri_off[p]);
    p1[B] = std::max(p1[B], ctx->ri_off[p + 1]);
    if (A != B) {
      lam_atoms[A].push_back(B);
      p0[A] = std::min(p0[A], ctx->ri_off[p]);
      p1[A] = std::max(p1[A], ctx->ri_off[p + 1]);
    }
  }
  ctx->panels.assign(n, PanelDesc{});
  std::vector<int> lam;
  std::vector<std::map<int, int>> rowmap(n);
  long long off = 0;
  for (int s = 0; s < n; ++s) {
    auto& la = lam_atoms[s];
    std::sort(la.begin(), la.end());
    la.erase(std::unique(la.begin(), la.end()), la.end());
    PanelDesc d{};
    d.owner = s;
    d.nsig = ctx->n_ao[s];
    d.lam_off = (int)lam.size();
    int K = 0;
    for (int a : la) {
      rowmap[s][a] = K;
      for (int i = ctx->ao_off[a]; i < ctx->ao_off[a + 1]; ++i) lam.push_back(i);
      K += ctx->n_ao[a];
    }
    d.K = K;
    if (K > 0) {
      d.p0 = p0[s];
      d.npw = p1[s] - p0[s];
    }
    d.off = off;
    off += (long long)K * d.npw * d.nsig;
    ctx->panels[s] = d;
  }
  ctx->panel_elems = off;
  ctx->lam_total = (long long)lam.size();
  // per atom: the kept blocks in which it is an owner (B, or A != B)
  ctx->plan_atom_off.assign(n + 1, 0);
  for (int b : kept) {
    const int A = ctx->blk[3 * b], B = ctx->blk[3 * b + 1];
    ++ctx->plan_atom_off[B + 1];
    if (A != B) ++ctx->plan_atom_off[A + 1];
  }
  for (int a = 0; a < n; ++a) ctx->plan_atom_off[a + 1] += ctx->plan_atom_off[a];
  {
    std::vector<int> fill(ctx->plan_atom_off.begin(), ctx->plan_atom_off.end() - 1);
    ctx->plan_atom_blk.assign(ctx->plan_atom_off[n], 0);
    for (size_t i = 0; i < kept.size(); ++i) {
      const int b = kept[i];
      const int A = ctx->blk[3 * b], B = ctx->blk[3 * b + 1];
      ctx->plan_atom_blk[fill[B]++] = (int)i;
      if (A != B) ctx->plan_atom_blk[fill[A]++] = (int)i;
    }
  }
  // flop weights of steps A and B per (owner, lambda-atom)
  {
    std::vector<std::map<int, double>> wl(n);
    for (int b : kept) {
      const int A = ctx->blk[3 * b], B = ctx->blk[3 * b + 1], p = ctx->blk[3 * b + 2];
      const double w = 2.0 * ctx->n_ao[A] * ctx->n_ao[B] * ctx->n_ri[p];
      wl[B][A] += w;
      if (A != B) wl[A][B] += w;
    }
    ctx->wl_off.assign(n + 1, 0);
    ctx->wl_atom.clear();
    ctx->wl_w.clear();
    for (int s = 0; s < n; ++s) {
      for (const auto& kv : wl[s]) {
        ctx->wl_atom.push_back(kv.first);
        ctx->wl_w.push_back(kv.second);
      }
      ctx->wl_off[s + 1] = (int)ctx->wl_atom.size();
    }
  }
  ctx->plan_kB.resize(kept.size());
  ctx->plan_kA.resize(kept.size());
  for (size_t i = 0; i < kept.size(); ++i) {
    const int b = kept[i];
    const int A = ctx->blk[3 * b], B = ctx->blk[3 * b + 1];
    ctx->plan_kB[i] = rowmap[B][A];
    ctx->plan_kA[i] = rowmap[A][B];
  }
  free_dev(ctx->d_lam);
  ctx->d_lam = nullptr;
  GW_TRY(cudaMalloc(&ctx->d_lam, std::max<size_t>(lam.size(), 1) * sizeof(int)));
  if (!lam.empty())
    GW_TRY(cudaMemcpy(ctx->d_lam, lam.data(), lam.size() * sizeof(int), cudaMemcpyHostToDevice));
  ctx->plan_ok = true;
  ctx->plan_thr = thr;
  return GW_OK;
}

// The FP64 owner panels of the plan (the CUDA-core routes, the self-energy
// and the allocation-free entry point).
int build_panels(gw_ctx* ctx, double thr) {
  if (ctx->d_t3f)
    return fail(ctx, GW_ERR_UNSUPPORTED,
                "the FP64 panels need the tensor in FP64 (it is kept in FP32: option tensor_fp32)");
  int rc;
  if ((rc = plan_panels(ctx, thr))) return rc;
  if (ctx->panels_ok && ctx->panels_thr == thr) return GW_OK;
  // the pool (and its FP32 copy) stops being valid until rebuilt below
  ctx->panels_ok = false;
  ctx->panels_thr = -1.0;
  ctx->panel32_ok = false;
  const std::vector<int>& kept = ctx->plan_kept;
  const long long off = ctx->panel_elems;
  // destinations of each kept block
  std::vector<long long> dstB(kept.size()), dstA(kept.size());
  std::vector<int> ldB(kept.size()), ldA(kept.size());
  for (size_t i = 0; i < kept.size(); ++i) {
    int b = kept[i];
    int A = ctx->blk[3 * b], B = ctx->blk[3 * b + 1], p = ctx->blk[3 * b + 2];
    const PanelDesc& pb = ctx->panels[B];
    ldB[i] = pb.npw * pb.nsig;
    dstB[i] = pb.off + (long long)ctx->plan_kB[i] * ldB[i] + (long long)(ctx->ri_off[p] - pb.p0) * pb.nsig;
    const PanelDesc& pa = ctx->panels[A];
    ldA[i] = pa.npw * pa.nsig;
    dstA[i] = pa.off + (long long)ctx->plan_kA[i] * ldA[i] + (long long)(ctx->ri_off[p] - pa.p0) * pa.nsig;
  }
  free_dev(ctx->d_panel64);
  free_dev(ctx->d_panel32);
  ctx->d_panel64 = nullptr;
  ctx->d_panel32 = nullptr;
  GW_TRY(cudaMalloc(&ctx->d_panel64, std::max<long long>(off, 1) * sizeof(double)));
  GW_TRY(cudaMemsetAsync(ctx->d_panel64, 0, std::max<long long>(off, 1) * sizeof(double), ctx->stream));
  int *d_kept, *d_ldB, *d_ldA;
  long long *d_dstB, *d_dstA;
  if ((rc = upload(ctx, "kept", kept, &d_kept))) return rc;
  if ((rc = upload(ctx, "dstB", dstB, &d_dstB))) return rc;
  if ((rc = upload(ctx, "dstA", dstA, &d_dstA))) return rc;
  if ((rc = upload(ctx, "ldB", ldB, &d_ldB))) return rc;
  if ((rc = upload(ctx, "ldA", ldA, &d_ldA))) return rc;
  int *d_nao, *d_nri;
  if ((rc = upload(ctx, "n_ao", ctx->n_ao, &d_nao))) return rc;
  if ((rc = upload(ctx, "n_ri", ctx->n_ri, &d_nri))) return rc;
  gw::launch_panel_scatter(ctx->d_t3, ctx->d_blk, ctx->d_blk_off, d_nao, d_nri, ctx->d_ri_off,
                           d_kept, (int)kept.size(), d_dstB, d_dstA, d_ldB, d_ldA, ctx->d_panel64,
                           ctx->stream);
  GW_CHECK_LAUNCH();
  GW_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->panels_ok = true;
  ctx->panels_thr = thr;
  return GW_OK;
}

int ensure_panel32(gw_ctx* ctx) {
  if (ctx->panel32_ok) return GW_OK;
  free_dev(ctx->d_panel32);
  ctx->d_panel32 = nullptr;
  GW_TRY(cudaMalloc(&ctx->d_panel32, std::max<long long>(ctx->panel_elems, 1) * sizeof(float)));
  gw::launch_cast_f64_f32(ctx->d_panel64, ctx->d_panel32, ctx->panel_elems, ctx->stream);
  GW_CHECK_LAUNCH();
  ctx->panel32_ok = true;
  return GW_OK;
}

// ---------------------------------------------------------------------------
// batches of owner atoms
// ---------------------------------------------------------------------------
// Batches of consecutive owner atoms under a byte budget for the X and Y
// operands.  With align_rows > 0 a batch is cut, among the last half of the
// atoms that fit, where its primary-function count wastes the least of the
// last align_rows-row tile (step B runs on the batch's rows in such tiles).
std::vector<Batch> plan_batches(gw_ctx* ctx, size_t elem_bytes, double budget_bytes,
                                int align_rows = 0) {
  std::vector<Batch> out;
  const int n = ctx->n_at;
  int s = 0;
  while (s < n) {
    int e_max = s;
    {
      int P0 = INT32_MAX, P1 = 0;
      long long K = 0;
      while (e_max < n) {
        const PanelDesc& d = ctx->panels[e_max];
        int q0 = P0, q1 = P1;
        if (d.K > 0) {
          q0 = std::min(q0, d.p0);
          q1 = std::max(q1, d.p0 + d.npw);
        }
        const long long K2 = K + (long long)ctx->naop * d.nsig;
        const double bytes = (double)K2 * ((q1 > q0 ? q1 - q0 : 0) + ctx->nri) * elem_bytes;
        const bool limit = ctx->batch_atoms > 0 && e_max - s >= ctx->batch_atoms;
        if (e_max > s && (bytes > budget_bytes || limit)) break;
        P0 = q0;
        P1 = q1;
        K = K2;
        ++e_max;
      }
    }
    int e_cut = e_max;
    if (align_rows > 0 && e_max < n) {
      double best = 2.0;
      for (int e = e_max; e > s && e >= s + (e_max - s + 1) / 2; --e) {
        const int R = ctx->ao_off[e] - ctx->ao_off[s];
        const int Rp = (R + align_rows - 1) / align_rows * align_rows;
        const double waste = (double)(Rp - R) / Rp;
        if (waste < best - 1e-12) {
          best = waste;
          e_cut = e;
        }
      }
    }
    Batch b{};
    b.s0 = s;
    b.P0 = INT32_MAX;
    b.P1 = 0;
    long long K = 0;
    int e = s;
    while (e < e_cut) {
      const PanelDesc& d = ctx->panels[e];
      int P0 = b.P0, P1 = b.P1;
      if (d.K > 0) {
        P0 = std::min(P0, d.p0);
        P1 = std::max(P1, d.p0 + d.npw);
      }
      long long K2 = K + (long long)ctx->naop * d.nsig;
      b.P0 = P0;
      b.P1 = P1;
      b.seg.push_back(K);
      K = K2;
      ++e;
    }
    b.s1 = e;
    b.Kb = K;
    if (b.P1 <= b.P0) {
      b.P0 = 0;
      b.P1 = 0;
    }
    b.nslab = (b.s1 - b.s0) * (ctx->naop / kSlabAO);
    b.m0 = 0;
    b.m1 = n;
    b.mu0 = 0;
    b.nmu = ctx->nao;
    b.Lc = ctx->naop;
    b.Q0 = 0;
    b.Q1 = ctx->nri;
    out.push_back(b);
    s = e;
  }
  return out;
}

// RI window [q0, q1) of the panels of atoms [a0, a1) (q0 = q1 = 0: none).
void panel_window(const gw_ctx* ctx, int a0, int a1, int* q0, int* q1) {
  int lo = INT32_MAX, hi = 0;
  for (int a = a0; a < a1; ++a) {
    const PanelDesc& d = ctx->panels[a];
    if (d.K == 0) continue;
    lo = std::min(lo, d.p0);
    hi = std::max(hi, d.p0 + d.npw);
  }
  if (hi <= lo) lo = hi = 0;
  *q0 = lo;
  *q1 = hi;
}

// 2-D batches of the tensor-core route: chunks of mu-atoms, and in each
// chunk batches of consecutive owner atoms under the byte budget for X and
// Y (elem_bytes per operand element), cut where the batch's primary-function
// count wastes the least of its last align_rows-row tile (step B runs on the
// batch's rows in such tiles).  One chunk of every atom keeps Y over all RI
// functions; several chunks give each its panels' RI window.
std::vector<Batch> plan_batches_tc(gw_ctx* ctx, size_t elem_bytes, double budget_bytes, int align_rows) {
  const int n = ctx->n_at;
  auto seg_len = [&](int m0, int m1) {
    const int nmu = ctx->ao_off[m1] - ctx->ao_off[m0];
    return (nmu + kSlabAO - 1) / kSlabAO * kSlabAO;
  };
  int cs = ctx->mu_chunk_atoms;
  if (cs <= 0 || cs > n) {
    // fewest equal chunks for which one owner's operands stay within a
    // budget share of 1/8 (so that batches hold several owners)
    for (int nc = 1; nc <= n; ++nc) {
      cs = (n + nc - 1) / nc;
      bool ok = true;
      for (int m0 = 0; m0 < n && ok; m0 += cs) {
        const int m1 = std::min(n, m0 + cs);
        int q0 = 0, q1 = ctx->nri;
        if (nc > 1) panel_window(ctx, m0, m1, &q0, &q1);
        const double lc = seg_len(m0, m1);
        for (int s = 0; s < n && ok; ++s) {
          const PanelDesc& d = ctx->panels[s];
          if (d.K == 0) continue;
          ok = lc * d.nsig * (double)(d.npw + (q1 - q0)) * elem_bytes <= budget_bytes / 8;
        }
      }
      if (ok) break;
    }
  }
  const bool single = cs >= n;
  std::vector<Batch> out;
  for (int m0 = 0; m0 < n; m0 += cs) {
    const int m1 = std::min(n, m0 + cs);
    int Q0 = 0, Q1 = ctx->nri;
    if (!single) panel_window(ctx, m0, m1, &Q0, &Q1);
    if (Q1 <= Q0) continue;  // no panel in the chunk: its Y is zero
    const int Lc = seg_len(m0, m1);
    const int qrow = Q1 - Q0;
    int s = 0;
    while (s < n) {
      int e_max = s;
      {
        int P0 = INT32_MAX, P1 = 0;
        long long K = 0;
        while (e_max < n) {
          const PanelDesc& d = ctx->panels[e_max];
          int q0 = P0, q1 = P1;
          if (d.K > 0) {
            q0 = std::min(q0, d.p0);
            q1 = std::max(q1, d.p0 + d.npw);
          }
          const long long K2 = K + (long long)Lc * d.nsig;
          const double bytes = (double)K2 * ((q1 > q0 ? q1 - q0 : 0) + qrow) * elem_bytes;
          const bool limit = ctx->batch_atoms > 0 && e_max - s >= ctx->batch_atoms;
          if (e_max > s && (bytes > budget_bytes || limit)) break;
          P0 = q0;
          P1 = q1;
          K = K2;
          ++e_max;
        }
      }
      int e_cut = e_max;
      if (align_rows > 0 && e_max < n) {
        double best = 2.0;
        for (int e = e_max; e > s && e >= s + (e_max - s + 1) / 2; --e) {
          const int R = ctx->ao_off[e] - ctx->ao_off[s];
          const int Rp = (R + align_rows - 1) / align_rows * align_rows;
          const double waste = (double)(Rp - R) / Rp;
          if (waste < best - 1e-12) {
            best = waste;
            e_cut = e;
          }
        }
      }
      Batch b{};
      b.s0 = s;
      b.P0 = INT32_MAX;
      b.P1 = 0;
      long long K = 0;
      for (int e = s; e < e_cut; ++e) {
        const PanelDesc& d = ctx->panels[e];
        if (d.K > 0) {
          b.P0 = std::min(b.P0, d.p0);
          b.P1 = std::max(b.P1, d.p0 + d.npw);
        }
        b.seg.push_back(K);
        K += (long long)Lc * d.nsig;
      }
      b.s1 = e_cut;
      b.Kb = K;
      if (b.P1 <= b.P0) {
        b.P0 = 0;
        b.P1 = 0;
      }
      b.nslab = (b.s1 - b.s0) * (Lc / kSlabAO);
      b.m0 = m0;
      b.m1 = m1;
      b.mu0 = ctx->ao_off[m0];
      b.nmu = ctx->ao_off[m1] - ctx->ao_off[m0];
      b.Lc = Lc;
      b.Q0 = Q0;
      b.Q1 = Q1;
      out.push_back(b);
      s = e_cut;
    }
  }
  return out;
}

// Useful flops of steps A and B of one batch from the kept G blocks of this
// tau point (flags [n_at][n_at], symmetric): step A multiplies each kept
// block (l, s, P) of an owner s of the batch by every kept G^occ block
// (m, l) with m in the chunk, step B each kept block (l, m, Q) of a chunk
// atom m by every kept G^virt block (s, l) with s an owner of the batch.
// kao[l] = sum over the chunk's atoms m of n(m) [G^occ block (m, l) kept],
// computed once per chunk by chunk_kao.
void chunk_kao(const gw_ctx* ctx, int m0, int m1, const std::vector<unsigned char>& fo,
               std::vector<double>& kao) {
  const int n = ctx->n_at;
  kao.assign(n, 0.0);
  for (int m = m0; m < m1; ++m)
    for (int l = 0; l < n; ++l)
      if (fo[(size_t)m * n + l]) kao[l] += ctx->n_ao[m];
}
void batch_flops_ab(const gw_ctx* ctx, const Batch& b, const std::vector<double>& kao,
                    const std::vector<unsigned char>& fv, double* fa, double* fb) {
  const int n = ctx->n_at;
  std::vector<double> kav(n, 0.0);
  for (int s = b.s0; s < b.s1; ++s)
    for (int l = 0; l < n; ++l)
      if (fv[(size_t)s * n + l]) kav[l] += ctx->n_ao[s];
  double a = 0.0, v = 0.0;
  for (int s = b.s0; s < b.s1; ++s)
    for (int i = ctx->wl_off[s]; i < ctx->wl_off[s + 1]; ++i) a += ctx->wl_w[i] * kao[ctx->wl_atom[i]];
  for (int m = b.m0; m < b.m1; ++m)
    for (int i = ctx->wl_off[m]; i < ctx->wl_off[m + 1]; ++i) v += ctx->wl_w[i] * kav[ctx->wl_atom[i]];
  *fa = a;
  *fb = v;
}

// CUDA events bracketing the step launches of each batch (two pairs per
// batch: 2 b for step C, 2 b + 1 for steps A/B), kept in the context
int c_event_pair(gw_ctx* ctx, size_t idx, cudaEvent_t* a, cudaEvent_t* b) {
  auto& v = ctx->events;
  while (v.size() < 2 * (idx + 1)) {
    cudaEvent_t e;
    GW_TRY(cudaEventCreate(&e));
    v.push_back(e);
  }
  *a = v[2 * idx];
  *b = v[2 * idx + 1];
  return GW_OK;
}

template <typename T>
int chi_one_batch(gw_ctx* ctx, const Batch& b, const T* g_occ, const T* g_virt, const T* pool,
                  double thr, double* acc, std::vector<double>& fc_host, int /*precision*/,
                  size_t batch_idx) {
  const int ns = b.s1 - b.s0;
  gw::TraceRange trace("chi: batch, CUDA cores");
  const int prow = b.P1 - b.P0;
  const long long Kb = b.Kb;
  int rc;
  if (prow == 0 || Kb == 0) return GW_OK;
  T *X, *Y;
  if ((rc = wsT<T>(ctx, "X", (size_t)prow * Kb, &X))) return rc;
  if ((rc = wsT<T>(ctx, "Y", (size_t)ctx->nri * Kb, &Y))) return rc;
  GW_TRY(cudaMemsetAsync(X, 0, (size_t)prow * Kb * sizeof(T), ctx->stream));
  GW_TRY(cudaMemsetAsync(Y, 0, (size_t)ctx->nri * Kb * sizeof(T), ctx->stream));

  // step A tasks: owners of the batch, rows mu = all AOs
  std::vector<PanelTask> ta;
  int maxNa = 0;
  for (int s = b.s0; s < b.s1; ++s) {
    const PanelDesc& d = ctx->panels[s];
    if (d.K == 0) continue;
    PanelTask t{};
    t.panel_off = d.off;
    t.K = d.K;
    t.N = d.npw * d.nsig;
    t.lam_off = d.lam_off;
    t.npw = d.npw;
    t.nsig = d.nsig;
    t.p0 = d.p0;
    t.aom = ctx->ao_off[s];
    t.seg = b.seg[s - b.s0];
    maxNa = std::max(maxNa, t.N);
    ta.push_back(t);
  }
  // step B tasks: every panel, rows sigma of the batch
  std::vector<PanelTask> tb;
  int maxNb = 0;
  for (int m = 0; m < ctx->n_at; ++m) {
    const PanelDesc& d = ctx->panels[m];
    if (d.K == 0) continue;
    PanelTask t{};
    t.panel_off = d.off;
    t.K = d.K;
    t.N = d.npw * d.nsig;
    t.lam_off = d.lam_off;
    t.npw = d.npw;
    t.nsig = d.nsig;
    t.p0 = d.p0;
    t.aom = ctx->ao_off[m];
    t.seg = 0;
    maxNb = std::max(maxNb, t.N);
    tb.push_back(t);
  }
  const int r0 = ctx->ao_off[b.s0];
  const int R = ctx->ao_off[b.s1] - r0;
  std::vector<long long> rowbase(R);
  std::vector<int> rowmul(R);
  for (int s = b.s0; s < b.s1; ++s)
    for (int i = 0; i < ctx->n_ao[s]; ++i) {
      rowbase[ctx->ao_off[s] - r0 + i] = b.seg[s - b.s0] + i;
      rowmul[ctx->ao_off[s] - r0 + i] = ctx->n_ao[s];
    }
  PanelTask *d_ta, *d_tb;
  long long* d_rowbase;
  int* d_rowmul;
  if ((rc = upload(ctx, "tasksA", ta, &d_ta))) return rc;
  if ((rc = upload(ctx, "tasksB", tb, &d_tb))) return rc;
  if ((rc = upload(ctx, "rowbase", rowbase, &d_rowbase))) return rc;
  if ((rc = upload(ctx, "rowmul", rowmul, &d_rowmul))) return rc;

  gw::launch_panel_gemm<T>(g_occ, ctx->nao, pool, ctx->d_lam, d_ta, (int)ta.size(), maxNa, 0, 0,
                           ctx->nao, b.P0, Kb, nullptr, nullptr, X, ctx->stream);
  GW_CHECK_LAUNCH();
  gw::launch_panel_gemm<T>(g_virt, ctx->nao, pool, ctx->d_lam, d_tb, (int)tb.size(), maxNb, 1, r0,
                           R, 0, Kb, d_rowbase, d_rowmul, Y, ctx->stream);
  GW_CHECK_LAUNCH();
  ctx->stats.kernel_launches += 2;
  ctx->stats.bytes_operands += (double)(prow + ctx->nri) * Kb * sizeof(T);

  // block filter of X and Y, occupancy flags
  const bool tcpath = false;
  const int slices = 1;
  const int tile = 64;
  const int nslab = b.nslab;
  const int npt = (prow + tile - 1) / tile, nqt = (ctx->nri + tile - 1) / tile;
  const int pa0 = [&] {
    int a = 0;
    while (ctx->ri_off[a + 1] <= b.P0) ++a;
    return a;
  }();
  int pa1 = pa0;
  while (pa1 < ctx->n_at && ctx->ri_off[pa1] < b.P1) ++pa1;
  const int npa = pa1 - pa0;
  unsigned char *bx, *by, *fx, *fy;
  if ((rc = wsT(ctx, "bx", (size_t)ns * ctx->n_at * npa, &bx))) return rc;
  if ((rc = wsT(ctx, "by", (size_t)ns * ctx->n_at * ctx->n_at, &by))) return rc;
  if ((rc = wsT(ctx, "fx", (size_t)ns * ctx->n_at * npt, &fx))) return rc;
  if ((rc = wsT(ctx, "fy", (size_t)ns * ctx->n_at * nqt, &fy))) return rc;
  GW_TRY(cudaMemsetAsync(fx, 0, (size_t)ns * ctx->n_at * npt, ctx->stream));
  GW_TRY(cudaMemsetAsync(fy, 0, (size_t)ns * ctx->n_at * nqt, ctx->stream));
  long long* d_seg;
  if ((rc = upload(ctx, "seg", b.seg, &d_seg))) return rc;
  int* d_nao;
  if ((rc = upload(ctx, "n_ao_b", ctx->n_ao, &d_nao))) return rc;
  gw::launch_operand_block_filter<T>(X, Kb, b.P0, ctx->d_ri_off, ctx->d_ao_off, d_nao, b.s0, ns,
                                     d_seg, pa0, npa, ctx->n_at, thr, ctx->naop, bx, fx, npt, tile,
                                     ctx->stream);
  GW_CHECK_LAUNCH();
  gw::launch_operand_block_filter<T>(Y, Kb, 0, ctx->d_ri_off, ctx->d_ao_off, d_nao, b.s0, ns, d_seg,
                                     0, ctx->n_at, ctx->n_at, thr, ctx->naop, by, fy, nqt, tile,
                                     ctx->stream);
  GW_CHECK_LAUNCH();
  // slabs
  std::vector<long long> slab_k0(nslab);
  std::vector<int> slab_len(nslab);
  const int per = ctx->naop / kSlabAO;
  for (int sl = 0; sl < ns; ++sl)
    for (int c = 0; c < per; ++c) {
      int nsig = ctx->n_ao[b.s0 + sl];
      slab_k0[sl * per + c] = b.seg[sl] + (long long)c * kSlabAO * nsig;
      slab_len[sl * per + c] = kSlabAO * nsig;
    }
  long long* d_k0;
  int* d_len;
  if ((rc = upload(ctx, "slab_k0", slab_k0, &d_k0))) return rc;
  if ((rc = upload(ctx, "slab_len", slab_len, &d_len))) return rc;
  int *tasks, *counts;
  long long* kacc;
  if ((rc = wsT(ctx, "tasks", (size_t)npt * nqt * nslab, &tasks))) return rc;
  if ((rc = wsT(ctx, "counts", (size_t)npt * nqt, &counts))) return rc;
  if ((rc = wsT(ctx, "kacc", (size_t)npt * nqt, &kacc))) return rc;
  gw::launch_build_tasks(fx, fy, nslab, npt, nqt, b.P0, prow, 0, ctx->nri, ctx->d_atom_of_ri, d_len,
                         tasks, counts, kacc, tile, per, 0, ctx->n_at, 0, ctx->nao, ctx->d_atom_of_ao,
                         ctx->stream);
  GW_CHECK_LAUNCH();
  double* d_fc;
  if ((rc = wsT(ctx, "fc", (size_t)ns * ctx->n_at, &d_fc))) return rc;
  int* d_nri;
  if ((rc = upload(ctx, "n_ri_b", ctx->n_ri, &d_nri))) return rc;
  gw::launch_count_c(bx, by, ns, 0, ctx->n_at, pa0, npa, 0, ctx->n_at, d_nri, d_nao, b.s0, d_fc,
                     ctx->stream);
  GW_CHECK_LAUNCH();
  ctx->stats.kernel_launches += 5;

  // step C
  cudaEvent_t ec0, ec1;
  if ((rc = c_event_pair(ctx, 2 * batch_idx, &ec0, &ec1))) return rc;
  std::vector<int> h_counts((size_t)npt * nqt);
  int* d_err = nullptr;
  {
    GW_TRY(cudaEventRecord(ec0, ctx->stream));
    gw::launch_chi_tiles<T, T>(X, Y, Kb, b.P0, prow, ctx->nri, tasks, counts, nslab, npt, nqt, d_k0,
                               d_len, acc, ctx->stream);
    GW_CHECK_LAUNCH();
    GW_TRY(cudaEventRecord(ec1, ctx->stream));
    ctx->stats.c_launches += 1;
    ctx->stats.kernel_launches += 1;
  }
  // counters (small D2H)
  std::vector<long long> h_kacc((size_t)npt * nqt);
  std::vector<double> h_fc((size_t)ns * ctx->n_at);
  GW_TRY(cudaMemcpyAsync(h_counts.data(), counts, h_counts.size() * sizeof(int),
                         cudaMemcpyDeviceToHost, ctx->stream));
  GW_TRY(cudaMemcpyAsync(h_kacc.data(), kacc, h_kacc.size() * sizeof(long long),
                         cudaMemcpyDeviceToHost, ctx->stream));
  GW_TRY(cudaMemcpyAsync(h_fc.data(), d_fc, h_fc.size() * sizeof(double), cudaMemcpyDeviceToHost,
                         ctx->stream));
  int h_err = 0;
  if (d_err) GW_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GW_TRY(cudaStreamSynchronize(ctx->stream));
  if (h_err)
    return fail(ctx, GW_ERR_TIMEOUT,
                "tensor-core step C: a bounded wait gave up (flags " + std::to_string(h_err) + ")");
  float ms_ck = 0.f;
  GW_TRY(cudaEventElapsedTime(&ms_ck, ec0, ec1));
  ctx->stats.ms_step_c_kernel += ms_ck;
  long long act = 0, sl_act = 0;
  for (int c : h_counts) {
    act += c > 0;
    sl_act += c;
  }
  ctx->stats.tiles_total += (long long)npt * nqt;
  ctx->stats.tiles_active += act;
  ctx->stats.slabs_total += (long long)npt * nqt * nslab;
  ctx->stats.slabs_active += sl_act;
  for (double v : h_fc) fc_host.push_back(v);
  // issued by step C: 2 * tile area * K over active tiles (x products per product)
  double ksum = 0.0;
  for (long long k : h_kacc) ksum += (double)k;
  (void)tcpath;
  (void)slices;
  ctx->stats.flops_issued += 2.0 * tile * tile * ksum;
  return GW_OK;
}

// ---------------------------------------------------------------------------
// tensor-core route: transposed split panels (once per thr and slice count)
// ---------------------------------------------------------------------------
int ensure_pt(gw_ctx* ctx, int slices, int f16) {
  if (ctx->pt_ok && ctx->pt_slices == slices && ctx->pt_f16 == f16 && ctx->pt_thr == ctx->plan_thr)
    return GW_OK;
  free_dev(ctx->d_pt);
  ctx->d_pt = nullptr;
  ctx->pt_ok = false;
  ctx->pt_tasks.assign(ctx->n_at, gw::PanelTaskTC{});
  long long rows = 0;
  int kmax = 64;
  for (int s = 0; s < ctx->n_at; ++s) {
    const PanelDesc& d = ctx->panels[s];
    gw::PanelTaskTC t{};
    t.K = d.K;
    if (d.K == 0) {
      ctx->pt_tasks[s] = t;
      continue;
    }
    t.panel_off = d.off;
    t.N = d.npw * d.nsig;
    t.npw = d.npw;
    t.nsig = d.nsig;
    t.p0 = d.p0;
    t.aom = ctx->ao_off[s];
    t.owner = s;
    t.lam_off = d.lam_off;
    t.ksteps = (d.K + 63) / 64;  // K steps of 64 (the tensor-core stage width)
    t.p_row0 = (int)rows;
    rows += (t.N + 127) / 128 * 128;
    kmax = std::max(kmax, t.ksteps * 64);
    ctx->pt_tasks[s] = t;
  }
  if (rows > INT32_MAX) return fail(ctx, GW_ERR_INVALID_ARG, "transposed panels exceed 2^31 rows");
  ctx->ptB_m0 = ctx->ptB_m1 = -1;
  // stream the panels per batch when the whole set, with the operand batch
  // budget, chi and the Green's functions, does not fit in free memory
  {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const double need = (double)slices * rows * kmax * 2 + ctx->batch_bytes +
                        3.0 * ctx->nri * (double)ctx->nri * 8 + 5.0 * ctx->nao * (double)ctx->nao * 8 + 2e9;
    ctx->pt_stream = ctx->panel_stream || need > (double)free_b;
  }
  if (ctx->pt_stream) {
    double pt_scale = 1.0;
    int rc;
    if (f16) {
      double *st2, h[4] = {0, 0, 0, 0};
      if ((rc = wsT(ctx, "pt_absmax", 4, &st2))) return rc;
      const long long n = ctx->n_elems, nrow = n / 1024;
      if (ctx->d_t3f) {
        gw::launch_absmax_f32(ctx->d_t3f, n, st2, ctx->stream);
        GW_TRY(cudaMemsetAsync(st2 + 2, 0, 2 * sizeof(double), ctx->stream));
      } else {
        gw::launch_absmax_rowsum(ctx->d_t3, 1024, (int)nrow, 1024, st2, ctx->stream);
        gw::launch_absmax_rowsum(ctx->d_t3 + nrow * 1024, 1024, n > nrow * 1024 ? 1 : 0,
                                 (int)(n - nrow * 1024), st2 + 2, ctx->stream);
      }
      GW_CHECK_LAUNCH();
      GW_TRY(cudaMemcpyAsync(h, st2, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
      GW_TRY(cudaStreamSynchronize(ctx->stream));
      ctx->t_absmax = std::max(h[0], h[2]);
      pt_scale = gw::pow2_scale(ctx->t_absmax);
    }
    ctx->pt_rows = 0;
    ctx->pt_kmax = kmax;
    ctx->pt_slices = slices;
    ctx->pt_f16 = f16;
    ctx->pt_scale = pt_scale;
    ctx->pt_thr = ctx->plan_thr;
    ctx->pt_ok = true;
    return GW_OK;
  }
  // rows of each kept block in the two panels it lands in: (pw of its first
  // RI function, s' = 0)
  const std::vector<int>& kept = ctx->plan_kept;
  std::vector<long long> rowB(kept.size()), rowA(kept.size());
  for (size_t i = 0; i < kept.size(); ++i) {
    const int b = kept[i];
    const int A = ctx->blk[3 * b], B = ctx->blk[3 * b + 1], p = ctx->blk[3 * b + 2];
    const gw::PanelTaskTC& tb = ctx->pt_tasks[B];
    const gw::PanelTaskTC& ta = ctx->pt_tasks[A];
    rowB[i] = tb.p_row0 + (long long)(ctx->ri_off[p] - tb.p0) * tb.nsig;
    rowA[i] = ta.p_row0 + (long long)(ctx->ri_off[p] - ta.p0) * ta.nsig;
  }
  const size_t bytes = (size_t)slices * rows * kmax * 2;
  GW_TRY(cudaMalloc(&ctx->d_pt, std::max<size_t>(bytes, 16)));
  GW_TRY(cudaMemsetAsync(ctx->d_pt, 0, std::max<size_t>(bytes, 16), ctx->stream));
  int rc;
  int *d_kept, *d_kB, *d_kA, *d_nao, *d_nri;
  long long *d_rowB, *d_rowA;
  if ((rc = upload(ctx, "kept", kept, &d_kept)) || (rc = upload(ctx, "pt_kB", ctx->plan_kB, &d_kB)) ||
      (rc = upload(ctx, "pt_kA", ctx->plan_kA, &d_kA)) || (rc = upload(ctx, "pt_rowB", rowB, &d_rowB)) ||
      (rc = upload(ctx, "pt_rowA", rowA, &d_rowA)) || (rc = upload(ctx, "n_ao", ctx->n_ao, &d_nao)) ||
      (rc = upload(ctx, "n_ri", ctx->n_ri, &d_nri)))
    return rc;
  double pt_scale = 1.0;
  if (f16) {
    // exact max |T| over the stored tensor (viewed as rows of 1024 plus a
    // tail): a bound on every panel entry
    double *st2, h[4] = {0, 0, 0, 0};
    if ((rc = wsT(ctx, "pt_absmax", 4, &st2))) return rc;
    const long long n = ctx->n_elems, nrow = n / 1024;
    if (ctx->d_t3f) {
      gw::launch_absmax_f32(ctx->d_t3f, n, st2, ctx->stream);
      GW_TRY(cudaMemsetAsync(st2 + 2, 0, 2 * sizeof(double), ctx->stream));
    } else {
      gw::launch_absmax_rowsum(ctx->d_t3, 1024, (int)nrow, 1024, st2, ctx->stream);
      gw::launch_absmax_rowsum(ctx->d_t3 + nrow * 1024, 1024, n > nrow * 1024 ? 1 : 0,
                               (int)(n - nrow * 1024), st2 + 2, ctx->stream);
    }
    GW_CHECK_LAUNCH();
    GW_TRY(cudaMemcpyAsync(h, st2, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    GW_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->t_absmax = std::max(h[0], h[2]);
    pt_scale = gw::pow2_scale(ctx->t_absmax);
  }
  if (ctx->d_t3f)
    gw::launch_pt_scatter_f32(ctx->d_t3f, ctx->d_blk, ctx->d_blk_off, d_nao, d_nri, d_kept,
                              (long long)kept.size(), d_rowB, d_kB, d_rowA, d_kA, kmax, slices, rows * kmax,
                              f16, pt_scale, ctx->d_pt, ctx->stream);
  else
    gw::launch_pt_scatter(ctx->d_t3, ctx->d_blk, ctx->d_blk_off, d_nao, d_nri, d_kept, (long long)kept.size(),
                          d_rowB, d_kB, d_rowA, d_kA, kmax, slices, rows * kmax, f16, pt_scale, ctx->d_pt,
                          ctx->stream);
  GW_CHECK_LAUNCH();
  GW_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->pt_rows = rows;
  ctx->pt_kmax = kmax;
  ctx->pt_slices = slices;
  ctx->pt_f16 = f16;
  ctx->pt_scale = pt_scale;
  ctx->pt_thr = ctx->plan_thr;
  ctx->pt_ok = true;
  return GW_OK;
}

// Streamed split panels of the atoms in [a0, a1) into the named region: rows
// per atom in that order (row0[atom], -1 for atoms without a panel), the
// region zeroed and scattered from the kept blocks in which the atom is an
// owner.  *rows_out = the region's rows.
int build_pt_region(gw_ctx* ctx, const char* name, int a0, int a1, void** buf, long long* rows_out,
                    std::vector<int>& row0) {
  const int slices = ctx->pt_slices, kmax = ctx->pt_kmax;
  row0.assign(ctx->n_at, -1);
  long long rows = 0;
  for (int s = a0; s < a1; ++s) {
    const gw::PanelTaskTC& t = ctx->pt_tasks[s];
    if (t.K == 0) continue;
    row0[s] = (int)rows;
    rows += (t.N + 127) / 128 * 128;
  }
  *rows_out = rows;
  const size_t bytes = std::max<size_t>((size_t)slices * rows * kmax * 2, 16);
  int rc;
  if ((rc = ws(ctx, name, bytes, buf))) return rc;
  GW_TRY(cudaMemsetAsync(*buf, 0, bytes, ctx->stream));
  // one entry per (kept block, owner side in the range)
  std::vector<int> ent_blk, ent_kB, ent_kA;
  std::vector<long long> ent_rowB, ent_rowA;
  for (int s = a0; s < a1; ++s) {
    if (row0[s] < 0) continue;
    const gw::PanelTaskTC& t = ctx->pt_tasks[s];
    for (int e = ctx->plan_atom_off[s]; e < ctx->plan_atom_off[s + 1]; ++e) {
      const int i = ctx->plan_atom_blk[e];
      const int b = ctx->plan_kept[i];
      const int B = ctx->blk[3 * b + 1], p = ctx->blk[3 * b + 2];
      const long long r = row0[s] + (long long)(ctx->ri_off[p] - t.p0) * t.nsig;
      ent_blk.push_back(b);
      if (B == s) {
        ent_rowB.push_back(r);
        ent_kB.push_back(ctx->plan_kB[i]);
        ent_rowA.push_back(-1);
        ent_kA.push_back(0);
      } else {
        ent_rowB.push_back(-1);
        ent_kB.push_back(0);
        ent_rowA.push_back(r);
        ent_kA.push_back(ctx->plan_kA[i]);
      }
    }
  }
  int *d_blk, *d_kB, *d_kA, *d_nao, *d_nri;
  long long *d_rowB, *d_rowA;
  if ((rc = upload(ctx, "ptr_blk", ent_blk, &d_blk)) || (rc = upload(ctx, "ptr_kB", ent_kB, &d_kB)) ||
      (rc = upload(ctx, "ptr_kA", ent_kA, &d_kA)) || (rc = upload(ctx, "ptr_rowB", ent_rowB, &d_rowB)) ||
      (rc = upload(ctx, "ptr_rowA", ent_rowA, &d_rowA)) || (rc = upload(ctx, "n_ao", ctx->n_ao, &d_nao)) ||
      (rc = upload(ctx, "n_ri", ctx->n_ri, &d_nri)))
    return rc;
  if (ctx->d_t3f)
    gw::launch_pt_scatter_f32(ctx->d_t3f, ctx->d_blk, ctx->d_blk_off, d_nao, d_nri, d_blk,
                              (long long)ent_blk.size(), d_rowB, d_kB, d_rowA, d_kA, kmax, slices,
                              rows * kmax, ctx->pt_f16, ctx->pt_scale, *buf, ctx->stream);
  else
    gw::launch_pt_scatter(ctx->d_t3, ctx->d_blk, ctx->d_blk_off, d_nao, d_nri, d_blk,
                          (long long)ent_blk.size(), d_rowB, d_kB, d_rowA, d_kA, kmax, slices, rows * kmax,
                          ctx->pt_f16, ctx->pt_scale, *buf, ctx->stream);
  GW_CHECK_LAUNCH();
  // the host tables are read by the copies above before they go out of scope
  GW_TRY(cudaStreamSynchronize(ctx->stream));
  return GW_OK;
}

// Owners covering each RI row (for zeroing only the unwritten part of Y):
// once per panel build.
int ensure_ycover(gw_ctx* ctx) {
  if (ctx->ycov_valid) return GW_OK;
  free_dev(ctx->d_ycov_lo);
  free_dev(ctx->d_ycov_hi);
  ctx->d_ycov_lo = ctx->d_ycov_hi = nullptr;
  const int nri = ctx->nri;
  std::vector<int> lo(nri, INT32_MAX), hi(nri, -1), cnt(nri, 0);
  for (int m = 0; m < ctx->n_at; ++m) {
    const PanelDesc& d = ctx->panels[m];
    if (d.K == 0) continue;
    for (int q = d.p0; q < d.p0 + d.npw; ++q) {
      lo[q] = std::min(lo[q], m);
      hi[q] = std::max(hi[q], m);
      ++cnt[q];
    }
  }
  bool ok = true;
  for (int q = 0; q < nri && ok; ++q) {
    if (cnt[q] == 0) {
      lo[q] = -1;
      hi[q] = -1;
    } else if (hi[q] - lo[q] + 1 != cnt[q]) {
      ok = false;
    }
  }
  if (!ok) {
    ctx->ycov_ok = false;
    ctx->ycov_valid = true;
    return GW_OK;
  }
  // valid only once both tables are on the device
  GW_TRY(cudaMalloc(&ctx->d_ycov_lo, std::max(nri, 1) * sizeof(int)));
  GW_TRY(cudaMalloc(&ctx->d_ycov_hi, std::max(nri, 1) * sizeof(int)));
  GW_TRY(cudaMemcpy(ctx->d_ycov_lo, lo.data(), nri * sizeof(int), cudaMemcpyHostToDevice));
  GW_TRY(cudaMemcpy(ctx->d_ycov_hi, hi.data(), nri * sizeof(int), cudaMemcpyHostToDevice));
  ctx->ycov_ok = true;
  ctx->ycov_valid = true;
  return GW_OK;
}

// One batch on the tensor cores: steps A and B straight into bf16 slices,
// block filter from the accumulated norms, task lists, step C.
int chi_one_batch_tc(gw_ctx* ctx, const Batch& b, const double* g_occ, const double* g_virt,
                     double thr, double* acc, std::vector<double>& fc_host, int precision,
                     size_t batch_idx) {
  const int slices = precision == GW_BF16X6 ? 3 : 2;
  gw::TraceRange trace("chi: batch, tensor cores");
  const int f16 = precision == GW_FP16X3;
  const double prods = slices == 3 ? 6.0 : 3.0;
  const int tile = gw::tc_tile_rows();
  // binary16 scales (powers of two; 1 for bf16): G^occ, G^virt, X, Y, T
  const double s_go = f16 ? ctx->tc_scale[0] : 1.0, s_gv = f16 ? ctx->tc_scale[1] : 1.0;
  const double s_x = f16 ? ctx->tc_scale[2] : 1.0, s_y = f16 ? ctx->tc_scale[3] : 1.0;
  const double s_t = f16 ? ctx->pt_scale : 1.0;
  const int ns = b.s1 - b.s0;
  const int prow = b.P1 - b.P0;
  const int qrow = b.Q1 - b.Q0;  // Y rows: RI functions [Q0, Q1)
  const int nmc = b.m1 - b.m0;   // mu-atoms of the chunk
  const long long Kb = b.Kb;
  const int n_at = ctx->n_at, nri = ctx->nri;
  int rc;
  if (prow == 0 || qrow == 0 || Kb == 0) return GW_OK;
  const int kmax = ctx->pt_kmax;
  void *xs, *ys;
  if ((rc = ws(ctx, "Xs", (size_t)slices * prow * Kb * 2, &xs))) return rc;
  if ((rc = ws(ctx, "Ys", (size_t)slices * qrow * Kb * 2, &ys))) return rc;
  GW_TRY(cudaMemsetAsync(xs, 0, (size_t)slices * prow * Kb * 2, ctx->stream));
  if ((rc = ensure_ycover(ctx))) return rc;
  if (ctx->ycov_ok) {
    // step B writes every (q, s, mu of a covering owner, sigma); zero the rest
    long long* d_seg0;
    int* d_nao0;
    if ((rc = upload(ctx, "seg_y", b.seg, &d_seg0))) return rc;
    if ((rc = upload(ctx, "n_ao_y", ctx->n_ao, &d_nao0))) return rc;
    gw::launch_zero_unwritten_y(ys, slices, (long long)qrow * Kb, Kb, b.Q0, qrow, ns, d_seg0, d_nao0,
                                b.s0, ctx->d_ao_off, b.m0, b.m1, b.Lc, ctx->d_ycov_lo,
                                ctx->d_ycov_hi, ctx->stream);
    GW_CHECK_LAUNCH();
  } else {
    GW_TRY(cudaMemsetAsync(ys, 0, (size_t)slices * qrow * Kb * 2, ctx->stream));
  }
  const int pa0 = [&] {
    int a = 0;
    while (ctx->ri_off[a + 1] <= b.P0) ++a;
    return a;
  }();
  int pa1 = pa0;
  while (pa1 < n_at && ctx->ri_off[pa1] < b.P1) ++pa1;
  const int npa = pa1 - pa0;
  // RI atoms of the Y rows
  const int qa0 = [&] {
    int a = 0;
    while (ctx->ri_off[a + 1] <= b.Q0) ++a;
    return a;
  }();
  int qa1 = qa0;
  while (qa1 < n_at && ctx->ri_off[qa1] < b.Q1) ++qa1;
  const int nqa = qa1 - qa0;
  float *bx2, *by2;
  if ((rc = wsT(ctx, "bx2", (size_t)ns * nmc * npa, &bx2))) return rc;
  if ((rc = wsT(ctx, "by2", (size_t)ns * nmc * nqa, &by2))) return rc;
  GW_TRY(cudaMemsetAsync(bx2, 0, (size_t)ns * nmc * npa * sizeof(float), ctx->stream));
  GW_TRY(cudaMemsetAsync(by2, 0, (size_t)ns * nmc * nqa * sizeof(float), ctx->stream));
  int* d_err;  // zeroed once per tau point by gw_chi_tau
  if ((rc = wsT(ctx, "tc_err", 1, &d_err))) return rc;
  // split panels: the resident set for both steps, or streamed regions (A:
  // the batch's owners, rebuilt per batch; B: the chunk's atoms, rebuilt when
  // the chunk changes)
  CUtensorMap mpA, mpB;
  std::vector<int> row0A;
  if (ctx->pt_stream) {
    void* bufA;
    long long rowsA = 0;
    if ((rc = build_pt_region(ctx, "ptA", b.s0, b.s1, &bufA, &rowsA, row0A))) return rc;
    if (ctx->ptB_m0 != b.m0 || ctx->ptB_m1 != b.m1) {
      ctx->ptB_m0 = ctx->ptB_m1 = -1;
      if ((rc = build_pt_region(ctx, "ptB", b.m0, b.m1, &ctx->d_ptB_region, &ctx->ptB_rows, ctx->ptB_row0)))
        return rc;
      ctx->ptB_m0 = b.m0;
      ctx->ptB_m1 = b.m1;
    }
    if (gw::make_slice_map(&mpA, bufA, kmax, std::max<long long>(rowsA, 1), slices, tile, f16) ||
        gw::make_slice_map(&mpB, ctx->d_ptB_region, kmax, std::max<long long>(ctx->ptB_rows, 1), slices, tile,
                           f16))
      return fail(ctx, GW_ERR_CUDA, "cuTensorMapEncodeTiled failed for the streamed panels");
  } else {
    if (gw::make_slice_map(&mpA, ctx->d_pt, kmax, ctx->pt_rows, slices, tile, f16))
      return fail(ctx, GW_ERR_CUDA, "cuTensorMapEncodeTiled failed for the panels");
    mpB = mpA;
  }
  double issued = 0.0;
  cudaEvent_t ea0, ea1;
  if ((rc = c_event_pair(ctx, 2 * batch_idx + 1, &ea0, &ea1))) return rc;
  GW_TRY(cudaEventRecord(ea0, ctx->stream));

  int* d_nao_a;
  if ((rc = upload(ctx, "n_ao_b", ctx->n_ao, &d_nao_a))) return rc;
  // the staged epilogue (two slices) writes whole runs of X and Y: its tiles
  // start at pw boundaries (and at owner atoms for step B's rows), which
  // needs every atom's function count to be at most one tile
  bool staged = ctx->panel_staged && slices == 2;
  for (int a = 0; a < n_at && staged; ++a) staged = ctx->n_ao[a] <= tile;
  // ---- step A: X[P][(s, mu, s')] for the owners of the batch, rows mu of the chunk ----
  {
    const int rows_a = (b.nmu + tile - 1) / tile * tile;
    const int nmt = rows_a / tile;
    std::vector<gw::PanelTaskTC> ta;
    std::vector<int4> tiles;
    // mu tiles of the chunk whose G^occ rows against every lambda atom of
    // the owner's panel are dropped blocks (zero) give exact zeros: X is
    // zeroed before the step, so they are left out.  Their X blocks keep
    // zero norms, and step C never lists their slabs.
    std::vector<char> live(nmt, 1), reach(n_at, 0);
    for (int s = b.s0; s < b.s1; ++s) {
      gw::PanelTaskTC t = ctx->pt_tasks[s];
      if (t.K == 0) continue;
      if (ctx->cur_fo) {
        const std::vector<unsigned char>& fo = *ctx->cur_fo;
        std::fill(reach.begin(), reach.end(), 0);
        for (int i = ctx->wl_off[s]; i < ctx->wl_off[s + 1]; ++i) {
          const size_t a = (size_t)ctx->wl_atom[i] * n_at;
          for (int m = b.m0; m < b.m1; ++m) reach[m] |= fo[a + m];
        }
        for (int mt = 0; mt < nmt; ++mt) {
          const int c0 = b.mu0 + mt * tile, c1 = std::min(b.mu0 + b.nmu, c0 + tile) - 1;
          char on = 0;
          for (int m = ctx->h_atom_of_ao[c0]; m <= ctx->h_atom_of_ao[c1] && !on; ++m) on = reach[m];
          live[mt] = on;
        }
      }
      if (ctx->pt_stream) t.p_row0 = row0A[s];
      t.g_row0 = (int)ta.size() * rows_a;
      t.seg = b.seg[s - b.s0];
      t.s_local = s - b.s0;
      if (staged) {
        // panel rows from pw boundaries: (tile / nsig) whole runs per tile
        const int meff = tile / t.nsig * t.nsig;
        int ntn = 0, nlive = 0;
        for (int ra = 0; ra < t.N; ra += meff, ++ntn)
          for (int mt = 0; mt < nmt; ++mt) {
            if (!live[mt]) continue;
            const int rv = std::min(meff, t.N - ra), cv = std::min(tile, b.nmu - mt * tile);
            tiles.push_back(make_int4((int)ta.size(), ra, mt * tile, (rv << 16) | cv));
            ++nlive;
          }
        issued += 2.0 * tile * tile * 64.0 * t.ksteps * prods * nlive;
      } else {
        const int ntn = (t.N + tile - 1) / tile;
        int nlive = 0;
        for (int nt = 0; nt < ntn; ++nt)
          for (int mt = 0; mt < nmt; ++mt)
            if (live[mt]) {
              tiles.push_back(make_int4((int)ta.size(), nt, mt, 0));
              ++nlive;
            }
        issued += 2.0 * tile * tile * 64.0 * t.ksteps * prods * nlive;
      }
      ta.push_back(t);
    }
    if (!ta.empty()) {
      gw::PanelTaskTC* d_ta;
      int4* d_tiles;
      void* gg;
      if ((rc = upload(ctx, "tc_tasksA", ta, &d_ta))) return rc;
      if ((rc = upload(ctx, "tc_tilesA", tiles, &d_tiles))) return rc;
      const long long g_elems = (long long)ta.size() * rows_a * kmax;
      if ((rc = ws(ctx, "GgA", (size_t)slices * g_elems * 2, &gg))) return rc;
      gw::launch_gather_g(g_occ, ctx->nao, d_ta, (int)ta.size(), ctx->d_lam, b.mu0, b.nmu, rows_a, kmax,
                          slices, g_elems, f16, s_go, gg, ctx->stream);
      GW_CHECK_LAUNCH();
      CUtensorMap mg;
      if (gw::make_slice_map(&mg, gg, kmax, (long long)ta.size() * rows_a, slices, tile, f16))
        return fail(ctx, GW_ERR_CUDA, "cuTensorMapEncodeTiled failed for G (step A)");
      const int lrc =
          staged ? gw::launch_panel_tc_staged(f16, (float)(1.0 / (s_go * s_t)), (float)s_x, mg, mpA, d_tiles,
                                              (int)tiles.size(), d_ta, 0, xs, (long long)prow * Kb, Kb,
                                              b.P0, b.Lc, 0, b.s0, nullptr, bx2, ctx->d_atom_of_ri,
                                              ctx->d_atom_of_ao, ctx->d_ao_off, ctx->d_ri_off, d_nao_a,
                                              npa, pa0, b.mu0, b.m0, nmc, ctx->flush_k, d_err, ctx->stream)
                 : gw::launch_panel_tc(slices, f16, (float)(1.0 / (s_go * s_t)), (float)s_x, mg, mpA, d_tiles,
                                       (int)tiles.size(), d_ta, 0, b.nmu, xs,
                                       (long long)prow * Kb, Kb, b.P0, nullptr, nullptr, nullptr, bx2,
                                       ctx->d_atom_of_ri, ctx->d_atom_of_ao, ctx->d_ao_off, n_at, npa,
                                       pa0, b.mu0, b.m0, nmc, ctx->flush_k, d_err, ctx->stream);
      if (lrc) return fail(ctx, GW_ERR_CUDA, "tensor-core step A launch setup failed");
      GW_CHECK_LAUNCH();
      ctx->stats.kernel_launches += 2;
    }
  }
  // ---- step B: Y[Q][(s, mu, s')] for the panels of the chunk, rows sigma of the batch ----
  {
    const int r0 = ctx->ao_off[b.s0];
    const int R = ctx->ao_off[b.s1] - r0;
    const int rows_b = (R + tile - 1) / tile * tile;
    std::vector<gw::PanelTaskTC> tb;
    std::vector<int4> tiles;
    // staged: batch rows in groups of whole owner atoms, at most one tile each
    std::vector<std::pair<int, int>> groups, group_atoms;
    bool staged_b = staged;
    if (staged_b)
      for (int s = b.s0; s < b.s1;) {
        const int g0 = ctx->ao_off[s] - r0, a0 = s;
        while (s < b.s1 && ctx->ao_off[s + 1] - r0 - g0 <= tile) ++s;
        groups.push_back({g0, ctx->ao_off[s] - r0 - g0});
        group_atoms.push_back({a0, s});
      }
    // every (owner, row group) tile must fit in the staging area
    for (int m = b.m0; m < b.m1 && staged_b; ++m)
      if (ctx->pt_tasks[m].K > 0)
        for (const auto& ga : group_atoms)
          if (!gw::staged_fits_mode1(ctx->n_ao[m], ctx->n_ao.data() + ga.first, ga.second - ga.first)) {
            staged_b = false;
            break;
          }
    // staged: a (row group, owner) pair whose G^virt rows against every
    // lambda atom of the owner's panel are dropped blocks gives exact zeros;
    // its tiles are left out and its Y runs zeroed by a store-only kernel
    // (Y is not zeroed as a whole before the step)
    std::vector<gw::DeadY> dead;
    std::vector<char> reachv(n_at, 0), glive(groups.size(), 1);
    for (int m = b.m0; m < b.m1; ++m) {
      gw::PanelTaskTC t = ctx->pt_tasks[m];
      if (t.K == 0) continue;
      if (ctx->pt_stream) t.p_row0 = ctx->ptB_row0[m];
      t.aom -= b.mu0;  // chunk-local first AO of the panel's owner
      t.g_row0 = (int)tb.size() * rows_b;
      if (staged_b) {
        if (ctx->cur_fv) {
          const std::vector<unsigned char>& fv = *ctx->cur_fv;
          std::fill(reachv.begin(), reachv.end(), 0);
          for (int i = ctx->wl_off[m]; i < ctx->wl_off[m + 1]; ++i) {
            const size_t a = (size_t)ctx->wl_atom[i] * n_at;
            for (int s = b.s0; s < b.s1; ++s) reachv[s] |= fv[a + s];
          }
          for (size_t gi = 0; gi < groups.size(); ++gi) {
            char on = 0;
            for (int s = group_atoms[gi].first; s < group_atoms[gi].second && !on; ++s) on = reachv[s];
            glive[gi] = on;
            if (!on)
              dead.push_back(gw::DeadY{t.p0 - b.Q0, t.npw, group_atoms[gi].first - b.s0,
                                       group_atoms[gi].second - b.s0, t.aom, t.nsig});
          }
        }
        const int meff = tile / t.nsig * t.nsig;  // whole runs of the owner's functions
        int nlive = 0;
        for (int rb = 0; rb < t.N; rb += meff)
          for (size_t gi = 0; gi < groups.size(); ++gi) {
            if (!glive[gi]) continue;
            const auto& g = groups[gi];
            const int cv = std::min(meff, t.N - rb);
            tiles.push_back(make_int4((int)tb.size(), g.first, rb, (g.second << 16) | cv));
            ++nlive;
          }
        issued += 2.0 * tile * tile * 64.0 * t.ksteps * prods * nlive;
      } else {
        const int ntn = (t.N + tile - 1) / tile;
        for (int nt = 0; nt < ntn; ++nt)
          for (int mt = 0; mt < rows_b / tile; ++mt) tiles.push_back(make_int4((int)tb.size(), mt, nt, 0));
        issued += 2.0 * tile * tile * 64.0 * t.ksteps * prods * (rows_b / tile) * ntn;
      }
      tb.push_back(t);
    }
    std::vector<long long> rowbase(R);
    std::vector<int> rowmul(R), rowsl(R);
    for (int s = b.s0; s < b.s1; ++s)
      for (int i = 0; i < ctx->n_ao[s]; ++i) {
        rowbase[ctx->ao_off[s] - r0 + i] = b.seg[s - b.s0] + i;
        rowmul[ctx->ao_off[s] - r0 + i] = ctx->n_ao[s];
        rowsl[ctx->ao_off[s] - r0 + i] = s - b.s0;
      }
    if (!tb.empty() && R > 0) {
      gw::PanelTaskTC* d_tb;
      int4* d_tiles;
      long long* d_rowbase;
      int *d_rowmul, *d_rowsl;
      void* gg;
      if ((rc = upload(ctx, "tc_tasksB", tb, &d_tb))) return rc;
      if ((rc = upload(ctx, "tc_tilesB", tiles, &d_tiles))) return rc;
      if ((rc = upload(ctx, "rowbase", rowbase, &d_rowbase))) return rc;
      if ((rc = upload(ctx, "rowmul", rowmul, &d_rowmul))) return rc;
      if ((rc = upload(ctx, "rowsl", rowsl, &d_rowsl))) return rc;
      const long long g_elems = (long long)tb.size() * rows_b * kmax;
      if ((rc = ws(ctx, "GgB", (size_t)slices * g_elems * 2, &gg))) return rc;
      gw::launch_gather_g(g_virt, ctx->nao, d_tb, (int)tb.size(), ctx->d_lam, r0, R, rows_b, kmax, slices,
                          g_elems, f16, s_gv, gg, ctx->stream);
      GW_CHECK_LAUNCH();
      CUtensorMap mg;
      if (gw::make_slice_map(&mg, gg, kmax, (long long)tb.size() * rows_b, slices, tile, f16))
        return fail(ctx, GW_ERR_CUDA, "cuTensorMapEncodeTiled failed for G (step B)");
      const int lrc =
          staged_b ? gw::launch_panel_tc_staged(f16, (float)(1.0 / (s_gv * s_t)), (float)s_y, mg, mpB, d_tiles,
                                              (int)tiles.size(), d_tb, 1, ys, (long long)qrow * Kb, Kb,
                                              b.Q0, b.Lc, r0, b.s0, d_rowbase, by2, ctx->d_atom_of_ri,
                                              ctx->d_atom_of_ao, ctx->d_ao_off, ctx->d_ri_off, d_nao_a,
                                              nqa, qa0, b.mu0, b.m0, nmc, ctx->flush_k, d_err, ctx->stream)
                 : gw::launch_panel_tc(slices, f16, (float)(1.0 / (s_gv * s_t)), (float)s_y, mg, mpB, d_tiles,
                                       (int)tiles.size(), d_tb, 1, R, ys,
                                       (long long)qrow * Kb, Kb, b.Q0, d_rowbase, d_rowmul, d_rowsl, by2,
                                       ctx->d_atom_of_ri, ctx->d_atom_of_ao, ctx->d_ao_off, n_at, nqa,
                                       qa0, b.mu0, b.m0, nmc, ctx->flush_k, d_err, ctx->stream);
      if (lrc) return fail(ctx, GW_ERR_CUDA, "tensor-core step B launch setup failed");
      GW_CHECK_LAUNCH();
      ctx->stats.kernel_launches += 2;
      if (!dead.empty()) {
        gw::DeadY* d_dead;
        long long* d_segb;
        if ((rc = upload(ctx, "dead_y", dead, &d_dead))) return rc;
        if ((rc = upload(ctx, "seg_b", b.seg, &d_segb))) return rc;
        gw::launch_zero_dead_y(ys, slices, (long long)qrow * Kb, Kb, qrow, d_dead, (int)dead.size(), d_segb,
                               d_nao_a, b.s0, ctx->stream);
        GW_CHECK_LAUNCH();
        ctx->stats.kernel_launches += 1;
      }
    }
  }
  GW_TRY(cudaEventRecord(ea1, ctx->stream));
  ctx->stats.bytes_operands += (double)(prow + qrow) * Kb * 2.0 * slices;

  // ---- block filter, occupancy, task lists ----
  const int nslab = b.nslab;
  const int npt = (prow + tile - 1) / tile, nqt = (qrow + tile - 1) / tile;
  unsigned char *bx, *by, *fx, *fy;
  if ((rc = wsT(ctx, "bx", (size_t)ns * nmc * npa, &bx))) return rc;
  if ((rc = wsT(ctx, "by", (size_t)ns * nmc * nqa, &by))) return rc;
  if ((rc = wsT(ctx, "fx", (size_t)ns * nmc * npt, &fx))) return rc;
  if ((rc = wsT(ctx, "fy", (size_t)ns * nmc * nqt, &fy))) return rc;
  GW_TRY(cudaMemsetAsync(fx, 0, (size_t)ns * nmc * npt, ctx->stream));
  GW_TRY(cudaMemsetAsync(fy, 0, (size_t)ns * nmc * nqt, ctx->stream));
  long long* d_seg;
  int* d_nao;
  if ((rc = upload(ctx, "seg", b.seg, &d_seg))) return rc;
  if ((rc = upload(ctx, "n_ao_b", ctx->n_ao, &d_nao))) return rc;
  // queue of filtered blocks to zero (shared by the two stream-ordered calls)
  int *zlist, *zcount;
  if ((rc = wsT(ctx, "zlist", (size_t)ns * nmc * std::max(npa, nqa), &zlist))) return rc;
  if ((rc = wsT(ctx, "zcount", 1, &zcount))) return rc;
  gw::launch_slices_block_filter(xs, slices, (long long)prow * Kb, Kb, b.P0, ctx->d_ri_off,
                                 ctx->d_ao_off, d_nao, b.s0, ns, d_seg, pa0, npa, b.m0, nmc, b.mu0, thr,
                                 bx2, bx, fx, npt, tile, zlist, zcount, ctx->stream);
  gw::launch_slices_block_filter(ys, slices, (long long)qrow * Kb, Kb, b.Q0, ctx->d_ri_off,
                                 ctx->d_ao_off, d_nao, b.s0, ns, d_seg, qa0, nqa, b.m0, nmc, b.mu0, thr,
                                 by2, by, fy, nqt, tile, zlist, zcount, ctx->stream);
  GW_CHECK_LAUNCH();
  std::vector<long long> slab_k0(nslab);
  std::vector<int> slab_len(nslab);
  const int per = b.Lc / kSlabAO;
  for (int sl = 0; sl < ns; ++sl)
    for (int c = 0; c < per; ++c) {
      const int nsig = ctx->n_ao[b.s0 + sl];
      slab_k0[sl * per + c] = b.seg[sl] + (long long)c * kSlabAO * nsig;
      slab_len[sl * per + c] = kSlabAO * nsig;
    }
  long long* d_k0;
  int* d_len;
  if ((rc = upload(ctx, "slab_k0", slab_k0, &d_k0))) return rc;
  if ((rc = upload(ctx, "slab_len", slab_len, &d_len))) return rc;
  int *tasks, *counts;
  long long* kacc;
  if ((rc = wsT(ctx, "tasks", (size_t)npt * nqt * nslab, &tasks))) return rc;
  if ((rc = wsT(ctx, "counts", (size_t)npt * nqt, &counts))) return rc;
  if ((rc = wsT(ctx, "kacc", (size_t)npt * nqt, &kacc))) return rc;
  gw::launch_build_tasks(fx, fy, nslab, npt, nqt, b.P0, prow, b.Q0, qrow, ctx->d_atom_of_ri, d_len,
                         tasks, counts, kacc, tile, per, b.m0, nmc, b.mu0, b.nmu, ctx->d_atom_of_ao,
                         ctx->stream);
  double* d_fc;
  int* d_nri;
  if ((rc = wsT(ctx, "fc", (size_t)ns * nmc, &d_fc))) return rc;
  if ((rc = upload(ctx, "n_ri_b", ctx->n_ri, &d_nri))) return rc;
  gw::launch_count_c(bx, by, ns, b.m0, nmc, pa0, npa, qa0, nqa, d_nri, d_nao, b.s0, d_fc, ctx->stream);
  GW_CHECK_LAUNCH();
  // two block filters of two kernels each, the task lists and the count
  ctx->stats.kernel_launches += 6;
  double fc_scale = 1.0;
  if (ctx->mlp_mode) {
    gw::MlpBatch mb{};
    mb.s0 = b.s0;
    mb.ns = ns;
    mb.P0 = b.P0;
    mb.prow = prow;
    mb.nslab = nslab;
    mb.npt = npt;
    mb.nqt = nqt;
    mb.tile = tile;
    mb.per = per;
    mb.pa0 = pa0;
    mb.npa = npa;
    mb.slices = slices;
    mb.m0 = b.m0;
    mb.nmc = nmc;
    mb.mu0 = b.mu0;
    mb.nmu = b.nmu;
    mb.Q0 = b.Q0;
    mb.qrow = qrow;
    mb.qa0 = qa0;
    mb.nqa = nqa;
    mb.f16 = f16;
    mb.xinv = (float)(1.0 / s_x);
    mb.yinv = (float)(1.0 / s_y);
    mb.Kb = Kb;
    mb.xs = xs;
    mb.ys = ys;
    mb.bx2 = bx2;
    mb.by2 = by2;
    mb.bx = bx;
    mb.by = by;
    mb.tasks = tasks;
    mb.counts = counts;
    mb.kacc = kacc;
    mb.slab_k0 = d_k0;
    mb.slab_len = d_len;
    mb.tau = ctx->cur_tau;
    mb.thr = thr;
    const double kb0 = ctx->mlp_k_before, ka0 = ctx->mlp_k_after;
    if ((rc = gw::mlp_batch_hook(ctx, mb))) return rc;
    // learned skips are not credited as useful work: step C's count is
    // scaled by the fraction of its reduction length that is still issued
    if (ctx->mlp_mode == 2 && ctx->mlp_k_before > kb0)
      fc_scale = (ctx->mlp_k_after - ka0) / (ctx->mlp_k_before - kb0);
    ctx->stats.kernel_launches += 4;
  }
  CUtensorMap mx, my;
  if (gw::make_slice_map(&mx, xs, Kb, prow, slices, tile, f16) ||
      gw::make_slice_map(&my, ys, Kb, qrow, slices, tile, f16))
    return fail(ctx, GW_ERR_CUDA, "cuTensorMapEncodeTiled failed for the step-C operands");
  cudaEvent_t ec0, ec1;
  if ((rc = c_event_pair(ctx, 2 * batch_idx, &ec0, &ec1))) return rc;
  const double fc_scale_dev = fc_scale;
  if (ctx->c_split_k > 0 && !ctx->mlp_mode) {
    // step-C work units planned on the device: no host synchronisation; the
    // task statistics are read at the end of the tau point
    const int ntiles = npt * nqt;
    const size_t cap = std::max<size_t>((size_t)ntiles * nslab, 1);
    gw::UnitScratch w{};
    unsigned long long* tstat;
    if ((rc = wsT(ctx, "u_ucnt", std::max(ntiles, 1), &w.ucnt)) ||
        (rc = wsT(ctx, "u_uoff", std::max(ntiles, 1), &w.uoff)) ||
        (rc = wsT(ctx, "u_ttile", cap, &w.t_tile)) || (rc = wsT(ctx, "u_tfirst", cap, &w.t_first)) ||
        (rc = wsT(ctx, "u_tcount", cap, &w.t_count)) || (rc = wsT(ctx, "u_tkey", cap, &w.t_key)) ||
        (rc = wsT(ctx, "u_tile", cap, &w.u_tile)) || (rc = wsT(ctx, "u_first", cap, &w.u_first)) ||
        (rc = wsT(ctx, "u_count", cap, &w.u_count)) ||
        (rc = wsT(ctx, "u_hist", std::max(nslab, 1), &w.hist)) ||
        (rc = wsT(ctx, "u_start", std::max(nslab, 1), &w.start)) ||
        (rc = wsT(ctx, "u_nunits", 1, &w.n_units)) || (rc = wsT(ctx, "u_nkeys", 1, &w.total_keys)) ||
        (rc = wsT(ctx, "task_stats", 3, &tstat)))
      return rc;
    gw::launch_plan_units(tasks, counts, kacc, d_len, ntiles, nslab, ctx->c_split_k, w, tstat,
                          ctx->stream);
    GW_CHECK_LAUNCH();
    ctx->stats.kernel_launches += 5;
    ctx->tc_issue_per_k = 2.0 * tile * tile * prods;
    GW_TRY(cudaEventRecord(ec0, ctx->stream));
    int* d_work;  // the units' counter (zeroed by the launch)
    if ((rc = wsT(ctx, "tc_work", 1, &d_work))) return rc;
    if (gw::launch_chi_tc_units(slices, f16, (float)(1.0 / (s_x * s_y)), mx, my, w.u_tile, w.u_first,
                                w.u_count, (int)std::min<size_t>(cap, INT32_MAX), w.n_units, tasks,
                                counts, nslab, d_k0, d_len, b.P0, prow, nri, b.Q0, qrow, nqt, acc,
                                ctx->flush_k, ctx->c_dynamic ? d_work : nullptr, d_err, ctx->stream))
      return fail(ctx, GW_ERR_CUDA, "tensor-core step C launch setup failed");
    GW_CHECK_LAUNCH();
    GW_TRY(cudaEventRecord(ec1, ctx->stream));
    ctx->stats.c_launches += 1;
    ctx->stats.kernel_launches += 1;
    double* d_fc_all;
    if ((rc = wsT(ctx, "fc_all", (size_t)n_at * n_at, &d_fc_all))) return rc;
    GW_TRY(cudaMemcpyAsync(d_fc_all + ctx->tc_fc_used, d_fc, (size_t)ns * nmc * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->tc_pending.push_back({batch_idx, ctx->tc_fc_used, ns * nmc, fc_scale_dev});
    ctx->tc_fc_used += (long long)ns * nmc;
    ctx->stats.tiles_total += (long long)ntiles;
    ctx->stats.slabs_total += (long long)ntiles * nslab;
    ctx->stats.flops_issued += issued;
    return GW_OK;
  }
  std::vector<int> h_counts((size_t)npt * nqt);
  std::vector<long long> h_kacc((size_t)npt * nqt);
  GW_TRY(cudaMemcpyAsync(h_counts.data(), counts, h_counts.size() * sizeof(int),
                         cudaMemcpyDeviceToHost, ctx->stream));
  GW_TRY(cudaMemcpyAsync(h_kacc.data(), kacc, h_kacc.size() * sizeof(long long),
                         cudaMemcpyDeviceToHost, ctx->stream));
  GW_TRY(cudaStreamSynchronize(ctx->stream));
  // active tiles in the order the persistent CTAs take them round-robin:
  // longest first (c_order 0), or grouped raster (c_order 1: groups of 8 row
  // tiles swept along the columns, so that CTAs running side by side share
  // operand tiles in L2)
  std::vector<int> active;
  for (size_t t = 0; t < h_counts.size(); ++t)
    if (h_counts[t] > 0) active.push_back((int)t);
  if (ctx->c_order == 1) {
    std::stable_sort(active.begin(), active.end(), [&](int a, int c) {
      const int pa = a / nqt, qa = a % nqt, pc = c / nqt, qc = c % nqt;
      if (pa / 8 != pc / 8) return pa / 8 < pc / 8;
      if (qa != qc) return qa < qc;
      return pa < pc;
    });
  } else {
    std::stable_sort(active.begin(), active.end(),
                     [&](int a, int c) { return h_kacc[a] > h_kacc[c]; });
  }
  if (ctx->c_split_k > 0) {
    // split every tile's list into units of about c_split_k reduction
    // elements
    std::vector<int> h_tasks((size_t)npt * nqt * nslab);
    GW_TRY(cudaMemcpy(h_tasks.data(), tasks, h_tasks.size() * sizeof(int), cudaMemcpyDeviceToHost));
    // active tiles in grouped raster order (groups of 8 row tiles swept
    // along the columns)
    std::vector<int> raster;
    for (int pg = 0; pg < npt; pg += 8)
      for (int qt = 0; qt < nqt; ++qt)
        for (int pt = pg; pt < std::min(npt, pg + 8); ++pt)
          if (h_counts[(size_t)pt * nqt + qt] > 0) raster.push_back(pt * nqt + qt);
    // units: runs of a tile's slab list of about c_split_k elements, keyed by
    // their first slab (slab ids follow the reduction index)
    std::vector<int> r_tile, r_first, r_count, r_key;
    for (const int t : raster) {
      const int* lst = &h_tasks[(size_t)t * nslab];
      int i0 = 0;
      long long kk = 0;
      for (int i = 0; i < h_counts[t]; ++i) {
        kk += slab_len[lst[i]];
        if (kk >= ctx->c_split_k || i == h_counts[t] - 1) {
          r_tile.push_back(t);
          r_first.push_back(i0);
          r_count.push_back(i + 1 - i0);
          r_key.push_back(lst[i0]);
          i0 = i + 1;
          kk = 0;
        }
      }
    }
    // order by first reduction index, raster order among equal keys
    // (counting sort): CTAs that run side by side stream the same K window
    // of X and Y through L2
    std::vector<int> start((size_t)nslab + 1, 0);
    for (const int k : r_key) ++start[(size_t)k + 1];
    for (int k = 0; k < nslab; ++k) start[(size_t)k + 1] += start[k];
    const size_t nu = r_key.size();
    std::vector<int> u_tile(nu), u_first(nu), u_count(nu);
    for (size_t u = 0; u < nu; ++u) {
      const int pos = start[r_key[u]]++;
      u_tile[pos] = r_tile[u];
      u_first[pos] = r_first[u];
      u_count[pos] = r_count[u];
    }
    int *d_ut, *d_uf, *d_uc;
    if ((rc = upload(ctx, "unit_tile", u_tile, &d_ut))) return rc;
    if ((rc = upload(ctx, "unit_first", u_first, &d_uf))) return rc;
    if ((rc = upload(ctx, "unit_count", u_count, &d_uc))) return rc;
    int* d_work;  // the units' counter (zeroed by the launch)
    if ((rc = wsT(ctx, "tc_work", 1, &d_work))) return rc;
    GW_TRY(cudaEventRecord(ec0, ctx->stream));
    if (gw::launch_chi_tc_units(slices, f16, (float)(1.0 / (s_x * s_y)), mx, my, d_ut, d_uf, d_uc,
                                (int)u_tile.size(), nullptr, tasks, counts,
                                nslab, d_k0, d_len, b.P0, prow, nri, b.Q0, qrow, nqt, acc, ctx->flush_k,
                                ctx->c_dynamic ? d_work : nullptr, d_err, ctx->stream))
      return fail(ctx, GW_ERR_CUDA, "tensor-core step C launch setup failed");
  } else {
    int* d_active;
    if ((rc = upload(ctx, "active_tiles", active, &d_active))) return rc;
    GW_TRY(cudaEventRecord(ec0, ctx->stream));
    if (gw::launch_chi_tc(slices, f16, (float)(1.0 / (s_x * s_y)), mx, my, d_active,
                          (int)active.size(), tasks, counts, nslab, d_k0,
                          d_len, b.P0, prow, nri, b.Q0, qrow, nqt, acc, ctx->flush_k, d_err,
                          ctx->stream))
      return fail(ctx, GW_ERR_CUDA, "tensor-core step C launch setup failed");
  }
  GW_CHECK_LAUNCH();
  GW_TRY(cudaEventRecord(ec1, ctx->stream));
  ctx->stats.c_launches += 1;
  ctx->stats.kernel_launches += 1;
  // this batch's flop counts, error flag and timings are read at the end of
  // the tau point (tc_finish_tau), so the next batch is queued without a wait
  double* d_fc_all;  // sized n_at * n_at by gw_chi_tau
  if ((rc = wsT(ctx, "fc_all", (size_t)n_at * n_at, &d_fc_all))) return rc;
  GW_TRY(cudaMemcpyAsync(d_fc_all + ctx->tc_fc_used, d_fc, (size_t)ns * nmc * sizeof(double),
                         cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->tc_pending.push_back({batch_idx, ctx->tc_fc_used, ns * nmc, fc_scale});
  ctx->tc_fc_used += (long long)ns * nmc;
  long long act = 0, sl_act = 0;
  double ksum = 0.0;
  for (size_t t = 0; t < h_counts.size(); ++t) {
    act += h_counts[t] > 0;
    sl_act += h_counts[t];
    ksum += (double)h_kacc[t];
  }
  ctx->stats.tiles_total += (long long)npt * nqt;
  ctx->stats.tiles_active += act;
  ctx->stats.slabs_total += (long long)npt * nqt * nslab;
  ctx->stats.slabs_active += sl_act;
  (void)fc_host;
  ctx->stats.flops_issued += issued + 2.0 * tile * tile * ksum * prods;
  return GW_OK;
}

// Start of a tau point on the tensor-core route: error flag and flop-count
// staging for its batches.
int tc_begin_tau(gw_ctx* ctx) {
  int* d_err;
  double* d_fc_all;
  int rc;
  if ((rc = wsT(ctx, "tc_err", 1, &d_err))) return rc;
  if ((rc = wsT(ctx, "fc_all", (size_t)ctx->n_at * ctx->n_at, &d_fc_all))) return rc;
  GW_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), ctx->stream));
  unsigned long long* tstat;
  if ((rc = wsT(ctx, "task_stats", 3, &tstat))) return rc;
  GW_TRY(cudaMemsetAsync(tstat, 0, 3 * sizeof(unsigned long long), ctx->stream));
  ctx->tc_pending.clear();
  ctx->tc_fc_used = 0;
  ctx->tc_issue_per_k = 0.0;
  return GW_OK;
}

// End of a tau point (after the stream is synchronised): error flag, step
// timings and step-C flop counts of its tensor-core batches.
int tc_finish_tau(gw_ctx* ctx, std::vector<double>& fc_host) {
  int* d_err;
  double* d_fc_all;
  int rc;
  if ((rc = wsT(ctx, "tc_err", 1, &d_err))) return rc;
  if ((rc = wsT(ctx, "fc_all", (size_t)ctx->n_at * ctx->n_at, &d_fc_all))) return rc;
  int h_err = 0;
  GW_TRY(cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h_err)
    return fail(ctx, GW_ERR_TIMEOUT,
                "tensor-core kernel: a bounded wait gave up (flags " + std::to_string(h_err) + ")");
  std::vector<double> h_fc((size_t)ctx->tc_fc_used);
  if (!h_fc.empty())
    GW_TRY(cudaMemcpy(h_fc.data(), d_fc_all, h_fc.size() * sizeof(double), cudaMemcpyDeviceToHost));
  // task statistics of the batches whose units were planned on the device
  unsigned long long* tstat;
  unsigned long long h_stat[3] = {0, 0, 0};
  if ((rc = wsT(ctx, "task_stats", 3, &tstat))) return rc;
  GW_TRY(cudaMemcpy(h_stat, tstat, sizeof(h_stat), cudaMemcpyDeviceToHost));
  ctx->stats.tiles_active += (long long)h_stat[0];
  ctx->stats.slabs_active += (long long)h_stat[1];
  ctx->stats.flops_issued += ctx->tc_issue_per_k * (double)h_stat[2];
  for (const auto& p : ctx->tc_pending) {
    cudaEvent_t ec0, ec1, ea0, ea1;
    if ((rc = c_event_pair(ctx, 2 * p.batch_idx, &ec0, &ec1))) return rc;
    if ((rc = c_event_pair(ctx, 2 * p.batch_idx + 1, &ea0, &ea1))) return rc;
    float ms_ck = 0.f, ms_ab = 0.f;
    GW_TRY(cudaEventElapsedTime(&ms_ck, ec0, ec1));
    GW_TRY(cudaEventElapsedTime(&ms_ab, ea0, ea1));
    ctx->stats.ms_step_c_kernel += ms_ck;
    ctx->stats.ms_step_ab += ms_ab;
    for (int i = 0; i < p.fc_n; ++i) fc_host.push_back(h_fc[(size_t)p.fc_off + i] * p.fc_scale);
  }
  ctx->tc_pending.clear();
  ctx->tc_fc_used = 0;
  return GW_OK;
}

}  // namespace

namespace gw {
int build_panels_for(gw_ctx* ctx, double thr) { return build_panels(ctx, thr); }
}  // namespace gw

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int gw_create(gw_ctx** out, int device, void* cuda_stream) {
  if (!out) return GW_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GW_ERR_INVALID_ARG;
  }
  gw_ctx* ctx = new gw_ctx();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return GW_ERR_CUDA;
  }
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return GW_ERR_CUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return GW_OK;
}

void gw_destroy(gw_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  reset_tensor(ctx);
  reset_greens(ctx);
  free_dev(ctx->d_ao_off);
  free_dev(ctx->d_ri_off);
  free_dev(ctx->d_atom_of_ri);
  free_dev(ctx->d_atom_of_ao);
  free_dev(ctx->d_mlp_theta);
  free_dev(ctx->d_mlp_wb);
  free_dev(ctx->d_mlp_m);
  free_dev(ctx->d_mlp_v);
  free_dev(ctx->d_ycov_lo);
  free_dev(ctx->d_ycov_hi);
  for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
  ctx->events.clear();
  for (auto& kv : ctx->work) free_dev(kv.second.first);
  ctx->work.clear();
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* gw_last_error(const gw_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int gw_set_basis(gw_ctx* ctx, int n_atoms, const double* xyz, const int* n_ao, const int* n_ri) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (n_atoms <= 0 || !xyz || !n_ao || !n_ri) return fail(ctx, GW_ERR_INVALID_ARG, "set_basis: bad arguments");
  long long nao = 0, nri = 0;
  for (int a = 0; a < n_atoms; ++a) {
    if (n_ao[a] <= 0 || n_ri[a] <= 0 || n_ao[a] > 4096 || n_ri[a] > 4096)
      return fail(ctx, GW_ERR_INVALID_ARG, "set_basis: per-atom sizes must be in 1..4096");
    if (!std::isfinite(xyz[3 * a]) || !std::isfinite(xyz[3 * a + 1]) || !std::isfinite(xyz[3 * a + 2]))
      return fail(ctx, GW_ERR_NONFINITE, "set_basis: non-finite coordinate");
    nao += n_ao[a];
    nri += n_ri[a];
  }
  if (nao > 1000000 || nri > 1000000) return fail(ctx, GW_ERR_INVALID_ARG, "set_basis: basis too large");
  GW_TRY(cudaSetDevice(ctx->device));
  reset_tensor(ctx);
  reset_greens(ctx);
  ctx->n_at = n_atoms;
  ctx->xyz.assign(xyz, xyz + 3 * n_atoms);
  ctx->n_ao.assign(n_ao, n_ao + n_atoms);
  ctx->n_ri.assign(n_ri, n_ri + n_atoms);
  ctx->ao_off.assign(n_atoms + 1, 0);
  ctx->ri_off.assign(n_atoms + 1, 0);
  for (int a = 0; a < n_atoms; ++a) {
    ctx->ao_off[a + 1] = ctx->ao_off[a] + n_ao[a];
    ctx->ri_off[a + 1] = ctx->ri_off[a] + n_ri[a];
  }
  ctx->nao = (int)nao;
  ctx->nri = (int)nri;
  ctx->naop = (int)((nao + kSlabAO - 1) / kSlabAO * kSlabAO);
  std::vector<int> atom_of_ri(nri), atom_of_ao(nao);
  for (int a = 0; a < n_atoms; ++a) {
    for (int i = ctx->ri_off[a]; i < ctx->ri_off[a + 1]; ++i) atom_of_ri[i] = a;
    for (int i = ctx->ao_off[a]; i < ctx->ao_off[a + 1]; ++i) atom_of_ao[i] = a;
  }
  ctx->h_atom_of_ao = atom_of_ao;
  free_dev(ctx->d_ao_off);
  free_dev(ctx->d_ri_off);
  free_dev(ctx->d_atom_of_ri);
  free_dev(ctx->d_atom_of_ao);
  GW_TRY(cudaMalloc(&ctx->d_ao_off, (n_atoms + 1) * sizeof(int)));
  GW_TRY(cudaMalloc(&ctx->d_ri_off, (n_atoms + 1) * sizeof(int)));
  GW_TRY(cudaMalloc(&ctx->d_atom_of_ri, nri * sizeof(int)));
  GW_TRY(cudaMalloc(&ctx->d_atom_of_ao, nao * sizeof(int)));
  GW_TRY(cudaMemcpy(ctx->d_ao_off, ctx->ao_off.data(), (n_atoms + 1) * sizeof(int), cudaMemcpyHostToDevice));
  GW_TRY(cudaMemcpy(ctx->d_ri_off, ctx->ri_off.data(), (n_atoms + 1) * sizeof(int), cudaMemcpyHostToDevice));
  GW_TRY(cudaMemcpy(ctx->d_atom_of_ri, atom_of_ri.data(), nri * sizeof(int), cudaMemcpyHostToDevice));
  GW_TRY(cudaMemcpy(ctx->d_atom_of_ao, atom_of_ao.data(), nao * sizeof(int), cudaMemcpyHostToDevice));
  return GW_OK;
}

int gw_set_3c_tensor(gw_ctx* ctx, long long n_blocks, const int* blk_abp, const double* data,
                     long long n_elems) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_at == 0) return fail(ctx, GW_ERR_ORDER, "set_3c_tensor: call gw_set_basis first");
  if (n_blocks < 0 || n_elems < 0 || (n_blocks > 0 && (!blk_abp || !data)))
    return fail(ctx, GW_ERR_INVALID_ARG, "set_3c_tensor: bad arguments");
  GW_TRY(cudaSetDevice(ctx->device));
  reset_tensor(ctx);
  std::vector<long long> off(n_blocks + 1, 0);
  long long prev = -1;
  for (long long b = 0; b < n_blocks; ++b) {
    int A = blk_abp[3 * b], B = blk_abp[3 * b + 1], P = blk_abp[3 * b + 2];
    if (A < 0 || B < 0 || P < 0 || A >= ctx->n_at || B >= ctx->n_at || P >= ctx->n_at || A > B)
      return fail(ctx, GW_ERR_INVALID_ARG,
                  "set_3c_tensor: block " + std::to_string(b) + " has an atom index out of range or A > B");
    long long key = ((long long)A * ctx->n_at + B) * ctx->n_at + P;
    if (key <= prev)
      return fail(ctx, GW_ERR_INVALID_ARG,
                  "set_3c_tensor: blocks must be sorted by (A, B, P) without duplicates");
    prev = key;
    off[b + 1] = off[b] + (long long)ctx->n_ao[A] * ctx->n_ao[B] * ctx->n_ri[P];
  }
  if (off[n_blocks] != n_elems)
    return fail(ctx, GW_ERR_INVALID_ARG,
                "set_3c_tensor: n_elems " + std::to_string(n_elems) + " does not match the block sizes (" +
                    std::to_string(off[n_blocks]) + ")");
  ctx->blk.assign(blk_abp, blk_abp + 3 * n_blocks);
  ctx->blk_off = off;
  ctx->n_blocks = n_blocks;
  ctx->n_elems = n_elems;
  GW_TRY(cudaMalloc(&ctx->d_blk, std::max<long long>(3 * n_blocks, 1) * sizeof(int)));
  GW_TRY(cudaMalloc(&ctx->d_blk_off, (n_blocks + 1) * sizeof(long long)));
  GW_TRY(cudaMalloc(&ctx->d_blk_norm, std::max<long long>(n_blocks, 1) * sizeof(double)));
  if (n_blocks > 0) {
    GW_TRY(cudaMemcpyAsync(ctx->d_blk, blk_abp, 3 * n_blocks * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  }
  GW_TRY(cudaMemcpyAsync(ctx->d_blk_off, off.data(), (n_blocks + 1) * sizeof(long long),
                         cudaMemcpyHostToDevice, ctx->stream));
  int* d_bad;
  int rc;
  if ((rc = wsT(ctx, "bad", 1, &d_bad))) return rc;
  GW_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), ctx->stream));
  int *d_nao, *d_nri;
  if ((rc = upload(ctx, "n_ao", ctx->n_ao, &d_nao))) return rc;
  if ((rc = upload(ctx, "n_ri", ctx->n_ri, &d_nri))) return rc;
  if (!ctx->tensor_fp32) {
    GW_TRY(cudaMalloc(&ctx->d_t3, std::max<long long>(n_elems, 1) * sizeof(double)));
    // copy in chunks of 1 GiB (pageable host memory)
    const long long chunk = 1LL << 27;
    for (long long i = 0; i < n_elems; i += chunk) {
      long long n = std::min(chunk, n_elems - i);
      GW_TRY(cudaMemcpyAsync(ctx->d_t3 + i, data + i, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    }
    gw::launch_block_norms_3c(ctx->d_t3, 0, ctx->d_blk, ctx->d_blk_off, d_nao, d_nri, n_blocks,
                              ctx->d_blk_norm, d_bad, ctx->stream);
    GW_CHECK_LAUNCH();
  } else {
    // FP32 copy on the device: runs of whole blocks (up to 1 GiB of FP64, or
    // one block) pass through an FP64 staging buffer, where their norms,
    // finiteness and symmetry are taken before the cast
    GW_TRY(cudaMalloc(&ctx->d_t3f, std::max<long long>(n_elems, 1) * sizeof(float)));
    const long long chunk = 1LL << 27;
    long long max_run = 1;
    for (long long b0 = 0; b0 < n_blocks;) {
      long long b1 = b0 + 1;
      while (b1 < n_blocks && off[b1 + 1] - off[b0] <= chunk) ++b1;
      max_run = std::max(max_run, off[b1] - off[b0]);
      b0 = b1;
    }
    double* stage;
    if ((rc = wsT(ctx, "t3_stage", (size_t)max_run, &stage))) return rc;
    for (long long b0 = 0; b0 < n_blocks;) {
      long long b1 = b0 + 1;
      while (b1 < n_blocks && off[b1 + 1] - off[b0] <= chunk) ++b1;
      const long long n = off[b1] - off[b0];
      GW_TRY(cudaMemcpyAsync(stage, data + off[b0], n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      gw::launch_block_norms_3c(stage, off[b0], ctx->d_blk + 3 * b0, ctx->d_blk_off + b0, d_nao, d_nri,
                                b1 - b0, ctx->d_blk_norm + b0, d_bad, ctx->stream);
      gw::launch_cast_f64_f32(stage, ctx->d_t3f + off[b0], n, ctx->stream);
      GW_CHECK_LAUNCH();
      b0 = b1;
    }
    // the staging buffer is needed only here
    GW_TRY(cudaStreamSynchronize(ctx->stream));
    auto it = ctx->work.find("t3_stage");
    if (it != ctx->work.end()) {
      cudaFree(it->second.first);
      ctx->work.erase(it);
    }
  }
  int bad = 0;
  ctx->blk_norm.resize(n_blocks);
  GW_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (n_blocks > 0)
    GW_TRY(cudaMemcpyAsync(ctx->blk_norm.data(), ctx->d_blk_norm, n_blocks * sizeof(double),
                           cudaMemcpyDeviceToHost, ctx->stream));
  GW_TRY(cudaStreamSynchronize(ctx->stream));
  if (bad & 1) {
    reset_tensor(ctx);
    return fail(ctx, GW_ERR_NONFINITE, "set_3c_tensor: NaN or Inf in the tensor data");
  }
  if (bad & 2) {
    reset_tensor(ctx);
    return fail(ctx, GW_ERR_ASYM, "set_3c_tensor: an (A, A, P) block is not symmetric in its primary indices");
  }
  return GW_OK;
}

int gw_set_greens(gw_ctx* ctx, const double* C, const double* eps, int n_occ, double mu_fermi,
                  const double* tau, int n_tau) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_at == 0) return fail(ctx, GW_ERR_ORDER, "set_greens: call gw_set_basis first");
  const int nao = ctx->nao;
  if (!C || !eps || !tau || n_tau <= 0 || n_occ < 0 || n_occ > nao)
    return fail(ctx, GW_ERR_INVALID_ARG, "set_greens: bad arguments");
  if (!std::isfinite(mu_fermi)) return fail(ctx, GW_ERR_NONFINITE, "set_greens: mu_fermi not finite");
  for (int j = 0; j < n_tau; ++j)
    if (!(tau[j] > 0.0) || !std::isfinite(tau[j]))
      return fail(ctx, GW_ERR_INVALID_ARG, "set_greens: tau points must be finite and > 0");
  for (int i = 0; i < nao; ++i)
    if (!std::isfinite(eps[i])) return fail(ctx, GW_ERR_NONFINITE, "set_greens: non-finite orbital energy");
  for (long long i = 0; i < (long long)nao * nao; ++i)
    if (!std::isfinite(C[i])) return fail(ctx, GW_ERR_NONFINITE, "set_greens: non-finite orbital coefficient");
  GW_TRY(cudaSetDevice(ctx->device));
  reset_greens(ctx);
  GW_TRY(cudaMalloc(&ctx->d_C, (size_t)nao * nao * sizeof(double)));
  GW_TRY(cudaMalloc(&ctx->d_eps, (size_t)nao * sizeof(double)));
  GW_TRY(cudaMemcpyAsync(ctx->d_C, C, (size_t)nao * nao * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  GW_TRY(cudaMemcpyAsync(ctx->d_eps, eps, (size_t)nao * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  GW_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->n_occ = n_occ;
  ctx->mu = mu_fermi;
  ctx->tau.assign(tau, tau + n_tau);
  ctx->h_eps.assign(eps, eps + nao);
  ctx->have_greens = true;
  return GW_OK;
}

int gw_set_option(gw_ctx* ctx, const char* key, double value) {
  if (!ctx || !key) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!strcmp(key, "batch_bytes")) {
    if (!(value >= 1e6)) return fail(ctx, GW_ERR_INVALID_ARG, "batch_bytes must be >= 1e6");
    ctx->batch_bytes = value;
    return GW_OK;
  }
  if (!strcmp(key, "test_fail_alloc")) {
    ctx->test_fail_alloc = value != 0.0;
    return GW_OK;
  }
  if (!strcmp(key, "test_stall_tc")) {
    ctx->test_stall = value != 0.0;
    return GW_OK;
  }
  if (!strcmp(key, "c_dynamic")) {
    if (value != 0 && value != 1) return fail(ctx, GW_ERR_INVALID_ARG, "c_dynamic must be 0 or 1");
    ctx->c_dynamic = (int)value;
    return GW_OK;
  }
  if (!strcmp(key, "c_split_k")) {
    if (!(value >= 0 && value <= (1 << 30))) return fail(ctx, GW_ERR_INVALID_ARG, "c_split_k must be in [0, 2^30]");
    ctx->c_split_k = (int)value;
    return GW_OK;
  }
  if (!strcmp(key, "c_order")) {
    if (value != 0 && value != 1) return fail(ctx, GW_ERR_INVALID_ARG, "c_order must be 0 or 1");
    ctx->c_order = (int)value;
    return GW_OK;
  }
  if (!strcmp(key, "mlp_margin")) {
    if (!std::isfinite(value)) return fail(ctx, GW_ERR_INVALID_ARG, "mlp_margin must be finite");
    ctx->mlp_margin = value;
    return GW_OK;
  }
  if (!strcmp(key, "flush_k")) {
    if (!(value >= 16 && value <= (1 << 30))) return fail(ctx, GW_ERR_INVALID_ARG, "flush_k must be in [16, 2^30]");
    ctx->flush_k = (int)value;
    return GW_OK;
  }
  if (!strcmp(key, "panel_stream")) {
    if (value != 0 && value != 1) return fail(ctx, GW_ERR_INVALID_ARG, "panel_stream must be 0 or 1");
    ctx->panel_stream = (int)value;
    ctx->pt_ok = false;
    return GW_OK;
  }
  if (!strcmp(key, "tensor_fp32")) {
    if (value != 0 && value != 1) return fail(ctx, GW_ERR_INVALID_ARG, "tensor_fp32 must be 0 or 1");
    ctx->tensor_fp32 = (int)value;
    return GW_OK;
  }
  if (!strcmp(key, "panel_staged")) {
    if (value != 0 && value != 1) return fail(ctx, GW_ERR_INVALID_ARG, "panel_staged must be 0 or 1");
    ctx->panel_staged = (int)value;
    return GW_OK;
  }
  if (!strcmp(key, "mu_chunk_atoms")) {
    if (!(value >= 0 && value <= 1e9)) return fail(ctx, GW_ERR_INVALID_ARG, "mu_chunk_atoms must be >= 0");
    ctx->mu_chunk_atoms = (int)value;
    return GW_OK;
  }
  if (!strcmp(key, "batch_atoms")) {
    if (!(value >= 0)) return fail(ctx, GW_ERR_INVALID_ARG, "batch_atoms must be >= 0");
    ctx->batch_atoms = (int)value;
    return GW_OK;
  }
  return fail(ctx, GW_ERR_INVALID_ARG, std::string("unknown option '") + key + "'");
}

int gw_mlp_log(gw_ctx* ctx, int tau_first, int tau_count, double thr, int precision, float* feat_out,
               float* target_out, long long cap, long long* n_out) {
  if (!ctx || !n_out || cap < 0 || (cap > 0 && (!feat_out || !target_out))) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (precision != GW_BF16X3 && precision != GW_BF16X6 && precision != GW_FP16X3)
    return fail(ctx, GW_ERR_UNSUPPORTED, "gw_mlp_log: tasks are logged on the tensor-core route");
  if (tau_count < 0 || tau_first < 0 || tau_first + tau_count > (int)ctx->tau.size())
    return fail(ctx, GW_ERR_INVALID_ARG, "gw_mlp_log: tau range out of bounds");
  GW_TRY(cudaSetDevice(ctx->device));
  double* chi = nullptr;
  GW_TRY(cudaMalloc(&chi, std::max<size_t>((size_t)tau_count * ctx->nri * ctx->nri, 1) * sizeof(double)));
  ctx->mlp_log_feat.clear();
  ctx->mlp_log_tgt.clear();
  ctx->mlp_mode = 1;
  int rc = gw_chi_tau(ctx, tau_first, tau_count, thr, precision, GW_SCREEN_BOUND, chi, 1);
  ctx->mlp_mode = 0;
  cudaFree(chi);
  if (rc) return rc;
  const long long n = (long long)ctx->mlp_log_tgt.size();
  *n_out = n;
  const long long m = std::min(n, cap);
  if (m > 0) {
    std::memcpy(feat_out, ctx->mlp_log_feat.data(), (size_t)m * gw::kMlpFeatures * sizeof(float));
    std::memcpy(target_out, ctx->mlp_log_tgt.data(), (size_t)m * sizeof(float));
  }
  return GW_OK;
}

int gw_get_stats(const gw_ctx* ctx, gw_stats* out) {
  if (!ctx || !out) return GW_ERR_INVALID_ARG;
  *out = ctx->stats;
  return GW_OK;
}

int gw_chi_tau(gw_ctx* ctx, int tau_first, int tau_count, double thr, int precision, int screening,
               double* chi_out, int out_on_device) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_chi_tau");
  ctx->err.clear();
  if (ctx->n_at == 0 || (ctx->d_t3 == nullptr && ctx->d_t3f == nullptr && ctx->n_blocks > 0))
    return fail(ctx, GW_ERR_ORDER, "chi_tau: call gw_set_basis and gw_set_3c_tensor first");
  if (ctx->blk_off.empty()) return fail(ctx, GW_ERR_ORDER, "chi_tau: call gw_set_3c_tensor first");
  if (!ctx->have_greens) return fail(ctx, GW_ERR_ORDER, "chi_tau: call gw_set_greens first");
  if (tau_first < 0 || tau_count < 0 || tau_first + tau_count > (int)ctx->tau.size())
    return fail(ctx, GW_ERR_INVALID_ARG, "chi_tau: tau range out of bounds");
  if (!(thr >= 0.0) || !std::isfinite(thr)) return fail(ctx, GW_ERR_INVALID_ARG, "chi_tau: thr must be finite and >= 0");
  if (precision < GW_FP64 || precision > GW_FP16X3)
    return fail(ctx, GW_ERR_INVALID_ARG, "chi_tau: unknown precision");
  if (screening != GW_SCREEN_BOUND && screening != GW_SCREEN_MLP)
    return fail(ctx, GW_ERR_INVALID_ARG, "chi_tau: unknown screening mode");
  const bool tc_prec = precision == GW_BF16X3 || precision == GW_BF16X6 || precision == GW_FP16X3;
  if (screening == GW_SCREEN_MLP && !tc_prec)
    return fail(ctx, GW_ERR_UNSUPPORTED,
                "chi_tau: learned screening acts on the tensor-core route (GW_BF16X3 / GW_BF16X6 / "
                "GW_FP16X3)");
  if (screening == GW_SCREEN_MLP && !ctx->mlp_ready)
    return fail(ctx, GW_ERR_ORDER, "chi_tau: learned screening needs gw_mlp_init/gw_mlp_train first");
  if (tau_count > 0 && !chi_out) return fail(ctx, GW_ERR_INVALID_ARG, "chi_tau: chi_out is null");
  GW_TRY(cudaSetDevice(ctx->device));
  ctx->stats = gw_stats{};
  if (ctx->mlp_mode != 1) ctx->mlp_mode = screening == GW_SCREEN_MLP ? 2 : 0;
  ctx->mlp_skipped = ctx->mlp_seen = 0;
  ctx->mlp_k_before = ctx->mlp_k_after = 0.0;
  auto t_start = std::chrono::steady_clock::now();
  // test hook "test_stall_tc", on for this call only
  struct StallScope {
    explicit StallScope(int on) { gw::tc_set_stall_test(on); }
    ~StallScope() { gw::tc_set_stall_test(0); }
  } stall_scope(ctx->test_stall);
  if (!tc_prec && ctx->d_t3f)
    return fail(ctx, GW_ERR_UNSUPPORTED,
                "chi_tau: the tensor is kept in FP32 (option tensor_fp32); the CUDA-core forms need it in FP64");
  int rc;
  // the tensor-core route needs the panel plan only; the CUDA-core routes
  // also the FP64 panel pool
  if ((rc = tc_prec ? plan_panels(ctx, thr) : build_panels(ctx, thr))) return rc;
  const bool f64 = precision == GW_FP64;
  const bool tcpath = tc_prec;
  const int f16 = precision == GW_FP16X3;
  if (ctx->last_precision != precision) {
    ws_release_all(ctx);
    ctx->last_precision = precision;
  }
  if (!f64 && !tcpath && (rc = ensure_panel32(ctx))) return rc;
  if (tcpath && (rc = ensure_pt(ctx, precision == GW_BF16X6 ? 3 : 2, f16))) return rc;
  const int nao = ctx->nao, nri = ctx->nri, n_at = ctx->n_at;
  // device bytes per operand element: FP64, FP32, or FP32 plus bf16 slices
  const size_t esz = f64 ? sizeof(double)
                         : precision == GW_BF16X6 ? 6 : tcpath ? 4 : sizeof(float);
  std::vector<Batch> batches =
      tcpath ? plan_batches_tc(ctx, esz, ctx->batch_bytes, gw::tc_tile_rows())
             : plan_batches(ctx, esz, ctx->batch_bytes, 0);
  ctx->stats.n_batches = (int)batches.size();

  double *cso, *csv, *go, *gv, *acc, *stage = nullptr;
  float *go32 = nullptr, *gv32 = nullptr;
  unsigned char *flo, *flv;
  if ((rc = wsT(ctx, "cso", (size_t)nao * std::max(ctx->n_occ, 1), &cso))) return rc;
  if ((rc = wsT(ctx, "csv", (size_t)nao * std::max(nao - ctx->n_occ, 1), &csv))) return rc;
  if ((rc = wsT(ctx, "g_occ", (size_t)nao * nao, &go))) return rc;
  if ((rc = wsT(ctx, "g_virt", (size_t)nao * nao, &gv))) return rc;
  if ((rc = wsT(ctx, "chi_acc", (size_t)nri * nri, &acc))) return rc;
  if ((rc = wsT(ctx, "flag_occ", (size_t)n_at * n_at, &flo))) return rc;
  if ((rc = wsT(ctx, "flag_virt", (size_t)n_at * n_at, &flv))) return rc;
  if (!out_on_device && (rc = wsT(ctx, "chi_stage", (size_t)nri * nri, &stage))) return rc;
  if (!f64 && !tcpath) {
    if ((rc = wsT(ctx, "g_occ32", (size_t)nao * nao, &go32))) return rc;
    if ((rc = wsT(ctx, "g_virt32", (size_t)nao * nao, &gv32))) return rc;
  }

  gw::ScopedEvents<3> ev;
  GW_TRY(ev.create());
  double ms_g = 0, ms_c = 0;
  for (int j = tau_first; j < tau_first + tau_count; ++j) {
    gw::TraceRange trace_tau("chi: one tau point");
    GW_TRY(cudaEventRecord(ev[0], ctx->stream));
    ctx->cur_tau = ctx->tau[j];
    gw::launch_greens(ctx->d_C, ctx->d_eps, nao, ctx->n_occ, ctx->mu, ctx->tau[j], cso, csv, go, gv,
                      ctx->stream);
    GW_CHECK_LAUNCH();
    ctx->stats.kernel_launches += 3;
    if (f16) {
      // binary16 scales of this tau: max |G| for the G slices, and the bounds
      // |X| <= max_mu sum_lambda |G^occ| * max |T| (Y alike with G^virt)
      double* gst;
      double h[4];
      if ((rc = wsT(ctx, "g_absmax", 4, &gst))) return rc;
      gw::launch_absmax_rowsum(go, nao, nao, nao, gst, ctx->stream);
      gw::launch_absmax_rowsum(gv, nao, nao, nao, gst + 2, ctx->stream);
      GW_CHECK_LAUNCH();
      ctx->stats.kernel_launches += 2;
      GW_TRY(cudaMemcpyAsync(h, gst, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
      GW_TRY(cudaStreamSynchronize(ctx->stream));
      ctx->tc_scale[0] = gw::pow2_scale(h[0]);
      ctx->tc_scale[1] = gw::pow2_scale(h[2]);
      ctx->tc_scale[2] = gw::pow2_scale(h[1] * ctx->t_absmax);
      ctx->tc_scale[3] = gw::pow2_scale(h[3] * ctx->t_absmax);
    }
    std::vector<unsigned char> hfo((size_t)n_at * n_at, 1), hfv((size_t)n_at * n_at, 1);
    if (thr > 0.0) {
      gw::launch_sym_block_filter(go, nao, ctx->d_ao_off, n_at, thr, flo, ctx->stream);
      gw::launch_sym_block_filter(gv, nao, ctx->d_ao_off, n_at, thr, flv, ctx->stream);
      GW_CHECK_LAUNCH();
      ctx->stats.kernel_launches += 2;
      GW_TRY(cudaMemcpyAsync(hfo.data(), flo, hfo.size(), cudaMemcpyDeviceToHost, ctx->stream));
      GW_TRY(cudaMemcpyAsync(hfv.data(), flv, hfv.size(), cudaMemcpyDeviceToHost, ctx->stream));
      GW_TRY(cudaStreamSynchronize(ctx->stream));  // the batch plan below reads the flags
    }
    if (!f64 && !tcpath) {
      gw::launch_cast_f64_f32(go, go32, (long long)nao * nao, ctx->stream);
      gw::launch_cast_f64_f32(gv, gv32, (long long)nao * nao, ctx->stream);
      GW_CHECK_LAUNCH();
      ctx->stats.kernel_launches += 2;
    }
    GW_TRY(cudaMemsetAsync(acc, 0, (size_t)nri * nri * sizeof(double), ctx->stream));
    GW_TRY(cudaEventRecord(ev[1], ctx->stream));
    std::vector<double> fc;
    if (tcpath && (rc = tc_begin_tau(ctx))) return rc;
    double fa = 0.0, fb = 0.0;
    std::vector<double> kao;
    int kao_m0 = -1;
    ctx->cur_fo = thr > 0.0 ? &hfo : nullptr;
    ctx->cur_fv = thr > 0.0 ? &hfv : nullptr;
    for (size_t bi = 0; bi < batches.size(); ++bi) {
      const Batch& b = batches[bi];
      // useful flops of steps A and B; a batch whose X or Y is all zero
      // (every G block it needs was filtered) adds nothing to chi: skipped
      if (b.m0 != kao_m0) {
        chunk_kao(ctx, b.m0, b.m1, hfo, kao);
        kao_m0 = b.m0;
      }
      double ba = 0.0, bb = 0.0;
      batch_flops_ab(ctx, b, kao, hfv, &ba, &bb);
      if (ba == 0.0 || bb == 0.0) {
        ++ctx->stats.batches_skipped;
        continue;
      }
      fa += ba;
      fb += bb;
      if (f64)
        rc = chi_one_batch<double>(ctx, b, go, gv, ctx->d_panel64, thr, acc, fc, precision, bi);
      else if (tcpath)
        rc = chi_one_batch_tc(ctx, b, go, gv, thr, acc, fc, precision, bi);
      else
        rc = chi_one_batch<float>(ctx, b, go32, gv32, ctx->d_panel32, thr, acc, fc, precision, bi);
      if (rc) {
        ctx->cur_fo = ctx->cur_fv = nullptr;
        return rc;
      }
    }
    ctx->cur_fo = ctx->cur_fv = nullptr;
    GW_TRY(cudaEventRecord(ev[2], ctx->stream));
    double* dst = out_on_device ? chi_out + (size_t)(j - tau_first) * nri * nri : stage;
    gw::launch_mirror(acc, dst, nri, ctx->d_atom_of_ri, ctx->stream);
    GW_CHECK_LAUNCH();
    ctx->stats.kernel_launches += 1;
    if (!out_on_device)
      GW_TRY(cudaMemcpyAsync(chi_out + (size_t)(j - tau_first) * nri * nri, stage,
                             (size_t)nri * nri * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GW_TRY(cudaStreamSynchronize(ctx->stream));
    if (tcpath && (rc = tc_finish_tau(ctx, fc))) return rc;
    float t01, t12;
    GW_TRY(cudaEventElapsedTime(&t01, ev[0], ev[1]));
    GW_TRY(cudaEventElapsedTime(&t12, ev[1], ev[2]));
    ms_g += t01;
    ms_c += t12;
    double fcs = 0.0;
    for (double v : fc) fcs += v;
    ctx->stats.flops_a += fa;
    ctx->stats.flops_b += fb;
    ctx->stats.flops_c += fcs;
  }
  ctx->stats.flops_useful = ctx->stats.flops_a + ctx->stats.flops_b + ctx->stats.flops_c;
  ctx->stats.tasks_seen = ctx->mlp_seen;
  ctx->stats.tasks_skipped = ctx->mlp_skipped;
  if (ctx->mlp_mode == 2) ctx->mlp_mode = 0;
  ctx->stats.ms_greens = ms_g;
  ctx->stats.ms_step_c = ms_c;
  ctx->stats.ms_total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return GW_OK;
}

}  // extern "C"
