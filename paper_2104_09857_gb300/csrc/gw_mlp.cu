// Learned screening of step-C tasks (not in the paper): the batch hook that
// logs or screens (chi tile, slab) tasks, and the C ABI to log training data,
// initialise, train, evaluate and query the network.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "gw_internal.h"
#include "k_mlp.h"

namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

#define ML_TRY(call)                                                                 \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      ctx->err = std::string("mlp: ") + #call + ": " + cudaGetErrorString(e_);       \
      return e_ == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA;             \
    }                                                                                \
  } while (0)

int ensure_params(gw_ctx* ctx) {
  if (ctx->d_mlp_theta) return GW_OK;
  ML_TRY(cudaMalloc(&ctx->d_mlp_theta, gw::kMlpParams * sizeof(float)));
  ML_TRY(cudaMalloc(&ctx->d_mlp_wb, gw::kMlpParams * 2));
  ML_TRY(cudaMalloc(&ctx->d_mlp_m, gw::kMlpParams * sizeof(float)));
  ML_TRY(cudaMalloc(&ctx->d_mlp_v, gw::kMlpParams * sizeof(float)));
  return GW_OK;
}

int upload_params(gw_ctx* ctx, const float* theta) {
  int rc = ensure_params(ctx);
  if (rc) return rc;
  ML_TRY(cudaMemcpyAsync(ctx->d_mlp_theta, theta, gw::kMlpParams * sizeof(float),
                         cudaMemcpyHostToDevice, ctx->stream));
  ML_TRY(cudaMemsetAsync(ctx->d_mlp_m, 0, gw::kMlpParams * sizeof(float), ctx->stream));
  ML_TRY(cudaMemsetAsync(ctx->d_mlp_v, 0, gw::kMlpParams * sizeof(float), ctx->stream));
  gw::mlp_round(ctx->d_mlp_theta, ctx->d_mlp_wb, ctx->stream);
  ML_TRY(cudaGetLastError());
  ML_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->mlp_step = 0;
  ctx->mlp_ready = true;
  return GW_OK;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return ((splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

}  // namespace

namespace gw {

int mlp_batch_hook(gw_ctx* ctx, const MlpBatch& mb) {
  cudaStream_t st = ctx->stream;
  const int F = kMlpFeatures;
  const int ntiles = mb.npt * mb.nqt;
  const long long slots = (long long)ntiles * mb.nslab;
  if (slots == 0) return GW_OK;
  DevBuf xn, yn, cp, cq, cc, xyz, feat, aux, skipped;
  ML_TRY(cudaMalloc(&xn.p, (size_t)mb.nslab * mb.npt * sizeof(float)));
  ML_TRY(cudaMalloc(&yn.p, (size_t)mb.nslab * mb.nqt * sizeof(float)));
  gw::mlp_slab_tile_norms(mb.bx2, mb.bx, mb.nmc, mb.m0, mb.npa, mb.pa0, mb.per, kSlabAO, ctx->d_atom_of_ao,
                          ctx->d_atom_of_ri, mb.mu0, mb.nmu, mb.P0, mb.prow, mb.npt, mb.tile, mb.nslab,
                          (float*)xn.p, st);
  gw::mlp_slab_tile_norms(mb.by2, mb.by, mb.nmc, mb.m0, mb.nqa, mb.qa0, mb.per, kSlabAO, ctx->d_atom_of_ao,
                          ctx->d_atom_of_ri, mb.mu0, mb.nmu, mb.Q0, mb.qrow, mb.nqt, mb.tile, mb.nslab,
                          (float*)yn.p, st);
  // centroids of row tiles, column tiles and AO chunks (weighted by functions)
  auto centroid = [&](const std::vector<int>& off, int lo, int hi, float* out3) {
    double w = 0, x = 0, y = 0, z = 0;
    for (int a = 0; a < ctx->n_at; ++a) {
      const int a0 = std::max(off[a], lo), a1 = std::min(off[a + 1], hi);
      if (a1 <= a0) continue;
      const double c = a1 - a0;
      w += c;
      x += c * ctx->xyz[3 * a];
      y += c * ctx->xyz[3 * a + 1];
      z += c * ctx->xyz[3 * a + 2];
    }
    if (w == 0) w = 1;
    out3[0] = (float)(x / w);
    out3[1] = (float)(y / w);
    out3[2] = (float)(z / w);
  };
  std::vector<float> h_cp(3 * mb.npt), h_cq(3 * mb.nqt), h_cc(3 * mb.per), h_xyz(3 * ctx->n_at);
  for (int t = 0; t < mb.npt; ++t)
    centroid(ctx->ri_off, mb.P0 + t * mb.tile, std::min(mb.P0 + mb.prow, mb.P0 + (t + 1) * mb.tile), &h_cp[3 * t]);
  for (int t = 0; t < mb.nqt; ++t)
    centroid(ctx->ri_off, mb.Q0 + t * mb.tile, std::min(mb.Q0 + mb.qrow, mb.Q0 + (t + 1) * mb.tile),
             &h_cq[3 * t]);
  for (int c = 0; c < mb.per; ++c)
    centroid(ctx->ao_off, mb.mu0 + c * kSlabAO, std::min(mb.mu0 + mb.nmu, mb.mu0 + (c + 1) * kSlabAO),
             &h_cc[3 * c]);
  for (int i = 0; i < 3 * ctx->n_at; ++i) h_xyz[i] = (float)ctx->xyz[i];
  ML_TRY(cudaMalloc(&cp.p, h_cp.size() * 4));
  ML_TRY(cudaMalloc(&cq.p, h_cq.size() * 4));
  ML_TRY(cudaMalloc(&cc.p, h_cc.size() * 4));
  ML_TRY(cudaMalloc(&xyz.p, h_xyz.size() * 4));
  ML_TRY(cudaMemcpyAsync(cp.p, h_cp.data(), h_cp.size() * 4, cudaMemcpyHostToDevice, st));
  ML_TRY(cudaMemcpyAsync(cq.p, h_cq.data(), h_cq.size() * 4, cudaMemcpyHostToDevice, st));
  ML_TRY(cudaMemcpyAsync(cc.p, h_cc.data(), h_cc.size() * 4, cudaMemcpyHostToDevice, st));
  ML_TRY(cudaMemcpyAsync(xyz.p, h_xyz.data(), h_xyz.size() * 4, cudaMemcpyHostToDevice, st));
  DevBuf nao_d;
  ML_TRY(cudaMalloc(&nao_d.p, ctx->n_at * sizeof(int)));
  ML_TRY(cudaMemcpyAsync(nao_d.p, ctx->n_ao.data(), ctx->n_at * sizeof(int), cudaMemcpyHostToDevice, st));
  ML_TRY(cudaMalloc(&feat.p, (size_t)slots * F * sizeof(float)));
  ML_TRY(cudaMalloc(&aux.p, (size_t)slots * sizeof(float)));
  gw::mlp_task_features(mb.tasks, mb.counts, mb.nslab, mb.npt, mb.nqt, mb.per, mb.s0, (float*)xn.p,
                        (float*)yn.p, (float*)cp.p, (float*)cq.p, (float*)cc.p, (float*)xyz.p,
                        (int*)nao_d.p, (float)std::log10(mb.tau), (float*)feat.p, st);
  ML_TRY(cudaGetLastError());
  std::vector<int> h_counts(ntiles);
  ML_TRY(cudaMemcpyAsync(h_counts.data(), mb.counts, ntiles * sizeof(int), cudaMemcpyDeviceToHost, st));
  ML_TRY(cudaStreamSynchronize(st));
  int max_count = 0;
  long long n_tasks = 0;
  for (int c : h_counts) {
    max_count = std::max(max_count, c);
    n_tasks += c;
  }
  if (ctx->mlp_mode == 1) {
    gw::mlp_task_norms(mb.xs, mb.ys, mb.slices, mb.f16, mb.xinv, mb.yinv, (long long)mb.prow * mb.Kb,
                       (long long)mb.qrow * mb.Kb,
                       mb.Kb, mb.prow, mb.qrow, mb.tasks, mb.counts, mb.nslab, mb.npt, mb.nqt, max_count,
                       mb.tile, mb.slab_k0, mb.slab_len, (float*)aux.p, st);
    ML_TRY(cudaGetLastError());
    std::vector<float> h_feat((size_t)slots * F), h_tgt(slots);
    ML_TRY(cudaMemcpyAsync(h_feat.data(), feat.p, h_feat.size() * 4, cudaMemcpyDeviceToHost, st));
    ML_TRY(cudaMemcpyAsync(h_tgt.data(), aux.p, h_tgt.size() * 4, cudaMemcpyDeviceToHost, st));
    ML_TRY(cudaStreamSynchronize(st));
    for (int t = 0; t < ntiles; ++t)
      for (int i = 0; i < h_counts[t]; ++i) {
        const size_t slot = (size_t)t * mb.nslab + i;
        ctx->mlp_log_feat.insert(ctx->mlp_log_feat.end(), &h_feat[slot * F], &h_feat[slot * F] + F);
        ctx->mlp_log_tgt.push_back(h_tgt[slot]);
      }
    return GW_OK;
  }
  // mode 2: screen
  if (!ctx->mlp_ready) {
    ctx->err = "learned screening: the network is not initialised or trained";
    return GW_ERR_ORDER;
  }
  ML_TRY(cudaMalloc(&skipped.p, ntiles * sizeof(int)));
  std::vector<long long> kb(ntiles), ka(ntiles);
  ML_TRY(cudaMemcpyAsync(kb.data(), mb.kacc, ntiles * sizeof(long long), cudaMemcpyDeviceToHost, st));
  gw::mlp_forward(ctx->d_mlp_wb, (float*)feat.p, slots, mb.counts, mb.nslab, nullptr, nullptr,
                  (float*)aux.p, st);
  gw::mlp_compact(mb.tasks, mb.counts, mb.kacc, ntiles, mb.nslab, (float*)aux.p, (float*)feat.p,
                  (float)ctx->mlp_margin, (float)std::log10(mb.thr), mb.slab_len, (int*)skipped.p, st);
  ML_TRY(cudaGetLastError());
  std::vector<int> h_sk(ntiles);
  ML_TRY(cudaMemcpyAsync(h_sk.data(), skipped.p, ntiles * sizeof(int), cudaMemcpyDeviceToHost, st));
  ML_TRY(cudaMemcpyAsync(ka.data(), mb.kacc, ntiles * sizeof(long long), cudaMemcpyDeviceToHost, st));
  ML_TRY(cudaStreamSynchronize(st));
  for (int t = 0; t < ntiles; ++t) {
    ctx->mlp_skipped += h_sk[t];
    ctx->mlp_k_before += (double)kb[t];
    ctx->mlp_k_after += (double)ka[t];
  }
  ctx->mlp_seen += n_tasks;
  return GW_OK;
}

}  // namespace gw

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int gw_mlp_init(gw_ctx* ctx, unsigned long long seed) {
  if (!ctx) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  ML_TRY(cudaSetDevice(ctx->device));
  // He-scaled normal weights (SplitMix64 + Box-Muller), zero biases
  const int F = gw::kMlpFeatures, H = gw::kMlpHidden;
  std::vector<float> th(gw::kMlpParams, 0.f);
  uint64_t s = seed * 0x2545F4914F6CDD1Dull + 1;
  auto normal = [&]() {
    const double u1 = uniform01(s), u2 = uniform01(s);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  int o = 0;
  for (int i = 0; i < H * F; ++i) th[o++] = (float)(normal() * std::sqrt(2.0 / F));
  o += H;
  for (int i = 0; i < H * H; ++i) th[o++] = (float)(normal() * std::sqrt(2.0 / H));
  o += H;
  for (int i = 0; i < H; ++i) th[o++] = (float)(normal() * std::sqrt(1.0 / H));
  return upload_params(ctx, th.data());
}

int gw_mlp_set_params(gw_ctx* ctx, const float* theta, long long n) {
  if (!ctx || !theta) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (n != gw::kMlpParams) {
    ctx->err = "gw_mlp_set_params: expected " + std::to_string(gw::kMlpParams) + " parameters";
    return GW_ERR_INVALID_ARG;
  }
  ML_TRY(cudaSetDevice(ctx->device));
  return upload_params(ctx, theta);
}

int gw_mlp_get_params(gw_ctx* ctx, float* theta, long long n) {
  if (!ctx || !theta) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (n != gw::kMlpParams || !ctx->mlp_ready) {
    ctx->err = "gw_mlp_get_params: network not initialised or wrong size";
    return ctx->mlp_ready ? GW_ERR_INVALID_ARG : GW_ERR_ORDER;
  }
  ML_TRY(cudaMemcpy(theta, ctx->d_mlp_theta, n * sizeof(float), cudaMemcpyDeviceToHost));
  return GW_OK;
}

// loss and gradient (w.r.t. the bf16-rounded weights) on the given samples
int gw_mlp_grad(gw_ctx* ctx, const float* feat, const float* tgt, long long n, float* loss,
                float* grad) {
  if (!ctx || !feat || !tgt || n <= 0 || !loss || !grad) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->mlp_ready) {
    ctx->err = "gw_mlp_grad: network not initialised";
    return GW_ERR_ORDER;
  }
  ML_TRY(cudaSetDevice(ctx->device));
  const int F = gw::kMlpFeatures, H = gw::kMlpHidden;
  cudaStream_t st = ctx->stream;
  DevBuf x, t, z1, z2, y, dy, dz1, dz2, g;
  ML_TRY(cudaMalloc(&x.p, n * F * 4));
  ML_TRY(cudaMalloc(&t.p, n * 4));
  ML_TRY(cudaMalloc(&z1.p, n * H * 4));
  ML_TRY(cudaMalloc(&z2.p, n * H * 4));
  ML_TRY(cudaMalloc(&y.p, n * 4));
  ML_TRY(cudaMalloc(&dy.p, n * 4));
  ML_TRY(cudaMalloc(&dz1.p, n * H * 4));
  ML_TRY(cudaMalloc(&dz2.p, n * H * 4));
  ML_TRY(cudaMalloc(&g.p, gw::kMlpParams * 4));
  ML_TRY(cudaMemcpyAsync(x.p, feat, n * F * 4, cudaMemcpyHostToDevice, st));
  ML_TRY(cudaMemcpyAsync(t.p, tgt, n * 4, cudaMemcpyHostToDevice, st));
  gw::mlp_forward(ctx->d_mlp_wb, (float*)x.p, n, nullptr, 1, (float*)z1.p, (float*)z2.p, (float*)y.p, st);
  gw::mlp_backward(ctx->d_mlp_wb, (float*)x.p, (float*)z1.p, (float*)z2.p, (float*)y.p, (float*)t.p, n,
                   (float*)dy.p, (float*)dz1.p, (float*)dz2.p, (float*)g.p, st);
  ML_TRY(cudaGetLastError());
  std::vector<float> hy(n);
  ML_TRY(cudaMemcpyAsync(hy.data(), y.p, n * 4, cudaMemcpyDeviceToHost, st));
  ML_TRY(cudaMemcpyAsync(grad, g.p, gw::kMlpParams * 4, cudaMemcpyDeviceToHost, st));
  ML_TRY(cudaStreamSynchronize(st));
  double l = 0;
  for (long long i = 0; i < n; ++i) l += (double)(hy[i] - tgt[i]) * (hy[i] - tgt[i]);
  *loss = (float)(l / n);
  return GW_OK;
}

int gw_mlp_predict(gw_ctx* ctx, const float* feat, long long n, float* pred) {
  if (!ctx || !feat || !pred || n <= 0) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->mlp_ready) {
    ctx->err = "gw_mlp_predict: network not initialised";
    return GW_ERR_ORDER;
  }
  ML_TRY(cudaSetDevice(ctx->device));
  DevBuf x, y;
  ML_TRY(cudaMalloc(&x.p, n * gw::kMlpFeatures * 4));
  ML_TRY(cudaMalloc(&y.p, n * 4));
  ML_TRY(cudaMemcpyAsync(x.p, feat, n * gw::kMlpFeatures * 4, cudaMemcpyHostToDevice, ctx->stream));
  gw::mlp_forward(ctx->d_mlp_wb, (float*)x.p, n, nullptr, 1, nullptr, nullptr, (float*)y.p, ctx->stream);
  ML_TRY(cudaGetLastError());
  ML_TRY(cudaMemcpyAsync(pred, y.p, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  ML_TRY(cudaStreamSynchronize(ctx->stream));
  return GW_OK;
}

// Adam on mini-batches of a per-epoch shuffled copy (batch <= 0: full batch);
// loss_per_epoch[e] = training loss after epoch e
int gw_mlp_train(gw_ctx* ctx, const float* feat, const float* tgt, long long n, int epochs, long long batch,
                 float lr, unsigned long long seed, float* loss_per_epoch) {
  if (!ctx || !feat || !tgt || n <= 0 || epochs < 0 || !(lr > 0.f)) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (!ctx->mlp_ready) {
    ctx->err = "gw_mlp_train: call gw_mlp_init or gw_mlp_set_params first";
    return GW_ERR_ORDER;
  }
  ML_TRY(cudaSetDevice(ctx->device));
  const int F = gw::kMlpFeatures, H = gw::kMlpHidden;
  if (batch <= 0 || batch > n) batch = n;
  cudaStream_t st = ctx->stream;
  DevBuf x, t, z1, z2, y, dy, dz1, dz2, g, xa, ta, ya;
  ML_TRY(cudaMalloc(&x.p, batch * F * 4));
  ML_TRY(cudaMalloc(&t.p, batch * 4));
  ML_TRY(cudaMalloc(&z1.p, batch * H * 4));
  ML_TRY(cudaMalloc(&z2.p, batch * H * 4));
  ML_TRY(cudaMalloc(&y.p, batch * 4));
  ML_TRY(cudaMalloc(&dy.p, batch * 4));
  ML_TRY(cudaMalloc(&dz1.p, batch * H * 4));
  ML_TRY(cudaMalloc(&dz2.p, batch * H * 4));
  ML_TRY(cudaMalloc(&g.p, gw::kMlpParams * 4));
  ML_TRY(cudaMalloc(&xa.p, n * F * 4));
  ML_TRY(cudaMalloc(&ya.p, n * 4));
  ML_TRY(cudaMemcpyAsync(xa.p, feat, n * F * 4, cudaMemcpyHostToDevice, st));
  std::vector<long long> perm(n);
  for (long long i = 0; i < n; ++i) perm[i] = i;
  std::vector<float> bx((size_t)batch * F), bt(batch), hy(n);
  uint64_t s = seed ^ 0x5DEECE66Dull;
  for (int e = 0; e < epochs; ++e) {
    if (batch < n)
      for (long long i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(s) % (uint64_t)(i + 1)]);
    for (long long b0 = 0; b0 < n; b0 += batch) {
      const long long m = std::min(batch, n - b0);
      for (long long i = 0; i < m; ++i) {
        const long long src = perm[b0 + i];
        std::memcpy(&bx[i * F], &feat[src * F], F * 4);
        bt[i] = tgt[src];
      }
      ML_TRY(cudaMemcpyAsync(x.p, bx.data(), m * F * 4, cudaMemcpyHostToDevice, st));
      ML_TRY(cudaMemcpyAsync(t.p, bt.data(), m * 4, cudaMemcpyHostToDevice, st));
      gw::mlp_forward(ctx->d_mlp_wb, (float*)x.p, m, nullptr, 1, (float*)z1.p, (float*)z2.p, (float*)y.p, st);
      gw::mlp_backward(ctx->d_mlp_wb, (float*)x.p, (float*)z1.p, (float*)z2.p, (float*)y.p, (float*)t.p, m,
                       (float*)dy.p, (float*)dz1.p, (float*)dz2.p, (float*)g.p, st);
      gw::mlp_adam(ctx->d_mlp_theta, (float*)g.p, ctx->d_mlp_m, ctx->d_mlp_v, ++ctx->mlp_step, lr,
                   ctx->d_mlp_wb, st);
      ML_TRY(cudaGetLastError());
      // the host staging vectors are reused: wait before the next batch overwrites them
      ML_TRY(cudaStreamSynchronize(st));
    }
    if (loss_per_epoch) {
      gw::mlp_forward(ctx->d_mlp_wb, (float*)xa.p, n, nullptr, 1, nullptr, nullptr, (float*)ya.p, st);
      ML_TRY(cudaMemcpyAsync(hy.data(), ya.p, n * 4, cudaMemcpyDeviceToHost, st));
      ML_TRY(cudaStreamSynchronize(st));
      double l = 0;
      for (long long i = 0; i < n; ++i) l += (double)(hy[i] - tgt[i]) * (hy[i] - tgt[i]);
      loss_per_epoch[e] = (float)(l / n);
    }
  }
  return GW_OK;
}

}  // extern "C"
