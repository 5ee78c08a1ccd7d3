// gw_autotune: picks the schedule of the tensor-core chi route for a given
// system, threshold and form by measurement.  The knobs searched change the
// work's order and grouping only (the result moves by rounding order, not by
// accuracy): the staged step-A/B epilogue, the step-C work-unit length, the
// operand batch budget and the mu-chunk size of the 2-D batches.  The drain
// cadence of the FP32 accumulator (flush_k) sets the accuracy and is left
// alone.
//
// Search: coordinate descent from the context's current settings.  Each knob
// in turn takes each of its candidate values with the others fixed; a
// candidate is timed as the device time (CUDA events on the context's
// stream) of gw_chi_tau on one tau point after one untimed call, and the
// fastest value is kept before the next knob.  Every trial is logged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "gw_internal.h"

namespace {

struct Knob {
  const char* name;
  std::vector<double> values;
};

double current(const gw_ctx* ctx, const std::string& k) {
  if (k == "panel_staged") return ctx->panel_staged;
  if (k == "c_split_k") return ctx->c_split_k;
  if (k == "c_dynamic") return ctx->c_dynamic;
  if (k == "batch_bytes") return ctx->batch_bytes;
  if (k == "mu_chunk_atoms") return ctx->mu_chunk_atoms;
  return 0.0;
}

}  // namespace

extern "C" int gw_autotune(gw_ctx* ctx, int tau_index, double thr, int precision, gw_tune_trial* trials,
                           int max_trials, int* n_trials) {
  if (!ctx || !n_trials || max_trials < 0 || (max_trials > 0 && !trials)) return GW_ERR_INVALID_ARG;
  gw::TraceRange trace("gw_autotune");
  ctx->err.clear();
  if (precision != GW_BF16X3 && precision != GW_BF16X6 && precision != GW_FP16X3) {
    ctx->err = "gw_autotune: the searched knobs belong to the tensor-core route (GW_BF16X3, GW_BF16X6, GW_FP16X3)";
    return GW_ERR_UNSUPPORTED;
  }
  if (ctx->n_at == 0 || ctx->blk_off.empty() || !ctx->have_greens) {
    ctx->err = "gw_autotune: call gw_set_basis, gw_set_3c_tensor and gw_set_greens first";
    return GW_ERR_ORDER;
  }
  if (tau_index < 0 || tau_index >= (int)ctx->tau.size()) {
    ctx->err = "gw_autotune: tau_index out of range";
    return GW_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return GW_ERR_CUDA;
  double* out = nullptr;
  const size_t bytes = (size_t)ctx->nri * ctx->nri * sizeof(double);
  if (cudaMalloc(&out, std::max<size_t>(bytes, 8)) != cudaSuccess) {
    cudaGetLastError();
    ctx->err = "gw_autotune: cudaMalloc of the chi buffer failed";
    return GW_ERR_OOM;
  }
  gw::ScopedEvents<2> ev;
  if (ev.create() != cudaSuccess) {
    cudaFree(out);
    ctx->err = "gw_autotune: cudaEventCreate failed";
    return GW_ERR_CUDA;
  }
  // device memory left for the operand batches bounds the budgets tried
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const double budget_now = ctx->batch_bytes;
  std::vector<double> budgets;
  for (double f : {0.5, 1.0, 1.5})
    if (f == 1.0 || budget_now * f < 0.6 * (double)free_b + budget_now) budgets.push_back(budget_now * f);
  std::vector<Knob> knobs = {
      {"panel_staged", {1, 0}},
      {"c_split_k", {1024, 2048, 4096, 8192}},
      {"c_dynamic", {1, 0}},
      {"batch_bytes", budgets},
      {"mu_chunk_atoms", {0, (double)std::max(1, ctx->n_at / 4), (double)std::max(1, ctx->n_at / 2)}},
  };
  int nt = 0, rc = GW_OK;
  auto time_once = [&](float* ms) -> int {
    int r = gw_chi_tau(ctx, tau_index, 1, thr, precision, GW_SCREEN_BOUND, out, 1);
    if (r) return r;
    if (cudaEventRecord(ev[0], ctx->stream) != cudaSuccess) return GW_ERR_CUDA;
    r = gw_chi_tau(ctx, tau_index, 1, thr, precision, GW_SCREEN_BOUND, out, 1);
    if (r) return r;
    if (cudaEventRecord(ev[1], ctx->stream) != cudaSuccess) return GW_ERR_CUDA;
    if (cudaEventSynchronize(ev[1]) != cudaSuccess) return GW_ERR_CUDA;
    if (cudaEventElapsedTime(ms, ev[0], ev[1]) != cudaSuccess) return GW_ERR_CUDA;
    return GW_OK;
  };
  auto record = [&](const char* knob, double value, float ms) {
    if (nt < max_trials) {
      gw_tune_trial& t = trials[nt];
      std::snprintf(t.knob, sizeof(t.knob), "%s", knob);
      t.value = value;
      t.ms = ms;
      t.panel_staged = ctx->panel_staged;
      t.c_split_k = ctx->c_split_k;
      t.batch_bytes = ctx->batch_bytes;
      t.mu_chunk_atoms = ctx->mu_chunk_atoms;
    }
    ++nt;
  };
  float best = 0.f;
  if ((rc = time_once(&best))) goto done;
  record("start", 0.0, best);
  for (const Knob& k : knobs) {
    const double keep = current(ctx, k.name);
    double best_v = keep;
    for (double v : k.values) {
      if (v == keep) continue;
      if ((rc = gw_set_option(ctx, k.name, v))) goto done;
      float ms = 0.f;
      rc = time_once(&ms);
      if (rc == GW_ERR_OOM) {  // a budget that does not fit: not a candidate
        rc = GW_OK;
        ctx->err.clear();
        continue;
      }
      if (rc) goto done;
      record(k.name, v, ms);
      if (ms < best) {
        best = ms;
        best_v = v;
      }
    }
    if ((rc = gw_set_option(ctx, k.name, best_v))) goto done;
  }
done:
  cudaFree(out);
  *n_trials = nt;
  return rc;
}
