// gw_chi_tau_noalloc: the FP64 chi(i tau) path for one tau point with every
// per-call work buffer taken from a fixed array in device global memory.
//
// Why: some callers cannot call cudaMalloc when they need chi -- a host
// framework whose caching allocator owns the device memory budget and must not
// see allocations behind its back, a process that reserved all device memory
// up front, or latency-bound code that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree.  For them this entry point runs the
// same kernels as gw_chi_tau(precision = GW_FP64) for one tau point without
// any allocation: Green's functions, the chi accumulator, the step-A/B
// operands of one batch of sigma-atoms, filter flags and task lists all live
// in the array below.
//
// Limits and sharing:
//  * The array holds kNoAllocBytes (64 MiB).  A system is accepted when its
//    Green's functions (3 n_AO^2 doubles), chi accumulator (n_RI^2 doubles),
//    small tables, and the operands of one single-atom batch
//    ((rows of its RI window + n_RI) * n_AO(rounded to 64) * n_ao(atom)
//    doubles) fit; otherwise the call returns GW_ERR_INVALID_ARG and says how
//    many bytes were needed.
//  * The array is a module-scope variable: every GPU on which the library's
//    module is loaded holds it until the process exits.
//  * All calls in the process share it and it keeps the previous call's
//    contents; everything that must start at zero is cleared by each call.
//    Two calls whose GPU work overlaps (other streams, other threads, other
//    contexts on the same device) race on the array and corrupt each other:
//    serialise them.
//  * The first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture begins.
//  * Each call copies its per-batch tables from pageable host memory and
//    synchronises the context's stream after every batch and at its end.
//  * The FP64 3c tensor panels are built by gw_chi_tau on its CUDA-core
//    routes (they depend on thr); call gw_chi_tau once with the same thr and
//    precision GW_FP64 (or GW_FP32) before using this entry point.
//  * No cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "gw_internal.h"
#include "k_simt.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per device).
int scratch_address(gw_ctx* ctx, int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) {
    ctx->err = "gw_chi_tau_noalloc: device index out of range";
    return GW_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      ctx->err = std::string("gw_chi_tau_noalloc: cudaGetSymbolAddress failed: ") +
                 cudaGetErrorString(e);
      return GW_ERR_CUDA;
    }
    g_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[device]);
  return GW_OK;
}

// Bump allocator over the fixed array (256-byte aligned pieces).
struct Carve {
  unsigned char* base;
  size_t used = 0;
  size_t need = 0;  // bytes requested so far, even past the end
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) / 256 * 256;
    size_t at = need;
    need += bytes;
    if (need > kNoAllocBytes) return nullptr;
    used = need;
    return reinterpret_cast<T*>(base + at);
  }
};

#define NA_TRY(call)                                                         \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      ctx->err = std::string("gw_chi_tau_noalloc: ") + #call + ": " +        \
                 cudaGetErrorString(e_);                                     \
      return GW_ERR_CUDA;                                                    \
    }                                                                        \
  } while (0)

#define NA_LAUNCHED()                                                        \
  do {                                                                       \
    cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess) {                                                 \
      ctx->err = std::string("gw_chi_tau_noalloc: kernel launch: ") +        \
                 cudaGetErrorString(e_);                                     \
      return GW_ERR_CUDA;                                                    \
    }                                                                        \
  } while (0)

}  // namespace

extern "C" int gw_chi_tau_noalloc(gw_ctx* ctx, int tau_index, double thr, double* chi_out_device) {
  using gw::kSlabAO;
  using gw::PanelDesc;
  using gw::PanelTask;
  if (!ctx) return GW_ERR_INVALID_ARG;
  ctx->err.clear();
  if (ctx->n_at == 0 || ctx->blk_off.empty() || !ctx->have_greens) {
    ctx->err = "gw_chi_tau_noalloc: call gw_set_basis, gw_set_3c_tensor and gw_set_greens first";
    return GW_ERR_ORDER;
  }
  if (tau_index < 0 || tau_index >= (int)ctx->tau.size()) {
    ctx->err = "gw_chi_tau_noalloc: tau_index out of range";
    return GW_ERR_INVALID_ARG;
  }
  if (!(thr >= 0.0) || !std::isfinite(thr)) {
    ctx->err = "gw_chi_tau_noalloc: thr must be finite and >= 0";
    return GW_ERR_INVALID_ARG;
  }
  if (!chi_out_device) {
    ctx->err = "gw_chi_tau_noalloc: chi_out_device is null";
    return GW_ERR_INVALID_ARG;
  }
  if (!ctx->panels_ok || ctx->panels_thr != thr) {
    ctx->err =
        "gw_chi_tau_noalloc: the FP64 3c panels for this thr are not built; call gw_chi_tau "
        "once with the same thr and precision GW_FP64 (or GW_FP32) first";
    return GW_ERR_ORDER;
  }
  NA_TRY(cudaSetDevice(ctx->device));
  unsigned char* base = nullptr;
  int rc = scratch_address(ctx, ctx->device, &base);
  if (rc) return rc;

  const int nao = ctx->nao, nri = ctx->nri, n_at = ctx->n_at, naop = ctx->naop;
  const int n_occ = ctx->n_occ;
  cudaStream_t st = ctx->stream;

  // fixed pieces
  Carve cv{base};
  double* cso = cv.take<double>((size_t)nao * std::max(n_occ, 1));
  double* csv = cv.take<double>((size_t)nao * std::max(nao - n_occ, 1));
  double* go = cv.take<double>((size_t)nao * nao);
  double* gv = cv.take<double>((size_t)nao * nao);
  double* acc = cv.take<double>((size_t)nri * nri);
  unsigned char* flo = cv.take<unsigned char>((size_t)n_at * n_at);
  unsigned char* flv = cv.take<unsigned char>((size_t)n_at * n_at);
  int* d_nao = cv.take<int>(n_at);
  int* d_nri = cv.take<int>(n_at);
  PanelTask* d_tb = cv.take<PanelTask>(n_at);
  const size_t fixed_need = cv.need;

  // largest single-atom batch (operands + its tables), to size the batch area
  auto batch_need = [&](int s0, int s1, int P0, int P1) {
    const int ns = s1 - s0;
    const long long Kb = [&] {
      long long k = 0;
      for (int s = s0; s < s1; ++s) k += (long long)naop * ctx->n_ao[s];
      return k;
    }();
    const int prow = P1 - P0;
    const int npt = (prow + 63) / 64, nqt = (nri + 63) / 64;
    const int nslab = ns * (naop / kSlabAO);
    const int R = ctx->ao_off[s1] - ctx->ao_off[s0];
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t b = 0;
    b += al((size_t)prow * Kb * sizeof(double)) + al((size_t)nri * Kb * sizeof(double));
    b += al(ns * sizeof(PanelTask)) + al(R * sizeof(long long)) + al(R * sizeof(int));
    b += al(ns * sizeof(long long));
    b += al((size_t)ns * n_at * n_at) * 2 + al((size_t)ns * n_at * npt) + al((size_t)ns * n_at * nqt);
    b += al((size_t)nslab * sizeof(long long)) + al((size_t)nslab * sizeof(int));
    b += al((size_t)npt * nqt * nslab * sizeof(int)) + al((size_t)npt * nqt * sizeof(int)) +
         al((size_t)npt * nqt * sizeof(long long));
    return b;
  };
  // plan batches greedily within what is left of the array
  struct B {
    int s0, s1, P0, P1;
  };
  std::vector<B> batches;
  {
    int s = 0;
    while (s < n_at) {
      B b{s, s, INT32_MAX, 0};
      int e = s;
      while (e < n_at) {
        const PanelDesc& d = ctx->panels[e];
        int P0 = b.P0, P1 = b.P1;
        if (d.K > 0) {
          P0 = std::min(P0, d.p0);
          P1 = std::max(P1, d.p0 + d.npw);
        }
        int q0 = P1 > P0 ? P0 : 0, q1 = P1 > P0 ? P1 : 0;
        size_t need = fixed_need + batch_need(s, e + 1, q0, q1);
        if (need > kNoAllocBytes) {
          if (e == s) {
            ctx->err = "gw_chi_tau_noalloc: system too large for the fixed " +
                       std::to_string(kNoAllocBytes >> 20) + " MiB work array (needs " +
                       std::to_string(need) + " bytes for one sigma-atom batch)";
            return GW_ERR_INVALID_ARG;
          }
          break;
        }
        b.P0 = P0;
        b.P1 = P1;
        ++e;
      }
      b.s1 = e;
      if (b.P1 <= b.P0) b.P0 = b.P1 = 0;
      batches.push_back(b);
      s = e;
    }
  }

  // Green's functions (Eq. 2) and their block filter
  NA_TRY(cudaMemcpyAsync(d_nao, ctx->n_ao.data(), n_at * sizeof(int), cudaMemcpyHostToDevice, st));
  NA_TRY(cudaMemcpyAsync(d_nri, ctx->n_ri.data(), n_at * sizeof(int), cudaMemcpyHostToDevice, st));
  gw::launch_greens(ctx->d_C, ctx->d_eps, nao, n_occ, ctx->mu, ctx->tau[tau_index], cso, csv, go, gv, st);
  NA_LAUNCHED();
  if (thr > 0.0) {
    gw::launch_sym_block_filter(go, nao, ctx->d_ao_off, n_at, thr, flo, st);
    gw::launch_sym_block_filter(gv, nao, ctx->d_ao_off, n_at, thr, flv, st);
    NA_LAUNCHED();
  }
  NA_TRY(cudaMemsetAsync(acc, 0, (size_t)nri * nri * sizeof(double), st));

  // step-B problems: every panel (same for all batches)
  std::vector<PanelTask> tb;
  int maxNb = 0;
  for (int m = 0; m < n_at; ++m) {
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
    maxNb = std::max(maxNb, t.N);
    tb.push_back(t);
  }
  if (!tb.empty())
    NA_TRY(cudaMemcpyAsync(d_tb, tb.data(), tb.size() * sizeof(PanelTask), cudaMemcpyHostToDevice, st));

  for (const B& b : batches) {
    const int ns = b.s1 - b.s0;
    const int prow = b.P1 - b.P0;
    std::vector<long long> seg(ns);
    long long Kb = 0;
    for (int s = b.s0; s < b.s1; ++s) {
      seg[s - b.s0] = Kb;
      Kb += (long long)naop * ctx->n_ao[s];
    }
    if (prow == 0 || Kb == 0) continue;
    const int npt = (prow + 63) / 64, nqt = (nri + 63) / 64;
    const int nslab = ns * (naop / kSlabAO);
    const int r0 = ctx->ao_off[b.s0];
    const int R = ctx->ao_off[b.s1] - r0;
    Carve bc{base};
    bc.need = fixed_need;
    double* X = bc.take<double>((size_t)prow * Kb);
    double* Y = bc.take<double>((size_t)nri * Kb);
    PanelTask* d_ta = bc.take<PanelTask>(ns);
    long long* d_rowbase = bc.take<long long>(R);
    int* d_rowmul = bc.take<int>(R);
    long long* d_seg = bc.take<long long>(ns);
    unsigned char* bx = bc.take<unsigned char>((size_t)ns * n_at * n_at);
    unsigned char* by = bc.take<unsigned char>((size_t)ns * n_at * n_at);
    unsigned char* fx = bc.take<unsigned char>((size_t)ns * n_at * npt);
    unsigned char* fy = bc.take<unsigned char>((size_t)ns * n_at * nqt);
    long long* d_k0 = bc.take<long long>(nslab);
    int* d_len = bc.take<int>(nslab);
    int* tasks = bc.take<int>((size_t)npt * nqt * nslab);
    int* counts = bc.take<int>((size_t)npt * nqt);
    long long* kacc = bc.take<long long>((size_t)npt * nqt);
    if (!kacc) {
      ctx->err = "gw_chi_tau_noalloc: internal batch sizing error";
      return GW_ERR_INVALID_ARG;
    }
    // host tables
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
      t.seg = seg[s - b.s0];
      maxNa = std::max(maxNa, t.N);
      ta.push_back(t);
    }
    std::vector<long long> rowbase(R);
    std::vector<int> rowmul(R);
    for (int s = b.s0; s < b.s1; ++s)
      for (int i = 0; i < ctx->n_ao[s]; ++i) {
        rowbase[ctx->ao_off[s] - r0 + i] = seg[s - b.s0] + i;
        rowmul[ctx->ao_off[s] - r0 + i] = ctx->n_ao[s];
      }
    std::vector<long long> k0(nslab);
    std::vector<int> len(nslab);
    const int per = naop / kSlabAO;
    for (int sl = 0; sl < ns; ++sl)
      for (int c = 0; c < per; ++c) {
        int nsig = ctx->n_ao[b.s0 + sl];
        k0[sl * per + c] = seg[sl] + (long long)c * kSlabAO * nsig;
        len[sl * per + c] = kSlabAO * nsig;
      }
    if (!ta.empty())
      NA_TRY(cudaMemcpyAsync(d_ta, ta.data(), ta.size() * sizeof(PanelTask), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_rowbase, rowbase.data(), R * sizeof(long long), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_rowmul, rowmul.data(), R * sizeof(int), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_seg, seg.data(), ns * sizeof(long long), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_k0, k0.data(), nslab * sizeof(long long), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_len, len.data(), nslab * sizeof(int), cudaMemcpyHostToDevice, st));
    // cleared every call: the array keeps the previous call's contents
    NA_TRY(cudaMemsetAsync(X, 0, (size_t)prow * Kb * sizeof(double), st));
    NA_TRY(cudaMemsetAsync(Y, 0, (size_t)nri * Kb * sizeof(double), st));
    NA_TRY(cudaMemsetAsync(fx, 0, (size_t)ns * n_at * npt, st));
    NA_TRY(cudaMemsetAsync(fy, 0, (size_t)ns * n_at * nqt, st));
    // steps A and B (Eq. 3 brackets), block filter, task lists, step C
    gw::launch_panel_gemm<double>(go, nao, ctx->d_panel64, ctx->d_lam, d_ta, (int)ta.size(), maxNa, 0,
                                  0, nao, b.P0, Kb, nullptr, nullptr, X, st);
    gw::launch_panel_gemm<double>(gv, nao, ctx->d_panel64, ctx->d_lam, d_tb, (int)tb.size(), maxNb, 1,
                                  r0, R, 0, Kb, d_rowbase, d_rowmul, Y, st);
    NA_LAUNCHED();
    int pa0 = 0;
    while (ctx->ri_off[pa0 + 1] <= b.P0) ++pa0;
    int pa1 = pa0;
    while (pa1 < n_at && ctx->ri_off[pa1] < b.P1) ++pa1;
    gw::launch_operand_block_filter<double>(X, Kb, b.P0, ctx->d_ri_off, ctx->d_ao_off, d_nao, b.s0, ns,
                                            d_seg, pa0, pa1 - pa0, n_at, thr, naop, bx, fx, npt, 64, st);
    gw::launch_operand_block_filter<double>(Y, Kb, 0, ctx->d_ri_off, ctx->d_ao_off, d_nao, b.s0, ns,
                                            d_seg, 0, n_at, n_at, thr, naop, by, fy, nqt, 64, st);
    NA_LAUNCHED();
    gw::launch_build_tasks(fx, fy, nslab, npt, nqt, b.P0, prow, 0, nri, ctx->d_atom_of_ri, d_len, tasks,
                           counts, kacc, 64, per, 0, n_at, 0, nao, ctx->d_atom_of_ao, st);
    gw::launch_chi_tiles<double, double>(X, Y, Kb, b.P0, prow, nri, tasks, counts, nslab, npt, nqt,
                                         d_k0, d_len, acc, st);
    NA_LAUNCHED();
    // the host tables above are staged by the copies before the next batch
    // rewrites them; wait so that the vectors can go out of scope safely
    NA_TRY(cudaStreamSynchronize(st));
  }
  gw::launch_mirror(acc, chi_out_device, nri, ctx->d_atom_of_ri, st);
  NA_LAUNCHED();
  NA_TRY(cudaStreamSynchronize(st));
  (void)d_nri;
  return GW_OK;
}
