// Internal declarations shared by the translation units of libgwchi.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/gwchi.h"

namespace gw {

// Named NVTX range over a scope, for profilers (Nsight Compute's --nvtx
// filters, timeline tools); costs a predicted branch when no tool is attached.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// CUDA events destroyed with the scope, also on early error returns.
template <int N>
struct ScopedEvents {
  cudaEvent_t ev[N];
  int made = 0;
  cudaError_t create() {
    for (; made < N; ++made) {
      const cudaError_t e = cudaEventCreate(&ev[made]);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaEvent_t operator[](int i) const { return ev[i]; }
  ~ScopedEvents() {
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  }
};

// Slab: 64 consecutive primary functions mu of one sigma-atom segment of the
// K dimension of the step-C operands.
constexpr int kSlabAO = 64;

// Per-owner-atom dense panel of the three-centre tensor:
//   panel[k][pw][s'] = T[lambda_k, sigma = ao_off(owner) + s', P = p0 + pw]
// k runs over the primary functions of the atoms that share a stored block
// with the owner (ascending atom order), pw over the contiguous RI window
// [p0, p0 + npw) of those blocks, s' over the owner's primary functions.
struct PanelDesc {
  long long off;  // element offset of the panel in the panel pool
  int K;          // rows (gathered lambda functions)
  int nsig;       // n_ao(owner)
  int p0, npw;    // RI window
  int lam_off;    // offset into the lambda-index pool (K entries)
  int owner;
};

// One grouped-GEMM problem of steps A/B: Z[r][n] = sum_k G[lam[k]][r] P[k][n].
struct PanelTask {
  long long panel_off;
  int K, N;       // N = npw * nsig
  int lam_off;
  int npw, nsig;  // panel window and owner size (n = pw * nsig + s')
  int p0;
  int aom;        // mode B: AO offset of the panel owner (mu = aom + s')
  long long seg;  // mode A: K offset of the owner's segment in X
};

// One panel problem of the tensor-core steps A/B (see k_tc.cu):
//   Z[r][n] = sum_k Gg[g_row0 + r][k] * PT[p_row0 + n][k],  k < 64 * ksteps
struct PanelTaskTC {
  long long panel_off;  // FP64 panel in the pool (transpose build)
  long long seg;        // mode 0: K offset of the owner's segment in X
  int g_row0, p_row0, ksteps;  // ksteps: K steps of 64
  int K, N, npw, nsig, p0, aom;
  int s_local, owner, lam_off;
};

// One operand batch: the sigma-atoms (owners) [s0, s1) against the chunk of
// mu-atoms [m0, m1).  K runs over (owner s, chunk-local mu < Lc, sigma' of s);
// X rows are the RI window [P0, P1) of the owners' panels, Y rows the RI
// window [Q0, Q1) of the chunk's panels.  A chunk of every atom has Lc =
// n_AO rounded to kSlabAO and Y over all RI functions.
struct Batch {
  int s0, s1;         // owner atoms [s0, s1)
  int P0, P1;         // RI window of X rows
  long long Kb;       // K length (sum over owners of Lc * nsig)
  int nslab;          // (s1 - s0) * Lc / kSlabAO
  std::vector<long long> seg;  // per owner: K offset
  int m0 = 0, m1 = 0;          // mu-atom chunk
  int mu0 = 0, nmu = 0, Lc = 0;  // its AOs [mu0, mu0 + nmu), K segment length per sigma'
  int Q0 = 0, Q1 = 0;          // RI window of Y rows
};

// Builds (or reuses) the owner panels of the 3c tensor for filter threshold
// thr; defined with the chi orchestration.
int build_panels_for(gw_ctx* ctx, double thr);

// Learned-screening hook of a tensor-core batch, called after the task lists
// are built and before step C (defined in gw_mlp.cu).  Mode 1 logs
// (features, log10 contribution norm) of every task; mode 2 drops the tasks
// the network predicts below thr (minus the margin) from the lists.
struct MlpBatch {
  int s0, ns, P0, prow, nslab, npt, nqt, tile, per, pa0, npa, slices;
  int m0, nmc, mu0, nmu;  // mu-atom chunk and its AOs
  int Q0, qrow, qa0, nqa; // Y rows (RI functions) and their RI atoms
  int f16;           // slices in binary16 holding X / xinv and Y / yinv
  float xinv, yinv;
  long long Kb;
  const void* xs;
  const void* ys;
  const float* bx2;
  const float* by2;
  const unsigned char* bx;
  const unsigned char* by;
  int* tasks;
  int* counts;
  long long* kacc;
  const long long* slab_k0;
  const int* slab_len;
  double tau, thr;
};
int mlp_batch_hook(gw_ctx* ctx, const MlpBatch& mb);

}  // namespace gw

struct gw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;

  // basis
  int n_at = 0, nao = 0, nri = 0, naop = 0;  // naop = nao rounded up to kSlabAO
  std::vector<double> xyz;
  std::vector<int> n_ao, n_ri, ao_off, ri_off;  // offsets have n_at + 1 entries
  int* d_ao_off = nullptr;
  int* d_ri_off = nullptr;
  int* d_atom_of_ri = nullptr;
  int* d_atom_of_ao = nullptr;
  std::vector<int> h_atom_of_ao;  // host copy

  // three-centre tensor (A <= B blocks as given)
  long long n_blocks = 0, n_elems = 0;
  std::vector<int> blk;              // 3 per block
  std::vector<long long> blk_off;    // n_blocks + 1
  double* d_t3 = nullptr;
  float* d_t3f = nullptr;  // the tensor kept in FP32 instead (option tensor_fp32)
  int tensor_fp32 = 0;     // option: applies at the next gw_set_3c_tensor
  int* d_blk = nullptr;
  long long* d_blk_off = nullptr;
  double* d_blk_norm = nullptr;
  std::vector<double> blk_norm;
  double t_absmax = 0.0;  // max |(mu sigma|P)| over the stored blocks

  // Green's function inputs
  bool have_greens = false;
  double* d_C = nullptr;
  double* d_eps = nullptr;
  std::vector<double> h_eps;  // host copy of the levels given to gw_set_greens
  int n_occ = 0;
  double mu = 0.0;
  std::vector<double> tau;

  // panel plan (depends on thr through the 3c block filter): descriptors,
  // the kept blocks with the K offset of their partner atom in each owner's
  // panel, and the device lambda lists; every route needs it
  bool plan_ok = false;
  double plan_thr = -1.0;
  std::vector<gw::PanelDesc> panels;   // per atom (K == 0: no panel)
  std::vector<int> plan_kept;          // kept 3c blocks
  std::vector<int> plan_kB, plan_kA;   // per kept block (A, B, P): K offset of A in panel(B), of B in panel(A)
  // per owner s: (lambda-atom l, sum over its kept blocks (l, s, P) of
  // 2 n(l) n(s) n(P)), CSR; the useful flops of steps A and B per batch
  std::vector<int> wl_off, wl_atom;
  std::vector<double> wl_w;
  // FP64 panel pool (CUDA-core routes, the self-energy and the allocation-free
  // entry point; the tensor-core route builds its split panels from the
  // stored blocks instead)
  bool panels_ok = false;
  double panels_thr = -1.0;
  long long panel_elems = 0;
  double* d_panel64 = nullptr;
  float* d_panel32 = nullptr;
  bool panel32_ok = false;
  int* d_lam = nullptr;
  long long lam_total = 0;

  // transposed, split panels for the tensor-core steps A/B
  bool pt_ok = false;
  int pt_slices = 0, pt_f16 = 0;
  double pt_thr = -1.0;
  double pt_scale = 1.0;          // binary16 slices hold pt_scale * T
  double tc_scale[4] = {1, 1, 1, 1};  // binary16 scales of G^occ, G^virt, X, Y (current tau)
  void* d_pt = nullptr;           // [slices][pt_rows][pt_kmax] 16-bit slices
  long long pt_rows = 0;
  int pt_kmax = 0;
  std::vector<gw::PanelTaskTC> pt_tasks;  // per atom (K == 0: none)
  // streamed split panels: when the whole set does not fit, step A builds
  // the panels of a batch's owners and step B those of a chunk's atoms, each
  // in a region of its own, from the stored blocks
  bool pt_stream = false;
  int panel_stream = 0;            // option: 1 always stream
  int ptB_m0 = -1, ptB_m1 = -1;    // chunk whose panels region B holds
  long long ptB_rows = 0;
  void* d_ptB_region = nullptr;    // region B's buffer (a named work buffer)
  std::vector<int> ptB_row0;       // per atom: first row in region B (-1: absent)
  std::vector<int> plan_atom_off, plan_atom_blk;  // per atom: indices into plan_kept of its blocks
  // per RI row q: the owner atoms whose panel windows cover q, [ycov_lo,
  // ycov_hi] (lo < 0: none); valid when they are contiguous for every q
  // tensor-core batches of the current tau point whose flop counts and
  // timings are read once at its end (no per-batch host synchronisation)
  struct TcPending {
    size_t batch_idx;
    long long fc_off;
    int fc_n;
    double fc_scale;
  };
  std::vector<TcPending> tc_pending;
  long long tc_fc_used = 0;
  double tc_issue_per_k = 0.0;  // issued flops per reduction element of a step-C tile
  bool ycov_valid = false;  // cleared whenever the panels are rebuilt
  bool ycov_ok = false;
  int* d_ycov_lo = nullptr;
  int* d_ycov_hi = nullptr;

  // learned screening: network (FP32 master, bf16 copy, Adam moments)
  float* d_mlp_theta = nullptr;
  void* d_mlp_wb = nullptr;
  float* d_mlp_m = nullptr;
  float* d_mlp_v = nullptr;
  int mlp_step = 0;
  bool mlp_ready = false;
  double mlp_margin = 0.5;          // log10 units added to the prediction
  int mlp_mode = 0;                 // 0 off, 1 log tasks, 2 screen tasks (set per call)
  std::vector<float> mlp_log_feat;  // logged features / targets (mode 1)
  std::vector<float> mlp_log_tgt;
  long long mlp_skipped = 0, mlp_seen = 0;
  double cur_tau = 0.0;  // tau of the point being computed
  double mlp_k_before = 0.0, mlp_k_after = 0.0;

  // options
  double batch_bytes = 40e9;
  int batch_atoms = 0;
  // tensor cores: main FP32 accumulator drained every flush_k reduction elements
  int flush_k = 64;
  int last_precision = -1;
  int c_order = 0;   // step-C tile order: 0 longest first, 1 grouped raster
  // step-C work units: tiles split into runs of about c_split_k reduction
  // elements, FP64 atomics into chi (0: whole tiles, bitwise reproducible)
  int c_split_k = 2048;
  // step-C work units handed out in order from a counter (1) or a fixed
  // share per CTA (0)
  int c_dynamic = 1;
  // G block flags of the current tau point (host copies, n_at x n_at; null
  // or all kept when nothing is filtered): steps A/B leave out the tiles
  // whose G rows are all dropped blocks
  const std::vector<unsigned char>* cur_fo = nullptr;
  const std::vector<unsigned char>* cur_fv = nullptr;
  // mu-atoms per chunk of the tensor-core route's 2-D batches (0: the fewest
  // equal chunks that keep one owner's operands within budget / 8)
  int mu_chunk_atoms = 0;
  // two-slice forms: steps A/B stage each finished tile in shared memory and
  // write whole runs of X and Y (0: per-element stores from registers)
  int panel_staged = 1;

  // named device work buffers (grown on demand) and the step timing events
  // of this context; a context is used by one host thread at a time
  std::map<std::string, std::pair<void*, size_t>> work;
  std::vector<cudaEvent_t> events;

  // test hooks (options "test_fail_alloc", "test_stall_tc")
  int test_fail_alloc = 0;  // the next new work-buffer allocation fails
  int test_stall = 0;       // tensor-core kernels wait on a dependency never met

  gw_stats stats{};
};
