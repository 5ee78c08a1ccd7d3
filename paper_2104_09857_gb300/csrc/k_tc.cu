// Tensor-core (tcgen05) kernels of the mixed-precision chi(i tau) path.
//
// Split-BF16 products: every operand value x is stored as S bfloat16 slices
// x = x_0 + x_1 + ... (x_0 = bf16(x), x_{i+1} = bf16(x - x_0 - .. - x_i)).  A
// product a*b is formed from the slice pairs (i, j) with i + j <= S - 1:
// S = 2 gives 3 products (a0b0 + a0b1 + a1b0), S = 3 gives 6.
//
// One persistent, warp-specialised kernel template serves the three
// contractions of Eq. 3.  A job supplies, per output tile, the rows of the A
// and B operands (both K-major bf16 slices behind 3-D TMA maps) and the
// sequence of 64-wide K steps; and it writes the finished tile:
//   ChiJob    step C:  chi[P][Q] -= sum_k X[P][k] Y[Q][k] over the tile's slabs
//   PanelJob  steps A/B: Z[r][n] = sum_k Gg[r][k] PT[n][k] (Gg = G gathered on
//             the panel's lambda functions, PT = transposed 3c panel), split
//             into bf16 slices and scattered into X or Y, with the squared
//             Frobenius norms of its atom blocks accumulated on the way.
// Warp roles (320 threads):
//   warp 0      TMA producer (one thread): A and B slices of each K step
//   warp 1      TMEM allocator and MMA issuer (one thread)
//   warps 2..9  epilogue: every chunk of `per_chunk` K steps the TMEM
//               accumulators are read into an FP32 register sum per element;
//               the job writes it out at the end of a tile (ChiJob also every
//               kFlushChunks chunks).
// The tensor cores' FP32 accumulation loses precision with every addition
// into a large accumulator (the error grows linearly with their number), so
// the main slice product (0, 0) and the small ones accumulate separately and
// both are drained every chunk.  TMEM: 2 buffers x (main 128 + small 128)
// columns.  Every mbarrier wait is bounded; on time-out the CTA raises the
// error flag, waits (bounded) for the copies and products it issued, frees
// its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gw_internal.h"
#include "k_tc.h"

namespace gw {
namespace tc {

constexpr int kTileM = 128;
constexpr int kTileN = 128;
constexpr int kStageK = 64;   // bf16 elements per K step: one 128-byte swizzled row
constexpr int kMmaK = 16;
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kEpiCols = kTileN / 2;
constexpr int kFlushChunks = 8;
constexpr int kTmemCols = 512;
constexpr uint32_t kMaxPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false on time-out or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t i = 0; i < kMaxPolls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u) {
      if (*abort_flag) return false;
      __nanosleep(128);
    }
  }
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 128-byte rows
// (64 bf16), 8-row groups 1024 bytes apart, 1024-aligned tile base.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}
// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Per-epilogue-warp staging for coalesced stores: 32 rows x 34 bf16, or
// 32 rows x 17 floats (both 2176 bytes).
constexpr int kStgBytes = 2176;

template <int S>
struct Smem {
  static constexpr int kStages = (S == 2) ? 3 : 2;
  static constexpr int kTileBytes = kTileM * kStageK * 2;  // 16 KB, A and B alike
  static constexpr int kStageBytes = 2 * S * kTileBytes;
  static constexpr int kOperandBytes = kStages * kStageBytes;
  static constexpr int kStagingBytes = kEpiWarps * kStgBytes;
  static constexpr int kTotal = kOperandBytes + kStagingBytes + 256 + 1024;
};

// ---------------------------------------------------------------------------
// step C job
// ---------------------------------------------------------------------------
struct ChiJob {
  const int* tile_list;  // active tiles, tile = pt * nqt + qt
  int n_tiles;
  const int* tasks;
  const int* counts;
  int max_slab;
  const long long* slab_k0;
  const int* slab_len;
  int nqt, P0, prow, nri;
  double* chi;
  static constexpr bool kPeriodic = true;

  struct Tile {
    int ya, yb, cnt;
    const int* list;
  };
  __device__ Tile tile(int t) const {
    const int id = tile_list[t];
    Tile T;
    T.ya = (id / nqt) * kTileM;
    T.yb = (id % nqt) * kTileN;
    T.cnt = counts[id];
    T.list = tasks + static_cast<long long>(id) * max_slab;
    return T;
  }
  __device__ long long nsteps(const Tile& T) const {
    long long n = 0;
    for (int i = 0; i < T.cnt; ++i) n += slab_len[T.list[i]] / kStageK;
    return n;
  }
  struct Iter {
    const ChiJob* j;
    const int* list;
    int cnt, i, kk, len;
    long long k0;
    __device__ void init(const ChiJob* jj, const Tile& T) {
      j = jj;
      list = T.list;
      cnt = T.cnt;
      i = 0;
      kk = 0;
      len = cnt > 0 ? j->slab_len[list[0]] : 0;
      k0 = cnt > 0 ? j->slab_k0[list[0]] : 0;
    }
    __device__ int next() {
      const int x = static_cast<int>(k0 + kk);
      kk += kStageK;
      if (kk >= len) {
        ++i;
        kk = 0;
        if (i < cnt) {
          len = j->slab_len[list[i]];
          k0 = j->slab_k0[list[i]];
        }
      }
      return x;
    }
  };
  // Add the register sums of a warp (rows quad*32.., 64 columns from c0) into
  // chi, 16 columns at a time through the warp's staging buffer so that each
  // store instruction covers two rows of 16 consecutive doubles.
  __device__ void write(float (&acc)[kEpiCols], const Tile& T, int quad, int lane, int c0,
                        uint8_t* stg) const {
    float* f = reinterpret_cast<float*>(stg);  // [32][17]
#pragma unroll
    for (int cc = 0; cc < kEpiCols; cc += 16) {
#pragma unroll
      for (int j = 0; j < 16; ++j) f[lane * 17 + j] = acc[cc + j];
      __syncwarp();
      const int col = lane & 15, sub = lane >> 4;
      const int q = T.yb + c0 + cc + col;
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        const int p = T.ya + quad * 32 + i + sub;
        if (p < prow && q < nri) chi[static_cast<long long>(P0 + p) * nri + q] -= static_cast<double>(f[(i + sub) * 17 + col]);
      }
      __syncwarp();
    }
  }
};

// ---------------------------------------------------------------------------
// steps A / B job
// ---------------------------------------------------------------------------
struct PanelJob {
  const int4* tiles;          // (task, m-tile, n-tile, 0)
  int n_tiles;
  const PanelTaskTC* tasks;
  int mode;                   // 0: X (rows mu), 1: Y (rows sigma of the batch)
  int rows_valid;             // mode 0: n_AO; mode 1: batch AO count
  __nv_bfloat16* out;         // slices [S][slice_elems]
  long long slice_elems, ldk;
  int P0b;
  const long long* rowbase;   // mode 1, per batch row
  const int* rowmul;
  const int* row_slocal;
  float* norm2;               // mode 0: [ns][n_at][npa], mode 1: [ns][n_at][n_at]
  const int* atom_of_ri;
  const int* atom_of_ao;
  int n_at, npa, pa0, slices;
  static constexpr bool kPeriodic = false;

  struct Tile {
    int ya, yb, ksteps, task, mt, nt;
  };
  __device__ Tile tile(int t) const {
    const int4 e = tiles[t];
    const PanelTaskTC& tk = tasks[e.x];
    Tile T;
    T.task = e.x;
    T.mt = e.y;
    T.nt = e.z;
    T.ya = tk.g_row0 + e.y * kTileM;
    T.yb = tk.p_row0 + e.z * kTileN;
    T.ksteps = tk.ksteps;
    return T;
  }
  __device__ long long nsteps(const Tile& T) const { return T.ksteps; }
  struct Iter {
    int x;
    __device__ void init(const PanelJob*, const Tile&) { x = 0; }
    __device__ int next() {
      const int v = x;
      x += kStageK;
      return v;
    }
  };
  __device__ void write(float (&acc)[kEpiCols], const Tile& T, int quad, int lane, int c0,
                        uint8_t* stg) const {
    const PanelTaskTC& tk = tasks[T.task];
    const int r = T.mt * kTileM + quad * 32 + lane;
    const bool row_ok = r < rows_valid;
    long long rb = 0;
    int rm = 0, s_local = 0, m_row = 0;
    if (row_ok) {
      if (mode == 0) {
        rb = tk.seg + static_cast<long long>(r) * tk.nsig;
        s_local = tk.s_local;
        m_row = atom_of_ao[r];
      } else {
        rb = rowbase[r];
        rm = rowmul[r];
        s_local = row_slocal[r];
        m_row = tk.owner;
      }
    }
    // Walk this row's columns n = nbase + j in 16-column groups parked in the
    // thread's own staging row (no cross-lane traffic, so no warp sync): the
    // squared block norms for both modes, and the Y stores of mode 1 (there
    // consecutive rows sigma are consecutive in memory).
    float* f = reinterpret_cast<float*>(stg) + lane * 17;
    const int nbase = T.nt * kTileN + c0;
    int pw = nbase / tk.nsig;
    int sp = nbase - pw * tk.nsig;
    int key = -1;
    float ss = 0.f;
    int patom = -1, patom_pw = -1;
#pragma unroll
    for (int cc = 0; cc < kEpiCols; cc += 16) {
#pragma unroll
      for (int j = 0; j < 16; ++j) f[j] = acc[cc + j];
      if (row_ok) {
        for (int j = 0; j < 16; ++j) {
          const int n = nbase + cc + j;
          if (n >= tk.N) break;
          if (pw != patom_pw) {
            patom = atom_of_ri[tk.p0 + pw];
            patom_pw = pw;
          }
          const int blk = mode == 0 ? (s_local * n_at + m_row) * npa + (patom - pa0)
                                    : (s_local * n_at + m_row) * n_at + patom;
          float v = f[j];
          if (blk != key) {
            if (key >= 0 && ss != 0.f) atomicAdd(norm2 + key, ss);
            key = blk;
            ss = 0.f;
          }
          ss += v * v;
          if (mode == 1) {
            const long long dst = static_cast<long long>(tk.p0 + pw) * ldk + rb +
                                  static_cast<long long>(tk.aom + sp) * rm;
            for (int s = 0; s < slices; ++s) {
              const __nv_bfloat16 h = __float2bfloat16_rn(v);
              out[s * slice_elems + dst] = h;
              v -= __bfloat162float(h);
            }
          }
          if (++sp == tk.nsig) {
            sp = 0;
            ++pw;
          }
        }
      }
    }
    if (key >= 0 && ss != 0.f) atomicAdd(norm2 + key, ss);
    if (mode == 1) return;
    // X: consecutive columns (s' of one RI function) are consecutive in
    // memory; stage each slice through smem and store column-wise.
    __syncwarp();
    __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(stg);  // [32][34]
    const int mu0 = T.mt * kTileM + quad * 32;
#pragma unroll
    for (int cc = 0; cc < kEpiCols; cc += 32) {
      const int n = nbase + cc + lane;
      const bool n_ok = n < tk.N;
      const int cpw = n_ok ? n / tk.nsig : 0;
      const int csp = n - cpw * tk.nsig;
      const long long colbase = static_cast<long long>(tk.p0 + cpw - P0b) * ldk + tk.seg + csp;
      for (int s = 0; s < slices; ++s) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const __nv_bfloat16 b = __float2bfloat16_rn(acc[cc + j]);
          h[lane * 34 + j] = b;
          acc[cc + j] -= __bfloat162float(b);
        }
        __syncwarp();
        if (n_ok) {
          for (int i = 0; i < 32; ++i) {
            const int mu = mu0 + i;
            if (mu < rows_valid)
              out[s * slice_elems + colbase + static_cast<long long>(mu) * tk.nsig] = h[i * 34 + lane];
          }
        }
        __syncwarp();
      }
    }
  }
};

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <int S, class Job>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_persistent(const __grid_constant__ CUtensorMap map_a,
                    const __grid_constant__ CUtensorMap map_b, const Job job, int per_chunk,
                    int* __restrict__ err_flag) {
  using L = Smem<S>;
  constexpr int kStages = L::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* operands = smem;
  uint8_t* staging = smem + L::kOperandBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOperandBytes + L::kStagingBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* acc_full = bars + 2 * kStages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed_parity[kStages];
      bool armed[kStages];
      for (int s = 0; s < kStages; ++s) armed[s] = false, armed_parity[s] = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < job.n_tiles && ok; t += gridDim.x) {
        const typename Job::Tile T = job.tile(t);
        const long long n = job.nsteps(T);
        typename Job::Iter it;
        it.init(&job, T);
        for (long long i = 0; i < n; ++i) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* st = operands + stage * L::kStageBytes;
          mbar_expect_tx(&full[stage], L::kStageBytes);
          armed[stage] = true;
          armed_parity[stage] = phase;
          const int x = it.next();
          for (int s = 0; s < S; ++s) {
            tma_load_3d(st + s * L::kTileBytes, &map_a, x, T.ya, s, &full[stage]);
            tma_load_3d(st + (S + s) * L::kTileBytes, &map_b, x, T.yb, s, &full[stage]);
          }
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(err_flag, 1);
        for (int s = 0; s < kStages; ++s)
          if (armed[s])
            for (uint32_t t = 0; t < kMaxPolls && !mbar_try_wait(&full[s], armed_parity[s]); ++t) {
            }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(kTileM, kTileN);
      int stage = 0;
      uint32_t phase = 0;
      int chunk = 0;
      bool ok = true, issued_any = false;
      for (int t = blockIdx.x; t < job.n_tiles && ok; t += gridDim.x) {
        const typename Job::Tile T = job.tile(t);
        const long long n = job.nsteps(T);
        int step = 0;
        for (long long i = 0; i < n; ++i) {
          const int buf = chunk & 1;
          if (step == 0) {
            const uint32_t use = static_cast<uint32_t>(chunk >> 1);
            if (!mbar_wait(&acc_empty[buf], (use & 1u) ^ 1u, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          if (!mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_main = tmem + static_cast<uint32_t>(buf * 256);
          const uint32_t d_small = d_main + 128u;
          const uint32_t st = smem_u32(operands + stage * L::kStageBytes);
#pragma unroll
          for (int k = 0; k < kStageK / kMmaK; ++k) {
            const uint64_t koff = static_cast<uint64_t>((k * kMmaK * 2) >> 4);
            const bool chunk_start = (step == 0 && k == 0);
            mma_bf16(d_main, desc_sw128(st) + koff, desc_sw128(st + S * L::kTileBytes) + koff, idesc,
                     chunk_start ? 0u : 1u);
            bool first_small = true;
#pragma unroll
            for (int a = 0; a < S; ++a) {
#pragma unroll
              for (int b = 0; b < S - a; ++b) {
                if (a == 0 && b == 0) continue;
                mma_bf16(d_small, desc_sw128(st + a * L::kTileBytes) + koff,
                         desc_sw128(st + (S + b) * L::kTileBytes) + koff, idesc,
                         (chunk_start && first_small) ? 0u : 1u);
                first_small = false;
              }
            }
          }
          issued_any = true;
          mma_commit(&empty[stage]);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
          if (++step == per_chunk || i == n - 1) {
            mma_commit(&acc_full[buf]);
            ++chunk;
            step = 0;
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(err_flag, 2);
        if (issued_any) {
          mma_commit(drain);
          for (uint32_t t = 0; t < kMaxPolls && !mbar_try_wait(drain, 0); ++t) {
          }
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int c0 = half * kEpiCols;
    uint8_t* stg = staging + (warp - 2) * kStgBytes;
    const uint32_t row_addr = tmem + (static_cast<uint32_t>(quad * 32) << 16);
    float acc[kEpiCols];
    int chunk = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < job.n_tiles && ok; t += gridDim.x) {
      const typename Job::Tile T = job.tile(t);
      const long long n = job.nsteps(T);
      const long long nch = (n + per_chunk - 1) / per_chunk;
#pragma unroll
      for (int j = 0; j < kEpiCols; ++j) acc[j] = 0.f;
      for (long long c = 0; c < nch; ++c, ++chunk) {
        const int buf = chunk & 1;
        const uint32_t use = static_cast<uint32_t>(chunk >> 1);
        if (!mbar_wait(&acc_full[buf], use & 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int g = 0; g < kEpiCols / 8; ++g) {
          const uint32_t col = static_cast<uint32_t>(buf * 256 + c0 + g * 8);
          uint32_t vm[8], vs[8];
          tmem_ld8(row_addr + col, vm);
          tmem_ld8(row_addr + col + 128u, vs);
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[g * 8 + j] += __uint_as_float(vm[j]) + __uint_as_float(vs[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
        if (Job::kPeriodic && (c + 1) % kFlushChunks == 0 && c + 1 < nch) {
          job.write(acc, T, quad, lane, c0, stg);
#pragma unroll
          for (int j = 0; j < kEpiCols; ++j) acc[j] = 0.f;
        }
      }
      if (!ok) break;
      if (nch > 0) job.write(acc, T, quad, lane, c0, stg);
    }
    if (!ok) {
      *abort_flag = 1;
      if (lane == 0) atomicOr(err_flag, 4);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
// Gathered, split Green's function for the panel tasks:
//   Gg[s][g_row0 + r][k] = slice s of G[rbase + r][lam[lam_off + k]]
// for r < rows_valid and k < K, zero elsewhere up to (rows, kmax).
__global__ void k_gather_g(const double* __restrict__ g, int nao, const PanelTaskTC* __restrict__ tasks,
                           const int* __restrict__ lam, int rbase, int rows_valid, int rows_per_task,
                           int kmax, int slices, long long slice_elems,
                           __nv_bfloat16* __restrict__ out) {
  const PanelTaskTC tk = tasks[blockIdx.y];
  const long long n = static_cast<long long>(rows_per_task) * kmax;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / kmax), k = static_cast<int>(i % kmax);
    double v = 0.0;
    if (r < rows_valid && k < tk.K) v = g[static_cast<long long>(rbase + r) * nao + lam[tk.lam_off + k]];
    const long long dst = static_cast<long long>(tk.g_row0 + r) * kmax + k;
    for (int s = 0; s < slices; ++s) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      out[s * slice_elems + dst] = h;
      v -= static_cast<double>(__bfloat162float(h));
    }
  }
}

// Transposed, split panel: PT[s][p_row0 + n][k] = slice s of panel[k][n]
// (k < K, n < N; zero padding up to (npad, kmax)).  32x32 tiles via smem.
__global__ void k_transpose_panel(const double* __restrict__ pool, const PanelTaskTC* __restrict__ tasks,
                                  int kmax, int slices, long long slice_elems,
                                  __nv_bfloat16* __restrict__ out) {
  __shared__ double tile[32][33];
  const PanelTaskTC tk = tasks[blockIdx.z];
  const int npad = (tk.N + kTileN - 1) / kTileN * kTileN;
  const int n0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  if (n0 >= npad || k0 >= kmax) return;
  const double* p = pool + tk.panel_off;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int k = k0 + i, nn = n0 + tx;
    tile[i][tx] = (k < tk.K && nn < tk.N) ? p[static_cast<long long>(k) * tk.N + nn] : 0.0;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int nn = n0 + i, k = k0 + tx;
    double v = tile[tx][i];
    const long long dst = static_cast<long long>(tk.p_row0 + nn) * kmax + k;
    for (int s = 0; s < slices; ++s) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      out[s * slice_elems + dst] = h;
      v -= static_cast<double>(__bfloat162float(h));
    }
  }
}

// Norms of the atom blocks of an operand from the accumulated squares; zero
// the filtered ones (norm < thr, norm > 0) in every slice; flag the kept
// nonzero blocks and the (slab, tile) pairs they touch.
__global__ void k_slices_block_filter(__nv_bfloat16* __restrict__ Z, int slices, long long slice_elems,
                                      long long ldk, int rowoff, const int* __restrict__ ri_off,
                                      const int* __restrict__ ao_off, const int* __restrict__ n_ao,
                                      int s0, int ns, const long long* __restrict__ seg, int pa0,
                                      int npa, int n_at, double thr, int naop,
                                      const float* __restrict__ norm2,
                                      unsigned char* __restrict__ blockflag,
                                      unsigned char* __restrict__ tileflag, int ntile,
                                      int tile_rows) {
  long long w = static_cast<long long>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  const long long nblk = static_cast<long long>(ns) * n_at * npa;
  if (w >= nblk) return;
  const int pl = static_cast<int>(w % npa);
  const long long t = w / npa;
  const int m = static_cast<int>(t % n_at);
  const int sl = static_cast<int>(t / n_at);
  const int s = s0 + sl, p = pa0 + pl;
  const double nrm = sqrt(static_cast<double>(norm2[w]));
  const bool kept = !(nrm < thr);
  const bool nz = kept && nrm > 0.0;
  if (lane == 0) blockflag[w] = nz;
  const int nsig = n_ao[s];
  const int rows0 = ri_off[p] - rowoff, nrows = ri_off[p + 1] - ri_off[p];
  const long long c0 = seg[sl] + static_cast<long long>(ao_off[m]) * nsig;
  const int ncols = n_ao[m] * nsig;
  if (!kept && nrm > 0.0) {
    for (int r = 0; r < nrows; ++r)
      for (int c = lane; c < ncols; c += 32)
        for (int sc = 0; sc < slices; ++sc)
          Z[sc * slice_elems + static_cast<long long>(rows0 + r) * ldk + c0 + c] = __float2bfloat16_rn(0.f);
  }
  if (nz) {
    const int ts = rows0 / tile_rows, te = (rows0 + nrows - 1) / tile_rows;
    for (int tt = ts + lane; tt <= te; tt += 32)
      tileflag[(static_cast<long long>(sl) * n_at + m) * ntile + tt] = 1;
    (void)naop;
  }
}

// FP64 [rows][cols] (row stride ld) -> bf16 slices [S][rows][kpad], zero for
// k >= cols
__global__ void k_split_f64(const double* __restrict__ a, long long ld, int rows, int cols, int kpad,
                            int slices, __nv_bfloat16* __restrict__ out) {
  const long long n = static_cast<long long>(rows) * kpad;
  const long long slice = n;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / kpad), k = static_cast<int>(i % kpad);
    double v = k < cols ? a[static_cast<long long>(r) * ld + k] : 0.0;
    for (int s = 0; s < slices; ++s) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      out[s * slice + i] = h;
      v -= static_cast<double>(__bfloat162float(h));
    }
  }
}

}  // namespace tc

void launch_split_f64(const double* a, long long ld, int rows, int cols, int kpad, int slices,
                      void* out, cudaStream_t st) {
  const long long n = static_cast<long long>(rows) * kpad;
  if (n == 0) return;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  tc::k_split_f64<<<static_cast<unsigned>(blocks), 256, 0, st>>>(a, ld, rows, cols, kpad, slices,
                                                                static_cast<__nv_bfloat16*>(out));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

template <int S, class Job>
int launch_persistent(const CUtensorMap& ma, const CUtensorMap& mb, const Job& job, int per_chunk,
                      int* err_flag, cudaStream_t st) {
  if (job.n_tiles == 0) return 0;
  constexpr int smem = tc::Smem<S>::kTotal;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tc::k_tc_persistent<S, Job>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess)
      return -1;
    attr = true;
  }
  const int grid = job.n_tiles < num_sms() ? job.n_tiles : num_sms();
  tc::k_tc_persistent<S, Job><<<grid, tc::kThreads, smem, st>>>(ma, mb, job, per_chunk, err_flag);
  return 0;
}
}  // namespace

int make_slice_map(CUtensorMap* map, const void* base, long long k_len, long long rows, int slices,
                   int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return -1;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (k_len * 2) % 16 != 0) return -2;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(k_len), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(slices)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(k_len * 2),
                           static_cast<cuuint64_t>(k_len * 2 * rows)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(tc::kStageK), static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int tc_tile_rows() { return tc::kTileM; }

int launch_chi_tc(int slices, const CUtensorMap& mx, const CUtensorMap& my, const int* tile_list,
                  int n_tiles, const int* tasks, const int* counts, int max_slab,
                  const long long* slab_k0, const int* slab_len, int P0, int prow, int nri, int nqt,
                  double* chi, int flush_k, int* err_flag, cudaStream_t st) {
  tc::ChiJob job{tile_list, n_tiles, tasks, counts, max_slab, slab_k0, slab_len, nqt, P0, prow, nri, chi};
  const int per_chunk = flush_k / tc::kStageK > 0 ? flush_k / tc::kStageK : 1;
  if (slices == 2) return launch_persistent<2>(mx, my, job, per_chunk, err_flag, st);
  if (slices == 3) return launch_persistent<3>(mx, my, job, per_chunk, err_flag, st);
  return -4;
}

int launch_panel_tc(int slices, const CUtensorMap& mg, const CUtensorMap& mp, const int4* tiles,
                    int n_tiles, const PanelTaskTC* tasks, int mode, int rows_valid, void* out,
                    long long slice_elems, long long ldk, int P0b, const long long* rowbase,
                    const int* rowmul, const int* row_slocal, float* norm2, const int* atom_of_ri,
                    const int* atom_of_ao, int n_at, int npa, int pa0, int flush_k, int* err_flag,
                    cudaStream_t st) {
  tc::PanelJob job{tiles, n_tiles, tasks, mode, rows_valid, static_cast<__nv_bfloat16*>(out),
                   slice_elems, ldk, P0b, rowbase, rowmul, row_slocal, norm2, atom_of_ri,
                   atom_of_ao, n_at, npa, pa0, slices};
  const int per_chunk = flush_k / tc::kStageK > 0 ? flush_k / tc::kStageK : 1;
  if (slices == 2) return launch_persistent<2>(mg, mp, job, per_chunk, err_flag, st);
  if (slices == 3) return launch_persistent<3>(mg, mp, job, per_chunk, err_flag, st);
  return -4;
}

void launch_gather_g(const double* g, int nao, const PanelTaskTC* tasks, int ntasks, const int* lam,
                     int rbase, int rows_valid, int rows_per_task, int kmax, int slices,
                     long long slice_elems, void* out, cudaStream_t st) {
  if (ntasks == 0) return;
  long long per = static_cast<long long>(rows_per_task) * kmax;
  int bx = static_cast<int>((per + 255) / 256);
  if (bx > 1024) bx = 1024;
  dim3 grid(bx, ntasks);
  tc::k_gather_g<<<grid, 256, 0, st>>>(g, nao, tasks, lam, rbase, rows_valid, rows_per_task, kmax,
                                       slices, slice_elems, static_cast<__nv_bfloat16*>(out));
}

void launch_transpose_panels(const double* pool, const PanelTaskTC* tasks, int ntasks, int max_npad,
                             int kmax, int slices, long long slice_elems, void* out, cudaStream_t st) {
  if (ntasks == 0) return;
  for (int z0 = 0; z0 < ntasks; z0 += 65535) {
    const int nz = ntasks - z0 < 65535 ? ntasks - z0 : 65535;
    dim3 grid((max_npad + 31) / 32, (kmax + 31) / 32, nz);
    tc::k_transpose_panel<<<grid, 256, 0, st>>>(pool, tasks + z0, kmax, slices, slice_elems,
                                                static_cast<__nv_bfloat16*>(out));
  }
}

void launch_slices_block_filter(void* Z, int slices, long long slice_elems, long long ldk, int rowoff,
                                const int* ri_off, const int* ao_off, const int* n_ao, int s0,
                                int ns, const long long* seg, int pa0, int npa, int n_at,
                                double thr, int naop, const float* norm2, unsigned char* blockflag,
                                unsigned char* tileflag, int ntile, int tile_rows, cudaStream_t st) {
  const long long nblk = static_cast<long long>(ns) * n_at * npa;
  if (nblk == 0) return;
  tc::k_slices_block_filter<<<static_cast<unsigned>((nblk + 7) / 8), 256, 0, st>>>(
      static_cast<__nv_bfloat16*>(Z), slices, slice_elems, ldk, rowoff, ri_off, ao_off, n_ao, s0, ns,
      seg, pa0, npa, n_at, thr, naop, norm2, blockflag, tileflag, ntile, tile_rows);
}

}  // namespace gw
