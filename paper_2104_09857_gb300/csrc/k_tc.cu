// Tensor-core (tcgen05) kernels of the mixed-precision chi(i tau) path.
//
// Split products: every operand value x is stored as S 16-bit slices
// x = x_0 + x_1 + ... (x_0 = h(x), x_{i+1} = h(x - x_0 - .. - x_i)), h the
// rounding to bfloat16 or, for the FP16 form, to binary16 after scaling the
// whole operand by a power of two c (slices of c x; the epilogues multiply by
// the exact reciprocal).  A product a*b is formed from the slice pairs (i, j)
// with i + j <= S - 1: S = 2 gives 3 products (a0b0 + a0b1 + a1b0), S = 3
// gives 6.  With 8 significant bits per bf16 slice, S = 3 carries 24 bits;
// with 11 per binary16 slice, S = 2 carries 22.
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
// Warp roles (576 threads):
//   warp 0      TMA producer (one thread): A and B slices of each K step
//   warp 1      TMEM allocator and MMA issuer (one thread)
//   warps 2..17 epilogue (4 lane quadrants x 4 groups of 32 columns): the
//               TMEM accumulators are read into an FP32
//               register sum per element; the job writes it out at the end
//               of a tile (ChiJob also every kWriteK reduction elements), or
//               stages it in shared memory and copies it out from there
// The tensor cores' FP32 accumulation rounds each MMA step's result toward
// zero (measured: a bias of about half an ulp of the running sum per step,
// so the relative error grows with the number of steps between drains), so
// the accumulator is drained every few MMA steps (flush_k reduction
// elements).  Within one drain interval the small slice products (2^-8 of
// the main one or less) are issued first, while the sum is small: their
// roundings fall below the main product's ulp, and the interval costs the
// main product's few roundings only.  TMEM: four accumulators of 128 columns,
// used in turn (the MMA may run three drains ahead of the epilogue, and a
// tile starts without waiting for the previous one's last drain).  Every
// mbarrier wait is bounded; on time-out the CTA raises the error flag, waits
// (bounded) for the copies and products it issued, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>

#include "gw_internal.h"
#include "k_tc.h"

namespace gw {
namespace tc {

constexpr int kTileM = 128;
constexpr int kTileN = 128;
constexpr int kStageK = 64;   // bf16 elements per K step: one 128-byte swizzled row
constexpr int kMmaK = 16;
constexpr int kEpiWarps = 16;                 // 4 TMEM lane quadrants x 4 column groups
constexpr int kEpiCols = kTileN / 4;          // accumulator columns per epilogue warp
constexpr int kWriteK = 2048;  // reduction elements between ChiJob write-outs (one per split-K unit)
constexpr int kTmemCols = 512;
constexpr int kAccBufs = 4;   // accumulators: TMEM columns [128 b, 128 b + 128)
constexpr uint32_t kSuspendNs = 20000;            // longest suspension of one try_wait
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // a wait gives up after 2 s

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
// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps in hardware (up to kSuspendNs) instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of the given parity; false on time-out
// (kWaitLimitNs) or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait_sleep(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait_sleep(bar, parity)) return true;
    if (*abort_flag) return false;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}
// Bounded wait without abort check (clean-up after an abort).
__device__ __forceinline__ void mbar_wait_cleanup(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait_sleep(bar, parity) && global_ns() - t0 < kWaitLimitNs) {
  }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// Bulk copy of `bytes` (a multiple of 16) from shared to global memory, both
// addresses 16-byte aligned, as a bulk async-group of the issuing thread.
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
               "r"(smem_u32(ssrc)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of this thread's bulk groups have been read
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// this thread's bulk groups have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's shared-memory writes before later async-proxy reads
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
// Instruction descriptor of kind::f16: BF16 x BF16 (or F16 x F16) -> FP32,
// both operands K-major.
__host__ __device__ constexpr uint32_t idesc_f32(int m, int n, bool f16) {
  return (1u << 4) | (f16 ? 0u : ((1u << 7) | (1u << 10))) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}
// One slice of v (bf16, or binary16 when f16): returns its bits and leaves
// the remainder v - slice in v (exact).
__device__ __forceinline__ uint16_t take_slice(float& v, bool f16) {
  if (f16) {
    const __half h = __float2half_rn(v);
    v -= __half2float(h);
    return __half_as_ushort(h);
  }
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  v -= __bfloat162float(h);
  return __bfloat16_as_ushort(h);
}
__device__ __forceinline__ uint16_t take_slice(double& v, bool f16) {
  if (f16) {
    const __half h = __double2half(v);
    v -= static_cast<double>(__half2float(h));
    return __half_as_ushort(h);
  }
  const __nv_bfloat16 h = __double2bfloat16(v);
  v -= static_cast<double>(__bfloat162float(h));
  return __bfloat16_as_ushort(h);
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
// acc[j] += TMEM[lane row][taddr column + j], j < 32: one 32-column load and
// its wait, or (kHalves = 2) two 16-column loads and waits, which keeps 16
// fewer registers live.  The registers pass through the wait's asm so that
// no use of them can be scheduled before it.
template <int kHalves>
__device__ __forceinline__ void tmem_add32(uint32_t taddr, float (&acc)[32]) {
  if (kHalves == 1) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] += __uint_as_float(r[k]);
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + static_cast<uint32_t>(h * 16)));
      asm volatile("tcgen05.wait::ld.sync.aligned;"
                   : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                   :
                   : "memory");
#pragma unroll
      for (int k = 0; k < 16; ++k) acc[h * 16 + k] += __uint_as_float(r[k]);
    }
  }
}
// Drain cadence of the persistent kernel, in MMA steps of kMmaK reduction
// elements: the accumulator every `main` steps; periodic jobs write out
// every `write_every` drains.
struct Cadence {
  int main, write_every;
  int stall;  // test hook: the epilogue first waits on a barrier nothing arrives at
};

// Per-epilogue-warp staging: 32 rows x kStgCols floats, row pitch
// kStgCols + 1 (no bank conflicts on column reads).
constexpr int kStgCols = 8;
constexpr int kStgPitch = kStgCols + 1;
constexpr int kStgBytes = 32 * kStgPitch * 4;

// Whole-tile staging (jobs with kTileStaging): the finished tile as its two
// 16-bit slices, two planes of kPlaneElems elements each, laid out in the
// order of the output runs (see PanelStagedJob).
constexpr int kPlaneElems = 23040;
constexpr int kTileStgBytes = 2 * kPlaneElems * 2;

// Threads of a launch: producer, MMA issuer and the epilogue warps.
constexpr int kThreads = (2 + kEpiWarps) * 32;

template <int S, class Job>
struct Smem {
  // a job that stages whole tiles keeps two operand stages to make room
  static constexpr int kStages = Job::kTileStaging ? 2 : ((S == 2) ? 3 : 2);
  static constexpr int kTileBytes = kTileM * kStageK * 2;  // 16 KB, A and B alike
  static constexpr int kStageBytes = 2 * S * kTileBytes;
  static constexpr int kOperandBytes = kStages * kStageBytes;
  static constexpr int kStagingBytes = Job::kTileStaging ? kTileStgBytes : kEpiWarps * kStgBytes;
  static constexpr int kTotal = kOperandBytes + kStagingBytes + 256 + 1024;
};

// What a tile-staging job's epilogue needs besides its registers: the
// staging area, two barriers (tile staged by every epilogue warp; staging
// area free again), the abort flag, the warp's index among the epilogue
// warps and the number of tiles this CTA has staged so far.
struct EpiCtx {
  uint8_t* staging;
  uint64_t* staged;
  uint64_t* freed;
  volatile int* abort;
  int warp;
  int tile_no;
};

// ---------------------------------------------------------------------------
// step C job
// ---------------------------------------------------------------------------
struct ChiJob {
  const int* tile_list;  // work units: tile = pt * nqt + qt of unit u
  int n_tiles;           // number of units
  const int* unit_first; // optional (split K): first list entry and entry
  const int* unit_count; // count of unit u; null = the tile's whole list
  const int* tasks;
  const int* counts;
  int max_slab;
  const long long* slab_k0;
  const int* slab_len;
  int nqt, P0, prow, nri;
  int qlim;         // Y row ql adds into chi column Q0 + ql; written while ql < qlim = n_RI - Q0
  double* chi;      // chi + Q0 (row stride nri)
  float out_scale;  // 1 / (scale of the A operand x scale of the B operand)
  const int* n_dev; // optional: number of units in device memory (n_tiles = capacity)
  int* work;        // optional: counter handing the units out in order (zeroed before the launch)
  static constexpr bool kPeriodic = true;
  static constexpr bool kTileStaging = false;
  static constexpr bool kDynamic = true;
  static constexpr int kDrainHalves = 2;  // 96 registers: one 32-column load would spill

  struct Tile {
    int ya, yb, cnt;
    const int* list;
  };
  __device__ Tile tile(int t) const {
    const int id = tile_list[t];
    Tile T;
    T.ya = (id / nqt) * kTileM;
    T.yb = (id % nqt) * kTileN;
    if (unit_first) {
      T.cnt = unit_count[t];
      T.list = tasks + static_cast<long long>(id) * max_slab + unit_first[t];
    } else {
      T.cnt = counts[id];
      T.list = tasks + static_cast<long long>(id) * max_slab;
    }
    return T;
  }
  __device__ long long nsteps(const Tile& T) const {
    long long n = 0;
    for (int i = 0; i < T.cnt; ++i) n += slab_len[T.list[i]] / kStageK;
    return n;
  }
  __device__ int items() const { return n_dev ? *n_dev : n_tiles; }
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
  // Add the register sums of a warp (rows quad*32.., kEpiCols columns from
  // c0) into chi, kStgCols columns at a time through the warp's staging
  // buffer, so that each store instruction covers 4 rows of 8 consecutive
  // doubles.
  __device__ void write(float (&acc)[kEpiCols], const Tile& T, int quad, int lane, int c0,
                        uint8_t* stg) const {
    float* f = reinterpret_cast<float*>(stg);  // [32][kStgPitch]
    constexpr int kRowsPer = 32 / kStgCols;    // rows covered by one warp store
#pragma unroll
    for (int cc = 0; cc < kEpiCols; cc += kStgCols) {
#pragma unroll
      for (int j = 0; j < kStgCols; ++j) f[lane * kStgPitch + j] = acc[cc + j];
      __syncwarp();
      const int col = lane % kStgCols, sub = lane / kStgCols;
      // Y row ql; rows past the Y operand read as zeros (TMA fill), so
      // every ql < qlim may be written
      const int q = T.yb + c0 + cc + col;
      if (unit_first) {
        // units of one tile may run concurrently when K is split
#pragma unroll
        for (int i = 0; i < 32; i += kRowsPer) {
          const int p = T.ya + quad * 32 + i + sub;
          if (p < prow && q < qlim)
            atomicAdd(chi + static_cast<long long>(P0 + p) * nri + q,
                      -static_cast<double>(f[(i + sub) * kStgPitch + col] * out_scale));
        }
      } else {
        // one owner per tile: all loads in flight, then the stores
        double old[32 / kRowsPer];
#pragma unroll
        for (int i = 0; i < 32 / kRowsPer; ++i) {
          const int p = T.ya + quad * 32 + kRowsPer * i + sub;
          old[i] = (p < prow && q < qlim) ? chi[static_cast<long long>(P0 + p) * nri + q] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 32 / kRowsPer; ++i) {
          const int p = T.ya + quad * 32 + kRowsPer * i + sub;
          if (p < prow && q < qlim)
            chi[static_cast<long long>(P0 + p) * nri + q] =
                old[i] - static_cast<double>(f[(kRowsPer * i + sub) * kStgPitch + col] * out_scale);
        }
      }
      __syncwarp();
    }
  }
};

// ---------------------------------------------------------------------------
// grouped products (the batched self-energy): independent problems of their
// own sizes in one launch
// ---------------------------------------------------------------------------
struct GroupJob {
  const GroupTile* tiles;
  int n_tiles;
  double* out;
  static constexpr bool kPeriodic = true;
  static constexpr bool kTileStaging = false;
  static constexpr bool kDynamic = false;
  static constexpr int kDrainHalves = 2;

  struct Tile {
    int ya, yb, idx;
    long long ks;
  };
  __device__ Tile tile(int t) const {
    const GroupTile& g = tiles[t];
    Tile T;
    T.ya = g.a_row;
    T.yb = g.b_row;
    T.idx = t;
    T.ks = g.ksteps;
    return T;
  }
  __device__ long long nsteps(const Tile& T) const { return T.ks; }
  __device__ int items() const { return n_tiles; }
  struct Iter {
    int x;
    __device__ void init(const GroupJob*, const Tile&) { x = 0; }
    __device__ int next() {
      const int v = x;
      x += kStageK;
      return v;
    }
  };
  // out -= scale * acc through the warp's staging buffer (4 rows of 8
  // consecutive doubles per store); one owner per tile
  __device__ void write(float (&acc)[kEpiCols], const Tile& T, int quad, int lane, int c0,
                        uint8_t* stg) const {
    const GroupTile g = tiles[T.idx];
    float* f = reinterpret_cast<float*>(stg);
    constexpr int kRowsPer = 32 / kStgCols;
#pragma unroll
    for (int cc = 0; cc < kEpiCols; cc += kStgCols) {
#pragma unroll
      for (int j = 0; j < kStgCols; ++j) f[lane * kStgPitch + j] = acc[cc + j];
      __syncwarp();
      const int col = lane % kStgCols, sub = lane / kStgCols;
      const int c = c0 + cc + col;
#pragma unroll
      for (int i = 0; i < 32 / kRowsPer; ++i) {
        const int r = quad * 32 + kRowsPer * i + sub;
        if (r < g.rows && c < g.cols) {
          double* o = out + g.out_off + static_cast<long long>(r) * g.ld + c;
          *o -= static_cast<double>(f[(kRowsPer * i + sub) * kStgPitch + col] * g.scale);
        }
      }
      __syncwarp();
    }
  }
};

// ---------------------------------------------------------------------------
// steps A / B job
// ---------------------------------------------------------------------------
// Adds each lane's ss into norm2[key] (key < 0: nothing).  Lanes with equal
// keys form contiguous runs; each run is summed by a segmented suffix scan
// and its first lane issues one atomic.  Called by all 32 lanes.
__device__ __forceinline__ void flush_norm(float ss, int key, float* norm2, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float up = __shfl_down_sync(0xffffffffu, ss, o);
    const int kup = __shfl_down_sync(0xffffffffu, key, o);
    if (lane + o < 32 && kup == key) ss += up;
  }
  const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
  if (key >= 0 && (lane == 0 || kprev != key) && ss != 0.f) atomicAdd(norm2 + key, ss);
}

struct PanelJob {
  // mode 0 (X): A operand = transposed panel rows n = (pw, s'), B operand =
  //   gathered G^occ rows mu; tile entry (task, PT tile, G tile).
  // mode 1 (Y): A operand = gathered G^virt rows sigma (batch), B operand =
  //   transposed panel rows n = (pw, mu); tile entry (task, G tile, PT tile).
  // Either way a thread of the epilogue owns one A row, so its stores run
  // along the contiguous index of the K layout (s, mu, s'): s' for X, the
  // batch row sigma for Y.
  const int4* tiles;
  int n_tiles;
  const PanelTaskTC* tasks;
  int mode;
  int rows_valid;             // G rows: mode 0 n_AO, mode 1 batch AO count
  uint16_t* out;              // slices [S][slice_elems] (bf16 or binary16 bits)
  long long slice_elems, ldk;
  int P0b;
  const long long* rowbase;   // mode 1, per batch row
  const int* rowmul;
  const int* row_slocal;
  float* norm2;               // [ns][nmc][npa]: sigma-atom of the batch, mu-atom of the chunk, RI atom
  const int* atom_of_ri;
  const int* atom_of_ao;
  const int* ao_off;
  int n_at, npa, pa0, slices;
  int mu_base, m_base, nmc;   // mu chunk: first AO, first atom, atom count
  int f16;                    // slices in binary16 (else bf16)
  float unscale;              // 1 / (scale of Gg x scale of PT): true Z = acc * unscale
  float out_scale;            // scale of the Z slices
  static constexpr bool kPeriodic = false;
  static constexpr bool kTileStaging = false;
  static constexpr bool kDynamic = false;
  static constexpr int kDrainHalves = 1;

  struct Tile {
    int ya, yb, ksteps, task, mt, nt;
  };
  __device__ Tile tile(int t) const {
    const int4 e = tiles[t];
    const PanelTaskTC& tk = tasks[e.x];
    Tile T;
    T.task = e.x;
    T.mt = e.y;  // tile of the A operand's rows
    T.nt = e.z;  // tile of the B operand's rows
    if (mode == 0) {
      T.ya = tk.p_row0 + e.y * kTileM;
      T.yb = tk.g_row0 + e.z * kTileN;
    } else {
      T.ya = tk.g_row0 + e.y * kTileM;
      T.yb = tk.p_row0 + e.z * kTileN;
    }
    T.ksteps = tk.ksteps;
    return T;
  }
  __device__ long long nsteps(const Tile& T) const { return T.ksteps; }
  __device__ int items() const { return n_tiles; }
  struct Iter {
    int x;
    __device__ void init(const PanelJob*, const Tile&) { x = 0; }
    __device__ int next() {
      const int v = x;
      x += kStageK;
      return v;
    }
  };
  // The register sums go through the thread's own staging row kStgCols at a
  // time, so that the per-column loops stay rolled (small code).
  __device__ void write(float (&acc)[kEpiCols], const Tile& T, int quad, int lane, int c0,
                        uint8_t* stg) const {
    const PanelTaskTC& tk = tasks[T.task];
    const bool f = f16 != 0;
    float* fr = reinterpret_cast<float*>(stg) + lane * kStgPitch;
    if (mode == 0) {
      // row n = (pw, s') of the owner's panel; columns mu = G rows
      const int n = T.mt * kTileM + quad * 32 + lane;
      const bool n_ok = n < tk.N;
      const int pw = n_ok ? n / tk.nsig : 0;
      const int sp = n - pw * tk.nsig;
      const int patom = n_ok ? atom_of_ri[tk.p0 + pw] : 0;
      uint16_t* o = out + static_cast<long long>(tk.p0 + pw - P0b) * ldk + tk.seg + sp;
      const int mu0 = T.nt * kTileN + c0;  // chunk-local
      const int base_key = n_ok ? tk.s_local * nmc * npa + (patom - pa0) : -1;
      int m = atom_of_ao[mu_base + (mu0 < rows_valid ? mu0 : rows_valid - 1)];
      int mend = ao_off[m + 1] - mu_base;
      float ss = 0.f;
#pragma unroll
      for (int cc = 0; cc < kEpiCols; cc += kStgCols) {
#pragma unroll
        for (int j = 0; j < kStgCols; ++j) fr[j] = acc[cc + j];
#pragma unroll 1
        for (int j = 0; j < kStgCols; ++j) {
          const int mu = mu0 + cc + j;
          if (mu >= rows_valid) break;  // warp-uniform
          float v = fr[j] * unscale;
          ss += v * v;
          if (n_ok) {
            v *= out_scale;
            uint16_t* d = o + static_cast<long long>(mu) * tk.nsig;
            for (int s = 0; s < slices; ++s) d[s * slice_elems] = take_slice(v, f);
          }
          if (mu + 1 == mend || cc + j == kEpiCols - 1 || mu + 1 == rows_valid) {  // warp-uniform
            flush_norm(ss, base_key < 0 ? -1 : base_key + (m - m_base) * npa, norm2, lane);
            ss = 0.f;
            if (mu + 1 == mend && m + 1 < n_at) mend = ao_off[++m + 1] - mu_base;
          }
        }
      }
    } else {
      // row = batch AO sigma; columns n = (pw, mu') of the panel of atom tk.owner
      const int r = T.mt * kTileM + quad * 32 + lane;
      const bool r_ok = r < rows_valid;
      const long long rb = r_ok ? rowbase[r] : 0;
      const int rm = r_ok ? rowmul[r] : 0;
      const int s_local = r_ok ? row_slocal[r] : 0;
      const int n0 = T.nt * kTileN + c0;
      int pw = n0 / tk.nsig;
      int sp = n0 - pw * tk.nsig;
      int patom = atom_of_ri[tk.p0 + (pw < tk.npw ? pw : tk.npw - 1)];
      long long pwbase = static_cast<long long>(tk.p0 + pw - P0b) * ldk + rb;
      // key of (sigma-atom, mu-atom = owner, RI atom patom) is row_key + patom
      const int row_key = r_ok ? (s_local * nmc + (tk.owner - m_base)) * npa - pa0 : -1;
      float ss = 0.f;
#pragma unroll
      for (int cc = 0; cc < kEpiCols; cc += kStgCols) {
#pragma unroll
        for (int j = 0; j < kStgCols; ++j) fr[j] = acc[cc + j];
#pragma unroll 1
        for (int j = 0; j < kStgCols; ++j) {
          const int n = n0 + cc + j;
          if (n >= tk.N) break;  // warp-uniform
          float v = fr[j] * unscale;
          ss += v * v;
          if (r_ok) {
            v *= out_scale;
            uint16_t* d = out + pwbase + static_cast<long long>(tk.aom + sp) * rm;
            for (int s = 0; s < slices; ++s) d[s * slice_elems] = take_slice(v, f);
          }
          const bool last = (cc + j == kEpiCols - 1) || (n + 1 == tk.N);
          if (++sp == tk.nsig) {
            sp = 0;
            ++pw;
            pwbase += ldk;
            const int pa = (pw < tk.npw) ? atom_of_ri[tk.p0 + pw] : -1;
            if (pa != patom || last) {  // warp-uniform
              flush_norm(ss, r_ok ? row_key + patom : -1, norm2, lane);
              ss = 0.f;
              patom = pa;
            }
          } else if (last) {
            flush_norm(ss, r_ok ? row_key + patom : -1, norm2, lane);
            ss = 0.f;
          }
        }
      }
    }
  }
};

// Steps A / B with a staged epilogue (two slices only).  Tiles are aligned
// to whole output runs:
//   mode 0 (X): A operand = owner panel rows n = (pw, s'); a tile starts at a
//     pw boundary and covers rv = (128 / nsig) nsig rows or the panel's rest,
//     B operand = 128 G^occ rows mu (chunk-local).  For each of its pw the
//     tile is the contiguous run X[P0 + pw][seg + mu0 nsig, + ncol nsig).
//   mode 1 (Y): A operand = batch rows sigma, a group of whole owner atoms
//     (<= 128 rows); B operand = panel rows n = (pw, mu') of atom tk.owner, a
//     tile starting at a pw boundary with (128 / n_ao) n_ao rows or the rest.
//     For each (owner s, pw) the tile is the contiguous run
//     Y[pw - Q0][seg(s) + aom n(s), + n(owner) n(s)].
// The 16 epilogue warps turn their accumulators into the two 16-bit slices
// and store them in shared memory in the order of the output runs; on the
// way they add the squared Frobenius norms of the tile's atom blocks into
// norm2, one atomic per rectangle and group of rows (mu-atom x RI atom in
// mode 0, owner x pw's RI atom in mode 1).  The runs then leave shared
// memory:
//   mode 0 (runs of 64 or 128 nsig elements): one epilogue warp issues one
//     bulk copy per (run, slice) and returns to the accumulators; it waits
//     for the copies' reads before the next tile is staged;
//   mode 1 (runs of n(owner) n(s) elements, many per tile): the 16 warps copy
//     the runs themselves, the 8-aligned body of each in 16-byte vectors and
//     the few elements before and after it one by one.
// A run starts in shared memory at the same offset modulo 8 elements as in
// global memory, so that its body moves in aligned vectors:
//   mode 0: run g at g (128 nsig + kRunSkew) (every X run is 8-aligned);
//   mode 1: sigma-atom a of the tile owns a region at U_a + d_a, d_a = the
//     global offset of its runs modulo 8, U_a = sum over the tile's earlier
//     atoms b of round8(d_b + ng round8(n(owner) n(b))); run (a, g) at
//     U_a + d_a + g round8(n(owner) n(a)).
// The host checks that a tile fits in kPlaneElems (mode 1) and that the row
// stride and the slice offset of the output are multiples of 8 elements.
constexpr int kRunSkew = 16;  // mode 0 run pitch 128 nsig + 16: conflict-free staging stores

__host__ __device__ constexpr int round8(int x) { return (x + 7) & ~7; }

struct PanelStagedJob {
  const int4* tiles;          // (task, A row offset, B row offset, rows_valid << 16 | cols_valid)
  int n_tiles;
  const PanelTaskTC* tasks;
  int mode;
  uint16_t* out;              // slices [2][slice_elems]
  long long slice_elems, ldk;
  int P0b;                    // first RI function of the output rows
  int Lc;                     // mode 0: chunk segment length (X columns per s' run)
  int row_ao0;                // mode 1: global AO of batch row 0
  int s0b;                    // mode 1: first owner atom of the batch
  const long long* rowbase;   // mode 1, per batch row: seg(s) + sigma'
  float* norm2;               // [ns][nmc][npa]
  const int* atom_of_ri;
  const int* atom_of_ao;
  const int* ao_off;
  const int* ri_off;
  const int* n_ao;
  int npa, pa0, mu_base, m_base, nmc;
  int f16;
  float unscale, out_scale;
  static constexpr bool kPeriodic = false;
  static constexpr bool kTileStaging = true;
  static constexpr bool kDynamic = false;
  static constexpr int kDrainHalves = 1;
  // arrivals that free the staging area: the issuing warp (mode 0) or every
  // epilogue warp (mode 1)
  __device__ int freed_count() const { return mode == 0 ? 1 : kEpiWarps; }

  struct Tile {
    int ya, yb, ksteps, task, ra, rb, rv, cv;
  };
  __device__ Tile tile(int t) const {
    const int4 e = tiles[t];
    const PanelTaskTC& tk = tasks[e.x];
    Tile T;
    T.task = e.x;
    T.ra = e.y;
    T.rb = e.z;
    T.rv = e.w >> 16;
    T.cv = e.w & 0xffff;
    if (mode == 0) {
      T.ya = tk.p_row0 + e.y;
      T.yb = tk.g_row0 + e.z;
    } else {
      T.ya = tk.g_row0 + e.y;
      T.yb = tk.p_row0 + e.z;
    }
    T.ksteps = tk.ksteps;
    return T;
  }
  __device__ long long nsteps(const Tile& T) const { return T.ksteps; }
  __device__ int items() const { return n_tiles; }
  struct Iter {
    int x;
    __device__ void init(const PanelStagedJob*, const Tile&) { x = 0; }
    __device__ int next() {
      const int v = x;
      x += kStageK;
      return v;
    }
  };

  __device__ static void pack_slices(float v, bool f, uint16_t& h0, uint16_t& h1) {
    h0 = take_slice(v, f);
    h1 = take_slice(v, f);
  }
  // Mode 1: global offset (row pw run 0) of the runs of sigma-atom a (task
  // with RI base p0 and chunk-local owner AO offset aom).
  __device__ long long run_dst(int p0, int aom, int pw0, int a) const {
    return static_cast<long long>(p0 + pw0 - P0b) * ldk + rowbase[ao_off[a] - row_ao0] +
           static_cast<long long>(aom) * n_ao[a];
  }
  // Mode 1: shared-memory extent of sigma-atom a's region (ng runs).
  __device__ int region_len(int p0, int aom, int pw0, int ng, int nm, int a) const {
    const int d = static_cast<int>(run_dst(p0, aom, pw0, a) & 7);
    return round8(d + ng * round8(nm * n_ao[a]));
  }

  // Adds ss of every lane into the rectangle (row group key rk, column key
  // ck >= 0); lanes with equal rk are contiguous.  uni: every row key of the
  // warp is rk of lane 0 or -1.  Called by all 32 lanes.
  __device__ __forceinline__ void add_norm(float ss, int rk, int ck, bool uni, int lane, int s_local,
                                           int owner) const {
    auto index = [&](int r) {
      return mode == 0 ? (s_local * nmc + (ck - m_base)) * npa + (r - pa0)
                       : ((r - s0b) * nmc + (owner - m_base)) * npa + (ck - pa0);
    };
    if (uni) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const int r0 = __shfl_sync(0xffffffffu, rk, 0);
      if (lane == 0 && r0 >= 0 && ss != 0.f) atomicAdd(norm2 + index(r0), ss);
    } else {
      flush_norm(ss, rk >= 0 ? index(rk) : -1, norm2, lane);
    }
  }

  // Mode 1: run geometry of sigma-atom a in a tile of ng runs starting at pw
  // run pw0: global offset of run 0 (d0), padded run pitch in shared memory
  // (preg), head / 8-element vectors / tail of a run (h, nb, t) and the
  // region length in shared memory (reg).
  struct Geom {
    long long d0;
    int preg, h, nb, t, reg;
  };
  __device__ Geom geom(int p0, int aom, int pw0, int ng, int nm, int a) const {
    Geom G;
    const int len = nm * n_ao[a];
    G.preg = round8(len);
    G.d0 = run_dst(p0, aom, pw0, a);
    const int d = static_cast<int>(G.d0 & 7);
    G.h = min((8 - d) & 7, len);
    G.nb = (len - G.h) >> 3;
    G.t = len - G.h - 8 * G.nb;
    G.reg = round8(d + ng * G.preg);
    return G;
  }

  // Epilogue warps, end of a tile: wait until the staging area is free,
  // stage this warp's 32 rows x 32 columns as slices, add the block norms,
  // and copy the tile out (see above).
  __device__ bool stage(float (&acc)[kEpiCols], const Tile& T, int quad, int lane, int c0,
                        EpiCtx& ep) const {
    uint16_t* pl0 = reinterpret_cast<uint16_t*>(ep.staging);
    uint16_t* pl1 = pl0 + kPlaneElems;
    uint16_t* o1 = out + slice_elems;
    // the task's fields in registers before the first store or atomic (which
    // the compiler cannot prove not to alias them)
    const PanelTaskTC& tk = tasks[T.task];
    const int t_nsig = tk.nsig, t_p0 = tk.p0, t_sl = tk.s_local, t_owner = tk.owner, t_aom = tk.aom;
    const long long t_seg = tk.seg;
    const bool f = f16 != 0;
    const int r = quad * 32 + lane;  // this thread's tile row
    const bool valid = r < T.rv;
    int rk = -1;       // row group key: RI atom (mode 0) or sigma-atom (mode 1)
    int ckl = -1;      // column key of column c0 + lane: mu-atom (mode 0) or RI atom (mode 1)
    int pos = 0;       // staging position of column c0
    int step = 0;      // mode 0: position step per column
    int nm = 0, mu = 0, nsg = 0, gap = 0;  // mode 1 walk over (pw run, mu')
    int ncol;          // columns that exist in the output
    int sf = 0, sl = -1, ng = 0, pw0 = 0;
    Geom G{0, 0, 0, 0, 0, 0};  // mode 1: lane i holds atom sf + i (first 32 atoms)
    int g_U = 0;               // ... and its region's start
    if (mode == 0) {
      const int nsig = t_nsig;
      const int gr = r / nsig, sp = r - gr * nsig;
      pw0 = T.ra / nsig;
      ng = T.rv / nsig;
      ncol = min(kTileN, Lc - T.rb);
      if (valid) rk = atom_of_ri[t_p0 + pw0 + gr];
      if (c0 + lane < T.cv) ckl = atom_of_ao[mu_base + T.rb + c0 + lane];
      step = nsig;
      pos = gr * (kTileN * nsig + kRunSkew) + c0 * nsig + sp;
    } else {
      nm = t_nsig;  // the owner's function count
      ng = T.cv / nm;
      pw0 = T.rb / nm;
      ncol = T.cv;
      sf = atom_of_ao[row_ao0 + T.ra];
      sl = atom_of_ao[row_ao0 + T.ra + T.rv - 1];
      int s = sf, sp = 0;
      if (valid) {
        const int a = row_ao0 + T.ra + r;
        s = atom_of_ao[a];
        sp = a - ao_off[s];
        nsg = n_ao[s];
        rk = s;
      }
      if (sf + lane <= sl) G = geom(t_p0, t_aom, pw0, ng, nm, sf + lane);
      int inc = sf + lane <= sl ? G.reg : 0;
      const int mine = inc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      g_U = inc - mine;
      // U_s of this row's atom: from its lane, or summed when the tile has
      // more than 32 atoms and s is past the first 32
      int U = __shfl_sync(0xffffffffu, g_U, valid && s - sf <= 31 ? s - sf : 0);
      if (valid && s - sf > 31) {
        U = 0;
        for (int b = sf; b < s; ++b) U += geom(t_p0, t_aom, pw0, ng, nm, b).reg;
      }
      if (valid) {
        const int d = static_cast<int>(run_dst(t_p0, t_aom, pw0, s) & 7);
        const int preg = round8(nm * nsg);
        gap = preg - nm * nsg;
        const int g = c0 / nm;
        mu = c0 - g * nm;
        pos = U + d + g * preg + mu * nsg + sp;
      }
      if (c0 + lane < T.cv) ckl = atom_of_ri[t_p0 + pw0 + (c0 + lane) / nm];
    }
    // the staging area is free: mode 0, the issuing warp's copies of the
    // previous tile have read it; mode 1, every warp has copied its runs
    if (ep.tile_no > 0) {
      if (mode == 0 && ep.warp == 0) {
        bulk_wait_read();
        __syncwarp();
        if (lane == 0) mbar_arrive(ep.freed);
      }
      if (!mbar_wait(ep.freed, static_cast<uint32_t>(ep.tile_no - 1) & 1u, ep.abort)) return false;
    }
    // row keys uniform across the warp's valid rows?
    const int rk0 = __shfl_sync(0xffffffffu, rk, 0);
    const bool uni = __all_sync(0xffffffffu, rk == rk0 || rk < 0);
    // bit j: column j starts a new column key (warp-uniform)
    const int ck_up = __shfl_up_sync(0xffffffffu, ckl, 1);
    const unsigned kmask = __ballot_sync(0xffffffffu, lane == 0 || ckl != ck_up);
    float ss = 0.f;
#pragma unroll
    for (int j = 0; j < kEpiCols; ++j) {
      const float v = acc[j] * unscale;
      if (valid && c0 + j < ncol) {
        uint16_t h0, h1;
        pack_slices(v * out_scale, f, h0, h1);
        pl0[pos] = h0;
        pl1[pos] = h1;
        ss += v * v;
      }
      if (mode == 0) {
        pos += step;
      } else {
        pos += nsg;
        if (++mu == nm) {  // next pw run of the owner: the next padded slot
          mu = 0;
          pos += gap;
        }
      }
      // the column key changes after column j: flush the segment
      if (j == kEpiCols - 1 || ((kmask >> (j + 1)) & 1u)) {
        const int ck = __shfl_sync(0xffffffffu, ckl, j);
        if (ck >= 0) add_norm(ss, rk, ck, uni, lane, t_sl, t_owner);
        ss = 0.f;
      }
    }
    if (mode == 0) {
      // the bulk copies read the staged slices through the async proxy
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(ep.staged);
      if (ep.warp != 0) return true;
      if (!mbar_wait(ep.staged, static_cast<uint32_t>(ep.tile_no) & 1u, ep.abort)) return false;
      const int nsig = t_nsig;
      const int pitch = kTileN * nsig + kRunSkew;
      const long long d0 = static_cast<long long>(t_p0 + pw0 - P0b) * ldk + t_seg +
                           static_cast<long long>(T.rb) * nsig;
      // X runs are 8-aligned by construction (segments of multiples of 64
      // columns); refuse rather than issue a misaligned copy
      if (((d0 | ldk | slice_elems) & 7) != 0 || ((ncol * nsig) & 7) != 0) return false;
      const uint32_t bytes = static_cast<uint32_t>(ncol * nsig) * 2u;
      bool issued = false;
      for (int u = lane; u < 2 * ng; u += 32) {  // (run, slice) pairs
        const int gr = u >> 1;
        const long long dst = d0 + gr * ldk;
        if (u & 1)
          bulk_store(o1 + dst, pl1 + gr * pitch, bytes);
        else
          bulk_store(out + dst, pl0 + gr * pitch, bytes);
        issued = true;
      }
      if (issued) bulk_commit();
      return true;
    }
    // mode 1: every warp copies runs (atom i of the group, run g), warps
    // striding over them
    __syncwarp();
    if (lane == 0) mbar_arrive(ep.staged);
    if (!mbar_wait(ep.staged, static_cast<uint32_t>(ep.tile_no) & 1u, ep.abort)) return false;
    int U0 = 0;  // first region of the current group of 32 atoms
    for (int base = sf; base <= sl; base += 32) {
      if (base > sf) {
        G = Geom{0, 0, 0, 0, 0, 0};
        if (base + lane <= sl) G = geom(t_p0, t_aom, pw0, ng, nm, base + lane);
        int inc = base + lane <= sl ? G.reg : 0;
        const int mine = inc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        g_U = inc - mine;
      }
      const int cnt = min(32, sl - base + 1);
      for (int k = ep.warp; k < cnt * ng; k += kEpiWarps) {
        const int i = k / ng, g = k - i * ng;
        const long long d0 = __shfl_sync(0xffffffffu, G.d0, i);
        const int preg = __shfl_sync(0xffffffffu, G.preg, i);
        const int h = __shfl_sync(0xffffffffu, G.h, i);
        const int nb = __shfl_sync(0xffffffffu, G.nb, i);
        const int t = __shfl_sync(0xffffffffu, G.t, i);
        const int R = U0 + __shfl_sync(0xffffffffu, g_U, i) + static_cast<int>(d0 & 7);
        const long long dst = d0 + g * ldk;
        const int src = R + g * preg;
        // lane l: head element l < h, vector l - h < nb, tail element after
        for (int l = lane; l < h + nb + t; l += 32) {
          if (l < h) {
            out[dst + l] = pl0[src + l];
            o1[dst + l] = pl1[src + l];
          } else if (l < h + nb) {
            const int e = h + 8 * (l - h);
            const uint4 x = *reinterpret_cast<const uint4*>(pl0 + src + e);
            const uint4 y = *reinterpret_cast<const uint4*>(pl1 + src + e);
            *reinterpret_cast<uint4*>(out + dst + e) = x;
            *reinterpret_cast<uint4*>(o1 + dst + e) = y;
          } else {
            const int e = h + 8 * nb + (l - h - nb);
            out[dst + e] = pl0[src + e];
            o1[dst + e] = pl1[src + e];
          }
        }
      }
      // the group's total region length
      int tot = base + lane <= sl ? G.reg : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
      U0 += tot;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(ep.freed);
    return true;
  }

  // After the last tile: the issuing warp's bulk copies have completed.
  __device__ void finish(const EpiCtx& ep) const {
    if (mode == 0 && ep.warp == 0) bulk_wait_all();
  }
};

// ---------------------------------------------------------------------------
// work distribution
// ---------------------------------------------------------------------------
constexpr int kSchedSlots = 4;
// The work items of one role of a CTA: blockIdx.x, + gridDim.x, ... (static),
// or, for a job that hands items out from an atomic counter, whatever item
// the producer thread takes next: it passes each to the MMA issuer and the
// epilogue warps through a ring of shared-memory slots, so that the CTAs
// together work through the items in order (and the operand slabs of the
// items in flight stay few).  -1 ends the sequence.
struct Sched {
  volatile int* slot;  // [kSchedSlots]
  uint64_t* full;      // [kSchedSlots] item written by the producer
  uint64_t* empty;     // [kSchedSlots] item read by the MMA issuer and every epilogue warp
  int* counter;        // null: static
  int n;
  volatile int* abort;
  int s;
  uint32_t ph;
  int t;               // static: the next item
  int ahead;           // dynamic: the producer's next item, taken one item early (-2: none yet)
  __device__ int next_static() {
    const int v = t;
    t += gridDim.x;
    return v < n ? v : -1;
  }
  __device__ void advance() {
    if (++s == kSchedSlots) {
      s = 0;
      ph ^= 1u;
    }
  }
  // producer (one thread)
  __device__ int produce(bool& ok) {
    if (!counter) return next_static();
    if (!mbar_wait(&empty[s], ph ^ 1u, abort)) {
      ok = false;
      return -1;
    }
    // the counter's next value is fetched while this item runs; the counter
    // only grows, so the value left unused after the last item is past n
    int v = ahead >= -1 ? ahead : atomicAdd(counter, 1);
    if (v >= n) v = -1;
    ahead = v >= 0 ? atomicAdd(counter, 1) : -1;
    slot[s] = v;
    mbar_arrive(&full[s]);
    advance();
    return v;
  }
  // the MMA issuer (one thread)
  __device__ int consume_one(bool& ok) {
    if (!counter) return next_static();
    if (!mbar_wait(&full[s], ph, abort)) {
      ok = false;
      return -1;
    }
    const int v = slot[s];
    mbar_arrive(&empty[s]);
    advance();
    return v;
  }
  // an epilogue warp (all 32 lanes)
  __device__ int consume_warp(int lane, bool& ok) {
    if (!counter) return next_static();
    if (!mbar_wait(&full[s], ph, abort)) {
      ok = false;
      return -1;
    }
    const int v = slot[s];
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    advance();
    return v;
  }
};
template <class Job>
__device__ int* work_counter(const Job& j) {
  if constexpr (Job::kDynamic)
    return j.work;
  else
    return nullptr;
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <int S, class Job, bool F16>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_persistent(const __grid_constant__ CUtensorMap map_a,
                    const __grid_constant__ CUtensorMap map_b, const Job job, Cadence cad,
                    int* __restrict__ err_flag) {
  using L = Smem<S, Job>;
  constexpr int kStages = L::kStages;
  constexpr int kSub = kStageK / kMmaK;  // MMA steps per K step
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* operands = smem;
  uint8_t* staging = smem + L::kOperandBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOperandBytes + L::kStagingBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* acc_full = bars + 2 * kStages;  // [kAccBufs] accumulator buffers
  uint64_t* acc_empty = acc_full + kAccBufs;
  uint64_t* drain = acc_empty + kAccBufs;
  uint64_t* never = drain + 1;  // arrived at by nothing (stall test hook)
  uint64_t* tile_staged = never + 1;  // tile-staging jobs: every epilogue warp staged its part
  uint64_t* tile_freed = tile_staged + 1;  // ... and finished writing the tile out
  uint64_t* sched_full = tile_freed + 1;           // [kSchedSlots]
  uint64_t* sched_empty = sched_full + kSchedSlots;  // [kSchedSlots]
  int* sched_slot = reinterpret_cast<int*>(sched_empty + kSchedSlots);  // [kSchedSlots]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sched_slot + kSchedSlots);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    mbar_init(never, 1);
    mbar_init(tile_staged, kEpiWarps);
    int freed_arrivals = 1;
    if constexpr (Job::kTileStaging) freed_arrivals = job.freed_count();
    mbar_init(tile_freed, static_cast<uint32_t>(freed_arrivals));
    for (int k = 0; k < kSchedSlots; ++k) {
      mbar_init(&sched_full[k], 1);
      mbar_init(&sched_empty[k], 1 + kEpiWarps);
    }
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
  const int n_items = job.items();  // work items (tiles or units) of the launch
  Sched sch{sched_slot, sched_full, sched_empty, work_counter(job), n_items, abort_flag, 0, 0,
            static_cast<int>(blockIdx.x), -2};

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed_parity[kStages];
      bool armed[kStages];
      for (int s = 0; s < kStages; ++s) armed[s] = false, armed_parity[s] = 0;
      bool ok = true;
      for (int t = sch.produce(ok); t >= 0 && ok; t = sch.produce(ok)) {
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
          if (armed[s]) mbar_wait_cleanup(&full[s], armed_parity[s]);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    // Each drain interval (cad.main MMA steps, or the tile's rest) goes to
    // the next accumulator buffer; within the part of an interval that lies
    // in one K step, the small slice products come first, then the main
    // product (0, 0).
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f32(kTileM, kTileN, F16);
      // slice tiles are kTileBytes apart: descriptor start addresses
      // advance by kTileBytes >> 4
      constexpr uint64_t kStep = static_cast<uint64_t>(L::kTileBytes >> 4);
      int stage = 0;
      uint32_t phase = 0;
      int chunk = 0;
      bool ok = true, issued_any = false;
      for (int t = sch.consume_one(ok); t >= 0 && ok; t = sch.consume_one(ok)) {
        const typename Job::Tile T = job.tile(t);
        const long long n = job.nsteps(T);
        const long long nsub = n * kSub;
        long long js = 0;
        int sub = 0;  // MMA steps into the drain interval
        for (long long i = 0; i < n && ok; ++i) {
          if (!mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(operands + stage * L::kStageBytes);
          const uint64_t da = desc_sw128(st), db = desc_sw128(st + S * L::kTileBytes);
          int k = 0;
          while (k < kSub) {
            const int mb = chunk % kAccBufs;
            if (sub == 0) {
              ok = mbar_wait(&acc_empty[mb], ((static_cast<uint32_t>(chunk / kAccBufs)) & 1u) ^ 1u,
                             abort_flag);
              tc_fence_after();
              if (!ok) break;
            }
            // MMA steps [k, ke) of this K step belong to the current interval
            const int ke = min(kSub, k + (cad.main - sub));
            const uint32_t d = tmem + static_cast<uint32_t>(mb * 128);
            uint32_t accf = sub == 0 ? 0u : 1u;
            for (int kk = k; kk < ke; ++kk) {
              const uint64_t koff = static_cast<uint64_t>((kk * kMmaK * 2) >> 4);
#pragma unroll
              for (int a = 0; a < S; ++a) {
#pragma unroll
                for (int b = 0; b < S - a; ++b) {
                  if (a == 0 && b == 0) continue;
                  mma_bf16(d, da + a * kStep + koff, db + b * kStep + koff, idesc, accf);
                  accf = 1u;
                }
              }
            }
            for (int kk = k; kk < ke; ++kk) {
              const uint64_t koff = static_cast<uint64_t>((kk * kMmaK * 2) >> 4);
              mma_bf16(d, da + koff, db + koff, idesc, accf);
              accf = 1u;
            }
            issued_any = true;
            js += ke - k;
            sub += ke - k;
            k = ke;
            if (sub == cad.main || js == nsub) {
              mma_commit(&acc_full[mb]);
              ++chunk;
              sub = 0;
            }
          }
          if (!ok) break;
          mma_commit(&empty[stage]);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(err_flag, 2);
        if (issued_any) {
          mma_commit(drain);
          mbar_wait_cleanup(drain, 0);
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2..17) ----------------
    const int quad = warp & 3;
    const int cgroup = (warp - 2) >> 2;  // warps 2..17: 4 per column group, one per lane quadrant
    const int c0 = cgroup * kEpiCols;
    uint8_t* stg = staging + (warp - 2) * kStgBytes;
    const uint32_t row_addr = tmem + (static_cast<uint32_t>(quad * 32) << 16) + static_cast<uint32_t>(c0);
    float acc[kEpiCols];
    int chunk = 0;
    EpiCtx ep{staging, tile_staged, tile_freed, abort_flag, warp - 2, 0};
    (void)ep;
    // test hook: a dependency that is never satisfied; the bounded wait
    // gives up and the kernel reports a time-out instead of hanging
    bool ok = cad.stall ? mbar_wait(never, 0, abort_flag) : true;
    for (int t = ok ? sch.consume_warp(lane, ok) : -1; t >= 0 && ok; t = sch.consume_warp(lane, ok)) {
      const typename Job::Tile T = job.tile(t);
      const long long n = job.nsteps(T);
      const long long nch = (n * kSub + cad.main - 1) / cad.main;
#pragma unroll
      for (int j = 0; j < kEpiCols; ++j) acc[j] = 0.f;
      for (long long c = 0; c < nch; ++c, ++chunk) {
        const int mb = chunk % kAccBufs;
        if (!mbar_wait(&acc_full[mb], static_cast<uint32_t>(chunk / kAccBufs) & 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        tmem_add32<Job::kDrainHalves>(row_addr + static_cast<uint32_t>(mb * 128), acc);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[mb]);
        if constexpr (Job::kPeriodic) {
          if ((c + 1) % cad.write_every == 0 && c + 1 < nch) {
            job.write(acc, T, quad, lane, c0, stg);
#pragma unroll
            for (int j = 0; j < kEpiCols; ++j) acc[j] = 0.f;
          }
        }
      }
      if (!ok) break;
      if (nch > 0) {
        if constexpr (Job::kTileStaging) {
          ok = job.stage(acc, T, quad, lane, c0, ep);
          ++ep.tile_no;
          if (!ok) break;
        } else {
          job.write(acc, T, quad, lane, c0, stg);
        }
      }
    }
    // bulk copies still in flight complete before the CTA exits
    if constexpr (Job::kTileStaging) job.finish(ep);
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
                           int kmax, int slices, long long slice_elems, int f16, double scale,
                           uint16_t* __restrict__ out) {
  const PanelTaskTC tk = tasks[blockIdx.y];
  const long long n = static_cast<long long>(rows_per_task) * kmax;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / kmax), k = static_cast<int>(i % kmax);
    double v = 0.0;
    if (r < rows_valid && k < tk.K)
      v = scale * g[static_cast<long long>(rbase + r) * nao + lam[tk.lam_off + k]];
    const long long dst = static_cast<long long>(tk.g_row0 + r) * kmax + k;
    for (int s = 0; s < slices; ++s) out[s * slice_elems + dst] = take_slice(v, f16 != 0);
  }
}

// Split, transposed owner panels straight from the stored 3c blocks.  The
// panel of owner atom s is PT[slice][p_row0(s) + pw * n_ao(s) + s'][k] =
// slice of scale * T[lambda_k, sigma = s', P = p0(s) + pw] (k over the
// functions of the atoms sharing a kept block with s).  Kept block (A, B, P)
// [lambda' in A][sigma' in B][P'] lands in
//   panel B: row rowB + P' n(B) + sigma', column kB + lambda'
//   panel A (A != B): row rowA + P' n(A) + lambda', column kA + sigma'
// (T symmetric in its primary indices).  Consecutive threads take
// consecutive columns of a row.  One CTA per kept block, striding; the
// buffer is zeroed beforehand (padding and blocks not stored).
template <typename T>
__global__ void k_pt_scatter(const T* __restrict__ t3, const int* __restrict__ blk,
                             const long long* __restrict__ off, const int* __restrict__ n_ao,
                             const int* __restrict__ n_ri, const int* __restrict__ kept,
                             long long n_kept, const long long* __restrict__ rowB,
                             const int* __restrict__ kB, const long long* __restrict__ rowA,
                             const int* __restrict__ kA, int kmax, int slices, long long slice_elems,
                             int f16, double scale, uint16_t* __restrict__ out) {
  for (long long kb = blockIdx.x; kb < n_kept; kb += gridDim.x) {
    const int b = kept[kb];
    const int A = blk[3 * b], B = blk[3 * b + 1], p = blk[3 * b + 2];
    const int na = n_ao[A], nb = n_ao[B], np = n_ri[p];
    const T* x = t3 + off[b];
    const long long n = static_cast<long long>(na) * nb * np;
    // panel B: i = (P' nb + sigma') na + lambda' (a row below 0: the side is
    // not built in this call)
    for (long long i = threadIdx.x; rowB[kb] >= 0 && i < n; i += blockDim.x) {
      const int al = static_cast<int>(i % na);
      const long long r = i / na;  // P' nb + sigma'
      const int be = static_cast<int>(r % nb), pl = static_cast<int>(r / nb);
      double v = scale * static_cast<double>(x[(static_cast<long long>(al) * nb + be) * np + pl]);
      const long long dst = (rowB[kb] + r) * kmax + kB[kb] + al;
      for (int s = 0; s < slices; ++s) out[s * slice_elems + dst] = take_slice(v, f16 != 0);
    }
    if (A == B || rowA[kb] < 0) continue;
    // panel A: i = (P' na + lambda') nb + sigma'
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      const int be = static_cast<int>(i % nb);
      const long long r = i / nb;  // P' na + lambda'
      const int al = static_cast<int>(r % na), pl = static_cast<int>(r / na);
      double v = scale * static_cast<double>(x[(static_cast<long long>(al) * nb + be) * np + pl]);
      const long long dst = (rowA[kb] + r) * kmax + kA[kb] + be;
      for (int s = 0; s < slices; ++s) out[s * slice_elems + dst] = take_slice(v, f16 != 0);
    }
  }
}

// Norms of the atom blocks of an operand from the accumulated squares, one
// thread per block (sigma-atom, mu-atom, RI atom): flag the kept nonzero
// blocks and the (slab, tile) pairs they touch; queue the filtered nonzero
// ones (norm < thr) for zeroing.
__global__ void k_slices_block_flags(const int* __restrict__ ri_off, int rowoff, int pa0, int npa,
                                     int nmc, int ns, double thr, const float* __restrict__ norm2,
                                     unsigned char* __restrict__ blockflag,
                                     unsigned char* __restrict__ tileflag, int ntile, int tile_rows,
                                     int* __restrict__ zlist, int* __restrict__ zcount) {
  const long long nblk = static_cast<long long>(ns) * nmc * npa;
  for (long long w = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; w < nblk;
       w += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int pl = static_cast<int>(w % npa);
    const long long t = w / npa;  // sl * nmc + (m - m0)
    const double nrm = sqrt(static_cast<double>(norm2[w]));
    const bool kept = !(nrm < thr);
    const bool nz = kept && nrm > 0.0;
    blockflag[w] = nz;
    if (!kept && nrm > 0.0) zlist[atomicAdd(zcount, 1)] = static_cast<int>(w);
    if (nz) {
      const int p = pa0 + pl;
      const int rows0 = ri_off[p] - rowoff, nrows = ri_off[p + 1] - ri_off[p];
      const int ts = rows0 / tile_rows, te = (rows0 + nrows - 1) / tile_rows;
      for (int tt = ts; tt <= te; ++tt) tileflag[t * ntile + tt] = 1;
    }
  }
}

// Zero, in every slice, the blocks queued by k_slices_block_flags: one warp
// per queued block, the warps striding over the queue.  Each row of a block
// is one contiguous run: its 8-aligned body in 16-byte stores, the elements
// before and after one by one (slice_elems and ldk are multiples of 8 when
// vec is set).
__global__ void k_slices_zero_blocks(uint16_t* __restrict__ Z, int slices, long long slice_elems,
                                     long long ldk, int rowoff, const int* __restrict__ ri_off,
                                     const int* __restrict__ ao_off, const int* __restrict__ n_ao,
                                     int s0, const long long* __restrict__ seg, int pa0, int npa,
                                     int m0, int nmc, int mu0, const int* __restrict__ zlist,
                                     const int* __restrict__ zcount, int vec) {
  const int lane = threadIdx.x & 31;
  const int nq = *zcount;
  const int nwarps = gridDim.x * (blockDim.x / 32);
  for (int q = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; q < nq; q += nwarps) {
    const long long w = zlist[q];
    const int pl = static_cast<int>(w % npa);
    const long long t = w / npa;
    const int m = m0 + static_cast<int>(t % nmc);
    const int sl = static_cast<int>(t / nmc);
    const int nsig = n_ao[s0 + sl];
    const int p = pa0 + pl;
    const int rows0 = ri_off[p] - rowoff, nrows = ri_off[p + 1] - ri_off[p];
    const long long c0 = seg[sl] + static_cast<long long>(ao_off[m] - mu0) * nsig;
    const int ncols = n_ao[m] * nsig;
    if (vec) {
      for (int r = 0; r < nrows; ++r) {
        const long long row = static_cast<long long>(rows0 + r) * ldk + c0;
        const int h = min(static_cast<int>((8 - (row & 7)) & 7), ncols);
        const int nb = (ncols - h) >> 3, t = ncols - h - 8 * nb;
        for (int l = lane; l < h + nb + t; l += 32) {
          for (int sc = 0; sc < slices; ++sc) {
            uint16_t* z = Z + sc * slice_elems + row;
            if (l < h)
              z[l] = 0;  // +0 in both formats
            else if (l < h + nb)
              *reinterpret_cast<uint4*>(z + h + 8 * (l - h)) = make_uint4(0, 0, 0, 0);
            else
              z[h + 8 * nb + (l - h - nb)] = 0;
          }
        }
      }
    } else {
      for (int r = 0; r < nrows; ++r)
        for (int c = lane; c < ncols; c += 32)
          for (int sc = 0; sc < slices; ++sc)
            Z[sc * slice_elems + static_cast<long long>(rows0 + r) * ldk + c0 + c] = 0;
    }
  }
}

// Zero n 16-bit elements from p with the whole CTA (16-byte stores in the
// aligned body).
__device__ __forceinline__ void zero_run(uint16_t* p, long long n) {
  long long head = (8 - static_cast<long long>((reinterpret_cast<uintptr_t>(p) >> 1) & 7)) & 7;
  if (head > n) head = n;
  for (long long i = threadIdx.x; i < head; i += blockDim.x) p[i] = 0;
  uint4* q = reinterpret_cast<uint4*>(p + head);
  const long long nv = (n - head) >> 3;
  for (long long i = threadIdx.x; i < nv; i += blockDim.x) q[i] = make_uint4(0, 0, 0, 0);
  for (long long i = head + nv * 8 + threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

// The part of Y that step B does not write: for row Q and batch atom s, the
// mu outside the atoms [lo[Q], hi[Q]] whose panel windows cover Q (all of
// the segment when lo[Q] < 0), which includes the padding mu >= n_AO.  One
// CTA per (Q, s) pair, striding.
__global__ void k_zero_unwritten_y(uint16_t* __restrict__ Y, int slices, long long slice_elems,
                                   long long ldk, int Q0, int qrow, int ns,
                                   const long long* __restrict__ seg, const int* __restrict__ n_ao,
                                   int s0, const int* __restrict__ ao_off, int m0, int m1, int Lc,
                                   const int* __restrict__ lo, const int* __restrict__ hi) {
  const long long npair = static_cast<long long>(qrow) * ns;
  const int mu0 = ao_off[m0];
  for (long long w = blockIdx.x; w < npair; w += gridDim.x) {
    const int ql = static_cast<int>(w / ns), sl = static_cast<int>(w % ns);
    const int q = Q0 + ql;
    const int nsig = n_ao[s0 + sl];
    const long long L = static_cast<long long>(Lc) * nsig;
    // covering owners inside the chunk [m0, m1)
    const int a0 = lo[q] < 0 ? m1 : max(lo[q], m0);
    const int a1 = lo[q] < 0 ? m0 - 1 : min(hi[q], m1 - 1);
    const long long a = a0 > a1 ? L : static_cast<long long>(ao_off[a0] - mu0) * nsig;
    const long long b = a0 > a1 ? L : static_cast<long long>(ao_off[a1 + 1] - mu0) * nsig;
    for (int sc = 0; sc < slices; ++sc) {
      uint16_t* base = Y + sc * slice_elems + static_cast<long long>(ql) * ldk + seg[sl];
      zero_run(base, a);
      zero_run(base + b, L - b);
    }
  }
}

// Zero the Y runs of the step-B pairs left out (see DeadY): one CTA per
// pair in turn, one warp per row.
__global__ void k_zero_dead_y(uint16_t* __restrict__ Y, int slices, long long slice_elems, long long ldk,
                              int qrow, const DeadY* __restrict__ pairs, int n_pairs,
                              const long long* __restrict__ seg, const int* __restrict__ n_ao, int s0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
    const DeadY e = pairs[p];
    for (int q = warp; q < e.nq; q += nw) {
      const int row = e.q0 + q;
      if (row < 0 || row >= qrow) continue;
      for (int a = e.a0; a < e.a1; ++a) {
        const int na = n_ao[s0 + a];
        const long long base = static_cast<long long>(row) * ldk + seg[a] + static_cast<long long>(e.aom) * na;
        const int len = e.nm * na;
        for (int i = lane; i < len; i += 32)
          for (int sc = 0; sc < slices; ++sc) Y[sc * slice_elems + base + i] = 0;
      }
    }
  }
}

// FP64 [rows][cols] (row stride ld), times scale -> 16-bit slices
// [S][rows][kpad], zero for k >= cols
__global__ void k_split_f64(const double* __restrict__ a, long long ld, int rows, int cols, int kpad,
                            int slices, int f16, double scale, uint16_t* __restrict__ out) {
  const long long n = static_cast<long long>(rows) * kpad;
  const long long slice = n;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / kpad), k = static_cast<int>(i % kpad);
    double v = k < cols ? scale * a[static_cast<long long>(r) * ld + k] : 0.0;
    for (int s = 0; s < slices; ++s) out[s * slice + i] = take_slice(v, f16 != 0);
  }
}

// Grouped split: problem p's FP64 matrix src[off + r * ld + k] (r < rows,
// k < cols), times its scale, into slice rows dst_row + r of [S][..][kmax],
// zero for k >= cols.  blockIdx.y = problem.
__global__ void k_split_group(const double* __restrict__ src, const SplitDesc* __restrict__ desc,
                              int kmax, int slices, long long slice_elems, int f16,
                              uint16_t* __restrict__ out) {
  const SplitDesc d = desc[blockIdx.y];
  const long long n = static_cast<long long>(d.rows) * kmax;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(i / kmax), k = static_cast<int>(i % kmax);
    double v = k < d.cols ? d.scale * src[d.src_off + static_cast<long long>(r) * d.ld + k] : 0.0;
    const long long dst = (d.dst_row + r) * kmax + k;
    for (int s = 0; s < slices; ++s) out[s * slice_elems + dst] = take_slice(v, f16 != 0);
  }
}

// Grouped magnitudes: out[2p] = max |x|, out[2p + 1] = max over rows of
// sum |x[r][:]| of problem p (out zeroed by the caller; non-negative doubles
// order like their bit patterns).  A warp per row, blockIdx.y = problem.
__global__ void k_absmax_group(const double* __restrict__ src, const SplitDesc* __restrict__ desc,
                               unsigned long long* __restrict__ out) {
  const SplitDesc d = desc[blockIdx.y];
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  double mx = 0.0, rs_max = 0.0;
  for (long long r = static_cast<long long>(blockIdx.x) * (blockDim.x / 32) + warp; r < d.rows;
       r += static_cast<long long>(gridDim.x) * (blockDim.x / 32)) {
    double rs = 0.0;
    for (int c = lane; c < d.cols; c += 32) {
      const double v = fabs(src[d.src_off + r * d.ld + c]);
      rs += v;
      mx = fmax(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
    rs_max = fmax(rs_max, rs);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    atomicMax(out + 2 * blockIdx.y, static_cast<unsigned long long>(__double_as_longlong(mx)));
    atomicMax(out + 2 * blockIdx.y + 1, static_cast<unsigned long long>(__double_as_longlong(rs_max)));
  }
}

// ---------------------------------------------------------------------------
// step-C work units planned on the device
// ---------------------------------------------------------------------------
// A tile's slab list is cut into units: consecutive slabs until at least
// split reduction elements (the last unit takes the rest).  One thread per
// tile counts its units and adds the tile to the task statistics
// (stat[0] active tiles, stat[1] listed slabs, stat[2] reduction elements).
__global__ void k_units_count(const int* __restrict__ tasks, const int* __restrict__ counts,
                              const long long* __restrict__ kacc, const int* __restrict__ slab_len,
                              int ntiles, int nslab, int split, int* __restrict__ ucnt,
                              unsigned long long* __restrict__ stat) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    const int c = counts[t];
    const int* lst = tasks + static_cast<long long>(t) * nslab;
    int nu = 0;
    long long kk = 0;
    for (int i = 0; i < c; ++i) {
      kk += slab_len[lst[i]];
      if (kk >= split || i == c - 1) {
        ++nu;
        kk = 0;
      }
    }
    ucnt[t] = nu;
    if (c > 0) {
      atomicAdd(stat, 1ull);
      atomicAdd(stat + 1, static_cast<unsigned long long>(c));
      atomicAdd(stat + 2, static_cast<unsigned long long>(kacc[t]));
    }
  }
}

// Exclusive scan of v[0..n) into out[0..n) with one CTA of 1024 threads;
// *total = the sum.  Optionally zeroes zero[0..nz).
__global__ void k_scan_1cta(const int* __restrict__ v, int n, int* __restrict__ out,
                            int* __restrict__ total, int* __restrict__ zero, int nz) {
  __shared__ int part[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) zero[i] = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int x = i < n ? v[i] : 0;
    part[threadIdx.x] = x;
    __syncthreads();
    for (int o = 1; o < static_cast<int>(blockDim.x); o <<= 1) {  // inclusive Hillis-Steele scan
      const int y = threadIdx.x >= static_cast<unsigned>(o) ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < n) out[i] = carry + part[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// One thread per tile writes its units at uoff[t] with the key of each (its
// first slab) and counts the keys.
__global__ void k_units_emit(const int* __restrict__ tasks, const int* __restrict__ counts,
                             const int* __restrict__ slab_len, int ntiles, int nslab, int split,
                             const int* __restrict__ uoff, int* __restrict__ t_tile,
                             int* __restrict__ t_first, int* __restrict__ t_count,
                             int* __restrict__ t_key, int* __restrict__ hist) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    const int c = counts[t];
    const int* lst = tasks + static_cast<long long>(t) * nslab;
    int u = uoff[t], i0 = 0;
    long long kk = 0;
    for (int i = 0; i < c; ++i) {
      kk += slab_len[lst[i]];
      if (kk >= split || i == c - 1) {
        t_tile[u] = t;
        t_first[u] = i0;
        t_count[u] = i + 1 - i0;
        t_key[u] = lst[i0];
        atomicAdd(hist + lst[i0], 1);
        ++u;
        i0 = i + 1;
        kk = 0;
      }
    }
  }
}

// Units in order of their key (first slab, i.e. first reduction index):
// start[k] = first position of key k, advanced atomically.
__global__ void k_units_scatter(const int* __restrict__ n_units, const int* __restrict__ t_tile,
                                const int* __restrict__ t_first, const int* __restrict__ t_count,
                                const int* __restrict__ t_key, int* __restrict__ start,
                                int* __restrict__ u_tile, int* __restrict__ u_first,
                                int* __restrict__ u_count) {
  const int n = *n_units;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const int pos = atomicAdd(start + t_key[u], 1);
    u_tile[pos] = t_tile[u];
    u_first[pos] = t_first[u];
    u_count[pos] = t_count[u];
  }
}

// out[0] = max |x| of an FP32 array (as a double; out zeroed by the caller).
__global__ void k_absmax_f32(const float* __restrict__ x, long long n, unsigned long long* __restrict__ out) {
  float mx = 0.f;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    mx = fmaxf(mx, fabsf(x[i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(mx))));
}

// out[0] = max |a|, out[1] = max over rows of sum |a[r][:]| (out zeroed by
// the caller): non-negative doubles order like their bit patterns.
__global__ void k_absmax_rowsum(const double* __restrict__ a, long long ld, int rows, int cols,
                                unsigned long long* __restrict__ out) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  double mx = 0.0, rs_max = 0.0;
  for (long long r = static_cast<long long>(blockIdx.x) * (blockDim.x / 32) + warp; r < rows;
       r += static_cast<long long>(gridDim.x) * (blockDim.x / 32)) {
    double rs = 0.0;
    for (int c = lane; c < cols; c += 32) {
      const double v = fabs(a[r * ld + c]);
      rs += v;
      mx = fmax(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
    rs_max = fmax(rs_max, rs);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(mx)));
    atomicMax(out + 1, static_cast<unsigned long long>(__double_as_longlong(rs_max)));
  }
}

}  // namespace tc

void launch_absmax_rowsum(const double* a, long long ld, int rows, int cols, double* out2,
                          cudaStream_t st) {
  cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
  if (rows <= 0 || cols <= 0) return;
  int blocks = (rows + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  tc::k_absmax_rowsum<<<blocks, 256, 0, st>>>(a, ld, rows, cols, reinterpret_cast<unsigned long long*>(out2));
}

double pow2_scale(double bound) {
  if (!(bound > 0.0) || !std::isfinite(bound)) return 1.0;
  // the scaled bound is at most 2^14: four times below the binary16 maximum
  return std::ldexp(1.0, 14 - static_cast<int>(std::ceil(std::log2(bound))));
}

void launch_plan_units(const int* tasks, const int* counts, const long long* kacc, const int* slab_len,
                       int ntiles, int nslab, int split, UnitScratch w, unsigned long long* stat,
                       cudaStream_t st) {
  if (ntiles == 0) {
    cudaMemsetAsync(w.n_units, 0, sizeof(int), st);
    return;
  }
  const int g = (ntiles + 255) / 256;
  tc::k_units_count<<<g, 256, 0, st>>>(tasks, counts, kacc, slab_len, ntiles, nslab, split, w.ucnt, stat);
  tc::k_scan_1cta<<<1, 1024, 0, st>>>(w.ucnt, ntiles, w.uoff, w.n_units, w.hist, nslab);
  tc::k_units_emit<<<g, 256, 0, st>>>(tasks, counts, slab_len, ntiles, nslab, split, w.uoff, w.t_tile,
                                      w.t_first, w.t_count, w.t_key, w.hist);
  tc::k_scan_1cta<<<1, 1024, 0, st>>>(w.hist, nslab, w.start, w.total_keys, nullptr, 0);
  tc::k_units_scatter<<<152 * 4, 256, 0, st>>>(w.n_units, w.t_tile, w.t_first, w.t_count, w.t_key,
                                               w.start, w.u_tile, w.u_first, w.u_count);
}

void launch_zero_unwritten_y(void* Y, int slices, long long slice_elems, long long ldk, int Q0, int qrow,
                             int ns, const long long* seg, const int* n_ao, int s0, const int* ao_off,
                             int m0, int m1, int Lc, const int* lo, const int* hi, cudaStream_t st) {
  if (qrow == 0 || ns == 0) return;
  tc::k_zero_unwritten_y<<<152 * 16, 256, 0, st>>>(static_cast<uint16_t*>(Y), slices, slice_elems, ldk,
                                                   Q0, qrow, ns, seg, n_ao, s0, ao_off, m0, m1, Lc, lo,
                                                   hi);
}

void launch_zero_dead_y(void* Y, int slices, long long slice_elems, long long ldk, int qrow,
                        const DeadY* pairs, int n_pairs, const long long* seg, const int* n_ao, int s0,
                        cudaStream_t st) {
  if (n_pairs == 0) return;
  const int grid = n_pairs < 152 * 8 ? n_pairs : 152 * 8;
  tc::k_zero_dead_y<<<grid, 256, 0, st>>>(static_cast<uint16_t*>(Y), slices, slice_elems, ldk, qrow, pairs,
                                          n_pairs, seg, n_ao, s0);
}

void launch_split_f64(const double* a, long long ld, int rows, int cols, int kpad, int slices,
                      int f16, double scale, void* out, cudaStream_t st) {
  const long long n = static_cast<long long>(rows) * kpad;
  if (n == 0) return;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  tc::k_split_f64<<<static_cast<unsigned>(blocks), 256, 0, st>>>(a, ld, rows, cols, kpad, slices, f16,
                                                                scale, static_cast<uint16_t*>(out));
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
  // resolved once per process (a function-local static is initialised once,
  // even under concurrent first calls)
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return EncodeTiledFn{nullptr};
  }();
  return fn;
}

thread_local int g_stall_test = 0;  // test hook, per host thread

// SM count of the current device (queried per call: contexts of one process
// may sit on different devices)
int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

template <int S, class Job, bool F16>
int launch_persistent_t(const CUtensorMap& ma, const CUtensorMap& mb, const Job& job, tc::Cadence cad,
                        int* err_flag, cudaStream_t st) {
  if (job.n_tiles == 0) return 0;
  constexpr int smem = tc::Smem<S, Job>::kTotal;
  // the shared-memory opt-in is a per-device attribute of the kernel; setting
  // it twice (two threads racing on a first launch) is harmless
  static std::atomic<unsigned long long> attr_set{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
    if (cudaFuncSetAttribute(tc::k_tc_persistent<S, Job, F16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return -1;
    attr_set.fetch_or(bit, std::memory_order_release);
  }
  const int grid = job.n_tiles < num_sms() ? job.n_tiles : num_sms();
  tc::k_tc_persistent<S, Job, F16><<<grid, tc::kThreads, smem, st>>>(ma, mb, job, cad, err_flag);
  return 0;
}
// slices 2 or 3 in bf16, or 2 in binary16; flush_k = reduction elements
// between drains of the main accumulator (rounded down to a multiple of 16)
template <class Job>
int launch_persistent(int slices, int f16, const CUtensorMap& ma, const CUtensorMap& mb, const Job& job,
                      int flush_k, int* err_flag, cudaStream_t st) {
  tc::Cadence cad;
  cad.stall = g_stall_test;
  cad.main = flush_k / tc::kMmaK > 0 ? flush_k / tc::kMmaK : 1;
  const int fk = cad.main * tc::kMmaK;
  cad.write_every = tc::kWriteK / fk > 0 ? tc::kWriteK / fk : 1;
  if (f16) {
    if (slices == 2) return launch_persistent_t<2, Job, true>(ma, mb, job, cad, err_flag, st);
    return -4;
  }
  if (slices == 2) return launch_persistent_t<2, Job, false>(ma, mb, job, cad, err_flag, st);
  if (slices == 3) return launch_persistent_t<3, Job, false>(ma, mb, job, cad, err_flag, st);
  return -4;
}
}  // namespace

int make_slice_map(CUtensorMap* map, const void* base, long long k_len, long long rows, int slices,
                   int box_rows, int f16) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return -1;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (k_len * 2) % 16 != 0) return -2;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(k_len), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(slices)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(k_len * 2),
                           static_cast<cuuint64_t>(k_len * 2 * rows)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(tc::kStageK), static_cast<cuuint32_t>(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int tc_tile_rows() { return tc::kTileM; }

void tc_set_stall_test(int on) { g_stall_test = on; }

int launch_chi_tc(int slices, int f16, float out_scale, const CUtensorMap& mx, const CUtensorMap& my,
                  const int* tile_list, int n_tiles, const int* tasks, const int* counts, int max_slab,
                  const long long* slab_k0, const int* slab_len, int P0, int prow, int nri, int Q0,
                  int qrow, int nqt, double* chi, int flush_k, int* err_flag, cudaStream_t st) {
  (void)qrow;
  tc::ChiJob job{tile_list, n_tiles, nullptr, nullptr, tasks, counts, max_slab, slab_k0, slab_len, nqt,
                 P0, prow, nri, nri - Q0, chi + Q0, out_scale, nullptr, nullptr};
  return launch_persistent(slices, f16, mx, my, job, flush_k, err_flag, st);
}

int launch_chi_tc_units(int slices, int f16, float out_scale, const CUtensorMap& mx,
                        const CUtensorMap& my, const int* unit_tile, const int* unit_first,
                        const int* unit_count, int n_units, const int* n_units_dev, const int* tasks,
                        const int* counts, int max_slab, const long long* slab_k0, const int* slab_len,
                        int P0, int prow, int nri, int Q0, int qrow, int nqt, double* chi, int flush_k,
                        int* work, int* err_flag, cudaStream_t st) {
  (void)qrow;
  tc::ChiJob job{unit_tile, n_units, unit_first, unit_count, tasks, counts, max_slab, slab_k0, slab_len,
                 nqt, P0, prow, nri, nri - Q0, chi + Q0, out_scale, n_units_dev, work};
  if (work && cudaMemsetAsync(work, 0, sizeof(int), st) != cudaSuccess) return -6;
  return launch_persistent(slices, f16, mx, my, job, flush_k, err_flag, st);
}

int launch_panel_tc(int slices, int f16, float unscale, float out_scale, const CUtensorMap& mg,
                    const CUtensorMap& mp, const int4* tiles, int n_tiles, const PanelTaskTC* tasks,
                    int mode, int rows_valid, void* out, long long slice_elems, long long ldk, int P0b,
                    const long long* rowbase, const int* rowmul, const int* row_slocal, float* norm2,
                    const int* atom_of_ri, const int* atom_of_ao, const int* ao_off, int n_at, int npa,
                    int pa0, int mu_base, int m_base, int nmc, int flush_k, int* err_flag,
                    cudaStream_t st) {
  tc::PanelJob job{tiles, n_tiles, tasks, mode, rows_valid, static_cast<uint16_t*>(out), slice_elems,
                   ldk, P0b, rowbase, rowmul, row_slocal, norm2, atom_of_ri, atom_of_ao, ao_off, n_at,
                   npa, pa0, slices, mu_base, m_base, nmc, f16, unscale, out_scale};
  // mode 0: the panel rows are the A operand
  if (mode == 0) return launch_persistent(slices, f16, mp, mg, job, flush_k, err_flag, st);
  return launch_persistent(slices, f16, mg, mp, job, flush_k, err_flag, st);
}

void launch_split_group(const double* src, const SplitDesc* desc, int n_prob, int max_rows, int kmax,
                        int slices, long long slice_elems, int f16, void* out, cudaStream_t st) {
  if (n_prob == 0 || max_rows == 0) return;
  long long bx = (static_cast<long long>(max_rows) * kmax + 255) / 256;
  if (bx > 256) bx = 256;
  for (int p0 = 0; p0 < n_prob; p0 += 65535) {
    const int np = n_prob - p0 < 65535 ? n_prob - p0 : 65535;
    tc::k_split_group<<<dim3(static_cast<unsigned>(bx), np), 256, 0, st>>>(
        src, desc + p0, kmax, slices, slice_elems, f16, static_cast<uint16_t*>(out));
  }
}

void launch_absmax_group(const double* src, const SplitDesc* desc, int n_prob, int max_rows, double* out2,
                         cudaStream_t st) {
  if (n_prob == 0) return;
  cudaMemsetAsync(out2, 0, 2 * sizeof(double) * n_prob, st);
  int bx = (max_rows + 7) / 8;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  for (int p0 = 0; p0 < n_prob; p0 += 65535) {
    const int np = n_prob - p0 < 65535 ? n_prob - p0 : 65535;
    tc::k_absmax_group<<<dim3(bx, np), 256, 0, st>>>(src, desc + p0,
                                                     reinterpret_cast<unsigned long long*>(out2) + 2 * p0);
  }
}

int launch_group_tc(int slices, int f16, const CUtensorMap& ma, const CUtensorMap& mb,
                    const GroupTile* tiles, int n_tiles, double* out, int flush_k, int* err_flag,
                    cudaStream_t st) {
  tc::GroupJob job{tiles, n_tiles, out};
  return launch_persistent(slices, f16, ma, mb, job, flush_k, err_flag, st);
}

bool staged_fits_mode1(int nm, const int* n_sig, int count) {
  if (nm <= 0 || nm > tc::kTileN) return false;
  const int ng = tc::kTileN / nm;
  long long need = 0;
  for (int i = 0; i < count; ++i) need += tc::round8(7 + ng * tc::round8(nm * n_sig[i]));
  return need <= tc::kPlaneElems;
}

int launch_panel_tc_staged(int f16, float unscale, float out_scale, const CUtensorMap& mg,
                           const CUtensorMap& mp, const int4* tiles, int n_tiles,
                           const PanelTaskTC* tasks, int mode, void* out, long long slice_elems,
                           long long ldk, int P0b, int Lc, int row_ao0, int s0b,
                           const long long* rowbase, float* norm2, const int* atom_of_ri,
                           const int* atom_of_ao, const int* ao_off, const int* ri_off,
                           const int* n_ao, int npa, int pa0, int mu_base, int m_base, int nmc,
                           int flush_k, int* err_flag, cudaStream_t st) {
  tc::PanelStagedJob job{tiles, n_tiles, tasks, mode, static_cast<uint16_t*>(out), slice_elems, ldk,
                         P0b, Lc, row_ao0, s0b, rowbase, norm2, atom_of_ri, atom_of_ao, ao_off, ri_off,
                         n_ao, npa, pa0, mu_base, m_base, nmc, f16, unscale, out_scale};
  // the staged runs leave in aligned 8-element vectors in both slices
  if (ldk % 8 != 0 || slice_elems % 8 != 0 || (reinterpret_cast<uintptr_t>(out) & 15) != 0) return -5;
  // mode 0: the panel rows are the A operand
  if (mode == 0) return launch_persistent(2, f16, mp, mg, job, flush_k, err_flag, st);
  return launch_persistent(2, f16, mg, mp, job, flush_k, err_flag, st);
}

void launch_gather_g(const double* g, int nao, const PanelTaskTC* tasks, int ntasks, const int* lam,
                     int rbase, int rows_valid, int rows_per_task, int kmax, int slices,
                     long long slice_elems, int f16, double scale, void* out, cudaStream_t st) {
  if (ntasks == 0) return;
  long long per = static_cast<long long>(rows_per_task) * kmax;
  int bx = static_cast<int>((per + 255) / 256);
  if (bx > 1024) bx = 1024;
  dim3 grid(bx, ntasks);
  tc::k_gather_g<<<grid, 256, 0, st>>>(g, nao, tasks, lam, rbase, rows_valid, rows_per_task, kmax,
                                       slices, slice_elems, f16, scale, static_cast<uint16_t*>(out));
}

void launch_pt_scatter(const double* t3, const int* blk, const long long* off, const int* n_ao,
                       const int* n_ri, const int* kept, long long n_kept, const long long* rowB,
                       const int* kB, const long long* rowA, const int* kA, int kmax, int slices,
                       long long slice_elems, int f16, double scale, void* out, cudaStream_t st) {
  if (n_kept == 0) return;
  const long long grid = n_kept < 152LL * 64 ? n_kept : 152LL * 64;
  tc::k_pt_scatter<double><<<static_cast<unsigned>(grid), 128, 0, st>>>(
      t3, blk, off, n_ao, n_ri, kept, n_kept, rowB, kB, rowA, kA, kmax, slices, slice_elems, f16, scale,
      static_cast<uint16_t*>(out));
}

void launch_pt_scatter_f32(const float* t3, const int* blk, const long long* off, const int* n_ao,
                           const int* n_ri, const int* kept, long long n_kept, const long long* rowB,
                           const int* kB, const long long* rowA, const int* kA, int kmax, int slices,
                           long long slice_elems, int f16, double scale, void* out, cudaStream_t st) {
  if (n_kept == 0) return;
  const long long grid = n_kept < 152LL * 64 ? n_kept : 152LL * 64;
  tc::k_pt_scatter<float><<<static_cast<unsigned>(grid), 128, 0, st>>>(
      t3, blk, off, n_ao, n_ri, kept, n_kept, rowB, kB, rowA, kA, kmax, slices, slice_elems, f16, scale,
      static_cast<uint16_t*>(out));
}

void launch_absmax_f32(const float* x, long long n, double* out2, cudaStream_t st) {
  cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
  if (n <= 0) return;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  tc::k_absmax_f32<<<static_cast<unsigned>(blocks), 256, 0, st>>>(x, n,
                                                                 reinterpret_cast<unsigned long long*>(out2));
}

void launch_slices_block_filter(void* Z, int slices, long long slice_elems, long long ldk, int rowoff,
                                const int* ri_off, const int* ao_off, const int* n_ao, int s0,
                                int ns, const long long* seg, int pa0, int npa, int m0, int nmc,
                                int mu0, double thr, const float* norm2, unsigned char* blockflag,
                                unsigned char* tileflag, int ntile, int tile_rows, int* zlist,
                                int* zcount, cudaStream_t st) {
  const long long nblk = static_cast<long long>(ns) * nmc * npa;
  if (nblk == 0) return;
  cudaMemsetAsync(zcount, 0, sizeof(int), st);
  long long blocks = (nblk + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  tc::k_slices_block_flags<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
      ri_off, rowoff, pa0, npa, nmc, ns, thr, norm2, blockflag, tileflag, ntile, tile_rows, zlist,
      zcount);
  // many warps: each queued block is a few kilobytes of scattered rows
  const int vec = (slice_elems % 8 == 0 && ldk % 8 == 0 && (reinterpret_cast<uintptr_t>(Z) & 15) == 0) ? 1 : 0;
  tc::k_slices_zero_blocks<<<152 * 64, 256, 0, st>>>(static_cast<uint16_t*>(Z), slices, slice_elems, ldk,
                                                  rowoff, ri_off, ao_off, n_ao, s0, seg, pa0, npa, m0,
                                                  nmc, mu0, zlist, zcount, vec);
}

}  // namespace gw
