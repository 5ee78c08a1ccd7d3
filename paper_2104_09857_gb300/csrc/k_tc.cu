// Tensor-core (tcgen05) kernels of the mixed-precision chi(i tau) path.
//
// Split-BF16 products: every FP32 operand value x is stored as S bfloat16
// slices x = x_0 + x_1 + ... (x_0 = bf16(x), x_{i+1} = bf16(x - x_0 - .. - x_i),
// each residual exact in FP32).  A product a*b is formed from the slice pairs
// (i, j) with i + j <= S - 1: S = 2 gives 3 products (a0b0 + a0b1 + a1b0),
// S = 3 gives 6.
//
// Step C (Eq. 3):  chi[P][Q] -= sum_k X[P][k] Y[Q][k]  over the tile's slabs.
// One CTA per active 128 x 128 tile of chi; warp roles:
//   warp 0      TMA producer: slices of the X and Y K-steps into smem stages
//   warp 1      TMEM allocator and MMA issuer (one elected thread)
//   warps 2..9  epilogue: every chunk of `flush_k` reduction elements, TMEM
//               accumulators -> registers (FP32 sum); every few chunks and at
//               the end of the tile the sum is added to chi in FP64.
// The tensor cores' FP32 accumulation rounds each addition toward zero-ish
// (its error grows linearly with the number of accumulations), so the
// accumulators are kept short: the main slice product and the small ones go
// to separate accumulators and both are drained every chunk.
// Every mbarrier wait is bounded; on time-out the CTA raises the error flag,
// drains the copies and products it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gw_internal.h"
#include "k_tc.h"

namespace gw {
namespace tc {

constexpr int kTileM = 128;  // chi rows (P) per tile
constexpr int kTileN = 128;  // chi columns (Q) per tile
constexpr int kStageK = 64;  // bf16 elements per K step = one 128-byte swizzled row
constexpr int kMmaK = 16;
constexpr int kThreads = 320;  // 2 + 8 warps
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

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart; the tile base is 1024-aligned.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;            // leading byte offset 16 B (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;    // stride byte offset: 8 rows x 128 B
  d |= static_cast<uint64_t>(1) << 46;            // descriptor version
  d |= static_cast<uint64_t>(2) << 61;            // 128-byte swizzle
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

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int S>
struct ChiTcSmem {
  static constexpr int kStages = (S == 2) ? 3 : 2;
  static constexpr int kTileBytes = kTileM * kStageK * 2;   // 16 KB, same for A and B
  static constexpr int kStageBytes = 2 * S * kTileBytes;
  static constexpr int kOperandBytes = kStages * kStageBytes;
  static constexpr int kTotal = kOperandBytes + 256 + 1024;  // + barriers + alignment
};

// TMEM columns: buffer b holds the main accumulator (slice products (0, 0))
// at columns [256 b, 256 b + 128) and the small accumulator (all other slice
// products, about 2^-8 of the main one) at [256 b + 128, 256 b + 256).
constexpr int kTmemCols = 512;
constexpr int kEpiWarps = 8;
constexpr int kEpiCols = kTileN / 2;  // columns per epilogue thread
constexpr int kFlushChunks = 8;       // chunks summed in FP32 registers before an FP64 flush

template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    k_chi_tc(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_y,
             const int* __restrict__ tile_list, const int* __restrict__ tasks,
             const int* __restrict__ counts, int max_slab, int nqt64,
             const long long* __restrict__ slab_k0, const int* __restrict__ slab_len, int P0,
             int prow, int nri, int nqt, double* __restrict__ chi, int flush_k,
             int* __restrict__ err_flag) {
  using L = ChiTcSmem<S>;
  constexpr int kStages = L::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* operands = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOperandBytes);
  uint64_t* full = bars;                     // [kStages]
  uint64_t* empty = bars + kStages;          // [kStages]
  uint64_t* acc_full = bars + 2 * kStages;   // [2]
  uint64_t* acc_empty = acc_full + 2;        // [2]
  uint64_t* drain = acc_empty + 2;           // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int tile = tile_list[blockIdx.x];
  const int pt = tile / nqt, qt = tile % nqt;
  const int p_base = pt * kTileM, q_base = qt * kTileN;
  const int cnt = counts[tile];
  const int* list = tasks + static_cast<long long>(tile) * max_slab;
  (void)nqt64;
  // K steps of the tile and the chunking: a chunk is `per_chunk` K steps
  const int per_chunk = flush_k / kStageK > 0 ? flush_k / kStageK : 1;

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
    if (lane == 0 && cnt > 0) {
      int stage = 0;
      uint32_t phase = 0;
      int armed_parity[kStages];
      bool armed[kStages];
      for (int s = 0; s < kStages; ++s) armed[s] = false, armed_parity[s] = 0;
      bool ok = true;
      for (int i = 0; i < cnt && ok; ++i) {
        const int sl = list[i];
        const long long k0 = slab_k0[sl];
        const int len = slab_len[sl];
        for (int kk = 0; kk < len; kk += kStageK) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* st = operands + stage * L::kStageBytes;
          mbar_expect_tx(&full[stage], L::kStageBytes);
          armed[stage] = true;
          armed_parity[stage] = phase;
          const int kx = static_cast<int>(k0 + kk);
          for (int s = 0; s < S; ++s) {
            tma_load_3d(st + s * L::kTileBytes, &map_x, kx, p_base, s, &full[stage]);
            tma_load_3d(st + (S + s) * L::kTileBytes, &map_y, kx, q_base, s, &full[stage]);
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
          if (armed[s]) {
            for (uint32_t t = 0; t < kMaxPolls && !mbar_try_wait(&full[s], armed_parity[s]); ++t) {
            }
          }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && cnt > 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(kTileM, kTileN);
      int stage = 0;
      uint32_t phase = 0;
      int step = 0;  // K steps issued in the current chunk
      int chunk = 0;
      bool ok = true;
      bool issued_any = false;
      for (int i = 0; i < cnt && ok; ++i) {
        const int len = slab_len[list[i]];
        for (int kk = 0; kk < len; kk += kStageK) {
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
            mma_bf16(d_main, desc_sw128(st) + koff, desc_sw128(st + S * L::kTileBytes) + koff,
                     idesc, chunk_start ? 0u : 1u);
            bool first_small = true;
#pragma unroll
            for (int a = 0; a < S; ++a) {
#pragma unroll
              for (int b = 0; b < S - a; ++b) {
                if (a == 0 && b == 0) continue;
                const uint64_t da = desc_sw128(st + a * L::kTileBytes) + koff;
                const uint64_t db = desc_sw128(st + (S + b) * L::kTileBytes) + koff;
                mma_bf16(d_small, da, db, idesc, (chunk_start && first_small) ? 0u : 1u);
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
          const bool last = (i == cnt - 1) && (kk + kStageK >= len);
          if (++step == per_chunk || last) {
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
    // warp w reads TMEM lanes of quadrant w % 4 (rows 32 q .. 32 q + 31) and
    // the 64 columns of half (w - 2) / 4.  Each chunk's main and small
    // accumulators are added (round-to-nearest FP32) into a register sum;
    // every kFlushChunks chunks, and at the end, the sum is added to chi in FP64.
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int p = p_base + quad * 32 + lane;
    double* row = chi + static_cast<long long>(P0 + (p < prow ? p : 0)) * nri;
    float acc[kEpiCols];
#pragma unroll
    for (int j = 0; j < kEpiCols; ++j) acc[j] = 0.f;
    auto flush = [&]() {
      if (p < prow) {
#pragma unroll
        for (int j = 0; j < kEpiCols; ++j) {
          const int q = q_base + half * kEpiCols + j;
          if (q < nri) row[q] -= static_cast<double>(acc[j]);
          acc[j] = 0.f;
        }
      }
    };
    long long nsteps = 0;
    for (int i = 0; i < cnt; ++i) nsteps += slab_len[list[i]] / kStageK;
    const long long nchunks = (nsteps + per_chunk - 1) / per_chunk;
    bool ok = true;
    for (long long c = 0; c < nchunks; ++c) {
      const int buf = static_cast<int>(c & 1);
      const uint32_t use = static_cast<uint32_t>(c >> 1);
      if (!mbar_wait(&acc_full[buf], use & 1u, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t row_addr = tmem + (static_cast<uint32_t>(quad * 32) << 16);
#pragma unroll
      for (int g = 0; g < kEpiCols / 8; ++g) {
        const uint32_t col = static_cast<uint32_t>(buf * 256 + half * kEpiCols + g * 8);
        uint32_t vm[8], vs[8];
        tmem_ld8(row_addr + col, vm);
        tmem_ld8(row_addr + col + 128u, vs);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          acc[g * 8 + j] += __uint_as_float(vm[j]) + __uint_as_float(vs[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      if ((c + 1) % kFlushChunks == 0 || c + 1 == nchunks) flush();
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

// FP32 -> S bfloat16 slices, slices stored [S][n] (n = rows * ld elements).
template <int S>
__global__ void k_split_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ out,
                             long long n) {
  long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (; i < n; i += stride) {
    float r = x[i];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      __nv_bfloat16 h = __float2bfloat16_rn(r);
      out[s * n + i] = h;
      r -= __bfloat162float(h);
    }
  }
}

}  // namespace tc

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

template <int S>
int launch_chi_tc_impl(const CUtensorMap& mx, const CUtensorMap& my, const int* tile_list,
                       int n_tiles, const int* tasks, const int* counts, int max_slab,
                       const long long* slab_k0, const int* slab_len, int P0, int prow, int nri,
                       int nqt, double* chi, int flush_k, int* err_flag, cudaStream_t st) {
  if (n_tiles == 0) return 0;
  constexpr int smem = tc::ChiTcSmem<S>::kTotal;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(tc::k_chi_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
      return -1;
    attr = true;
  }
  tc::k_chi_tc<S><<<n_tiles, tc::kThreads, smem, st>>>(mx, my, tile_list, tasks, counts, max_slab, 0,
                                                       slab_k0, slab_len, P0, prow, nri, nqt, chi,
                                                       flush_k, err_flag);
  return 0;
}

int launch_chi_tc(int slices, const CUtensorMap& mx, const CUtensorMap& my, const int* tile_list,
                  int n_tiles, const int* tasks, const int* counts, int max_slab,
                  const long long* slab_k0, const int* slab_len, int P0, int prow, int nri, int nqt,
                  double* chi, int flush_k, int* err_flag, cudaStream_t st) {
  if (slices == 2)
    return launch_chi_tc_impl<2>(mx, my, tile_list, n_tiles, tasks, counts, max_slab, slab_k0,
                                 slab_len, P0, prow, nri, nqt, chi, flush_k, err_flag, st);
  if (slices == 3)
    return launch_chi_tc_impl<3>(mx, my, tile_list, n_tiles, tasks, counts, max_slab, slab_k0,
                                 slab_len, P0, prow, nri, nqt, chi, flush_k, err_flag, st);
  return -4;
}

void launch_split_bf16(int slices, const float* x, void* out, long long n, cudaStream_t st) {
  if (n == 0) return;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (slices == 2)
    tc::k_split_bf16<2><<<(unsigned)blocks, 256, 0, st>>>(x, static_cast<__nv_bfloat16*>(out), n);
  else
    tc::k_split_bf16<3><<<(unsigned)blocks, 256, 0, st>>>(x, static_cast<__nv_bfloat16*>(out), n);
}

}  // namespace gw
