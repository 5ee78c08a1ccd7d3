// Launchers of the tensor-core kernels (k_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace gw {

// 3D TMA map over bf16 slices stored [slices][rows][k_len] (k contiguous);
// box = 64 k x box_rows rows x 1 slice, 128-byte swizzle.  0 on success.
int make_slice_map(CUtensorMap* map, const void* base, long long k_len, long long rows, int slices,
                   int box_rows);
// Rows (and columns) of one step-C tile of the tensor-core kernel.
int tc_tile_rows();
// Step C on the tensor cores: chi[P0 + p][q] -= sum over the tile's slabs of
// X[p][k] Y[q][k], split-BF16 with `slices` slices; one CTA per entry of
// tile_list (tile = pt * nqt + qt, 128 x 128).  err_flag != 0 after the
// kernel means a bounded wait gave up.  Returns 0 or a negative setup error.
int launch_chi_tc(int slices, const CUtensorMap& mx, const CUtensorMap& my, const int* tile_list,
                  int n_tiles, const int* tasks, const int* counts, int max_slab,
                  const long long* slab_k0, const int* slab_len, int P0, int prow, int nri, int nqt,
                  double* chi, int flush_k, int* err_flag, cudaStream_t st);
// FP32 -> `slices` bf16 slices, out[s * n + i].
void launch_split_bf16(int slices, const float* x, void* out, long long n, cudaStream_t st);

}  // namespace gw
