// Learned block-norm predictor (k_mlp.cu): constants and launchers.
#pragma once

#include <cuda_runtime.h>

namespace gw {

constexpr int kMlpFeatures = 8;
constexpr int kMlpHidden = 64;
constexpr int kMlpBound = 7;  // feature index of log10(norm-product bound)
constexpr int kMlpParams = kMlpHidden * kMlpFeatures + kMlpHidden + kMlpHidden * kMlpHidden +
                           kMlpHidden + kMlpHidden + 1;

// Norm of the X (or Y) part of every (slab, row tile): flags and squared
// norms [sigma-atom][mu-atom of the chunk [mc0, mc0 + nmc)][RI atom from
// pa0]; the chunk's AOs are [mu0, mu0 + nmu); tiles of `tile` rows from row0.
void mlp_slab_tile_norms(const float* norm2, const unsigned char* flag, int nmc, int mc0, int npa, int pa0,
                         int per, int naop_chunk, const int* atom_of_ao, const int* atom_of_ri, int mu0,
                         int nmu, int row0, int rows, int ntile, int tile, int nslab, float* out,
                         cudaStream_t st);
void mlp_task_features(const int* tasks, const int* counts, int nslab, int npt, int nqt, int per, int s0,
                       const float* xn, const float* yn, const float* cent_p, const float* cent_q,
                       const float* cent_c, const float* xyz, const int* n_ao, float log_tau,
                       float* feat, cudaStream_t st);
void mlp_task_norms(const void* xs, const void* ys, int slices, int f16, float xinv, float yinv,
                    long long xslice, long long yslice, long long ldk, int prow, int nri, const int* tasks,
                    const int* counts, int nslab, int npt, int nqt, int max_count, int tile,
                    const long long* slab_k0, const int* slab_len, float* target, cudaStream_t st);
void mlp_forward(const void* wb, const float* x, long long n, const int* valid, int stride, float* z1,
                 float* z2, float* y, cudaStream_t st);
void mlp_backward(const void* wb, const float* x, const float* z1, const float* z2, const float* y,
                  const float* t, long long n, float* dy, float* dz1, float* dz2, float* grad,
                  cudaStream_t st);
void mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, void* wb,
              cudaStream_t st);
void mlp_round(const float* theta, void* wb, cudaStream_t st);
// Drop from each tile's list the tasks whose prediction + margin is below
// log_thr + min(0, largest log10 norm-product bound among the tile's tasks)
// (feat: [tiles][nslab][kMlpFeatures], the bound is feature 7).
void mlp_compact(int* tasks, int* counts, long long* kacc, int ntiles, int nslab, const float* pred,
                 const float* feat, float margin, float log_thr, const int* slab_len, int* skipped,
                 cudaStream_t st);

}  // namespace gw
