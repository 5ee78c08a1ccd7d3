// Launchers of the CUDA-core kernels (k_simt.cu).
#pragma once

#include <cuda_runtime.h>

#include "gw_internal.h"

namespace gw {

// Per-block Frobenius norms, finiteness and (A, A, P) symmetry of blocks
// [0, n_blocks) of blk/off; block b's data starts at t3 + off[b] - base_off.
void launch_block_norms_3c(const double* t3, long long base_off, const int* blk, const long long* off,
                           const int* n_ao, const int* n_ri, long long n_blocks, double* norms, int* bad,
                           cudaStream_t st);
void launch_panel_scatter(const double* t3, const int* blk, const long long* off, const int* n_ao,
                          const int* n_ri, const int* ri_off, const int* kept_idx, int n_kept,
                          const long long* dstB, const long long* dstA, const int* ldB,
                          const int* ldA, double* pool, cudaStream_t st);
void launch_cast_f64_f32(const double* x, float* y, long long n, cudaStream_t st);
void launch_greens(const double* C, const double* eps, int nao, int n_occ, double mu, double tau,
                   double* cso, double* csv, double* g_occ, double* g_virt, cudaStream_t st);
void launch_sym_block_filter(double* g, int nao, const int* ao_off, int n_at, double thr,
                             unsigned char* flags, cudaStream_t st);
template <typename T>
void launch_panel_gemm(const T* G, int nao, const T* pool, const int* lam, const PanelTask* tasks,
                       int ntasks, int maxN, int mode, int r0, int R, int P0b, long long ldk,
                       const long long* rowbase, const int* rowmul, T* out, cudaStream_t st);
template <typename T>
void launch_operand_block_filter(T* Z, long long ldk, int rowoff, const int* ri_off,
                                 const int* ao_off, const int* n_ao, int s0, int ns,
                                 const long long* seg, int pa0, int npa, int n_at, double thr,
                                 int naop, unsigned char* blockflag, unsigned char* tileflag,
                                 int ntile, int tile_rows, cudaStream_t st);
// Occupancy flags are per (sigma-atom of the batch, mu-atom of the chunk,
// tile): fx[(sl * nmc + m - m0) * npt + pt], fy[(sl * nmc + m - m0) * nqt + qt].
// The chunk's AOs are [mu0, mu0 + nmu); slabs are 64 chunk-local AOs (per
// slabs per sigma-atom); the Y rows are RI functions [Q0, Q0 + qrow).
void launch_build_tasks(const unsigned char* fx, const unsigned char* fy, int nslab, int npt,
                        int nqt, int P0, int prow, int Q0, int qrow, const int* atom_of_ri,
                        const int* slab_len, int* tasks, int* counts, long long* kacc,
                        int tile_rows, int per, int m0, int nmc, int mu0, int nmu,
                        const int* atom_of_ao, cudaStream_t st);
void launch_count_c(const unsigned char* bx, const unsigned char* by, int ns, int m0, int nmc, int pa0,
                    int npa, int qa0, int nqa, const int* n_ri, const int* n_ao, int s0, double* out,
                    cudaStream_t st);
template <typename T, typename AccT>
void launch_chi_tiles(const T* X, const T* Y, long long ldk, int P0, int prow, int nri,
                      const int* tasks, const int* counts, int max_slab, int npt, int nqt,
                      const long long* slab_k0, const int* slab_len, double* chi, cudaStream_t st);
void launch_mirror(const double* acc, double* out, int nri, const int* atom_of_ri, cudaStream_t st);

}  // namespace gw
