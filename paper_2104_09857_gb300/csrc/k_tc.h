// Launchers of the tensor-core kernels (k_tc.cu).
//
// Operands are 16-bit slices (bf16, or binary16 when f16 != 0) stored
// [slices][rows][k] with k contiguous.  Binary16 slices hold the operand
// times a power of two (pow2_scale of a bound on its magnitude); the
// launchers take the scale of what they write and the reciprocal of the
// product of the input scales, both exact powers of two.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "gw_internal.h"

namespace gw {

// 3D TMA map over 16-bit slices stored [slices][rows][k_len] (k contiguous);
// box = 64 k x box_rows rows x 1 slice, 128-byte swizzle.  0 on success.
int make_slice_map(CUtensorMap* map, const void* base, long long k_len, long long rows, int slices,
                   int box_rows, int f16);
// Rows (and columns) of one step-C tile of the tensor-core kernel.
int tc_tile_rows();
// Test hook (process-wide): while on, every tensor-core kernel launched has
// its epilogue wait first on a barrier that nothing arrives at, so that the
// bounded waits expire (about 2 s) and the kernel returns its error flag.
void tc_set_stall_test(int on);
// 2^(14 - ceil(log2 bound)): scales a value of magnitude <= bound to <= 2^14
// (1 for a zero or non-finite bound).
double pow2_scale(double bound);
// out2[0] = max |a|, out2[1] = max_r sum_c |a[r][c]| of an FP64 [rows][cols]
// matrix (row stride ld), on the stream.
void launch_absmax_rowsum(const double* a, long long ld, int rows, int cols, double* out2,
                          cudaStream_t st);
// Step C on the tensor cores: chi[P0 + p][Q0 + q] -= out_scale * sum over
// the tile's slabs of X[p][k] Y[q][k] with `slices` slices (p < prow,
// q < qrow); one work item per entry of tile_list (tile = pt * nqt + qt,
// 128 x 128).  err_flag != 0 after
// the kernel means a bounded wait gave up.  Returns 0 or a negative setup
// error (-4: unsupported slice count / format).
int launch_chi_tc(int slices, int f16, float out_scale, const CUtensorMap& mx, const CUtensorMap& my,
                  const int* tile_list, int n_tiles, const int* tasks, const int* counts, int max_slab,
                  const long long* slab_k0, const int* slab_len, int P0, int prow, int nri, int Q0,
                  int qrow, int nqt, double* chi, int flush_k, int* err_flag, cudaStream_t st);
// Step C over work units that split tiles along K: unit u computes tile
// unit_tile[u] over list entries [unit_first[u], unit_first[u] + unit_count[u])
// of that tile's task list and adds into chi with FP64 atomics.  The number
// of units is n_units, or *n_units_dev (device memory) when that is not null,
// n_units then being the capacity of the unit arrays.  work (one device int,
// zeroed here on the stream; may be null): the CTAs take the units in order
// from this counter instead of a fixed share each.
int launch_chi_tc_units(int slices, int f16, float out_scale, const CUtensorMap& mx,
                        const CUtensorMap& my, const int* unit_tile, const int* unit_first,
                        const int* unit_count, int n_units, const int* n_units_dev, const int* tasks,
                        const int* counts, int max_slab, const long long* slab_k0, const int* slab_len,
                        int P0, int prow, int nri, int Q0, int qrow, int nqt, double* chi, int flush_k,
                        int* work, int* err_flag, cudaStream_t st);
// Device scratch of launch_plan_units: per tile (ntiles) ucnt, uoff; per unit
// (capacity ntiles * nslab) t_tile, t_first, t_count, t_key, u_tile, u_first,
// u_count; per slab (nslab) hist, start; and the counters n_units,
// total_keys.
struct UnitScratch {
  int *ucnt, *uoff, *t_tile, *t_first, *t_count, *t_key, *u_tile, *u_first, *u_count, *hist, *start;
  int *n_units, *total_keys;
};
// Step-C work units planned on the device from the task lists: tiles cut
// into units of at least `split` reduction elements (the last of a tile
// takes the rest), ordered by first slab (first reduction index); counts in
// *w.n_units.  Adds the active tiles, listed slabs and reduction elements
// into stat[0..2].
void launch_plan_units(const int* tasks, const int* counts, const long long* kacc, const int* slab_len,
                       int ntiles, int nslab, int split, UnitScratch w, unsigned long long* stat,
                       cudaStream_t st);
// Steps A/B on the tensor cores (PanelJob in k_tc.cu): mode 0 writes X, mode
// 1 writes Y, as slices of out_scale * (unscale * accumulator), and
// accumulates the squared atom-block norms of unscale * accumulator.  Tile
// entries (task, i, j): mode 0 i = panel-row tile, j = G-row tile; mode 1
// i = G-row tile, j = panel-row tile.  The G rows are local to a chunk of
// mu-atoms (nmc atoms from m_base, AOs from mu_base); norm2 is
// [ns][nmc][npa] over the RI atoms [pa0, pa0 + npa) of the output's rows,
// which start at RI function P0b.
int launch_panel_tc(int slices, int f16, float unscale, float out_scale, const CUtensorMap& mg,
                    const CUtensorMap& mp, const int4* tiles, int n_tiles, const PanelTaskTC* tasks,
                    int mode, int rows_valid, void* out, long long slice_elems, long long ldk, int P0b,
                    const long long* rowbase, const int* rowmul, const int* row_slocal, float* norm2,
                    const int* atom_of_ri, const int* atom_of_ao, const int* ao_off, int n_at, int npa,
                    int pa0, int mu_base, int m_base, int nmc, int flush_k, int* err_flag,
                    cudaStream_t st);
// One tile of a grouped product (GroupJob in k_tc.cu): out[off + r * ld + c]
// -= scale * sum_{k < 64 ksteps} A[a_row + r][k] B[b_row + c][k] for
// r < rows, c < cols (one owner per tile, FP64 read-modify-write).
struct GroupTile {
  long long out_off;
  int a_row, b_row, ksteps, rows, cols, ld;
  float scale;
  int pad;
};
// One matrix of a grouped split / magnitude pass: FP64 rows [rows][cols]
// (row stride ld) at src + src_off, written to slice rows dst_row.. with
// factor scale.
struct SplitDesc {
  long long src_off, dst_row;
  int rows, cols, ld, pad;
  double scale;
};
// scale * matrix -> 16-bit slices [S][..][kmax] for every problem in one launch
// (zero for k >= cols); max_rows bounds the problems' row counts.
void launch_split_group(const double* src, const SplitDesc* desc, int n_prob, int max_rows, int kmax,
                        int slices, long long slice_elems, int f16, void* out, cudaStream_t st);
// out2[2p] = max |x|, out2[2p + 1] = max row sum |x| of every problem.
void launch_absmax_group(const double* src, const SplitDesc* desc, int n_prob, int max_rows, double* out2,
                         cudaStream_t st);
// Many independent products of 16-bit slices in one persistent launch: A and
// B are slices [S][rows][k_len] behind 3-D TMA maps, each tile reads its own
// rows and reduction length and writes its own FP64 output block.
int launch_group_tc(int slices, int f16, const CUtensorMap& ma, const CUtensorMap& mb,
                    const GroupTile* tiles, int n_tiles, double* out, int flush_k, int* err_flag,
                    cudaStream_t st);
// Steps A/B with the staged epilogue (two slices; PanelStagedJob in k_tc.cu).
// Tile entries (task, A row offset, B row offset, rows_valid << 16 |
// cols_valid): mode 0 A = owner panel rows from a pw boundary, B = G^occ rows
// of the chunk; mode 1 A = batch rows of whole owner atoms (<= 128), B =
// panel rows from a pw boundary.  Lc: chunk segment length (mode 0);
// row_ao0, s0b: first AO and first owner atom of the batch (mode 1).
// Needs ldk and slice_elems to be multiples of 8 (returns -5 otherwise) and,
// in mode 1, every tile's staged runs to fit: staged_fits_mode1() of each
// (owner function count, row group) pair.
int launch_panel_tc_staged(int f16, float unscale, float out_scale, const CUtensorMap& mg,
                           const CUtensorMap& mp, const int4* tiles, int n_tiles,
                           const PanelTaskTC* tasks, int mode, void* out, long long slice_elems,
                           long long ldk, int P0b, int Lc, int row_ao0, int s0b,
                           const long long* rowbase, float* norm2, const int* atom_of_ri,
                           const int* atom_of_ao, const int* ao_off, const int* ri_off,
                           const int* n_ao, int npa, int pa0, int mu_base, int m_base, int nmc,
                           int flush_k, int* err_flag, cudaStream_t st);
// A (row group, owner) pair of step B whose products are all zero: Y rows
// [q0, q0 + nq) (batch-local), batch atoms [a0, a1), the owner's chunk-local
// first AO aom and function count nm.
struct DeadY {
  int q0, nq, a0, a1, aom, nm;
};
// Zero, in both slices, the Y runs of the pairs: for each row and atom s of
// the pair, Y[row][seg[s] + aom n(s), + nm n(s)) (seg per batch atom, n_ao
// per atom, s0 the batch's first atom).
void launch_zero_dead_y(void* Y, int slices, long long slice_elems, long long ldk, int qrow,
                        const DeadY* pairs, int n_pairs, const long long* seg, const int* n_ao, int s0,
                        cudaStream_t st);
// Whether a mode-1 staged tile fits in the staging area: the owner has nm
// functions and the tile's rows are the whole sigma-atoms with function
// counts n_sig[0..count) (padding of every run taken at its worst).
bool staged_fits_mode1(int nm, const int* n_sig, int count);
// Zero the part of the step-B operand Y that step B does not write: for each
// Y row (RI function Q0 + ql, ql < qrow) and batch atom s, the chunk-local mu
// (chunk atoms [m0, m1), segment Lc functions) outside the owner atoms
// [lo[q], hi[q]] whose panel windows cover q (the whole segment when none of
// them lies in the chunk).  Valid when the owners covering each q form one
// contiguous range.
void launch_zero_unwritten_y(void* Y, int slices, long long slice_elems, long long ldk, int Q0, int qrow,
                             int ns, const long long* seg, const int* n_ao, int s0, const int* ao_off,
                             int m0, int m1, int Lc, const int* lo, const int* hi, cudaStream_t st);
// scale * FP64 [rows][cols] (row stride ld) -> `slices` slices [S][rows][kpad],
// zero-padded in k.
void launch_split_f64(const double* a, long long ld, int rows, int cols, int kpad, int slices,
                      int f16, double scale, void* out, cudaStream_t st);
void launch_gather_g(const double* g, int nao, const PanelTaskTC* tasks, int ntasks, const int* lam,
                     int rbase, int rows_valid, int rows_per_task, int kmax, int slices,
                     long long slice_elems, int f16, double scale, void* out, cudaStream_t st);
// The same from the tensor kept in FP32 (option tensor_fp32).
void launch_pt_scatter_f32(const float* t3, const int* blk, const long long* off, const int* n_ao,
                           const int* n_ri, const int* kept, long long n_kept, const long long* rowB,
                           const int* kB, const long long* rowA, const int* kA, int kmax, int slices,
                           long long slice_elems, int f16, double scale, void* out, cudaStream_t st);
// out2[0] = max |x| of an FP32 array (out2[1] untouched but zeroed).
void launch_absmax_f32(const float* x, long long n, double* out2, cudaStream_t st);
// Split, transposed owner panels [slices][rows][kmax] straight from the
// kept 3c blocks (see k_pt_scatter); out must be zeroed beforehand.
void launch_pt_scatter(const double* t3, const int* blk, const long long* off, const int* n_ao,
                       const int* n_ri, const int* kept, long long n_kept, const long long* rowB,
                       const int* kB, const long long* rowA, const int* kA, int kmax, int slices,
                       long long slice_elems, int f16, double scale, void* out, cudaStream_t st);
// Atom-block filter of an operand (X or Y) from the squared norms its panel
// job accumulated: blockflag = kept and nonzero, tileflag per (sigma-atom,
// mu-atom of the chunk [m0, m0 + nmc), row tile) touched, and the filtered
// nonzero blocks zeroed in every slice (K offsets relative to the chunk's
// first AO mu0).  zlist (ns * nmc * npa ints) and zcount (one int) are
// scratch.
void launch_slices_block_filter(void* Z, int slices, long long slice_elems, long long ldk, int rowoff,
                                const int* ri_off, const int* ao_off, const int* n_ao, int s0,
                                int ns, const long long* seg, int pa0, int npa, int m0, int nmc,
                                int mu0, double thr, const float* norm2, unsigned char* blockflag,
                                unsigned char* tileflag, int ntile, int tile_rows, int* zlist,
                                int* zcount, cudaStream_t st);

}  // namespace gw
