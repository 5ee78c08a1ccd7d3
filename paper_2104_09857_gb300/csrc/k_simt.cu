// CUDA-core kernels of the chi(i tau) path: 3c block norms and panel build,
// Green's functions (Eq. 2), the two brackets of Eq. 3 as grouped panel
// GEMMs (steps A and B), the block filter of the intermediates, per-tile task
// lists, the step-C contraction in FP64 and FP32, and the final mirror.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gw_internal.h"
#include "k_simt.h"

namespace gw {

// ---------------------------------------------------------------------------
// three-centre tensor: per-block Frobenius norm, finiteness, symmetry of
// (A, A, P) blocks
// ---------------------------------------------------------------------------
__global__ void k_block_norms_3c(const double* __restrict__ t3, long long base_off,
                                 const int* __restrict__ blk, const long long* __restrict__ off,
                                 const int* __restrict__ n_ao, const int* __restrict__ n_ri,
                                 long long n_blocks, double* __restrict__ norms, int* __restrict__ bad) {
  long long b = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (b >= n_blocks) return;
  const double* x = t3 + (off[b] - base_off);
  long long n = off[b + 1] - off[b];
  double s = 0.0;
  bool nonfinite = false;
  for (long long i = lane; i < n; i += 32) {
    double v = x[i];
    if (!isfinite(v)) nonfinite = true;
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  unsigned nf = __ballot_sync(0xffffffffu, nonfinite);
  int a = blk[3 * b], bb = blk[3 * b + 1], p = blk[3 * b + 2];
  bool asym = false;
  if (a == bb) {
    int na = n_ao[a], np = n_ri[p];
    double mx = 0.0, md = 0.0;
    for (long long i = lane; i < n; i += 32) {
      int pl = (int)(i % np);
      long long r = i / np;
      int j = (int)(r % na), k = (int)(r / na);
      double v = x[i];
      double w = x[((long long)j * na + k) * np + pl];
      mx = fmax(mx, fabs(v));
      md = fmax(md, fabs(v - w));
    }
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
    }
    asym = md > 1e-12 * mx;
  }
  if (lane == 0) {
    norms[b] = sqrt(s);
    if (nf) atomicOr(bad, 1);
    if (asym) atomicOr(bad, 2);
  }
}

// Scatter the kept A <= B blocks into the owner panels:
//   block (A, B, p) -> panel(B) rows of A (value blk[a][b][P]),
//                      panel(A) rows of B (value blk[a][b][P]) if A != B.
__global__ void k_panel_scatter(const double* __restrict__ t3, const int* __restrict__ blk,
                                const long long* __restrict__ off, const int* __restrict__ n_ao,
                                const int* __restrict__ n_ri, const int* __restrict__ ri_off,
                                const int* __restrict__ kept_idx, int n_kept,
                                const long long* __restrict__ dstB, const long long* __restrict__ dstA,
                                const int* __restrict__ ldB, const int* __restrict__ ldA,
                                double* __restrict__ pool) {
  int kb = blockIdx.x;
  if (kb >= n_kept) return;
  int b = kept_idx[kb];
  int A = blk[3 * b], B = blk[3 * b + 1], p = blk[3 * b + 2];
  int na = n_ao[A], nb = n_ao[B], np = n_ri[p];
  const double* x = t3 + off[b];
  long long n = (long long)na * nb * np;
  // dstB[kb]: element offset of (row of alpha = 0, pw = ri_off[p] - p0(B), s' = 0)
  // in panel(B); row stride ldB = npw(B) * nb.
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    int pl = (int)(i % np);
    long long r = i / np;
    int be = (int)(r % nb), al = (int)(r / nb);
    double v = x[i];
    pool[dstB[kb] + (long long)al * ldB[kb] + (long long)pl * nb + be] = v;
    if (A != B) pool[dstA[kb] + (long long)be * ldA[kb] + (long long)pl * na + al] = v;
  }
}

__global__ void k_cast_f64_f32(const double* __restrict__ x, float* __restrict__ y, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stride) y[i] = (float)x[i];
}

// ---------------------------------------------------------------------------
// Eq. 2: scaled orbital columns.  occupied: C[mu][i] exp((eps_i - mu_F) tau/2),
// virtual: C[mu][a] exp(-(eps_a - mu_F) tau/2); G = Cs Cs^T.
// ---------------------------------------------------------------------------
__global__ void k_scale_orbitals(const double* __restrict__ C, const double* __restrict__ eps,
                                 int nao, int n_occ, double mu, double tau,
                                 double* __restrict__ cso, double* __restrict__ csv) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)nao * nao;
  if (i >= n) return;
  int row = (int)(i / nao), col = (int)(i % nao);
  double e = eps[col] - mu;
  if (col < n_occ) {
    cso[(long long)row * n_occ + col] = C[i] * exp(0.5 * e * tau);
  } else {
    int nv = nao - n_occ;
    csv[(long long)row * nv + (col - n_occ)] = C[i] * exp(-0.5 * e * tau);
  }
}

// Frobenius norms of the (A <= B) atom blocks of a symmetric matrix; blocks
// with norm < thr are zeroed together with their mirror.  flags[A*n+B] =
// flags[B*n+A] = kept.
__global__ void k_sym_block_filter(double* __restrict__ g, int nao, const int* __restrict__ ao_off,
                                   int n_at, double thr, unsigned char* __restrict__ flags) {
  int pair = blockIdx.x;
  int A = pair / n_at, B = pair % n_at;
  if (A > B) return;
  int a0 = ao_off[A], na = ao_off[A + 1] - a0;
  int b0 = ao_off[B], nb = ao_off[B + 1] - b0;
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < na * nb; i += blockDim.x) {
    double v = g[(long long)(a0 + i / nb) * nao + b0 + i % nb];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  bool keep = !(sqrt(red[0]) < thr);
  if (threadIdx.x == 0) {
    flags[A * n_at + B] = keep;
    flags[B * n_at + A] = keep;
  }
  if (!keep) {
    for (int i = threadIdx.x; i < na * nb; i += blockDim.x) {
      g[(long long)(a0 + i / nb) * nao + b0 + i % nb] = 0.0;
      g[(long long)(b0 + i % nb) * nao + a0 + i / nb] = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// CUDA-core tile GEMM, both operands K-major:
//   C[m][n] += alpha * sum_{k in runs} A[m][k] * B[n][k]
// 64 x 64 tile, 256 threads, thread (tx, ty) owns rows ty + 16 i and columns
// tx + 16 j (i, j < 4).  Accumulation in AccT per run; runs are added into
// FP64 registers, so FP32 products are summed in FP32 within a run only.
// ---------------------------------------------------------------------------
template <typename T, typename AccT>
__device__ __forceinline__ void tile_nt_run(const T* __restrict__ A, long long lda, int mrows,
                                            const T* __restrict__ B, long long ldb, int nrows,
                                            long long k0, int klen, T (*As)[65], T (*Bs)[65],
                                            double (&acc64)[4][4]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  AccT acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = AccT(0);
  for (int kk0 = 0; kk0 < klen; kk0 += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + 256 * e;
      int row = idx >> 4, kk = idx & 15;
      bool kin = kk0 + kk < klen;
      As[kk][row] = (row < mrows && kin) ? A[(long long)row * lda + k0 + kk0 + kk] : T(0);
      Bs[kk][row] = (row < nrows && kin) ? B[(long long)row * ldb + k0 + kk0 + kk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma((AccT)a[i], (AccT)b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc64[i][j] += (double)acc[i][j];
}

// G = Cs Cs^T (full K), written (not accumulated) into g[m][n]: tiles on
// and above the diagonal are computed and also stored transposed, so G is
// exactly symmetric (inside a diagonal tile both halves use the same k order
// and commutative products).
__global__ void k_syrk64(const double* __restrict__ cs, int nao, int K, double* __restrict__ g) {
  __shared__ double As[16][65];
  __shared__ double Bs[16][65];
  if (blockIdx.x < blockIdx.y) return;
  int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  double acc[4][4] = {};
  if (K > 0)
    tile_nt_run<double, double>(cs + (long long)m0 * K, K, min(64, nao - m0), cs + (long long)n0 * K,
                                K, min(64, nao - n0), 0, K, As, Bs, acc);
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < nao && n < nao) {
        g[(long long)m * nao + n] = acc[i][j];
        if (m0 != n0) g[(long long)n * nao + m] = acc[i][j];
      }
    }
}

// Step C: chi[P][Q] -= sum over the tile's slab list of X[P][k] Y[Q][k].
// Tile (pt, qt) covers P in [P0 + 64 pt, ...) and Q in [64 qt, ...).
template <typename T, typename AccT>
__global__ void k_chi_tiles(const T* __restrict__ X, const T* __restrict__ Y, long long ldk, int P0,
                            int prow, int nri, const int* __restrict__ tasks,
                            const int* __restrict__ counts, int max_slab, int nqt,
                            const long long* __restrict__ slab_k0, const int* __restrict__ slab_len,
                            double* __restrict__ chi) {
  __shared__ T As[16][65];
  __shared__ T Bs[16][65];
  int pt = blockIdx.y, qt = blockIdx.x;
  int tile = pt * nqt + qt;
  int cnt = counts[tile];
  if (cnt == 0) return;
  int p0 = pt * 64, q0 = qt * 64;
  int mrows = min(64, prow - p0), nrows = min(64, nri - q0);
  double acc[4][4] = {};
  const int* list = tasks + (long long)tile * max_slab;
  for (int t = 0; t < cnt; ++t) {
    int s = list[t];
    tile_nt_run<T, AccT>(X + (long long)p0 * ldk, ldk, mrows, Y + (long long)q0 * ldk, ldk, nrows,
                         slab_k0[s], slab_len[s], As, Bs, acc);
  }
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int m = p0 + ty + 16 * i, n = q0 + tx + 16 * j;
      if (m < prow && n < nri) chi[(long long)(P0 + m) * nri + n] -= acc[i][j];
    }
}

// ---------------------------------------------------------------------------
// Steps A / B: grouped panel GEMM Z[r][n] = sum_k G[lam[k]][r] * panel[k][n],
// scattered into the K-major operands.
//   mode 0 (X, Eq. 3 first bracket, G = G^occ, r = mu over all AOs):
//     X[(p0 + pw - P0b) * ldk + seg + r * nsig + s']
//   mode 1 (Y, Eq. 3 second bracket, G = G^virt, r = sigma of the batch):
//     Y[(p0 + pw) * ldk + rowbase[r] + (aom + s') * rowmul[r]]
// with n = pw * nsig + s'.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_panel_gemm(const T* __restrict__ G, int nao, const T* __restrict__ pool,
                             const int* __restrict__ lam, const PanelTask* __restrict__ tasks,
                             int mode, int r0, int R, int P0b, long long ldk,
                             const long long* __restrict__ rowbase, const int* __restrict__ rowmul,
                             T* __restrict__ out) {
  __shared__ T As[16][65];
  __shared__ T Bs[16][65];
  const PanelTask tk = tasks[blockIdx.z];
  int n0 = blockIdx.x * 64, m0 = blockIdx.y * 64;
  if (n0 >= tk.N || m0 >= R) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const T* P = pool + tk.panel_off;
  const int* lk = lam + tk.lam_off;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < tk.K; k0 += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + 256 * e;
      int kk = idx >> 6, c = idx & 63;
      bool kin = k0 + kk < tk.K;
      int r = m0 + c;
      As[kk][c] = (kin && r < R) ? G[(long long)lk[k0 + kk] * nao + r0 + r] : T(0);
      int n = n0 + c;
      Bs[kk][c] = (kin && n < tk.N) ? P[(long long)(k0 + kk) * tk.N + n] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int n = n0 + tx + 16 * j;
    if (n >= tk.N) continue;
    int pw = n / tk.nsig, sp = n - pw * tk.nsig;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r = m0 + ty + 16 * i;
      if (r >= R) continue;
      long long dst;
      if (mode == 0) {
        dst = (long long)(tk.p0 + pw - P0b) * ldk + tk.seg + (long long)(r0 + r) * tk.nsig + sp;
      } else {
        dst = (long long)(tk.p0 + pw) * ldk + rowbase[r] + (long long)(tk.aom + sp) * rowmul[r];
      }
      out[dst] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// Block filter of the intermediates and slab/tile occupancy.
// Block (m, s, p) of an operand buffer Z[row][k]: rows = RI functions of atom
// p (offset by rowoff), columns [seg(s) + ao(m) nsig(s), + n_ao(m) nsig(s)).
// Norm < thr -> zeroed.  Kept and nonzero -> flag byte of the block and of
// every (slab, row tile) it touches.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_operand_block_filter(T* __restrict__ Z, long long ldk, int rowoff,
                                       const int* __restrict__ ri_off, const int* __restrict__ ao_off,
                                       const int* __restrict__ n_ao, int s0, int ns,
                                       const long long* __restrict__ seg, int pa0, int npa, int n_at,
                                       double thr, int naop, unsigned char* __restrict__ blockflag,
                                       unsigned char* __restrict__ tileflag, int ntile,
                                       int tile_rows) {
  long long w = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  long long nblk = (long long)ns * n_at * npa;
  if (w >= nblk) return;
  int pl = (int)(w % npa);
  long long t = w / npa;
  int m = (int)(t % n_at);
  int sl = (int)(t / n_at);
  int s = s0 + sl, p = pa0 + pl;
  int nsig = n_ao[s];
  int rows0 = ri_off[p] - rowoff, nrows = ri_off[p + 1] - ri_off[p];
  long long c0 = seg[sl] + (long long)ao_off[m] * nsig;
  int ncols = n_ao[m] * nsig;
  double acc = 0.0;
  for (int r = 0; r < nrows; ++r) {
    const T* row = Z + (long long)(rows0 + r) * ldk + c0;
    for (int c = lane; c < ncols; c += 32) {
      double v = (double)row[c];
      acc += v * v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  double nrm = sqrt(acc);
  bool kept = !(nrm < thr);
  if (!kept) {
    for (int r = 0; r < nrows; ++r) {
      T* row = Z + (long long)(rows0 + r) * ldk + c0;
      for (int c = lane; c < ncols; c += 32) row[c] = T(0);
    }
  }
  bool nz = kept && nrm > 0.0;
  if (lane == 0) blockflag[w] = nz;
  if (nz) {
    // flag (sigma-atom, mu-atom, tile) for every tile the block's rows touch
    int ts = rows0 / tile_rows, te = (rows0 + nrows - 1) / tile_rows;
    for (int tt = ts + lane; tt <= te; tt += 32) tileflag[((long long)sl * n_at + m) * ntile + tt] = 1;
    (void)naop;
  }
}

// Task list per (P tile, Q tile): slabs whose X part touches the P tile and
// whose Y part touches the Q tile.  Tiles entirely below the atom-block
// diagonal (atom(first P) > atom(last Q)) get no tasks.
__global__ void k_build_tasks(const unsigned char* __restrict__ fx, const unsigned char* __restrict__ fy,
                              int nslab, int npt, int nqt, int P0, int prow, int Q0, int qrow,
                              const int* __restrict__ atom_of_ri, const int* __restrict__ slab_len,
                              int* __restrict__ tasks, int* __restrict__ counts,
                              long long* __restrict__ kacc, int tile_rows, int per, int m0, int nmc,
                              int mu0, int nmu, const int* __restrict__ atom_of_ao) {
  int tile = blockIdx.x;
  int pt = tile / nqt, qt = tile % nqt;
  int pfirst = P0 + pt * tile_rows;
  int qlast = Q0 + min(qrow, (qt + 1) * tile_rows) - 1;
  bool upper = atom_of_ri[pfirst] <= atom_of_ri[qlast];
  // warp-serial compaction in slab order (deterministic)
  if (threadIdx.x >= 32) return;
  int lane = threadIdx.x;
  int cnt = 0;
  long long ksum = 0;
  if (upper) {
    for (int base = 0; base < nslab; base += 32) {
      int s = base + lane;
      bool on = false;
      if (s < nslab) {
        // a slab is a task iff one of its mu atoms has both an X block in the
        // row tile and a Y block in the column tile (otherwise the product is
        // exactly zero)
        const int sl = s / per, c = s % per;
        const int a_lo = c * kSlabAO;  // chunk-local AO
        if (a_lo < nmu) {
          const int ma = atom_of_ao[mu0 + a_lo] - m0;
          const int mb = atom_of_ao[mu0 + min(nmu, a_lo + kSlabAO) - 1] - m0;
          for (int m = ma; m <= mb && !on; ++m)
            on = fx[((long long)sl * nmc + m) * npt + pt] && fy[((long long)sl * nmc + m) * nqt + qt];
        }
      }
      unsigned m = __ballot_sync(0xffffffffu, on);
      if (on) {
        tasks[(long long)tile * nslab + cnt + __popc(m & ((1u << lane) - 1))] = s;
        ksum += slab_len[s];
      }
      cnt += __popc(m);
    }
  }
  for (int o = 16; o > 0; o >>= 1) ksum += __shfl_xor_sync(0xffffffffu, ksum, o);
  if (lane == 0) {
    counts[tile] = cnt;
    kacc[tile] = ksum;
  }
  (void)prow;
}

// Useful flops of step C for one batch: for each (s, m) pair of the batch's
// sigma-atoms and the chunk's mu-atoms,
//   sum_{p <= q} 2 n(m) n(s) nP nQ [X(m,s,p) kept][Y(m,s,q) kept],
// X flags over RI atoms [pa0, pa0 + npa), Y flags over [qa0, qa0 + nqa).
__global__ void k_count_c(const unsigned char* __restrict__ bx, const unsigned char* __restrict__ by,
                          int ns, int m0, int nmc, int pa0, int npa, int qa0, int nqa,
                          const int* __restrict__ n_ri, const int* __restrict__ n_ao, int s0,
                          double* __restrict__ out) {
  int pair = blockIdx.x * blockDim.x + threadIdx.x;
  if (pair >= ns * nmc) return;
  int sl = pair / nmc, ml = pair % nmc;
  const unsigned char* fx = bx + ((long long)sl * nmc + ml) * npa;
  const unsigned char* fy = by + ((long long)sl * nmc + ml) * nqa;
  // suffix sums of Y over q
  double tot = 0.0, suffix = 0.0;
  int q = qa0 + nqa - 1;
  for (int pl = npa - 1; pl >= 0; --pl) {
    int p = pa0 + pl;
    while (q >= p && q >= qa0) {
      if (fy[q - qa0]) suffix += n_ri[q];
      --q;
    }
    if (fx[pl]) tot += (double)n_ri[p] * suffix;
  }
  out[pair] = 2.0 * tot * n_ao[m0 + ml] * n_ao[s0 + sl];
}

// chi_out[P][Q] = acc[P][Q] if atom(P) <= atom(Q) else acc[Q][P]
__global__ void k_mirror(const double* __restrict__ acc, double* __restrict__ out, int nri,
                         const int* __restrict__ atom_of_ri) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)nri * nri;
  if (i >= n) return;
  int P = (int)(i / nri), Q = (int)(i % nri);
  out[i] = atom_of_ri[P] <= atom_of_ri[Q] ? acc[i] : acc[(long long)Q * nri + P];
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
void launch_block_norms_3c(const double* t3, long long base_off, const int* blk, const long long* off,
                           const int* n_ao, const int* n_ri, long long n_blocks, double* norms, int* bad,
                           cudaStream_t st) {
  if (n_blocks == 0) return;
  long long grid = (n_blocks + 7) / 8;
  k_block_norms_3c<<<(unsigned)grid, 256, 0, st>>>(t3, base_off, blk, off, n_ao, n_ri, n_blocks, norms,
                                                    bad);
}

void launch_panel_scatter(const double* t3, const int* blk, const long long* off, const int* n_ao,
                          const int* n_ri, const int* ri_off, const int* kept_idx, int n_kept,
                          const long long* dstB, const long long* dstA, const int* ldB,
                          const int* ldA, double* pool, cudaStream_t st) {
  if (n_kept == 0) return;
  k_panel_scatter<<<n_kept, 256, 0, st>>>(t3, blk, off, n_ao, n_ri, ri_off, kept_idx, n_kept, dstB,
                                          dstA, ldB, ldA, pool);
}

void launch_cast_f64_f32(const double* x, float* y, long long n, cudaStream_t st) {
  if (n == 0) return;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_cast_f64_f32<<<(unsigned)blocks, 256, 0, st>>>(x, y, n);
}

void launch_greens(const double* C, const double* eps, int nao, int n_occ, double mu, double tau,
                   double* cso, double* csv, double* g_occ, double* g_virt, cudaStream_t st) {
  long long n = (long long)nao * nao;
  k_scale_orbitals<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(C, eps, nao, n_occ, mu, tau, cso, csv);
  dim3 grid((nao + 63) / 64, (nao + 63) / 64);
  k_syrk64<<<grid, 256, 0, st>>>(cso, nao, n_occ, g_occ);
  k_syrk64<<<grid, 256, 0, st>>>(csv, nao, nao - n_occ, g_virt);
}

void launch_sym_block_filter(double* g, int nao, const int* ao_off, int n_at, double thr,
                             unsigned char* flags, cudaStream_t st) {
  k_sym_block_filter<<<n_at * n_at, 256, 0, st>>>(g, nao, ao_off, n_at, thr, flags);
}

template <typename T>
void launch_panel_gemm(const T* G, int nao, const T* pool, const int* lam, const PanelTask* tasks,
                       int ntasks, int maxN, int mode, int r0, int R, int P0b, long long ldk,
                       const long long* rowbase, const int* rowmul, T* out, cudaStream_t st) {
  if (ntasks == 0 || R == 0 || maxN == 0) return;
  for (int z0 = 0; z0 < ntasks; z0 += 65535) {
    int nz = ntasks - z0 < 65535 ? ntasks - z0 : 65535;
    dim3 grid((maxN + 63) / 64, (R + 63) / 64, nz);
    k_panel_gemm<T><<<grid, 256, 0, st>>>(G, nao, pool, lam, tasks + z0, mode, r0, R, P0b, ldk,
                                         rowbase, rowmul, out);
  }
}
template void launch_panel_gemm<double>(const double*, int, const double*, const int*,
                                        const PanelTask*, int, int, int, int, int, int, long long,
                                        const long long*, const int*, double*, cudaStream_t);
template void launch_panel_gemm<float>(const float*, int, const float*, const int*,
                                       const PanelTask*, int, int, int, int, int, int, long long,
                                       const long long*, const int*, float*, cudaStream_t);

template <typename T>
void launch_operand_block_filter(T* Z, long long ldk, int rowoff, const int* ri_off,
                                 const int* ao_off, const int* n_ao, int s0, int ns,
                                 const long long* seg, int pa0, int npa, int n_at, double thr,
                                 int naop, unsigned char* blockflag, unsigned char* tileflag,
                                 int ntile, int tile_rows, cudaStream_t st) {
  long long nblk = (long long)ns * n_at * npa;
  if (nblk == 0) return;
  k_operand_block_filter<T><<<(unsigned)((nblk + 7) / 8), 256, 0, st>>>(
      Z, ldk, rowoff, ri_off, ao_off, n_ao, s0, ns, seg, pa0, npa, n_at, thr, naop, blockflag,
      tileflag, ntile, tile_rows);
}
template void launch_operand_block_filter<double>(double*, long long, int, const int*, const int*,
                                                  const int*, int, int, const long long*, int, int,
                                                  int, double, int, unsigned char*, unsigned char*,
                                                  int, int, cudaStream_t);
template void launch_operand_block_filter<float>(float*, long long, int, const int*, const int*,
                                                 const int*, int, int, const long long*, int, int,
                                                 int, double, int, unsigned char*, unsigned char*,
                                                 int, int, cudaStream_t);

void launch_build_tasks(const unsigned char* fx, const unsigned char* fy, int nslab, int npt,
                        int nqt, int P0, int prow, int Q0, int qrow, const int* atom_of_ri,
                        const int* slab_len, int* tasks, int* counts, long long* kacc,
                        int tile_rows, int per, int m0, int nmc, int mu0, int nmu,
                        const int* atom_of_ao, cudaStream_t st) {
  if (npt * nqt == 0) return;
  k_build_tasks<<<npt * nqt, 32, 0, st>>>(fx, fy, nslab, npt, nqt, P0, prow, Q0, qrow, atom_of_ri,
                                          slab_len, tasks, counts, kacc, tile_rows, per, m0, nmc, mu0,
                                          nmu, atom_of_ao);
}

void launch_count_c(const unsigned char* bx, const unsigned char* by, int ns, int m0, int nmc, int pa0,
                    int npa, int qa0, int nqa, const int* n_ri, const int* n_ao, int s0, double* out,
                    cudaStream_t st) {
  int n = ns * nmc;
  if (n == 0) return;
  k_count_c<<<(n + 127) / 128, 128, 0, st>>>(bx, by, ns, m0, nmc, pa0, npa, qa0, nqa, n_ri, n_ao, s0,
                                             out);
}

template <typename T, typename AccT>
void launch_chi_tiles(const T* X, const T* Y, long long ldk, int P0, int prow, int nri,
                      const int* tasks, const int* counts, int max_slab, int npt, int nqt,
                      const long long* slab_k0, const int* slab_len, double* chi, cudaStream_t st) {
  dim3 grid(nqt, npt);
  k_chi_tiles<T, AccT><<<grid, 256, 0, st>>>(X, Y, ldk, P0, prow, nri, tasks, counts, max_slab, nqt,
                                             slab_k0, slab_len, chi);
}
template void launch_chi_tiles<double, double>(const double*, const double*, long long, int, int, int,
                                               const int*, const int*, int, int, int,
                                               const long long*, const int*, double*, cudaStream_t);
template void launch_chi_tiles<float, float>(const float*, const float*, long long, int, int, int,
                                             const int*, const int*, int, int, int,
                                             const long long*, const int*, double*, cudaStream_t);

void launch_mirror(const double* acc, double* out, int nri, const int* atom_of_ri, cudaStream_t st) {
  long long n = (long long)nri * nri;
  k_mirror<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(acc, out, nri, atom_of_ri);
}

}  // namespace gw
