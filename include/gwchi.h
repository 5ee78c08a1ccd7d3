/*
 * gwchi -- imaginary-time polarizability chi_PQ(i tau) of the low-scaling GW
 * method in a Gaussian basis with resolution of the identity in the overlap
 * metric (Wilhelm, Golze, Talirz, Hutter, Pignedoli, arXiv 2104.09857),
 * computed on one NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Every call returns GW_OK (0) or a negative GW_ERR_* code; the text of
 * the last error of a context is available from gw_last_error().  All device
 * work of a context runs on the CUDA stream given to gw_create (or a stream the
 * library creates).  Host arrays passed in are copied before the call returns;
 * the library never keeps or frees caller memory.
 *
 * Threads: all state (device buffers, events, options, errors) belongs to a
 * context, so separate contexts may be driven from separate host threads at
 * the same time.  One context must not be used by two threads at once.
 *
 * Units: distances in Angstrom, energies in Hartree, imaginary time in a.u.
 * Layouts are row-major.  Atom-blocked basis: atom a owns n_ao[a] consecutive
 * primary (AO) functions and n_ri[a] consecutive auxiliary (RI) functions, in
 * atom order.
 */
#ifndef GWCHI_H
#define GWCHI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gw_ctx gw_ctx;

enum gw_status {
  GW_OK = 0,
  GW_ERR_INVALID_ARG = -1, /* bad size, null pointer, out-of-range index     */
  GW_ERR_ORDER = -2,       /* a prerequisite set_* call is missing          */
  GW_ERR_ASYM = -3,        /* an (A, A, P) 3c block is not symmetric        */
  GW_ERR_NONFINITE = -4,   /* NaN or Inf in an input                         */
  GW_ERR_OOM = -5,         /* device allocation failed                       */
  GW_ERR_CUDA = -6,        /* a CUDA runtime call or kernel failed           */
  GW_ERR_TIMEOUT = -7,     /* a bounded device wait gave up                  */
  GW_ERR_NOT_SPD = -8,     /* a Cholesky factorisation met a non-positive pivot */
  GW_ERR_UNSUPPORTED = -9, /* combination of options the library does not offer */
  GW_ERR_NOT_CONVERGED = -10 /* an iterative host solve did not converge       */
};

/* Arithmetic of the contraction steps (Eq. 3).  Green's functions are always
 * built in FP64; chi is always accumulated across blocks in FP64. */
enum gw_precision {
  GW_FP64 = 0,   /* FP64 operands, FP64 accumulation (CUDA cores)                  */
  GW_FP32 = 1,   /* FP32 operands, FP32 accumulation per block slab (CUDA cores)   */
  GW_BF16X3 = 2, /* two-term BF16 split, 3 products per product, FP32 accumulation
                    on the tensor cores (tcgen05)                                  */
  GW_BF16X6 = 3, /* three-term BF16 split, 6 products per product, FP32
                    accumulation on the tensor cores (tcgen05)                     */
  GW_FP16X3 = 4  /* two-term binary16 split of each operand scaled by a power of
                    two (from a bound on its magnitude: no overflow), 3 products
                    per product, FP32 accumulation on the tensor cores; 22
                    significant bits per operand against 24 for GW_BF16X6, at
                    half the products and two thirds of the operand bytes      */
};

enum gw_screening {
  GW_SCREEN_BOUND = 0, /* exact block filter of the paper (norm < thr dropped)    */
  GW_SCREEN_MLP = 1    /* additionally skip work a learned norm model predicts to
                          fall below thr                                          */
};

typedef struct gw_stats {
  double flops_useful;   /* 2*n*m*k summed over the surviving atom-block products
                            of steps A, B and C (padding and split products not
                            counted)                                              */
  double flops_a, flops_b, flops_c;  /* the same, per step                       */
  double flops_issued;   /* arithmetic the kernels actually issued (padded tiles,
                            all split products)                                   */
  double ms_greens, ms_step_ab, ms_filter, ms_step_c, ms_total; /* last chi call */
  double ms_step_c_kernel; /* device time of the step-C kernels alone           */
  long long c_launches;  /* step-C kernel launches in the last call            */
  long long tiles_total, tiles_active, slabs_total, slabs_active;
  long long kernel_launches; /* all kernel launches of the last call           */
  double bytes_operands; /* bytes of X and Y operands written by steps A/B      */
  int n_batches;
  long long tasks_seen;    /* learned screening: step-C tasks examined            */
  long long tasks_skipped; /* learned screening: tasks dropped by the prediction  */
  long long batches_skipped; /* operand batches whose X or Y was entirely
                              filtered (their contribution to chi is zero) */
} gw_stats;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (may be NULL: the library creates and owns one). */
int gw_create(gw_ctx** out, int device, void* cuda_stream);
void gw_destroy(gw_ctx* ctx);
/* Message of the last failed call on this context ("" if none).  Owned by the
 * context; valid until the next call on it. */
const char* gw_last_error(const gw_ctx* ctx);

/* Atom-blocked basis (Eq. 1 primary functions, auxiliary RI functions).
 * xyz[n_atoms*3] Angstrom, n_ao[n_atoms] >= 1, n_ri[n_atoms] >= 1.
 * Resets any tensor or Green's function set before. */
int gw_set_basis(gw_ctx* ctx, int n_atoms, const double* xyz, const int* n_ao,
                 const int* n_ri);

/* Three-centre overlap tensor (mu sigma | P) of Eq. 4 in atom blocks.
 * blk_abp[n_blocks*3] = (A, B, P) with A <= B, no duplicates; `data` holds the
 * blocks back to back in that order, block i being [n_ao[A]][n_ao[B]][n_ri[P]]
 * row-major; n_elems = sum of block sizes.  The (B, A, P) block is implied as
 * the transpose in the first two indices.  (A, A, P) blocks must be symmetric
 * in their two primary indices (GW_ERR_ASYM otherwise, tolerance 1e-12
 * relative).  The data is copied to the device. */
int gw_set_3c_tensor(gw_ctx* ctx, long long n_blocks, const int* blk_abp,
                     const double* data, long long n_elems);

/* Mean-field orbitals and the imaginary-time grid of Eq. 2.
 * C[n_ao_total * n_ao_total]: column n is orbital n (C[mu*n_ao_total + n] is the
 * paper's C_{n mu}); eps[n_ao_total] the orbital energies (ascending as a rule;
 * the order is not used); orbitals 0..n_occ-1 occupied; mu_fermi the energy
 * zero of the exponentials, which decay only if every occupied level lies
 * below it and every virtual level above (not checked); tau[n_tau] > 0.
 * Minimax tau points come from gw_minimax_grid. */
int gw_set_greens(gw_ctx* ctx, const double* C, const double* eps, int n_occ,
                  double mu_fermi, const double* tau, int n_tau);

/* chi_PQ(i tau_j), Eq. 3, for tau indices tau_first .. tau_first+tau_count-1,
 * as real matrices: the returned chi is the paper's chi^0 divided by i, which
 * is symmetric and negative semidefinite.
 *
 * Filter (Computational Methods): every atom block of the 3c tensor, of
 * G^occ(tau)/G^virt(tau) and of the two intermediates of Eq. 3 whose Frobenius
 * norm is < thr is dropped (thr = 0: nothing is dropped, exact zeros are still
 * skipped).  chi is formed on atom blocks atom(P) <= atom(Q) and mirrored.
 *
 * precision (enum gw_precision): GW_FP64 and GW_FP32 on the CUDA cores;
 * GW_BF16X3, GW_BF16X6 and GW_FP16X3 as split 16-bit products on the tensor
 * cores with FP64 accumulation of chi across work units.  screening:
 * GW_SCREEN_BOUND (the exact filter above) or GW_SCREEN_MLP (tensor-core forms
 * only, after gw_mlp_init/gw_mlp_train: step-C tasks the network predicts
 * below thr are skipped as well).
 *
 * Reproducibility: FP64, FP32 and the tensor-core forms with option
 * c_split_k = 0 give bitwise identical results run to run; with the default
 * split-K work units the tensor-core forms add into chi with FP64 atomics,
 * so the last bits can vary.
 *
 * chi_out: [tau_count][n_ri_total][n_ri_total] FP64, a device pointer if
 * out_on_device != 0, else a host pointer.  Work buffers are allocated on the
 * device and kept in the context between calls (released by gw_destroy).
 * Errors: GW_ERR_ORDER (inputs missing), GW_ERR_INVALID_ARG (range, thr,
 * precision), GW_ERR_UNSUPPORTED (learned screening with a CUDA-core form),
 * GW_ERR_OOM, GW_ERR_CUDA, GW_ERR_TIMEOUT (a bounded wait of a tensor-core
 * kernel gave up; the context stays usable). */
int gw_chi_tau(gw_ctx* ctx, int tau_first, int tau_count, double thr, int precision,
               int screening, double* chi_out, int out_on_device);

/* Diagonal correlation self-energy of Eq. 10 for the orbitals listed:
 *   B^n[mu][P] = sum_nu C[nu][n] (nu mu | P)  (half transform of the 3c tensor)
 *   S^g_n(tau) = sum_{mu nu} G^g_{mu nu}(tau) sum_{PQ} B^n_{mu P} W_PQ(tau) B^n_{nu Q}
 *   sigma_out[a][j][0] = Sigma^c_n(i tau_j)  = -S^occ_n(tau_j)
 *   sigma_out[a][j][1] = Sigma^c_n(-i tau_j) = +S^virt_n(tau_j),  n = orbitals[a]
 * (real, phases removed as for chi; W even in tau; RI metric = identity).
 * W_tau[n_tau][n_ri][n_ri]: device if w_on_device else host (e.g. the output
 * of gw_chi_to_w).  Filter: 3c, G and (mu-atom, P-atom) blocks of B^n with
 * norm < thr are dropped.  precision: GW_FP64 (CUDA cores) or GW_BF16X3 /
 * GW_BF16X6 / GW_FP16X3 (the two products B W and (B W) B^T on the tensor
 * cores as split 16-bit tile jobs with FP64 outputs; G, B^n and the traces
 * stay FP64).
 * sigma_out: host, [n_orb][n_tau][2].  Uses the tensor, orbitals and tau grid
 * of the context. */
int gw_sigma_tau(gw_ctx* ctx, const double* W_tau, int w_on_device, const int* orbitals,
                 int n_orb, double thr, int precision, double* sigma_out);

/* Screening chain from chi(i tau) to the correlation part of the screened
 * interaction W^c(i tau), all in FP64 on the device:
 *   chi(i omega_k) = sum_j gamma[k][j] chi(i tau_j)        (cosine transform)
 *   eps_k = 1 - L^T chi(i omega_k) L,  V = L L^T              (Eq. 7, Eq. 8)
 *   W^c(i omega_k) = L (eps_k^-1 - 1) L^T, eps_k inverted through its
 *   Cholesky factor eps_k = R R^T as Z^T Z - V, Z = R^-1 L^T  (Eq. 9)
 *   W^c(i tau_j) = sum_k delta[j][k] W^c(i omega_k)           (back transform)
 * The RI overlap metric is taken as the identity (Eqs. 5-6 reduce to chi).
 * V[n_ri*n_ri]: host, symmetric positive definite (GW_ERR_NOT_SPD otherwise);
 * gamma[n_omega][n_tau], delta[n_tau][n_omega]: host transform weights;
 * chi_tau[n_tau][n_ri][n_ri] (device if chi_on_device, else host), as returned
 * by gw_chi_tau; w_tau_out[n_tau][n_ri][n_ri] (device if out_on_device).
 * GW_ERR_NOT_SPD also when some eps_k is not positive definite (chi must be
 * negative semidefinite).  Requires gw_set_basis and gw_set_greens (tau grid). */
int gw_chi_to_w(gw_ctx* ctx, const double* V, int n_omega, const double* gamma,
                const double* delta, const double* chi_tau, int chi_on_device,
                double* w_tau_out, int out_on_device);

/* chi_PQ(i tau) for one tau point in FP64 without allocating device memory.
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc when they need chi -- a host framework whose caching
 * allocator owns the device memory budget and must not see allocations behind
 * its back, a process that reserved all device memory up front, or
 * latency-bound code that cannot afford the implicit device synchronisation
 * of cudaMalloc/cudaFree.  Same result as gw_chi_tau(tau_index, 1, thr,
 * GW_FP64, GW_SCREEN_BOUND) up to summation order.
 *
 * Every per-call work buffer lives in one fixed 64 MiB array of device
 * global memory inside the library (held on each GPU that loads the library
 * until the process exits).  Systems whose Green's functions, chi and the
 * operands of one single-sigma-atom batch do not fit are rejected with
 * GW_ERR_INVALID_ARG and a message giving the bytes needed.  The FP64 tensor
 * panels depend on thr and are built by gw_chi_tau on its CUDA-core routes:
 * call it once with the same thr and precision GW_FP64 (or GW_FP32) first
 * (GW_ERR_ORDER otherwise).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture begins.  Each call copies its small per-batch
 * tables from pageable host memory and synchronises the context's stream
 * once per batch of sigma-atoms and once at its end.  All calls share the
 * array: calls whose GPU work overlaps race and corrupt each other's results.
 * chi_out_device: [n_ri_total][n_ri_total] FP64 on the context's device.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
int gw_chi_tau_noalloc(gw_ctx* ctx, int tau_index, double thr, double* chi_out_device);

/* Learned screening of step-C tasks.  Not in the paper: a learned predictor
 * of block norms that skips work on top of the exact filter.  A task is one (128 x 128 chi tile, 64-function K
 * slab) pair of the tensor-core route that survives the exact block filter;
 * its 8 features are log10 of the norm bounds of its X and Y parts (from the
 * accumulated atom-block norms), log10 tau, three centroid distances (sigma
 * atom to row tile, AO chunk to column tile, row tile to column tile, in
 * units of 10 A), the sigma atom's basis size / 13, and the log10 norm-product
 * bound.  The network (8 -> 64 -> 64 -> 1, ReLU, bf16 weights, FP32
 * accumulation) plus the log bound feature (a skip connection: it learns
 * log10 of actual norm / bound) predicts log10 of the task's contribution
 * norm; with
 * screening = GW_SCREEN_MLP, gw_chi_tau drops a task when
 * prediction + margin < log10(thr * min(1, B)) (option "mlp_margin", default
 * 0.5), B the largest norm-product bound among the tasks of the task's chi
 * tile: an absolute cut at thr where the tile's scale is 1 or more, a cut
 * relative to the tile's scale where it is smaller (chi(i tau) falls as
 * exp(-gap tau), and an absolute cut would dominate it at large tau).
 *
 * gw_mlp_log: run gw_chi_tau on the tensor-core route and record every task's
 *   features [n][8] and the log10 Frobenius norm of its actual contribution
 *   (computed from the same operands); up to cap rows are copied out, n_out =
 *   rows logged.
 * gw_mlp_init: seeded He-normal weights, zero biases.
 * gw_mlp_set_params / gw_mlp_get_params: flat FP32 master weights, layout
 *   W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3[1] (n = 4801).
 * gw_mlp_grad: mean-squared-error loss and its gradient w.r.t. the bf16
 *   weights on the given samples (forward and backward kernels).
 * gw_mlp_train: Adam (lr) on mini-batches of a shuffled copy for `epochs`;
 *   loss_per_epoch[e] (may be NULL) = training loss after epoch e.
 * gw_mlp_predict: forward pass. */
int gw_mlp_log(gw_ctx* ctx, int tau_first, int tau_count, double thr, int precision,
               float* feat_out, float* target_out, long long cap, long long* n_out);
int gw_mlp_init(gw_ctx* ctx, unsigned long long seed);
int gw_mlp_set_params(gw_ctx* ctx, const float* theta, long long n);
int gw_mlp_get_params(gw_ctx* ctx, float* theta, long long n);
int gw_mlp_grad(gw_ctx* ctx, const float* feat, const float* target, long long n, float* loss,
                float* grad);
int gw_mlp_train(gw_ctx* ctx, const float* feat, const float* target, long long n, int epochs,
                 long long batch, float lr, unsigned long long seed, float* loss_per_epoch);
int gw_mlp_predict(gw_ctx* ctx, const float* feat, long long n, float* pred);

/* RI metric of Eqs. 5, 10 and 11: out[k] = S^-1 M[k] S^-1 for n_mat symmetric
 * [n_ri][n_ri] matrices (chi~ = S^-1 chi S^-1 before gw_chi_to_w, W~ before
 * gw_sigma_tau, V~ before gw_sigma_x), FP64 on the device through the
 * Cholesky factor S = R R^T.  S: host [n_ri][n_ri], symmetric positive
 * definite (GW_ERR_NOT_SPD otherwise).  M and out: device or host as flagged;
 * out may not alias M. */
int gw_ri_metric(gw_ctx* ctx, const double* S, int n_mat, const double* M, int m_on_device,
                 double* out, int out_on_device);

/* The full atomic-orbital matrix of the correlation self-energy of Eq. 10,
 * before projection on an orbital (C_n^T Sigma C_n is the Sigma^c_n of
 * gw_sigma_tau):
 *   Sigma_{mu nu}(+i tau) = -sum (mu lam|P) G^occ_{lam sig}(tau) W_PQ(tau) (sig nu|Q)
 *   Sigma_{mu nu}(-i tau) = +sum (mu lam|P) G^virt_{lam sig}(tau) W_PQ(tau) (sig nu|Q)
 * for every tau point of gw_set_greens.  FP64 dense route on the CUDA cores
 * for molecules (n_AO^2 n_RI <= 3*2^30 and n_AO <= 2047, GW_ERR_INVALID_ARG
 * otherwise; three arrays of n_AO^2 n_RI doubles on the device).  Filter: 3c
 * blocks and G blocks with Frobenius norm < thr are dropped.  W_tau:
 * [n_tau][n_ri][n_ri], device if w_on_device else host.  sigma_out:
 * [n_tau][2][n_ao][n_ao] (index 0: +i tau, 1: -i tau), device if
 * out_on_device else host. */
int gw_sigma_ao_tau(gw_ctx* ctx, const double* W_tau, int w_on_device, double thr,
                    double* sigma_out, int out_on_device);

/* Static exchange self-energy of Eq. 11 for the orbitals listed, with the RI
 * metric S = 1:
 *   Sigma^x_n = - sum_{mu nu} D_{mu nu} sum_{PQ} B^n_{mu P} V_PQ B^n_{nu Q},
 *   D = sum_{i occ} C_mu,i C_nu,i  (the density matrix, G^occ at tau = 0)
 * computed by the engine of gw_sigma_tau with W = V at tau = 0.  V[n_ri][n_ri]:
 * device if v_on_device else host.  Filter and precision as gw_sigma_tau.
 * sx_out: host, [n_orb]. */
int gw_sigma_x(gw_ctx* ctx, const double* V, int v_on_device, const int* orbitals, int n_orb,
               double thr, int precision, double* sx_out);

/* Batched form of gw_sigma_tau for many molecules (the uneven molecule set of
 * the batched self-energy workload): Eq. 10 for the orbitals orbitals[i][0 ..
 * n_orb[i]) of the molecule held by context ctxs[i] (basis, tensor and
 * Green's functions set; every context on the same device, all with the same
 * number of tau points).  W_tau[i]: [n_tau][n_ri_i][n_ri_i] FP64, host (or
 * device when w_on_device); sigma_out[i]: [n_orb[i]][n_tau][2] host, the
 * layout of gw_sigma_tau.  Split forms (GW_BF16X3, GW_BF16X6, GW_FP16X3):
 * per tau point, each of the two products of Eq. 10 -- Y = B^n W and
 * Z = Y B^nT, every (molecule, orbital) pair -- is one persistent
 * tensor-core launch over all pairs' tiles, and the traces with G^occ and
 * G^virt one more launch; B^n is formed once per molecule from its FP64
 * panels, which are then released (one molecule's panels are resident at a
 * time).  GW_FP64 runs gw_sigma_tau's FP64 route molecule by molecule.
 * Runs on the stream of ctxs[0]; messages go to ctxs[0]'s gw_last_error.
 * Errors: GW_ERR_INVALID_ARG (null or mismatched arguments, devices or tau
 * counts, orbital index), GW_ERR_ORDER (a context without inputs),
 * GW_ERR_UNSUPPORTED (precision), GW_ERR_OOM, GW_ERR_CUDA, GW_ERR_TIMEOUT. */
int gw_sigma_tau_batch(gw_ctx* const* ctxs, int n_mol, const double* const* W_tau, int w_on_device,
                       const int* const* orbitals, const int* n_orb, double thr, int precision,
                       double* const* sigma_out);

/* G0W0 quasiparticle energies, Eq. 12, FP64 on the device, from the diagonal
 * self-energy on imaginary time (the output layout of gw_sigma_tau):
 *   Sigma^c_n(i omega_k) = sum_j [gamma_kj / 2 (S+_j + S-_j) - i s_kj (S+_j - S-_j)]
 * with S+_j = sigma_c[a][j][0] = Sigma^c_n(i tau_j), S-_j = sigma_c[a][j][1]
 * = Sigma^c_n(-i tau_j) (the sine and cosine transform of the paper's
 * quasiparticle step, Fourier kernel e^{-i omega tau}); gamma [n_omega][n_tau]
 * are full-line cosine weights (those of gw_chi_to_w; gamma/2 is the
 * half-line transform) and s_weights [n_omega][n_tau] half-line sine weights.
 * Sigma^c_n is continued to the real axis by a Pade interpolant through the
 * n_omega points i omega_k (Thiele continued fraction, Vidberg-Serene
 * coefficients) and
 *   e = eps[a] - vxc[a] + sx[a] + Re Sigma^c_n(e)
 * is solved by Newton-Raphson from eps[a] (derivative of Re Sigma^c by
 * central differences, step 1e-6; |step| < 1e-12 max(1, |e|); at most 100
 * iterations).  iters_out[a] (if not NULL) holds the iterations to
 * convergence, or minus the iterations done when the solve of orbital a
 * stopped without converging (a zero or non-finite derivative or step, or
 * 100 iterations); then qp_out[a] is the last iterate and the call returns
 * GW_ERR_NOT_CONVERGED after writing every output.  sx is the exchange term
 * of Eq. 11 and vxc the mean-field exchange-correlation level.  All arrays
 * are host memory; 2 <= n_omega <= 128, every omega positive and all distinct
 * (GW_ERR_INVALID_ARG), finite inputs (GW_ERR_NONFINITE).  Independent of the
 * context's basis and tensor. */
int gw_qp_g0w0(gw_ctx* ctx, int n_orb, int n_tau, int n_omega, const double* sigma_c,
               const double* omega, const double* gamma, const double* s_weights,
               const double* eps, const double* vxc, const double* sx, double* qp_out,
               int* iters_out);

/* Minimax grids of the imaginary-time / imaginary-frequency method (the grids
 * chi is computed on and cosine-transformed over; the passage before Eq. 7
 * and the Computational Details).  With transition energies E in
 * [e_min, e_max], x = E / e_min and R = e_max / e_min, the grid is the n-term
 * best approximation of 1/x on [1, R] in the maximum norm:
 *   GW_GRID_TIME: 1/E ~ sum_j weights[j] exp(-nodes[j] E)
 *                 (nodes = tau_j in a.u., from 1/E = int_0^inf e^{-E t} dt)
 *   GW_GRID_FREQ: 1/E ~ sum_k weights[k] E^2 / (E^2 + nodes[k]^2)^2
 *                 (nodes = omega_k, from 1/E = 4/pi int_0^inf E^2/(E^2+w^2)^2 dw)
 * Its error equioscillates at 2n + 1 energies; *max_err = max |1/E - sum| over
 * [e_min, e_max].  nodes ascending, weights positive.  Host code only: needs
 * no context and no GPU; thread-safe.  nodes, weights: caller arrays of n
 * doubles.  Errors: GW_ERR_INVALID_ARG (kind, 1 <= n <= GW_GRID_MAX_N,
 * 0 < e_min, e_max > e_min (1 + 1e-9), null pointers), GW_ERR_NONFINITE,
 * GW_ERR_NOT_CONVERGED where the best error falls to the FP64 rounding level
 * (about 1e-10 relative to 1/e_min: fewer points suffice there).  Remez
 * exchange with Levenberg-Marquardt levelling; about a millisecond to a
 * second depending on n and R. */
enum gw_grid_kind { GW_GRID_TIME = 0, GW_GRID_FREQ = 1 };
#define GW_GRID_MAX_N 64
int gw_minimax_grid(int kind, int n, double e_min, double e_max, double* nodes, double* weights,
                    double* max_err);

/* Weights of the transforms between imaginary time and frequency, for the
 * tau grid tau[n_tau] and frequency grid omega[n_omega] (both > 0) and
 * transition energies in [e_min, e_max] (the cosine transform before Eq. 7
 * and its inverse after Eq. 9; the sine and cosine transform of Sigma^c in
 * the quasiparticle step).  Least squares over 400 energies x log-spaced on
 * [e_min, e_max], minimum-norm solution with singular values below 1e-14 of
 * the largest dropped (one-sided Jacobi SVD):
 *   gamma[n_omega][n_tau]:  sum_j gamma_kj e^{-x tau_j}           ~ 2x/(x^2+omega_k^2)
 *   delta[n_tau][n_omega]:  sum_k delta_jk 2x/(x^2+omega_k^2)    ~ e^{-x tau_j}
 *   s_weights[n_omega][n_tau]: sum_j s_kj e^{-x tau_j}           ~ omega_k/(x^2+omega_k^2)
 * gamma and delta are the inputs of gw_chi_to_w; gamma and s_weights those of
 * gw_qp_g0w0 (gamma/2 is the half-line cosine transform).  Any output may be
 * NULL to skip it.  fit_err[3] (may be NULL): for gamma, delta, s_weights the
 * largest deviation over 997 energies divided by the largest target value
 * (0 for a skipped output).  Host code only: needs no context and no GPU;
 * thread-safe.  Errors: GW_ERR_INVALID_ARG (null grid, n_tau or n_omega
 * outside 1..400, a grid point <= 0, e_max <= e_min or e_min <= 0),
 * GW_ERR_NONFINITE. */
int gw_transform_weights(const double* tau, int n_tau, const double* omega, int n_omega,
                         double e_min, double e_max, double* gamma, double* delta,
                         double* s_weights, double* fit_err);

/* Eigenvalue-self-consistent GW (the paragraph after Eq. 12).  Each cycle
 * builds G of Eq. 2 from the current levels and runs gw_chi_tau (all tau
 * points, filter thr, `precision`, bound screening), gw_chi_to_w (V, gamma,
 * delta), gw_sigma_tau for `orbitals` and gw_qp_g0w0 (omega, gamma,
 * s_weights, vxc, and Sigma^x_n of gw_sigma_x computed once).  The
 * quasiparticle equation keeps the levels given to gw_set_greens as eps_n.
 * The next cycle's levels: each level moves by the shift e_k - eps_k of the
 * nearest listed orbital on its side of the gap (nearest by index; on a tie
 * the one nearer the gap; a side with no listed orbital keeps its levels);
 * with HOMO and LUMO listed this is the scissor shift.  The first cycle is
 * G0W0.  Stops when no energy changes by tol or more between two cycles.
 * Arrays as in the calls above, host memory; qp_out[n_orb] receives the last
 * energies and cycles_out (may be NULL) the cycles run.  The context's levels
 * are restored before return.  Errors: those of the calls above;
 * GW_ERR_ORDER (inputs missing); GW_ERR_INVALID_ARG (null array, n_orb < 1,
 * orbital out of range, n_omega < 2, max_cycles < 1, tol <= 0);
 * GW_ERR_NOT_CONVERGED after max_cycles, or when a shifted level crosses
 * mu_fermi (qp_out then holds the last energies). */
int gw_evgw(gw_ctx* ctx, const double* V, int n_omega, const double* omega, const double* gamma,
            const double* delta, const double* s_weights, const int* orbitals, int n_orb,
            const double* vxc, double thr, int precision, int max_cycles, double tol,
            double* qp_out, int* cycles_out);

/* Schedule search of the tensor-core chi route (no counterpart in the paper;
 * a tuner for this library's own schedule).  Searches, by coordinate descent
 * from the context's current options, the knobs that change only the order
 * and grouping of the work -- "panel_staged", "c_split_k", "c_dynamic", "batch_bytes"
 * (0.5x, 1x, 1.5x of the current budget, where device memory allows) and
 * "mu_chunk_atoms" (automatic, n_atoms/4, n_atoms/2) -- timing each candidate
 * as the device time of gw_chi_tau on tau point tau_index (one untimed call
 * first), and leaves the fastest value of each knob set in the context.
 * "flush_k" is not searched: it sets the accuracy of the FP32 accumulation.
 * trials[0 .. min(*n_trials, max_trials)) log every timing (the first is the
 * starting point).  Needs the inputs set (GW_ERR_ORDER); precision must be a
 * tensor-core form (GW_ERR_UNSUPPORTED).  Allocates one n_RI^2 FP64 chi
 * buffer for the duration of the call. */
typedef struct gw_tune_trial {
  char knob[32];     /* knob varied in this trial ("start" for the first)     */
  double value;      /* its value                                            */
  double ms;         /* device time of one gw_chi_tau(tau_index) call        */
  int panel_staged;  /* the full setting timed                               */
  int c_split_k;
  double batch_bytes;
  int mu_chunk_atoms;
} gw_tune_trial;
int gw_autotune(gw_ctx* ctx, int tau_index, double thr, int precision, gw_tune_trial* trials,
                int max_trials, int* n_trials);

/* Counters and timings of the last gw_chi_tau call. */
int gw_get_stats(const gw_ctx* ctx, gw_stats* out);

/* Tuning knobs (no effect on results beyond rounding order):
 *   "batch_bytes"  device bytes allowed for the per-batch X and Y operands
 *                  (default 40e9)
 *   "batch_atoms"  upper limit on sigma-atoms per batch (0 = no limit)
 *   "panel_stream" split forms: 1 builds the split panels per operand batch
 *                  (the owners' for step A, the chunk's atoms' for step B)
 *                  instead of keeping the whole set resident; 0 (default)
 *                  streams only when the whole set, the batch budget, chi and
 *                  the Green's functions do not fit in free device memory
 *   "tensor_fp32"  1: the next gw_set_3c_tensor keeps the device copy of the
 *                  tensor in FP32 (half the bytes; block norms, finiteness
 *                  and symmetry are still taken from the FP64 input).  Only
 *                  the tensor-core forms can then run (the CUDA-core forms,
 *                  the self-energies and the allocation-free entry point
 *                  return GW_ERR_UNSUPPORTED or GW_ERR_ORDER); rounding T to
 *                  FP32 (2^-24) is below the split forms' own representation
 *                  error.  Default 0.
 *   "panel_staged" two-slice forms (FP16x3, BF16x3): 1 (default) steps A/B
 *                  stage each finished tile in shared memory and write whole
 *                  runs of X and Y; 0 per-element stores from registers
 *   "mu_chunk_atoms" split forms: mu-atoms per chunk of the 2-D operand
 *                  batches (0 = automatic: the fewest equal chunks for which
 *                  one sigma-atom's X and Y fit in batch_bytes / 8; one chunk
 *                  keeps Y over every RI function, several give each chunk
 *                  the RI window of its atoms' 3c blocks)
 *   "flush_k"      split forms: reduction elements between drains of the
 *                  tensor cores' FP32 accumulator (rounded down to a
 *                  multiple of 16, default 64; each 16-element MMA step of the
 *                  accumulation loses about half an ulp of the running sum
 *                  toward zero; within one 64-element step of a drain
 *                  interval the smaller slice products enter first, so an
 *                  interval of at most 64 costs the main product's roundings
 *                  only)
 *   "c_split_k"    split forms: step-C work units cover about this many
 *                  reduction elements of one 128 x 128 chi tile and add into
 *                  chi with FP64 atomics, so the summation order (and the
 *                  last bits) vary from run to run; 0 = one unit per tile,
 *                  bitwise reproducible (default 2048)
 *   "c_dynamic"    split forms with c_split_k > 0: 1 (default) the CTAs take
 *                  the step-C units in order from a shared counter, so that
 *                  the units in flight read few operand slabs; 0 each CTA
 *                  takes a fixed share (every 152nd unit)
 *   "c_order"      with c_split_k = 0: tile order, 0 longest first (default),
 *                  1 grouped raster
 *   "mlp_margin"   learned screening: decades added to the predicted norm
 * Fault-injection hooks for tests (no effect on results when 0):
 *   "test_fail_alloc"  1: the next new device work buffer fails to allocate
 *                      (the call returns GW_ERR_OOM; the hook then clears)
 *   "test_stall_tc"    1: in gw_chi_tau, every tensor-core kernel waits first
 *                      on a dependency that is never met; its bounded waits
 *                      expire after about 2 s and the call returns
 *                      GW_ERR_TIMEOUT (the context stays usable)
 * Unknown keys and out-of-range values return GW_ERR_INVALID_ARG.            */
int gw_set_option(gw_ctx* ctx, const char* key, double value);

#ifdef __cplusplus
}
#endif
#endif /* GWCHI_H */
