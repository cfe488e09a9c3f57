/*
 * sgtn -- tensor-network branch-and-bound for Ising spin glasses on
 * quasi-2D lattices of unit cells (arXiv:2411.16431), CUDA for sm_103a.
 *
 * C ABI.  All functions return an sgtn_status (0 on success); no exception
 * crosses the boundary.  A failed call leaves the handle usable and
 * sgtn_last_error() returns a text description.  Calls out of order (a
 * search before set_beta, ...) return SGTN_ERR_STATE.  A handle is bound to
 * the CUDA device that was current at sgtn_build_instance and to the stream
 * given there.  One handle must not be used by two threads at once; distinct
 * handles on distinct streams may be driven by concurrent host threads (the
 * library's mode flags are per thread, its device scratch per stream and its
 * allocator cache is locked) -- sgtn_batch_search does exactly that.
 *
 * Conventions shared by every entry point
 *  - H(s) = sum_{<ij>} J_ij s_i s_j + sum_i h_i s_i        (Sec. II, Eq. 1)
 *    with J_ij = j_num / denom, h_i = h_num / denom, s_i = +-1; lower energy
 *    is better and p(s) ~ exp(-beta H(s))                (Sec. III.A, Eq. 5).
 *  - Spins are grouped into an R x C grid of clusters ("sites"); site (r, c)
 *    has index r*C + c.  Couplings may join a site only to its eight
 *    king's-graph neighbours (nearest and diagonal, Sec. III, Fig. 1b/d);
 *    anything else is SGTN_ERR_ARG.
 *  - A cluster state is a bit pattern over the site's spins in increasing
 *    global index; bit value 0 means s = +1, bit value 1 means s = -1.
 *  - Host input arrays are copied during the call; the caller keeps
 *    ownership.  Output pointers are host pointers owned by the caller.
 */
#ifndef SGTN_H
#define SGTN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgtn_inst* sgtn_h;

typedef enum {
  SGTN_OK = 0,
  SGTN_ERR_ARG = -1,        /* bad size, pointer or lattice                */
  SGTN_ERR_STATE = -2,      /* call out of order                           */
  SGTN_ERR_OOM = -3,        /* device allocation failed                    */
  SGTN_ERR_NUMERICAL = -4,  /* NaN / zero norm / SVD did not converge      */
  SGTN_ERR_TIMEOUT = -5,    /* a bounded device-side loop gave up          */
  SGTN_ERR_CUDA = -6        /* any other CUDA error                        */
} sgtn_status;

/* SGTN_FP64: everything in double.  SGTN_FP32 (mixed): every contraction
 * (site diagrams, environments, projections, conditional scores) multiplies
 * and accumulates in FP32 while tensors are stored, truncated (SVD) and
 * normalised (log-norms) in FP64.  SGTN_TF32 (mixed, tensor cores): as FP32,
 * and the sparse site diagrams and environment updates with blocks of at
 * least 32 x 16 x 16, and dense GEMMs large enough for 128 x 128 tiles, run on
 * the tcgen05 tensor cores with 3xTF32 splitting (about FP32 accuracy).
 * SGTN_BF16 (mixed, tensor cores): as SGTN_TF32, but the sparse site diagrams
 * and environment updates split each operand into three BF16 slices and add
 * the six products of slice orders up to 2 (kind::f16 MMAs, FP32
 * accumulation; about FP32 accuracy again); dense GEMMs stay 3xTF32.
 * The conditionals, branch step and search run in the precision of the last
 * sgtn_contract_boundary unless sgtn_set_search_precision chose another. */
typedef enum { SGTN_FP64 = 0, SGTN_TF32 = 1, SGTN_BF16 = 2, SGTN_FP32 = 3 } sgtn_precision;

/* Build the generalized Potts model of Sec. III, Eqs. (2)-(4): cluster
 * states, intra-cluster energies E_x, projectors P^{mn} onto the spins that
 * couple to each neighbour, and compressed energies Ebar^{mn}.
 *   n_spins, n_edges          sizes; edges (ei[k], ej[k]) with ei < ej
 *   j_num[n_edges], h_num[n_spins], denom > 0
 *   site_of_spin[n_spins]     r*cols + c
 *   state_offsets, states     optional (both NULL or both set): explicit
 *                             state list of each site, site s owning
 *                             states[state_offsets[s] .. state_offsets[s+1]),
 *                             each a bit pattern as above (used for cells of
 *                             more than 16 spins or for reduced state sets);
 *                             when NULL every site enumerates all 2^k states
 *                             and k must be <= 16.
 *   stream                    cudaStream_t to run on (NULL = legacy stream)
 * On success *out receives a new handle (free with sgtn_destroy). */
int sgtn_build_instance(int32_t n_spins, int64_t n_edges, const int32_t* ei, const int32_t* ej,
                        const int32_t* j_num, const int32_t* h_num, int32_t denom,
                        const int32_t* site_of_spin, int32_t rows, int32_t cols,
                        const int64_t* state_offsets, const int64_t* states, void* stream,
                        sgtn_h* out);

/* Inverse temperature of Eq. (5).  Forms on the device the shifted site
 * weights w_x = exp(-beta (E_x - min E)) and bond factors
 * exp(-beta (Ebar - min Ebar)); the removed minima are kept as a log offset.
 * Invalidates boundary MPSs computed for another beta. */
int sgtn_set_beta(sgtn_h h, double beta);

/* Boundary-MPS contraction of Sec. III.B (Figs. 6-8): for r = R-1 .. 1,
 * psi_{r-1} ~ T_r psi_r by the right-to-left zipper keeping 2*chi singular
 * values, each zipper step followed by a one-site variational sweep of the
 * instantaneous stage (Sec. III.B "Variational zipper algorithm", Fig. 8d;
 * its range is set by sgtn_set_zipper_window), then a cut to chi and
 * n_sweeps full sweeps at chi.  All boundary MPSs stay resident on the device for the
 * branch step.  precision: SGTN_FP64 (everything in double) or a mixed mode
 * (contractions on tensor cores, truncation and log-norms in double).
 *   out_logz            log Z of Eq. (9) (may be NULL); NaN when the
 *                       approximate psi_0 has a non-positive overlap with the
 *                       top row (log Z undefined; the call still succeeds and
 *                       the boundary MPSs serve the branch step)
 *   out_worst_trunc_sv  largest, over all cuts, of the smallest retained
 *                       singular value relative to the largest (may be NULL) */
int sgtn_contract_boundary(sgtn_h h, int32_t chi, int32_t precision, int32_t n_sweeps,
                           double* out_logz, double* out_worst_trunc_sv);

/* Conditional marginals p(x_{n+1} | x_n) of Eq. (6) / Fig. 6 for a set of
 * partial configurations.  step = n+1 is the row-major index of the cluster
 * being placed; configs[count][step] holds the state index (position in the
 * site's state list) of every already placed cluster.  out_p[count][d] with
 * d the number of states of cluster `step`.  Requires contract_boundary. */
int sgtn_conditionals(sgtn_h h, int32_t step, int32_t count, const int32_t* configs, double* out_p);

/* Largest number of partial configurations one call scores together: `count`
 * of sgtn_conditionals(_noalloc) and `in_count` of sgtn_branch_step (larger
 * values return SGTN_ERR_ARG before anything is copied or launched), and the
 * number of live branches in sgtn_search / sgtn_batch_search /
 * sgtn_search_droplets: M itself may be larger (a cap the bounding never
 * reaches), but a step whose beam would exceed SGTN_MAX_BEAM returns
 * SGTN_ERR_ARG before its launches. */
#define SGTN_MAX_BEAM 1024

/* One branch-and-bound step (Sec. III.A, Fig. 3): branch every input
 * configuration over all states of cluster `step`, score candidates with the
 * chain rule (Eq. 6), keep the most probable candidate of every boundary
 * (Eq. 7), then the M most probable; ties go to the lexicographically smaller
 * configuration.
 *   in_configs[in_count][step], in_logp[in_count]
 *   out_configs[M][step+1], out_logp[M], *out_count <= M
 *   *io_pd: on entry the largest discarded log-probability so far (or
 *           -inf), on exit updated with this step's discards. */
int sgtn_branch_step(sgtn_h h, int32_t step, int32_t M, int32_t in_count, const int32_t* in_configs,
                     const double* in_logp, int32_t* out_configs, double* out_logp, int32_t* out_count,
                     double* io_pd);

/* Full search: all R*C steps from the empty configuration.  Writes up to
 * n_out final configurations (the search's merging leaves one at the end)
 *   out_spins[n_out][n_spins] (+1/-1), out_energy_num[n_out] (exact
 *   H * denom, int64), out_logp[n_out]; *out_pd = largest discarded log p;
 *   *out_count = number written. */
int sgtn_search(sgtn_h h, int32_t M, int32_t n_out, int8_t* out_spins, int64_t* out_energy_num,
                double* out_logp, double* out_pd, int32_t* out_count);

/* Search with the excitation bookkeeping of Fig. 4: as sgtn_search (n_out =
 * 1), and the droplets of the best configuration -- low-energy excitations
 * found where the bounding merged candidates with the same boundary (Eq. 7).
 * A merged-away candidate gives the main branch a droplet (the spins where it
 * differs, and the exact energy change dE, numerator over denom); its own
 * droplets are carried over too.  Kept: dE <= max_dE_num, spins connected in
 * the interaction graph (couplings J != 0), and pairwise more than
 * min_hamming flips apart (a closer droplet replaces the ones it clashes
 * with only if its dE is lower than theirs).
 *   out_spins[n_spins], *out_energy_num, *out_logp, *out_pd: the best
 *     configuration, as sgtn_search
 *   *out_ndrop   number of droplets (may exceed cap)
 *   out_dE[cap], out_offsets[cap+1], out_flips[cap * n_spins]: the first
 *     min(cap, ndrop) droplets in order of (dE, flipped spins); the spins of
 *     droplet i are out_flips[out_offsets[i] .. out_offsets[i+1]), increasing.
 * Flipping them in out_spins gives a configuration of energy
 * out_energy_num + out_dE[i].  Host buffers. */
int sgtn_search_droplets(sgtn_h h, int32_t M, int64_t max_dE_num, int32_t min_hamming, int32_t cap,
                         int8_t* out_spins, int64_t* out_energy_num, double* out_logp, double* out_pd,
                         int32_t* out_ndrop, int64_t* out_dE, int32_t* out_offsets, int32_t* out_flips);

/* Many independent searches at once (instances of different sizes, or the
 * eight grid symmetries of one instance, Sec. IV): for every handle i,
 * set_beta(beta), contract_boundary(chi, precision, n_sweeps) and
 * search(M, n_out), exactly as the three calls would do one after another.
 * Handles that share a CUDA stream run in order on one host thread; handles
 * on different streams run concurrently on up to n_threads host threads
 * (0: one per stream), so their kernels overlap on the device.  Each handle
 * must appear once.
 *   out_spins[i], out_energy_num[i], out_logp[i]: host buffers of handle i as
 *     in sgtn_search (n_out x n_spins_i, n_out, n_out)
 *   out_logz[i]  log Z of handle i (NaN if undefined or if it failed first)
 *   out_pd[i], out_count[i]  as in sgtn_search
 *   status[i]    that handle's return code (its sgtn_last_error has the text)
 * Returns SGTN_OK if every handle succeeded, else the first failing handle's
 * code; SGTN_ERR_ARG for null arrays or a repeated handle (nothing runs). */
int sgtn_batch_search(sgtn_h* hs, int32_t n, double beta, int32_t chi, int32_t precision, int32_t n_sweeps,
                      int32_t M, int32_t n_out, int8_t** out_spins, int64_t** out_energy_num, double** out_logp,
                      double* out_logz, double* out_pd, int32_t* out_count, int32_t n_threads, int32_t* status);

/* Loopy belief propagation over the clusters (Sec. IV) at the current beta,
 * for the local dimensional reduction: approximate marginals of every
 * cluster's states from messages indexed by the projected classes of Eq. (4)
 *   mu_{s->t}(a) = sum_{x: P^{st}(x)=a} exp(-beta E_x) prod_{t'!=t} nu_{t'->s}(P^{st'}(x))
 *   nu_{s->t}(b) = sum_a exp(-beta Ebar^{st}[a,b]) mu_{s->t}(a)
 *   p(x_s) ~ exp(-beta E_x) prod_t nu_{t->s}(P^{st}(x)),
 * t running over the sites that share a coupling with s.  n_iter synchronous
 * iterations from nu = 1, every nu scaled to sum 1 after its update.
 *   out_index[R*C][k]   positions (in the site's state list) of the k most
 *                       probable states of every site, most probable first,
 *                       ties to the smaller position; -1 past out_count
 *   out_marginal[R*C][k] their marginals (a site's marginals sum to 1 over
 *                       all of its states)
 *   out_count[R*C]      min(k, states of the site)
 *   *out_change         largest |nu_new - nu_old| of the last iteration (may
 *                       be NULL; 0 when n_iter = 0)
 * Host buffers.  Requires set_beta; sites of at most 2^20 states (the
 * ranking is quadratic in the states of a site). */
int sgtn_lbp(sgtn_h h, int32_t n_iter, int32_t k, int32_t* out_index, double* out_marginal, int32_t* out_count,
             double* out_change);

/* Gradient of log Z (Eq. 9): dJ[k] = d log Z / dJ_k = -beta <s_i s_j> for edge
 * k, dh[i] = -beta <s_i>, *dbeta = -<H>, evaluated as environment
 * correlators: row r is averaged in the sandwich <E_r| T_r |psi_r> of the
 * bottom-up boundary MPS psi_r and an upper boundary MPS E_r built top-down
 * with the same chi, sweeps and zipper window.  The row MPOs stay in their
 * sparse projector form throughout (Fig. 7): the transposed MPO of the
 * top-down pass is a column over (state, lower class) pairs, and dZ/dW is
 * formed only where a state reads it, so any cell size the contraction
 * takes is accepted.  Exact when the contraction is exact; with truncation
 * (chi, or the rank rule dropping singular values below 1e-12 of the
 * largest, which at low temperature can remove parts of E_r that the
 * sandwich weights heavily) it differs from the derivative of the computed
 * log Z by the truncation error.  Precision: that of the last
 * contract_boundary (with SGTN_FP32, SGTN_TF32 or SGTN_BF16 the contractions
 * of the top-down pass and of the sandwiches run in that arithmetic, while
 * truncations, environment norms, the correlator sums and the outputs stay
 * FP64; with SGTN_FP64 everything is FP64).  Requires
 * contract_boundary with n_sweeps >= 1 (SGTN_ERR_ARG otherwise; SGTN_ERR_STATE
 * before any contraction); SGTN_ERR_NUMERICAL if an environment has a zero or
 * non-finite norm.  dJ[n_edges], dh[n_spins]: host buffers. */
int sgtn_logz_grad(sgtn_h h, double* dJ, double* dh, double* dbeta);

/* Exact int64 energies (numerators over denom) of n configurations of +-1
 * spins, computed on the device: out[k] = sum j_num s_i s_j + sum h_num s_i. */
int sgtn_energies(sgtn_h h, int32_t n, const int8_t* spins, int64_t* out);

/* Introspection for tests.  sgtn_site_dims: number of states of a site.
 * sgtn_mps_shape: physical and bond dimensions of the boundary MPS psi_row
 * (phys[cols], bond[cols+1]) and its log-norm.  sgtn_mps_tensor copies
 * column `col` of psi_row to out ([phys][bond_l][bond_r], double). */
int sgtn_site_dims(sgtn_h h, int32_t site, int32_t* d);
/* After contract_boundary: number of iterative truncations that stopped at
 * their iteration cap because the singular values at the cut were not
 * separated (the truncation is then ambiguous; 0 for exact truncations), and
 * the precision the boundary was computed in. */
/* Precision of sgtn_conditionals, sgtn_conditionals_noalloc, sgtn_branch_step
 * and sgtn_search on this handle (the paper has no counterpart: its branch
 * and bound runs in the precision of its contraction).  -1 (the default)
 * follows the last sgtn_contract_boundary; SGTN_FP64, SGTN_FP32, SGTN_TF32 or
 * SGTN_BF16 fix it, e.g. an FP64 boundary (exact log Z) with FP32 conditional
 * scores.
 * SGTN_ERR_ARG for any other value. */
int sgtn_set_search_precision(sgtn_h h, int32_t precision);

/* Range of the variational sweep that follows each zipper step of
 * sgtn_contract_boundary (Sec. III.B, "Variational zipper algorithm", Fig.
 * 8d): the sweep re-optimises the boundary-MPS tensors built so far, or, to
 * limit the effort as the paper allows, only the `window` tensors next to the
 * zipper centre.  0 (the default): every tensor built so far; 1: no sweep
 * (the plain zipper of Fig. 8c); w > 1: columns c..c+w-1 after the step at
 * column c.  Takes effect at the next sgtn_contract_boundary (and
 * sgtn_logz_grad); SGTN_ERR_ARG for a negative value. */
int sgtn_set_zipper_window(sgtn_h h, int32_t window);

/* In a mixed-precision sgtn_contract_boundary (SGTN_FP32, SGTN_TF32 or SGTN_BF16), run
 * the n_sweeps full variational sweeps that follow the cut to chi (Fig. 8d)
 * with FP64 contractions (on != 0; default off).  The zipper stages, which
 * hold most of the work, stay in the mixed precision; the final sweeps then
 * converge each boundary MPS toward the variational fixed point of the FP64
 * target, which removes most of the FP32 rounding those stages leave in
 * log Z (measured on Pegasus P16 15x15, beta 2, chi 64: 1.5e-7 relative to
 * the FP64 boundary instead of about 1e-6, for 4% more boundary time).  The
 * paper has no counterpart (its contraction runs in one precision).  No
 * effect on an SGTN_FP64 contraction. */
int sgtn_set_final_sweeps_fp64(sgtn_h h, int32_t on);

/* How the one-site updates of the variational sweeps (Fig. 8d) are made
 * orthonormal before the sweep moves on.  Only the span of an updated tensor
 * matters there (the next update projects the target onto it again) and
 * nothing is truncated, so where the truncated SVD would keep every direction
 * any orthonormal basis of the same span gives the same boundary MPS in
 * another gauge, without the SVD's Jacobi rotations.  mode 1 (the default):
 * one CholeskyQR pass, Q1 = M R^{-1}, when its FP64 Cholesky factor R keeps
 * every pivot above 1e-10 of its diagonal entry and ||M||_F ||R^{-1}||_F <
 * 1e12 for the matrix M being orthonormalised (an upper bound on its
 * condition number, so no singular value falls below the rank rule's 1e-12
 * of the largest), then one Newton step toward the polar factor,
 * Q = Q1 (3 I - Q1^T Q1) / 2, accepted when max |Q1^T Q1 - I| <= 1e-6 (its
 * orthogonality error is then about the square of that or less); otherwise
 * the SVD.  mode 0:
 * always the SVD.  The paper leaves the orthonormalisation open.
 * SGTN_ERR_ARG for any other mode. */
int sgtn_set_sweep_orthonormalisation(sgtn_h h, int32_t mode);
/* Sweep orthonormalisations done so far on this handle by CholeskyQR2 and by
 * the SVD (either pointer may be NULL). */
int sgtn_sweep_orthonormalisations(sgtn_h h, int64_t* by_qr, int64_t* by_svd);

int sgtn_boundary_info(sgtn_h h, int32_t* unconverged_cuts, int32_t* precision);
int sgtn_mps_shape(sgtn_h h, int32_t row, int32_t* phys, int32_t* bond, double* lognorm);
int sgtn_mps_tensor(sgtn_h h, int32_t row, int32_t col, double* out);

/* Allocation-free variant of sgtn_conditionals (the paper has no
 * counterpart; this is a service for callers that must not let the library
 * allocate device memory at run time -- e.g. a server that hands all device
 * memory to its own pool at start-up, or a real-time loop that cannot absorb
 * the device-wide synchronisation of cudaMalloc / cudaFree).  Same arguments
 * and results as sgtn_conditionals (configs and out_p are host pointers), but
 * every device temporary is taken from one static device array of
 * SGTN_NOALLOC_SCRATCH_BYTES bytes that each GPU loading the library reserves
 * until the process exits; the call performs no device allocation.
 *  - Set-up: every call looks up the array's device address
 *    (cudaGetSymbolAddress) with the handle's device current, so the address
 *    stays right after a cudaDeviceReset; the first call on a device loads
 *    the library's device code there, so make it before any stream capture
 *    is started.
 *  - A call whose temporaries (about 8 bytes x count x states, plus the
 *    projected boundary MPS of the row) exceed the array returns SGTN_ERR_ARG
 *    and sgtn_last_error() states the bytes needed; nothing is launched.
 *  - All calls share the array and it keeps the previous call's contents;
 *    everything that must start at zero is cleared by the call itself.  Calls
 *    that overlap on the GPU (other threads, other handles, other streams)
 *    race on the array: serialise them. */
#define SGTN_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int sgtn_conditionals_noalloc(sgtn_h h, int32_t step, int32_t count, const int32_t* configs, double* out_p);

/* Dense product C[m x n] = X[m x k] Y[k x n] (row-major FP64 device
 * arrays) with the library's own GEMM in `precision` (the paper has no
 * counterpart: this is the building block of every contraction of the method,
 * exposed so that its arithmetic can be checked and timed on its own).
 * SGTN_FP64: FP64 SIMT.  SGTN_FP32: FP32 SIMT (FP32 products and sums).
 * SGTN_TF32: tcgen05 tensor cores (TMA-fed, TMEM accumulators) with 3xTF32
 * splitting -- the operands split into TF32 high and low parts, the three
 * products hi*hi + hi*lo + lo*hi summed in FP32 -- when m >= 128, n >= 64
 * and k >= 32, else FP32 SIMT; |error| <= (2^-20 + k 2^-24) (|X| |Y|)_ij.
 * `stream` is a cudaStream_t (NULL: the legacy default stream); the call is
 * asynchronous except for SGTN_TF32, which synchronises to read the kernel's
 * timeout flag (SGTN_ERR_TIMEOUT if a bounded wait gave up).  SGTN_ERR_ARG
 * for non-positive sizes, NULL pointers or another precision. */
int sgtn_gemm(int32_t precision, int32_t m, int32_t n, int32_t k, const double* X, const double* Y, double* C,
              void* stream);

/* The segmented gathered product behind the sparse site diagram of Fig. 7(b)
 * (Sec. III.B, "Employing sparsity of tensors": one chi x chi product per
 * cluster state, weighted by its Boltzmann factor, summed into the block of
 * its projected indices), exposed to test the library's contraction kernels
 * on their own.  All pointers are device memory; the work runs on `stream`
 * (NULL: the default stream), which the call synchronises to check the term
 * tables first and, in SGTN_TF32 and SGTN_BF16, to read the tensor-core
 * kernel's timeout flag afterwards.  For segment g = 0..nseg-1:
 *   O[g] = sum_{t = seg_ptr[g]}^{seg_ptr[g+1]-1} c_t X[xr[t]] Y[yr[t]],
 * c_t = coef[cidx[t]] (1 if cidx is NULL), X[i] the i-th of nx row-major
 * p x q blocks of X, Y[j] the j-th of ny row-major q x s blocks of Y, O[g]
 * the g-th row-major p x s block of O (overwritten; zero for an empty
 * segment).  seg_ptr has nseg + 1 nondecreasing entries from 0 to nterm,
 * 0 <= xr[t] < nx, 0 <= yr[t] < ny and 0 <= cidx[t] < nterm (coef holds
 * nterm values); the call copies these tables to the host and checks them
 * (synchronising the stream) before it launches anything.
 * precision: SGTN_FP64 or SGTN_FP32 (SIMT kernel), SGTN_TF32 (3xTF32 on the
 * tcgen05 tensor cores, operand tiles brought in by TMA, when p >= 32,
 * q >= 16, s >= 16 and q, s are even; else FP32), SGTN_BF16 (the same
 * tensor-core kernel with three BF16 slices per operand and six kind::f16
 * products; else FP32).  SGTN_ERR_ARG for non-positive sizes, NULL arrays,
 * an index out of range or another precision; SGTN_ERR_TIMEOUT if a bounded
 * wait of the tensor-core kernel gave up. */
int sgtn_seg_gemm(int32_t precision, int32_t p, int32_t q, int32_t s, int32_t nseg, int32_t nterm, int32_t nx,
                  int32_t ny, const int32_t* seg_ptr, const int32_t* xr, const int32_t* yr, const int32_t* cidx,
                  const double* coef, const double* X, const double* Y, double* O, void* stream);

/* Cholesky factor and inverse used by the CholeskyQR orthonormalisations of
 * the truncation (Sec. III.B; the paper truncates by SVD and does not fix
 * how), exposed to test the kernel on its own.  All pointers are device
 * memory: G (n x n, row-major; only its upper triangle is read), outputs
 * R (upper triangular, R^T R = G + shift I) and Rinv = R^{-1} (n x n,
 * row-major, zero below the diagonal; Rinv may be G), status[0] = 0, or
 * j + 1 for the first pivot j that was not positive (it is then replaced by
 * 1 and the factorisation goes on), minratio[0] (may be NULL) = the smallest
 * pivot over the matching diagonal entry of G + shift I.  FP64; orders up
 * to 48 on one CTA, larger ones as a recursive blocked factorisation (one-CTA
 * diagonal blocks, off-diagonal GEMMs over many CTAs).  Asynchronous on
 * `stream`.  SGTN_ERR_ARG for n <= 0 or a NULL output. */
int sgtn_cholesky(int32_t n, double shift, const double* G, double* R, double* Rinv, int32_t* status,
                  double* minratio, void* stream);

/* Process-wide diagnostics (the paper has no counterpart): cumulative
 * number of kernel launches issued by this library, algorithmic
 * floating-point operations of its contractions (2 m n k per gathered
 * matrix product, no padding; SVD work excluded) and number of conditional
 * marginals evaluated (one per branch x cluster state).  Any pointer may be
 * NULL.  The counters are atomic and summed over all threads. */
void sgtn_stats(int64_t* launches, double* flops, int64_t* evals);

/* Number of device allocations (cudaMalloc calls) the library has made so far
 * in this process, over all handles and threads (the paper has no
 * counterpart; it lets a caller check that a call allocated nothing). */
int64_t sgtn_device_allocations(void);

/* Optional per-kernel timing (the paper has no counterpart): when enabled,
 * every launch of the library's kernels is bracketed by CUDA events on its
 * stream, booked under a label naming the kernel and its role (for example
 * "site_diagram_f64", "theta_mul_f64", "gemm_f32", "tc_gemm_3xtf32",
 * "jacobi_f64", "cholesky_f64", "score_f32"); reset clears the totals.
 * sgtn_kernel_time returns the summed device time in ms, the number of timed
 * launches and their algorithmic flops (SGTN_ERR_ARG if the label was not
 * seen).  sgtn_kernel_names writes the labels seen so far, comma-separated and
 * NUL-terminated, into buf (at most cap bytes, truncated) and returns the
 * length the full list needs (without the NUL). */
void sgtn_kernel_timing(int32_t enable, int32_t reset);
int sgtn_kernel_time(const char* name, double* ms, int64_t* launches, double* flops);
int32_t sgtn_kernel_names(char* buf, int32_t cap);

const char* sgtn_last_error(sgtn_h h);
void sgtn_destroy(sgtn_h h);

#ifdef __cplusplus
}
#endif
#endif
