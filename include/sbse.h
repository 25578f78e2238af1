/*
 * sbse.h - C ABI of the GB300 library for the stochastic Bethe-Salpeter hot path of
 * Bradbury, Nguyen, Caram & Neuhauser, "Bethe Salpeter Equation Spectra for Very Large Systems"
 * (arXiv 2205.06690):
 *
 *   the action of the screened interaction W on occupied pair densities phi_i phi_j, computed by
 *   stochastic time-dependent-Hartree (TDH) propagation (Sec. II.B, Eqs. 10-15); the
 *   contraction of the screened potentials into the Tamm-Dancoff matrix A of Eq. (1); and the
 *   lowest eigenvalues (excitons) of A.
 *
 * Conventions for every function:
 *  - Returns SBSE_OK (0) or a negative SBSE_ERR_* code; sbse_last_error() gives the message.
 *    No exception crosses the ABI. A failed call leaves the context usable unless it returned
 *    SBSE_ERR_CUDA or SBSE_ERR_DEVICE_TIMEOUT, after which the context should be destroyed.
 *  - Host buffers belong to the caller. Inputs are copied; nothing is retained after return.
 *  - Calls are synchronous: on return all device work of the call has finished.
 *  - One context per host thread. A context owns its device memory and one CUDA stream.
 *  - Call order: sbse_set_grid -> sbse_set_orbitals -> sbse_apply_W (all pairs) ->
 *    sbse_build_A -> sbse_spectrum. Out-of-order calls return SBSE_ERR_NOT_READY.
 *  - Grid layout: a field on the N^3 periodic grid of the cubic box [0, L)^3 is N^3 doubles,
 *    point r = h (ix, iy, iz), h = L/N, index ix + N (iy + N iz) (x fastest).
 *  - Units: Hartree atomic units (bohr, Hartree, hbar = 1).
 */
#ifndef SBSE_H
#define SBSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SBSE_OK 0
#define SBSE_ERR_INVALID_ARG (-1)   /* NULL pointer, value out of range */
#define SBSE_ERR_SHAPE (-2)         /* unsupported grid size or window sizes */
#define SBSE_ERR_OOM (-3)           /* device allocation failed */
#define SBSE_ERR_DEVICE_TIMEOUT (-4)/* a bounded device-side wait gave up */
#define SBSE_ERR_NOT_READY (-5)     /* call order violated */
#define SBSE_ERR_NUMERIC (-6)       /* NaN or Inf in an input or a result */
#define SBSE_ERR_CUDA (-7)          /* CUDA runtime error */
#define SBSE_ERR_UNSUPPORTED (-8)   /* option not implemented in this build */

/* precision modes (sbse_create) */
#define SBSE_FP64 0  /* every step in FP64 */
#define SBSE_MIXED 1 /* FFTs, propagation, cleaning in FP32; W accumulator, A, eigensolve FP64 */

/* distribution of the stochastic coefficients c[l][s] of Eq. (14) */
#define SBSE_COEFF_GAUSSIAN 0 /* N(0, 1) */
#define SBSE_COEFF_SIGN 1     /* +-1, as printed in Eq. (14) */

/* terms of Eq. (1) included by sbse_build_A (the diagonal eps_a - eps_i + Delta is always in) */
#define SBSE_EXCHANGE 1u /* + 2 (ia|jb) */
#define SBSE_DIRECT 2u   /* - (phi_a phi_b | W | phi_i phi_j) */
#define SBSE_DIRECT_PARTIAL 4u /* the direct term from the pairs that have W; the others count as zero */

typedef struct sbse_ctx sbse_ctx;

/* Parameters of one stochastic-TDH run (Sec. II.B; values used in Sec. III: L = 10,
 * dt = 0.1, M = 10, gamma = 0.1 Ha).
 *   n_s         L, number of stochastic occupied orbitals eta_l (Eq. 14), 1..64
 *   n_steps     N_t, number of split-operator steps; W^pol integrates t in [0, N_t dt] (Eq. 13)
 *   clean_every M of Eq. (15) (0 = never clean); cleaning happens before step n when n % M == 0
 *   dt          time step (a.u.)
 *   gamma       Gaussian damping width of Eq. (13) (Ha)
 *   alpha       kick strength of psi_s(0) = exp(-i alpha q_ij) phi_s (paper: 1e-6 .. 1e-4)
 *   seed        key of the counter-based splitmix64 stream for c[l][s] (see sbse_coefficients)
 *   coeff_dist  SBSE_COEFF_GAUSSIAN or SBSE_COEFF_SIGN
 *   feedback    1 = TDH (u enters the propagation, RPA screening); 0 = propagate with H0 only
 *               (u is still recorded), which gives v chi0 v instead of v chi v */
typedef struct {
  int n_s;
  int n_steps;
  int clean_every;
  double dt;
  double gamma;
  double alpha;
  uint64_t seed;
  int coeff_dist;
  int feedback;
} sbse_tdh_params;

/* Create a context on CUDA device `device` with precision SBSE_FP64 or SBSE_MIXED.
 * *out receives the context (NULL on failure). Errors: INVALID_ARG, CUDA. */
int sbse_create(sbse_ctx **out, int device, int precision);

/* Free all device memory and the stream of the context. NULL is allowed. */
void sbse_destroy(sbse_ctx *ctx);

/* Define the grid and the local potential V_loc of H0 = -1/2 Laplacian + V_loc.
 * n: points per axis, with prime factors in {2, 3, 5}, 4 <= n <= 128.
 * box: edge L of the cubic box (bohr, > 0).
 * v_loc: host, n^3 doubles, x fastest; copied.
 * The kinetic operator is spectral (plane waves of the periodic box), the Coulomb operator is
 * the periodic 4 pi / |G|^2 with the G = 0 term removed (the paper's finite-box treatment,
 * Sec. II.B). Resets orbitals and results. Errors: INVALID_ARG, SHAPE, OOM, NUMERIC, CUDA. */
int sbse_set_grid(sbse_ctx *ctx, int n, double box, const double *v_loc);

/* Set the orbitals of the closed-shell system (Sec. II, "Method": 2 N_occ electrons, n_o valence
 * states phi_i and n_c conduction states phi_a, eigenstates of H0).
 * phi: host, (n_occ + n_c) x n^3 doubles, states in ascending energy, real, normalised so that
 *      sum_r phi_s(r)^2 h^3 = 1; rows 0..n_occ-1 are all occupied states.
 * eps: host, n_occ + n_c eigenvalues (Ha).
 * The valence window is the top n_o occupied states (i = 0..n_o-1 <-> state n_occ - n_o + i) and
 * the conduction window the bottom n_c virtual states (a = 0..n_c-1 <-> state n_occ + a).
 * scissor: Delta of Eq. (9), added to every eps_a - eps_i on the diagonal of A.
 * Requires sbse_set_grid. Resets results. Errors: INVALID_ARG, NOT_READY, OOM, NUMERIC, CUDA. */
int sbse_set_orbitals(sbse_ctx *ctx, int n_occ, int n_o, int n_c, const double *phi,
                      const double *eps, double scissor);

/* Host-only helper: the coefficient matrix c[l][s] (n_s x n_occ, row-major) that sbse_apply_W
 * draws for `seed`. Output k of splitmix64 started from state `seed` is
 * z = mix(seed + (k + 1) * 0x9E3779B97F4A7C15). SIGN: c = -1 if bit 63 of output l*n_occ + s is
 * set, else +1. GAUSSIAN: u1, u2 = 53-bit uniforms (z >> 11) * 2^-53 of outputs 2(l*n_occ + s)
 * and 2(l*n_occ + s) + 1; c = sqrt(-2 ln(1 - u1)) cos(2 pi u2). Errors: INVALID_ARG. */
int sbse_coefficients(uint64_t seed, int n_s, int n_occ, int dist, double *out);

/* Compute the screened potentials W_ij(r) = q_ij(r) + W^pol_ij(r) (Sec. II.B: q_ij = v phi_i phi_j,
 * W^pol_ij from Eq. 13) for n_pairs pairs (pi[k], pj[k]) of valence-window indices,
 * 0 <= pi[k] <= pj[k] < n_o, by stochastic TDH with the parameters p:
 *   eta_l = L^-1/2 sum_{s <= N_occ} c[l][s] phi_s (Eq. 14); kick exp(-i alpha q_ij);
 *   split-operator propagation of Eq. (10) with u_ij = v (n^alpha - n^0) (Eq. 11), both sets
 *   propagated; cleaning (Eq. 15) plus renormalisation every M steps; damped trapezoid
 *   integral of alpha^-1 u_ij (Eq. 13).
 * coeff: optional host n_s x n_occ matrix c[l][s]; NULL draws it from p->seed, p->coeff_dist.
 * w_out: optional host buffer n_pairs x n^3 doubles receiving W_ij; NULL keeps the results on
 *        the device only. Results are always kept on the device for sbse_build_A.
 * Requires sbse_set_orbitals. Errors: INVALID_ARG, NOT_READY, OOM, NUMERIC, DEVICE_TIMEOUT (a
 * bounded device-side wait of a bulk-copy, tensor-core or persistent kernel ran out; results are
 * not valid), CUDA. */
int sbse_apply_W(sbse_ctx *ctx, const sbse_tdh_params *p, int n_pairs, const int *pi,
                 const int *pj, const double *coeff, double *w_out);

/* Store externally computed screened potentials W_ij (for example from the learned surrogate) for
 * n_pairs pairs (pi[k] <= pj[k] < n_o), so that sbse_build_A uses them instead of running
 * sbse_apply_W for these pairs. w: host, n_pairs x n^3 doubles, copied.
 * Requires sbse_set_orbitals. Errors: INVALID_ARG, NOT_READY, NUMERIC, CUDA. */
int sbse_set_W(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, const double *w);

/* Copy W_ij of n_pairs pairs out of the context (host, n_pairs x n^3 doubles). Errors: INVALID_ARG,
 * NOT_READY (a pair has no W yet), CUDA. */
int sbse_get_W(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, double *w);

/* Assemble the Tamm-Dancoff matrix of Eq. (1), in FP64:
 *   A(ia, jb) = (eps_a - eps_i + Delta) delta_ij delta_ab + 2 (ia|jb) - (phi_a phi_b|W|phi_i phi_j)
 * with (ia|jb) = sum_r phi_i phi_a (r) [v phi_j phi_b](r) h^3 (exchange element after Eq. 1) and
 * (phi_a phi_b|W|phi_i phi_j) = sum_r phi_a phi_b (r) W_ij(r) h^3 (direct element), W_ji = W_ij.
 * Index ia = i * n_c + a. terms: bitwise OR of SBSE_EXCHANGE and SBSE_DIRECT (0 gives the
 * diagonal only). SBSE_DIRECT requires W for all n_o (n_o + 1) / 2 pairs; SBSE_DIRECT_PARTIAL
 * takes W = 0 for the pairs without one (screened-out pairs of a localized window, see
 * sbse_localize_occupied). After sbse_localize_occupied the diagonal term is
 * delta_ab (eps_a delta_ij - F_ij) + Delta delta_ij delta_ab with F the occupied block of H0 in the
 * rotated window.
 * a_out: optional host (n_o n_c)^2 doubles, row-major; NULL keeps A on the device.
 * Errors: INVALID_ARG, NOT_READY, OOM, CUDA. */
int sbse_build_A(sbse_ctx *ctx, unsigned terms, double *a_out);

/* The direct element split by pairs, for one system spread over several GPUs (each rank propagates a
 * block of pairs; the pairs are independent W applications): sbse_get_direct returns, for n_pairs
 * pairs (i, j) with W available, the columns D[ab][k] = sum_r phi_a phi_b (r) W_{i_k j_k}(r) h^3,
 * ab = a n_c + b (all n_c^2 products), as a host n_c^2 x n_pairs row-major array; sbse_set_direct
 * takes the n_c^2 x n_o (n_o + 1) / 2 array of every pair in the canonical order (the ranks'
 * columns gathered) and makes the next sbse_build_A with SBSE_DIRECT use it instead of W (until W
 * changes). Errors: INVALID_ARG, NOT_READY (W missing), NUMERIC, OOM, CUDA. */
int sbse_get_direct(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, double *dab);
int sbse_set_direct(sbse_ctx *ctx, const double *dab);

/* Lowest k eigenvalues of A (Eq. 1; the exciton energies, Ha), ascending, by an FP64
 * Householder tridiagonalisation and Sturm bisection on the device.
 * evals: host, k doubles. evecs: optional host (n_o n_c) x k doubles, row-major (component ia of
 * exciton j at evecs[ia * k + j]): orthonormal eigenvectors by inverse iteration on the
 * tridiagonal matrix (vectors of eigenvalues closer than 1e-3 |T| orthogonalised against each
 * other) and the Householder back-transformation, each with its largest-magnitude component
 * positive; NULL returns eigenvalues only. For degenerate excitons only the spanned subspace is
 * defined. Requires sbse_build_A. Errors: INVALID_ARG, NOT_READY, OOM, NUMERIC, CUDA. */
int sbse_spectrum(sbse_ctx *ctx, int k, double *evals, double *evecs);

/* Absorption spectrum from A by a Chebyshev expansion (Sec. II.C, electron-hole basis, the
 * paragraph after Eq. 18): sigma(omega) = omega <f0| G_s(A - omega) |f0>, the dipole correlation
 * with the delta function smoothed by a normalised Gaussian G_s of standard deviation
 * `broadening` (Ha) and the start vector f0_ia = <phi_a| x |phi_i> (x along `axis`: 0 = x, 1 = y,
 * 2 = z, measured from the box centre; index ia = i * n_c + a). A is scaled to
 * A~ = (A - c) / w from its Gershgorin bounds [lo, hi] (c = (lo + hi) / 2, w = 1.01 (hi - lo) / 2);
 * the residues R_n = <f0| T_n(A~) |f0>, n < n_terms, come from the Chebyshev recursion applied to
 * f0 on the device, and the Gaussian's Chebyshev coefficients from Chebyshev-Gauss quadrature on
 * n_terms nodes. All FP64. More terms resolve narrower broadenings: n_terms of several times
 * w / broadening.
 * omega: host, n_omega frequencies (Ha). sigma: host out, n_omega values. residues: optional host
 * out, n_terms values (NULL: not returned). Requires sbse_build_A.
 * Errors: INVALID_ARG (axis, n_terms outside [2, 65536], broadening <= 0, n_omega outside
 * [1, 2^24], NULL arrays), NOT_READY, OOM, NUMERIC (non-finite result), CUDA. */
int sbse_absorption(sbse_ctx *ctx, int axis, int n_terms, double broadening, int n_omega,
                    const double *omega, double *sigma, double *residues);

/* Finite-box correction W(k -> 0) (Sec. III, paragraph before the algorithm summary): the scissor
 * shift is lowered by W(k -> 0) = eps_eff^-1 v_bndry, with v_bndry the average Kohn-Sham potential
 * on the box boundary of a run and eps_eff^-1 fitted so that the spectra of runs in boxes of
 * several sizes overlap.
 * sbse_boundary_potential: v_bndry of the context's system, FP64 on the device. Reading: the model's
 * Kohn-Sham potential is V_loc - mean(V_loc) + v n0, n0 = 2 sum_{s <= N_occ} |phi_s|^2, v the
 * periodic Coulomb operator with G = 0 dropped; the boundary is the grid points with ix, iy or
 * iz = 0, averaged with equal weights. v_bndry: host out, Ha. Requires sbse_set_orbitals.
 * Errors: INVALID_ARG, NOT_READY, OOM, NUMERIC, CUDA. */
int sbse_boundary_potential(sbse_ctx *ctx, double *v_bndry);
/* sbse_fit_inverse_dielectric (host only, no context): E is n_box x k (row-major, box-major) lowest
 * excitons of the runs, v their v_bndry; returns in *eps_inv the least-squares s minimising
 * sum_{b,j} (E[b,j] - s v[b] - mean_b'(E[b',j] - s v[b']))^2. Errors: INVALID_ARG (n_box < 2, k < 1,
 * null arrays, all v equal); message from sbse_last_error(NULL). */
int sbse_fit_inverse_dielectric(int n_box, int k, const double *E, const double *v, double *eps_inv);
/* Localized occupied window (Forward perspective: localized occupied orbitals reduce the number of
 * (i, j) pairs whose W_ij is needed). sbse_localize_occupied rotates the n_o window orbitals,
 * phi'_k = sum_i U_ik phi_i with U orthogonal, to maximise the periodic localization functional
 * sum_{alpha = x,y,z} sum_k |Z'_alpha,kk|^2, Z_alpha,ij = sum_r phi_i phi_j exp(i 2 pi x_alpha / L) h^3
 * (Jacobi sweeps; at most max_sweeps, stopping when a sweep gains less than tol relative). The
 * context then works in the rotated window: W, A (with F = U^T diag(eps_o) U on its diagonal term)
 * and the spectra refer to it; W computed before is dropped. U_out: optional host n_o x n_o,
 * row-major (U_out[i n_o + k] = U_ik). Errors: INVALID_ARG, NOT_READY, OOM, CUDA.
 * sbse_pair_weights: w_p = (sum_r (phi_i phi_j)^2 h^3)^1/2 for the n_o (n_o + 1) / 2 window pairs in
 * the canonical order (0,0), (0,1), .., (1,1), ..: the norms by which pairs are screened before
 * sbse_apply_W. w_out: host out. Errors: INVALID_ARG, NOT_READY, OOM, CUDA. */
int sbse_localize_occupied(sbse_ctx *ctx, int max_sweeps, double tol, double *U_out);
int sbse_pair_weights(sbse_ctx *ctx, double *w_out);

/* Mixed hole-grid representation (Sec. II.C, "Mixed Representation Iterative Solution"): the BSE
 * operator A = Q A-bar on vectors f_j(r), one grid function per window state j (n_o x n^3, x
 * fastest, FP64), (A-bar f)_j = (H0 + Delta - eps_j) f_j + dv phi_j - sum_i f_i W_ij with
 * dv = v dn, dn = 2 sum_i phi_i f_i (the window's exciton density), W_ji = W_ij from sbse_apply_W.
 * projector: 0 = SBSE_Q_OCCUPIED, Q = 1 - sum_{s <= N_occ} |phi_s><phi_s| (the whole virtual space
 * of the grid); 1 = SBSE_Q_CONDUCTION, Q = sum_{c <= n_c} |phi_c><phi_c| (the electron-hole-basis
 * variant; A restricted to span{phi_c} is then the matrix of Eq. 1). All FP64 on the device in
 * either precision mode. Require W for every window pair and the canonical (not localized) window.
 * sbse_apply_A_mixed: f_out = A f_in (host arrays, n_o x n^3 each).
 * sbse_mixed_bounds: an interval [lo, hi] enclosing the spectrum of A on the range of Q: the
 *   extreme Ritz values of n_lanczos Lanczos steps from f0_j = Q x phi_j (x along `axis` from the box
 *   centre; each vector projected by Q), widened by 5 % of their spread on each side.
 * sbse_absorption_mixed: sigma(omega) = omega <f0| delta(A - omega) |f0> with f0_j = Q x phi_j, from
 *   n_terms residues R_n = <f0| T_n(A~) |f0>, A~ f = Q(A-bar f - c f) / w, c = (lo + hi) / 2,
 *   w = (hi - lo) / 2 for the interval [lo, hi] the caller gives (it must enclose the spectrum), and
 *   the Gaussian-smoothed delta of sbse_absorption (Chebyshev-Gauss quadrature on n_terms nodes).
 *   sigma: host n_omega; residues: optional host n_terms.
 * Errors: INVALID_ARG, NOT_READY (orbitals or some W missing), UNSUPPORTED (localized window), OOM,
 * NUMERIC, CUDA. */
#define SBSE_Q_OCCUPIED 0
#define SBSE_Q_CONDUCTION 1
int sbse_apply_A_mixed(sbse_ctx *ctx, int projector, const double *f_in, double *f_out);
int sbse_mixed_bounds(sbse_ctx *ctx, int projector, int axis, int n_lanczos, double *lo, double *hi);
int sbse_absorption_mixed(sbse_ctx *ctx, int projector, int axis, int n_terms, double lo, double hi,
                          double broadening, int n_omega, const double *omega, double *sigma, double *residues);

/* Replace the scissor shift Delta of Eq. (9) (e.g. by Delta - eps_eff^-1 v_bndry) without touching
 * orbitals or W; A must be built again. Errors: INVALID_ARG, NOT_READY, NUMERIC. */
int sbse_set_scissor(sbse_ctx *ctx, double scissor);

/* Allocation-free variant of sbse_spectrum, for callers that cannot allocate device memory (for
 * example a host framework whose memory pool has reserved the whole GPU, or code that must not
 * trigger an allocation once it runs). The paper has no counterpart: it is an interface addition.
 * It computes the lowest k eigenvalues of the real symmetric n x n matrix at a_dev (device pointer,
 * FP64, row-major, not modified) into evals_dev (device pointer, k doubles, ascending) with the
 * same kernels as sbse_spectrum, on `stream` (a cudaStream_t; NULL = default stream), and
 * returns after the stream has synchronised. It calls no cudaMalloc, cudaFree or allocating
 * library routine: its scratch (n^2 + 2n doubles) is a fixed device array of
 * SBSE_NOALLOC_MAX_N^2 + 2 SBSE_NOALLOC_MAX_N doubles (about 2 MB) that every GPU loading the
 * library holds until the process exits. Each call looks up that array's device address on the
 * current device (cudaGetSymbolAddress). The array is reserved when the library's device code is
 * loaded on a device, which under CUDA's default lazy loading is the first call there: a caller
 * whose memory pool will take the whole GPU should make one call (or set
 * CUDA_MODULE_LOADING=EAGER) before the pool reserves it, else that first call can fail with CUDA.
 * Every call synchronises `stream` before it returns, so it must not be called on a stream that is
 * being captured into a graph (the synchronisation would end the capture). All calls on a device
 * share the array, so calls that overlap on the GPU race; the
 * array keeps the last call's contents, and nothing in it needs to start at zero.
 * Errors: INVALID_ARG (null pointer, k outside 1..n), SHAPE (n > SBSE_NOALLOC_MAX_N), CUDA;
 * the message is available from sbse_last_error(NULL). */
#define SBSE_NOALLOC_MAX_N 512
int sbse_spectrum_noalloc(const double *a_dev, int n, int k, double *evals_dev, void *stream);

/* Message of the last failed call on ctx ("" if none). The pointer stays valid until the next
 * call on ctx. ctx may be NULL: message of the last failed context-free call on this thread
 * (sbse_create, sbse_spectrum_noalloc). */
const char *sbse_last_error(const sbse_ctx *ctx);

/* The CUDA stream (cudaStream_t) all device work of ctx is issued on, for event timing by the
 * caller. Errors: INVALID_ARG. */
int sbse_get_stream(const sbse_ctx *ctx, void **stream);

/* Options. SBSE_OPT_TENSOR_CORES (default 1): in SBSE_MIXED, run the grid-sum contractions of
 * sbse_build_A on the tensor cores (tcgen05, BF16 high/low split of both operands, three products
 * per term, FP32 accumulation); 0 uses FP32 CUDA-core arithmetic. Errors: INVALID_ARG. */
#define SBSE_OPT_TENSOR_CORES 1
/* SBSE_OPT_CHUNK_MB (default 0): sbse_apply_W advances the pairs in chunks holding about this many
 * MiB of propagated orbitals, so that the three passes of a split-operator step find a chunk in the
 * L2 cache; 0 advances all pairs at once (fastest as separate launches: small launches leave
 * SMs idle). Results do not depend on it. */
#define SBSE_OPT_CHUNK_MB 2
/* SBSE_OPT_PERSISTENT (default 0): advance the eta0 set and all pairs by one split-operator step in
 * a single persistent kernel whose blocks pull tiles from a dependency-ordered queue (grids with a
 * register-pencil FFT); 0 uses three separate pass kernels, which are faster on GB300 (the merged
 * kernel is register-limited to fewer resident warps). Results do not depend on it. */
#define SBSE_OPT_PERSISTENT 3
/* SBSE_OPT_TMA_PLANES (default 1): in SBSE_MIXED on grids of 32, 40, 48 or 64 points per axis, the
 * inverse plane pass of the pair batch (with the induced density of Eq. 11) and the z-column passes
 * run as persistent kernels fed by bulk asynchronous copies (TMA) of their next planes or column
 * slabs; 0 uses the plain pass kernels. Results do not depend on it. */
#define SBSE_OPT_TMA_PLANES 4
/* SBSE_OPT_GRAPH (default 1): sbse_apply_W captures its time loop (all launches of all steps, on
 * the context's two streams) into a CUDA graph and replays it on later calls whose buffers, sizes,
 * parameters and options are unchanged, removing the host launch cost per step (which dominates
 * on small grids). Not used while sbse_profile is enabled. Results do not depend on it. */
#define SBSE_OPT_GRAPH 5
/* SBSE_OPT_MEM_LIMIT_MB (default 0 = none): device memory, in MiB, that the context may hold in
 * total (grid tables, orbitals, results and scratch). An allocation that would exceed it fails with
 * SBSE_ERR_OOM and leaves the context as it was before the failing call. */
#define SBSE_OPT_MEM_LIMIT_MB 6
/* SBSE_OPT_WAIT_LIMIT (default 0 = 2^23 polls, about a second): iteration limit of the bounded waits
 * with which the persistent step kernel (SBSE_OPT_PERSISTENT) waits for the tiles it depends on.
 * A wait that runs out skips its tile's work, the kernel still ends, and sbse_apply_W returns
 * SBSE_ERR_DEVICE_TIMEOUT with the context still usable. */
#define SBSE_OPT_WAIT_LIMIT 7
int sbse_set_option(sbse_ctx *ctx, int option, int value);

/* Number of CUDA kernel launches the library has issued in this process (all contexts), for
 * counting the kernels inside a timed region. Errors: INVALID_ARG. */
int sbse_kernel_launches(long long *count);

/* Per-phase device timing. When enabled, CUDA events bracket each phase launch group inside
 * sbse_apply_W and sbse_build_A; sbse_phase_time reports the summed device milliseconds and the
 * number of launches of one phase since the last reset (enable resets the counters).
 * phase: 0 = orbital propagation step (phase + 3D FFT + kinetic + inverse FFT + induced density),
 *        1 = Poisson solve and time-integral accumulation, 2 = cleaning, 3 = contractions (K, D),
 *        4 = A assembly + eigensolve; inside phase 0, the three passes over the pair batch on
 *        grids with the register-pencil FFT: 5 = forward plane pass (potential phase + x, y FFTs),
 *        6 = z-column pass (z FFT, kinetic phase, inverse z FFT), 7 = inverse plane pass (+ density).
 *        Errors: INVALID_ARG, CUDA. */
int sbse_profile(sbse_ctx *ctx, int enable);
int sbse_phase_time(sbse_ctx *ctx, int phase, double *ms, long long *launches);

/* ---- learned surrogate (not in the paper; the workload's learned form) ----------------------
 * A Fourier neural operator mapping (rho_ij, V_loc) on an n^3 grid to W^pol_ij: lift 2 -> width
 * channels, `layers` Fourier layers U = K(V) + W V + b with K(V) = irfftn(R . rfftn(V)) on the kept
 * modes kx < modes, ky, kz in [0, modes) U [n - modes, n), V' = GELU(U) except after the last layer,
 * then a linear projection to one channel. Spectral and pointwise weights are used in BF16, sums in
 * FP32; FP32 master weights and Adam moments are kept on the device.
 * Parameter vector (FP32, sbse_fno_num_params entries): lift W [width][2], lift b [width], then per
 * layer spectral R [2 modes][2 modes][modes][width][width] complex (re, im interleaved), pointwise
 * W [width][width] (W[co][ci]), b [width]; then projection w [width], b [1].
 * Tensors are DEVICE pointers, FP32: x [batch][2][n^3] (channel 0 = rho, 1 = V_loc), y and targets
 * [batch][n^3]. Calls are synchronous. Errors: INVALID_ARG, OOM, CUDA. */
typedef struct sbse_fno sbse_fno;
int sbse_fno_create(sbse_fno **out, int device, int n, int width, int modes, int layers, int max_batch);
void sbse_fno_destroy(sbse_fno *fno);
const char *sbse_fno_last_error(const sbse_fno *fno);
long long sbse_fno_num_params(const sbse_fno *fno);
/* copy the FP32 parameter vector in (resets the Adam state) / out (params and/or last gradients) */
int sbse_fno_set_params(sbse_fno *fno, const float *host);
int sbse_fno_get_params(sbse_fno *fno, float *host, float *grad_host);
int sbse_fno_forward(sbse_fno *fno, int batch, const float *x_dev, float *y_dev);
/* forward, then backward from dL/dy = dy_dev: gradients available through sbse_fno_get_params */
int sbse_fno_gradients(sbse_fno *fno, int batch, const float *x_dev, const float *dy_dev);
/* one Adam step (b1 0.9, b2 0.999, eps 1e-8) on the loss 0.5 mean((y - t)^2); *loss receives it */
int sbse_fno_train_step(sbse_fno *fno, int batch, const float *x_dev, const float *t_dev, float lr,
                        double *loss);
/* Surrogate inputs of pairs (i, j) of ctx's valence window, written to x_dev [n_pairs][2][n^3]:
 * channel 0 = phi_i phi_j / s_rho, channel 1 = V_loc / s_v. Errors: INVALID_ARG, NOT_READY, CUDA. */
int sbse_fno_pair_inputs(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, double s_rho, double s_v,
                         float *x_dev);
/* Surrogate screened potentials: W_ij = s_w * FNO(phi_i phi_j / s_rho, V_loc / s_v) for n_pairs pairs,
 * stored in ctx as if computed by sbse_apply_W (the grid of fno must equal ctx's). Errors:
 * INVALID_ARG, NOT_READY, SHAPE, OOM, CUDA. */
int sbse_surrogate_W(sbse_ctx *ctx, sbse_fno *fno, int n_pairs, const int *pi, const int *pj, double s_rho,
                     double s_v, double s_w);

/* Debug bounds checks (race detection and sanitizers are not available on the target; see the
 * debug build, SBSE_DEBUG_BOUNDS=1 in paper_2205_06690_gb300/build.py, libsbse_dbg.so). In that
 * build the kernels of the hot path check their global-memory indices; an out-of-range access is
 * recorded (first one per translation unit) and redirected to element 0 of its array instead of
 * faulting. *enabled = 1 in the debug build, 0 otherwise; *first_fault = 0 if nothing was recorded
 * since the last call, else (site << 40) | (index & (2^40 - 1)) of the first record, site =
 * translation unit * 100000 + source line. Reading clears the records. Host-synchronous.
 * Returns OK (no record), NUMERIC (records found), CUDA. */
int sbse_debug_bounds(int *enabled, unsigned long long *first_fault);

/* Checkpoint / resume of a propagation (not in the paper: long runs and restarts).
 * sbse_apply_W_range runs the time steps [n_begin, n_end) of the propagation sbse_apply_W would run
 * for these parameters and pairs (0 <= n_begin < n_end <= p->n_steps): n_begin = 0 starts it
 * (stochastic orbitals of Eq. 14 and the kick); n_begin > 0 continues the state this context holds,
 * which a range ending at n_begin with the same parameters and pairs left (or sbse_load_state
 * loaded); n_end = p->n_steps ends it and stores the pairs' W as sbse_apply_W does (w_out as there;
 * before that W is not touched and w_out is ignored). Calls in the same context between the range
 * calls may discard the state (they share its device memory): a later continuation then returns
 * NOT_READY. The continued run gives the same W as one sbse_apply_W call, to the bit in both
 * precision modes (the partial FP32 time integral is part of the state).
 * sbse_state_bytes / sbse_save_state copy the held state (the difference orbitals d, eta0 of the next
 * step, the FP64 and partial FP32 time integrals, E - 1 of the pending half step, the orbitals'
 * norms, and the parameters, pairs and next step) into a HOST buffer of at least that many bytes;
 * sbse_load_state puts such a buffer into a context of the same grid, orbitals and precision (for
 * example a new process) for the next sbse_apply_W_range call.
 * Errors: INVALID_ARG (range, buffer), NOT_READY (no such state), SHAPE (other grid or precision),
 * NUMERIC, OOM, CUDA, DEVICE_TIMEOUT. */
int sbse_apply_W_range(sbse_ctx *ctx, const sbse_tdh_params *p, int n_pairs, const int *pi, const int *pj,
                       const double *coeff, double *w_out, int n_begin, int n_end);
int sbse_state_bytes(sbse_ctx *ctx, size_t *bytes);
int sbse_save_state(sbse_ctx *ctx, void *host, size_t bytes);
int sbse_load_state(sbse_ctx *ctx, const void *host, size_t bytes);

/* Bare potentials q_ij = v (phi_i phi_j) (FP64 Poisson, the first term of W_ij = q_ij + W^pol_ij,
 * Sec. II.B) stored as the W of the given pairs of the valence window, as a starting point for a
 * polarisation part added by sbse_add_W. Errors: INVALID_ARG (indices, duplicates), NOT_READY, OOM,
 * CUDA. */
int sbse_bare_W(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj);
/* W_ij += scale * y_k for the k-th pair (i, j): y_dev is a DEVICE array [n_pairs][n^3] of FP32 fields
 * on ctx's grid (for example the surrogate's W^pol). The pairs' W must be available (sbse_bare_W or
 * sbse_apply_W). Errors: INVALID_ARG, NOT_READY, CUDA. */
int sbse_add_W(sbse_ctx *ctx, int n_pairs, const int *pi, const int *pj, const float *y_dev, double scale);
/* Periodic trilinear resampling of `count` FP32 fields (DEVICE arrays, [count][n^3], x fastest) from an
 * n_src^3 grid onto an n_dst^3 grid of the same box (point i of the new grid at i n_src / n_dst old
 * grid units), on ctx's stream; src and dst must not overlap. Connects the surrogate's grid to a
 * system's grid. Errors: INVALID_ARG, CUDA. */
int sbse_resample(sbse_ctx *ctx, int count, int n_src, const float *src_dev, int n_dst, float *dst_dev);

#ifdef __cplusplus
}
#endif

#endif /* SBSE_H */
