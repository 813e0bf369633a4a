/*
 * gw.h -- C ABI of the GB300 periodic G0W0 hot path (localized RI, imaginary axis).
 *
 * The operations follow Ren et al., "All-electron periodic G0W0 implementation
 * with numerical atomic orbital basis functions" (arXiv:2011.01400):
 *   gw_chi0   -- Eqs. (AO_triple_split2), (AO_MO_transform), (chi0_matrix):
 *                LRI triple coefficients -> band-pair coefficients M -> chi0(q, i w)
 *   gw_screen -- Eqs. (symm_dielec_func), (screened_W_matr); Gamma point per
 *                Eq. (dielectric_func_gamma): eps~ = 1 - V^1/2 chi0 V^1/2,
 *                W^c = V^1/2 (eps~^{-1} - 1) V^1/2
 *   gw_sigma  -- Eq. (GW_selfe_element) with W^c: Sigma_c_n(k, i w), one q term
 *   gw_qp     -- continuation of Sigma_c to the real axis (Sec. II.A) and the
 *                quasiparticle equation; indirect gap
 *
 * Conventions (all calls):
 *   - Atomic units (Hartree, bohr). Complex numbers are gw_complex {re, im}
 *     (layout of C99 double _Complex, numpy complex128, cuDoubleComplex).
 *   - Mesh: Gamma-centred, k index = (i1*n2 + i2)*n3 + i3, fractional
 *     coordinate (i1/n1, i2/n2, i3/n3); the q mesh equals the k mesh.
 *   - "device" pointers are CUDA device memory owned by the caller; the
 *     library only reads inputs and writes the outputs named per call.
 *     "host" pointers are ordinary CPU memory.
 *   - Every call is ordered on the plan's stream and returns a gw_status; none
 *     aborts or throws. A failed call leaves the plan in an error state that
 *     sticks until gw_plan_destroy (later calls return GW_ERR_STATE).
 *     gw_last_error() returns a text for the last failure of this thread.
 *   - Matrices are row-major. Hermitian outputs are written in full.
 *   - No call uses more than the one current CUDA device.
 *   - Environment (read at gw_plan_create, split precision only):
 *     GW_CHI0_SEG_ROWS      pair rows per FP64 promotion segment of the tensor-core
 *                           chi0 (default 8192; at least 32);
 *     GW_CHI0_COMPRESS_TOL  per-frequency residual bound of the chi0 weight-matrix
 *                           compression (default 3e-8; 0 keeps all frequencies).
 *   - Environment (read at gw_plan_create, all precisions):
 *     GW_WORKSPACE_LIMIT    bytes of device memory one plan may allocate for its workspace
 *                           (default: no limit). An allocation that would pass it fails with
 *                           GW_ERR_NOMEM before cudaMalloc is called.
 *   - Autotuning: the first split-precision call that generates band-pair rows
 *     of a given shape in this process times two thread mappings of that kernel
 *     (one warm-up and one timed launch each). It then waits for the plan's stream
 *     once, to read the timings. Both mappings write identical rows, so the
 *     results never depend on the choice, and later calls of that shape do not wait.
 */
#ifndef GW_H
#define GW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GW_OK = 0,
  GW_ERR_ARG = 1,        /* invalid argument or size; nothing was launched           */
  GW_ERR_NOMEM = 2,      /* device workspace allocation failed                       */
  GW_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed               */
  GW_ERR_NOT_PD = 4,     /* eps~ had a non-positive Cholesky pivot (chi0 not NSD)    */
  GW_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up (pipeline stalled)     */
  GW_ERR_STATE = 6,      /* call out of order (e.g. gw_screen before gw_chi0 for q)  */
  GW_ERR_UNSUPPORTED = 7 /* valid request that the library does not implement          */
} gw_status;

typedef enum {
  GW_FP64 = 0,    /* plain method: every contraction in FP64 on CUDA cores          */
  GW_3XTF32 = 1,  /* contractions as 3 TF32 split products on tcgen05, FP32 accum.   */
  GW_3XBF16 = 2,  /* contractions as BF16 split products on tcgen05 (chi0: 3 pieces, 6
                     products; Sigma_c: 2 pieces, 3 products), FP32 accumulation          */
  GW_3XFP16 = 3   /* chi0 as 3 FP16 split products (2 pieces, power-of-two scaled) on
                     tcgen05, FP32 accumulation; the other contractions as GW_3XBF16     */
} gw_precision;

typedef struct { double re, im; } gw_complex;

typedef struct gw_plan_s* gw_plan;

/* The problem, Sec. II of the paper. Sizes:
 *   N_k = nk[0]*nk[1]*nk[2];  n_b(A), n_aux(A) = basis / ABF functions on atom A. */
typedef struct {
  int32_t nk[3];                 /* k mesh (= q mesh), each >= 1                            */
  int32_t n_atoms, n_basis, n_bands, n_occ, n_aux;
  const int32_t* basis_atom;     /* host [n_basis]: atom of each NAO, non-decreasing        */
  const int32_t* aux_atom;       /* host [n_aux]:   atom of each ABF, non-decreasing        */
  int32_t n_R;                   /* number of lattice vectors with stored LRI coefficients */
  const int32_t* R;              /* host [n_R][3] lattice vectors in lattice coordinates    */
  const double* eps;             /* device [N_k][n_bands] KS energies, ascending per k      */
  const gw_complex* evec;        /* device [N_k][n_basis][n_bands] KS eigenvectors c_{i,n}(k) */
  const double* ctil_R;          /* device: atoms concatenated in order; atom A block is
                                    [n_R][n_aux(A)][n_b(A)][n_basis] = C~_{i(0),j(R)}^{mu(0)},
                                    mu and i on A, j any (Eq. two_center_coeff_determination) */
  const gw_complex* V;           /* device [N_k][n_aux][n_aux] Coulomb matrix V(q), Hermitian
                                    positive definite (the truncated V^cut at q = 0)          */
  const gw_complex* pmom;        /* device [N_k][3][n_bands][n_bands] momentum matrix p_mn(k);
                                    may be NULL when head_wings == 0                          */
  double omega_cell;             /* unit-cell volume (bohr^3), > 0 when head_wings != 0      */
  double qhat[3];                /* direction of q -> 0 for the head and wings: a unit vector
                                    (|qhat|^2 = 1 within 1e-9, checked when head_wings == 1) */
  int32_t head_wings;            /* 1: Gamma point by Eq. dielectric_func_gamma along qhat;
                                    2: the same with eps~^-1 - 1 averaged over the direction
                                    of q -> 0 (128-point product rule on the sphere: 8 Gauss-
                                    Legendre nodes in cos(theta) x 16 equally spaced phi,
                                    offset by half a step; qhat unused); 0: regular formula */
  int32_t n_freq;                /* imaginary frequencies, 1..256                            */
  double omega0;                 /* scale of the default grid (freq NULL): modified Gauss-
                                    Legendre w_j = omega0 (1+x_j)/(1-x_j), g_j = 2 omega0 v_j /
                                    (1-x_j)^2 (x_j, v_j Gauss-Legendre on (-1, 1)); Ha, > 0     */
  int32_t sigma_lo, sigma_hi;    /* self-energy bands [sigma_lo, sigma_hi), 0-based          */
  double spin;                   /* spin factor in chi0 (2 for doubly occupied bands)        */
  double mu;                     /* chemical potential (finite); NaN selects midgap          */
  gw_precision prec;
  int32_t time_reversal;         /* 1: the inputs are time-reversal symmetric (real NAOs and
                                    ABFs, no magnetism): eps(-k) = eps(k), c(-k) = conj(c(k))
                                    up to a phase per band, V(-q) = conj(V(q)), p(-k) =
                                    -conj(p(k)). Then chi0(-q) = conj(chi0(q)) and W^c(-q) =
                                    conj(W^c(q)), and gw_g0w0 / gw_g0w0_qset compute chi0, eps~
                                    and W^c for one q of each pair (q, -q) of their q list, the
                                    Sigma_c term of -q from the conjugate W^c. gw_plan_create
                                    checks eps and V (GW_ERR_ARG beyond rounding). 0: no
                                    symmetry assumed.                                          */
  double k_offset[3];            /* shift of the k mesh in fractional coordinates, each in
                                    [-1, 1]: the k points are k0 + (i1/n1, i2/n2, i3/n3), and
                                    eps, evec and pmom are given at those points (same index
                                    order); the q mesh is never shifted, so k + q and k - q stay
                                    on the shifted mesh. All zero: the Gamma-centred mesh. A
                                    shifted plan gives Sigma_c at off-mesh k (its point 0 is k0)
                                    through gw_sigma_ext with the W^c of an unshifted plan.    */
  const double* freq;            /* host [n_freq]: the caller's imaginary frequencies w_j > 0
                                    (Ha, distinct), the grid of chi0 / eps~ / W^c and of the
                                    Sigma_c output; NULL: the default grid above (copied)      */
  const double* freq_w;          /* host [n_freq]: their weights g_j > 0 for the folded w'
                                    integral over (0, inf) of Eq. GW_selfe_element; NULL with
                                    freq NULL (both or neither)                                */
} gw_problem;

/* sizeof(gw_problem) as compiled into the library (a binding checks its own layout against it). */
size_t gw_problem_bytes(void);

/* Build a plan: validates `prob`, copies the host arrays, allocates the
 * library's own workspace, and on `stream` precomputes the half-transformed
 * LRI coefficients (Eqs. expan_coeff_FT1/2 contracted with c(k)), V(q)^{1/2}
 * for every q and the Coulomb eigenvector lambda = 1 at q = 0.
 * `stream` is a cudaStream_t (NULL = legacy default).
 * n_sys > 1 (batch of independent systems, sizes free per system): `prob` points to an array of
 * n_sys problems; the plan holds one plan per system, each on a stream of its own created by the
 * library (all of them resident at once). The per-system calls (gw_chi0, gw_screen, gw_sigma,
 * gw_g0w0, gw_qp, gw_qp_static, gw_surrogate_modes, gw_surrogate_data) take `sys` in [0, n_sys);
 * on a batch plan each such call starts after the work queued on `stream` and returns after its
 * own work. gw_plan_freq / gw_plan_mu / gw_plan_chi0_terms / gw_plan_last_chi0_stats report
 * system 0; gw_surrogate_enable is not available on a batch plan. n_sys in [1, 4096].
 * On success *out owns the workspace until gw_plan_destroy.
 * Errors: GW_ERR_ARG (bad sizes/pointers; for a batch the message names the system),
 * GW_ERR_NOMEM, GW_ERR_CUDA. */
gw_status gw_plan_create(const gw_problem* prob, int32_t n_sys, void* stream, gw_plan* out);

/* Release the plan and its workspace (waits for the plan's stream). NULL is a no-op. */
gw_status gw_plan_destroy(gw_plan plan);

/* chi0_{mu nu}(q, i w_j) for all j (Eq. chi0_matrix, Hermitised, occupations restored):
 *   chi0 = -(s/N_k) sum_k sum_{i occ, a unocc} M^mu_{ai}(k,q) M^nu_{ai}(k,q)^* 2D/(w^2+D^2),
 *   D = eps_a(k+q) - eps_i(k), M from the LRI coefficients (Eqs. AO_triple_split2, AO_MO_transform).
 * chi0_out: device [n_freq][n_aux][n_aux] or NULL (kept only inside the plan).
 * Errors: GW_ERR_ARG (sys, q out of range), GW_ERR_CUDA, GW_ERR_TIMEOUT. */
gw_status gw_chi0(gw_plan plan, int32_t sys, int32_t q, gw_complex* chi0_out);

/* W^c(q, i w_j) = V^1/2 (eps~^{-1} - 1) V^1/2, eps~ = 1 - V^1/2 chi0 V^1/2 (Eqs. symm_dielec_func,
 * screened_W_matr); at q = 0 with head_wings, eps~ is assembled in the Coulomb eigenbasis
 * with the head and wings of Eq. dielectric_func_gamma (insulator: f' term dropped).
 * Uses the chi0 of the last gw_chi0 call, which must be for the same q (else GW_ERR_STATE).
 * wc_out: device [n_freq][n_aux][n_aux] or NULL. eps~ is factorised and inverted in FP64.
 * Errors: GW_ERR_STATE, GW_ERR_NOT_PD, GW_ERR_CUDA. */
gw_status gw_screen(gw_plan plan, int32_t sys, int32_t q, gw_complex* wc_out);

/* Adds the q term of Eq. (GW_selfe_element) with W^c in place of W:
 *   Sigma_c_n(k, i w) += -(1/(2 pi N_q)) sum_m sum_j g_j S_nm(k,q,w'_j) 2z/(z^2 + w'_j^2),
 *   S_nm = sum_{mu nu} C^mu_{nm}(k,k-q) W^c_{mu nu}(q, i w'_j) C^nu_{mn}(k-q,k),
 *   z = i w + mu - eps_m(k-q), n in [sigma_lo, sigma_hi), m over all bands.
 * Uses the W^c of the last gw_screen call, which must be for the same q (else GW_ERR_STATE).
 * sigma_acc: device [N_k][sigma_hi-sigma_lo][n_freq], accumulated into (caller zeroes it),
 *            or NULL to accumulate into the plan's own buffer (zeroed at plan creation). */
gw_status gw_sigma(gw_plan plan, int32_t sys, int32_t q, gw_complex* sigma_acc);

/* The q term of Sigma_c (as gw_sigma) with a caller-supplied W^c(q) (device [n_freq][n_aux][n_aux],
 * Hermitian, same grid), for the target k in [k_lo, k_hi) only. On a plan whose k mesh is shifted
 * (gw_problem.k_offset = k0), with the W^c of an unshifted plan of the same system, the sum over
 * q gives Sigma_c at the off-mesh points k0 + mesh (point 0 is k0 itself): band energies along
 * lines through the Brillouin zone. sigma_acc: device [N_k][n_sigma][n_freq] (rows outside the
 * k range untouched) or NULL for the plan's own accumulator.
 * Errors: GW_ERR_ARG (q, k range, NULL wc), GW_ERR_CUDA. */
gw_status gw_sigma_ext(gw_plan plan, int32_t sys, int32_t q, const gw_complex* wc, int32_t k_lo, int32_t k_hi,
                       gw_complex* sigma_acc);

/* Exchange self-energy, the bare-Coulomb part of Eq. (GW_selfe_element) (W = V + W^c): the
 * frequency integral of V G leaves the occupied bands,
 *   Sigma_x_n(k) = -(1/N_q) sum_q sum_{m occ} sum_{mu nu} C^mu_{nm}(k,k-q) V_{mu nu}(q) C^nu_{mn}(k-q,k),
 * n in [sigma_lo, sigma_hi), V(0) the (truncated) Coulomb matrix as given.
 * sigx: device [N_k][n_sigma] FP64 output (overwritten). The products run in FP64 on the FP64
 * path and in FP32 on the split paths. For the QP equation, pass dxv = Sigma_x - v_xc to gw_qp.
 * Errors: GW_ERR_ARG, GW_ERR_NOMEM, GW_ERR_CUDA. */
gw_status gw_sigma_x(gw_plan plan, int32_t sys, double* sigx);

/* The whole q loop of the G0W0 pass in one call: for every q on the mesh, chi0 (as gw_chi0),
 * eps~ and W^c (as gw_screen) and the Sigma_c term (as gw_sigma), accumulated into sigma_acc
 * (device [N_k][n_sigma][n_freq], caller zeroes it) or, if NULL, the plan's own accumulator.
 * q points are processed in groups whose FP64 factorisations of eps~ run as one batched launch;
 * the group buffers (about 8 GB at most) are allocated on the first call and kept by the plan.
 * Results equal those of the per-q calls. Errors: as gw_chi0 / gw_screen / gw_sigma. */
gw_status gw_g0w0(gw_plan plan, int32_t sys, gw_complex* sigma_acc);

/* gw_g0w0 over the listed q points only (q_list: host [n_q], distinct, in [0, N_k)): their chi0,
 * eps~, W^c and Sigma_c terms, accumulated into sigma_acc (device [N_k][n_sigma][n_freq]; the
 * caller zeroes it). The q terms are independent, so disjoint lists that cover the mesh, run
 * on several devices (one plan each) and summed, give gw_g0w0's Sigma_c: the q-parallel form of
 * the pass, whose only exchange is that sum. Not available with a surrogate attached.
 * Errors: GW_ERR_ARG (NULL, out-of-range or repeated q), GW_ERR_UNSUPPORTED, as gw_g0w0. */
gw_status gw_g0w0_qset(gw_plan plan, int32_t sys, const int32_t* q_list, int32_t n_q, gw_complex* sigma_acc);

/* gw_g0w0 for every system of a batch plan: the systems' q loops run concurrently, each on its
 * own stream, driven by n_threads host threads (0: min(n_sys, 8)), so that small systems
 * together fill the GPU. sigma_accs: host array of n_sys device accumulators
 * ([N_k][n_sigma][n_freq] of each system, zeroed by the caller; an entry may be NULL for the
 * plan's own accumulator), or NULL for all own accumulators. Returns after all systems are done.
 * On a single-system plan it is gw_g0w0(plan, 0, sigma_accs[0]).
 * Errors: the first failing system's status, its message prefixed with "system i". */
gw_status gw_g0w0_batch(gw_plan plan, gw_complex* const* sigma_accs, int32_t n_threads);

/* Number of systems of a plan (host scalar). */
gw_status gw_plan_n_sys(gw_plan plan, int32_t* n_sys);

/* Quasiparticle energies: Sigma_c(i w) continued with the two-pole model
 * (p1 z + p0)/(z^2 + q1 z + q0) fitted by linear least squares on all n_freq points,
 * then E = eps_n + Re Sigma_c(E - mu) + dxv_n by Newton (tolerance 1e-10 Ha; linearised
 * fallback flagged by a negative converged count). All in FP64 on the device.
 * sigma:  device [N_k][n_sigma][n_freq], or NULL for the plan's own accumulator.
 * dxv:    device [N_k][n_sigma] (Sigma_x - v_xc) or NULL for zero.
 * e_qp:   host [N_k][n_sigma] output.
 * gap:    host scalar output, min_k E_LUMO - max_k E_HOMO when both are in the window, else NaN.
 * n_conv: host scalar output (may be NULL): number of (k, n) whose Newton iteration converged. */
gw_status gw_qp(gw_plan plan, int32_t sys, const gw_complex* sigma, const double* dxv,
                double* e_qp, double* gap, int32_t* n_conv);

/* Capacity of the fixed device scratch of gw_qp_static, in (k, n) pairs (12 bytes each). */
#define GW_QP_STATIC_MAX 16384

/* gw_qp without any device allocation (the paper has no counterpart: a deployment variant).
 * Same arguments, arithmetic and results as gw_qp; the per-(k, n) QP energies and Newton flags
 * live in one fixed file-scope device array of GW_QP_STATIC_MAX pairs instead of a
 * cudaMalloc/cudaFree pair per call. For callers that cannot allocate device memory when
 * they solve the QP equation: a process whose device memory is held by a caching allocator,
 * or a serving loop that must not take the device-wide synchronisation of cudaFree.
 * The plan itself still owns the workspace gw_plan_create allocated.
 * - N_k * (sigma_hi - sigma_lo) > GW_QP_STATIC_MAX: GW_ERR_ARG, nothing launched (use gw_qp).
 * - The current CUDA device must be the plan's device (the one current at gw_plan_create):
 *   the scratch address is per device. Otherwise GW_ERR_STATE, nothing launched.
 * - The first call on a device looks up the scratch address with cudaGetSymbolAddress (this
 *   may load the library's device code) and caches it for the life of the process.
 * - The call is synchronous: it reads the energies back to the host and waits for the plan's
 *   stream, so it cannot be called while that stream is being captured.
 * - Nothing in the scratch has to start at zero: every call writes each element it reads.
 * - One scratch array per device: calls that overlap in time on the same device (from any
 *   thread, stream or plan) race on it. Serialise them.
 * Errors: as gw_qp, plus GW_ERR_STATE (wrong current device) and GW_ERR_CUDA if the address
 * lookup fails. */
gw_status gw_qp_static(gw_plan plan, int32_t sys, const gw_complex* sigma, const double* dxv,
                       double* e_qp, double* gap, int32_t* n_conv);

/* Host copies of the plan's frequency grid (w_j and quadrature weights g_j), [n_freq] each. */
gw_status gw_plan_freq(gw_plan plan, double* freq, double* weight);

/* Chemical potential the plan uses (host scalar). */
gw_status gw_plan_mu(gw_plan plan, double* mu);

/* Device time of the last chi0 contraction launch (ms, CUDA events on the plan's stream),
 * and its algorithmic flop count (8 per complex multiply-add, Hermitian lower triangle). */
gw_status gw_plan_last_chi0_stats(gw_plan plan, double* ms, double* flops);

/* Weight rows the split-precision chi0 contraction used for the last q. The frequency
 * compression writes the Lorentzian weight matrix W [n_freq][pairs] as E V with T <= n_freq rows
 * in V, T the smallest count for which every frequency's row keeps a relative residual
 * |W_j - (E V)_j| / |W_j| <= 3e-8 (FP64 over all pairs); chi0(w_j) = sum_t E_jt C_t.
 * 0 before the first split-precision chi0; compression is off on the FP64 path and for
 * n_freq < 4 or > 64. */
gw_status gw_plan_chi0_terms(gw_plan plan, int32_t* terms);

/* Number of CUDA kernels this library has launched in the calling process so far (host-side count). */
gw_status gw_kernel_launches(uint64_t* count);

/* Number of device allocations (cudaMalloc calls) this library has made in the calling process
 * so far (host-side count; failed attempts included). */
gw_status gw_device_allocations(uint64_t* count);

/* ------------------------------------------------------------------------------------------
 * Learned frequency surrogate (no counterpart in the paper).
 *
 * The plain method evaluates chi0 and eps~^-1 at every imaginary frequency of the grid.
 * With a surrogate attached, only a coarse subset C of the grid is computed. X = eps~^-1 - 1
 * on the other ("fine") frequencies F is reconstructed as
 *   X(w_m) = sum_c L_mc X(w_c) + U diag(sigma_l g_l(w_m)) U^H,
 * where U are Ritz modes of eps~(w_ref) - 1 (w_ref = the first coarse frequency),
 * d_l(w) = u_l^H X(w) u_l is the mode diagonal, sigma_l = |d_l(w_ref)|, and the network maps
 * x_l = d_l(C)/sigma_l to f(x) = L x + g(x), the predicted d_l(F)/sigma_l.
 *   g(x) = s * (W4 h3 + b4), h3 = silu(W3 h2 + b3), h2 = silu(W2 h1 + b2), h1 = silu(W1 x + b1).
 * Parameters: one fp32 vector in this order (row-major):
 *   W1 [H][I], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], W4 [O][H], b4 [O], L [O][I], s [1]
 * with I = n_in (coarse frequencies), H = n_hidden, O = n_out (fine frequencies).
 * Matrix products use bf16 copies of W1..W4 (round to nearest even) with fp32 accumulation;
 * biases, L and s stay fp32. All model calls are ordered on the caller's stream given at
 * creation (the model works on its own stream, joined by events).
 * ------------------------------------------------------------------------------------------ */
typedef struct gw_surrogate_s* gw_surrogate;

typedef struct {
  int32_t n_in;      /* coarse frequencies, 1..64          */
  int32_t n_hidden;  /* hidden width, 1..4096               */
  int32_t n_out;     /* fine frequencies, 1..1024           */
} gw_surrogate_dims;

/* Length of the parameter vector for dims (host scalar). */
gw_status gw_surrogate_param_count(const gw_surrogate_dims* dims, int64_t* count);

/* New model with parameters copied from `params` (device fp32 [count]); Adam state zeroed.
 * `stream`: the caller's cudaStream_t (NULL = legacy default). */
gw_status gw_surrogate_create(const gw_surrogate_dims* dims, const float* params, void* stream, gw_surrogate* out);
gw_status gw_surrogate_destroy(gw_surrogate model);
/* Copy the fp32 parameters out (device [count]) / in (device [count]; the bf16 copies and s follow). */
gw_status gw_surrogate_get_params(gw_surrogate model, float* params);
gw_status gw_surrogate_set_params(gw_surrogate model, const float* params);

/* f = L x + g(x) and/or g(x) for n rows: x device [n][I]; f, g device [n][O] (either may be NULL). */
gw_status gw_surrogate_forward(gw_surrogate model, const float* x, int64_t n, float* f, float* g);

/* Mean squared error of f(x) against y over all n*O outputs, and its gradient with respect to
 * every parameter (device [count]; the entry of s is 0: s is fixed). 1 <= n <= 65536.
 * loss: host scalar. Weights enter through their bf16 copies (gradient of the rounded weights). */
gw_status gw_surrogate_loss_grad(gw_surrogate model, const float* x, const float* y, int64_t n, double* loss,
                                 float* grad);

/* Closed-form ridge fit of L: L = argmin |x L^T - y|^2 + ridge*n*|L|^2, normal equations
 * accumulated and solved in FP64 (Cholesky). Then s = rms of the residual y - x L^T
 * (s = 1 if that is 0); rms: host output (may be NULL). Errors: GW_ERR_NOT_PD. */
gw_status gw_surrogate_fit_linear(gw_surrogate model, const float* x, const float* y, int64_t n, double ridge,
                                  double* rms);

/* Ridge fit of L from frequency moments (device FP64 [n_in][n_in + n_out], as accumulated by
 * gw_surrogate_data): with G = moments[:, :n_in], R = moments[:, n_in:],
 * (G + ridge * tr(G)/n_in * 1) L^T = R, solved in FP64 (Cholesky). s is not changed.
 * Errors: GW_ERR_NOT_PD. */
gw_status gw_surrogate_fit_moments(gw_surrogate model, const double* moments, double ridge);

/* s = rms of the residual y - x L^T over n rows (s = 1 if that is 0); rms: host output or NULL. */
gw_status gw_surrogate_fit_scale(gw_surrogate model, const float* x, const float* y, int64_t n, double* rms);

/* Adam (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on W1..b4 over `epochs` passes of
 * mini-batches of `batch` rows (1..min(n, 4096)), rows shuffled every epoch with a generator
 * seeded by `seed` (the last n % batch rows of each shuffled epoch are skipped). L and s are
 * not changed. The MLP is fitted to the residual targets (y - x L^T)/s, whose mean squared
 * error is the loss of f divided by s^2 (the same minimiser; Adam is invariant to that scale).
 * One step (gather, forward, backward, Adam) runs as a captured CUDA graph. Adam's moments and
 * step count persist across calls. loss_hist: host [epochs] mean loss of f per epoch, or NULL. */
gw_status gw_surrogate_train(gw_surrogate model, const float* x, const float* y, int64_t n, int32_t epochs,
                             int32_t batch, double lr, uint64_t seed, double* loss_hist);

/* Surrogate configuration of a plan. */
typedef struct {
  int32_t n_coarse;          /* coarse frequencies computed exactly (= the model's n_in), 1..64   */
  const int32_t* coarse;     /* host [n_coarse]: ascending grid indices; coarse[0] is w_ref        */
  int32_t n_modes;           /* modes the network corrects, 1..n_block                            */
  int32_t n_block;           /* subspace iteration block width, n_modes..min(64, n_aux); it must
                                not exceed the rank of eps~(w_ref) - 1                          */
  int32_t n_iter;            /* subspace iteration steps, 0..1000                                 */
  const gw_complex* start;   /* device [n_aux][n_block]: start block of the iteration (caller's
                                seeded random numbers); copied                                  */
} gw_surrogate_cfg;

/* Attach a surrogate to the plan. With a model, gw_g0w0 computes chi0, eps~ and W^c on the
 * coarse frequencies only: per q it finds U, the n_modes Ritz vectors of eps~(w_ref) - 1 of
 * largest Ritz value after n_iter steps of subspace iteration (two Cholesky-QR passes per step,
 * FP64) and Rayleigh-Ritz, forms the mode diagonal d on the coarse frequencies, evaluates the
 * network, and adds to Sigma_c the fine frequencies through
 *   S_nm(w_m) = sum_c L_mc S_nm(w_c) + sum_l |(a^T V^1/2 U)_l|^2 sigma_l g_l(w_m),
 * which is the S of the reconstructed X above (S is linear in X). The quadrature, the
 * continuation and the QP solve use the full grid. The per-q calls (gw_chi0, gw_screen,
 * gw_sigma) keep the full grid. model NULL with cfg: only gw_surrogate_modes is enabled;
 * model and cfg NULL: detach. The model's n_in / n_out must be n_coarse / n_freq - n_coarse,
 * and it must not be used elsewhere while the plan runs. Sizes cannot change once set. */
gw_status gw_surrogate_enable(gw_plan plan, gw_surrogate model, const gw_surrogate_cfg* cfg);

/* Training data from the plain method: after gw_chi0(q) on the full grid, eps~ and eps~^-1 - 1
 * at every frequency, the modes U of eps~(w_coarse[0]) - 1 (as above), and (device outputs,
 * each may be NULL, not all):
 *   d_out     fp32 [n_modes][n_freq]: d_l(w_j) = u_l^H (eps~^-1(w_j) - 1) u_l
 *   theta_out [n_modes] Ritz values, descending
 *   x_out     fp32 [n_modes][n_coarse]: network inputs d_l(C) / sigma_l, sigma_l = |d_l(w_coarse[0])|
 *   y_out     fp32 [n_modes][n_freq - n_coarse]: targets d_l(F) / sigma_l
 * Needs gw_surrogate_enable. */
gw_status gw_surrogate_modes(gw_plan plan, int32_t sys, int32_t q, float* d_out, double* theta_out, float* x_out,
                             float* y_out);

/* The training data of all q of the plan at once:
 *   x_out, y_out: the rows of gw_surrogate_modes for q = 0 .. N_k-1, in that order: device fp32
 *     [N_k * n_modes][n_coarse] and [N_k * n_modes][n_freq - n_coarse];
 *   moments (device FP64 [n_coarse][n_freq], or NULL): accumulated (the caller zeroes it) with
 *     sum over q and all elements e of X = eps~^-1 - 1 of Re(conj(X_e(w_a)) X_e(w_b)), a coarse,
 *     b the coarse frequencies then the fine ones (needs n_freq <= 64, n_coarse*n_freq <= 1024).
 * q points run in groups (batched factorisations and modes) with the buffers of gw_g0w0.
 * Needs gw_surrogate_enable; leaves no chi0 / W^c in the plan. */
gw_status gw_surrogate_data(gw_plan plan, int32_t sys, float* x_out, float* y_out, double* moments);

/* Text of the last error on the calling thread ("" if none). Never NULL. */
const char* gw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GW_H */
