/*
 * pprpa.h - C ABI of the GB300 (sm_103a) particle-particle RPA hot path.
 *
 * The library solves the spin-adapted ppRPA eigenproblem of the LibppRPA
 * paper (arXiv 2512.12515, Sec. "ppRPA Equation"):
 *
 *     [ A   B ] [X]           [ I  0 ] [X]
 *     [ B^T C ] [Y] = omega * [ 0 -I ] [Y]
 *
 * with singlet or triplet matrix elements built from density-fitted
 * integrals, <pq|rs> = (pr|qs) = sum_P L^P_pr L^P_qs.  The inputs follow the
 * paper's input set (Sec. "Implementation Details"): occupation numbers,
 * orbital energies, and either MO coefficients with three-center AO
 * integrals or the MO-space fitting integrals directly.  The outputs are
 * the two-electron addition energies omega^{N+2}, the eigenvectors X/Y
 * (normalised X^T X - Y^T Y = +1, Eq. xy_norm), the correlation energy
 * (Eq. correlation_energy) and Hellmann-Feynman gradients
 * (Sec. "Analytic Gradient").
 *
 * Conventions (every entry point):
 *  - Arrays are row-major, float64, C-contiguous.  A pointer argument is a
 *    HOST pointer unless the call takes a `where` flag equal to
 *    PPRPA_DEVICE (then it is a device pointer on the context's GPU).
 *  - The caller owns every buffer it passes.  Inputs are copied (or
 *    transformed) into library-owned device memory before the call returns;
 *    outputs are written into caller buffers before the call returns.
 *  - Every call returns 0 (PPRPA_OK) or a negative error code; no call
 *    aborts the process or throws.  pprpa_strerror() names a code and
 *    pprpa_last_error() gives a message for the last failure on the
 *    calling thread.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Active orbitals are ordered occupied first, then virtual.  Pair
 *    vectors use the row-major upper triangle: singlet pairs (p <= q),
 *    triplet pairs (p < q); X (virtual pairs) comes first, then Y
 *    (occupied pairs): z = [X; Y], length N = nvv + noo.
 */
#ifndef PPRPA_H
#define PPRPA_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define PPRPA_OK 0
#define PPRPA_ERR_ARG (-1)      /* bad shape, null pointer, bad option, wrong call order */
#define PPRPA_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define PPRPA_ERR_OOM (-3)      /* device allocation failed */
#define PPRPA_ERR_NOCONV (-4)   /* Davidson hit max_iter; outputs hold the last iterate */
#define PPRPA_ERR_UNSTABLE (-5) /* no shift makes M - mu W positive definite, and (Davidson) the
                                   lowest roots are interleaved with complex pairs */
#define PPRPA_ERR_TIMEOUT (-6)  /* a device-side bounded wait expired */
#define PPRPA_ERR_STATE (-7)    /* required data not set yet (e.g. no integrals) */
#define PPRPA_ERR_UNSUPPORTED (-8) /* the GPU lacks sm_103a features */

/* ---- enums ------------------------------------------------------------ */
#define PPRPA_HOST 0
#define PPRPA_DEVICE 1

#define PPRPA_SINGLET 1
#define PPRPA_TRIPLET 3
#define PPRPA_AB 2 /* "mult" code of the alpha-beta subspace of spin-unrestricted ppRPA (pprpa_set_beta) */

#define PPRPA_METHOD_FULL 0     /* explicit A/B/C build + dense diagonalisation */
#define PPRPA_METHOD_DAVIDSON 1 /* density-fitted sigma + Davidson */

#define PPRPA_PREC_FP64 0       /* every contraction in FP64 */
#define PPRPA_PREC_BF16 1       /* BF16 tensor-core sigma, then BF16x3 split sigma */
#define PPRPA_PREC_FP8 2        /* FP8 (E4M3, per-P / per-vector scaled) first stage, then BF16x3 */

#define PPRPA_CHANNEL_PP 0      /* lowest two-electron addition roots (N+2) */
#define PPRPA_CHANNEL_HH 1      /* highest two-electron removal roots (N-2) */

typedef struct pprpa_ctx pprpa_ctx;

typedef struct pprpa_options {
    int mult;          /* PPRPA_SINGLET or PPRPA_TRIPLET */
    int channel;       /* PPRPA_CHANNEL_PP or PPRPA_CHANNEL_HH */
    int method;        /* PPRPA_METHOD_FULL or PPRPA_METHOD_DAVIDSON */
    int precision;     /* PPRPA_PREC_* (Davidson only; FULL is always FP64) */
    int nroots;        /* roots wanted: 1..nvv lowest N+2 roots (pp), 1..noo highest N-2 roots (hh) */
    double conv_tol;   /* residual 2-norm ||M z - omega W z|| for converged roots */
    int max_iter;      /* Davidson iteration cap */
    int max_subspace;  /* Davidson subspace cap (<= 128); 0 = automatic: 112, with restarts at 72
                          while the shifted pencil is definite and one sigma vector costs under
                          5e11 flop (3 naux n (nv^2 + no^2); PPRPA_SOFT_CAP_FLOPS) */
    int want_ec;       /* also return the correlation energy: FULL, or Davidson asked for every
                          root of its channel (nroots = nvv for pp, noo for hh) */
    int require_definite; /* Davidson: 1 = return PPRPA_ERR_UNSTABLE as soon as the subspace
                          pencil has no definite shift (the stability test of a screen), instead
                          of continuing with the general subspace solver; 0 = default */
} pprpa_options;

typedef struct pprpa_info {
    int iters;            /* Davidson iterations (both stages) */
    int iters_stage1;     /* iterations spent in the low-precision stage */
    int n_sigma;          /* single-vector sigma applications */
    int converged;        /* 1 if every root met conv_tol */
    double max_resid;     /* largest residual norm of the returned roots */
    double mu;            /* shift used by the last Rayleigh-Ritz step */
    double max_imag;      /* Davidson: largest |Im| of complex Ritz values below the highest
                             target at the last iteration (0 if none); FULL: 0 */
    double t_sigma_ms;    /* device time in sigma (CUDA events) */
    double t_total_ms;    /* device time of the whole solve */
    double sigma_flops;   /* algorithmic sigma flops 3*naux*n*(nv^2+no^2) per vector, summed */
    int nconv;            /* returned roots whose residual met conv_tol (the lowest ones need
                             not be among them when the solve did not converge) */
    int n_real;           /* Davidson: real positive-norm Ritz values in the last subspace; 0 when
                             the solve returned no iterate (stopped by require_definite) */
} pprpa_info;

/* ---- context ------------------------------------------------------------
 * pprpa_create: make a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to run on, or NULL for a library-owned stream.  Returns
 * PPRPA_ERR_UNSUPPORTED when the device is not compute capability 10.3.
 * pprpa_destroy frees every device buffer of the context (NULL is a no-op).
 */
int pprpa_create(pprpa_ctx** out, int device, void* cuda_stream);
void pprpa_destroy(pprpa_ctx* ctx);

/* ---- inputs ---------------------------------------------------------------
 * pprpa_set_orbitals: occupation numbers occ[nmo] per spatial orbital (the same for both
 * spins) and orbital energies eps[nmo] in Hartree, sorted ascending.  Inputs of Sec.
 * "Implementation Details" (a) and (b).  Occupations lie in [0, 1] and do not increase with
 * the orbital index: 1 (closed shell), fractional (Sec. "ppRPA for Fractional Charge
 * Systems") or 0.  Hole slots are orbitals with occ > 0 and particle slots orbitals with
 * occ < 1, so a fractionally occupied orbital is both; the fractional matrix elements
 * factor into one weight per slot, sqrt(occ) on holes and sqrt(1 - occ) on particles, which
 * multiply the integrals: L~^P_st = w_s w_t L^P_st (B's weight read as sqrt((1-n_a)(1-n_b)
 * n_k n_l)).  With 0/1 occupations every weight is 1.  Host pointers.
 */
int pprpa_set_orbitals(pprpa_ctx* ctx, int nmo, const double* occ, const double* eps);

/* pprpa_set_active: active space = the highest nocc_act hole slots (orbitals with occ > 0)
 * and the lowest nvir_act particle slots (occ < 1) (the active-space formalism of
 * Sec. "ppRPA Equation").  n = nocc_act + nvir_act slots, holes first; everything below
 * (pair lists, L, gradients, analysis) is indexed by slot.  Must follow set_orbitals and
 * precede set_ao / set_mo.  Default: every slot active.
 */
int pprpa_set_active(pprpa_ctx* ctx, int nocc_act, int nvir_act);

/* pprpa_set_ao: three-center AO integrals ao3c[naux][nbasis][nbasis]
 * (symmetric in the last two indices, already contracted with the fitting
 * metric) and MO coefficients C[nbasis][nmo].  Runs the AO->MO transform
 * L^P_pq = sum_{mu,nu} C_{mu p} (P|mu nu) C_{nu q} on the device in FP64
 * for the active orbitals (input (c) of Sec. "Implementation Details" in
 * its AO form; Abstract).  `where` = PPRPA_HOST or PPRPA_DEVICE for both
 * arrays.  Host input is streamed in slices; device input is read in place.
 */
int pprpa_set_ao(pprpa_ctx* ctx, int nbasis, int naux, const double* C,
                 const double* ao3c, int where);

/* pprpa_set_mo: MO-space fitting integrals L[naux][nmo][nmo] (input (c) of
 * Sec. "Implementation Details").  Only the active block is kept. */
int pprpa_set_mo(pprpa_ctx* ctx, int naux, const double* L, int where);

/* pprpa_set_beta: the beta orbitals of a spin-unrestricted reference, for the
 * (alpha alpha; beta beta) subspace (Sec. "Implementation Details": spin-unrestricted
 * ppRPA is built and diagonalised in three subspaces).  The context's own active orbitals,
 * energies and integrals (set_orbitals / set_active / set_ao or set_mo) are the alpha set;
 * this call gives the beta active space: nocc_b occupied then nvir_b virtual orbitals,
 * their energies eps_b[nb] and MO-space fitting integrals L_b[naux][nb][nb]
 * (nb = nocc_b + nvir_b; naux must equal the alpha one).  Host or device per `where`; the
 * data is copied.  mult = PPRPA_AB then selects the alpha-beta subspace in pprpa_dims,
 * pprpa_diag, pprpa_sigma (FP64), pprpa_build_matrix and pprpa_solve (FULL, or Davidson in
 * FP64): pairs (a_alpha, b_beta) over every virtual x virtual and (i_alpha, j_beta) over
 * every occupied x occupied, row-major, with A_{ab,cd} = d d (eps_a + eps_b) + (ac|bd),
 * B_{ab,kl} = (ak|bl), C_{ij,kl} = -d d (eps_i + eps_j) + (ik|jl) and
 * (pr|qs) = sum_P L^{alpha P}_pr L^{beta P}_qs (no exchange between opposite spins).  The
 * same-spin subspaces are the PPRPA_TRIPLET problem of one spin's orbitals and integrals
 * (a context per spin).  Gradients of alpha-beta roots: pprpa_grad_ab; analysis outputs:
 * pprpa_analyze (spin-resolved density blocks, rectangular NTOs). */
int pprpa_set_beta(pprpa_ctx* ctx, int nocc_b, int nvir_b, int naux, const double* eps_b,
                   const double* L_b, int where);

/* pprpa_grad_ab: Hellmann-Feynman gradient (Sec. "Analytic Gradient") of root `root` of the
 * last pprpa_solve, which must have been of the alpha-beta subspace (mult = PPRPA_AB; either
 * channel, the sign z^T W z = -1 of a removal root applied).  With Zt the n_alpha x n_beta
 * matrix of the root's pair vector (X on its virtual block, Y on its occupied block) and
 * s = z^T W z:
 *   dLa[P] = d omega / d L^{alpha P} = s Zt L^{beta P} Zt^T      (naux x n_alpha x n_alpha)
 *   dLb[P] = d omega / d L^{beta P}  = s Zt^T L^{alpha P} Zt     (naux x n_beta x n_beta)
 *   deps_a[p] = d omega / d eps^alpha_p,  deps_b[q] = d omega / d eps^beta_q
 * (entries of L treated as independent; n_alpha = nocc_act + nvir_act, n_beta = nocc_b +
 * nvir_b, occupied first).  Any output may be NULL; all live on the host or all on the
 * device per `where`.  Errors: PPRPA_ERR_STATE without an alpha-beta solve,
 * PPRPA_ERR_ARG for a root index out of range. */
int pprpa_grad_ab(pprpa_ctx* ctx, int root, double* dLa, double* dLb, double* deps_a, double* deps_b,
                  int where);

/* pprpa_get_L: copy the active-space L^P_pq (naux x n x n, n = nocc_act +
 * nvir_act, hole slots first; with fractional occupations the weighted L~ that the
 * matrix elements use, which pprpa_grad also differentiates) into `out` (host or device
 * per `where`). */
int pprpa_get_L(pprpa_ctx* ctx, double* out, int where);

/* pprpa_dims: sizes of the current problem: n active orbitals, naux, and
 * the pair counts nvv / noo for multiplicity `mult`.  Any out pointer may
 * be NULL. */
int pprpa_dims(pprpa_ctx* ctx, int mult, int* n, int* naux, int* nvv, int* noo);

/* ---- hot-path kernels (also used by pprpa_solve) ------------------------
 * pprpa_diag: diagonal of the ppRPA matrix M (Sec. "ppRPA Equation"):
 *   singlet D_(pq) = w (eps_p + eps_q) + ((pp|qq) + (pq|pq)) / (1 + d_pq),
 *   triplet D_(pq) = w (eps_p + eps_q) + (pp|qq) - (pq|pq),
 * w = +1 on virtual pairs, -1 on occupied pairs.  out[N]. */
int pprpa_diag(pprpa_ctx* ctx, int mult, double* out, int where);

/* pprpa_sigma: sigma_k = M z_k for k vectors z[k][N] -> sigma[k][N]
 * (the Davidson matrix-vector product of Sec. "ppRPA Equation", evaluated
 * as sum_P L^P Zt L^P with the pair packing of Zt).  precision selects
 * the contraction arithmetic: PPRPA_PREC_FP64, PPRPA_PREC_BF16 (BF16
 * operands, FP32 accumulation), PPRPA_PREC_BF16 + 16 (BF16x3 split:
 * hi*hi + hi*lo + lo*hi), or PPRPA_PREC_FP8 (first product L^P Zt with E4M3
 * operands scaled per P and per vector, second in BF16).  Result is FP64.
 * Device or host per `where`. */
int pprpa_sigma(pprpa_ctx* ctx, int mult, int precision, int k, const double* z,
                double* sigma, int where);

/* pprpa_sigma_batch: sigma for many molecules at once (each its own context with its own
 * integrals; all on one device).  Molecule m applies its matrix (multiplicity mults[m]) to
 * ks[m] vectors z[m] -> sigma[m] (DEVICE pointers, layout of pprpa_sigma).  Molecules whose
 * first stage alone fills the GPU many times over (about 26 waves of tiles) run on their own
 * clustered launches; the stage-1 products of all other molecules run in one persistent
 * tensor-core launch and their stage-2 products in a second one; flags & 1 captures that
 * persistent part in a CUDA graph that is replayed while the arguments (pointers and sizes)
 * stay the same.  Runs on ctxs[0]'s stream; returns after the work completes.  precision: PPRPA_PREC_BF16 or
 * PPRPA_PREC_BF16 + 16.  The tile widths are each context's autotuned ones (pprpa_autotune)
 * or the model's choice. */
int pprpa_sigma_batch(int nmol, pprpa_ctx* const* ctxs, const int* mults, const int* ks,
                      const double* const* z, double* const* sigma, int precision, int flags);

/* pprpa_autotune: time the candidate tensor-core tile widths of both sigma stages on this
 * context's problem (multiplicity mult, k vectors) and keep the fastest for later sigma
 * calls.  tiles (nullable, host int[4]) receives the chosen widths: stage 1 virtual,
 * stage 1 occupied, stage 2 virtual, stage 2 occupied (0 = block empty). */
int pprpa_autotune(pprpa_ctx* ctx, int mult, int k, int precision, int* tiles);

/* pprpa_build_matrix: explicit M = [[A, B], [B^T, C]] (N x N, FP64) from
 * the fitted integrals (Sec. "ppRPA Equation", spin-adapted elements). */
int pprpa_build_matrix(pprpa_ctx* ctx, int mult, double* M, int where);

/* pprpa_sigma_noalloc: the FP64 sigma of pprpa_sigma (precision PPRPA_PREC_FP64) for callers
 * that cannot allocate device memory, e.g. code running inside another framework's
 * fixed-budget memory pool, latency-critical loops that cannot afford the device
 * synchronisation of cudaMalloc/cudaFree, or plugins whose host forbids allocation in its
 * callbacks.  The paper has no counterpart: this is a deployment variant of the same
 * contraction.  It needs no context and allocates nothing; every argument is a DEVICE
 * pointer on the current device: L[naux][n][n] active-space fitted integrals (occupied
 * orbitals first, n = nocc_act + nvir_act), eps[n] active orbital energies, z[k][N] trial
 * vectors, sigma[k][N] output (pair order of this header).  Intermediates live in one
 * 64 MiB file-scope device array, so the call is limited to 3*k*n^2*8 + 8*N + ~1 KB bytes
 * of intermediates and returns PPRPA_ERR_ARG beyond that (use pprpa_sigma).  The first call
 * on a device looks up that array's device address; make that first call before any stream
 * capture.  Work is enqueued on `cuda_stream` (NULL = default stream) and the call returns
 * without waiting for it.  All calls share the array and it keeps the last call's contents
 * (the call clears what must start at zero): calls whose work overlaps on the GPU race, so
 * keep them on one stream or serialise them. */
int pprpa_sigma_noalloc(int mult, int nocc_act, int nvir_act, int naux, const double* L,
                        const double* eps, int k, const double* z, double* sigma,
                        void* cuda_stream);

/* ---- solve -----------------------------------------------------------------
 * pprpa_solve: pp channel (opts->channel = PPRPA_CHANNEL_PP): the lowest
 * opts->nroots two-electron addition roots, omega ascending, X^T X - Y^T Y = +1.
 * hh channel (PPRPA_CHANNEL_HH): the highest opts->nroots two-electron removal
 * roots, omega descending, X^T X - Y^T Y = -1 (the lower sign of Eq. xy_norm);
 * they are found as the lowest positive-norm roots of the pencil (M, -W).
 * X[nroots][nvv] and Y[nroots][noo] (either may be NULL), largest-magnitude
 * component positive; ec (may be NULL; written when opts->want_ec is set): correlation
 * energy of Eq. correlation_energy for this multiplicity, sum(Omega^{N+2}) - Tr A from every
 * addition root (pp) or -sum(Omega^{N-2}) - Tr C from every removal root (hh), summed in
 * FP64 on the device; the two agree for a stable problem.  FULL always has every root;
 * Davidson gives ec only when nroots is every root of its channel (noo for hh, the
 * affordable form when the occupied block is small) and they converged, NaN otherwise.
 * info may be NULL.
 * Host output pointers.  Returns PPRPA_ERR_NOCONV (outputs filled with the
 * last iterate) or PPRPA_ERR_UNSTABLE when no positive-definite shift
 * exists and the roots cannot be separated: FULL when the root count by norm fails;
 * Davidson when its subspace pencil has no definite shift, complex Ritz pairs lie below the
 * highest target in at least half of the last PPRPA_UNSTABLE_WINDOW (default 40) iterations
 * and the largest residual has not dropped tenfold over them (outputs hold the last iterate,
 * info->max_imag the largest imaginary part below the targets), or at once when
 * opts->require_definite is set.  Lowest real roots isolated below any
 * complex pairs still converge through the general (non-symmetric) subspace solver.
 * The converged eigenvectors stay on the device for pprpa_grad. */
int pprpa_solve(pprpa_ctx* ctx, const pprpa_options* opts, double* omega, double* X,
                double* Y, double* ec, pprpa_info* info);

/* pprpa_solve_batch: pprpa_solve (Davidson) for nmol molecules at once, each its own context
 * on one device with its own options opts[m] (multiplicity, channel, precision, roots,
 * tolerance; method must be PPRPA_METHOD_DAVIDSON).  Every molecule's iteration runs on its
 * own host thread and its context's stream, so the per-molecule FP64 steps (projections,
 * the Rayleigh-Ritz eigensolve, residuals, corrections) of different molecules overlap on
 * the GPU; their BF16 and BF16x3 sigma products (precision PPRPA_PREC_BF16) are gathered
 * into one batched tensor-core sigma per round (pprpa_sigma_batch's launches, replayed from a
 * CUDA graph while the set of molecules and block sizes stays the same) once every molecule
 * still iterating has asked for one.  FP64 and FP8 solves compute their sigma alone.
 * Outputs per molecule as pprpa_solve: omega[m][nroots], X[m], Y[m] (X, Y or any X[m], Y[m]
 * may be NULL), infos[m] (NULL allowed), host pointers; rcs[m] receives each molecule's
 * return code.  The correlation energy is not returned here.  Returns PPRPA_OK when every
 * molecule returned PPRPA_OK, otherwise the first failing molecule's code (its message
 * names the molecule).  The contexts must not be used by other threads during the call. */
int pprpa_solve_batch(int nmol, pprpa_ctx* const* ctxs, const pprpa_options* opts, double* const* omega,
                      double* const* X, double* const* Y, pprpa_info* infos, int* rcs);

/* pprpa_grad: Hellmann-Feynman gradient (Sec. "Analytic Gradient") of root
 * `root` of the last pprpa_solve (either channel; the sign z^T W z = -1 of a
 * removal root is applied): d omega / d L^P_pq -> dL[naux][n][n]
 * (entries treated as independent) and d omega / d eps_p -> deps[n]
 * (active orbitals).  Computed in FP64 on the device.  Either output may
 * be NULL.  Host or device per `where`. */
int pprpa_grad(pprpa_ctx* ctx, int root, double* dL, double* deps, int where);

/* pprpa_analyze: analysis outputs of root `root` of the last pprpa_solve (either channel).
 * With the root's X (nv x nv) and Y (no x no) viewed as upper-triangular matrices over the
 * pair list (Sec. "Natural Transition Orbital"):
 *   D2e[n][n]: the two-electron addition/removal density matrix of Sec. "Density Matrix",
 *     active-orbital order (occupied first): virtual block X X^T + X^T X, occupied block
 *     -(Y Y^T + Y^T Y), zero elsewhere; its trace is +2 (addition) or -2 (removal), and its
 *     diagonal times z^T W z is d omega / d eps.
 *   lam_p[nv], Cp1[nv][nv], Cp2[nv][nv]: NTO weights (descending) and coefficient matrices of
 *     X = Cp1 diag(sqrt(lam_p)) Cp2^T (Eq. nto_pp); lam_h[no], Ch1, Ch2 likewise for Y
 *     (Eq. nto_hh).  sum(lam_p) - sum(lam_h) = +-1.  Each Cp1 / Ch1 column has its
 *     largest-magnitude entry positive; columns of Cp2 / Ch2 with zero weight are zero.
 * Any output may be NULL; NTOs need nv (no) <= 1024.  FP64 on the device (the NTOs through a
 * one-CTA Jacobi eigensolver of X X^T); outputs host or device per `where`.
 * Alpha-beta roots (last solve with mult = PPRPA_AB): X is the full nv_alpha x nv_beta
 * rectangle and Y the no_alpha x no_beta one; the two orbital slots are told apart by spin:
 *   D2e[(na+nb)][(na+nb)] = diag(D^alpha, D^beta), alpha orbitals first, each spin occupied
 *     first; D^alpha has X X^T on its virtual block and -Y Y^T on its occupied block, D^beta
 *     X^T X and -Y^T Y; each block traces to z^T W z, and its diagonal times z^T W z is that
 *     spin's d omega / d eps (pprpa_grad_ab).
 *   lam_p[nv_alpha], Cp1[nv_alpha][nv_alpha], Cp2[nv_beta][nv_alpha] (zero weights beyond the
 *     rank of X, zero Cp2 columns there); lam_h[no_alpha], Ch1[no_alpha][no_alpha],
 *     Ch2[no_beta][no_alpha] likewise. */
int pprpa_analyze(pprpa_ctx* ctx, int root, double* D2e, double* lam_p, double* lam_h,
                  double* Cp1, double* Cp2, double* Ch1, double* Ch2, int where);

/* pprpa_grad_ao: adjoint of the AO->MO transform of pprpa_set_ao, the step from the
 * MO-space gradient of pprpa_grad / pprpa_grad_ec / pprpa_grad_vector back to the AO inputs
 * (the chain toward the nuclear gradients of Sec. "Analytic Gradient").  With
 * L^P = C_act^T (P|..) C_act (entries independent):
 *   dAO[P][mu][nu] = sum_pq C[mu][p] dL[P][p][q] C[nu][q]            (naux x nbasis x nbasis)
 *   dC[mu][r]      = sum_P (H^P dL^P^T + H^P dL^P)[mu][r],  H^P = (P|..) C_act,
 * for the active columns r of C (nbasis x nmo); every other column is zero.  The AO slices
 * are taken as symmetric (as pprpa_set_ao requires).  Inputs: C[nbasis][nmo] and
 * dL[naux][n][n] (n active orbitals, occupied first); ao3c[naux][nbasis][nbasis] is needed
 * only for dC and may be NULL otherwise.  Either output may be NULL.  All arrays host or
 * device per `where`; FP64 on the device, in slices of the auxiliary index. */
int pprpa_grad_ao(pprpa_ctx* ctx, int nbasis, int naux, const double* C, const double* ao3c,
                  const double* dL, double* dAO, double* dC, int where);

/* pprpa_grad_ec: gradient of the correlation energy of Eq. correlation_energy of the last
 * solve's multiplicity, with respect to L^P_pq (dL[naux][n][n], entries independent) and
 * eps_p (deps[n]).  After a solve of the pp channel that returned every addition root
 * (nroots = nvv): the sum of their Hellmann-Feynman gradients z^T (dM) z minus the
 * derivative of Tr A (E_c = sum(Omega^{N+2}) - Tr A).  After a solve of the hh channel that
 * returned every removal root (nroots = noo, FULL or converged Davidson): E_c =
 * -sum(Omega^{N-2}) - Tr C, i.e. the sum of z^T (dM) z over the removal roots (their
 * d Omega is -z^T (dM) z) minus the derivative of Tr C.  PPRPA_ERR_STATE without such a
 * solve.  FP64 on the device (batched over roots); outputs host or device per `where`,
 * either may be NULL. */
int pprpa_grad_ec(pprpa_ctx* ctx, double* dL, double* deps, int where);

/* pprpa_grad_sum: gradient of sum_{r < nw} w[r] omega_r over the first nw roots of the last
 * pprpa_solve (either channel, removal roots carrying their sign z^T W z = -1), i.e.
 * sum_r w[r] (d omega_r / d L^P_pq, d omega_r / d eps_p) of pprpa_grad in one call (the
 * backward step of a function of several roots, Sec. "Analytic Gradient").  w: host
 * float64[nw], finite, 1 <= nw <= roots of the last solve.  dL[naux][n][n], deps[n]: host or
 * device per `where`, either may be NULL.  FP64 on the device, the roots batched through
 * one reduction per slice of the auxiliary index.  PPRPA_ERR_STATE without a solve. */
int pprpa_grad_sum(pprpa_ctx* ctx, int nw, const double* w, double* dL, double* deps, int where);

/* pprpa_grad_vector: the same Hellmann-Feynman contraction for an explicit pair vector
 * z[N] of multiplicity `mult` (Sec. "Analytic Gradient": d(z^T M z)/d theta = z^T (dM/d theta) z),
 * i.e. the gradient of the Rayleigh quotient at fixed z; for a converged root normalised to
 * z^T W z = 1 it is d omega / d theta.  z, dL[naux][n][n] and deps[n] are host or device per
 * `where`; either output may be NULL. */
int pprpa_grad_vector(pprpa_ctx* ctx, int mult, const double* z, double* dL, double* deps,
                      int where);

/* ---- diagnostics ----------------------------------------------------------
 * pprpa_profile: CUDA-event timing of every tensor-core sigma GEMM launch,
 * recorded on the context's stream.  enable = 1 clears the records and
 * starts recording, 0 stops.  `out` (host, nullable) receives 4 rows of
 * {launches, total_ms, algorithmic_flops}: stage 1 BF16, stage 2 BF16,
 * stage 1 BF16x3, stage 2 BF16x3.  algorithmic_flops counts the sigma work
 * 3*naux*n*(nv^2+no^2) per vector split as 2/3 (stage 1) and 1/3 (stage 2),
 * independent of padding and of the number of split products.  Reading
 * synchronises the context's stream. */
int pprpa_profile(pprpa_ctx* ctx, int enable, double* out);

const char* pprpa_strerror(int code);
const char* pprpa_last_error(void);
/* Number of kernels this library has launched on the calling process. */
long long pprpa_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* PPRPA_H */
