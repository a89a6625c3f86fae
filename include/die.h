/*
 * libdie -- C ABI of the GB300 TE domain-integral-equation solver.
 *
 * Zouros & Budko, "Transverse electric scattering on inhomogeneous objects:
 * spectrum of integral operator and preconditioning" (arXiv 1104.4263).
 *
 * The operator.  On an n1 x n2 grid of square cells of side h (cell centres
 * x_i = (i + 1/2) h - n h / 2), with relative permittivity eps_r(x), contrast
 * chi = eps_r - 1 (Eq. (2.11), eps_b = 1) and unknowns u = (E1, E2), the
 * midpoint-collocation system of Section 4, Eqs. (4.1)-(4.5), restricted to the
 * electric unknowns (no magnetic contrast, so Eqs. (4.6)-(4.11) drop out) is
 *     A u = b,   A = I - G X(chi),
 *     (G w)_l(x_n) = sum_m sum_q G_lq(x_n - x_m) w_q(x_m),
 * with G_lq from Eqs. (4.3)-(4.5) (Hankel functions of k_b |x_n - x_m|; the
 * diagonal from the equal-area disc of Eq. (4.4)).  The regularised operator of
 * Eq. (3.19) and Section 5 is A_R A with A_R = A(chi'), chi' = 1/eps_r - 1
 * (Eq. (3.18)).  G is block-Toeplitz, so every product runs as a zero-padded 2-D
 * FFT convolution (Sections 1 and 5).
 *
 * Vector layout.  A field vector is 2 * n1 * n2 interleaved complex numbers in
 * the order [component][x2][x1] (x1 fastest): E1 plane, then E2 plane.  For the
 * polarisation DIE_TE_MAG it is 3 * n1 * n2: E1, E2, then H3.  Wherever a size below
 * says "2 n1 n2", read "3 n1 n2" for DIE_TE_MAG.
 * Complex128 = two doubles (re, im); complex64 = two floats.
 *
 * Conventions for every call:
 *  - device pointers are CUDA global-memory pointers on the current device; the
 *    caller owns them and must keep them alive until the stream reaches the call;
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream); every call is
 *    stream-ordered on it; calls that report values to the host synchronise it;
 *  - handles are not thread-safe: one host thread at a time per handle;
 *  - no call aborts or traps: failures return a die_status; after DIE_ECUDA the
 *    handle should be destroyed.
 */
#ifndef LIBDIE_DIE_H
#define LIBDIE_DIE_H

#ifdef __cplusplus
extern "C" {
#endif

#define DIE_ABI_VERSION 3

typedef enum die_status {
    DIE_OK = 0,
    DIE_EINVAL = 1,        /* bad argument (sizes, NULL pointer, unsupported option)          */
    DIE_ENOMEM = 2,        /* device or host allocation (or a host thread) could not be had    */
    DIE_ECUDA = 3,         /* a CUDA runtime call failed                                       */
    DIE_ESINGULAR = 4,     /* eps_r == 0 somewhere (existence condition, Eq. (3.17)), or T singular */
    DIE_ENOCONV = 5,       /* GMRES / eigensolver stopped at max_iters without reaching tol    */
    DIE_EBREAKDOWN = 6,    /* Arnoldi breakdown with a singular least-squares problem          */
    DIE_ENAN = 7,          /* NaN or Inf met in a residual or norm                             */
    DIE_ETIMEOUT = 8,      /* a bounded device-side wait gave up                               */
    DIE_EUNSUPPORTED = 9   /* FFT size or grid size outside what the kernels handle            */
} die_status;

typedef enum die_precision {
    DIE_FP64 = 0,          /* complex128 storage, FP64 arithmetic everywhere                  */
    DIE_FP32_INNER = 1     /* complex64 FFT products; FP64 for everything else                */
} die_precision;

/* Polarisation (Section 2).  DIE_TE: the unknowns (E1, E2) of Eq. (2.15) with the
 * Green's tensor of Eqs. (4.3)-(4.5).  DIE_TM: the scalar E-wave unknown E3 of Eq. (2.16),
 * E3_in = E3 - k_b^2 g * (chi E3), on the same grid with the scalar kernel
 * k_b^2 h^2 (i/4) H0(k_b r) and, on the diagonal, the integral of k_b^2 g over the
 * equal-area disc of Eq. (4.4), (i pi/2) k_b a H1(k_b a) - 1.  A TM field vector keeps the
 * two-plane layout below with E3 in the first plane and a zero second plane: the TM
 * operator acts on each plane separately (the off-diagonal kernel plane is zero), so a zero
 * second plane stays zero through every product, solve and deflation; the products cost
 * what a TE product costs.
 * DIE_TE_MAG: the full TE system with electric and magnetic contrast, unknowns
 * (E1, E2, H3) of Eq. (2.15) in three planes, A = I - G X, X = diag(chi_e, chi_e, chi_m),
 * chi_e = eps_r - 1, chi_m = mu_r - 1 (mu_r from dieop_set_permeability; 1 until then).
 * Besides the electric block of Eqs. (4.3)-(4.5), G has the couplings of Section 3's
 * compact kernels K13, K23, K31, K32, K33 (eps_b = mu_b = 1, omega = k_b):
 * G13 = G31 = (k_b^2 h^2 / 4) H1(k_b r) theta_2, G23 = G32 = -(k_b^2 h^2 / 4) H1(k_b r) theta_1,
 * G33 = k_b^2 h^2 (i/4) H0(k_b r), zero at r = 0 except G33(0) = (i pi/2) k_b a H1(k_b a) - 1
 * (the [A33]_nn of Section 4).  (The discrete relations A31 = -A13, A23 = -A32 printed in
 * Section 4 disagree with K31, K32 and are not used.)  The regulariser is A(chi'_e, chi_m),
 * chi'_e = 1/eps_r - 1: the symbol I + chi_e Q of Section 3 does not involve chi_m.  Its
 * products run on the runtime-plan kernels (no compile-time FFT path, no tile schedule, no
 * complex64 deflated first pass), and the learned preconditioner does not take it. */
typedef enum die_polarization {
    DIE_TE = 0,
    DIE_TM = 1,
    DIE_TE_MAG = 2
} die_polarization;

typedef struct dieop_s* dieop_t;
typedef struct defl_s* defl_t;

/* Operator description (Section 4: uniform grid of step h; units of the
 * background wavelength, so k_b = 2 pi by default). */
typedef struct dieop_desc {
    int n1, n2;            /* cells along x1 / x2; 2 <= n <= 2048                              */
    double h;              /* cell side in background wavelengths, > 0                         */
    double k_b;            /* background wavenumber; <= 0 selects 2 pi                         */
    die_precision prec;    /* element type of dieop_apply / dieop_apply_regularized I/O        */
    int M1, M2;            /* FFT sizes, 0 = smallest 2^a 3^b >= 2 n; else >= 2 n and 2^a 3^b */
    die_polarization pol;  /* DIE_TE (default, 0), DIE_TM or DIE_TE_MAG                         */
} dieop_desc;

/* dieop_create -- build the operator of Eqs. (4.3)-(4.5) for a permittivity map.
 *   eps_r: n1*n2 complex128 relative permittivities, layout [x2][x1]; host memory if
 *          eps_on_device == 0, else device memory.  Copied; the caller keeps ownership.
 *   Computes the Green's-tensor table and its 2-D FFT (FP64; a complex64 copy is kept
 *   too), the contrasts chi and chi', and the workspaces.
 *   Errors: DIE_EINVAL (sizes, h, NULL), DIE_ESINGULAR (|eps_r| <= 1e-12 in some cell:
 *   the existence condition eps != 0 of Eq. (3.17)), DIE_EUNSUPPORTED (FFT sizes),
 *   DIE_ENOMEM, DIE_ECUDA.  On error *out is NULL. */
die_status dieop_create(const dieop_desc* desc, const void* eps_r, int eps_on_device,
                        void* stream, dieop_t* out);

/* Replaces the permittivity map of an operator (same grid, h, FFT sizes: the Green
 * spectra of Eqs. (4.3)-(4.5) do not depend on it), recomputing chi and chi'.  eps_r as
 * for dieop_create.  On DIE_ESINGULAR (the existence condition of Eq. (3.17)) the operator
 * keeps its previous map.  The operator gets a new identity: deflation handles built
 * before the call are rejected by the solves.  Synchronises the stream.  Errors:
 * DIE_EINVAL, DIE_ESINGULAR, DIE_ENOMEM, DIE_ECUDA. */
die_status dieop_set_permittivity(dieop_t op, const void* eps_r, int eps_on_device, void* stream);

/* Sets the relative permeability map of a DIE_TE_MAG operator: chi_m = mu_r - 1 (Section 2's magnetic contrast).
 * mu_r: n1*n2 interleaved complex128, host (mu_on_device = 0) or device.  DIE_EINVAL for
 * another polarisation, DIE_ENAN for a non-finite value (the operator keeps its previous
 * map).  The operator gets a new identity, as for dieop_set_permittivity.  Synchronises
 * the stream.  Errors: DIE_EINVAL, DIE_ENAN, DIE_ENOMEM, DIE_ECUDA. */
die_status dieop_set_permeability(dieop_t op, const void* mu_r, int mu_on_device, void* stream);

/* Schedule of the complex64 products: the tile height (rows per block) of the row passes
 * (contrast multiply + row FFT, row inverse FFT + crop, and the fused pass of the
 * regularised product, Eq. (4.1)) on grids whose row FFT is the compile-time path
 * (M1 = 2 n1 = 2^a, 256 <= M1 <= 4096); other grids have one schedule.  Candidate heights
 * are 1, 2, 4 and 8 rows (at most 512 threads per block: M1 = 2048 allows up to 4, 4096
 * up to 2; the default is 4, 2 at M1 = 4096).  Every height gives bit-identical products.
 *
 * dieop_autotune times the complex64 regularised product A(chi') A(chi) at every
 * candidate height (CUDA events on `stream`, 3 warm-up and 20 timed products each, on
 * two 2 n1 n2 complex64 scratch vectors it allocates and frees) and keeps the default
 * unless another height is at least 3% faster, then the fastest (the timed product stands
 * in for the solver's passes, whose deflated first row pass may rank close heights
 * differently).
 * The choice is remembered per (device, M1, n2) for the process: a later call on an
 * operator of the same sizes reuses it without timing unless force != 0.  tile_rows
 * (host, may be NULL) receives the height used; us4 (host, may be NULL) receives the
 * microseconds per product at heights 1, 2, 4, 8 (0: not a candidate or not timed this
 * call).  Not concurrent with other calls on the operator (it uses the operator's
 * workspace).  Synchronises the stream.  Errors: DIE_EINVAL, DIE_ENOMEM, DIE_ECUDA. */
die_status dieop_autotune(dieop_t op, int force, void* stream, int* tile_rows, double* us4);

/* Sets the tile height (0 = the default; 1, 2, 4 or 8 where the grid allows it) and
 * returns DIE_EINVAL for any other value or a grid with one schedule.  Affects products
 * launched afterwards (a CUDA graph captured before keeps the height it captured). */
die_status dieop_set_tile_rows(dieop_t op, int tile_rows);

/* The tile height the complex64 row passes use (0 for a grid with one schedule). */
int dieop_tile_rows(dieop_t op);

/* Actual sizes chosen at create: out[0..5] = n1, n2, M1, M2, N = n1*n2, prec. */
die_status dieop_info(dieop_t op, long long* out6);

/* y = A x  (Eq. (4.1) with Eqs. (4.3)-(4.5)); x, y: device, 2*n1*n2 complex of the
 * type selected by desc.prec (complex128 for DIE_FP64, complex64 for DIE_FP32_INNER).
 * y may equal x (in place).  Errors: DIE_EINVAL, DIE_ECUDA. */
die_status dieop_apply(dieop_t op, const void* x, void* y, void* stream);

/* y = A(chi') A(chi) x, the regularised product of Eq. (3.19) / Section 5.
 * Same types, aliasing and errors as dieop_apply. */
die_status dieop_apply_regularized(dieop_t op, const void* x, void* y, void* stream);

/* y = A(chi') x alone (the regulariser; used for the right-hand side A_R b). */
die_status dieop_apply_regularizer(dieop_t op, const void* x, void* y, void* stream);

/* Batched products with one operator (many incidence angles of one scatterer):
 * y_k = A x_k (regularized == 0) or y_k = A(chi') A(chi) x_k (regularized != 0), k < nrhs.
 * x, y: device, nrhs field vectors one after another (vector k starts at element
 * k * 2 n1 n2), each laid out as for dieop_apply, complex128 (prec DIE_FP64) or complex64
 * (DIE_FP32_INNER); y may equal x.  Every pass of the product runs as one launch over all
 * right-hand sides, so the kernels see nrhs times more independent work per launch.  The
 * operator keeps a workspace of nrhs sets of row spectra (2 M1 n2) and middle vectors
 * (2 n1 n2), grown on the first call with a larger nrhs (that call synchronises the
 * device).  Results are identical to nrhs separate calls.  DIE_EINVAL: NULL pointer or
 * nrhs outside [1, 1024]; DIE_ENOMEM: the workspace does not fit. */
die_status dieop_apply_batch(dieop_t op, int nrhs, const void* x, void* y, int regularized, void* stream);

/* b = incident TE plane wave of unit |E| at angle psi to the x1 axis (Section 4, end):
 * H3 = exp(i k_b (x1 cos psi + x2 sin psi)), E1 = -sin(psi) H3, E2 = cos(psi) H3; for a
 * TM operator E3 = exp(i k_b (x1 cos psi + x2 sin psi)) in the first plane, 0 in the second;
 * for DIE_TE_MAG (E1, E2, H3) in three planes, as for TE.
 * b: device, 2*n1*n2 complex128.  Errors: DIE_EINVAL, DIE_ECUDA. */
die_status dieop_rhs_plane_wave(dieop_t op, double psi, void* b, void* stream);

void dieop_destroy(dieop_t op);

/* ----------------------------------------------------------------------------
 * Restarted GMRES (Sections 4-5) with optional regularisation and deflation.
 * Solves Atilde x = btilde with Atilde = A (regularized = 0) or A_R A and
 * btilde = A_R b (regularized = 1), right-preconditioned by the deflation
 * P^-1 of Eq. (4.12) when a defl_t is given: Atilde P^-1 v = btilde, x = P^-1 v.
 * Arnoldi by classical Gram-Schmidt with the DGKS criterion (a second pass when the
 * first left less than eta of ||w||; see reorth_eta), FP64; Hessenberg least squares by
 * Givens rotations, FP64, on the device.  With inner = DIE_FP32_INNER the products
 * with Atilde inside a cycle and the deflation P^-1 run in complex64 (a fixed
 * preconditioner for the whole solve); the restart residual stays FP64.
 * ------------------------------------------------------------------------- */
typedef struct gmres_opts {
    int restart;           /* Krylov dimension per cycle, 1..2048 (the basis holds restart + 1
                              FP64 vectors and their Re - Im planes: 24 (restart + 1) 2 n1 n2
                              bytes; bases longer than 256 vectors are swept in chunks)        */
    int max_iters;         /* cap on Arnoldi steps (applications of Atilde)                    */
    double tol;            /* stop when ||btilde - Atilde x|| / ||btilde|| <= tol              */
    int regularized;       /* 0: Atilde = A; 1: Atilde = A_R A                                 */
    int use_x0;            /* 1: x holds the initial guess on entry; 0: x0 = 0                 */
    die_precision inner;   /* DIE_FP64, or DIE_FP32_INNER: complex64 products inside a cycle,
                              FP64 restart residual (iterative refinement)                      */
    int timing;            /* 1: fill t_matvec/t_orth/t_defl (adds stream syncs)               */
    double reorth_eta;     /* DGKS threshold: second Gram-Schmidt pass when ||w'|| < eta ||w||;
                              <= 0 selects 0.01 for restart <= 64 and the classical 1/sqrt(2)
                              beyond (single-pass losses accumulate over a cycle: measured on
                              the 512^2 core-shell, max |V*V - I| 2.3e-11 after 64 steps at
                              0.01, 3e-6 after 300 steps at 0.01, < 1e-8 at 1/sqrt(2));
                              >= 1 always re-orthogonalises                                    */
    int graph;             /* 1: the Arnoldi steps of a cycle run as one CUDA graph launch.  A
                              configuration (operator context, deflation handle, options, cycle
                              length) is captured the first time it recurs after one direct run
                              and kept by the context (up to 4) for later cycles and solves;
                              results are bit-identical to graph = 0.  Ignored (no graph) when
                              timing = 1 or kernel timing (die_prof_*) is on                   */
} gmres_opts;

typedef struct gmres_report {
    int cycles;            /* restart cycles run                                               */
    int iters;             /* Arnoldi steps = applications of Atilde                           */
    int n_apply;           /* applications of A or A_R (a regularised step counts 2)           */
    double rel_res_solved; /* FP64 ||btilde - Atilde x|| / ||btilde|| at exit                  */
    double rel_res_orig;   /* FP64 ||b - A x|| / ||b|| at exit                                 */
    double t_matvec, t_orth, t_defl, t_total;   /* seconds                                    */
    double* history;       /* caller-owned host buffer for per-step residual estimates, or NULL */
    int history_cap;       /* its length                                                       */
    int history_len;       /* entries written                                                  */
    int n_reorth;          /* Arnoldi steps that needed the second Gram-Schmidt pass           */
    int graph_cycles;      /* cycles whose Arnoldi steps ran as a graph launch                 */
} gmres_report;

/* b, x: device complex128, 2*n1*n2.  defl may be NULL.  report may be NULL.
 * Returns DIE_OK when converged, DIE_ENOCONV at max_iters (x holds the last iterate),
 * DIE_ENAN if a norm became NaN/Inf, DIE_EBREAKDOWN on a singular Hessenberg system,
 * DIE_EINVAL on bad options (restart range, defl built for another operator), DIE_ENOMEM
 * when the solver context cannot be allocated, DIE_ECUDA on a CUDA error.  No call of
 * this library lets a C++ exception escape. */
die_status gmres_solve(dieop_t op, defl_t defl, const gmres_opts* opts, const void* b, void* x,
                       gmres_report* report, void* stream);

/* Copies `count` vectors of the Krylov basis held by the operator's solver context (the
 * one gmres_solve uses), starting at basis vector `first`, to out (device, count * 2 n1 n2
 * complex128, one vector after another); stream-ordered.  After gmres_solve returns,
 * vectors 1 .. k-1 of the context are the orthonormal Arnoldi vectors v_1 .. v_{k-1} of
 * the solve's last cycle (k = that cycle's Arnoldi steps; Section 4's restarted GMRES),
 * vector 0 holds the restart residual b~ - A~x computed after that cycle and vector k
 * the last, unnormalised, direction.  A diagnostic of the Gram-Schmidt orthogonality
 * (||V* V - I||); the paper has no counterpart.  DIE_EINVAL: NULL pointer, no solve run
 * on this operator yet, or [first, first + count) outside the basis (restart + 1). */
die_status gmres_basis(dieop_t op, int first, int count, void* out, void* stream);

/* nrhs independent solves with one operator and deflation handle (for example one
 * scatterer under several incidence angles), run concurrently: b, x hold nrhs complex128
 * field vectors one after another (vector k at element k * 2 n1 n2); reports: NULL or an
 * array of nrhs reports (each with its own optional history buffer).  Every right-hand
 * side gets its own solver context (Krylov basis, product workspace, deflation scratch,
 * streams, kept by the operator for later calls) and its own host thread, so that the
 * FP64-bound Gram-Schmidt passes of one system overlap the FFT passes of another.  Each
 * x_k is bit-identical to gmres_solve on b_k.  The L2 access-policy window of gmres_solve
 * is not used.  Returns the first error other than DIE_ENOCONV if any, else DIE_ENOCONV
 * if some system did not converge, else DIE_OK; DIE_EINVAL also for nrhs outside
 * [1, 16]. */
die_status gmres_solve_batch(dieop_t op, defl_t defl, const gmres_opts* opts, int nrhs, const void* b, void* x,
                             gmres_report* reports, void* stream);

/* count independent systems whose operators may differ (different scatterers and grid
 * sizes): system k solves with ops[k] and defls[k] (defls NULL, or an array whose
 * entries may be NULL) from b[k] into x[k] (device complex128, 2 n1 n2 of ops[k]; x[k]
 * holds an initial guess when opts->use_x0).  One set of options for all.  Up to 16
 * systems run at once, one host thread each, taking the systems in order from a shared
 * counter; a thread solves in the first batch context of the system's operator that no
 * other thread holds at that moment (created on first use and kept by the operator, as
 * for gmres_solve_batch), so an operator keeps as many contexts as it had systems in
 * flight at once.  Each x[k] is bit-identical to gmres_solve on b[k].  reports: NULL or
 * count reports.  Returns as gmres_solve_batch; DIE_EINVAL for count < 1, a NULL array or
 * entry, or any system's options or deflation handle that gmres_solve would reject
 * (checked before any solve starts). */
die_status gmres_solve_many(int count, const dieop_t* ops, const defl_t* defls, const gmres_opts* opts,
                            const void* const* b, void* const* x, gmres_report* reports, void* stream);

/* ----------------------------------------------------------------------------
 * Deflation (Eqs. (4.12)-(4.13)): V = orthonormal basis of the invariant subspace
 * of the r largest-magnitude eigenvalues of Atilde (Krylov-Schur Arnoldi on the
 * device; the paper uses Matlab eigs with tolerance 1e-4, Section 5), and
 * T = V^* Atilde V; the preconditioner is P^-1 = I + V (T^-1 - I) V^*.
 * ------------------------------------------------------------------------- */
typedef struct defl_opts {
    int r;                 /* eigenvalues to deflate, 1..256; 0 = count those outside the
                              deflation radius of Section 5 (capped at r_max)                  */
    int r_max;             /* cap for r = 0 (default 64 when <= 0), <= 256                    */
    double tol;            /* Ritz residual ||Atilde y - theta y|| <= tol |theta| (1e-4)       */
    int regularized;       /* deflate A_R A (1) or A (0)                                       */
    die_precision inner;   /* precision of the products inside the eigensolver               */
    int krylov_dim;        /* Krylov-Schur basis size, r + 2 .. 318; 0 = max(2 r + 16, r + 32)
                              capped at 318                                                     */
    int max_restarts;      /* 0 = 200                                                           */
    unsigned long long seed; /* start vector seed                                              */
} defl_opts;

/* eig_out: host, 2*r doubles (re, im of the deflated eigenvalues, |.| descending), or
 * NULL.  r_out (may be NULL) receives the r actually used.  Errors: DIE_EINVAL,
 * DIE_ENOCONV (not all r Ritz pairs reached tol; the handle is still returned and
 * usable), DIE_ESINGULAR (T singular), DIE_ENOMEM, DIE_ECUDA. */
die_status deflation_build(dieop_t op, const defl_opts* opts, void* stream, defl_t* out,
                           double* eig_out, int* r_out);

/* z = P^-1 x with P^-1 = I + V (T^-1 - I) V^* (Eq. (4.12)); x, z device complex128;
 * z may equal x. */
die_status deflation_apply(defl_t defl, const void* x, void* z, void* stream);

/* z = P^-1 x exactly as deflation_apply, but allocating nothing.  The paper has no
 * counterpart: this entry exists for callers that must not allocate device memory,
 * for example a solver embedded in another program that has already handed all
 * device memory to its own pool allocator, or a latency-critical loop where the
 * device-wide synchronisation that cudaMalloc and cudaFree can cause is not
 * acceptable.  Its scratch (projections, per-block and per-group partial sums and the
 * reduction's arrival counters, about 1.4 MB) is a static device array inside the
 * library that every GPU loading the library keeps until the process exits.
 *   - defl must have r <= 128, else DIE_EINVAL; x, z as for deflation_apply; the
 *     device current at the call must be the one defl was built on, else DIE_EINVAL.
 *   - The array's address is looked up once per device and kept: after a
 *     cudaDeviceReset of that device in this process the entry point must not be used.
 *   - The first call on a device looks up the array's address on that device (call
 *     it with that device current); make this first call before any stream capture.
 *   - All calls share the one array (it keeps the last call's contents; the counter
 *     are cleared at the start of each call): calls that overlap on the GPU, e.g. on
 *     two streams at once, race and give wrong results.  Serialise them. */
die_status deflation_apply_noalloc(defl_t defl, const void* x, void* z, void* stream);

void deflation_destroy(defl_t defl);

/* Deflation radius of Section 5: the largest |lambda'| over the images of the segments
 * [1, eps] under Eq. (5.3), lambda' = [1 + (1 - lambda)/eps] lambda, for every
 * permittivity value in eps_r (host, count complex128), each segment sampled at
 * `samples` points (1000 if <= 1).  Returns a negative value on bad arguments. */
double die_deflation_radius(const double* eps_r, long long count, int samples);

/* The memory rule of Section 5 (host only): for M bytes of memory, the eigenvalue
 * fraction beta (r = 3 N beta deflated eigenvalues), restart = x r, k_ppw points per
 * smallest medium wavelength and the largest relative permittivity eps_max:
 *   out3[0] = N_max = [sqrt(900 + M s) - 30] / (12 s), s = beta^2 + beta + x beta,
 *   out3[1] = [a/lambda]_max = (sqrt(N_max) - 1) / alpha,
 *   out3[2] = alpha = k_ppw sqrt(eps_max), so that N = (alpha a/lambda + 1)^2.
 * (The paper's counts are for its 3N-unknown system.)  DIE_EINVAL on a NULL pointer or a
 * non-positive input. */
die_status die_memory_plan(double M, double beta, double x, double k_ppw, double eps_max, double* out3);

/* ----------------------------------------------------------------------------
 * Kernel timing (a tracing aid; the paper has no counterpart).  Between
 * die_prof_begin and die_prof_end every kernel launch of the library is bracketed
 * by CUDA events on its stream; die_prof_end synchronises the device and sums the
 * durations per kernel class.  Not thread-safe; do not enable during CUDA-graph
 * capture.  die_prof_end returns DIE_ENOMEM if the event pool overflowed (the
 * sums then cover the launches recorded before the overflow).
 * ------------------------------------------------------------------------- */
die_status die_prof_begin(void);
die_status die_prof_end(void);
int die_prof_kernels(void);                       /* number of kernel classes          */
const char* die_prof_name(int id);                /* class name, static storage        */
die_status die_prof_read(int id, long long* launches, double* total_ms);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (an FMA-chain kernel over
 * every SM, best of three timed launches after a warm-up, CUDA events on `stream`): the
 * denominator of the FP64 kernels' roofline fractions.  A measurement aid; the paper has
 * no counterpart.  Synchronises the stream.  DIE_EINVAL on NULL, DIE_ENOMEM, DIE_ECUDA. */
die_status die_fp64_peak(double* tflops, void* stream);

/* Human-readable name of a status code (static storage). */
const char* die_status_str(die_status s);

/* sizeof of the public structures, for bindings that mirror them: sizes[0..n) receives
 * dieop_desc, gmres_opts, gmres_report, defl_opts (in this order; n <= 4).  DIE_EINVAL
 * if sizes is NULL or n is outside [1, 4]. */
die_status die_abi_sizes(long long* sizes, int n);

/* Library ABI version (DIE_ABI_VERSION) for binding checks. */
int die_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBDIE_DIE_H */
