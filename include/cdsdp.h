/*
 * cdsdp.h — C ABI of the GB300 chordally decomposed ADMM solver for sparse SDPs
 * (Zheng, Fantuzzi, Papachristodoulou, Goulart, Wynn, "Chordal decomposition in
 * operator-splitting methods for sparse semidefinite programs", arXiv 1707.05058).
 *
 * Problem (Section 1, Eqs. PrimalSDP / DualSDP):
 *     min <C, X>  s.t.  <A_i, X> = b_i (i = 0..m-1),  X PSD
 *     max b^T y   s.t.  Z + sum_i y_i A_i = C,        Z PSD
 *
 * Conventions for every function:
 *   - Return value is a cdsdp_status: negative values are errors, non-negative
 *     values are solve outcomes.  No function aborts, exits or traps.
 *   - Matrices are given as 0-based lower-triangle triplets (row >= col); an
 *     upper-triangle entry is an error (CDSDP_ERR_ARG).  Duplicate triplets are
 *     summed.  Off-diagonal entries stand for both (row,col) and (col,row).
 *   - Host arrays passed in are copied; the caller keeps ownership.
 *   - "d_" arguments are device pointers on the current CUDA device; the
 *     caller owns that memory.  The library itself never allocates device
 *     memory: the caller provides the workspace (cdsdp_workspace_bytes).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef CDSDP_H
#define CDSDP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cdsdp cdsdp; /* opaque; created by a cdsdp_setup* call, released by cdsdp_free */

typedef enum {
    CDSDP_PRIMAL = 0, /* Algorithm 1: domain-space decomposition (Section 4.1) */
    CDSDP_DUAL = 1,   /* Algorithm 2: range-space decomposition (Section 4.2)  */
    CDSDP_HSDE = 2    /* Algorithm 3: homogeneous self-dual embedding (Section 5) */
} cdsdp_form;

typedef enum {
    CDSDP_SOLVED = 0,
    CDSDP_MAX_ITER = 1,
    CDSDP_PRIMAL_INFEASIBLE = 2, /* HSDE only: certificate u_y / (b^T u_y)        */
    CDSDP_DUAL_INFEASIBLE = 3,   /* HSDE only: certificate -u_x / (c^T u_x)       */
    CDSDP_NOT_PD = 4,            /* completion: a clique block is not positive
                                    definite, so no max-det completion exists     */
    CDSDP_ERR_ARG = -1,          /* malformed argument                            */
    CDSDP_ERR_RANK = -2,         /* A not full row rank: Cholesky pivot <= 0      */
    CDSDP_ERR_CUDA = -3,         /* a CUDA runtime call failed                    */
    CDSDP_ERR_NOMEM = -4,        /* host allocation failed / workspace too small  */
    CDSDP_ERR_TIMEOUT = -5,      /* a bounded device wait gave up                 */
    CDSDP_ERR_NUMERIC = -6,      /* NaN or Inf met in the iteration               */
    CDSDP_ERR_STATE = -7,        /* call out of order (e.g. solve before bind)    */
    CDSDP_ERR_UNSUPPORTED = -8   /* size or option the library does not handle    */
} cdsdp_status;

typedef enum {
    CDSDP_FP32_PROJECTION = 0, /* eigensolve + rebuild in float32, clique state float32,
                                  affine step, residuals and tau/kappa in float64 */
    CDSDP_FP64 = 1             /* float64 everywhere */
} cdsdp_precision;

typedef struct {
    double eps;            /* stopping tolerance eps_tol (Sections 4.1.4, 4.2.4, 5.2.3) */
    int max_iter;          /* n_max                                                     */
    double rho;            /* ADMM penalty (Algorithms 1, 2); unused by HSDE            */
    int precision;         /* cdsdp_precision                                           */
    int use_graph;         /* 1: whole solve is one CUDA graph with a device-side while
                              loop; 0: one launch per phase, host polls every check_every */
    int check_every;       /* host poll period when use_graph = 0                       */
    int jacobi_max_sweeps; /* cap on Jacobi sweeps per projection                       */
    int warm_start;        /* 0: every eigensolve starts from the identity; N > 0: each
                              clique's Jacobi starts from its eigenvectors of the previous
                              iteration, with a cold start every N iterations          */
    int profile;           /* 1: run the use_graph = 0 path and bracket every projection
                              launch with CUDA events on `stream` (see cdsdp_profile)      */
    int component_stop;    /* Algorithms 1-2 on a problem with independent components
                              (see cdsdp_components): 1 = each component runs its own
                              stopping test and is frozen once it holds, so its result
                              is that of a solve of the component alone; 0 = one test
                              over the whole problem.  HSDE: 1 = one embedding (tau,
                              kappa) and one test per component; 0 = one embedding
                              over the whole problem.                                  */
    int adaptive_rho;      /* Algorithms 1-2: 0 = fixed rho; N > 0 = after every N-th
                              iteration whose stopping test failed, apply the adaptive
                              penalty rule of Section 7.1.2 to (eps_c, eps_lambda):
                              rho *= rho_mu if eps_c >= rho_nu eps_lambda, rho /= rho_mu
                              if eps_lambda >= rho_nu eps_c (per component with
                              component_stop).  The cached factor does not involve rho. */
    double rho_mu;         /* >= 1; the paper's default 2                              */
    double rho_nu;         /* >= 1; the paper's default 10                             */
    int x_update;          /* Algorithm 1, where x = D^-1 (bhat - A^T y) is formed:
                              0 = default (2); 1 = inside the projection's gather,
                              once per clique holding the entry; 2 = a separate
                              kernel over the A^T rows, once per entry             */
    int proj_warps_div;    /* warp-per-clique projections (orders <= 32): warps per
                              block = the kernel's maximum / this (1, 2 or 4)       */
    int linear_solver;     /* Algorithms 1-2, the system (A D^-1 A^T) y = r of Eqs.
                              OptCondMinYPrimal / OptCondMinYDual: 0 = the cached
                              inverse; 1 = conjugate gradient (Section 4.1.1), warm-
                              started from the previous y, stopped once
                              ||r - S y|| <= cg_tol ||r|| or after cg_max_steps steps;
                              runs one stopping test over the whole problem.  HSDE:
                              CDSDP_ERR_UNSUPPORTED.                                  */
    double cg_tol;         /* relative residual tolerance of the CG solve (>= 0)       */
    int cg_max_steps;      /* CG steps per ADMM iteration (0..1024)                    */
    int proj_streams;      /* with component_stop on a problem with independent
                              components: the projection launches of the size classes
                              (and the step of the cliques above order 128) run on this
                              many streams forked from `stream` and joined before the
                              stopping tests, largest work first, so that one class's
                              tail overlaps the next class (1..4; 1 = one after the
                              other on `stream`).  No effect otherwise.  Default 4.   */
    int proj_cta_kernel;   /* float32 projections of padded orders 36..64 (one thread
                              block per clique): 0 = eigenvectors in shared memory,
                              two barriers per Jacobi round; 1 = eigenvectors in
                              registers, one barrier per round (default).  Same
                              rotations and results up to rounding order.            */
    int row_threads;       /* threads per constraint row of the sparse A-row products
                              (A W v): 0 = from the average row length (default), or
                              32, 64, 128, 256.                                       */
} cdsdp_opts;

typedef struct {
    int n, m;
    int p;                   /* number of maximal cliques                           */
    int max_clique;          /* largest |C_k|                                        */
    long long nnz_pattern;   /* lower-triangle entries of the extended pattern E*   */
    long long n_d_lower;     /* sum_k |C_k|(|C_k|+1)/2                               */
    long long nnz_A;         /* stored nonzeros of A after merging duplicates        */
    long long n_fill;        /* fill edges added by the chordal extension            */
    int chordal;             /* 1 if the aggregate pattern was already chordal       */
    int diag_factor;         /* 1 if A D^-1 A^T is diagonal (e.g. MaxCut, Section 4.1.2) */
    long long upload_bytes;  /* size of the one host-to-device copy cdsdp_bind makes   */
    int ncomp;               /* independent components (see cdsdp_components)        */
    int cached_factor;       /* 1 if the inverse of A D^-1 A^T is cached (0 after
                                CDSDP_SETUP_NO_FACTOR)                               */
} cdsdp_info_t;

/* Fill `o` with defaults: eps 1e-4, max_iter 2000, rho 1, FP32 projection,
 * graph on, check_every 50, 30 Jacobi sweeps, warm start with a cold start every
 * 16 iterations, no profiling, per-component stopping, fixed rho (adaptive
 * rule off; rho_mu 2, rho_nu 10 when switched on), x formed by its own
 * kernel, cached inverse (CG tolerance 1e-10 and 50 steps when switched on). */
void cdsdp_default_opts(cdsdp_opts* o);

/* Data preprocessing of Algorithms 1-3 (host only, no GPU call):
 * aggregate sparsity pattern E* of C, every A_i and the optional extra
 * edges P (Section 2.1, Eq. AggregateSparsity), chordal extension and maximal
 * cliques (Section 7.1.1; maximum cardinality search when already chordal,
 * minimum-degree elimination otherwise; cliques sorted lexicographically),
 * the entry selectors H_k (Section 4), D = sum_k H_k^T H_k, and the cached
 * inverses of A D^-1 A^T (Eq. ADMMprimalFatorization) and of
 * I + A (I + D/2)^-1 A^T (Eq. HSDEFactorizationFinal), with
 * zeta_hat (Proposition 2).
 *   n, m        matrix order and number of constraints (n >= 1, m >= 1)
 *   A_*         nnzA triplets (constraint, row, col, value)
 *   b           m values
 *   C_*         nnzC triplets
 *   P_*         nnzP extra pattern edges (may be 0 / NULL)
 *   out         receives the handle
 * Errors: CDSDP_ERR_ARG (bad index, upper entry, non-finite value),
 *         CDSDP_ERR_RANK (A D^-1 A^T not positive definite), CDSDP_ERR_NOMEM. */
int cdsdp_setup(int n, int m,
                long long nnzA, const int* A_con, const int* A_row, const int* A_col, const double* A_val,
                const double* b,
                long long nnzC, const int* C_row, const int* C_col, const double* C_val,
                long long nnzP, const int* P_row, const int* P_col,
                cdsdp** out);

/* Same as cdsdp_setup, on data scaled as Section 7.1.3 describes (host only,
 * no GPU call).  The paper scales the decomposed problem by positive diagonal
 * matrices and two scalars and maps the scaled solution back; the reading used
 * here is a diagonal congruence, which keeps the PSD cone and every clique
 * block:  Abar_i = e_i D A_i D,  bbar = tau E b,  Cbar = sigma D C D,
 * D = diag(d), E = diag(e).  d and e come from scale_passes rounds of symmetric
 * Ruiz equilibration of the A triplets (e_i <- e_i / sqrt(||Abar_i||_F), then
 * d_j <- d_j / sqrt(max |Abar_i(j,k)|), each clipped to [1e-4, 1e4]; both
 * triangles of an off-diagonal entry counted), then tau = 1 / ||E b||_2 and
 * sigma = 1 / ||D C D||_F (1 where the norm is 0).  scale_passes = 0 keeps
 * d = e = 1 and only normalises b and C.
 * Solves on the handle run on the scaled data; cdsdp_solve / cdsdp_results
 * map X, y, Z back on the host (X = D Xbar D / tau, y_i = e_i ybar_i / sigma,
 * Z = D^-1 Zbar D^-1 / sigma) and certificates to the normalisation of an
 * unscaled solve (b^T y = 1, C . X = -1).  The residual history, the
 * per-component residuals and the stopping test are those of the scaled
 * problem.  cdsdp_unrolled_* return CDSDP_ERR_UNSUPPORTED on such a handle.
 * Errors: as cdsdp_setup, and CDSDP_ERR_ARG for scale_passes < 0. */
int cdsdp_setup_scaled(int n, int m,
                       long long nnzA, const int* A_con, const int* A_row, const int* A_col, const double* A_val,
                       const double* b,
                       long long nnzC, const int* C_row, const int* C_col, const double* C_val,
                       long long nnzP, const int* P_row, const int* P_col,
                       int scale_passes, cdsdp** out);

/* Setup flags (cdsdp_setup_flags). */
enum { CDSDP_SETUP_NO_FACTOR = 1, CDSDP_SETUP_MERGE_CLIQUES = 2 };

/* cdsdp_setup (scale_passes < 0) or cdsdp_setup_scaled (scale_passes >= 0)
 * with flags.  CDSDP_SETUP_NO_FACTOR skips the cached inverses of Algorithms
 * 1-3: the m x m blocks and their O(m^3) factorisation, which bound the
 * problem sizes the other paths take (a dense block above 8192 constraints is
 * CDSDP_ERR_UNSUPPORTED there).  Such a handle solves Algorithms 1-2 with
 * opts.linear_solver = 1 (conjugate gradient, Section 4.1.1) only; other
 * solves, the autotuner with the cached inverse and the unrolled passes return
 * CDSDP_ERR_UNSUPPORTED.  Without the factor no rank test of A is made.
 * CDSDP_SETUP_MERGE_CLIQUES replaces the maximal cliques of the extension by a
 * coarser clique cover of a further chordal extension wherever that lowers the
 * projection work sum_k |C_k|^3 (the paper decomposes along whatever chordal
 * extension it is given; this picks a coarser one).  The clique tree is the
 * maximum-weight spanning forest of the clique intersection graph (Kruskal,
 * edges (i < j) in the order weight |C_i ^ C_j| descending, i, j ascending);
 * the tree edge with the largest gain |C_i|^3 + |C_j|^3 - |C_i u C_j|^3 (ties:
 * smaller min(i, j), then max(i, j)) is merged while that gain is positive,
 * node min(i, j) keeping the union and the other node's tree edges; the
 * extended pattern becomes every pair within a merged clique.  It pays where
 * cliques overlap heavily (minimum-degree extensions of random graphs).  A
 * merged handle does not serve cdsdp_completion_sizes / cdsdp_complete
 * (CDSDP_ERR_UNSUPPORTED).
 * Errors: as cdsdp_setup_scaled, and CDSDP_ERR_ARG for an unknown flag. */
int cdsdp_setup_flags(int n, int m,
                      long long nnzA, const int* A_con, const int* A_row, const int* A_col, const double* A_val,
                      const double* b,
                      long long nnzC, const int* C_row, const int* C_col, const double* C_val,
                      long long nnzP, const int* P_row, const int* P_col,
                      int scale_passes, unsigned flags, cdsdp** out);

/* A batch of `count` independent SDPs set up as their direct sum (one handle;
 * each SDP is an independent component, so with opts.component_stop each
 * stops on its own test).  n[j], m[j], nnzA[j], nnzC[j], nnzP[j] (nnzP may be
 * NULL) describe problem j; its triplets follow those of problems 0..j-1 in
 * the concatenated arrays, with indices local to the problem (0-based, lower
 * triangle); b is the concatenation of the b vectors.  The sum numbers the
 * vertices and constraints of problem j after those of problems 0..j-1, so X
 * and Z (pattern order), y and cliques of problem j are contiguous in the
 * results.  scale_passes and flags as cdsdp_setup_flags; with scale_passes >= 0
 * every SDP is scaled as if alone (Section 7.1.3): d and e from the
 * equilibration passes (which act within each SDP), tau_j = 1 / ||E b_j|| and
 * sigma_j = 1 / ||D C_j D||_F of SDP j, so that each SDP's scaled problem,
 * iterates and stopping test are those of a scaled solve of that SDP alone
 * (cdsdp_scaling_batch reports tau_j, sigma_j).  Errors: as cdsdp_setup_flags;
 * CDSDP_ERR_ARG for a local index out of its problem's range. */
int cdsdp_setup_batch(int count, const int* n, const int* m,
                      const long long* nnzA, const int* A_con, const int* A_row, const int* A_col,
                      const double* A_val, const double* b,
                      const long long* nnzC, const int* C_row, const int* C_col, const double* C_val,
                      const long long* nnzP, const int* P_row, const int* P_col,
                      int scale_passes, unsigned flags, cdsdp** out);

/* Scaling factors of a handle (Section 7.1.3): d [n], e [m] (host buffers the
 * caller owns; any may be NULL), tau and sigma (for a scaled batch, those of
 * SDP 0).  A handle made by cdsdp_setup reports d = e = 1, tau = sigma = 1.
 * Errors: CDSDP_ERR_ARG (NULL handle). */
int cdsdp_scaling(const cdsdp* h, double* d, double* e, double* tau, double* sigma);

/* tau and sigma of every SDP of a scaled batch (cdsdp_setup_batch with
 * scale_passes >= 0, Section 7.1.3): *count (may be NULL) receives the number
 * of SDPs (1 for any other handle), tau [count] and sigma [count] (host
 * buffers the caller owns, large enough for the batch; may be NULL) the
 * factors; ones for an unscaled handle.  Errors: CDSDP_ERR_ARG (NULL handle). */
int cdsdp_scaling_batch(const cdsdp* h, int* count, double* tau, double* sigma);

/* Maximum-determinant positive definite completion (Section 7.1.1) of a
 * partial matrix X on the handle's extended pattern E* (the X that
 * cdsdp_solve returns).  The completion W is the unique positive definite
 * matrix with W = X on E* and (W^-1)_ij = 0 off E*; it exists exactly when
 * every clique block of X is positive definite.  It is computed along a
 * perfect elimination order of E* (Vandenberghe and Andersen, Chapter 10.2).
 * The output holds one dense row-major n_c x n_c block per independent
 * component c of the handle (cdsdp_components), rows and columns in
 * ascending vertex order, block c at element offset w_offsets[c]; entries
 * between components are zero and not stored.
 *
 * cdsdp_completion_sizes (host only):
 *   scratch_bytes  device scratch that cdsdp_complete needs
 *   w_elems        doubles of the dense output (sum of n_c^2)
 *   w_offsets      [ncomp + 1] element offsets of the blocks (may be NULL)
 * cdsdp_complete:
 *   d_X        device, nnz_pattern doubles in cdsdp_pattern order
 *   d_scratch  device, scratch_bytes, 256-byte aligned, caller-owned
 *   d_W        device, w_elems doubles (may be NULL: factor and log det only)
 *   logdet     host [ncomp], log det of each block (may be NULL)
 *   stream     CUDA stream; the call synchronises it once (to read the
 *              positive-definiteness flag) and returns with the dense
 *              blocks queued on it.
 * Returns CDSDP_SOLVED, CDSDP_NOT_PD (d_W and logdet untouched),
 * CDSDP_ERR_ARG (NULL or misaligned pointer), CDSDP_ERR_NOMEM (scratch too
 * small), CDSDP_ERR_UNSUPPORTED (largest clique above order 160), CDSDP_ERR_CUDA. */
int cdsdp_completion_sizes(const cdsdp* h, size_t* scratch_bytes, long long* w_elems, long long* w_offsets);
int cdsdp_complete(cdsdp* h, const double* d_X, void* d_scratch, size_t scratch_bytes, double* d_W, double* logdet,
                   void* stream);

int cdsdp_info(const cdsdp* h, cdsdp_info_t* info);

/* Maximal cliques in canonical order: offsets[p+1], vertices[offsets[p]],
 * each clique ascending (Section 2.1, natural ordering). */
int cdsdp_cliques(const cdsdp* h, int* offsets, int* vertices);

/* Extended pattern E*, lower triangle incl. diagonal, column-major order:
 * rows[nnz_pattern], cols[nnz_pattern].  X and Z are returned in this order. */
int cdsdp_pattern(const cdsdp* h, int* rows, int* cols);

/* Independent components: connected components of the extended pattern in
 * which every constraint also joins the vertices it touches.  A direct sum of
 * SDPs (a batch of independent problems given as one block-diagonal problem)
 * has one component per summand; A D^-1 A^T is then block diagonal and the
 * library caches one dense inverse block per component.  Components are
 * numbered by their smallest vertex.
 *   vertex_comp      [n] component of each vertex (may be NULL)
 *   constraint_comp  [m] component of each constraint (may be NULL)
 * Host only, valid right after cdsdp_setup. */
int cdsdp_components(const cdsdp* h, int* vertex_comp, int* constraint_comp);

/* Per-component outcome of the last solve (each output may be NULL):
 *   iters   [ncomp] iterations the component ran
 *   status  [ncomp] its outcome (CDSDP_SOLVED, CDSDP_MAX_ITER, CDSDP_ERR_NUMERIC)
 *   res     [ncomp x 8] its last stopping-test row (columns as in cdsdp_solve's hist)
 * When the last solve ran one test over the whole problem (component_stop = 0,
 * HSDE, or a single component) every component reports the global values.
 * Errors: CDSDP_ERR_STATE before the first solve. */
int cdsdp_component_results(cdsdp* h, void* stream, int* iters, int* status, double* res);

/* Device workspace the caller must provide for solves of up to max_iter
 * iterations (history included). */
int cdsdp_workspace_bytes(const cdsdp* h, int max_iter, size_t* bytes);

/* Attach a caller-owned device workspace (>= cdsdp_workspace_bytes, 256-byte
 * aligned) and upload the preprocessed problem into it with one host-to-device
 * copy on `stream`.  The workspace must stay allocated until cdsdp_free or the
 * next cdsdp_bind.  Errors: CDSDP_ERR_NOMEM (too small), CDSDP_ERR_ARG
 * (misaligned), CDSDP_ERR_CUDA. */
int cdsdp_bind(cdsdp* h, void* d_workspace, size_t bytes, int max_iter, void* stream);

/* Run Algorithm 1, 2 or 3 on the bound workspace from zero initial guesses
 * (HSDE: u = (0,..,0,1), v = (0,..,0,1)) until the stopping test of the form
 * holds or max_iter iterations.  Blocks until the solve is done.
 * Host outputs (each may be NULL):
 *   X     [nnz_pattern] primal solution on E* (pattern order)
 *   y     [m]           dual multipliers
 *   Z     [nnz_pattern] dual slack on E*
 *   hist  [iters x 8]   per-iteration residuals, row-major:
 *         primal/dual: eps_c, eps_lambda, rho, 0, <C,X>, b^T y, 0, 0
 *         HSDE tau>0:  eps_p, eps_d, eps_g, eps_c, <C,X>, b^T y, tau, kappa
 *         HSDE tau=0:  ||A^T u_y + H^T v_z||, ||A u_x||, b^T u_y, c^T u_x, 0, 0, tau, kappa
 *   iters number of iterations run (with per-component stopping: the largest
 *         over the components; hist then holds, per iteration, the largest
 *         eps_c and eps_lambda over the components tested, the summed
 *         objectives and, in column 6, the number of components still running)
 *   cert  HSDE certificate: [m] (primal infeasible) or [nnz_pattern] (dual
 *         infeasible); must hold max(m, nnz_pattern) doubles
 * Returns the outcome (CDSDP_SOLVED, CDSDP_MAX_ITER, CDSDP_*_INFEASIBLE) or
 * an error (CDSDP_ERR_STATE if no workspace is bound, CDSDP_ERR_NUMERIC on
 * NaN/Inf, CDSDP_ERR_CUDA). */
int cdsdp_solve(cdsdp* h, int form, const cdsdp_opts* opts, void* stream,
                double* X, double* y, double* Z, double* hist, int* iters, double* cert);

/* Kernel timings of the last solve run with opts.profile = 1:
 *   proj_ms       summed duration of the projection launches (CUDA events on
 *                 the solve's stream), over the iterations actually run
 *   proj_launches number of projection launches summed
 *   iter_ms       summed duration of whole iterations
 * Errors: CDSDP_ERR_STATE when the last solve was not profiled. */
int cdsdp_profile(const cdsdp* h, double* proj_ms, int* proj_launches, double* iter_ms);

/* Per size class of the projection kernels, for the last solve run with
 * opts.profile = 1 (not in the paper; measurement).  Cliques are bucketed by
 * padded order, one launch per non-empty class and iteration; each launch is
 * bracketed by CUDA events on the solve's stream.  Arrays of
 * CDSDP_PROJ_CLASSES entries, any of them may be NULL:
 *   orders         padded order of the class
 *   ms             total device time of its launches over the profiled iterations
 *   launches       its launches over the profiled iterations
 *   cliques        cliques in the class
 *   nominal_flops  sum over its cliques of 10 s^3 (9 s^3 for a symmetric
 *                  eigendecomposition with vectors, s^3 for the rebuild;
 *                  Golub and Van Loan, Section 8.3): the algorithmic work of
 *                  one launch
 * Errors: CDSDP_ERR_ARG, CDSDP_ERR_STATE when the last solve was not profiled. */
#define CDSDP_PROJ_CLASSES 22
int cdsdp_profile_orders(const cdsdp* h, int* orders, double* ms, int* launches, int* cliques, double* nominal_flops);

/* The cliques of order > 128 in the last profiled solve (opts.profile = 1):
 * their projection step (gather, sign iteration on the tensor cores, state
 * update, sums) bracketed by CUDA events once per iteration.  Any pointer may
 * be NULL.
 *   ms             total device time over the profiled iterations
 *   launches       iterations timed
 *   cliques        cliques of order > 128
 *   nominal_flops  sum of 10 s^3 over those cliques (the same nominal count as
 *                  cdsdp_profile_orders)
 *   tensor_flops   tensor-core work of one step: 59 products x 3 TF32 MMAs over
 *                  the lower 128 x 128 tiles of each padded block (2 flops per
 *                  multiply-add)
 * Errors: CDSDP_ERR_ARG, CDSDP_ERR_STATE when the last solve was not profiled. */
int cdsdp_profile_large(const cdsdp* h, double* ms, int* launches, int* cliques, double* nominal_flops,
                        double* tensor_flops);

/* Measured FMA throughput of the current GPU, the peak against which the
 * projection kernels (bound by the FP32, or FP64, FMA pipe) are reported.  Not
 * in the paper.  One launch of register-resident independent FMA chains over
 * every SM (8 blocks of 256 threads each), timed with CUDA events on `stream`
 * after a warm-up launch; flops = 2 x FMAs.
 *   precision  CDSDP_FP32_PROJECTION (float FMA) or CDSDP_FP64 (double FMA)
 *   iters      chain steps per thread (>= 1; about 10^5 for float and 2 x 10^4
 *              for double give launches of a few milliseconds)
 *   tflops     out: TFLOP/s
 * Synchronises `stream`.  Errors: CDSDP_ERR_ARG, CDSDP_ERR_CUDA. */
int cdsdp_fma_peak(int precision, int iters, void* stream, double* tflops);

/* Schedule autotuner (not in the paper; the launch schedule is a GPU choice):
 * times `iters` iterations (no early stop; graph or not as in opts) of `form`
 * for each candidate schedule and writes into *tuned a copy of *opts (the
 * defaults when opts is NULL) with the fastest candidate's fields:
 *   x_update        1 or 2 (Algorithm 1 only)
 *   proj_warps_div  1, 2 or 4
 *   warm_start      16 or 64 (only when opts->warm_start > 0)
 *   proj_streams    4 or 1
 *   proj_cta_kernel 0 or 1 (one more candidate: the fastest of the above with
 *                   the other value)
 *   row_threads     64, 128, 256 (three more candidates: the fastest of the
 *                   above with each value)
 * ms_per_iter[] receives each candidate's device time per iteration in
 * candidate order (at most 28 entries; may be NULL), *n_cand their number (may
 * be NULL).  Overwrites the last solve's state.  Errors as cdsdp_solve. */
int cdsdp_autotune(cdsdp* h, int form, const cdsdp_opts* opts, int iters, void* stream, cdsdp_opts* tuned,
                   double* ms_per_iter, int* n_cand);

/* Copy the last solve's results again (same meaning as in cdsdp_solve). */
int cdsdp_results(cdsdp* h, void* stream, double* X, double* y, double* Z, double* hist, double* cert);

int cdsdp_free(cdsdp* h);

const char* cdsdp_strerror(int status);

/* Standalone batched PSD projection P(W) = V max(Lambda, 0) V^T
 * (Section 4.1.2, Eq. XkUpdate) of p symmetric blocks, one warp per block
 * (block size <= 32) or one thread block per block (33..128).
 *   d_off[p+1]    offsets of each block's lower-packed storage (int32)
 *   d_size[p]     block orders s_k (1..128)
 *   d_W           lower-packed inputs, column-major within a block:
 *                 entry (a, b), a >= b, at d_off[k] + b*(2 s_k - b + 1)/2 + (a - b)
 *   d_X           lower-packed outputs, same layout (may alias d_W)
 *   d_eig         optional [sum_k s_k] eigenvalues (block k at its vertex
 *                 offset d_voff[k]); NULL to skip
 *   d_V           optional [sum_k s_k^2] eigenvectors, column-major per block
 *                 at d_vvoff[k]; NULL to skip
 *   d_voff/d_vvoff offsets for d_eig / d_V (int32, p entries); NULL if unused
 *   precision     CDSDP_FP32_PROJECTION: float data; CDSDP_FP64: double data
 * Errors: CDSDP_ERR_ARG (p < 0, size out of range), CDSDP_ERR_CUDA. */
int cdsdp_psd_project(int p, const int* d_off, const int* d_size, int max_size,
                      const void* d_W, void* d_X, void* d_eig, const int* d_voff, void* d_V, const int* d_vvoff,
                      int precision, int max_sweeps, void* stream);

/* Differentiation through unrolled Algorithm 1 (not in the paper).  The map
 * (c, b) -> x_N runs `iters` iterations of Algorithm 1 from the zero start
 * with the bound problem's A, cliques and cached factor but with the data c
 * (lower pattern order, nnz_pattern values, the off-diagonal value standing
 * for both entries) and b (m values) given on the device.  The forward stores
 * the clique state every `ckpt_every` iterations in the caller-owned device
 * buffer d_gws (cdsdp_grad_workspace_bytes); the backward replays each
 * segment from its checkpoint, recording the projection inputs, and runs the
 * reverse pass: the Daleckii-Krein adjoint of every clique projection on the
 * GPU (eigenpairs recomputed by the same Jacobi), the linear steps transposed.
 * Warm start is off and the solve never stops early, so the replay repeats
 * the forward bit for bit.  Only opts->rho, precision and jacobi_max_sweeps
 * are used.  Cliques of order > 32 return CDSDP_ERR_UNSUPPORTED; ckpt_every
 * must not exceed the bound max_iter.
 *   d_x     out [nnz_pattern] x_N (device)
 *   d_xbar  [nnz_pattern] dL/dx_N in the same coordinates (device)
 *   d_cbar  out [nnz_pattern] dL/dc;  d_bbar  out [m] dL/db (device)
 * The backward must follow a forward with the same arguments and d_gws. */
int cdsdp_grad_workspace_bytes(const cdsdp* h, int iters, int ckpt_every, int precision, size_t* bytes);
int cdsdp_unrolled_forward(cdsdp* h, const cdsdp_opts* opts, int iters, int ckpt_every, const double* d_c,
                           const double* d_b, void* d_gws, size_t gws_bytes, double* d_x, void* stream);
int cdsdp_unrolled_backward(cdsdp* h, const cdsdp_opts* opts, int iters, int ckpt_every, const double* d_c,
                            const double* d_b, void* d_gws, size_t gws_bytes, const double* d_xbar, double* d_cbar,
                            double* d_bbar, void* stream);

/* PSD projection of large blocks (order 129 .. 8192) on the tensor cores
 * (Section 4.1.2, Eq. XkUpdate, for cliques too large for one thread block's
 * Jacobi eigensolver).  P(W) = (W + W sign(W)) / 2 with sign(W) from an odd
 * polynomial (Newton-Schulz) iteration on W / ||W||_F: 16 steps of
 * X <- 3.30 X - 3.66 X^3 + 1.36 X^5, then 5 steps of X <- 1.5 X - 0.5 X^3,
 * every product of two (commuting, symmetric) matrices as three TF32
 * tcgen05 products (float32 accuracy), lower 128 x 128 tiles only.
 * Eigenvalues with |lambda| < 1e-8 ||W||_F may stay unconverged; each adds at
 * most |lambda| / 2 to the error of P.
 *   p        number of blocks
 *   h_size   [p] host: orders, 1 .. 8192
 *   h_off    [p] host: offset (elements) of each block's packed lower values
 *            (column-major lower packed, as in cdsdp_psd_project)
 *   d_W      device float32: input blocks;  d_X  device float32: P(W_k), same layout
 *   d_scratch  device scratch, 256-byte aligned, at least
 *            cdsdp_psd_project_large_bytes(p, h_size) bytes: the tensor maps
 *            of the iteration and ten dense float copies of every block
 *            (order rounded up to a multiple of 128)
 * Synchronises `stream`.  Errors: CDSDP_ERR_ARG, CDSDP_ERR_NOMEM (scratch too
 * small), CDSDP_ERR_CUDA (also when the driver's tensor-map encoder is
 * unavailable), CDSDP_ERR_TIMEOUT (a bounded wait inside the product kernel
 * ran out; the results are then invalid). */
int cdsdp_psd_project_large_bytes(int p, const int* h_size, size_t* bytes);
int cdsdp_psd_project_large(int p, const int* h_size, const long long* h_off, const float* d_W, float* d_X,
                            void* d_scratch, size_t scratch_bytes, void* stream);

/* PSD-violation measure of Section 7.2 (Eq. PSD-violation):
 *   alpha = -min{0, lambda_min(W_0), ..., lambda_min(W_{p-1})}
 * over p lower-packed symmetric blocks (layout and orders as in
 * cdsdp_psd_project; order <= 32).  With W_k = mat(H_k x) this is the bound
 * alpha in the paper's eps_alpha = alpha / (1 + ||X||_F).  One kernel: one warp
 * per block, per-thread-block minima in d_scratch, final reduction by the last
 * thread block.
 *   d_scratch  caller-owned device scratch, 256-byte aligned, at least
 *              cdsdp_psd_violation_scratch_bytes(p) bytes; its first word is
 *              cleared on `stream` before the launch
 *   d_alpha    device pointer receiving alpha (one double)
 * Asynchronous on `stream`.  Errors: CDSDP_ERR_ARG (p < 1, max_size outside
 * 1..32, misaligned scratch), CDSDP_ERR_NOMEM (scratch too small),
 * CDSDP_ERR_CUDA.  The orders in d_size are device data: if any lies outside
 * 1..max_size, alpha is written as NaN (no error code, the call is
 * asynchronous). */
size_t cdsdp_psd_violation_scratch_bytes(int p);
int cdsdp_psd_violation(int p, const int* d_off, const int* d_size, int max_size, const void* d_W, int precision,
                        int max_sweeps, void* d_scratch, size_t scratch_bytes, double* d_alpha, void* stream);

/* cdsdp_psd_violation for callers that cannot allocate device memory.  The
 * paper has no counterpart; this exists for callers that cannot call
 * cudaMalloc when they need the measure: code running inside a framework whose
 * caching allocator owns the device memory (a raw cudaMalloc there would
 * fragment or overcommit the pool it manages), a plugin whose host hands it
 * only input and output buffers, or a real-time loop that forbids the latency
 * and possible failure of an allocation.  Same arguments,
 * result and errors as cdsdp_psd_violation, minus the scratch: the scratch is
 * a fixed 1 MiB array inside the library, present on every GPU that loads it
 * until the process exits.  Limit: p <= 524160 blocks (131040 thread blocks of
 * 4); larger p returns CDSDP_ERR_UNSUPPORTED.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) and should therefore
 * come before any stream capture on that device.  Every call shares the array
 * and clears its counter word on `stream` before launching; calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * the array and must be serialised by the caller.  Allocates nothing: no
 * cudaMalloc, cudaFree or allocating library routine.  The array's device
 * address is kept for the life of the process: do not call this entry point on
 * a device after cudaDeviceReset (the library's module is loaded again there,
 * at a new address). */
int cdsdp_psd_violation_noalloc(int p, const int* d_off, const int* d_size, int max_size, const void* d_W,
                                int precision, int max_sweeps, double* d_alpha, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CDSDP_H */
