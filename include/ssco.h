/*
 * ssco.h -- C ABI of the fixed-pattern assemble / refactor / solve / adjoint
 * library for one GB300 (sm_103a).
 *
 * The setting is the paper's "compile once for a fixed structure, evaluate
 * for many value sets" (Sec. 3.3, requirement 2; Sec. 4.3 grouping of
 * structurally equal expressions by dependency level; Sec. 4.4 leaf tables
 * with uniform vs varying constants; Sec. 4.8 index arrays p, constants c,
 * consecutive outputs, coalesced layouts).  The fixed structure here is the
 * sparsity pattern of K = A^T diag(w) A + shift*I (or K = sum_e E_e K_e^0,
 * the tagged element blocks of Sec. 4.2.4); the evaluated program is the
 * assembly of K, its Cholesky factorization K~ = P K P^T = L L^T and the two
 * triangular solves, plus their adjoint.
 *
 * Conventions shared by every entry point
 *  - Every call returns an ssco_status; nothing throws across the ABI.
 *    ssco_last_error(plan) returns a message for the last failing call.
 *  - The caller owns every array it passes.  ssco_analyze copies what it
 *    needs; the library owns the host plan until ssco_destroy.
 *  - ALL device memory is caller-allocated: ssco_plan_info reports the
 *    sizes of the table buffer and the workspace, ssco_bind attaches them.
 *    The library never calls cudaMalloc.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *    Calls are asynchronous on it except where a comment says otherwise.
 *  - Batched values are INSTANCE-OUTERMOST: an array "[B][n]" holds value set
 *    b at offset b*n.  Several patterns in one plan are concatenated: their
 *    unknowns (and values) follow each other in pattern order.
 *  - A "system" is one (instance b, pattern k) pair, index b*n_pats + k.
 *  - A plan and its workspace must not be used on two streams at once.
 */
#ifndef SSCO_H
#define SSCO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SSCO_OK = 0,
    SSCO_ERR_INVALID_ARG = 1,  /* NULL pointer, bad size, bad enum          */
    SSCO_ERR_PATTERN = 2,      /* index out of range, bad rowptr, bad perm  */
    SSCO_ERR_NOT_SPD = 3,      /* a pivot was not > 0 (per system)          */
    SSCO_ERR_NONFINITE = 4,    /* NaN/Inf in values or right-hand side      */
    SSCO_ERR_NO_CONVERGE = 5,  /* refinement hit its cap or stagnated       */
    SSCO_ERR_TIMEOUT = 6,      /* a bounded device wait gave up (all systems) */
    SSCO_ERR_CUDA = 7,         /* a CUDA runtime call failed                */
    SSCO_ERR_OOM = 8,          /* a caller buffer is smaller than required  */
    SSCO_ERR_UNSUPPORTED = 9,  /* request outside what the library supports  */
    SSCO_ERR_STATE = 10        /* call order violated (e.g. solve unbound)  */
} ssco_status;

enum { SSCO_KIND_ATWA = 0, SSCO_KIND_ELEM = 1, SSCO_KIND_ELEM_BLOCKS = 2 };
enum { SSCO_FP64 = 0, SSCO_FP32_REFINE = 1 };
enum { SSCO_VALS_F64 = 0, SSCO_VALS_F32 = 1 };

typedef struct ssco_plan_s* ssco_plan;

/* One fixed sparsity structure.
 * kind = SSCO_KIND_ATWA:  K = A^T diag(w) A + shift*I.  A is m x n in CSR
 *   (rowptr[m+1] int64, colind[nnz] int32 in [0,n), aval[nnz] constant
 *   entries, e.g. +-1 for an incidence matrix).  The per-call values are w[m].
 *   Every diagonal of K receives the shift.
 * kind = SSCO_KIND_ELEM:  K = sum_e E_e K_e^0 over m elements.  elem_dofs
 *   [m][elem_dim] lists each element's global DOF (or -1 for a fixed DOF);
 *   elem_K0 [m][elem_dim*(elem_dim+1)/2] holds K_e^0 as a row-major packed
 *   lower triangle (i >= j).  The per-call values are E[m].  A DOF that no
 *   element references becomes an identity row/column (K_ii = 1); every
 *   referenced DOF's diagonal receives the shift.
 * kind = SSCO_KIND_ELEM_BLOCKS:  K = sum_e K_e with the element blocks
 *   themselves supplied per call: the per-call values are
 *   K_e [m][elem_dim*(elem_dim+1)/2] (row-major packed lower triangles, the
 *   layout of elem_K0, which is ignored), so the value count per set is
 *   m*elem_dim*(elem_dim+1)/2 (must stay below 2^31).  Entries on a fixed
 *   DOF (-1) are dropped; identity rows and the shift as for ELEM.  The
 *   element blocks may come from geometry on the device (ssco_tet_stiffness),
 *   which makes the mesh positions, not only the moduli, the per-call input.
 * perm[n] (perm[new] = old) is the fill-reducing order; NULL = natural.
 *   It must be a permutation of [0,n) (else SSCO_ERR_PATTERN).          */
typedef struct {
    int32_t kind;
    int32_t n;
    int32_t m;
    const int64_t* rowptr;
    const int32_t* colind;
    const double* aval;
    int32_t elem_dim;
    const int32_t* elem_dofs;
    const double* elem_K0;
    const int32_t* perm;
} ssco_pattern;

/* Options of the numeric phase.
 * precision: SSCO_FP64 factors and solves in FP64.  SSCO_FP32_REFINE factors
 *   in FP32 and refines in FP64: r = b - K x with the FP64 K, d = solve32(r),
 *   x += d, until ||r||_2 <= refine_tol*||b||_2, refine_max_iter iterations,
 *   or stagnation (||r|| not halved over two iterations).
 * batch: value sets per pattern (1 .. 65535).
 * small_front_max: fronts with more rows than this use the multi-CTA dense
 *   path (0 = default for the precision).
 * amalgamate: 0 = fundamental supernodes only; 1 = relaxed amalgamation of
 *   a front into its parent when the merge adds few explicit zeros
 *   (numeric partition only; exported structures stay exact).
 * tiny_front_max: subtrees whose fronts all have at most this many rows
 *   (<= 32) are factored and solved by one warp each, front in registers,
 *   in a single launch (0 = default 32, -1 = off).
 * tensor_cores: 0 = FP32 updates of multi-CTA fronts run on the tcgen05
 *   tensor cores (3xTF32), one CTA per 128 x 128 tile; 2 = the wide
 *   trailing updates in persistent CTAs (one per SM, two TMEM
 *   accumulators); -1 = SIMT FP32 only.
 * big_panel: columns of a multi-CTA front factored between two trailing
 *   updates (a multiple of 32 in [32, 1024]; 0 = default 256).
 * split_rows: fronts with at least this many rows (and more than
 *   small_front_max) are solved by multi-CTA launches over 256-column
 *   blocks (0 = default: 1024 with >= 8 value sets, else 2048; -1 = never).
 * warp_front_max: small fronts of at most this many rows (<= 64) are
 *   factored one warp per front on levels that supply at least 8 warps per
 *   SM (0 = default off; ssco_autotune may switch it on).
 * cluster_rows: fronts with at least this many rows (below split_rows)
 *   are solved by one 8-CTA thread-block cluster per value set
 *   (0 = default: 512 with <= 4 value sets, else never; -1 = never).
 * refine_mode (SSCO_FP32_REFINE): 0 = the plain refinement above; 1 =
 *   GMRES-IR: each correction solves K d = r by restarted GMRES in FP64,
 *   right-preconditioned by the FP32 factor (d = sum_i y_i M^-1 v_i with
 *   M = L L^T applied as two FP32 triangular solves), until the GMRES
 *   residual estimate falls by 1e-4 or gmres_restart steps; 2 = plain
 *   refinement first, then GMRES-IR for the systems where it stagnated or
 *   ran out of iterations (each phase has refine_max_iter corrections).  A
 *   plan with refine_mode != 0 holds 2*gmres_restart + 1 more FP64 vectors
 *   [B][n] in its workspace; its ssco_graph_run runs the eager calls (it
 *   synchronizes `stream`).  There the FP32 factor is only a preconditioner:
 *   a non-positive FP32 pivot is replaced by 1 and reported in bad_col, and
 *   the system's status is the refinement's (OK once the FP64 residual met
 *   refine_tol), not SSCO_ERR_NOT_SPD.
 * gmres_restart: Krylov vectors per GMRES-IR correction (1 .. 64; 0 =
 *   default 16).
 * vec2_max_cls (SSCO_FP32_REFINE): small-front size classes above the
 *   four-value-set classes and up to this many rows are factored two value
 *   sets per CTA (0 = default off; 128 or 160; ssco_autotune may switch it
 *   on).  */
typedef struct {
    int32_t precision;
    int32_t batch;
    double refine_tol;
    int32_t refine_max_iter;
    int32_t small_front_max;
    int32_t amalgamate;
    int32_t tiny_front_max;
    int32_t tensor_cores;
    int32_t big_panel;
    int32_t split_rows;
    int32_t warp_front_max;
    int32_t cluster_rows;
    int32_t refine_mode;
    int32_t gmres_restart;
    int32_t vec2_max_cls;
} ssco_op;

/* Sizes and counts of an analyzed plan (all for the concatenated system). */
typedef struct {
    int64_t n;               /* unknowns (sum over patterns)                 */
    int64_t n_pats;
    int64_t batch;
    int64_t n_systems;       /* batch * n_pats                               */
    int64_t m;               /* values per instance (sum over patterns)      */
    int64_t nnz_K;           /* lower triangle of K incl. diagonal           */
    int64_t nnz_L;           /* structural nonzeros of L incl. diagonal      */
    int64_t n_snodes;        /* fundamental supernodes                       */
    int64_t n_fronts;        /* supernodes of the numeric partition          */
    int64_t n_levels;        /* levels of the numeric supernodal forest      */
    int64_t max_col_level;   /* height of the column elimination forest      */
    int64_t panel_entries;   /* stored factor entries (per instance)         */
    int64_t update_entries;  /* stored update-matrix entries (per instance)  */
    int64_t max_front_rows;
    int64_t n_assembly_groups;
    int64_t assembly_terms;  /* total terms in the assembly leaf tables      */
    int64_t tables_bytes;    /* device table buffer size                     */
    int64_t workspace_bytes; /* device workspace size                        */
    double factor_flops;     /* sum_j c_j^2 over the numeric partition       */
    double factor_flops_exact; /* sum_j c_j^2 over the exact structure       */
    int64_t tune_warp_items; /* launch-shape knobs (see ssco_autotune)       */
    int64_t tune_vec_max_cls;
    int64_t tune_solve_threads_big;
    int64_t tuned;           /* 1 after a successful ssco_autotune           */
    int64_t tune_use_tc;     /* 1: FP32 big-front updates on tensor cores    */
    int64_t tune_big_panel;  /* big fronts: columns per trailing update      */
    int64_t tune_split_rows; /* fronts this large take the multi-CTA solves  */
    int64_t tune_warp_front_max; /* small-front classes factored warp-per-front */
    int64_t tune_cluster_rows;   /* fronts this large: one CTA cluster per solve */
    int64_t tune_flow;           /* persistent dataflow launches: bit 0 solve sweeps,
                                    bit 1 small-front factorization; bit 2 the panel
                                    core for per-level small fronts; bit 3 big-front
                                    steps with the diagonal factor fused; bit 4 no solve
                                    graphs (ssco_set_flow)                           */
    int64_t flow_fact_fronts;    /* fronts factored by the dataflow launches         */
    int64_t flow_solve_fronts;   /* fronts solved by the dataflow sweeps             */
    int64_t tune_vec2_max_cls;   /* FP32 classes above tune_vec_max_cls up to this
                                    size: two value sets per CTA (0 = none)          */
} ssco_info;

/* ssco_plan_export selectors (host copies; sizes in elements).          */
enum {
    SSCO_EXPORT_PERM = 0,        /* int32 [n]     concatenated perm (new->old) */
    SSCO_EXPORT_ETREE = 1,       /* int32 [n]     parent column, -1 = root     */
    SSCO_EXPORT_COLCOUNT = 2,    /* int32 [n]     nnz of each column of L      */
    SSCO_EXPORT_L_COLPTR = 3,    /* int64 [n+1]                                */
    SSCO_EXPORT_L_ROWIND = 4,    /* int32 [nnz_L] rows ascending per column    */
    SSCO_EXPORT_COL_LEVEL = 5,   /* int32 [n]     height in the column forest  */
    SSCO_EXPORT_SNODE_FIRST = 6, /* int32 [n_snodes+1] fundamental supernodes  */
    SSCO_EXPORT_SN_PARENT = 7,   /* int32 [n_snodes]                           */
    SSCO_EXPORT_SN_LEVEL = 8,    /* int32 [n_snodes] height in the sn forest   */
    SSCO_EXPORT_K_COLPTR = 9,    /* int64 [n+1]   pattern of K~ (lower, CSC)   */
    SSCO_EXPORT_K_ROWIND = 10,   /* int32 [nnz_K]                              */
    SSCO_EXPORT_GROUPS = 11,     /* int64 [n_assembly_groups][4]: members,     */
                                 /*   terms, coefficient mode (0 varying,      */
                                 /*   1 uniform), diagonal flag                */
    SSCO_EXPORT_GROUP_COEF = 12, /* double [n_assembly_groups]: the uniform     */
                                 /*   constant (0 for varying groups)          */
    SSCO_EXPORT_FRONT_FIRST = 13,/* int32 [n_fronts+1] numeric partition       */
    SSCO_EXPORT_FRONT_LEVEL = 14 /* int32 [n_fronts]                           */
};

/* Symbolic phase (host only, no GPU needed).  Validates every pattern,
 * builds K~'s pattern and the assembly leaf tables grouped by (term count,
 * uniform/varying constant, diagonal) [Sec. 4.3, 4.4, App. B], the
 * elimination forest, column counts, fundamental supernodes, level sets by
 * height, the numeric front partition and all index tables.
 * Errors: SSCO_ERR_INVALID_ARG, SSCO_ERR_PATTERN. */
ssco_status ssco_analyze(const ssco_pattern* const* pats, int32_t n_pats, const ssco_op* op,
                         ssco_plan* out);
ssco_status ssco_plan_info(ssco_plan plan, ssco_info* out);
/* Copies one exported structure into host_buf (bytes must be >= its size,
 * else SSCO_ERR_OOM).
 * No counterpart in the paper: it exposes the host phase's structures to
 * tests and tools. */
ssco_status ssco_plan_export(ssco_plan plan, int32_t what, void* host_buf, size_t bytes);

/* Attaches caller-allocated device memory: dev_tables (>= tables_bytes,
 * 256-byte aligned) receives the index tables (copied on `stream`);
 * dev_workspace (>= workspace_bytes, 256-byte aligned) holds K, the factor,
 * update matrices, vectors and status words.  Re-binding is allowed.
 * The device copy of the harvested tables that every grouped launch reads
 * (Sec. 4.4, 4.8). */
ssco_status ssco_bind(ssco_plan plan, void* dev_tables, size_t tables_bytes, void* dev_workspace,
                      size_t workspace_bytes, void* stream);

/* Defined by: the assembly K = A^T diag(w) A + shift*I (or the element-block
 * sum of Sec. 4.2.4) evaluated through the grouped leaf tables of Sec. 4.3
 * and 4.4, then the Cholesky factor P K P^T = L L^T by its textbook
 * definition (the paper factors nothing itself: Sec. 5.5 and 5.6 time an
 * external sparse factorization of such systems), scheduled as the level
 * groups of Sec. 4.3.
 * Numeric phase: assemble K from vals (device, [B][m], dtype
 * SSCO_VALS_F64/F32) and shift (device, double [n_systems]), then factor.
 * Asynchronous.  A non-positive pivot is recorded per system (read it with
 * ssco_status_get), never branched on. */
ssco_status ssco_numeric(ssco_plan plan, const void* vals, int32_t vals_dtype, const double* shift,
                         void* stream);

/* Defined by: forward substitution L y = P b and back substitution
 * L^T z = y, x = P^T z, with the factor of ssco_numeric, level by level in
 * the order of Sec. 4.3 (reversed for L^T); the FP32 form adds iterative
 * refinement in FP64, which the paper does not use.
 * x = K^-1 b for every system (device, double [B][n] each; b and x may not
 * alias).  Asynchronous.  In SSCO_FP32_REFINE mode the refinement loop runs
 * on the device as a captured CUDA graph with a conditional WHILE node,
 * captured on the first call for a (b, x) pointer pair (two pairs are kept)
 * and replayed afterwards; make that first call outside any stream capture
 * of your own.  With refine_mode != 0 (GMRES-IR), or while per-launch
 * profiling is on, the loop is host-driven and the call synchronizes
 * `stream`. */
ssco_status ssco_solve(ssco_plan plan, const double* b, double* x, void* stream);

/* Defined by: the reverse-mode derivative of x = K^-1 b (the derivatives
 * the paper obtains by symbolic differentiation of expression graphs, Sec.
 * 4.9, written out by hand for this program: one more solve with the same
 * factor, then one product per value).
 * Adjoint of x = K(vals, shift)^-1 b for a scalar loss with dloss/dx = xbar:
 * mu = K^-1 xbar (same factor, same refinement), then
 *   vals_bar_e = -(A mu)_e (A x)_e            (ATWA)
 *   vals_bar_e = -mu_e^T K_e^0 x_e            (ELEM, free DOFs)
 *   vals_bar_(e,r,s) = -(mu_u x_v + mu_v x_u), r > s; -mu_u x_u, r = s
 *                 (ELEM_BLOCKS: u, v the global DOFs of local r, s; 0 on
 *                  an entry with a fixed DOF)
 *   shift_bar  = -mu^T x over shifted diagonals, per system
 *   b_bar      = mu.
 * Device arrays: x, xbar, b_bar [B][n]; vals_bar [B][m]; shift_bar
 * [n_systems] (may be NULL).  Its solve behaves like ssco_solve's (a
 * captured graph for FP32 plans with plain refinement, keyed by xbar and
 * the workspace's adjoint vector). */
ssco_status ssco_backward(ssco_plan plan, const double* x, const double* xbar, double* vals_bar,
                          double* shift_bar, double* b_bar, void* stream);

/* Synchronizes `stream`, then copies per-system results to host arrays
 * (any may be NULL): status (ssco_status codes), iters (refinement
 * iterations of the last solve), resid (||b - K x||_2 / ||b||_2 of the last
 * solve, FP64), bad_col (first non-positive pivot in permuted numbering,
 * -1 if none).  Returns SSCO_OK or the worst system status.
 * Per-system outcome of the repeated evaluation (Sec. 3.3); the status
 * words have no counterpart in the paper. */
ssco_status ssco_status_get(ssco_plan plan, void* stream, int32_t* status, int32_t* iters,
                            double* resid, int32_t* bad_col);

/* Synchronizes `stream`, then writes the factor in the CSC order of
 * SSCO_EXPORT_L_ROWIND to the HOST array host_out, as double [B][nnz_L].
 * No counterpart in the paper: it copies a computed result out for
 * checking. */
ssco_status ssco_export_L(ssco_plan plan, double* host_out, void* stream);
/* Synchronizes `stream`, then writes K~ in the CSC order of
 * SSCO_EXPORT_K_ROWIND to the HOST array host_out, double [B][nnz_K].
 * No counterpart in the paper: it copies a computed result out for
 * checking. */
ssco_status ssco_export_K(ssco_plan plan, double* host_out, void* stream);

/* Autotuner of the launch shapes of the level groups: for each knob (the
 * item count from which a solve level runs warp-per-(front, instance), the
 * largest front size class factored several value sets per CTA, the CTA size
 * of solve levels with wide fronts, tensor cores on or off for the FP32
 * trailing updates of big fronts) every candidate is timed on the caller's
 * data (median of `reps` numeric + solve steps, CUDA events) and the fastest
 * is kept in the plan (saved by ssco_plan_save).  Synchronizes `stream`;
 * leaves a valid factor and solution (x) behind.  *best_ms (may be NULL)
 * receives the best step time.
 * No counterpart in the paper, which fixes launch shapes when it generates
 * code (App. F); here they are timed on the caller's data. */
ssco_status ssco_autotune(ssco_plan plan, const void* vals, int32_t vals_dtype, const double* shift, const double* b,
                          double* x, int32_t reps, void* stream, double* best_ms);

/* Dataflow launches (Sec. 4.3's level groups, scheduled by dependency).
 * The fronts below every big front are factored, and the fronts of at most
 * 256 rows solved, by persistent launches that walk all their levels: each
 * front (per value set) is an item taken in level order from a ticket
 * counter, and it waits only for the done flags of its children (factor,
 * forward sweep) or of its parent (backward sweep), never for a whole level.
 * flow: bit 0 the solve sweeps, bit 1 the factorization (default 3; 0 = one
 * launch per level and size class); bit 2: the per-level launches of small
 * fronts (those outside the dataflow) use the dataflow kernel's dense core
 * (a 16-column panel per three barriers) instead of the column-step
 * kernels; bit 3: big fronts factor each 32-column step's diagonal block
 * inside the triangular-solve launch (every CTA of the step factors it in
 * shared memory; the factor reaches the panel one step later), so only a
 * level's last step has a separate one-warp factor launch -- the same
 * arithmetic, so the same factor; bit 4: ssco_solve of an FP32 plan launches
 * its kernels one by one instead of replaying its cached solve graph (for
 * profilers that do not see kernels inside graphs; the call then
 * synchronizes once per refinement step).  max_polls bounds every wait (polls of
 * about 256 ns; 0 = keep the current bound, default 2^22): a wait that runs
 * out raises the plan's device error, the launch ends early and
 * ssco_status_get reports SSCO_ERR_TIMEOUT for every system (the results of
 * that call are invalid).  stall_item >= 0 is a test hook: that item of the
 * first dataflow launch of each numeric (else of each forward sweep) waits
 * on a flag that nothing sets, so the bounded wait runs out; -1 = off.
 * Host only; invalidates the captured graph of ssco_graph_run. */
ssco_status ssco_set_flow(ssco_plan plan, int32_t flow, int64_t max_polls, int32_t stall_item);

/* ssco_numeric + ssco_solve as ONE CUDA graph: the refinement loop runs on
 * the device as a conditional WHILE node (no host round trip per
 * iteration).  The graph is captured (on library-owned streams) on the first
 * call for this (vals, shift, b, x, workspace) tuple and replayed by later
 * calls with the same pointers; new pointers or ssco_bind re-capture.  Call
 * it outside any stream capture of your own.  Asynchronous on `stream`.
 * The same evaluation replayed for every new value set (Sec. 3.3); the CUDA
 * graph itself has no counterpart in the paper. */
ssco_status ssco_graph_run(ssco_plan plan, const void* vals, int32_t vals_dtype, const double* shift, const double* b,
                           double* x, void* stream);

/* ssco_graph_run over several plans as ONE CUDA graph: each plan's
 * assemble + refactor + solve (with its own device-side refinement loop)
 * is an independent branch of the graph, so the latency-bound levels of one
 * plan overlap the work of the others (e.g. many value sets on one pattern
 * beside single instances of patterns of uneven size).  Array arguments
 * have one entry per plan, as for ssco_graph_run.  The graph is held by
 * plans[0] and re-captured when a plan, a pointer or a dtype changes, or
 * after anything that releases a plan's graphs (ssco_bind, ssco_autotune,
 * ssco_set_flow).  No plan may appear twice; call it outside any stream
 * capture of your own.  Asynchronous on `stream`.
 * Several independent patterns' evaluations in one replay (Sec. 4.3
 * grouping across patterns); no counterpart in the paper as a call. */
ssco_status ssco_graph_run_many(const ssco_plan* plans, int32_t n_plans, const void* const* vals,
                                const int32_t* vals_dtype, const double* const* shift, const double* const* b,
                                double* const* x, void* stream);

/* ssco_autotune for the plans of one ssco_graph_run_many step: coordinate
 * descent (two sweeps over the plans) over each plan's dataflow choices
 * (the bits of ssco_set_flow 0..3 and the two-value-set classes of FP32
 * plans), every candidate timed on the multi-plan graph itself (median of
 * `reps` replays after a warm-up; kept when 0.5 % faster than the current
 * setting, re-timed beside each knob's candidates).  A plan's best choice
 * alone can differ from its
 * best choice beside the others, whose work it overlaps with (Sec. 4.3's
 * grouping decided across the patterns of a step).  Arguments as for
 * ssco_graph_run_many; run ssco_autotune on each plan first for its other
 * knobs.  Leaves valid results in x; *best_ms (may be NULL) receives the
 * best step time. */
ssco_status ssco_autotune_many(const ssco_plan* plans, int32_t n_plans, const void* const* vals,
                               const int32_t* vals_dtype, const double* const* shift, const double* const* b,
                               double* const* x, int32_t reps, void* stream, double* best_ms);

/* End-to-end call on HOST buffers: copies vals/shift/b to the device
 * (staging areas inside the workspace), runs numeric + solve as the captured
 * graph of ssco_graph_run, copies x back and synchronizes.  Host arrays use
 * the same layouts as above.
 * No counterpart in the paper: the host-buffer wrapper around
 * ssco_graph_run. */
ssco_status ssco_refactor_solve_host(ssco_plan plan, const void* vals, int32_t vals_dtype,
                                     const double* shift, const double* b, double* x, void* stream);

/* Allocation-free variant of ssco_solve for SSCO_FP64 plans.  The paper has
 * no counterpart; it exists for callers that must not allocate device
 * memory per call, for example a host application whose memory manager owns
 * every device allocation, or a latency-critical loop where a cudaMalloc /
 * cudaFree would synchronize the device.  It computes x = K^-1 b (device,
 * double [B][n] each, no aliasing) with the factor left in the bound
 * workspace by ssco_numeric, by direct forward/back substitution (no
 * refinement, no status words; ssco_status_get does not report it).  Its
 * scratch -- the permuted right-hand side, the solve vector and the
 * passing vectors, 2*B*n + B*(sum over fronts of rows-width) doubles -- lives
 * in one static device array of 64 MiB that every GPU loading the library
 * keeps until the process exits; plans needing more are rejected with
 * SSCO_ERR_UNSUPPORTED and a message giving both sizes.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (every
 * word is written before it is read, so nothing needs clearing): calls that
 * overlap on the GPU, on any stream or plan, race.  Calls no cudaMalloc,
 * cudaFree or other allocating routine. */
ssco_status ssco_solve_noalloc(ssco_plan plan, const double* b, double* x, void* stream);

/* Value construction upstream of assembly (no plan): cotangent edge weights
 * of a planar triangle mesh from vertex positions, per value set (the
 * cotangent Laplacian of Sec. 5.3's mesh experiments):
 *   w[b][e] = 1/2 * sum over the triangles holding edge e of
 *             cot(angle opposite e),  cot = (u . v) / |u x v|,
 * u, v the two edges leaving that corner (unsigned area, so weights may be
 * negative on obtuse angles).  All pointers are device pointers:
 *   tri      [n_tri][3] int32 vertex ids;
 *   tri_edge [n_tri][3] int32 id of the edge opposite each corner;
 *   xy       [batch][n_vert][2] double positions;
 *   w        [batch][n_edge] double, overwritten.
 *   n_bad    optional device int32: incremented once per triangle whose
 *            vertex or edge ids are out of range (such triangles are
 *            skipped, never dereferenced); may be NULL.
 * Each edge must belong to at most two triangles (then the result does not
 * depend on summation order); a degenerate triangle gives non-finite
 * weights (the numeric phase then reports SSCO_ERR_NONFINITE).  Async on
 * `stream`; returns SSCO_ERR_INVALID_ARG for inconsistent sizes or null
 * pointers, SSCO_ERR_CUDA if the launch fails. */
ssco_status ssco_cotan_weights(const int32_t* tri, const int32_t* tri_edge, int64_t n_tri, int64_t n_vert,
                               int64_t n_edge, int32_t batch, const double* xy, double* w, int32_t* n_bad,
                               void* stream);

/* Value construction upstream of assembly (no plan): stiffness blocks of
 * linear tetrahedra from vertex positions, per value set -- the element
 * blocks of the 3D elasticity configurations, for SSCO_KIND_ELEM_BLOCKS
 * patterns whose geometry changes per call.  For tet t with vertices
 * x_0..x_3 (local DOF 3a+c = component c of vertex a), J = [x_1-x_0,
 * x_2-x_0, x_3-x_0], V = |det J|/6, g_a = grad of the barycentric
 * coordinate of vertex a (rows of J^-1; g_0 = -(g_1+g_2+g_3)), and the
 * isotropic Lame constants lambda = E nu/((1+nu)(1-2nu)), mu = E/(2(1+nu)):
 *   K_t[3a+i][3b+j] = V (lambda g_a[i] g_b[j] + mu g_a[j] g_b[i]
 *                        + mu [i==j] g_a . g_b),
 * which equals V B^T D B of the strain-displacement matrix B and the
 * isotropic D (Voigt order, engineering shear).  All pointers are device
 * pointers:
 *   tets   [n_tet][4] int32 vertex ids;
 *   xyz    [batch][n_node][3] double positions;
 *   E      [batch][n_tet] double Young's moduli, or NULL for E = 1;
 *   K_e    [batch][n_tet][78] double, overwritten: the lower triangle of
 *          K_t packed row-major (entry (r, s), r >= s, at r(r+1)/2 + s);
 *   n_bad  optional device int32: incremented once per tet with an
 *          out-of-range vertex id and once per (tet, value set) with a zero
 *          or non-finite det J; such blocks are written as zeros and the ids
 *          are never dereferenced; may be NULL.
 * nu must lie in (-1, 0.5).  Async on `stream`; returns
 * SSCO_ERR_INVALID_ARG for inconsistent sizes, nu or null pointers,
 * SSCO_ERR_CUDA if the launch fails.
 * No counterpart in the paper: it builds, from vertex positions, the per-
 * call element blocks that SSCO_KIND_ELEM_BLOCKS patterns take (the element
 * form of Sec. 4.2.4). */
ssco_status ssco_tet_stiffness(const int32_t* tets, int64_t n_tet, int64_t n_node, int32_t batch, const double* xyz,
                               const double* E, double nu, double* K_e, int32_t* n_bad, void* stream);

/* ---------------------------------------------------------------------------
 * Fixed-pattern sparse matrix expressions (the paper's method applied to
 * sparse algebra, Sec. 4 and the sparse-expression experiments of Sec. 5):
 * a DAG of sparse matrices with fixed patterns is unrolled once on the host
 * into scalar expressions (every entry of a product or sum), structurally
 * identical scalar expressions are merged (hashing), each is assigned the
 * level = longest path from the leaves, and the level groups with their
 * harvested index tables are run by one gather-multiply-accumulate kernel
 * per level, for `batch` value sets at once.
 *
 * Node ids are positions in the node array; operands must come earlier.
 *   LEAF       a rows x cols CSR pattern (rowptr[rows+1] int64, colind
 *              int32 strictly increasing within each row); its values are
 *              supplied per call.  With vmap (int64 [nnz], values in
 *              [0, n_vals)) entry q takes the leaf's value vmap[q], so
 *              entries may share one value (a symmetric matrix stored once);
 *              the leaf then supplies n_vals values.  NULL vmap: one value
 *              per entry.
 *   ADD        a + b (same shape; pattern = union).
 *   SCALE      alpha * a.
 *   MUL        a * b (a.cols == b.rows; pattern = structural product).
 *   TRANSPOSE  a^T.
 * Every entry of a MUL, and (unless inlined, see inline_terms) every entry
 * of an ADD present in both operands, is stored once as an intermediate (a
 * global intermediate in the paper's terms) unless its canonical form is a
 * multiple of one slot or zero (A + A, A - A); scaling and transposition
 * only relabel entries.  The products of
 * an entry are summed in ascending order of their factor slots, after equal
 * factor pairs are merged (coefficients added) and zero coefficients
 * dropped; values are float or double (`precision` = SSCO_VALS_F64 /
 * SSCO_VALS_F32) and accumulate in that type.
 * Leaf values per set are the leaves' values (nnz each, or n_vals with a
 * vmap) concatenated in node order ([batch][n_leaf_vals]); outputs likewise ([batch][n_out_vals], in the
 * order of `outputs`, each in its CSR order). */
typedef struct ssco_expr_s* ssco_expr;
enum { SSCO_EXPR_LEAF = 0, SSCO_EXPR_ADD = 1, SSCO_EXPR_SCALE = 2, SSCO_EXPR_MUL = 3, SSCO_EXPR_TRANSPOSE = 4 };
typedef struct {
    int32_t op;            /* SSCO_EXPR_* */
    int32_t a, b;          /* operand node ids (-1 where unused) */
    double alpha;          /* SCALE factor */
    int32_t rows, cols;    /* LEAF shape */
    const int64_t* rowptr; /* LEAF pattern (host; copied by compile) */
    const int32_t* colind;
    const int64_t* vmap;   /* LEAF: value of each entry, or NULL (host) */
    int64_t n_vals;        /* LEAF with vmap: number of distinct values */
} ssco_expr_node;
typedef struct {
    int64_t n_leaf_vals;   /* values per set: all leaves' nnz */
    int64_t n_out_vals;    /* values per set: all outputs' nnz */
    int64_t n_slots;       /* 1 (the constant one) + leaf values + stored intermediates */
    int64_t n_ops;         /* stored intermediates (scalar expressions) */
    int64_t n_terms;       /* products over all of them */
    int64_t n_unrolled;    /* scalar expressions before hashing and relabelling */
    int32_t n_levels;
    int32_t batch;
    int32_t precision;
    int32_t unit_coef;     /* 1: every coefficient is 1 (no coefficient table) */
    uint64_t table_bytes;  /* device tables (ssco_expr_bind) */
    uint64_t workspace_bytes;
    /* what the optional steps of ssco_expr_compile_opts did (0 after load) */
    int64_t n_alg_merged;  /* expressions replaced by a multiple of an equal slot */
    int64_t n_alg_zero;    /* expressions found equal to zero */
    int64_t n_factored;    /* factorization steps */
    int64_t n_inlined;     /* linear intermediates substituted into their users */
} ssco_expr_info;
enum { SSCO_EXPR_EXPORT_LEVELS = 0,   /* int64 [n_levels+1] op ranges */
       SSCO_EXPR_EXPORT_TERM_OFF = 1, /* int64 [n_ops+1] */
       SSCO_EXPR_EXPORT_F1 = 2,       /* int32 [n_terms] first factor slot */
       SSCO_EXPR_EXPORT_F2 = 3,       /* int32 [n_terms] second factor slot (0 = the constant one) */
       SSCO_EXPR_EXPORT_COEF = 4,     /* double [n_terms] */
       SSCO_EXPR_EXPORT_OUT_SLOT = 5, /* int32 [n_out_vals] slot of each output value */
       SSCO_EXPR_EXPORT_OUT_COEF = 6  /* double [n_out_vals] its factor */ };

/* Host only.  inline_terms (0..16) chooses between storing and inlining a
 * sum (the paper's global / local decomposition): 0 stores every entry of a
 * sum present in both operands; k > 0 keeps a sum of at most k slot
 * multiples local instead, and the products that use it expand over its
 * terms (at most k x k products per factor pair), so fewer intermediates
 * and levels are stored at the cost of more products.
 * Slot layout: slot 0 = 1, slots 1..n_leaf_vals = leaf values,
 * then the intermediates of level 1, 2, ... (op i is slot
 * 1 + n_leaf_vals + i).  Returns INVALID_ARG / PATTERN for malformed nodes
 * (message in ssco_expr_last_error(NULL)), UNSUPPORTED beyond int32 slots.
 * The paper's method on sparse matrix expressions: unrolling, hashing,
 * levels and leaf harvesting (Sec. 4.1-4.4, App. A). */
ssco_status ssco_expr_compile(const ssco_expr_node* nodes, int32_t n_nodes, const int32_t* outputs, int32_t n_out,
                              int32_t batch, int32_t precision, int32_t inline_terms, ssco_expr* out);

/* ssco_expr_compile with the optional steps of the method (all off = 0,
 * which gives ssco_expr_compile's tables byte for byte).  Host only.
 *   algebraic   1: algebraic hashing (Sec. 4.1.2, App. A).  Every slot gets
 *               the value of its polynomial in the leaf variables at three
 *               seeded points of the field of integers mod 2^61 - 1
 *               (coefficients, finite doubles, map there exactly).  An
 *               expression whose values are all zero is dropped (the entry
 *               becomes 0, App. D "constant expressions"; with this op set
 *               no other constant can arise); one whose values are c times
 *               an existing slot's -- c a double confirmed exactly in the
 *               field -- becomes c times that slot (so (A+B)C and AC+BC,
 *               or the mirror entries of a symmetric product, are stored
 *               once).  Two different polynomials of degree d are merged
 *               with probability at most (d / (2^61 - 1))^3.
 *   factor_min  0 or >= 2: factorization (App. D).  While a slot is a factor
 *               of at least factor_min products of one sum, the slot shared
 *               by the most is taken out: its partners' sum is stored as a
 *               linear expression (hashed like any other) and those
 *               products become one.
 *   t_ref, t_compl  global decomposition (Sec. 4.2.1; 0 and 0 = off).  A
 *               linear intermediate (a sum of slot multiples) that is no
 *               output and is referenced fewer than t_ref times or has
 *               fewer than t_compl terms is not stored: its terms are
 *               substituted into the products that use it.  Products stay
 *               stored (substituting one would give three-factor terms).
 * Fraction reduction and square-root elimination (App. D) have nothing to
 * act on: the node set has no division and no roots.  These steps change
 * the order of the arithmetic (the paper notes the same): results agree
 * with the plain tables up to rounding, not bit for bit.  reserved must be
 * 0.  Errors as ssco_expr_compile, INVALID_ARG for options out of range. */
typedef struct {
    int32_t batch, precision, inline_terms; /* as in ssco_expr_compile */
    int32_t algebraic;                      /* 0 / 1 */
    int32_t factor_min;                     /* 0, or >= 2 */
    int32_t t_ref, t_compl;                 /* >= 0 */
    int32_t reserved;                       /* 0 */
} ssco_expr_opts;
ssco_status ssco_expr_compile_opts(const ssco_expr_node* nodes, int32_t n_nodes, const int32_t* outputs,
                                   int32_t n_out, const ssco_expr_opts* opts, ssco_expr* out);
ssco_status ssco_expr_get_info(ssco_expr e, ssco_expr_info* out);
ssco_status ssco_expr_export(ssco_expr e, int32_t what, void* host_buf, uint64_t bytes);
/* Shape and CSR pattern of the k-th output (rowptr [rows+1], colind [nnz]).
 * No counterpart in the paper: describes an output's pattern for the
 * caller. */
ssco_status ssco_expr_output_shape(ssco_expr e, int32_t k, int32_t* rows, int32_t* cols, int64_t* nnz);
ssco_status ssco_expr_output_pattern(ssco_expr e, int32_t k, int64_t* rowptr, int32_t* colind);
/* Caller-allocated device memory of table_bytes / workspace_bytes (256-byte
 * aligned); the tables are copied with `stream`, which is synchronized.
 * The device copy of the harvested tables (Sec. 4.4, 4.8). */
ssco_status ssco_expr_bind(ssco_expr e, void* dev_tables, void* dev_workspace, void* stream);
/* Evaluates every set: leaf_vals [batch][n_leaf_vals] and out_vals
 * [batch][n_out_vals] device arrays of the program's precision.  Async;
 * launches 2 + n_levels kernels on `stream`.
 * One launch per dependency level of grouped expressions (Sec. 4.3). */
ssco_status ssco_expr_run(ssco_expr e, const void* leaf_vals, void* out_vals, void* stream);
/* Versioned file of a compiled program (host tables only; digest-checked
 * like plan files).  Load refuses another version, damage, and tables that
 * index outside the program's slots; the caller owns the returned program
 * and binds it as after compile.
 * No counterpart in the paper: a compiled program kept on disk. */
ssco_status ssco_expr_save(ssco_expr e, const char* path);
ssco_status ssco_expr_load(const char* path, ssco_expr* out);
const char* ssco_expr_last_error(ssco_expr e);
void ssco_expr_destroy(ssco_expr e);

/* Number of kernel launches the last ssco_numeric / ssco_solve /
 * ssco_backward / ssco_refactor_solve_host call issued (host counter).
 * No counterpart in the paper: instrumentation. */
int64_t ssco_last_launch_count(ssco_plan plan);

/* Per-kernel timing.  ssco_profile_enable(plan, max_launches) creates a pool
 * of 2*max_launches CUDA events (0 releases it and turns profiling off);
 * while on, every kernel launch is bracketed by events on its own stream
 * and its algorithmic work (flops, bytes) is recorded.  Launches beyond the
 * pool are not recorded.  ssco_profile_read synchronizes the device, sums
 * the records by kernel kind into out[SSCO_K_COUNT] and clears them. */
enum {
    SSCO_K_ASSEMBLE = 0,     /* assembly gather-MAC over the leaf tables      */
    SSCO_K_FRONT_SMALL = 1,  /* one-CTA front factorization in shared memory  */
    SSCO_K_BIG_INIT = 2,     /* big front: pull children's update matrices    */
    SSCO_K_BIG_KSCATTER = 3, /* big front: add K entries                      */
    SSCO_K_BIG_GEMM = 4,     /* big front: right-looking trailing update       */
    SSCO_K_BIG_POTRF = 5,    /* big front: 32x32 diagonal block Cholesky      */
    SSCO_K_BIG_SYRK = 6,     /* (unused; kept for numbering)                  */
    SSCO_K_FWD = 7,          /* forward solve, one level                      */
    SSCO_K_BWD = 8,          /* backward solve, one level                     */
    SSCO_K_RESID = 9,        /* FP64 residual b - K x                         */
    SSCO_K_CHECK = 10,       /* per-system norms and refinement decision      */
    SSCO_K_VECTOR = 11,      /* permutations, casts, updates, status fills    */
    SSCO_K_GRAD = 12,        /* adjoint reductions                            */
    SSCO_K_FRONT_TINY = 13,  /* warp-per-subtree factorization, tiny fronts   */
    SSCO_K_BIG_TRSM = 14,    /* big front: rows below the diagonal block      */
    SSCO_K_FRONT_VEC = 15,   /* small fronts, V value sets per CTA            */
    SSCO_K_BIG_UPDATE_TC = 16, /* big front: trailing update on tcgen05 (3xTF32) */
    SSCO_K_COUNT = 17
};
typedef struct {
    int32_t kind;
    int32_t reserved;
    int64_t launches;
    double ms;     /* summed event time of the recorded launches */
    double flops;  /* summed algorithmic floating-point operations */
    double bytes;  /* summed algorithmic bytes moved              */
} ssco_kernel_stat;
ssco_status ssco_profile_enable(ssco_plan plan, int32_t max_launches);
ssco_status ssco_profile_read(ssco_plan plan, ssco_kernel_stat* out);
/* Per-launch trace: synchronizes the device and copies up to `cap` records
 * in launch order (kind, milliseconds, flops, bytes; any array may be NULL)
 * WITHOUT clearing them; *n receives the number of records held.
 * No counterpart in the paper: instrumentation. */
ssco_status ssco_profile_trace(ssco_plan plan, int32_t* kinds, float* ms, double* flops, double* bytes,
                               int64_t cap, int64_t* n);
const char* ssco_kernel_name(int32_t kind);

const char* ssco_last_error(ssco_plan plan);
const char* ssco_status_string(ssco_status s);

/* Versioned binary file of the host plan (no device state): magic, version,
 * the plan's tables, then a 64-bit FNV-1a digest of everything before it.
 * Load returns SSCO_ERR_INVALID_ARG for another version, a truncated file,
 * trailing bytes, a digest mismatch, or launch lists whose size fields
 * (largest rows, width, tiles) differ from the fronts they list or that point
 * outside the front tables; the caller owns the returned plan.  The digest
 * detects damage, not tampering: beyond these checks the tables are trusted,
 * so load only files that ssco_plan_save wrote.
 * No counterpart in the paper: the host phase's result kept on disk, so
 * that it runs once per pattern (Sec. 3.3). */
ssco_status ssco_plan_save(ssco_plan plan, const char* path);
ssco_status ssco_plan_load(const char* path, ssco_plan* out);
void ssco_destroy(ssco_plan plan);

#ifdef __cplusplus
}
#endif
#endif /* SSCO_H */
