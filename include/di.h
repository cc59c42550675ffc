/*
 * di.h — C ABI of the GB300 (sm_103a) D-iteration library.
 *
 * The library solves X = P.X + B (paper: "Revisiting the D-iteration method: runtime
 * comparison", Section 1) for a directed graph given as an edge list. P has d / out_j at (i, j)
 * for every distinct link j -> i (Section 2.4: column j of P holds the out-links of j, row i
 * the in-links of i); a dangling column (out_j = 0) is zero. B >= 0. With B = (1-d)/N this is
 * the unnormalised PageRank equation; with B = (1-d)/|S| on a seed set S it is personalised
 * PageRank.
 *
 * Conventions shared by every entry point
 *   - Pointers: every array argument may be host memory (pageable or pinned) or device memory
 *     of the graph's GPU; the library asks the CUDA runtime which one it is. The caller owns
 *     every array it passes and keeps it alive for the duration of the call. A graph handle owns
 *     its graph arrays; solve scratch is either allocated by the library on first use or laid
 *     out in a workspace the caller attaches (di_workspace_size, di_graph_set_workspace).
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     All device work of a call is ordered on that stream. Every call returns only after its
 *     results are written (it synchronises the stream before returning).
 *   - Errors: every call returns a di_status; DI_OK is 0. On error, di_last_error() returns a
 *     human-readable message for the calling thread. No call aborts the process.
 *   - Threads: calls on different graphs may run concurrently. Calls that use the same graph's
 *     solve workspace (di_solve*, di_power_iter, di_solve_batch, di_ppr_batch) are serialised
 *     by the graph; a call that finds the workspace busy returns DI_ERR_BUSY.
 */
#ifndef DI_GB300_H
#define DI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct di_graph di_graph;

typedef enum {
    DI_OK = 0,
    DI_ERR_INVALID_ARG = 1,      /* bad size, d outside [0,1), tol <= 0, B < 0 or not finite */
    DI_ERR_OUT_OF_RANGE_ID = 2,  /* an edge id outside [0, n_nodes) */
    DI_ERR_OOM = 3,              /* device or host allocation failed */
    DI_ERR_CUDA = 4,             /* a CUDA runtime call failed */
    DI_ERR_NOT_CONVERGED = 5,    /* the sweep cap was reached; outputs hold the current state */
    DI_ERR_BUSY = 6,             /* the graph's workspace is in use by another thread */
    DI_ERR_TIMEOUT = 7,          /* a bounded wait ran out */
    DI_ERR_CORRUPT = 8           /* di_csr_validate / di_graph_validate found an inconsistency */
} di_status;

/* Node selection rule of a sweep (Section 2.3). */
typedef enum {
    DI_CYC = 0,   /* visit every node with F_i != 0 */
    DI_SOP = 1    /* visit node i when |F_i| > (r / L) * out_i, r = ||F||_1 at the sweep start */
} di_schedule;

/* Storage of the fluid F. H, the residual and r are FP64 in both. */
typedef enum {
    DI_FLUID_F32 = 0,
    DI_FLUID_F64 = 1
} di_fluid;

/* Graph statistics (Section 2.4 notation). */
typedef struct {
    int64_t n_nodes;
    int64_t L;          /* distinct links, self-loops included */
    int64_t D;          /* dangling nodes (out-degree 0) */
    int64_t E;          /* recursively zero-in-degree nodes */
    int64_t O;          /* loop nodes (p_ii != 0) */
    int32_t max_in;
    int32_t max_out;
    int32_t e_levels;   /* 1 + largest peeling level in E (0 when E is empty) */
    int32_t reserved;
} di_graph_stats;

/* Options of di_solve_ex / di_solve_batch / di_ppr_batch. Zero-initialise, then set fields;
 * a zero field means "default". */
typedef struct {
    int32_t schedule;    /* di_schedule; default DI_CYC (0) */
    int32_t fluid;       /* di_fluid; default DI_FLUID_F32 (0) */
    int32_t max_sweeps;  /* cap on sweeps; <= 0: 100000; clamped to 1000000 */
    int32_t refine;      /* 0: default (on for F32, off for F64); 1: on; -1: off. Refinement
                            recomputes the exact FP64 residual F* = B + P.H - H and continues
                            sweeping from it until ||F*||_1 <= tol (at most 4 rounds). An FP32
                            solve refines first where ||F||_1 reaches sqrt(tol * ||F_0||_1),
                            before the FP32 rounding has grown comparable to tol, then at the
                            end. */
    int32_t host_loop;   /* 1: drive sweeps from the host (one sync per sweep) instead of a CUDA
                            graph WHILE node; default 0 */
    int32_t rhs_tile;    /* batched solves: RHS per tile, 4, 8, 16 or 32 (0: autotuned per graph) */
    int32_t profile;     /* 1: host-driven sweeps with CUDA events around every kernel launch;
                            fills the per-kernel times of di_solve_info (slower: one sync per
                            sweep). Batched solves time their select, push and reduce kernels */
    int32_t e_prediffuse;/* di_solve_ex only; 1: before the sweeps, visit every node of E once in
                            level order (Section 2.4: E converges in finitely many steps). Each
                            node of E then holds its exact value, up to rounding, and receives no
                            fluid afterwards, so no sweep selects it again. Default 0. */
    int32_t r_refresh;   /* single-RHS DI-SOP: a sweep selects in this many consecutive parts of
                            the node range (0 or 1: one part), and r = ||F||_1 is taken again
                            before each part, so a part's threshold sees the fluid that the parts
                            before it pushed (Section 2.3 takes r_n' once per cycle; this is the
                            variant that refreshes it within the cycle). At most 16. */
    int32_t exact_r;     /* single-RHS FP32 solves: 1 takes r from a sum of |F| after every sweep.
                            Default 0: while r is far above tol and the fluid is nonnegative, r is
                            tracked as the sum before the sweep less the fluid its visits absorbed,
                            with an exact sum every 8th sweep and at every sweep near tol. */
} di_solve_opts;

/* Per-solve report. */
typedef struct {
    int32_t sweeps;          /* sweeps (or PI iterations) executed */
    int32_t refine_rounds;   /* exact-residual recomputations */
    int64_t pushed_edges;    /* sum of out_i over visited nodes (PI: L * iterations) */
    int64_t visited_nodes;   /* node diffusions */
    double residual_l1;      /* ||F||_1 at exit (after refinement: exact FP64 ||F*||_1);
                                PI: ||X_k - X_(k-1)||_1 */
    double dangling_mass_e;  /* e = sum of H over dangling nodes (Section 2.5 DI-CYC) */
    double paper_error;      /* residual / (1 - d - d e), the paper's normalised error */
    double ms;               /* device time of the solve (CUDA events), copies excluded */
    int64_t kernel_launches; /* kernels of this library launched by the call */
    int64_t frontier_entries;/* nodes handed to the push kernel (visited nodes with out-links) */
    /* per-kernel device time and launch counts; filled only when opts.profile = 1
       (refine_* also holds the initialisation and the E pre-diffusion kernels;
       PI: push_* is the pull kernel, select_* the heavy-row pre-pass) */
    double select_ms, push_ms, reduce_ms, refine_ms;
    int32_t select_launches, push_launches, reduce_launches, refine_launches;
    int32_t rhs_tile;        /* batched solves: columns per tile that were used */
    int32_t e_visits;        /* visits of the E pre-diffusion (opts.e_prediffuse) */
    int64_t column_links;    /* batched solves: link-column updates the push made (for every
                                diffusion of a node in a column with a non-zero share, the
                                node's pushed links); 0 for single solves */
} di_solve_info;

/* Which internal array di_graph_export copies. */
typedef enum {
    DI_ARR_ROWPTR_OUT = 0,   /* int64[n+1]: out-CSR row pointers (column view of P, l_out) */
    DI_ARR_COL_OUT = 1,      /* int32[L]:   destinations, ascending within each row */
    DI_ARR_ROWPTR_IN = 2,    /* int64[n+1]: in-CSR row pointers (row view of P, l_in) */
    DI_ARR_COL_IN = 3,       /* int32[L]:   origins, ascending within each row */
    DI_ARR_OUT_DEG = 4,      /* int32[n] */
    DI_ARR_IN_DEG = 5,       /* int32[n] */
    DI_ARR_LOOP = 6,         /* uint8[n]:   1 when the node links to itself */
    DI_ARR_E_MASK = 7,       /* uint8[n]:   1 when the node is in E */
    DI_ARR_E_LEVEL = 8       /* int32[n]:   peeling level in E, -1 outside E */
} di_array;

/*
 * di_graph_create — iterator build ("Init", Section 2.1; Section 2.5 out[], in[], l_out,
 * l_in; Section 2.4 L, D, E, O, max_in, max_out).
 *   n_nodes   number of nodes, 1 .. 2^31-1.
 *   src, dst  int32[n_edges]: link src[e] -> dst[e]. Host or device memory. Any order;
 *             duplicates are dropped (a link counts once in L and in the degrees).
 *   n_edges   0 .. 2^31-1.
 *   out       receives a new graph handle owned by the caller (free with di_graph_destroy).
 *             The handle owns its device arrays; they live on the device current at the call.
 * Errors: DI_ERR_INVALID_ARG (sizes, NULL), DI_ERR_OUT_OF_RANGE_ID (the message names the first
 * bad edge), DI_ERR_OOM, DI_ERR_CUDA. On error *out is set to NULL.
 */
di_status di_graph_create(int32_t n_nodes, const int32_t *src, const int32_t *dst, int64_t n_edges,
                          void *stream, di_graph **out);

/* Releases the graph and its device memory. NULL is ignored. */
void di_graph_destroy(di_graph *g);

/* Copies the statistics of Section 2.4 into *out. */
di_status di_graph_stats_get(const di_graph *g, di_graph_stats *out);

/*
 * di_graph_export — copies one internal array (see di_array for type and length) into dst,
 * host or device memory of at least `capacity_bytes`. Errors: DI_ERR_INVALID_ARG when `which`
 * is unknown or the buffer is too small.
 */
di_status di_graph_export(const di_graph *g, int32_t which, void *dst, int64_t capacity_bytes,
                          void *stream);

/*
 * di_solve — D-iteration (Section 2.3 DI-CYC / DI-SOP, Section 2.5): H = 0, F = B, then sweeps
 * until ||F||_1 <= tol. A sweep takes r = ||F||_1, selects nodes by `schedule` (a DI-SOP sweep
 * that selects nothing is followed by a DI-CYC sweep), and diffuses every selected node: H_i
 * gains transit = F_i (F_i * out_i / (out_i - d) for a loop node), F_i becomes 0 and every
 * out-neighbour j != i gains d * transit / out_i. Selected nodes diffuse concurrently, so the
 * trajectory differs from the sequential one; the fixed point X = lim H does not.
 *   B          double[n]: right-hand side, >= 0 and finite.
 *   d          damping, 0 <= d < 1.   tol > 0: stop when ||F||_1 <= tol.
 *   X_out      double[n]: receives H (the approximation of X; ||X - H||_1 <= residual/(1-d)).
 *   residual_out (nullable) receives info.residual_l1.   info (nullable) receives the report.
 * Uses FP32 fluid with refinement (see di_solve_opts); di_solve_ex takes explicit options.
 * Errors: DI_ERR_INVALID_ARG, DI_ERR_NOT_CONVERGED (X_out and the residual still hold the
 * current state), DI_ERR_BUSY, DI_ERR_OOM, DI_ERR_CUDA.
 */
di_status di_solve(di_graph *g, const double *B, double d, double tol, int32_t schedule,
                   int32_t max_sweeps, double *X_out, double *residual_out, di_solve_info *info,
                   void *stream);

/* di_solve with explicit options (opts may be NULL for defaults). Same errors as di_solve. */
di_status di_solve_ex(di_graph *g, const double *B, double d, double tol, const di_solve_opts *opts,
                      double *X_out, double *residual_out, di_solve_info *info, void *stream);

/*
 * di_power_iter — power iteration PI (Section 2.3, Section 2.5 "PI": row vectors, i.e. a pull
 * over the in-links), applied to X = P.X + B as a Jacobi iteration: X_0 = 0,
 * X_(k+1) = B + P.X_k, stopping when ||X_(k+1) - X_k||_1 <= tol or after max_iters (<= 0:
 * 100000) iterations. This is di_power_iter_ex with default options: the increments
 * X_(k+1) - X_k = P (X_k - X_(k-1)) in FP32, X in FP64, and the exact
 * next increment B + P.X - X (double-float link sums, FP64 B and X) taken halfway and at the
 * end; the reported residual is that exact ||X_(k+1) - X_k||_1 of the returned X.
 * X_out double[n]; residual_out and info nullable. Errors as di_solve.
 */
di_status di_power_iter(di_graph *g, const double *B, double d, double tol, int32_t max_iters,
                        double *X_out, double *residual_out, di_solve_info *info, void *stream);

/*
 * di_power_iter_ex — di_power_iter with options (opts may be NULL):
 *   fluid      DI_FLUID_F32 (default): FP32 increments, X in FP64, exact FP64
 *              certification as described for di_power_iter.
 *              DI_FLUID_F64: FP64 throughout (y_j = d X_j / out_j, the link sums and X in FP64);
 *              the iterates and the iteration count are those of an FP64 Jacobi iteration.
 *   max_sweeps iteration cap (<= 0: 100000).   refine   -1: no exact certification (FP32
 *              increments only; the residual is the last FP32 increment's norm).
 *   profile    1: iterations driven from the host with CUDA events around every kernel
 *              (push_ms: the pull kernel, select_ms: the heavy rows' chunk sums).
 * Other fields are ignored. Errors as di_solve.
 */
di_status di_power_iter_ex(di_graph *g, const double *B, double d, double tol, const di_solve_opts *opts,
                           double *X_out, double *residual_out, di_solve_info *info, void *stream);

/*
 * di_solve_resume — D-iteration from a given state (H0, F0) instead of (0, B) (Section 2.5: the
 * visit keeps X = H + (I - P)^-1 F for any state, so a run can stop and continue).
 *   B       double[n] (host or device), >= 0 and finite: the problem X = P.X + B.
 *   H0      double[n] (host or device), finite: the starting history.
 *   F0      double[n] (host or device) or NULL. A run's final fluid (F_out below) resumes that
 *           run. NULL starts from the exact residual F0 = B + P.H0 - H0, which makes any
 *           approximate solution H0 (for instance the solution for an earlier B) a warm start.
 *           The fluid may be negative: a node is selected on |F_i|.
 *   F_out   double[n] (host or device) or NULL: the final fluid, the checkpoint that, with X_out
 *           as H0, resumes this run. After refinement it is the exact residual, rounded to the
 *           fluid's type.
 *   opts    as di_solve_ex (nullable).
 * X_out, residual_out, info, stream and errors as di_solve_ex. With refinement (the default for
 * FP32 fluid) the result is X = P.X + B's whatever F0 was; without it, the run converges to
 * H0 + (I - P)^-1 F0, which is X only when F0 is a state of this problem.
 */
di_status di_solve_resume(di_graph *g, const double *B, const double *H0, const double *F0, double d, double tol,
                          const di_solve_opts *opts, double *X_out, double *F_out, double *residual_out,
                          di_solve_info *info, void *stream);

/*
 * di_power_iter_push — power iteration per column PI' (Section 2.5 "PI'": column vectors l_out,
 * i.e. a push over the out-links), the same Jacobi iteration as di_power_iter with the same
 * stopping rule ||X_(k+1) - X_k||_1 <= tol (the paper's tables give PI and PI' equal iteration
 * counts). It pushes the increments X_(k+1) - X_k = P (X_k - X_(k-1)) with the D-iteration's
 * push kernels, a self-link being a plain link: the k-th sweep is iteration k.
 *   fluid  DI_FLUID_F64: FP64 increments; the iterates and the iteration count are PI's.
 *          DI_FLUID_F32: FP32 increments (faster push) with FP64 X; the reported residual is
 *          the exact FP64 ||B + P.X - X||_1 (= the next increment), with continuation sweeps
 *          until it is <= tol, which adds iterations when FP32 rounding of the increments
 *          exceeds tol.
 * Other arguments and errors as di_power_iter; info->sweeps counts iterations.
 */
di_status di_power_iter_push(di_graph *g, const double *B, double d, double tol, int32_t max_iters,
                             int32_t fluid, double *X_out, double *residual_out, di_solve_info *info,
                             void *stream);

/*
 * di_solve_batch — k independent D-iterations on one graph in one multi-RHS sweep loop: every
 * column r solves X_r = P.X_r + B_r and stops at its own tolerance tol[r]. Each column keeps its
 * own selection rule (Section 2.3; DI-SOP: |F_ir| > (r_r / L) * out_i); a node's out-links are
 * walked once per sweep for all the columns that selected it.
 *   B      double[k * n]: column r at B + r * n (host or device), >= 0 and finite.
 *   tol    double[k] (host or device), each > 0.
 *   opts   schedule, max_sweeps, refine (as di_solve_ex; fluid must be DI_FLUID_F32), rhs_tile
 *          (columns per tile: 4, 8, 16 or 32; 0 = autotuned once per graph and cached).
 *   X_out  double[k * n], same layout as B.   res_out (nullable) double[k]: final ||F_r||_1
 *          (exact FP64 residual of H_r when refinement is on).
 *   info   (nullable) aggregate report: sweeps summed over tiles, pushed_edges counted once per
 *          node visit (a visit serves every selected column), rhs_tile = tile width used.
 * The fluid is FP32, node-major within each tile; H is FP64.
 * Errors as di_solve; DI_ERR_NOT_CONVERGED when any column missed its tolerance (X_out and
 * res_out still hold every column's current state).
 */
di_status di_solve_batch(di_graph *g, int32_t k, const double *B, double d, const double *tol,
                         const di_solve_opts *opts, double *X_out, double *res_out,
                         di_solve_info *info, void *stream);

/*
 * di_ppr_batch — di_solve_batch with personalised right-hand sides given as seed sets
 * (personalised PageRank): column r has B_r = (1 - d) / |S_r| on every seed of
 * S_r = seeds[seed_offsets[r] .. seed_offsets[r+1]); a seed listed twice receives two shares.
 *   seed_offsets int64[k+1], ascending, seed_offsets[0] = 0, no empty set; seeds int32 ids.
 *   Both host or device.
 * Errors as di_solve_batch; DI_ERR_OUT_OF_RANGE_ID for a seed outside [0, n),
 * DI_ERR_INVALID_ARG for an empty set or bad offsets.
 */
di_status di_ppr_batch(di_graph *g, int32_t k, const int64_t *seed_offsets, const int32_t *seeds,
                       double d, const double *tol, const di_solve_opts *opts, double *X_out,
                       double *res_out, di_solve_info *info, void *stream);

/* ------------------------------------------------------------------------------------------
 * Caller-owned scratch ("workspace"). By default a graph's first solve allocates the scratch
 * it keeps for later solves (cudaMalloc). A caller whose own allocator must own all device
 * memory (PyTorch's caching allocator, a serving runtime's pool) asks for the size, allocates
 * the buffer itself and attaches it; from then on the solves of that kind lay their scratch out
 * in it and call no allocator. The paper has no counterpart: this is the ownership rule of the
 * C boundary.
 * ------------------------------------------------------------------------------------------ */
typedef enum {
    DI_WS_SOLVE = 0,   /* di_solve, di_solve_ex, di_solve_resume, di_power_iter,
                          di_power_iter_push (param: the fluid, DI_FLUID_F32 or DI_FLUID_F64;
                          power iteration uses the DI_FLUID_F32 size) */
    DI_WS_BATCH = 1    /* di_solve_batch, di_ppr_batch (param: the widest tile, 4, 8, 16 or 32
                          columns; 0 means 32). With a workspace for fewer than 32 columns the
                          autotuner only tries the widths it holds. */
} di_workspace_kind;

/*
 * di_workspace_size — bytes of device scratch the solves of `kind` need on graph g, for the
 * given param (see di_workspace_kind). The size grows with the graph (about 70 bytes per node
 * for DI_WS_SOLVE with FP32 fluid; about 44 * param bytes per node for DI_WS_BATCH).
 * Errors: DI_ERR_INVALID_ARG (NULL, unknown kind or param).
 */
di_status di_workspace_size(const di_graph *g, int32_t kind, int32_t param, int64_t *bytes);

/*
 * di_graph_set_workspace — attaches `bytes` of the caller's device memory at `workspace` (256-byte
 * aligned, on the graph's GPU) as the scratch of the solves of `kind`, or detaches it (workspace
 * NULL: later solves allocate their own again). Scratch the library had allocated for that kind
 * is freed at once. The caller keeps the memory alive and leaves it alone until it detaches it or
 * destroys the graph; the library keeps solver state there between calls, so two graphs must not
 * share one workspace. A solve that needs more than the attached size fails with
 * DI_ERR_INVALID_ARG (see di_workspace_size) and allocates nothing. The call waits for the device
 * to finish earlier work (cudaDeviceSynchronize), since that work may still use the old scratch.
 * Errors: DI_ERR_INVALID_ARG (NULL graph, kind, alignment, not device memory of the graph's
 * GPU), DI_ERR_BUSY (a solve on the graph is running), DI_ERR_CUDA.
 */
di_status di_graph_set_workspace(di_graph *g, int32_t kind, void *workspace, int64_t bytes);

/* ------------------------------------------------------------------------------------------
 * Autotuning of the push (the paper has no counterpart: it chooses how the GPU splits work).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t push_row;          /* single right-hand side: rows of at least this many links are
                                  pushed one at a time by a whole warp */
    int32_t heavy_cut;         /* nodes with more links than this are pushed in chunks spread over
                                  all warps of the grid ... */
    int32_t heavy_chunk;       /* ... of this many links each (so out / heavy_chunk warps share the
                                  row) */
    int32_t rhs_tile;          /* batched: columns per tile (0 before the first batched call) */
    int32_t batch_heavy_cut;   /* batched push: the same split for tiles */
    int32_t batch_heavy_chunk;
    double single_probe_ms;    /* device time of the chosen single-RHS probe solve (ms) */
    double batch_rate;         /* column-link updates per second of the chosen batched setting */
} di_tuning;

/*
 * di_autotune — times short probe solves on graph g (damping d, uniform right-hand sides) and
 * keeps the fastest push split for later solves on g. what: bit 0 tunes the single right-hand
 * side push (row cut-off, heavy cut-off, chunk length; probe: a DI-SOP solve to 1e-3 ||B||_1,
 * median of 3), bit 1 the batched tile width and its push split (probes of 6 and 24 sweeps),
 * bit 2 sets the single right-hand-side split to out's push_row, heavy_cut and heavy_chunk
 * without probing (heavy_cut >= 1024, 256 <= heavy_chunk <= heavy_cut; to repeat a tuned setting);
 * 0 only reports the current values. Untuned graphs use 64 / 4096 / 1024; a graph's first
 * batched call with rhs_tile 0 tunes the batched setting itself. out (nullable) receives the
 * values in use. Errors: DI_ERR_INVALID_ARG, DI_ERR_BUSY, DI_ERR_OOM, DI_ERR_CUDA.
 */
di_status di_autotune(di_graph *g, double d, int32_t what, di_tuning *out, void *stream);

/* Bytes of device memory this library holds from its own allocations (cudaMalloc), over every
 * graph of the process: the graphs' arrays and any scratch not attached by the caller. A
 * diagnostic: with workspaces attached, solves leave it unchanged. */
int64_t di_device_bytes_held(void);

/* ------------------------------------------------------------------------------------------
 * Serving: personalised-PageRank requests over resident graphs, continuously batched.
 * ------------------------------------------------------------------------------------------ */
typedef struct di_server di_server;

typedef struct {
    double d;                    /* damping of every request; 0 means 0.85 */
    int32_t slots;               /* request slots per graph (columns of its tile): 4, 8, 16 or 32;
                                    0 means 32 */
    int32_t sweeps_per_step;     /* sweeps between two admission / retirement points; 0 means 8 */
    int32_t max_request_sweeps;  /* a request still above its tolerance after this many sweeps
                                    ends with DI_ERR_NOT_CONVERGED; 0 means 100000 */
    int32_t tile_min_queue;      /* a graph whose tile is idle solves its queued requests one at a
                                    time on the single right-hand-side path until this many wait;
                                    then they share the tile's sweeps. 0 means 16; 1 always tiles */
    int64_t mem_budget;          /* device bytes for request state over all graphs (24 bytes per
                                    node and slot); slots halve until it fits; 0 means no limit */
} di_server_opts;

typedef struct {
    int32_t status;              /* di_status of the request */
    int32_t sweeps;              /* sweeps its slot took part in */
    int32_t graph, slot;
    double residual_l1;          /* final ||F||_1 of its column (exact FP64 when tol < 1e-6) */
    double queue_ms;             /* submit -> admitted into a slot */
    double service_ms;           /* admitted -> history in host memory */
    double total_ms;             /* submit -> history in host memory (done) */
} di_request_info;

/*
 * di_server_create — starts one worker (host thread + CUDA stream + a tile of request slots) per
 * resident graph. Every request is the personalised PageRank X = P.X + B with
 * B = (1 - d) / |S| on its seed set S (Section 1 problem, Section 2.3 DI-SOP sweeps, per-column
 * selection and retirement as in di_solve_batch). Requests that arrive while others are on the
 * GPU are admitted between sweep steps as slots free up, so their work overlaps; the workers of
 * different graphs run concurrently. A finished request's history is copied into a pinned host
 * buffer owned by the server (one per finished request not yet collected by di_server_wait, n
 * doubles each; four per graph are made at creation and reused, more only while more results
 * wait uncollected); the request is done when that copy has completed. The graphs must outlive
 * the server.
 * Errors: DI_ERR_INVALID_ARG, DI_ERR_OOM (mem_budget below 4 slots per graph), DI_ERR_CUDA.
 */
di_status di_server_create(di_graph *const *graphs, int32_t n_graphs, const di_server_opts *opts,
                           di_server **out);

/*
 * di_server_submit — queues a request on graph `graph` with seed ids seeds[0 .. n_seeds) (host
 * memory, copied; a seed listed twice gets two shares) and tolerance tol on ||F||_1. Returns at
 * once with *request_id. Errors: DI_ERR_INVALID_ARG, DI_ERR_OUT_OF_RANGE_ID (a seed), DI_ERR_CUDA
 * (the graph's worker stopped).
 */
di_status di_server_submit(di_server *srv, int32_t graph, const int32_t *seeds, int32_t n_seeds,
                           double tol, int64_t *request_id);

/*
 * di_server_wait — waits at most timeout_ms for a request. When it is done, copies its history H
 * (the approximation of X, n doubles) from the server's pinned buffer into X_out (host or device
 * memory; NULL skips the copy), releases the buffer, fills *info (nullable), forgets the request
 * and returns its status. DI_ERR_TIMEOUT leaves the request pending (wait again later).
 */
di_status di_server_wait(di_server *srv, int64_t request_id, double *X_out, di_request_info *info,
                         int32_t timeout_ms);

/* Stops the workers (requests not finished end with DI_ERR_BUSY) and frees the server. */
void di_server_destroy(di_server *srv);

/* ------------------------------------------------------------------------------------------
 * Diagnostics (host code, not on the solve path).
 * ------------------------------------------------------------------------------------------ */

/*
 * di_csr_validate — checks graph arrays in host memory, laid out as di_graph_export returns
 * them, against the build's invariants:
 *   - each CSR runs from 0 to L, with non-decreasing row pointers, ids in [0, n), and every row
 *     strictly ascending (sorted and free of duplicates);
 *   - the in-CSR is the transpose of the out-CSR (order-independent checksums of the link set);
 *   - the degrees are the row lengths, and loop[i] is set exactly when row i holds i;
 *   - E and its levels follow Section 2.4's definition: i is in E exactly when all of its
 *     in-neighbours are, with level 1 + their largest level (0 without in-neighbours), and -1
 *     outside E.
 * out_deg, in_deg, loop, e_mask and e_level may be NULL to skip their checks. Returns DI_OK, or
 * DI_ERR_CORRUPT with di_last_error() naming the first inconsistency; DI_ERR_INVALID_ARG for a
 * NULL CSR array or bad sizes. Time O(n + L); no GPU needed.
 */
di_status di_csr_validate(int32_t n, int64_t L, const int64_t *rp_out, const int32_t *col_out,
                          const int64_t *rp_in, const int32_t *col_in, const int32_t *out_deg,
                          const int32_t *in_deg, const uint8_t *loop, const uint8_t *e_mask,
                          const int32_t *e_level);

/*
 * di_graph_validate — copies every array of a built graph to the host and runs di_csr_validate
 * on them. It also checks the push kernels' copy of the out-links, where bit 31 marks the links
 * into a hub and a loop node's self-link is swapped with the last link of its row, and |E|
 * against the statistics. Same returns; DI_ERR_CUDA if a copy fails.
 */
di_status di_graph_validate(const di_graph *g);

/*
 * di_residual_noalloc — the exact residual F* = B + P.H - H of a history H and its norm
 * ||F*||_1 (by the identity X = H + (I - P)^-1 F*, ||X - H||_1 <= ||F*||_1 / (1 - d)), computed
 * without allocating any memory. The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc, such as hosts whose own pool owns all device memory and
 * forbids the runtime's allocator, or code that must not add the device-wide synchronisation
 * that cudaMalloc may cause. Its scratch is a static device array of about 8 MB that every GPU
 * which loads this library holds until the process exits.
 *   n          1 .. 1048576 nodes (the size the static scratch holds); larger n is rejected with
 *              DI_ERR_INVALID_ARG.
 *   rp_in, col_in  int64[n+1], int32[L]: rows of P (in-links), as di_graph_export returns them.
 *              Every id in col_in must lie in [0, n): the call does not check them (an id outside
 *              that range reads scratch left by an earlier call or past it). di_csr_validate
 *              checks a CSR that did not come from di_graph_export.
 *   out_deg    int32[n]: out-degrees.   B, H: double[n].   0 <= d < 1.
 *   Fstar_out  double[n] or NULL: receives F*.   norm_out: one double, receives ||F*||_1.
 * Every array must be device memory of the current device; the caller owns all of them. The call
 * only enqueues work on `stream` (no synchronisation, no allocation); results are ready when
 * the stream reaches that point. The first call on a device looks up the scratch array's device
 * address and keeps it for the life of the process, so make that first call before any stream
 * capture; a device reset (cudaDeviceReset) in between is not supported. Every call shares the one
 * scratch array: calls whose work can overlap on the GPU (different streams without ordering)
 * race and must not be issued. Errors: DI_ERR_INVALID_ARG (size, d, NULL pointer, host memory or
 * memory of another device), DI_ERR_CUDA.
 */
di_status di_residual_noalloc(int32_t n, const int64_t *rp_in, const int32_t *col_in,
                              const int32_t *out_deg, const double *B, double d, const double *H,
                              double *Fstar_out, double *norm_out, void *stream);

/* Thread-local message of the last failing call on this thread ("" when none). */
const char *di_last_error(void);

/* Library version string. */
const char *di_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DI_GB300_H */
