/*
 * amg.h -- C ABI of the GB300 (sm_103a) auxiliary-grid algebraic multigrid library
 * (libamg_gb300.so).
 *
 * The method is that of Wang, Hu, Cohen and Xu, "A Parallel Auxiliary Grid AMG Method for
 * GPU": unsmoothed aggregation from a region quadtree over a uniform auxiliary grid laid on
 * the finest mesh, Galerkin coarse operators, a quadtree-coloured Gauss-Seidel smoother and
 * the nonlinear AMLI-cycle (K-cycle) preconditioning a Krylov iteration. All of the work
 * runs in the library's CUDA kernels on one GPU.
 *
 * Conventions shared by every entry point:
 *  - Return value: an AMG_* status (0 = AMG_OK). No C++ exception crosses this interface.
 *  - Pointers marked "device or host" may point to device memory or to host memory (pageable
 *    or pinned); the library detects which and stages host data through device buffers
 *    inside the call. All other array pointers are host pointers unless stated.
 *  - Ownership: input arrays are borrowed for the duration of the call only; setup copies
 *    what it keeps. A hierarchy is owned by the library until amg_free.
 *  - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream). All device work
 *    of a call is ordered on it. Calls return after their results are complete (the status,
 *    iteration counts and residuals are host values).
 *  - Threads: a hierarchy may be used by one thread / one stream at a time; different
 *    hierarchies are independent.
 *  - Indices are 32-bit: n < 2^31 and nnz < 2^31.
 */
#ifndef AMG_GB300_AMG_H
#define AMG_GB300_AMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    AMG_OK = 0,
    AMG_ERR_INVALID_ARG = 1,   /* NULL pointer, n <= 0, bad option, non-finite coordinate */
    AMG_ERR_BAD_MATRIX = 2,    /* not square CSR with sorted unique in-range columns and a
                                  positive diagonal, non-finite value, or a coarsest matrix
                                  that is not positive definite */
    AMG_ERR_OOM = 3,           /* device allocation failed */
    AMG_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    AMG_ERR_NOT_CONVERGED = 5, /* max_iters reached; x, iters, relres are valid */
    AMG_ERR_BREAKDOWN = 6,     /* (p, Ap) <= 0 or non-finite in the outer Krylov iteration */
    AMG_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
    AMG_ERR_UNSUPPORTED = 8    /* outside the library's limits (see amg_options) */
};

/* Outer Krylov iteration. */
enum { AMG_OUTER_FCG = 0, AMG_OUTER_FGMRES = 1 };
/* Arithmetic of the AMLI-cycle (the preconditioner). */
enum { AMG_FP64 = 0, AMG_FP32 = 1 };

/*
 * Sparse SPD matrix A of the linear system A x = b (paper Sec. 1), in CSR:
 * rowptr[n+1], col[nnz], val[nnz]; columns ascending and unique within each row, the
 * diagonal present and positive. Arrays are device or host memory, borrowed.
 */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t *rowptr;
    const int32_t *col;
    const double *val;
} amg_csr;

/* Options; amg_options_default fills the defaults given in brackets. */
typedef struct {
    int aux_level;      /* depth L of the quadtree / auxiliary grid 2^L x 2^L (Sec. 3.1);
                           0 = automatic, the largest L with 4^L <= n [0]; at most 14 */
    int coarsest_max;   /* coarsen until a level has at most this many unknowns; that level
                           is solved exactly (Alg. 2, B_1 = A_1^{-1}) [64]; 1..256 */
    int kcycle_n;       /* steps n of Alg. 1 on each coarse level of the AMLI-cycle [2];
                           1..4 */
    int max_iters;      /* outer iterations [200] */
    int outer;          /* AMG_OUTER_FCG: Alg. 1 on the finest level (flexible CG with full
                           A-orthogonalisation) [default]; AMG_OUTER_FGMRES: restarted
                           flexible GMRES (requires cycle_prec = AMG_FP32 or FP64) */
    int cycle_prec;     /* AMG_FP64 [default] or AMG_FP32 (cycle in single precision, outer
                           residuals, updates and inner products in double) */
    int fgmres_restart; /* restart length of FGMRES [30] */
    int has_bbox;       /* 1: use bbox as the auxiliary box Omega_0^0 instead of the
                           coordinates' min/max (eq. ab12) [0] */
    double bbox[4];     /* a1, b1, a2, b2 */
    double zbox[2];     /* a3, b3: the box's third side (amg_setup3 with has_bbox) */
    int nu_pre;         /* Gauss-Seidel sweeps of the pre-smoothing R_k of Alg. 2 on every
                           level, the first from zero [1]; 1..4 (0 = 1) */
    int nu_post;        /* backward sweeps of the post-smoothing R_k^t [1]; 1..4 (0 = 1) */
} amg_options;

typedef struct amg_hierarchy amg_hierarchy;

/* Fill *opt with the defaults. */
void amg_options_default(amg_options *opt);

/*
 * Setup phase (paper Sec. 3 and Sec. 4.2-4.5): auxiliary box (eq. ab12), level-L aggregates
 * by binning the unknowns' coordinates into the 2^L x 2^L auxiliary cells (Sec. 4.2), coarse
 * aggregates from the quadtree parents (eq. agg_k), Galerkin operators A_{k-1} = P^t A_k P
 * (eq. acsum) on every level down to the first with at most coarsest_max unknowns, the
 * quadtree colouring of every level (Sec. 4.5), and the exact coarsest solve.
 *   A      : the fine matrix (device or host, borrowed).
 *   x, y   : coordinates (x_j, y_j) of unknown j, arrays of A->n doubles (device or host).
 *   opt    : options (host); NULL = defaults.
 *   stream : cudaStream_t for the device work.
 *   out    : receives the new hierarchy (owned by the library until amg_free).
 * Errors: AMG_ERR_INVALID_ARG, AMG_ERR_BAD_MATRIX (checked on the device),
 * AMG_ERR_UNSUPPORTED, AMG_ERR_OOM, AMG_ERR_CUDA. On error *out is NULL.
 */
int amg_setup(const amg_csr *A, const double *x, const double *y, const amg_options *opt,
              void *stream, amg_hierarchy **out);

/*
 * The octree variant (paper Sec. 3.1 and Sec. 6: the same construction in three dimensions,
 * 8 children per cell, 27-point coarse stencils, 8 colours): the setup above with node
 * coordinates (x, y, z). The auxiliary box gains [a3, b3] (min / max of z, or zbox with
 * has_bbox); cells have coordinates (t1, t2, t3) and index t1 + 2^k (t2 + 2^k t3) on level
 * k; the parent of a cell halves all three; colours are (t1 mod m) + m (t2 mod m) +
 * m^2 (t3 mod m); the automatic depth is the largest L with 8^L <= n. Coupling spans above 2
 * cells return AMG_ERR_UNSUPPORTED. Solve, inspection and batching work on the result as on
 * a quadtree hierarchy. Arguments and errors as amg_setup; z: n doubles (device or host).
 */
int amg_setup3(const amg_csr *A, const double *x, const double *y, const double *z,
               const amg_options *opt, void *stream, amg_hierarchy **out);

/*
 * Solve phase: x = A^{-1} b by the outer Krylov iteration preconditioned with the nonlinear
 * AMLI-cycle (Alg. 2 with Alg. 1 on the coarse levels), from x_0 = 0, until
 * ||b - A x||_2 / ||b||_2 <= tol.
 *   b      : right-hand side, n doubles (device or host, borrowed).
 *   tol    : relative residual target (>= 0).
 *   x      : output, n doubles (device or host, caller-allocated; initial content ignored).
 *   iters  : receives the number of outer iterations (preconditioner applications); may be
 *            NULL.
 *   relres : receives ||b - A x||_2 / ||b||_2 of the returned x; may be NULL.
 * Returns AMG_OK, or AMG_ERR_NOT_CONVERGED / AMG_ERR_BREAKDOWN with x, iters and relres
 * still valid, or another error.
 */
int amg_solve(amg_hierarchy *h, const double *b, double tol, double *x, int *iters,
              double *relres, void *stream);

/* Device memory held by the hierarchy, in bytes (for admission against a memory budget). */
int amg_hierarchy_bytes(const amg_hierarchy *h, size_t *bytes);

/* Release a hierarchy and its device memory (NULL is ignored). */
void amg_free(amg_hierarchy *h);

/*
 * Batched systems. The paper solves one system at a time and has no counterpart of these
 * calls: they apply the setup and solve above to many independent systems at once. Each
 * system gets its own hierarchy, exactly as amg_setup would build it from its block; the
 * solve runs every system's outer iteration and AMLI-cycle in one persistent kernel, one
 * CTA (or a team of CTAs for the largest systems) per system at a time, largest systems
 * first, with flexible CG as the outer method.
 */
typedef struct amg_batch amg_batch;

/*
 *   nprob   : number of systems (>= 1).
 *   row_off : host array of nprob + 1 row offsets, row_off[0] = 0, strictly increasing,
 *             row_off[nprob] = A->n: system p owns rows [row_off[p], row_off[p+1]).
 *   A       : the block-diagonal matrix of all systems as one CSR (global row pointers and
 *             global column indices; every column of a row of system p lies in system p),
 *             device or host, borrowed.
 *   x, y    : node coordinates of every row, A->n doubles each (device or host).
 *   opt     : options of every system (aux_level 0 = chosen per system); outer must be
 *             AMG_OUTER_FCG. NULL = defaults.
 *   out     : receives the batch (owned by the library until amg_batch_free).
 * The systems of more than opt->coarsest_max unknowns are set up together: every step of the
 * setup runs once, as one multi-system kernel launch, for all of them (the others, which are
 * their own coarsest level, take amg_setup's path). Each hierarchy is bit for bit the one
 * amg_setup builds from its block. Its arrays are pieces of a few large allocations of its own
 * (about 1 KB per unknown with the batched-solve workspace, charged in full to the
 * hierarchy); its amg_launch_counts setup figure is the whole batched setup's launches.
 * Errors: as amg_setup (a system's failure fails the call), AMG_ERR_UNSUPPORTED for the
 * FGMRES outer method. On error *out is NULL.
 */
int amg_batch_setup(int32_t nprob, const int64_t *row_off, const amg_csr *A, const double *x,
                    const double *y, const amg_options *opt, void *stream, amg_batch **out);

/*
 * amg_setup (the setup of paper Sec. 3.1-4.5: auxiliary grid, quadtree aggregates, colours,
 * Galerkin operators, exact coarsest inverse) of many systems at once, each hierarchy returned
 * on its own: the systems are given as for amg_batch_setup (row_off, A, x, y, opt; any outer
 * method) and set up together in the same way, but out[p] (a host array of nprob pointers,
 * caller-allocated) receives system p's hierarchy,
 * bit for bit the one amg_setup builds from its block, owned by the caller and released by
 * amg_free like any other, independently of the others. With the flexible-CG outer method
 * each hierarchy is also ready for batched solves (amg_batch_create). The paper sets up one
 * system at a time; this entry point serves callers with many new systems at once, such as a
 * server admitting several matrices.
 * Errors: as amg_setup (a system's failure fails the call; every out[p] is then NULL).
 */
int amg_setup_many(int32_t nprob, const int64_t *row_off, const amg_csr *A, const double *x,
                   const double *y, const amg_options *opt, void *stream, amg_hierarchy **out);

/*
 * A batch over hierarchies that already exist (built by amg_setup or amg_batch_setup; all
 * with the same cycle_prec, kcycle_n, nu_pre, nu_post and max_iters; borrowed: they must outlive the
 * batch, and a hierarchy must not be solved by two calls at the same time). System p is hs[p]; its rows in
 * the concatenated vectors follow those of hs[0..p-1]. threads: 0 = choose the launch shape
 * by timing on the first solve, with teams of CTAs for the largest systems (see
 * amg_batch_set_teams); 1024, 512 or 256 = that many threads per CTA (1, 2 or 4 CTAs per
 * SM), one CTA per system. With a fixed shape a system's result does not depend on the
 * other systems of the batch (each system is computed by one CTA in a fixed order). The batch allocates each
 * hierarchy's outer-iteration workspace: 32 FP64 directions and their images at first
 * (about 0.5 KB per unknown), the same directions amg_solve uses, owned by the hierarchy and
 * counted by amg_hierarchy_bytes.
 * Errors: AMG_ERR_INVALID_ARG (NULL, mixed options, a repeated hierarchy, other threads),
 * AMG_ERR_OOM, AMG_ERR_CUDA.
 */
int amg_batch_create(int32_t nprob, amg_hierarchy *const *hs, int32_t threads, void *stream,
                     amg_batch **out);

/*
 * Solves every system: b and x hold all right-hand sides / solutions concatenated in row_off
 * order (A->n doubles each, device or host; x caller-allocated). iters, relres, status: host
 * arrays of nprob entries receiving each system's outer iterations, true relative residual
 * and status (as amg_solve would return it); each may be NULL. The first call also times the
 * candidate launch shapes on this batch (every timed solve is a complete solve) and keeps
 * the fastest; the launch sequence is captured in a CUDA graph and replayed while b, x and
 * tol stay the same. The outer iteration keeps every direction (flexible CG with full
 * A-orthogonalisation, as amg_solve): a system that fills its allocated directions gets
 * twice as many (at most max_iters) and continues in a further launch, so its iterates are
 * those of an unbounded workspace. Returns AMG_OK if every system converged, else the first
 * non-OK system status in system order.
 */
int amg_batch_solve(amg_batch *bt, const double *b, double tol, double *x, int32_t *iters,
                    double *relres, int32_t *status, void *stream);

/*
 * nprob: systems; threads, ctas: the launch shape chosen by the first solve (0 before it);
 * tuned_ms: one batch solve's time for each of the 4 candidate shapes (1024 threads x 1 CTA
 * per SM, 512 x 2, 512 x 1, 256 x 4; -1 if not timed); bytes: device memory of the batch
 * with its hierarchies. Each output may be NULL.
 */
int amg_batch_info(const amg_batch *bt, int32_t *nprob, int32_t *threads, int32_t *ctas,
                   double tuned_ms[4], size_t *bytes);

/*
 * Algorithmic bytes the last amg_batch_solve moved (0 before a solve), for its roofline: per
 * system, every outer step's B^_0 application (Alg. 2 over every level, the per-op counts of
 * the single-system cycle: 4-byte indices, values in the cycle precision) and its FP64 outer
 * flexible-CG work (conversions, the dots and orthogonalisation against every kept direction,
 * the SpMV, the update), plus the gather of b and the true residual. Padding and re-reads
 * are not counted. bytes: host. Errors: AMG_ERR_INVALID_ARG (NULL).
 */
int amg_batch_moved_bytes(amg_batch *bt, double *bytes);

/*
 * When each system of the last amg_batch_solve started and finished on the device: host
 * arrays of nprob entries, ns after the earliest start (device clock); each may be NULL.
 * end_ns is each system's latency from the launch of the batch.
 */
int amg_batch_timeline(const amg_batch *bt, int64_t *start_ns, int64_t *end_ns);

/*
 * Teams of CTAs for the largest systems of a batch. A system far larger than the batch's
 * average work per CTA would alone set the batch's time on one CTA, so it can be solved by a
 * team of up to 8 CTAs that split every step's rows and meet at a barrier of their own
 * (bounded: a wait that runs out ends that system with AMG_ERR_TIMEOUT). A system gets about
 * ceil(its unknowns / (the batch's unknowns / CTAs of the launch)) CTAs, largest systems
 * first, while the teams hold at most half of the launch's CTAs. Team sums add the members'
 * partial sums in a fixed order, so results are reproducible, but they differ in rounding
 * from a one-CTA solve of the same system.
 *   max_team: 0 = teams sized as above (the default of a batch created with threads = 0),
 *             1 = one CTA per system (the default with a fixed shape: a system's result then
 *             does not depend on the other systems), 2..8 = sized as above, at most max_team.
 * A batch whose shape is chosen by timing times its shapes again on the next solve.
 * Teams expect the batch's kernel to have the GPU to itself (its CTAs resident together): when
 * several batches are solved at the same time on different streams, give them a fixed shape
 * or max_team = 1 (a team whose members cannot all run waits until its barrier's limit, and
 * that system ends with AMG_ERR_TIMEOUT).
 * Errors: AMG_ERR_INVALID_ARG (NULL, max_team outside 0..8).
 */
int amg_batch_set_teams(amg_batch *bt, int32_t max_team);

/* CTAs of each system's team in the launch shape in use: team is a host array of nprob
 * entries (-1 each before the first solve). Errors: AMG_ERR_INVALID_ARG (NULL). */
int amg_batch_teams(const amg_batch *bt, int32_t *team);

/* System p's hierarchy (owned by the batch; valid until amg_batch_free), NULL if none. */
amg_hierarchy *amg_batch_system(amg_batch *bt, int32_t p);

/* Release a batch and its device memory, and the hierarchies amg_batch_setup built (not
 * those given to amg_batch_create). NULL is ignored. */
void amg_batch_free(amg_batch *bt);

/* Static, human-readable text of a status code. */
const char *amg_status_string(int status);

/* Detail of the last failing call on the calling thread (valid until its next call). */
const char *amg_last_error(void);

/* ---------------------------------------------------------------------------------------
 * Inspection (host copies of what setup built), for checking and diagnostics.
 * Levels are numbered 0 = the given fine matrix, 1 = the auxiliary level L, 2 = level L-1,
 * ..., num_levels-1 = the coarsest. Rows of level l >= 1 are aggregates numbered in
 * ascending lexicographic cell order t1 + 2^k t2 (the numbering of Sec. 3.1), empty cells
 * skipped.
 * ------------------------------------------------------------------------------------- */

/* Number of levels and the depth L actually used. */
int amg_num_levels(const amg_hierarchy *h, int *num_levels, int *aux_level);

/* The auxiliary box a1, b1, a2, b2 actually used (eq. ab12). */
int amg_get_bbox(const amg_hierarchy *h, double bbox[4]);

/* Tree dimension (2 or 3) and the whole auxiliary box a1, b1, a2, b2, a3, b3 (a3 = b3 = 0
 * for a quadtree). Either output may be NULL. */
int amg_get_box3(const amg_hierarchy *h, int *dim, double box[6]);

/*
 * info[0] = n (unknowns), info[1] = stored entries of A_l (without padding),
 * info[2] = cells per side of the grid the rows live on (level 0: the level-L grid),
 * info[3] = span s (largest cell offset over the stored entries),
 * info[4] = colour modulus m = max(2, s+1) (m*m colours),
 * info[5] = padded entries in the on-device sliced-ELL layout,
 * info[6] = 1 if this is the coarsest level (solved exactly).
 */
int amg_level_info(const amg_hierarchy *h, int level, int64_t info[8]);

/*
 * Host copies of level `level` in natural row order (fine: the caller's unknown order;
 * coarse: aggregate number). Any pointer may be NULL to skip it. Sizes: n for agg, color,
 * t1, t2; n+1 for rowptr; info[1] for col and val (CSR, columns ascending).
 *   agg    : row of the next coarser level containing each row (-1 on the coarsest).
 *   color  : colour (t1 mod m) + m (t2 mod m) [+ m^2 (t3 mod m)] of each row's cell.
 *   t1, t2 : cell coordinates of each row (amg_level_t3 gives the octree's third).
 */
int amg_level_export(const amg_hierarchy *h, int level, int32_t *agg, int32_t *color,
                     int32_t *t1, int32_t *t2, int32_t *rowptr, int32_t *col, double *val);

/* Octree: the third cell coordinate t3 of every row of `level`, natural order (host, n). */
int amg_level_t3(const amg_hierarchy *h, int level, int32_t *t3);

/*
 * One application of the AMLI-cycle preconditioner z = B^_level[f] (Alg. 2) on level
 * `level` (0 = finest), vectors in that level's natural row order. Level 0 runs the solve's
 * preconditioner in the hierarchy's cycle precision (options.cycle_prec; with AMG_FP32 the
 * cycle computes in FP32 between FP64 f and z); coarser levels run in FP64.
 * f, z: device or host arrays of n doubles (z caller-allocated).
 */
int amg_apply_cycle(amg_hierarchy *h, int level, const double *f, double *z, void *stream);

/*
 * One Gauss-Seidel sweep of the quadtree-coloured smoother on level `level` (Sec. 4.5):
 * backward = 0: forward sweep R_k (colours ascending); 1: backward sweep R_k^t. Starts from
 * the given u (updated in place). f, u: device or host, natural row order.
 */
int amg_smooth(amg_hierarchy *h, int level, int backward, const double *f, double *u,
               void *stream);

/*
 * The ELL format of paper Sec. 4.1 (Fig. ellform): a CSR matrix of `rows` rows with at most
 * K = width entries per row stored as two rows x K arrays Aj (columns, -1 padding) and Ax
 * (values, 0 padding), written here column-major (entry (i, k) at [k * rows + i]).
 * diag_first = 1 moves each row's diagonal entry to slot 0 (as the paper's solver stores
 * it); 0 keeps the CSR order. Device kernel; all arrays are device or host memory.
 * rowptr must be non-decreasing from rowptr[0] = 0, and col and val must hold rowptr[rows]
 * entries: the packer reads that many and does not validate rowptr (unlike amg_setup, which
 * validates the whole matrix on the device); the Python binding checks host arrays.
 * Returns AMG_ERR_INVALID_ARG if a row has more than `width` entries.
 */
int amg_csr_to_ell(int32_t rows, const int32_t *rowptr, const int32_t *col, const double *val,
                   int32_t width, int diag_first, int32_t *Aj, double *Ax, void *stream);

/*
 * amg_csr_to_ell without any allocation, for callers that cannot allocate device memory
 * when they call in -- for example because another allocator already owns all of the GPU's
 * memory, or because a latency-critical loop forbids allocation calls. The paper has no
 * counterpart of this entry point; it takes the same arguments and gives the same results as
 * amg_csr_to_ell.
 *   - All arrays must be device memory (host arrays would need staging buffers):
 *     otherwise AMG_ERR_INVALID_ARG.
 *   - Its scratch is a fixed array inside the library (about 64 KiB per GPU, held until the
 *     process exits); rows is limited to 4,194,304: larger inputs return AMG_ERR_UNSUPPORTED.
 *   - The first call on a device looks up that array's device address (once per device);
 *     make that first call before any stream capture.
 *   - Every call on a device shares the array: calls that overlap on the GPU (other streams
 *     or host threads) race and must be ordered by the caller.
 *   - Every call synchronises: it reads the overflow count back into host memory and waits
 *     on `stream` (cudaStreamSynchronize) before it returns. A stream that is capturing does
 *     not allow that, so on such a stream the call returns AMG_ERR_UNSUPPORTED at once,
 *     before any work, and the caller's capture goes on undisturbed.
 *   - The same precondition on rowptr as amg_csr_to_ell.
 *   - Returns AMG_ERR_INVALID_ARG if a row has more than `width` entries. Every failure sets
 *     the text amg_last_error returns; a CUDA error left pending by other code on the calling
 *     thread is not taken for this call's.
 */
int amg_csr_to_ell_noalloc(int32_t rows, const int32_t *rowptr, const int32_t *col,
                           const double *val, int32_t width, int diag_first, int32_t *Aj,
                           double *Ax, void *stream);

/* ---------------------------------------------------------------------------------------
 * Diagnostics.
 * ------------------------------------------------------------------------------------- */

/* Kernel launches made by the last amg_setup and the last amg_solve on h. */
int amg_launch_counts(const amg_hierarchy *h, int64_t *setup_launches, int64_t *solve_launches);

/*
 * Per-kernel timing. enable = 0: off. enable = 1 or 2: every kernel of the following solves
 * is bracketed by CUDA events on the hierarchy's stream and its duration is accumulated per
 * (kernel kind, level) together with its algorithmic bytes: the bytes of every array it must
 * read or write once at its width (4-byte indices, value width of the cycle precision; no
 * padding). Inside the persistent cycle kernel every op is timed from in-kernel timestamps
 * (each op's time includes the grid barrier that ends it); with enable = 1 the ops of the
 * shared-memory tail are also timed one by one (SM clock cycles, which adds work to the tail),
 * with enable = 2 the tail is timed as a whole. Enabling or disabling resets the totals.
 * Measure throughput with profiling off. Errors: AMG_ERR_INVALID_ARG for another value.
 */
int amg_profile_enable(amg_hierarchy *h, int enable);

/*
 * Copies up to `capacity` accumulated records: kind (see amg_kernel_name), level, launches,
 * total milliseconds and total algorithmic bytes. *count receives the number of records.
 */
int amg_profile_read(const amg_hierarchy *h, int capacity, int32_t *kind, int32_t *level,
                     int64_t *launches, double *ms, double *bytes, int *count);

/* Static name of a kernel kind reported by amg_profile_read. */
const char *amg_kernel_name(int kind);

/* ---------------------------------------------------------------------------------------
 * Fault injection, for tests of the error paths. The paper has no counterpart. Every fault
 * is made on the host side or by a bounded wait that runs out: the GPU is never made to
 * fault, trap or hang, and the context stays usable.
 * ------------------------------------------------------------------------------------- */

/*
 * Barrier fault of h's cycle kernel for the following solves (until reset with 0, 0): every
 * grid barrier of the persistent kernel gives up after limit_ns nanoseconds (0 = the default
 * 2 s), and the first barrier of each launch waits for `extra` arrivals more than the grid
 * makes, so that it runs out (0 = none). The solve then returns AMG_ERR_TIMEOUT and leaves h
 * ready for the next solve. Errors: AMG_ERR_INVALID_ARG for NULL or negative arguments.
 */
int amg_debug_barrier_fault(amg_hierarchy *h, int64_t limit_ns, int32_t extra);

/*
 * The same for the team barriers of a batch (systems solved by a team of CTAs): their waits
 * give up after limit_ns (0 = 2 s), and with extra > 0 every team's first barrier runs out.
 * Those systems report AMG_ERR_TIMEOUT; systems solved by one CTA are unaffected. The next
 * solve re-captures the launch with the new arguments.
 */
int amg_debug_batch_barrier_fault(amg_batch *bt, int64_t limit_ns, int32_t extra);

/*
 * Allocation fault: with k > 0 the k-th device allocation the library makes from now on (any
 * thread, any call) fails as if the device were out of memory, so the call making it returns
 * AMG_ERR_OOM after releasing what it had allocated; later allocations succeed again. k = 0
 * disarms it. Errors: AMG_ERR_INVALID_ARG for k < 0.
 */
int amg_debug_fail_allocation(int64_t k);

/*
 * Index checks: in a library built with -DAMG_BOUNDS_CHECK (`python -m
 * paper_1209_5421_gb300.build --bounds-check`), every gather of the cycle's and the batch
 * kernel's ops checks its index against the vector's length; an index outside it is skipped
 * and sets a flag. *flags receives the flags set since the last call (0: none) and clears
 * them. Errors: AMG_ERR_UNSUPPORTED in a library built without the checks (the default).
 */
int amg_debug_bounds_flags(int32_t *flags);

/*
 * Bytes currently allocated from `device`'s default stream-ordered memory pool, which every
 * device allocation of the library uses (freed blocks return to it once their stream reaches
 * the free: synchronise first). A leak check compares it before and after a call.
 */
int amg_debug_pool_bytes_in_use(int32_t device, int64_t *bytes);

#ifdef __cplusplus
}
#endif

#endif /* AMG_GB300_AMG_H */
