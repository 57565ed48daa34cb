// Internal structures of the GB300 auxiliary-grid AMG library.
//
// Data layout in HBM (every level, "pi order"):
//   Rows of each level are stored permuted into the smoother's sweep order pi (colour
//   ascending, then aggregate, then -- on the finest level -- unknown ascending inside the
//   aggregate; paper Sec. 4.5). Every colour is therefore one contiguous row range, every
//   finest-level block (aggregate) a contiguous row range, and restriction from the finest
//   level is a contiguous segmented sum.
//   Matrices are sliced ELL with slices of 32 rows (one warp): inside a slice, entry k of row
//   r sits at sl_ptr[r/32] + 32*k + r%32, so a warp reading slot k of its 32 rows touches one
//   contiguous 256-byte (FP64) segment. Slot 0 holds the diagonal (paper Sec. 4.1 keeps the
//   diagonal first); padding has col = -1, val = 0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/amg.h"

namespace amg {

constexpr int kSliceH = 32;        // sliced-ELL slice height (one warp)
constexpr int kMaxKcycle = 4;      // largest supported kcycle_n
constexpr int kMaxSweeps = 4;      // largest supported nu_pre / nu_post
constexpr int kMaxLevels = 20;
constexpr int kRedBlocks = 608;    // blocks of the deterministic reductions (4 x 152 SMs)
constexpr int kRedThreads = 256;
constexpr int kMaxCoarsest = 256;  // largest exact coarsest level
constexpr int kBatchDirs = 32;     // outer directions a batched system starts with (grown on demand)

// scalar slots of a level's device scalar array
// (one slot per Alg. 1 step where a kernel reads the previous step's value while writing its
// own, so no grid-wide kernel reads a slot it also writes)
enum : int {
    SC_PQ0 = 0,       // (p_i, A p_i) for i = 0..kMaxKcycle-1
    SC_RP0 = 4,       // (r_i, p_i)
    SC_ZQ0 = 8,       // (z, A p_j) for j = 0..kMaxKcycle-1 (current step)
    SC_RR0 = 12,      // (r_{i+1}, r_{i+1}) written by step i
    SC_STOP0 = 16,    // 1.0 if Alg. 1 stopped at or before step i
    SC_N = 24
};

// Big aggregates of the finest level (graded meshes put thousands of unknowns in one
// auxiliary cell): their Gauss-Seidel sweep runs on a warp (blocks of up to kWarpBlockRows
// rows) or a whole CTA, in level order. The level of a row in a forward sweep is 1 + the
// largest level of the rows of its block it depends on (coupled rows earlier in the sweep),
// 0 if none; rows of one level are independent, and every earlier coupled row has a lower
// level, so sweeping level by level reads exactly the values the sequential sweep reads:
// the same result, bit for bit. The backward sweep has its own levels (dependencies on
// later rows).
constexpr int kBigBlockRows = 16;
constexpr int kWarpBlockRows = 128;
struct BigSched {
    int nbig;
    const int *ids;              // [nbig] big block ids: colour by colour (block order), and
                                 // inside a colour the warp-sized blocks first
    const int *lofs_f, *lofs_b;  // [nbig + 1]: block k's level boundaries start at lp_*[lofs_*[k]]
    const int *lp_f, *lp_b;      // level boundaries: positions in ent_* (level j of block k is
                                 // ent_*[lp[lofs[k] + j] .. lp[lofs[k] + j + 1]))
    const int4 *ent_f, *ent_b;   // rows of every big block in level order: (pi row, first
                                 // slot, slot count, offset of the row's off-diagonal slots
                                 // among the block's, in this order)
};

// shared-memory bytes of a big block's sweep in shared memory (big_block_smem): rows m,
// levels nl, off-diagonal slots ns, value size vb; 0 if it cannot be done there (16-bit
// row, slot and entry indices)
__host__ __device__ inline size_t big_smem_align(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ inline size_t big_smem_bytes(int m, int nl, int ns, int vb) {
    if (m > 65535 || ns > 65535) return 0;
    return big_smem_align((size_t)3 * m * vb) + big_smem_align((size_t)6 * m) +
           big_smem_align((size_t)2 * (nl + 1)) + big_smem_align((size_t)2 * ns * vb) +
           big_smem_align((size_t)2 * ns);
}

struct Sell {
    int n = 0;
    int nslices = 0;
    int *sl_ptr = nullptr;   // [nslices+1]
    int *col = nullptr;      // [padded]
    double *val = nullptr;   // [padded]
    float *val32 = nullptr;  // FP32 copy of val (FP32 cycle only)
    int64_t padded = 0;
    int64_t stored = 0;
    int uw = 0;              // > 0: every slice has this width (sl_ptr[s] = 32 uw s)
};

template <class T>
struct Vecs {
    T *rhs = nullptr, *e = nullptr, *r = nullptr, *z = nullptr;
    T *p[kMaxKcycle] = {}, *q[kMaxKcycle] = {};
};

struct Level {
    int n = 0;
    int cellw = 0;          // cells per side of the grid the rows live on
    int span = 0, m = 2, ncolors = 4;
    bool coarsest = false;
    Sell A;
    std::vector<int> color_rows;    // host [ncolors+1]: pi-row range of each colour
    std::vector<int64_t> color_nnz; // host [ncolors]: stored entries of each colour's rows
    unsigned long long *d_color_nnz = nullptr;  // the same on the device, read back at the
                                                // end of setup
    std::vector<int> color_blocks;  // host [ncolors+1] (finest level): block range per colour
    int nblocks = 0;
    int *bptr = nullptr;    // finest level: [nblocks+1] pi-row range of each block
    // finest level: blocks of more than kBigBlockRows rows, swept in level order by warps
    // and CTAs
    int nbig = 0;
    const BigSched *big_dev = nullptr;  // device copy of the schedule
    std::vector<int> color_big;     // host [ncolors+1]: each colour's range of big blocks
    std::vector<int> color_bigc;    // host [ncolors]: where each colour's CTA-sized ones start
    std::vector<size_t> big_smem[2];  // shared memory each CTA-sized big block's sweep
                                      // needs (big_smem_bytes; FP32, FP64 values)
    size_t big_smem_warp[2] = {0, 0};  // the most a warp-sized one needs
    int *parent = nullptr;  // [n] pi-row of the next coarser level
    int4 *children = nullptr;  // level >= 2: [n] children pi-rows in level-1 by quadrant
    int4 *children2 = nullptr; // octree: children 4..7 (octant (t1&1) + 2 (t2&1) + 4 (t3&1))
    int *nat = nullptr;     // [n] natural index of pi-row p
    int *inv = nullptr;     // [n] pi-row of natural index
    int *cell = nullptr;    // [n] cell index t1 + cellw * t2 of pi-row p
    int *agg_nat = nullptr; // [n] natural aggregate (next level) of natural row
    unsigned short *col16 = nullptr;  // 16-bit columns (a tail level read in place)
    double *dinv64 = nullptr;  // 1 / a_ii (smoother), FP64 and FP32
    float *dinv32 = nullptr;
    double *Ainv = nullptr; // coarsest: dense inverse, pi order, row-major
    float *Ainv32 = nullptr; // the same inverse as float high parts then low parts (2 n^2)
    Vecs<double> v64;
    Vecs<float> v32;
    double *sc = nullptr;   // [SC_N] device scalars of Alg. 1 on this level
};

struct Profiler;
struct EngineBase;

// outer-iteration workspace of a hierarchy solved inside a batch (batch.cu); allocated on the
// hierarchy's first batched solve and owned by it
struct BatchWs {
    double *bo = nullptr, *xo = nullptr, *to = nullptr;
    double *pq = nullptr;           // (p_j, q_j) of the outer directions (the hierarchy's P, Q)
    int *colors = nullptr;          // colour ranges of every level, concatenated
    int cofs[kMaxLevels] = {}, ncol[kMaxLevels] = {};
    int4 *bigr = nullptr;           // finest level's colours: their big blocks (bb0, bbc, bb1)
};

// Many small arrays carved from a few large allocations (a bump allocator over chunks): a
// hierarchy of the batched setup takes its arrays from its own arena, which it frees with
// itself. Every piece is 256-byte aligned.
struct Arena {
    cudaStream_t s = nullptr;
    std::vector<void *> chunks;
    char *cur = nullptr;
    size_t left = 0;
    size_t bytes = 0;                 // allocated chunk bytes
    size_t chunk = size_t(1) << 20;   // chunk size (a larger piece gets a chunk of its own)
    void *get(size_t b);
    void release();
};

}  // namespace amg

struct amg_hierarchy {
    amg_options opt{};
    int L = 0;
    int dim = 2;                        // 2: quadtree (x, y), 3: octree (x, y, z)
    double bbox[6] = {0, 0, 0, 0, 0, 0};  // a1, b1, a2, b2, a3, b3
    int nlev = 0;
    int64_t N = 0;
    std::vector<amg::Level> lev;
    cudaStream_t stream = nullptr;      // private non-blocking stream of the hierarchy
    cudaEvent_t order_ev = nullptr;     // orders it after the caller's stream
    int device = 0;
    // allocations owned by the hierarchy
    std::vector<void *> allocs;
    amg::Arena arena;                   // the batched setup's arrays of this hierarchy
    size_t bytes = 0;
    // deterministic reduction scratch
    double *red_partials = nullptr;   // [kRedBlocks * kMaxRed]
    unsigned int *red_counter = nullptr;
    int *err_flag = nullptr;
    // outer Krylov state
    double *xo = nullptr, *ro = nullptr, *zo = nullptr, *to = nullptr;  // pi order
    double *bo = nullptr;
    int outer_cap = 0;
    std::vector<double *> P, Q;        // directions p_j, A p_j
    double **dP = nullptr, **dQ = nullptr;
    double *osc = nullptr;             // outer scalars
    int *oit = nullptr;                // device iteration counter
    double *h_pinned = nullptr;        // pinned host scalars (allocated on first use)
    // FGMRES state (FP64 basis)
    double *gm_V = nullptr, *gm_Z = nullptr, *gm_H = nullptr;
    int gm_cap = 0;
    // FP32 cycle buffers for outer<->cycle conversion
    float *r32 = nullptr, *z32 = nullptr;
    // persistent cycle engines (FP64 / FP32 cycle), their reduction buffer and grid barrier
    amg::EngineBase *eng64 = nullptr, *eng32 = nullptr;
    double *cyc_partials = nullptr;    // [2][4][grid]
    unsigned long long *bar = nullptr; // grid-barrier arrival counter
    // host staging for host-memory arguments
    double *stage_b = nullptr, *stage_x = nullptr;
    // natural-order cells and colours of every level (inspection)
    std::vector<int *> cell_nat, color_nat;
    // per-level device tables (solve.cu)
    void *lev_tab64 = nullptr, *lev_tab32 = nullptr;
    int tail_level = -1;
    bool fp32_ready = false;
    amg::BatchWs bws;                  // batched solves (allocated on first use)
    // diagnostics: per-op CUDA-event profiling and launch counts (solve.cu)
    amg::Profiler *prof = nullptr;
    int64_t setup_launches = 0, solve_launches = 0;
    // host-set barrier fault of the cycle kernel (amg_debug_barrier_fault): 0 = none
    int64_t dbg_bar_limit_ns = 0;
    int dbg_bar_extra = 0;
};

namespace amg {

// ---- error handling -------------------------------------------------------------------
struct Error {
    int status;
    std::string what;
};

#define AMG_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            throw ::amg::Error{e_ == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA, \
                               std::string(#call) + ": " + cudaGetErrorString(e_)};      \
        }                                                                                \
    } while (0)

// records `what` as the text amg_last_error returns on this host thread; returns status
int set_last_error(int status, const char *what);

// every kernel launch is followed by AMG_LAUNCH_CHECK, which also counts it
extern thread_local int64_t g_launches;
#define AMG_LAUNCH_CHECK()            \
    do {                              \
        ++::amg::g_launches;          \
        AMG_CUDA(cudaGetLastError()); \
    } while (0)

inline int nblocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : b);
}

// ---- allocation (stream-ordered, tracked by the hierarchy) ----------------------------
// Every device allocation of the library goes through device_alloc. A host-set fault
// (amg_debug_fail_allocation) makes the k-th one from then on fail as if the device had no
// memory left: it throws the library's out-of-memory error without calling CUDA.
bool fail_this_allocation();  // capi.cu: counts down the armed fault
inline void device_alloc(void **p, size_t bytes, cudaStream_t s) {
    if (fail_this_allocation())
        throw Error{AMG_ERR_OOM, "device allocation failed (host-set fault)"};
    AMG_CUDA(cudaMallocAsync(p, bytes, s));
}

template <class T>
T *halloc(amg_hierarchy *h, size_t count) {
    void *p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    device_alloc(&p, bytes, h->stream);
    h->allocs.push_back(p);
    h->bytes += bytes;
    return (T *)p;
}

// Arena::get and Arena::release (declared before amg_hierarchy): a new chunk comes from
// device_alloc, so the host-set allocation fault reaches it too
inline void *Arena::get(size_t b) {
    b = (std::max<size_t>(b, 16) + 255) & ~size_t(255);
    if (b > left) {
        const size_t c = std::max(b, chunk);
        void *p = nullptr;
        device_alloc(&p, c, s);
        chunks.push_back(p);
        bytes += c;
        cur = (char *)p;
        left = c;
        chunk = std::max<size_t>(chunk / 4, size_t(1) << 20);  // the first chunk fell short
    }
    void *r = cur;
    cur += b;
    left -= b;
    return r;
}
inline void Arena::release() {
    for (void *p : chunks) cudaFreeAsync(p, s);
    chunks.clear();
    cur = nullptr;
    left = 0;
    bytes = 0;
}

// scratch allocation freed by the owner (RAII)
struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t s_) : s(s_) {}
    template <class T>
    T *get(size_t count) {
        void *p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        device_alloc(&p, bytes, s);
        ptrs.push_back(p);
        return (T *)p;
    }
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
};

// ---- primitives (scan_sort.cu) --------------------------------------------------------
// Exclusive prefix sum of in[0..n) into out (may alias in); the total goes to *d_total
// (device int) if non-null. Deterministic.
void exclusive_scan(const int *in, int *out, int n, int *d_total, cudaStream_t s);
// Stable sort of (key, val) pairs by key, keys in [0, 2^key_bits). Results replace the
// inputs. Deterministic (LSD radix sort, 8-bit digits).
void stable_sort_pairs(int *keys, int *vals, int n, int key_bits, cudaStream_t s);

// ---- setup (setup.cu) and solve (solve.cu) --------------------------------------------
// make the hierarchy's stream wait for all work already queued on the caller's stream
inline void bind_stream(amg_hierarchy *h, void *user_stream) {
    AMG_CUDA(cudaEventRecord(h->order_ev, (cudaStream_t)user_stream));
    AMG_CUDA(cudaStreamWaitEvent(h->stream, h->order_ev, 0));
}

// z: NULL for the quadtree (h->dim 2), the third coordinates for the octree (h->dim 3)
void build_hierarchy(amg_hierarchy *h, const amg_csr &A, const double *x, const double *y,
                     const double *z);
void free_engines(amg_hierarchy *h);
void profiler_enable(amg_hierarchy *h, int mode);
void profiler_free(amg_hierarchy *h);
int profiler_read(const amg_hierarchy *h, int cap, int32_t *kind, int32_t *level,
                  int64_t *launches, double *ms, double *bytes);
const char *kernel_name(int kind);
void allocate_solve_workspace(amg_hierarchy *h);
int solve(amg_hierarchy *h, const double *b, double tol, double *x, int *iters,
          double *relres);
void apply_cycle_level(amg_hierarchy *h, int level, const double *f_nat, double *z_nat);
void prepare_cycle(amg_hierarchy *h);
// what a batched solve needs of a hierarchy beyond its setup: the FP32 cycle's copies (FP32
// cycle) and the batched-solve workspace; idempotent, synchronises h->stream
void batch_prepare(amg_hierarchy *h);
// doubles of the outer iteration's device scalars (h->osc) for max_iters iterations
size_t outer_scalar_count(int max_iters);
// algorithmic bytes of one application of B^_0 (Alg. 2 over every level, values of
// value_bytes bytes; the per-op counts of the cycle's roofline)
double cycle_application_bytes(amg_hierarchy *h, int value_bytes);
// host image of h's device level table in the cycle precision fp32 (LevelDev<T, int>[nlev]):
// what the level table holds once the level arrays exist; returns its size in bytes
size_t level_table_image(amg_hierarchy *h, bool fp32, std::vector<unsigned char> &out);
// the finest level's big blocks and their level-ordered sweep schedules (setup.cu)
void build_fine_big_blocks(amg_hierarchy *h);
// Batched setup (setup_batch.cu): every hierarchy of hs (created, options and sizes set, no
// levels yet; system p is rows[p] of the block-diagonal A: rows r0 .. r0 + n, entries
// nz0 .. nz0 + nnz; x, y device; every system has more than coarsest_max unknowns) is built
// by one set of multi-system kernels on stream s, its arrays in its own arena; then each
// hierarchy is ready for amg_solve like one from amg_setup, and with batch_ws also for
// batched solves (as after batch_prepare). Throws amg::Error.
struct BatchRows {
    int r0, n, nz0, nnz;
};
void build_batch(const std::vector<amg_hierarchy *> &hs, const amg_csr &A, const double *x,
                 const double *y, const std::vector<BatchRows> &rows, cudaStream_t s,
                 bool batch_ws);
// the pinned host scalars of the single-system solver (allocated on first use)
void ensure_pinned(amg_hierarchy *h);
// outer directions P[j], Q[j] (and the device tables dP, dQ) for j < count at least, in
// chunks, at most max_iters; returns the number allocated. Synchronises h->stream.
int ensure_directions(amg_hierarchy *h, int count);
const void *level_table(const amg_hierarchy *h, bool fp32);

// ---- batched solves (batch.cu) ------------------------------------------------------------
struct BatchEngine;
// hierarchies of the systems (built, not owned); row_off[p] = first row of system p in the
// concatenated vectors (nprob + 1 entries); every hierarchy has the same options
// shape_threads: 0 = time the candidate launch shapes on the first solve and keep the
// fastest; 1024, 512 or 256 = that many threads per CTA (1, 2 or 4 CTAs per SM)
BatchEngine *batch_create(const std::vector<amg_hierarchy *> &hs, const std::vector<int64_t> &row_off,
                          cudaStream_t stream, int shape_threads);
void batch_destroy(BatchEngine *E);
size_t batch_bytes(const BatchEngine *E);
// b, x: device, concatenated; per-system results into host arrays (may be null); returns
// AMG_OK or the first failing system's status
int batch_solve(BatchEngine *E, const double *b, double tol, double *x, int *iters,
                double *relres, int *status);
// chosen launch shape (-1 before the first solve): threads per CTA, CTAs, and the time of
// one solve of the batch for every candidate shape (ms, -1 if not runnable)
int batch_shape(const BatchEngine *E, int *threads, int *ctas, double *tuned_ms);
// per-system start / end of the last solve (ns after the earliest start; host arrays)
void batch_timeline(const BatchEngine *E, int64_t *start_ns, int64_t *end_ns);
// teams: max_team 0 = sized per system, 1 = one CTA per system, 2..8 = sized, at most that
// many CTAs; an autotuned batch times its shapes again on the next solve
void batch_set_teams(BatchEngine *E, int max_team);
// CTAs of each system's team in the chosen launch shape (host array; -1 before a solve)
void batch_teams(const BatchEngine *E, int *team);
// algorithmic bytes the last batch_solve moved (every system's cycles and outer steps)
double batch_moved_bytes(BatchEngine *E);
// host-set fault of the team barriers for the following solves: limit_ns > 0 replaces the
// wait limit, extra > 0 makes every team's first barrier wait for that many more arrivals
// than its members make (so it runs out); 0, 0 restores the defaults
void batch_barrier_fault(BatchEngine *E, int64_t limit_ns, int extra);
void smooth_level(amg_hierarchy *h, int level, int backward, const double *f_nat,
                  double *u_nat);
// the bounds-checking build's flags of solve.cu's and batch.cu's kernels, read and cleared
// (-1: the library was built without index checks)
int bounds_flags_solve();
int bounds_flags_batch();

}  // namespace amg
