// Device building blocks of the AMLI-cycle (paper Alg. 1, Alg. 2, Sec. 4.3, Sec. 4.5): the
// operation descriptors, level views, deterministic reductions, the bounded grid barrier
// and every cycle operation as a row-parallel device function ("thread tid of nth").
// The same functions run in three executors (solve.cu): one multi-CTA kernel per op, a
// persistent cooperative kernel that runs a whole program of ops with grid barriers, and a
// single-CTA interpreter over levels staged in shared memory.
#pragma once

#include <stdint.h>

#include "amg_internal.cuh"

namespace amg {

enum OpKind : int {
    OP_ZERO = 0,      // u = 0
    OP_GS,            // one colour of a Gauss-Seidel sweep: rows/blocks [i0, i1)
    OP_RESTRICT,      // next.rhs = P^t (f - A u)
    OP_PROLONG,       // u += P next.e
    OP_COARSE,        // e = A^{-1} rhs (coarsest level)
    OP_MULTIDOT,      // sc[ZQ_j] = (p_i, q_j), j < i
    OP_ORTH,          // p_i += sum_j beta_ij p_j, beta_ij = -sc[ZQ_j] / sc[PQ_j]
    OP_SPMV_DOT,      // q_i = A p_i, sc[PQ_i] = (p_i, q_i), sc[RP_i] = (r_i, p_i)
    OP_UPDATE,        // alpha_i; e (+)= alpha_i p_i; r = r_i - alpha_i q_i; sc[RR_i] = (r, r)
    OP_TAIL,          // persistent program: CTA 0 runs the tail program in shared memory
    OP_NOP,           // persistent program: only the prologue (finalise a reduction)
    OP_GS_FIRST,      // point GS from zero, first colour: u_i = f_i / a_ii on [i0, i1), 0 elsewhere
    OP_RESID,         // first pass of a split restriction: q_step = f - A u (row by row)
    OP_GATHER,        // second pass: next.rhs[R] = sum of q_step over R's children
    OP_NKINDS
};

struct Op {
    int kind;
    int level;
    int i0, i1;       // GS range (blocks on the finest level, rows elsewhere)
    int backward;     // GS direction
    int step;         // Alg. 1 step index i
    int last;         // Alg. 1: last step
    int fsel, usel;   // vector selectors (vec_of)
    // persistent executor: reductions leave per-CTA partials in buffer red_pb; the next op
    // sums them (every CTA, same order) into sc of fin_level at fin_dst[0..fin_n)
    int red_pb;
    int fin_pb, fin_level, fin_n;
    int fin_dst[4];
    // RESTRICT / UPDATE: also do the first op of the next pre-smoothing, the point-GS first
    // colour [f0, f1) from zero (OP_GS_FIRST), on the value just computed in the same thread:
    // RESTRICT for B^ of the next level (u = next.p_0, f = next.rhs), UPDATE (not last) for
    // the next Alg. 1 step (u = p_{i+1}, f = r)
    int fuse, f0, f1;
    // finest level, grid-wide executors: big blocks (aggregates of more than kBigBlockRows
    // unknowns) [bb0, bb1) of L.big->ids, swept by warps ([bb0, bbc)) and whole CTAs ([bbc,
    // bb1)) for GS (this colour's), summed by CTAs for RESTRICT (all); 0, 0, 0 = none (every
    // block is one thread's, as in the batch and tail executors)
    int bb0, bbc, bb1;
};


enum : int { V_RHS = 0, V_E, V_R, V_P0 };  // V_P0 + i = p_i

// view of one level; I = column index type (int in HBM, uint16 in the shared-memory tail);
// B = 1 compiles the lane-parallel block smoother of finest levels with multi-row blocks
// (a separate kernel instance, so that the code of the others stays as it is)
template <class T, class I, int B = 0>
struct LevelDev {
    using val_t = T;
    using idx_t = I;
    static constexpr int coop = B;
    int n;
    int fine;                       // 1 on the finest level (block smoother, bptr)
    int bg;                         // finest level: lanes that share a block (kBlockLanes), or
                                    // 0: one thread per block
    int w;                          // > 0: every slice has width w (sl not read)
    const int *sl;
    const I *col;
    const T *val;
    const T *dinv;                  // 1 / a_ii (smoother)
    const unsigned short *col16;    // 16-bit copy of col (levels read by the tail from HBM)
    const int *bptr;
    const BigSched *big;            // finest level: the big blocks' sweep schedule, or NULL
    const int *parent;
    const int4 *children;           // children of the NEXT coarser level's rows
    const int4 *children2;          // octree: their children 4..7 (NULL on a quadtree)
    const double *Ainv;             // coarsest: dense inverse, FP64 (FP64 cycle)
    const float *Ainv2;             // coarsest, FP32 cycle: the same inverse as n*n high parts
                                    // followed by n*n low parts (Ainv ~ high + low)
    T *rhs, *e, *r;
    T *p[kMaxKcycle], *q[kMaxKcycle];
    double *sc;
    int nnext;
};

// view of a level staged in shared memory with one slice width for the whole level: entry k
// of row i at (i / 32) 32 w + 32 k + i % 32, w = W (compile-time) or the member w (W = 0).
// No slice pointers to load, and with W fixed every row loop is unrolled without bounds.
template <class T, int W>
struct StagedLevel {
    using val_t = T;
    using idx_t = unsigned short;
    static constexpr int fine = 0;  // point smoother (staged levels are coarse)
    static constexpr int bg = 0;
    static constexpr int coop = 0;
    int n, w;
    const unsigned short *col;
    const T *val;
    const T *dinv;
    const int *bptr;                // unused (fine = 0)
    static constexpr const BigSched *big = nullptr;
    const int *parent;
    const int4 *children;           // children of the NEXT coarser level's rows
    const int4 *children2;          // octree: their children 4..7 (NULL on a quadtree)
    const double *Ainv;
    const float *Ainv2;
    T *rhs, *e, *r;
    T *p[kMaxKcycle], *q[kMaxKcycle];
    double *sc;
    int nnext;
};

// first slot and slot count of row i
template <class T, class I, int B>
__device__ __forceinline__ void row_span(const LevelDev<T, I, B> &L, int i, int &base,
                                         int &width) {
    const int s = i >> 5;
    if (L.w > 0) {
        width = L.w;
        base = s * 32 * width + (i & 31);
    } else {
        const int a = L.sl[s];
        base = a + (i & 31);
        width = (L.sl[s + 1] - a) >> 5;
    }
}
template <class T, int W>
__device__ __forceinline__ void row_span(const StagedLevel<T, W> &L, int i, int &base,
                                         int &width) {
    width = W > 0 ? W : L.w;
    base = (i >> 5) * 32 * width + (i & 31);
}

// Index checks of the bounds-checking build (compiled with -DAMG_BOUNDS_CHECK): an index of
// a gather outside [0, n) sets this translation unit's flag (amg_debug_bounds_flags reads it)
// and the access is skipped, so a bad index is reported instead of read. The normal build
// checks nothing here: setup builds every index and validates the input matrix.
#ifdef AMG_BOUNDS_CHECK
static __device__ unsigned int g_bounds_err;
__device__ __forceinline__ bool idx_ok(int i, int n) {
    if ((unsigned)i < (unsigned)n) return true;
    atomicOr(&g_bounds_err, 1u);
    return false;
}
// this translation unit's flag, read and cleared (host; -1 when the flag is not built)
static inline int bounds_flag_read_clear() {
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_err, sizeof v) != cudaSuccess ||
        cudaMemcpyToSymbol(g_bounds_err, &zero, sizeof zero) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int)v;
}
#else
__device__ __forceinline__ constexpr bool idx_ok(int, int) { return true; }
static inline int bounds_flag_read_clear() { return -1; }
#endif

__device__ __forceinline__ bool col_ok(int c) { return c >= 0; }
__device__ __forceinline__ bool col_ok(unsigned short c) { return c != (unsigned short)0xFFFF; }

// a[i] for a run-time i, as a chain of selects: a view built in registers keeps its pointer
// arrays in registers (an indexed access would move them to the stack)
template <class P>
__device__ __forceinline__ P pick(const P (&a)[kMaxKcycle], int i) {
    P r = a[0];
#pragma unroll
    for (int k = 1; k < kMaxKcycle; k++)
        if (i == k) r = a[k];
    return r;
}

template <class LV>
__device__ __forceinline__ typename LV::val_t *vec_of(const LV &L, int sel) {
    return sel == V_RHS ? L.rhs : sel == V_E ? L.e : sel == V_R ? L.r : pick(L.p, sel - V_P0);
}

// ---------------------------------------------------------------------------------------
// the threads of one CTA that run an op together, and the barrier they meet at
struct BlockGroup {  // every thread of the CTA; barrier 0
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ int nwarps() const { return (blockDim.x + 31) >> 5; }
};
struct WarpGroup {  // warps [0, nthreads / 32) of the CTA; hardware barrier 1
    int nthreads;   // multiple of 32
    __device__ __forceinline__ void sync() const {
        asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
    }
    __device__ __forceinline__ int nwarps() const { return nthreads >> 5; }
};

// ---------------------------------------------------------------------------------------
// reductions: fixed-order trees, no floating-point atomics (bitwise reproducible)
enum : int { RM_LASTBLOCK = 0, RM_BLOCK = 1, RM_PARTIAL = 2, RM_TEAM = 3 };

// GB300 executes FP64 arithmetic at a small fraction of its FP32 rate, so reductions keep
// FP64 work low: in the FP32 cycle a block sums in FP32 (a warp tree, then one warp over the
// per-warp sums) and only the sum over CTAs is FP64; FP64 partials go through shared memory
// and one warp sums them (32 values per lane in fixed order, then a 5-level shuffle tree),
// about one FP64 add per partial instead of five for a shuffle tree over every warp.
__device__ __forceinline__ double *red_scratch() {
    __shared__ double s[1024];  // >= blockDim.x (1024 at most)
    return s;
}

__device__ __forceinline__ double warp_sum(double y) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
    return y;
}

// r[k] (valid in thread 0) = sum of v[k] over group g; every thread of g must call it. The
// caller synchronises g before the scratch is used again (every executor puts a barrier
// between two ops, and no op reduces twice).
template <int NV, class A, class G>
__device__ __forceinline__ void block_sum(const A (&v)[NV], double (&r)[NV], const G &g) {
    double *s = red_scratch();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = g.nwarps();
    if constexpr (sizeof(A) == 4) {
        // FP32 cycle: a warp tree, then one warp combines the per-warp sums, all in FP32
        float *sf = reinterpret_cast<float *>(s);
#pragma unroll
        for (int k = 0; k < NV; k++) {
            float x = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) sf[k * 32 + w] = x;
        }
        g.sync();
        if (w == 0)
#pragma unroll
            for (int k = 0; k < NV; k++) {
                float x = lane < nw ? sf[k * 32 + lane] : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                r[k] = (double)x;
            }
    } else {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            if (k > 0) g.sync();
            s[threadIdx.x] = (double)v[k];
            g.sync();
            if (w == 0) {
                double y = 0.0;
                for (int j = lane; j < 32 * nw; j += 32) y += s[j];
                r[k] = warp_sum(y);
            }
        }
    }
}

struct RedCtx {
    double *partials;        // LASTBLOCK: [NV][gridDim]; PARTIAL: [2][4][gridDim]; TEAM: [4][size]
    unsigned int *counter;   // LASTBLOCK and TEAM
    int rank = 0, size = 1;  // TEAM: this CTA's rank in the team of CTAs that runs the op
};

// RM_TEAM over more than one CTA (out of line: the one-CTA path of the same ops stays
// small). Every thread of the CTA calls it; r is valid in thread 0. The team's partials are
// summed in rank order by its last CTA to arrive, which also re-arms the counter.
static __device__ __noinline__ void team_reduce_store(const double *r, int nv,
                                                      double *const *out, RedCtx rc) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int k = 0; k < nv; k++) rc.partials[k * rc.size + rc.rank] = r[k];
        __threadfence();
        const unsigned t = atomicAdd(rc.counter, 1u);
        last = (t == (unsigned)rc.size - 1);
    }
    __syncthreads();
    if (last && threadIdx.x < 32) {
        __threadfence();
        for (int k = 0; k < nv; k++) {
            double y = 0.0;
            for (int b = threadIdx.x; b < rc.size; b += 32) y += __ldcg(&rc.partials[k * rc.size + b]);
            y = warp_sum(y);
            if (threadIdx.x == 0 && out[k]) *out[k] = y;
        }
        if (threadIdx.x == 0) *rc.counter = 0u;
    }
}

// RM_LASTBLOCK: per-block partial; the last block to finish sums them in block order.
// RM_BLOCK (one CTA): the block sum. RM_PARTIAL (persistent kernel): per-block partials
// into buffer pb; the next op sums them. RM_TEAM: LASTBLOCK over the rc.size CTAs of a team
// (team_reduce_store; a team of one is RM_BLOCK; the group must be the whole CTA). Final
// values are stored by thread 0 into out[k]; they are visible to the team after its next
// barrier.
template <int NV, int RM, class A, class G>
__device__ __forceinline__ void reduce_store(const A (&v)[NV], double *const (&out)[NV],
                                             const RedCtx &rc, int pb, const G &g) {
    double r[NV];
    block_sum<NV, A>(v, r, g);
    if (RM == RM_BLOCK || (RM == RM_TEAM && rc.size == 1)) {  // visible after the next barrier
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; k++)
                if (out[k]) *out[k] = r[k];
        return;
    }
    if (RM == RM_PARTIAL) {
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; k++)
                rc.partials[((size_t)pb * 4 + k) * gridDim.x + blockIdx.x] = r[k];
        return;
    }
    if (RM == RM_TEAM) {
        team_reduce_store(r, NV, out, rc);
        return;
    }
    __shared__ bool last;
    const int nb = (int)gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) rc.partials[k * nb + blockIdx.x] = r[k];
        __threadfence();
        unsigned t = atomicAdd(rc.counter, 1u);
        last = (t == (unsigned)nb - 1);
    }
    g.sync();
    if (last && threadIdx.x < 32) {
        __threadfence();
#pragma unroll
        for (int k = 0; k < NV; k++) {
            double y = 0.0;
            for (int b = threadIdx.x; b < nb; b += 32) y += __ldcg(&rc.partials[k * nb + b]);
            y = warp_sum(y);
            if (threadIdx.x == 0 && out[k]) *out[k] = y;
        }
        if (threadIdx.x == 0) *rc.counter = 0u;
    }
}

// ---------------------------------------------------------------------------------------
// grid barrier of the persistent cooperative kernel (all CTAs co-resident by construction).
// Every wait is bounded (kBarrierLimitNs); on expiry the CTA raises bit 16 of *err and every
// CTA leaves its op loop at its next barrier.
constexpr unsigned long long kBarrierLimitNs = 2000000000ull;  // 2 s
constexpr int kErrTimeout = 1 << 16;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_volatile_int(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}

// Monotonic counter barrier: every CTA adds 1 with a release reduction and polls with acquire
// loads until the counter reaches (k+1) * gridDim.x for its k-th barrier (the load that sees
// the last arrival orders every later access after the other CTAs' writes; the CTA's other
// threads follow through the closing __syncthreads). The counter is zeroed before every
// launch. Returns false if the kernel must stop.
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ bool grid_barrier(unsigned long long *count, int *err,
                                             unsigned long long &target, int &abort_flag,
                                             unsigned long long limit_ns = kBarrierLimitNs) {
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        red_release_add_u64(count, 1ull);
        unsigned long long t0 = 0;
        int spins = 0;
        while (ld_acquire_u64(count) < target) {
            if ((++spins & 1023) == 0) {
                if (t0 == 0) {
                    t0 = global_ns();
                } else if (global_ns() - t0 > limit_ns || (ld_volatile_int(err) & kErrTimeout)) {
                    atomicOr(err, kErrTimeout);
                    abort_flag = 1;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return abort_flag == 0;
}

// ---------------------------------------------------------------------------------------
// row kernels (sliced ELL: entry k of row i at sl[i/32] + 32 k + i%32, slot 0 = diagonal).
// The small levels are pure latency, so a row's slots are read in batches of 8: all column
// indices and values of a batch are loaded before any gathered x[c], which turns a chain of
// two dependent loads per slot into about three round trips per row.
constexpr int kRowBatch = 9;  // one batch for a 9-point row

// sum over slots k0 <= k < width of a_ik x[c_ik] (padding contributes nothing)
template <class LV>
__device__ __forceinline__ typename LV::val_t row_dot(const LV &L, int base, int k0, int width,
                                                      const typename LV::val_t *x) {
    using T = typename LV::val_t;
    using I = typename LV::idx_t;
    T acc = 0;
    for (int kb = k0; kb < width; kb += kRowBatch) {
        I c[kRowBatch];
        T a[kRowBatch];
#pragma unroll
        for (int j = 0; j < kRowBatch; j++) {
            const int k = kb + j;
            c[j] = k < width ? L.col[base + 32 * k] : (I)-1;
            a[j] = k < width ? L.val[base + 32 * k] : T(0);
        }
        T xv[kRowBatch];
#pragma unroll
        for (int j = 0; j < kRowBatch; j++)
            xv[j] = (col_ok(c[j]) && idx_ok((int)c[j], L.n)) ? x[c[j]] : T(0);
#pragma unroll
        for (int j = 0; j < kRowBatch; j++) acc += a[j] * xv[j];
    }
    return acc;
}

template <class LV>
__device__ __forceinline__ typename LV::val_t row_residual(const LV &L, int i,
                                                           const typename LV::val_t *f,
                                                           const typename LV::val_t *u) {
    int base, width;
    row_span(L, i, base, width);
    return f[i] - row_dot(L, base, 0, width, u);
}

// Gauss-Seidel update of row i: u_i = (f_i - sum_{j != i} a_ij u_j) / a_ii, the division
// taken as a product with the reciprocal diagonal stored at setup
template <class LV>
__device__ __forceinline__ void gs_row(const LV &L, int i, const typename LV::val_t *f,
                                       typename LV::val_t *u) {
    int base, width;
    row_span(L, i, base, width);
    u[i] = (f[i] - row_dot(L, base, 1, width, u)) * L.dinv[i];
}

// ---------------------------------------------------------------------------------------
// the ops
template <class LV>
__device__ void op_zero(const LV &L, typename LV::val_t *u, int tid, int nth) {
    for (int i = tid; i < L.n; i += nth) u[i] = 0;
}

// Block smoother with kBlockLanes lanes per block (finest level, blocks of several rows, as
// the octree's 2x2x2-node aggregates): lane q owns row r0 + q. Phase 1 (all lanes at once)
// gathers the row's terms whose values are final for this row: columns outside the block
// and block rows the sweep reaches after it (still old); the coefficients of block rows the
// sweep reaches before it are kept by local index. Phase 2 walks the block's rows in sweep
// order: the owner finishes its row, the new value goes to the other lanes by a shuffle, and
// each adds its coefficient times that value. The same Gauss-Seidel update as one thread per
// block, summed in another order. Blocks of more than kBlockLanes rows (none on the octree
// workloads) are swept by the group's first lane.
constexpr int kBlockLanes = 16;
constexpr int kBlockEarly = 8;  // coefficients of earlier block rows kept per row

template <class LV>
__device__ __forceinline__ void gs_block_seq(const LV &L, int b, bool backward,
                                             const typename LV::val_t *f, typename LV::val_t *u) {
    const int r0 = L.bptr[b], r1 = L.bptr[b + 1];
    if (!backward)
        for (int i = r0; i < r1; i++) gs_row(L, i, f, u);
    else
        for (int i = r1 - 1; i >= r0; i--) gs_row(L, i, f, u);
}

template <class LV>
__device__ void op_gs_blocks_coop(const LV &L, const Op &op, const typename LV::val_t *f,
                                  typename LV::val_t *u, int tid, int nth, bool skip_big) {
    using T = typename LV::val_t;
    using I = typename LV::idx_t;
    constexpr int G = kBlockLanes;
    const int q = tid & (G - 1);
    const unsigned gmask = 0xFFFFu << ((threadIdx.x & 31) & 16);  // this group's 16 lanes
    const int glane0 = (threadIdx.x & 31) & 16;
    const bool bwd = op.backward != 0;
    for (int base = op.i0; base < op.i1; base += nth / G) {
        const int b = base + tid / G;
        int r0 = 0, k = 0;
        if (b < op.i1) {
            r0 = L.bptr[b];
            k = L.bptr[b + 1] - r0;
        }
        if (k > G) {  // the same for the whole group
            if (q == 0 && !(skip_big && k > kBigBlockRows)) gs_block_seq(L, b, bwd, f, u);
            continue;
        }
        const bool has = q < k;
        const int i = r0 + q;
        T acc = 0, fi = 0, di = 0;
        T early[kBlockEarly];
        unsigned lidx = 0;  // local index of early[t], 4 bits each (t < nearly)
#pragma unroll
        for (int t = 0; t < kBlockEarly; t++) early[t] = 0;
        int nearly = 0;
        bool overflow = false;
        if (has) {
            fi = f[i];
            di = L.dinv[i];
            int rb, width;
            row_span(L, i, rb, width);
            for (int kb = 1; kb < width; kb += kRowBatch) {
                I c[kRowBatch];
                T a[kRowBatch];
#pragma unroll
                for (int j = 0; j < kRowBatch; j++) {
                    const int kk = kb + j;
                    c[j] = kk < width ? L.col[rb + 32 * kk] : (I)-1;
                    a[j] = kk < width ? L.val[rb + 32 * kk] : T(0);
                }
                T xv[kRowBatch];
#pragma unroll
                for (int j = 0; j < kRowBatch; j++) {
                    xv[j] = T(0);
                    if (col_ok(c[j])) {
                        const int li = (int)c[j] - r0;
                        const bool early_row = li >= 0 && li < k && (bwd ? li > q : li < q);
                        if (!early_row) {
                            xv[j] = u[c[j]];
                        } else {
#pragma unroll
                            for (int t = 0; t < kBlockEarly; t++)
                                if (t == nearly) early[t] = a[j];
                            if (nearly < kBlockEarly) lidx |= (unsigned)li << (4 * nearly);
                            else overflow = true;
                            nearly++;
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < kRowBatch; j++) acc += a[j] * xv[j];
            }
        }
        // more than kBlockEarly earlier block rows in a row: the group's first lane sweeps it
        if (__any_sync(gmask, overflow)) {
            if (q == 0) gs_block_seq(L, b, bwd, f, u);
            continue;
        }
        int kmax = k;  // the same in the group
        for (int s = 0; s < kmax; s++) {
            const int j = bwd ? kmax - 1 - s : s;  // block row updated at this step
            T vj = (has && q == j) ? (fi - acc) * di : T(0);
            vj = __shfl_sync(gmask, vj, glane0 + j);
            if (has && q == j) u[i] = vj;
            if (has) {
#pragma unroll
                for (int t = 0; t < kBlockEarly; t++)
                    if (t < nearly && ((lidx >> (4 * t)) & 15u) == (unsigned)j) acc += early[t] * vj;
            }
        }
    }
}

// asynchronous prefetch of [p, p + bytes) into L2 (cp.async.bulk.prefetch), trimmed inward to
// 16-byte boundaries so that it never reaches outside the range
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
    uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    while (a < e) {
        const unsigned chunk = (unsigned)((e - a) < 32768 ? (e - a) : 32768);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(chunk) : "memory");
        a += chunk;
    }
}

// L2 prefetch of what big block k's sweep reads: its level-ordered entries, its rows' slots
// (contiguous slices: the block's rows are consecutive) and its rows' f, 1/a_ii and u
template <class LV>
__device__ void prefetch_big_block(const LV &L, const int *lofs, const int *lp, const int4 *ent,
                                   int k, const typename LV::val_t *f,
                                   const typename LV::val_t *u) {
    using T = typename LV::val_t;
    const BigSched *S = L.big;
    const int blk = S->ids[k];
    const int r0 = L.bptr[blk], r1 = L.bptr[blk + 1];
    const int e0 = lp[lofs[k]], e1 = lp[lofs[k + 1]];
    prefetch_l2(ent + e0, sizeof(int4) * (size_t)(e1 - e0));
    const int s0 = L.sl[r0 >> 5], s1 = L.sl[((r1 - 1) >> 5) + 1];
    prefetch_l2(L.col + s0, sizeof(typename LV::idx_t) * (size_t)(s1 - s0));
    prefetch_l2(L.val + s0, sizeof(T) * (size_t)(s1 - s0));
    prefetch_l2(f + r0, sizeof(T) * (size_t)(r1 - r0));
    prefetch_l2(L.dinv + r0, sizeof(T) * (size_t)(r1 - r0));
    prefetch_l2(u + r0, sizeof(T) * (size_t)(r1 - r0));
}

// every big-block task's data on its way to L2 (one lane per warp task, one thread per CTA
// task), issued before the op's other work so that the level chains wait on L2, not DRAM
template <class LV>
__device__ void prefetch_big_tasks(const LV &L, const Op &op, const typename LV::val_t *f,
                                   const typename LV::val_t *u, int tid, int nth, int crank,
                                   int ccount) {
    const BigSched *S = L.big;
    const bool bwd = op.backward != 0;
    const int *lofs = bwd ? S->lofs_b : S->lofs_f;
    const int *lp = bwd ? S->lp_b : S->lp_f;
    const int4 *ent = bwd ? S->ent_b : S->ent_f;
    if ((tid & 31) == 0)
        for (int k = op.bb0 + (tid >> 5); k < op.bbc; k += nth >> 5)
            prefetch_big_block(L, lofs, lp, ent, k, f, u);
    if (threadIdx.x == 0)
        for (int k = op.bbc + crank; k < op.bb1; k += ccount)
            prefetch_big_block(L, lofs, lp, ent, k, f, u);
}

// Gauss-Seidel update of row i whose slots start at `base` (gs_row without the slice lookup)
template <class LV>
__device__ __forceinline__ void gs_row_at(const LV &L, int i, int base, int width,
                                          const typename LV::val_t *f, typename LV::val_t *u) {
    u[i] = (f[i] - row_dot(L, base, 1, width, u)) * L.dinv[i];
}

// Shared memory a grid-wide executor lends to the big blocks' sweeps: p (null on CTAs
// without it) and its size. With skip0, CTA 0 (whose shared memory holds the tail) takes no
// big block; the warp-sized blocks go to warps [0, wwarps) of the other CTAs, each with a
// slice of wslice bytes at p + warp * wslice (wwarps = 0: to every warp, from global memory).
struct BigScratch {
    unsigned char *p = nullptr;
    unsigned bytes = 0;
    bool skip0 = false;
    int wwarps = 0;
    unsigned wslice = 0;
};

// the threads that sweep one big block together: a CTA, or one warp
struct CtaGroup {
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ int size() const { return blockDim.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct LaneGroup {
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ int size() const { return 32; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// Big block k swept in shared memory (buf, bytes) by group g. Its rows' couplings are staged
// first, in one pass over the block with no dependence between rows: each off-diagonal
// slot's coefficient, and either the current value of a coupled unknown outside the block
// (this colour does not change it) or the index of one inside; with each row's f and
// 1/a_ii. The block's unknowns then live in shared memory and the level-ordered sweep reads
// nothing else: a group barrier between levels, no memory round trip. Every row's sum takes
// its slots in row_dot's order, with row_dot's zero terms up to the end of its last batch:
// the same operations, the same bits. Returns false (nothing done) when the block does not
// fit.
template <class LV, class G>
__device__ bool big_block_smem(const LV &L, const int *lofs, const int *lp, const int4 *ent,
                               int k, const typename LV::val_t *f, typename LV::val_t *u,
                               unsigned char *buf, size_t bytes, const G &g) {
    using T = typename LV::val_t;
    const BigSched *S = L.big;
    const int blk = S->ids[k];
    const int r0 = L.bptr[blk], m = L.bptr[blk + 1] - r0;
    const int l0 = lofs[k], nl = lofs[k + 1] - l0;
    const int e0 = lp[l0];  // the block's rows: ent[e0, e0 + m), level by level
    const int4 last = ent[e0 + m - 1];
    const int ns = last.w + last.z - 1;
    const size_t need = big_smem_bytes(m, nl, ns, (int)sizeof(T));
    if (need == 0 || need > bytes) return false;
    unsigned char *q = buf;
    T *su = (T *)q;  // the block's unknowns (local index = row - r0)
    T *ef = su + m, *ed = ef + m;  // per entry: f, 1/a_ii
    q += big_smem_align((size_t)3 * m * sizeof(T));
    // per entry: local row, first slot, slot count
    unsigned short *erow = (unsigned short *)q, *eo = erow + m, *ew = eo + m;
    q += big_smem_align((size_t)6 * m);
    unsigned short *slp = (unsigned short *)q;  // level boundaries, relative to e0
    q += big_smem_align((size_t)2 * (nl + 1));
    T *sa = (T *)q, *sx = sa + ns;  // per slot: coefficient, outside value
    q += big_smem_align((size_t)2 * ns * sizeof(T));
    unsigned short *si = (unsigned short *)q;  // per slot: inside index, 0xFFFF outside
    const int t = g.rank(), nt = g.size();
    for (int j = t; j <= nl; j += nt) slp[j] = (unsigned short)(lp[l0 + j] - e0);
    for (int i = t; i < m; i += nt) {
        const int4 e = ent[e0 + i];
        const int row = e.x;
        erow[i] = (unsigned short)(row - r0);
        eo[i] = (unsigned short)e.w;
        ew[i] = (unsigned short)e.z;
        ef[i] = f[row];
        ed[i] = L.dinv[row];
        su[row - r0] = u[row];
        for (int kk = 1; kk < e.z; kk++) {
            const auto c = L.col[e.y + 32 * kk];
            const int s = e.w + kk - 1;
            sa[s] = L.val[e.y + 32 * kk];
            unsigned short ix = 0xFFFF;
            T xv = T(0);
            if (col_ok(c) && idx_ok((int)c, L.n)) {
                const int ci = (int)c;
                if (ci >= r0 && ci < r0 + m) ix = (unsigned short)(ci - r0);
                else xv = u[ci];
            }
            si[s] = ix;
            sx[s] = xv;
        }
    }
    g.sync();
    for (int j = 0; j < nl; j++) {
        const int p1 = slp[j + 1];
        for (int i = slp[j] + t; i < p1; i += nt) {
            const int o = (int)eo[i] - 1, w = ew[i];
            T acc = 0;
            int kk = 1;
            for (; kk < w; kk++) {
                const unsigned short ix = si[o + kk];
                const T xv = ix != 0xFFFF ? su[ix] : sx[o + kk];
                acc += sa[o + kk] * xv;
            }
            for (const int kend = 1 + (w + kRowBatch - 2) / kRowBatch * kRowBatch; kk < kend; kk++)
                acc += T(0) * T(0);  // row_dot's zero terms to the end of its batch
            su[erow[i]] = (ef[i] - acc) * ed[i];
        }
        g.sync();
    }
    for (int i = t; i < m; i += nt) u[r0 + i] = su[i];
    g.sync();  // the buffer is used again by the group's next block
    return true;
}

// one big block swept from global memory by group g, level by level
template <class LV, class G>
__device__ void big_block_global(const LV &L, const int *lofs, const int *lp, const int4 *ent,
                                 int k, const typename LV::val_t *f, typename LV::val_t *u,
                                 const G &g) {
    const int l1 = lofs[k + 1];
    for (int j = lofs[k]; j < l1; j++) {
        const int b = lp[j + 1];
        for (int p = lp[j] + g.rank(); p < b; p += g.size()) {
            const int4 e = ent[p];
            gs_row_at(L, e.x, e.y, e.z, f, u);
        }
        g.sync();  // this level's values are read by the next level's rows
    }
}

// the big blocks of one colour in level order: [op.bb0, op.bbc) one warp each,
// [op.bbc, op.bb1) one CTA each; in shared memory where the executor lends it (sc). tid, nth:
// the executor's thread index and count (whole warps); crank, ccount: this CTA's index among
// the executor's CTAs and their number (the grid's, or a batch team's). Every thread of the
// executor calls this.
template <class LV>
__device__ void op_gs_big_blocks(const LV &L, const Op &op, const typename LV::val_t *f,
                                 typename LV::val_t *u, int tid, int nth, int crank,
                                 int ccount, const BigScratch &sc) {
    const BigSched *S = L.big;
    const bool bwd = op.backward != 0;
    const int *lofs = bwd ? S->lofs_b : S->lofs_f;
    const int *lp = bwd ? S->lp_b : S->lp_f;
    const int4 *ent = bwd ? S->ent_b : S->ent_f;
    if (sc.skip0) {  // CTA 0 lends no shared memory: the other CTAs take every big block
        if (blockIdx.x == 0) return;
        crank -= 1;
        ccount -= 1;
        const int w = (int)threadIdx.x >> 5;
        if (sc.wwarps > 0 && w < sc.wwarps) {  // warps with a slice: warp-sized blocks
            unsigned char *slice = sc.p + (size_t)w * sc.wslice;
            for (int k = op.bb0 + w * ccount + crank; k < op.bbc; k += sc.wwarps * ccount)
                if (!big_block_smem(L, lofs, lp, ent, k, f, u, slice, sc.wslice, LaneGroup{}))
                    big_block_global(L, lofs, lp, ent, k, f, u, LaneGroup{});
        } else if (sc.wwarps == 0) {
            const int nw = ((int)blockDim.x >> 5) * ccount;
            for (int k = op.bb0 + w * ccount + crank; k < op.bbc; k += nw)
                big_block_global(L, lofs, lp, ent, k, f, u, LaneGroup{});
        }
        __syncthreads();  // the slices are the CTA-sized blocks' buffer next
    } else {
        for (int k = op.bb0 + (tid >> 5); k < op.bbc; k += nth >> 5)  // warp-sized blocks
            big_block_global(L, lofs, lp, ent, k, f, u, LaneGroup{});
    }
    for (int k = op.bbc + crank; k < op.bb1; k += ccount) {  // larger blocks
        if (sc.p && big_block_smem(L, lofs, lp, ent, k, f, u, sc.p, sc.bytes, CtaGroup{}))
            continue;
        big_block_global(L, lofs, lp, ent, k, f, u, CtaGroup{});
    }
}

// one colour: independent blocks (finest level, rows of a block in sweep order) or rows.
// BIG (the grid-wide executors, whose programs set op.bb0, op.bb1): the colour's big blocks
// are left to the CTA phase at the end. Other executors never see big-block ranges and do
// not compile that phase (nor its shared memory).
template <class LV, bool BIG = false>
__device__ void op_gs(const LV &L, const Op &op, const typename LV::val_t *f,
                      typename LV::val_t *u, int tid, int nth, int crank = -1,
                      int ccount = -1, const BigScratch &sc = BigScratch{}) {
    const bool big = BIG && L.fine && op.bb1 > op.bb0;
    if constexpr (BIG) {
        if (crank < 0) {  // the grid's CTAs
            crank = (int)blockIdx.x;
            ccount = (int)gridDim.x;
        }
        if (big) prefetch_big_tasks(L, op, f, u, tid, nth, crank, ccount);
    } else {
        (void)crank;
        (void)ccount;
    }
    if constexpr (LV::coop) {
        if (L.fine && L.bg > 0) {
            op_gs_blocks_coop(L, op, f, u, tid, nth, big);
            if constexpr (BIG)
                if (big) op_gs_big_blocks(L, op, f, u, tid, nth, crank, ccount, sc);
            return;
        }
    }
    for (int b = op.i0 + tid; b < op.i1; b += nth) {
        if (L.fine) {
            const int r0 = L.bptr[b], r1 = L.bptr[b + 1];
            if (big && r1 - r0 > kBigBlockRows) continue;  // in level order, below
            if (!op.backward)
                for (int i = r0; i < r1; i++) gs_row(L, i, f, u);
            else
                for (int i = r1 - 1; i >= r0; i--) gs_row(L, i, f, u);
        } else {
            gs_row(L, b, f, u);
        }
    }
    if constexpr (BIG)
        if (big) op_gs_big_blocks(L, op, f, u, tid, nth, crank, ccount, sc);
}

// fc = P^t (f - A u): the finest level sums the contiguous block of each aggregate; the
// coarser levels the (up to four, octree eight) children of each coarse cell (Sec. 4.3
// explicit form), one lane per child and a shuffle tree (nth must be a multiple of 32)
// With un non-null, the next level's smoothing starts here as well (Op::fuse):
// un[R] = fc[R] / a_RR on the next level's first colour [f0, f1), 0 elsewhere.
// fc of the finest level's big blocks: a warp per block of up to kWarpBlockRows rows, a CTA
// per larger block; the rows' residuals summed per lane (thread), then over the warp (CTA)
// in a fixed order. tid, nth: the executor's global thread index and count (whole warps).
// Every thread of the grid calls this.
template <class LV>
__device__ void restrict_big_blocks(const LV &L, const typename LV::val_t *f,
                                    const typename LV::val_t *u, typename LV::val_t *fc,
                                    typename LV::val_t *un, const typename LV::val_t *dinv_n,
                                    int f0, int f1, int tid, int nth, int crank, int ccount) {
    using T = typename LV::val_t;
    const BigSched *S = L.big;
    const int lane = tid & 31;
    for (int k = tid >> 5; k < S->nbig; k += nth >> 5) {
        const int R = S->ids[k];
        const int r0 = L.bptr[R], r1 = L.bptr[R + 1];
        if (r1 - r0 > kWarpBlockRows) continue;  // a CTA's, below
        T v = 0;
        for (int i = r0 + lane; i < r1; i += 32) v += row_residual(L, i, f, u);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) {
            fc[R] = v;
            if (un) un[R] = (R >= f0 && R < f1) ? v * dinv_n[R] : T(0);
        }
    }
    for (int k = crank; k < S->nbig; k += ccount) {
        const int R = S->ids[k];
        const int r0 = L.bptr[R], r1 = L.bptr[R + 1];
        if (r1 - r0 <= kWarpBlockRows) continue;  // a warp's, above
        T v[1] = {T(0)};
        for (int i = r0 + (int)threadIdx.x; i < r1; i += (int)blockDim.x)
            v[0] += row_residual(L, i, f, u);
        double r[1];
        block_sum<1, T>(v, r, BlockGroup{});
        if (threadIdx.x == 0) {
            const T sum = (T)r[0];
            fc[R] = sum;
            if (un) un[R] = (R >= f0 && R < f1) ? sum * dinv_n[R] : T(0);
        }
        __syncthreads();  // the reduction scratch is used again by the next block
    }
}

// big = true (grid-wide executors, finest level with big blocks): blocks of more than
// kBigBlockRows rows are summed by warps and CTAs at the end (restrict_big_blocks)
template <class LV>
__device__ void op_restrict(const LV &L, const typename LV::val_t *f,
                            const typename LV::val_t *u, typename LV::val_t *fc, int tid,
                            int nth, typename LV::val_t *un = nullptr,
                            const typename LV::val_t *dinv_n = nullptr, int f0 = 0, int f1 = 0,
                            bool big = false, int crank = -1, int ccount = -1) {
    using T = typename LV::val_t;
    if (crank < 0) {  // the grid's CTAs
        crank = (int)blockIdx.x;
        ccount = (int)gridDim.x;
    }
    if constexpr (LV::coop) {  // kBlockLanes lanes per aggregate: a row each, then a shuffle sum
        if (L.fine && L.bg > 0) {
            constexpr int G = kBlockLanes;
            const int q = tid & (G - 1);
            for (int base = 0; base < L.nnext; base += nth / G) {
                const int R = base + tid / G;
                T v = 0;
                bool mine = R < L.nnext;
                if (mine && big && L.bptr[R + 1] - L.bptr[R] > kBigBlockRows) mine = false;
                if (mine)
                    for (int i = L.bptr[R] + q; i < L.bptr[R + 1]; i += G)
                        v += row_residual(L, i, f, u);
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (mine && q == 0) {
                    fc[R] = v;
                    if (un) un[R] = (R >= f0 && R < f1) ? v * dinv_n[R] : T(0);
                }
            }
            if (big)
                restrict_big_blocks(L, f, u, fc, un, dinv_n, f0, f1, tid, nth, crank, ccount);
            return;
        }
    }
    if (L.fine) {
        for (int R = tid; R < L.nnext; R += nth) {
            const int r0 = L.bptr[R], r1 = L.bptr[R + 1];
            if (big && r1 - r0 > kBigBlockRows) continue;  // by warps / CTAs, below
            T acc = 0;
            for (int i = r0; i < r1; i++) acc += row_residual(L, i, f, u);
            fc[R] = acc;
            if (un) un[R] = (R >= f0 && R < f1) ? acc * dinv_n[R] : T(0);
        }
        if (big)
            restrict_big_blocks(L, f, u, fc, un, dinv_n, f0, f1, tid, nth, crank, ccount);
        return;
    }
    const bool oct = L.children2 != nullptr;
    const int lg = oct ? 3 : 2;  // log2 of the lanes per coarse row
    const int q = tid & ((1 << lg) - 1), per_pass = nth >> lg;
    for (int base = 0; base < L.nnext; base += per_pass) {
        const int R = base + (tid >> lg);
        T v = 0;
        if (R < L.nnext) {
            const int4 ch = (q < 4 ? L.children : L.children2)[R];
            const int qq = q & 3;
            const int c = qq == 0 ? ch.x : qq == 1 ? ch.y : qq == 2 ? ch.z : ch.w;
            if (c >= 0 && idx_ok(c, L.n)) v = row_residual(L, c, f, u);
        }
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (oct) v += __shfl_xor_sync(0xffffffffu, v, 4);
        if (R < L.nnext && q == 0) {
            fc[R] = v;
            if (un) un[R] = (R >= f0 && R < f1) ? v * dinv_n[R] : T(0);
        }
    }
}

// The restriction of a coarse level in two passes, for executors where the children of
// consecutive coarse rows are far apart (they lie in different colours): t = f - A u row by
// row (consecutive rows, contiguous slots), then fc[R] = the sum of t over R's children.
// The sum is taken in op_restrict's order ((t0 + t1) + (t2 + t3), octree + ((t4 + t5) +
// (t6 + t7)), missing children as 0), so both forms give the same bits.
template <class LV>
__device__ void op_resid(const LV &L, const typename LV::val_t *f, const typename LV::val_t *u,
                         typename LV::val_t *t, int tid, int nth) {
    for (int i = tid; i < L.n; i += nth) t[i] = row_residual(L, i, f, u);
}

template <class LV>
__device__ void op_gather_children(const LV &L, const typename LV::val_t *t,
                                   typename LV::val_t *fc, int tid, int nth,
                                   typename LV::val_t *un = nullptr,
                                   const typename LV::val_t *dinv_n = nullptr, int f0 = 0,
                                   int f1 = 0) {
    using T = typename LV::val_t;
    const bool oct = L.children2 != nullptr;
    for (int R = tid; R < L.nnext; R += nth) {
        const int4 ch = L.children[R];
        auto at = [&](int c) { return (c >= 0 && idx_ok(c, L.n)) ? t[c] : T(0); };
        const T a0 = at(ch.x), a1 = at(ch.y), a2 = at(ch.z), a3 = at(ch.w);
        T v = (a0 + a1) + (a2 + a3);
        if (oct) {
            const int4 c2 = L.children2[R];
            const T b0 = at(c2.x), b1 = at(c2.y), b2 = at(c2.z), b3 = at(c2.w);
            v = v + ((b0 + b1) + (b2 + b3));
        }
        fc[R] = v;
        if (un) un[R] = (R >= f0 && R < f1) ? v * dinv_n[R] : T(0);
    }
}

// first colour of a forward sweep from u = 0 on a point-smoothed level: rows of one colour
// are never coupled, so u_i = f_i / a_ii there, and every other row is still 0
template <class LV>
__device__ void op_gs_first(const LV &L, const Op &op, const typename LV::val_t *f,
                            typename LV::val_t *u, int tid, int nth) {
    for (int i = tid; i < L.n; i += nth) u[i] = (i >= op.i0 && i < op.i1) ? f[i] * L.dinv[i] : 0;
}

// u_i += e_{agg(i)} (Sec. 4.3 prolongation)
template <class LV>
__device__ void op_prolong(const LV &L, const typename LV::val_t *e, typename LV::val_t *u,
                           int tid, int nth) {
    for (int i = tid; i < L.n; i += nth) {
        const int pr = L.parent[i];
        if (idx_ok(pr, L.nnext)) u[i] += e[pr];
    }
}

// e = A^{-1} rhs with the dense inverse of the coarsest level, g lanes per row (g = largest
// power of two <= 32 with g * n <= nth) and a shuffle tree. The FP64 cycle accumulates in
// FP64. The FP32 cycle keeps that accuracy with FP32 instructions (FP64 throughput is
// scarce on this GPU): the inverse is stored as float pairs (high + low) and the row sum is
// the compensated dot product "Dot2" of Ogita, Rump and Oishi (Accurate sum and dot
// product, SIAM J. Sci. Comput. 26, 2005): each product is split exactly into a float and
// its rounding error (one fma), each running sum into a float and its rounding error
// (Knuth's two-sum), and the errors are summed on the side; the result is as accurate as a
// sum in twice the working precision, rounded once to FP32 at the end as the FP64 sum is.
// Only the running sum's addition is on the loop-carried path.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    // (the _rn intrinsics keep these steps from being fused into FMAs)
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <class LV>
__device__ void op_coarse(const LV &L, int tid, int nth) {
    using T = typename LV::val_t;
    const int n = L.n;
    int g = 1;
    while (g < 32 && 2 * g * n <= nth) g *= 2;
    const int sub = tid & (g - 1), rows_per_pass = nth / g;
    // the lanes of a warp read 32 / g rows at once: lane `sub` of a row reads columns
    // sub + g t, t < T, starting at t = its row group in the warp, so that rows whose stride
    // is a multiple of the 32 shared-memory banks do not read the same banks in the same step
    const int T_ = (n + g - 1) / g, rot = ((tid & 31) / g) % T_;
    for (int base = 0; base < n; base += rows_per_pass) {
        const int i = base + tid / g;
        if constexpr (sizeof(T) == 4) {
            float s = 0.f, c = 0.f;  // running sum, sum of all rounding errors
            if (i < n) {
                const float *ah = L.Ainv2 + (size_t)i * n, *al = ah + (size_t)n * n;
                // column group tt' = (tt + rot) mod T_, wrapped by a compare (no division)
                for (int tt = 0, tw = rot; tt < T_; tt++, tw = (tw + 1 == T_) ? 0 : tw + 1) {
                    const int j = sub + g * tw;
                    if (j >= n) continue;
                    const float x = L.rhs[j];
                    const float ph = __fmul_rn(ah[j], x);
                    const float pe = fmaf(al[j], x, fmaf(ah[j], x, -ph));  // error + low part
                    float t, e;
                    two_sum(s, ph, t, e);
                    s = t;
                    c = __fadd_rn(c, __fadd_rn(e, pe));
                }
            }
            for (int o = g >> 1; o > 0; o >>= 1) {  // combine lanes: (s, c) + (s', c')
                const float so = __shfl_down_sync(0xffffffffu, s, o, g);
                const float co = __shfl_down_sync(0xffffffffu, c, o, g);
                float t, e;
                two_sum(s, so, t, e);
                s = t;
                c = __fadd_rn(c, __fadd_rn(co, e));
            }
            if (i < n && sub == 0) L.e[i] = __fadd_rn(s, c);
        } else {
            double s = 0.0;
            if (i < n) {
                const double *a = L.Ainv + (size_t)i * n;
                for (int tt = 0, tw = rot; tt < T_; tt++, tw = (tw + 1 == T_) ? 0 : tw + 1) {
                    const int j = sub + g * tw;
                    if (j < n) s += a[j] * (double)L.rhs[j];
                }
            }
            for (int o = g >> 1; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, g);
            if (i < n && sub == 0) L.e[i] = (T)s;
        }
    }
}

template <class LV, int RM, class G>
__device__ void op_multidot(const LV &L, const Op &op, const RedCtx &rc, int tid, int nth,
                            const G &g) {
    using T = typename LV::val_t;
    const int i = op.step;
    T v[kMaxKcycle] = {};
    const T *z = pick(L.p, i);
    for (int r = tid; r < L.n; r += nth) {
        T zr = z[r];
#pragma unroll
        for (int j = 0; j < kMaxKcycle; j++)
            if (j < i) v[j] += zr * L.q[j][r];
    }
    double *out[kMaxKcycle];
#pragma unroll
    for (int j = 0; j < kMaxKcycle; j++) out[j] = j < i ? &L.sc[SC_ZQ0 + j] : nullptr;
    reduce_store<kMaxKcycle, RM, T>(v, out, rc, op.red_pb, g);
}

// a / b for an Alg. 1 coefficient: in FP64 for the FP64 cycle, in FP32 for the FP32 cycle
// (whose vectors are FP32; an FP64 division is a long dependent chain of FP64 operations,
// which run at a small fraction of the FP32 rate on this GPU)
template <class T>
__device__ __forceinline__ double ratio(double a, double b) {
    if constexpr (sizeof(T) == 4)
        return (double)__fdiv_rn((float)a, (float)b);
    else
        return a / b;
}

// p_i = z + sum_j beta_ij p_j, beta_ij = -(z, p_j)_A / (p_j, p_j)_A  (Alg. 1, step 2).
// The coefficients are computed once per CTA (FP64 division is scarce on this GPU) and
// broadcast through shared memory.
template <class LV, class G>
__device__ void op_orth(const LV &L, const Op &op, int tid, int nth, const G &g) {
    using T = typename LV::val_t;
    __shared__ double beta_s[kMaxKcycle];
    const int i = op.step;
    if (threadIdx.x < kMaxKcycle) {
        const int j = threadIdx.x;
        double pq = L.sc[SC_PQ0 + j];
        beta_s[j] = (j < i && pq > 0.0) ? -ratio<T>(L.sc[SC_ZQ0 + j], pq) : 0.0;
    }
    g.sync();
    T beta[kMaxKcycle];
#pragma unroll
    for (int j = 0; j < kMaxKcycle; j++) beta[j] = (T)beta_s[j];
    T *p = pick(L.p, i);
    for (int r = tid; r < L.n; r += nth) {
        T acc = p[r];
#pragma unroll
        for (int j = 0; j < kMaxKcycle; j++)
            if (j < i) acc += beta[j] * L.p[j][r];
        p[r] = acc;
    }
}

// q_i = A p_i; (p_i, q_i); (r_i, p_i) with r_0 = rhs
template <class LV, int RM, class G>
__device__ void op_spmv_dot(const LV &L, const Op &op, const RedCtx &rc, int tid, int nth,
                            const G &g) {
    using T = typename LV::val_t;
    const int i = op.step;
    const T *p = pick(L.p, i);
    T *q = pick(L.q, i);
    const T *r = i == 0 ? L.rhs : L.r;
    T v[2] = {0, 0};
    for (int row = tid; row < L.n; row += nth) {
        int base, width;
        row_span(L, row, base, width);
        const T acc = row_dot(L, base, 0, width, p);
        q[row] = acc;
        T pr = p[row];
        v[0] += pr * acc;
        v[1] += r[row] * pr;
    }
    double *out[2] = {&L.sc[SC_PQ0 + i], &L.sc[SC_RP0 + i]};
    reduce_store<2, RM, T>(v, out, rc, op.red_pb, g);
}

// alpha_i = (r_i, p_i) / (p_i, p_i)_A; u_{i+1} = u_i + alpha_i p_i; r_{i+1} = r_i - alpha_i q_i.
// Alg. 1 stops (alpha = 0 from then on) once (p_i, p_i)_A <= 0 or a residual is exactly zero.
template <class LV, int RM, class G>
__device__ void op_update(const LV &L, const Op &op, const RedCtx &rc, int tid, int nth,
                          const G &g) {
    using T = typename LV::val_t;
    __shared__ double coef[2];  // alpha, stopped: computed once per CTA
    const int i = op.step, last = op.last;
    if (threadIdx.x == 0) {
        const double pq = L.sc[SC_PQ0 + i];
        const bool prev_stop =
            i > 0 && (L.sc[SC_STOP0 + i - 1] != 0.0 || L.sc[SC_RR0 + i - 1] == 0.0);
        const bool stopped = prev_stop || !(pq > 0.0) || !isfinite(pq);
        coef[0] = stopped ? 0.0 : ratio<T>(L.sc[SC_RP0 + i], pq);
        coef[1] = stopped ? 1.0 : 0.0;
    }
    g.sync();
    const T a = (T)coef[0];
    const bool stopped = coef[1] != 0.0;
    const T *p = pick(L.p, i);
    const T *q = pick(L.q, i);
    const T *r_in = i == 0 ? L.rhs : L.r;
    T *e = L.e;
    T v[1] = {0};
    T *pn = (op.fuse && !last) ? pick(L.p, i + 1) : nullptr;  // next step's first colour
    for (int row = tid; row < L.n; row += nth) {
        e[row] = (i == 0) ? a * p[row] : e[row] + a * p[row];
        if (!last) {
            T rn = r_in[row] - a * q[row];
            L.r[row] = rn;
            v[0] += rn * rn;
            if (pn) pn[row] = (row >= op.f0 && row < op.f1) ? rn * L.dinv[row] : T(0);
        }
    }
    if (!last) {
        double *out[1] = {&L.sc[SC_RR0 + i]};
        reduce_store<1, RM, T>(v, out, rc, op.red_pb, g);
    }
    if ((RM == RM_BLOCK || (RM == RM_TEAM ? rc.rank == 0 : blockIdx.x == 0)) && threadIdx.x == 0)
        L.sc[SC_STOP0 + i] = stopped ? 1.0 : 0.0;
}

// run one op (everything except OP_TAIL / OP_NOP) on level view L by threads tid < nth of
// group g; next() gives the view of the next coarser level (only its rhs and e are used)
template <class LV, int RM, class G, class Next>
__device__ __forceinline__ void run_op_on(const LV &L, const Next &next, const Op &op,
                                          const RedCtx &rc, int tid, int nth, const G &g,
                                          const BigScratch &sc = BigScratch{}) {
    switch (op.kind) {
        case OP_ZERO: op_zero(L, vec_of(L, op.usel), tid, nth); break;
        case OP_GS:
            op_gs<LV, true>(L, op, vec_of(L, op.fsel), vec_of(L, op.usel), tid, nth, -1, -1, sc);
            break;
        case OP_GS_FIRST: op_gs_first(L, op, vec_of(L, op.fsel), vec_of(L, op.usel), tid, nth); break;
        case OP_RESTRICT: {
            const auto &N = next();
            op_restrict(L, vec_of(L, op.fsel), vec_of(L, op.usel), N.rhs, tid, nth,
                        op.fuse ? N.p[0] : nullptr, N.dinv, op.f0, op.f1, op.bb1 > op.bb0);
            break;
        }
        case OP_RESID:
            op_resid(L, vec_of(L, op.fsel), vec_of(L, op.usel), pick(L.q, op.step), tid, nth);
            break;
        case OP_GATHER: {
            const auto &N = next();
            op_gather_children(L, pick(L.q, op.step), N.rhs, tid, nth, op.fuse ? N.p[0] : nullptr,
                               N.dinv, op.f0, op.f1);
            break;
        }
        case OP_PROLONG: op_prolong(L, next().e, vec_of(L, op.usel), tid, nth); break;
        case OP_COARSE: op_coarse(L, tid, nth); break;
        case OP_MULTIDOT: op_multidot<LV, RM>(L, op, rc, tid, nth, g); break;
        case OP_ORTH: op_orth(L, op, tid, nth, g); break;
        case OP_SPMV_DOT: op_spmv_dot<LV, RM>(L, op, rc, tid, nth, g); break;
        case OP_UPDATE: op_update<LV, RM>(L, op, rc, tid, nth, g); break;
        default: break;
    }
}

// run one op on level op.level of a table of views, every thread of the CTA taking part
template <class LV, int RM>
__device__ __forceinline__ void run_op(const LV *tab, const Op &op, const RedCtx &rc, int tid,
                                       int nth, const BigScratch &sc = BigScratch{}) {
    run_op_on<LV, RM>(tab[op.level], [&]() -> const LV & { return tab[op.level + 1]; }, op, rc,
                      tid, nth, BlockGroup{}, sc);
}

}  // namespace amg
