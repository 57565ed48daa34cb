// Solve phase on the GPU: the nonlinear AMLI-cycle (paper Alg. 2) with nonlinear PCG on the
// coarse levels (Alg. 1), the quadtree-coloured Gauss-Seidel smoother (Sec. 4.5), implicit
// prolongation / restriction (Sec. 4.3), and the outer Krylov iteration (Alg. 1 on the
// finest level, flexible CG with full A-orthogonalisation).
//
// Execution. One application of the preconditioner B^_fine is a fixed program of ops (see
// cycle_ops.cuh) over device-resident data; every scalar stays on the device. It runs as ONE
// persistent cooperative kernel (one CTA per SM): the CTAs execute each op row-parallel and
// meet at a bounded grid barrier before the next. The coarse levels from the "tail" level
// down (a few thousand rows or less: pure latency) are staged in shared memory by CTA 0 at
// kernel start, and CTA 0 alone runs their whole recursive Alg. 1 / Alg. 2 there with
// __syncthreads() between ops while the other CTAs wait at the barrier. The outer Krylov
// update is four small kernels per iteration; the host reads one residual per iteration.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "cycle_ops.cuh"

namespace amg {

template <class T>
using GLev = LevelDev<T, int>;                 // level in HBM
template <class T>
using SLev = LevelDev<T, unsigned short>;      // level staged in shared memory

// persistent kernel CTA size (one CTA per SM): the FP64 cycle runs with fewer threads and
// twice the registers each, as its ops at the 64-register cap of 1024 threads spill
constexpr int kPThreads = 1024;
constexpr int kPThreads64 = 512;
template <class T>
constexpr int cycle_threads() { return sizeof(T) == 8 ? kPThreads64 : kPThreads; }
constexpr int kTailRowsMax = 4096;  // levels larger than this are never staged
// coarse levels of at least this many rows restrict in two grid-wide passes (OP_RESID,
// OP_GATHER): their rows' children lie in different colours, far apart in HBM, and the
// one-pass form's four-lane gathers read scattered slots
constexpr int kSplitRestrictRows = 524288;


// shared-memory image of the tail levels (byte offsets into the dynamic shared memory)
struct TailLevelLayout {
    int n, nslices, padded;
    int gmem;    // 1: the level stays in HBM/L2 (top tail level only); its scalars are staged
    int w;       // staged: slice width of the image (every slice padded to it)
    int colors, ncolors;  // staged int[ncolors + 1]: pi-row range of each colour
    int col, val, dinv, parent, children, children2, Ainv, rhs, e, r;
    int p[kMaxKcycle], q[kMaxKcycle];
};
struct TailLayout {
    int tl;      // first tail level (nlev = none)
    int nlev;
    int narrow;  // threads (whole warps) that run the ops of the staged levels
    int kc;      // Alg. 1 steps (kcycle_n)
    int nu_pre, nu_post;  // smoothing sweeps
    int W;       // slice width of every staged level when fixed (9), else 0
    int bytes;
    int sc;      // the tail levels' Alg. 1 scalars, SC_N doubles per level
    TailLevelLayout lv[kMaxLevels];
};

constexpr int kTprofCount = 16 * kMaxLevels;  // tail profile slots: 16 op kinds per level

template <class T>
struct CycleArgs {
    const GLev<T> *tab;
    const Op *prog;
    int nops;
    const int *tail_colors;      // colour ranges of the tail levels, copied to shared memory
    int tail_color_words;
    TailLayout lay;
    double *partials;            // [2][4][gridDim]
    unsigned long long *bar;     // barrier counter (zeroed before every launch)
    int *err;
    unsigned long long *ts;      // per-op end timestamps (profiling) or null
    unsigned long long *tprof;   // tail: [16 level + kind] cycles, [kTprofCount + 16 level +
                                 // kind] count (profiling) or null
    // host-set barrier fault (amg_debug_barrier_fault): wait limit of every grid barrier, and
    // arrivals the first barrier waits for beyond the grid's (0: none)
    unsigned long long bar_limit_ns;
    int bar_extra;
    // the finest level's input and output vectors when not the table's (FGMRES basis vectors)
    T *rhs0, *e0;
    // CTAs 1.. lend their dynamic shared memory to the big blocks' sweeps; the warp-sized
    // ones go to warps [0, big_wwarps) with big_wslice bytes each (0: to every warp, from
    // global memory)
    int big_smem, big_wwarps;
    unsigned big_wslice;
};

// ---------------------------------------------------------------------------------------
// standalone executor (diagnostic path: amg_apply_cycle on coarse levels, amg_smooth)
template <class T>
__global__ void __launch_bounds__(kRedThreads) k_op(const GLev<T> *__restrict__ tab, Op op,
                                                    RedCtx rc) {
    run_op<GLev<T>, RM_LASTBLOCK>(tab, op, rc, blockIdx.x * blockDim.x + threadIdx.x,
                                  gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------------------
// persistent cycle kernel: the shared-memory tail
//
// CTA 0 runs B~ of the tail levels (Alg. 1 with Alg. 2 inside, down to the exact coarsest
// solve) as structured code: one device function per level depth, every op a direct call,
// no op decoding. Staged levels are addressed from the dynamic shared-memory base through
// the byte offsets of the layout (kept in shared memory), so every access is a shared-memory
// load, and their slices have one width W (compile-time 9 for the 3x3-cell stencils of
// span-1 levels). Their ops run on the first `narrow` threads (whole warps) with hardware
// barrier 1: the other warps would only add issue slots and barrier arrivals to ops of a
// few hundred rows. The ops of an HBM-resident top level (thousands of rows, each a chain
// of L2 round trips) run on the whole CTA with CTA-wide barriers.
extern __shared__ __align__(16) unsigned char amg_smem[];

struct TailCtl {
    int tl, nlev, narrow, kc, sc_off;
    int nu_pre, nu_post;
    int top_w;  // slice width of the HBM-resident top level when uniform, else 0
    int *err;
    unsigned long long *tprof;
    long long t0;
};
__shared__ TailCtl tail_ctl;
__shared__ TailLevelLayout tail_lay[kMaxLevels];
__shared__ __align__(16) unsigned char tail_gview[sizeof(SLev<double>)];  // SLev<T> of the top
// The same top level as a StagedLevel<T, W> whose arrays are in HBM (uniform slice width):
// its phases then run the code the staged levels run, so the tail executes one copy of the
// phase code instead of two (the tail's time goes largely to instruction fetch)
__shared__ __align__(16) unsigned char tail_sview[sizeof(StagedLevel<double, 0>)];

template <class T, int W>
__device__ __forceinline__ StagedLevel<T, W> staged_level(int l) {
    const TailLevelLayout &y = tail_lay[l];
    const int nlev = tail_ctl.nlev;
    auto at = [](int off) { return amg_smem + (off > 0 ? off : 0); };  // -1: absent, never read
    StagedLevel<T, W> V;
    V.n = y.n;
    V.w = y.w;
    V.col = (const unsigned short *)at(y.col);
    V.val = (const T *)at(y.val);
    V.dinv = (const T *)at(y.dinv);
    V.bptr = nullptr;
    V.parent = (const int *)at(y.parent);
    V.children = (const int4 *)at(l + 1 < nlev ? tail_lay[l + 1].children : -1);
    V.children2 = (l + 1 < nlev && tail_lay[l + 1].children2 >= 0)
                      ? (const int4 *)(amg_smem + tail_lay[l + 1].children2) : nullptr;
    V.Ainv = (const double *)at(y.Ainv);  // FP64 cycle: n*n doubles
    V.Ainv2 = (const float *)at(y.Ainv);  // FP32 cycle: 2*n*n floats, the same bytes
    V.rhs = (T *)at(y.rhs);
    V.e = (T *)at(y.e);
    V.r = (T *)at(y.r);
#pragma unroll
    for (int k = 0; k < kMaxKcycle; k++) {
        V.p[k] = (T *)at(y.p[k]);
        V.q[k] = (T *)at(y.q[k]);
    }
    V.sc = (double *)(amg_smem + tail_ctl.sc_off) + (size_t)(l - tail_ctl.tl) * SC_N;
    V.nnext = l + 1 < nlev ? tail_lay[l + 1].n : 0;
    return V;
}

// tail profiling: SM cycles of the op just finished, by level and kind (thread 0)
__device__ __forceinline__ void tail_mark(int l, int kind) {
    if (tail_ctl.tprof && threadIdx.x == 0) {
        const long long t1 = clock64();
        const int slot = 16 * l + kind;
        atomicAdd(&tail_ctl.tprof[slot], (unsigned long long)(t1 - tail_ctl.t0));
        atomicAdd(&tail_ctl.tprof[kTprofCount + slot], 1ull);
        tail_ctl.t0 = t1;
    }
}

__device__ __forceinline__ Op tail_op() {
    Op o;
    memset(&o, 0, sizeof o);
    o.red_pb = -1;
    o.fin_pb = -1;
    return o;
}

// The recursion of B~ (Alg. 1) and B^ (Alg. 2) over the tail levels is walked as a state
// machine with three phases per level: ENTER (B~_l starts: the exact solve on the coarsest
// level, else step 0), PRE (B^_l for step i up to the restriction, then B~_{l+1}) and POST
// (the prolongation, post-smoothing and the Alg. 1 updates of step i). Every thread of the
// CTA walks it with the same state, so all know which phases are the top level's.
enum : int { PH_ENTER = 0, PH_PRE, PH_POST };

// pre-smoothing from zero (colours ascending; the first non-empty colour is u = D^-1 f) and
// next.rhs = P^t (f - A u1), for z = p_i = B^_l [f], f = rhs (i = 0) or r
// first non-empty colour [r0, r1) of tail level l (its point-GS first colour)
__device__ __forceinline__ void tail_first_colour(int l, int &r0, int &r1) {
    const int *cr = (const int *)(amg_smem + tail_lay[l].colors);
    const int nc = tail_lay[l].ncolors;
    int c = 0;
    while (c < nc && cr[c + 1] == cr[c]) c++;
    r0 = c < nc ? cr[c] : 0;
    r1 = c < nc ? cr[c + 1] : 0;
}

// The first colour of a pre-smoothing was already done by the op before it, except for step
// 0 of the top tail level: by the last UPDATE (i > 0) or by the restriction into this level
// (i = 0), which also starts the next level's first colour unless that level is the coarsest.
template <class T, int W, class LV, class G>
__device__ __forceinline__ void phase_pre(const LV &L, const G &g, int nth, int l, int i) {
    const int tid = threadIdx.x;
    const T *f = i == 0 ? L.rhs : L.r;
    T *z = pick(L.p, i);
    const int *cr = (const int *)(amg_smem + tail_lay[l].colors);
    const int nc = tail_lay[l].ncolors;
    int c = 0;
    while (c < nc && cr[c + 1] == cr[c]) c++;
    Op op = tail_op();
    if (i == 0 && l == tail_ctl.tl) {
        op.i0 = c < nc ? cr[c] : 0;
        op.i1 = c < nc ? cr[c + 1] : 0;
        op_gs_first(L, op, f, z, tid, nth);
        g.sync();
        tail_mark(l, OP_GS_FIRST);
    }
    // the first sweep's remaining colours, then nu_pre - 1 further forward sweeps
    for (int sw = 0, c1 = c + 1; sw < tail_ctl.nu_pre; sw++, c1 = 0)
        for (c = c1; c < nc; c++) {
            if (cr[c + 1] == cr[c]) continue;
            op.i0 = cr[c];
            op.i1 = cr[c + 1];
            op_gs(L, op, f, z, tid, nth);
            g.sync();
            tail_mark(l, OP_GS);
        }
    // next.rhs = P^t (f - A u1) in two passes: the residual row by row into q_i (free until
    // step i's SpMV writes it), then the children sums
    T *t = pick(L.q, i);
    op_resid(L, f, z, t, tid, nth);
    g.sync();
    tail_mark(l, OP_RESID);
    const StagedLevel<T, W> N = staged_level<T, W>(l + 1);
    if (tail_lay[l + 1].Ainv < 0) {  // the next level smooths: its first colour too
        int f0, f1;
        tail_first_colour(l + 1, f0, f1);
        op_gather_children(L, t, N.rhs, tid, nth, N.p[0], N.dinv, f0, f1);
    } else {
        op_gather_children(L, t, N.rhs, tid, nth);
    }
    g.sync();
    tail_mark(l, OP_RESTRICT);
}

// u2 = u1 + P next.e, post-smoothing (colours descending), then Alg. 1 step i on level l
template <class T, int W, class LV, class G>
__device__ __forceinline__ void phase_post(const LV &L, const G &g, int nth, int l, int i) {
    const int tid = threadIdx.x;
    const T *f = i == 0 ? L.rhs : L.r;
    T *z = pick(L.p, i);
    op_prolong(L, staged_level<T, W>(l + 1).e, z, tid, nth);
    g.sync();
    tail_mark(l, OP_PROLONG);
    const int *cr = (const int *)(amg_smem + tail_lay[l].colors);
    Op op = tail_op();
    op.backward = 1;
    for (int sw = 0; sw < tail_ctl.nu_post; sw++)
        for (int c = tail_lay[l].ncolors - 1; c >= 0; c--) {
            if (cr[c + 1] == cr[c]) continue;
            op.i0 = cr[c];
            op.i1 = cr[c + 1];
            op_gs(L, op, f, z, tid, nth);
            g.sync();
            tail_mark(l, OP_GS);
        }
    const RedCtx rc{nullptr, nullptr};
    const int kc = tail_ctl.kc;
    op = tail_op();
    op.step = i;
    op.last = (i == kc - 1);
    if (!op.last) {  // the UPDATE also starts step i+1's pre-smoothing
        op.fuse = 1;
        tail_first_colour(l, op.f0, op.f1);
    }
    if (i > 0) {
        op_multidot<LV, RM_BLOCK>(L, op, rc, tid, nth, g);
        g.sync();
        tail_mark(l, OP_MULTIDOT);
        op_orth(L, op, tid, nth, g);
        g.sync();
        tail_mark(l, OP_ORTH);
    }
    op_spmv_dot<LV, RM_BLOCK>(L, op, rc, tid, nth, g);
    g.sync();
    tail_mark(l, OP_SPMV_DOT);
    op_update<LV, RM_BLOCK>(L, op, rc, tid, nth, g);
    g.sync();
    tail_mark(l, OP_UPDATE);
}

// ENTER on the coarsest level: e = A^{-1} rhs
template <class LV, class G>
__device__ __forceinline__ void phase_coarse(const LV &L, const G &g, int nth, int l) {
    op_coarse(L, threadIdx.x, nth);
    g.sync();
    tail_mark(l, OP_COARSE);
}

// e_tl = B~_tl [rhs_tl] over the whole tail (every thread of CTA 0 calls it)
template <class T, int W>
__device__ void tail_btilde(bool inplace) {
    const int tl = tail_ctl.tl, nlev = tail_ctl.nlev, kc = tail_ctl.kc, narrow = tail_ctl.narrow;
    const int tid = threadIdx.x;
    const SLev<T> &top_gv = *reinterpret_cast<const SLev<T> *>(tail_gview);
    const StagedLevel<T, W> &topv = *reinterpret_cast<const StagedLevel<T, W> *>(tail_sview);
    const bool top_staged_code = tail_ctl.top_w > 0 && (W == 0 || tail_ctl.top_w == W);
    int step[kMaxLevels] = {};
    int l = tl, ph = PH_ENTER;
    bool prev_top = true;  // the caller's barrier
    for (;;) {
        const bool coarsest = tail_lay[l].Ainv >= 0;
        const int i = step[l];
        if (inplace && l == tl) {  // the HBM-resident top level: the whole CTA
            if (!prev_top) __syncthreads();  // the narrow warps' phases are complete
            prev_top = true;
            const int nth = blockDim.x;
            if (top_staged_code) {  // every thread: barrier 1 over the whole CTA
                const WarpGroup all{nth};
                if (ph == PH_PRE) phase_pre<T, W>(topv, all, nth, l, i);
                else if (ph == PH_POST) phase_post<T, W>(topv, all, nth, l, i);
            } else {
                if (ph == PH_PRE) phase_pre<T, W>(top_gv, BlockGroup{}, nth, l, i);
                else if (ph == PH_POST) phase_post<T, W>(top_gv, BlockGroup{}, nth, l, i);
            }
        } else {
            prev_top = false;
            if (tid < narrow) {
                const WarpGroup ng{narrow};
                const StagedLevel<T, W> L = staged_level<T, W>(l);
                if (ph == PH_ENTER && coarsest) phase_coarse(L, ng, narrow, l);
                else if (ph == PH_PRE) phase_pre<T, W>(L, ng, narrow, l, i);
                else if (ph == PH_POST) phase_post<T, W>(L, ng, narrow, l, i);
            }
        }
        // next state (the same in every thread)
        if (ph == PH_ENTER && !coarsest) {
            step[l] = 0;
            ph = PH_PRE;
            continue;
        }
        if (ph == PH_PRE) {  // descend: B~_{l+1}
            if (l + 1 >= nlev || l + 1 - tl >= kMaxLevels) break;  // never: the coarsest ends it
            l++;
            ph = PH_ENTER;
            continue;
        }
        if (ph == PH_POST && i + 1 < kc) {
            step[l] = i + 1;
            ph = PH_PRE;
            continue;
        }
        // B~_l done (coarsest solved, or its last step): back to level l-1's POST
        if (l == tl) break;
        l--;
        ph = PH_POST;
    }
    if (inplace && !prev_top) __syncthreads();
}

// CTA 0, kernel start: copy the staged levels into shared memory (slices padded to width w)
template <class T>
__device__ void stage_tail(const CycleArgs<T> &a) {
    const TailLayout &Y = a.lay;
    const int tid = threadIdx.x, nth = blockDim.x;
    {
        const int words = Y.nlev * (int)(sizeof(TailLevelLayout) / sizeof(int));
        for (int i = tid; i < words; i += nth) ((int *)tail_lay)[i] = ((const int *)Y.lv)[i];
    }
    if (tid == 0) {
        tail_ctl.tl = Y.tl;
        tail_ctl.nlev = Y.nlev;
        tail_ctl.narrow = Y.narrow;
        tail_ctl.kc = Y.kc;
        tail_ctl.nu_pre = Y.nu_pre;
        tail_ctl.nu_post = Y.nu_post;
        tail_ctl.sc_off = Y.sc;
        tail_ctl.top_w = 0;
        tail_ctl.err = a.err;
        tail_ctl.tprof = a.tprof;
    }
    for (int l = Y.tl; l < Y.nlev; l++) {
        const TailLevelLayout &y = Y.lv[l];
        const GLev<T> &G = a.tab[l];
        if (y.gmem) {  // read in place from HBM / L2
            if (tid == 0) {
                SLev<T> &S = *reinterpret_cast<SLev<T> *>(tail_gview);
                S.n = G.n;
                S.fine = 0;
                S.bg = 0;
                S.w = G.w;
                S.sl = G.sl;
                S.col = G.col16;
                S.val = G.val;
                S.dinv = G.dinv;
                S.col16 = nullptr;
                S.bptr = nullptr;
                S.parent = G.parent;
                S.children = (l + 1 < Y.nlev && Y.lv[l + 1].children >= 0)
                                 ? (const int4 *)(amg_smem + Y.lv[l + 1].children) : nullptr;
                S.children2 = (l + 1 < Y.nlev && Y.lv[l + 1].children2 >= 0)
                                  ? (const int4 *)(amg_smem + Y.lv[l + 1].children2) : nullptr;
                S.Ainv = G.Ainv;
                S.Ainv2 = G.Ainv2;
                S.rhs = G.rhs;
                S.e = G.e;
                S.r = G.r;
                for (int k = 0; k < kMaxKcycle; k++) {
                    S.p[k] = G.p[k];
                    S.q[k] = G.q[k];
                }
                S.sc = (double *)(amg_smem + Y.sc) + (size_t)(l - Y.tl) * SC_N;
                S.nnext = G.nnext;
                StagedLevel<T, 0> &V = *reinterpret_cast<StagedLevel<T, 0> *>(tail_sview);
                V.n = G.n;
                V.w = G.w;
                V.col = G.col16;
                V.val = G.val;
                V.dinv = G.dinv;
                V.bptr = nullptr;
                V.parent = G.parent;
                V.children = S.children;
                V.children2 = S.children2;
                V.Ainv = nullptr;
                V.Ainv2 = nullptr;
                V.rhs = G.rhs;
                V.e = G.e;
                V.r = G.r;
                for (int k = 0; k < kMaxKcycle; k++) {
                    V.p[k] = G.p[k];
                    V.q[k] = G.q[k];
                }
                V.sc = S.sc;
                V.nnext = G.nnext;
                tail_ctl.top_w = G.w;  // 0 unless every slice has one width
            }
            continue;
        }
        // slot (s, k, lane) of the image <- slot k of slice s in HBM, or padding
        unsigned short *col = (unsigned short *)(amg_smem + y.col);
        T *val = (T *)(amg_smem + y.val);
        const int img = y.nslices * 32 * y.w;
        for (int i = tid; i < img; i += nth) {
            const int sidx = i / (32 * y.w), rem = i - sidx * 32 * y.w;
            const int k = rem >> 5, lane = rem & 31;
            const int s0 = G.sl[sidx], width = (G.sl[sidx + 1] - s0) >> 5;
            int c = -1;
            T v = 0;
            if (k < width) {
                c = G.col[s0 + 32 * k + lane];
                v = G.val[s0 + 32 * k + lane];
            }
            col[i] = c >= 0 ? (unsigned short)c : (unsigned short)0xFFFF;
            val[i] = c >= 0 ? v : T(0);
        }
        if (y.dinv >= 0)
            for (int i = tid; i < y.n; i += nth) ((T *)(amg_smem + y.dinv))[i] = G.dinv[i];
        if (y.parent >= 0)
            for (int i = tid; i < y.n; i += nth) ((int *)(amg_smem + y.parent))[i] = G.parent[i];
        if (y.children >= 0)  // children of this level's rows (in level l-1)
            for (int i = tid; i < y.n; i += nth)
                ((int4 *)(amg_smem + y.children))[i] = a.tab[l - 1].children[i];
        if (y.children2 >= 0)  // octree: children 4..7
            for (int i = tid; i < y.n; i += nth)
                ((int4 *)(amg_smem + y.children2))[i] = a.tab[l - 1].children2[i];
        if (y.Ainv >= 0) {  // n*n doubles or 2*n*n floats
            if (sizeof(T) == 8)
                for (int i = tid; i < y.n * y.n; i += nth)
                    ((double *)(amg_smem + y.Ainv))[i] = G.Ainv[i];
            else
                for (int i = tid; i < 2 * y.n * y.n; i += nth)
                    ((float *)(amg_smem + y.Ainv))[i] = G.Ainv2[i];
        }
    }
    // colour ranges: every level's int[ncolors + 1] at its offset, in one block of words
    if (a.tail_color_words > 0) {
        int *dst = (int *)(amg_smem + Y.lv[Y.tl].colors);
        for (int i = tid; i < a.tail_color_words; i += nth) dst[i] = a.tail_colors[i];
    }
}

template <class T, int W>
__device__ void run_tail(const CycleArgs<T> &a) {
    const int tl = a.lay.tl, n = tail_lay[tl].n;
    const int tid = threadIdx.x, nth = blockDim.x;
    const bool inplace = tail_lay[tl].gmem != 0;
    if (!inplace) {
        const T *grhs = a.tab[tl].rhs;
        T *srhs = (T *)(amg_smem + tail_lay[tl].rhs);
        for (int i = tid; i < n; i += nth) srhs[i] = grhs[i];
    }
    if (tid == 0) tail_ctl.t0 = clock64();
    __syncthreads();
    tail_btilde<T, W>(inplace);
    if (inplace) return;
    __syncthreads();
    T *ge = a.tab[tl].e;
    const T *se = (const T *)(amg_smem + tail_lay[tl].e);
    for (int i = tid; i < n; i += nth) ge[i] = se[i];
}

// sum the per-CTA partials of the previous op (every CTA, identical order) into sc; one
// warp does it, in FP64 for the FP64 cycle and in FP32 for the FP32 cycle (whose per-CTA
// partials are FP32 sums)
template <class T, class TAB>
__device__ __forceinline__ void finalize(const CycleArgs<T> &a, const TAB *tab, const Op &op) {
    if (threadIdx.x < 32) {
        const int G = gridDim.x;
        double *sc = tab[op.fin_level].sc;
        for (int k = 0; k < op.fin_n; k++) {
            const double *part = a.partials + ((size_t)op.fin_pb * 4 + k) * G;
            double y;
            if constexpr (sizeof(T) == 4) {
                float x = 0.f;
                for (int b = threadIdx.x; b < G; b += 32) x += (float)__ldcg(&part[b]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                y = (double)x;
            } else {
                y = 0.0;
                for (int b = threadIdx.x; b < G; b += 32) y += __ldcg(&part[b]);
                y = warp_sum(y);
            }
            if (threadIdx.x == 0 && op.fin_dst[k] >= 0) sc[op.fin_dst[k]] = y;
        }
    }
    __syncthreads();
}

// B = 1: finest-level blocks of several rows take the lane-parallel block smoother
template <class T, int W, int B>
__global__ void __launch_bounds__(cycle_threads<T>(), 1) k_cycle(CycleArgs<T> a) {
    using GL = LevelDev<T, int, B>;  // the same layout as GLev<T>
    __shared__ GL gtab[kMaxLevels];
    __shared__ unsigned long long target;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        target = (unsigned long long)a.bar_extra;  // > 0 only under a host-set barrier fault
        abort_flag = 0;
    }
    {  // the level table, read by every op, lives in shared memory
        const int words = a.lay.nlev * (int)(sizeof(GL) / sizeof(int));
        for (int i = threadIdx.x; i < words; i += blockDim.x)
            ((int *)gtab)[i] = ((const int *)a.tab)[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.rhs0) gtab[0].rhs = a.rhs0;
        if (a.e0) gtab[0].e = a.e0;
    }
    if (blockIdx.x == 0 && a.lay.tl < a.lay.nlev) stage_tail(a);
    __syncthreads();
    // the op descriptors pass through shared memory: a few threads fetch the next one while
    // the CTA waits at the barrier, and every thread reads its fields from there (a per-thread
    // copy would cost every thread a 72-byte global load and a local-memory round trip)
    __shared__ Op sop[2];
    constexpr int kOpWords = (int)(sizeof(Op) / sizeof(int));
    if (threadIdx.x < kOpWords) ((int *)&sop[0])[threadIdx.x] = ((const int *)a.prog)[threadIdx.x];
    __syncthreads();
    // rows go to warps in 32-row chunks with the CTA index fastest, so an op over a few
    // thousand rows (the coarse grid-wide levels) spreads over every SM instead of filling the
    // first few CTAs; a warp's rows stay consecutive (coalesced slots, lane = row mod 32)
    const int gtid = (((int)threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x) * 32 +
                     ((int)threadIdx.x & 31);
    const int gnth = gridDim.x * blockDim.x;
    const RedCtx rc{a.partials, nullptr};
    BigScratch sc;
    if (a.big_smem && gridDim.x > 1) {
        unsigned dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        sc.p = blockIdx.x ? amg_smem : nullptr;  // CTA 0's holds the tail
        sc.bytes = dyn;
        sc.skip0 = true;
        sc.wwarps = a.big_wwarps;
        sc.wslice = a.big_wslice;
    }
    for (int k = 0; k < a.nops; k++) {
        const Op &op = sop[k & 1];
        // the next descriptor into the other buffer (last read by op k-1), issued before op k
        // runs: a load still in flight at the barrier would delay its release fence
        if (threadIdx.x < kOpWords && k + 1 < a.nops)
            ((int *)&sop[(k + 1) & 1])[threadIdx.x] = ((const int *)(a.prog + k + 1))[threadIdx.x];
        if (op.fin_pb >= 0) finalize(a, gtab, op);
        if (op.kind == OP_TAIL) {
            if (blockIdx.x == 0) run_tail<T, W>(a);
        } else if (op.kind != OP_NOP) {
            run_op<GL, RM_PARTIAL>(gtab, op, rc, gtid, gnth, sc);
        }
        if (!grid_barrier(a.bar, a.err, target, abort_flag, a.bar_limit_ns)) break;
        if (a.ts && blockIdx.x == 0 && threadIdx.x == 0) a.ts[k] = global_ns();
    }
}

__global__ void k_timestamp(unsigned long long *t) { *t = global_ns(); }

// ---------------------------------------------------------------------------------------
// outer Krylov kernels (FP64, pi order)
__global__ void k_gather(int n, const int *__restrict__ idx, const double *__restrict__ src,
                         double *__restrict__ dst) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) dst[p] = src[idx[p]];
}

__global__ void k_scatter(int n, const int *__restrict__ idx, const double *__restrict__ src,
                          double *__restrict__ dst) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) dst[idx[p]] = src[p];
}

// 16-bit copy of column indices (padding -1 -> 0xFFFF)
__global__ void k_col16(int n, const int *__restrict__ col, unsigned short *__restrict__ c16) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c16[i] = col[i] >= 0 ? (unsigned short)col[i] : (unsigned short)0xFFFF;
}

// 1 / a_ii of every row (slot 0 of the sliced ELL holds the diagonal)
template <class T>
__global__ void k_inv_diag(int n, const int *__restrict__ sl, const double *__restrict__ val,
                           T *__restrict__ dinv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dinv[i] = (T)(1.0 / val[sl[i >> 5] + (i & 31)]);
}

template <class A, class B>
__global__ void k_convert(int n, const A *__restrict__ src, B *__restrict__ dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (B)src[i];
}

// (v, v) -> out
__global__ void __launch_bounds__(kRedThreads) k_norm2(int n, const double *__restrict__ v,
                                                       double *out, RedCtx rc) {
    double a[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        a[0] += v[i] * v[i];
    double *o[1] = {out};
    reduce_store<1, RM_LASTBLOCK, double>(a, o, rc, 0, BlockGroup{});
}

// t = b - A x, (t, t) -> out
__global__ void __launch_bounds__(kRedThreads) k_true_residual(GLev<double> L,
                                                               const double *__restrict__ b,
                                                               const double *__restrict__ x,
                                                               double *__restrict__ t,
                                                               double *out, RedCtx rc) {
    double a[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) {
        double ri = row_residual(L, i, b, x);
        t[i] = ri;
        a[0] += ri * ri;
    }
    double *o[1] = {out};
    reduce_store<1, RM_LASTBLOCK, double>(a, o, rc, 0, BlockGroup{});
}

// outer scalars: osc[OS_BB] = (b,b), osc[OS_RR] = (r,r), osc[OS_STOP] = breakdown flag,
// osc[OS_RP] = (r, p_i), osc[OS_TT] = (t, t), osc[OS_ZQ + j] = (z, A p_j); (p_j, A p_j) in opq
enum : int { OS_BB = 0, OS_RR = 1, OS_STOP = 2, OS_RP = 4, OS_TT = 5, OS_ZQ = 8 };

// Dots of w with the basis vectors V[0..m), kDotChunk vectors per sweep over the rows: each
// thread keeps one grid-stride partial sum per vector (in row order), each block reduces them
// vector by vector, and the last block to finish sums the block partials in block order.
constexpr int kDotChunk = 8;

__device__ __forceinline__ void mdot_chunk(int n, const double *__restrict__ w,
                                           double *const *__restrict__ V, int c0, int mc,
                                           double *partials) {
    const double *vp[kDotChunk];
#pragma unroll
    for (int i = 0; i < kDotChunk; i++) vp[i] = i < mc ? V[c0 + i] : nullptr;
    double a[kDotChunk] = {}, r[kDotChunk];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double wk = w[k];
#pragma unroll
        for (int i = 0; i < kDotChunk; i++)
            if (i < mc) a[i] += wk * vp[i][k];
    }
    block_sum<kDotChunk, double>(a, r, BlockGroup{});
    if (threadIdx.x == 0)
        for (int i = 0; i < mc; i++) partials[(size_t)(c0 + i) * gridDim.x + blockIdx.x] = r[i];
    __syncthreads();  // the reduction scratch is reused by the next chunk
}

__device__ __forceinline__ void mdot_finish(int m, double *out, const RedCtx &rc) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(rc.counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // vector i by warp i mod (warps): each sum in the same order as one warp summing them all
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = wid; i < m; i += nw) {
        double y = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32)
            y += __ldcg(&rc.partials[(size_t)i * gridDim.x + b]);
        y = warp_sum(y);
        if (lane == 0) out[i] = y;
    }
    __syncthreads();  // every warp's partial reads before the counter is re-armed
    if (threadIdx.x == 0) *rc.counter = 0u;
}

// (z, q_j) for all j < it: each block loops over j; the last block reduces every j
__global__ void __launch_bounds__(kRedThreads, 4)
    k_outer_multidot(int n, const double *__restrict__ z, double *const *__restrict__ Q,
                     const int *__restrict__ it_ptr, double *osc, RedCtx rc) {
    const int it = *it_ptr;
    for (int c0 = 0; c0 < it; c0 += kDotChunk)
        mdot_chunk(n, z, Q, c0, min(kDotChunk, it - c0), rc.partials);
    mdot_finish(it, osc + OS_ZQ, rc);
}

// p_it = z - sum_j (z, q_j) / (p_j, q_j) p_j   (Alg. 1 step 2 on the finest level)
// The coefficients are divided once per block (FP64 division is a long instruction sequence
// on this GPU), the same values as dividing per row.
constexpr int kOrthCoef = 256;

__global__ void k_outer_orth(int n, const double *__restrict__ z, double *const *__restrict__ P,
                             const int *__restrict__ it_ptr, const double *__restrict__ osc,
                             const double *__restrict__ opq) {
    const int it = *it_ptr;
    __shared__ double cf[kOrthCoef];
    for (int j = threadIdx.x; j < it && j < kOrthCoef; j += blockDim.x)
        cf[j] = -osc[OS_ZQ + j] / opq[j];
    __syncthreads();
    double *p = P[it];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = z[i];
        for (int j = 0; j < it; j++)
            acc += (j < kOrthCoef ? cf[j] : -osc[OS_ZQ + j] / opq[j]) * P[j][i];
        p[i] = acc;
    }
}

// q = A p, (p, q) -> opq[it], (r, p) -> osc[RP]
__global__ void __launch_bounds__(kRedThreads) k_outer_spmv_dot(GLev<double> L,
                                                                double *const *__restrict__ P,
                                                                double *const *__restrict__ Q,
                                                                const int *__restrict__ it_ptr,
                                                                const double *__restrict__ r,
                                                                double *osc, double *opq,
                                                                RedCtx rc) {
    const int it = *it_ptr;
    const double *p = P[it];
    double *q = Q[it];
    double v[2] = {0.0, 0.0};
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < L.n; row += gridDim.x * blockDim.x) {
        int base, width;
        row_span(L, row, base, width);  // computed, not loaded, for uniform slices
        const double acc = row_dot(L, base, 0, width, p);
        q[row] = acc;
        v[0] += p[row] * acc;
        v[1] += r[row] * p[row];
    }
    double *out[2] = {&opq[it], &osc[OS_RP]};
    reduce_store<2, RM_LASTBLOCK, double>(v, out, rc, 0, BlockGroup{});
}

// alpha = (r, p) / (p, Ap); x += alpha p; r -= alpha q; (r, r)
__global__ void __launch_bounds__(kRedThreads) k_outer_update(int n, double *const *__restrict__ P,
                                                              double *const *__restrict__ Q,
                                                              int *it_ptr, double *__restrict__ x,
                                                              double *__restrict__ r, double *osc,
                                                              const double *__restrict__ opq,
                                                              RedCtx rc) {
    const int it = *it_ptr;
    const double pq = opq[it];
    const bool bad = !(pq > 0.0) || !isfinite(pq);
    __shared__ double alpha_s;  // one FP64 division per block, not per thread
    if (threadIdx.x == 0) alpha_s = bad ? 0.0 : osc[OS_RP] / pq;
    __syncthreads();
    const double alpha = alpha_s;
    const double *p = P[it];
    const double *q = Q[it];
    double v[1] = {0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        double rn = r[i] - alpha * q[i];
        r[i] = rn;
        v[0] += rn * rn;
    }
    double *out[1] = {&osc[OS_RR]};
    reduce_store<1, RM_LASTBLOCK, double>(v, out, rc, 0, BlockGroup{});
    if (blockIdx.x == 0 && threadIdx.x == 0 && bad) osc[OS_STOP] = 1.0;
}

__global__ void k_bump(int *it_ptr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *it_ptr += 1;
}


// ---------------------------------------------------------------------------------------
// FGMRES kernels (FP64, pi order); V and Z are arrays of vector pointers
// w = A z
__global__ void k_spmv(GLev<double> L, const double *__restrict__ z, double *__restrict__ w) {
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < L.n; row += gridDim.x * blockDim.x) {
        int base, width;
        row_span(L, row, base, width);
        w[row] = row_dot(L, base, 0, width, z);
    }
}

// out[i] = (w, V[i]) for i < m
__global__ void __launch_bounds__(kRedThreads, 4) k_mdot(int n, const double *__restrict__ w,
                                                      double *const *__restrict__ V, int m,
                                                      double *out, RedCtx rc) {
    for (int c0 = 0; c0 < m; c0 += kDotChunk)
        mdot_chunk(n, w, V, c0, min(kDotChunk, m - c0), rc.partials);
    mdot_finish(m, out, rc);
}

// The second Gram-Schmidt pass's dots fused with the first pass's subtraction (both are
// row-local): w -= sum_i c[i] V[i], then out[i] = (w, V[i]) for i < m. Each row's new w is
// written by the thread that reads it again in the later chunks.
__global__ void __launch_bounds__(kRedThreads, 4) k_orth_mdot(int n, double *__restrict__ w,
                                                           double *const *__restrict__ V, int m,
                                                           const double *__restrict__ c,
                                                           double *out, RedCtx rc) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double x = w[k];
        for (int i = 0; i < m; i++) x -= c[i] * V[i][k];
        w[k] = x;
    }
    for (int c0 = 0; c0 < m; c0 += kDotChunk)
        mdot_chunk(n, w, V, c0, min(kDotChunk, m - c0), rc.partials);
    mdot_finish(m, out, rc);
}

// w -= sum_i c[i] V[i]; (w, w) -> *nrm2
__global__ void __launch_bounds__(kRedThreads) k_orth_sub(int n, double *__restrict__ w,
                                                          double *const *__restrict__ V, int m,
                                                          const double *__restrict__ c,
                                                          double *nrm2, RedCtx rc) {
    double a[1] = {0.0};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double x = w[k];
        for (int i = 0; i < m; i++) x -= c[i] * V[i][k];
        w[k] = x;
        a[0] += x * x;
    }
    double *o[1] = {nrm2};
    reduce_store<1, RM_LASTBLOCK, double>(a, o, rc, 0, BlockGroup{});
}

// v = w * s
__global__ void k_scale(int n, const double *__restrict__ w, double s, double *__restrict__ v) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) v[k] = w[k] * s;
}

// x += sum_j y[j] Z[j]
__global__ void k_lincomb(int n, double *__restrict__ x, double *const *__restrict__ Z, int m,
                          const double *__restrict__ y) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double acc = x[k];
        for (int j = 0; j < m; j++) acc += y[j] * Z[j][k];
        x[k] = acc;
    }
}

// =======================================================================================
// diagnostics: per-kernel timing and algorithmic bytes
thread_local int64_t g_launches = 0;

enum : int { K_CYCLE = OP_NKINDS, K_OUTER_MULTIDOT, K_OUTER_ORTH, K_OUTER_SPMV_DOT, K_OUTER_UPDATE,
             K_TRUE_RESIDUAL, K_FGMRES_SPMV, K_FGMRES_MDOT, K_FGMRES_ORTH, K_NUM };
constexpr int K_IN_CYCLE = 100;  // + op kind: an op timed inside the persistent kernel
constexpr int K_IN_TAIL = 200;   // + op kind: an op timed inside the shared-memory tail

const char *kernel_name(int kind) {
    static const char *names[K_NUM] = {"zero", "gs_colour", "resid_restrict", "prolong_correct",
                                       "coarse_solve", "alg1_multidot", "alg1_orth",
                                       "alg1_spmv_dot", "alg1_update", "tail_cta", "barrier_only",
                                       "gs_first_colour", "residual", "restrict_gather",
                                       "cycle_persistent", "outer_multidot", "outer_orth",
                                       "outer_spmv_dot", "outer_update", "true_residual",
                                       "fgmres_spmv", "fgmres_mdot", "fgmres_orth_sub"};
    static const char *incycle[OP_NKINDS] = {"in_cycle:zero", "in_cycle:gs_colour",
                                             "in_cycle:resid_restrict", "in_cycle:prolong_correct",
                                             "in_cycle:coarse_solve", "in_cycle:alg1_multidot",
                                             "in_cycle:alg1_orth", "in_cycle:alg1_spmv_dot",
                                             "in_cycle:alg1_update", "in_cycle:tail_cta",
                                             "in_cycle:barrier_only", "in_cycle:gs_first_colour",
                                             "in_cycle:residual", "in_cycle:restrict_gather"};
    static const char *intail[OP_NKINDS] = {"in_tail:zero", "in_tail:gs_colour",
                                            "in_tail:resid_restrict", "in_tail:prolong_correct",
                                            "in_tail:coarse_solve", "in_tail:alg1_multidot",
                                            "in_tail:alg1_orth", "in_tail:alg1_spmv_dot",
                                            "in_tail:alg1_update", "in_tail:?", "in_tail:?",
                                            "in_tail:gs_first_colour", "in_tail:residual",
                                            "in_tail:restrict_gather"};
    if (kind >= K_IN_CYCLE && kind < K_IN_CYCLE + OP_NKINDS) return incycle[kind - K_IN_CYCLE];
    if (kind >= K_IN_TAIL && kind < K_IN_TAIL + OP_NKINDS) return intail[kind - K_IN_TAIL];
    return (kind >= 0 && kind < K_NUM) ? names[kind] : "unknown";
}

struct Profiler {
    struct Rec {
        int kind, level;
        double bytes;
        cudaEvent_t a, b;
    };
    bool on = false;
    bool tail_ops = false;  // also time every op inside the shared-memory tail
    std::vector<Rec> pending;
    struct Acc {
        int64_t launches = 0;
        double ms = 0, bytes = 0;
    };
    std::vector<std::pair<std::pair<int, int>, Acc>> acc;

    Acc &slot(int kind, int level) {
        for (auto &e : acc)
            if (e.first.first == kind && e.first.second == level) return e.second;
        acc.push_back({{kind, level}, Acc()});
        return acc.back().second;
    }
    void add(int kind, int level, double ms, double bytes, int64_t launches = 1) {
        Acc &a = slot(kind, level);
        a.launches += launches;
        a.ms += ms;
        a.bytes += bytes;
    }
    Rec begin(int kind, int level, double bytes, cudaStream_t s) {
        Rec r{kind, level, bytes, nullptr, nullptr};
        AMG_CUDA(cudaEventCreate(&r.a));
        AMG_CUDA(cudaEventCreate(&r.b));
        AMG_CUDA(cudaEventRecord(r.a, s));
        return r;
    }
    void end(Rec &r, cudaStream_t s) {
        AMG_CUDA(cudaEventRecord(r.b, s));
        pending.push_back(r);
    }
    void harvest() {
        for (auto &r : pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) add(r.kind, r.level, ms, r.bytes);
            else cudaGetLastError();
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        pending.clear();
    }
    ~Profiler() {
        for (auto &r : pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    }
};

void profiler_enable(amg_hierarchy *h, int mode) {
    if (!h->prof) h->prof = new Profiler();
    h->prof->on = mode != 0;
    h->prof->tail_ops = mode == 1;
    h->prof->acc.clear();
}

void profiler_free(amg_hierarchy *h) {
    delete h->prof;
    h->prof = nullptr;
}

int profiler_read(const amg_hierarchy *h, int cap, int32_t *kind, int32_t *level,
                  int64_t *launches, double *ms, double *bytes) {
    if (!h->prof) return 0;
    int k = 0;
    for (auto &e : h->prof->acc) {
        if (k >= cap) break;
        if (kind) kind[k] = e.first.first;
        if (level) level[k] = e.first.second;
        if (launches) launches[k] = e.second.launches;
        if (ms) ms[k] = e.second.ms;
        if (bytes) bytes[k] = e.second.bytes;
        k++;
    }
    return (int)h->prof->acc.size();
}

static bool profiling(const amg_hierarchy *h) { return h->prof && h->prof->on; }

// algorithmic bytes of one op: every array the op must touch, once, at its width
// (w = value width, 4-byte column indices; padding of the sliced ELL is not counted)
static double op_bytes(const amg_hierarchy *h, const Op &op, int w) {
    const Level &lv = h->lev[op.level];
    const double n = lv.n, nnz = (double)lv.A.stored;
    const double nn = op.level + 1 < h->nlev ? h->lev[op.level + 1].n : 0;
    switch (op.kind) {
        case OP_ZERO: return w * n;
        case OP_GS_FIRST: return w * n + 2.0 * w * (op.i1 - op.i0);
        case OP_GS: {
            const std::vector<int> &ranges = op.level == 0 ? lv.color_blocks : lv.color_rows;
            int c = 0;
            while (c + 1 < (int)ranges.size() && ranges[c] != op.i0) c++;
            double rows = lv.color_rows[c + 1] - lv.color_rows[c];
            double e = c < (int)lv.color_nnz.size() ? (double)lv.color_nnz[c] : 0;
            double blocks = op.i1 - op.i0;
            return e * (4 + w) + rows * 3.0 * w + (op.level == 0 ? 4.0 * blocks : 0.0);
        }
        case OP_RESTRICT:
            return nnz * (4 + w) + 2.0 * w * n + w * nn + (op.level == 0 ? 4.0 * nn : 16.0 * nn);
        // the two passes of a split restriction: the restriction's bytes, shared out (the
        // intermediate residual vector is the split's own traffic, not the method's)
        case OP_RESID: return nnz * (4 + w) + 2.0 * w * n;
        case OP_GATHER: return w * nn + 16.0 * nn;
        case OP_PROLONG: return 2.0 * w * n + 4.0 * n + w * nn;
        case OP_COARSE: return w * n * n + 2.0 * w * n;
        case OP_MULTIDOT: return w * n * (1 + op.step);
        case OP_ORTH: return w * n * (2 + op.step);
        case OP_SPMV_DOT: return nnz * (4 + w) + 3.0 * w * n;
        case OP_UPDATE: return (op.step == 0 ? 2.0 : 3.0) * w * n + (op.last ? 0.0 : 3.0 * w * n);
    }
    return 0;
}

// =======================================================================================
// host side
struct EngineBase {
    Op *prog = nullptr;
    int nops = 0;
    int *tail_colors = nullptr;  // colour ranges of the tail levels
    int tail_color_words = 0;
    TailLayout lay{};
    size_t smem = 0;
    int grid = 0;
    int coop = 0;  // the cycle kernel instance with the lane-parallel block smoother
    int big_smem = 0;  // CTAs 1.. sweep the big blocks in their shared memory
    int big_wwarps = 0;  // warps of a CTA with a slice for the warp-sized blocks
    unsigned big_wslice = 0;
    std::vector<Op> hprog, htail;
    double tail_bytes = 0, cycle_bytes = 0;
    unsigned long long *ts = nullptr;
    unsigned long long *tprof = nullptr;
};

namespace {

template <class T>
Vecs<T> &vecs(Level &lv);
template <>
Vecs<double> &vecs<double>(Level &lv) { return lv.v64; }
template <>
Vecs<float> &vecs<float>(Level &lv) { return lv.v32; }

int red_grid(int64_t n) {
    return (int)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, (n + kRedThreads - 1) / kRedThreads));
}

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }


// finest-level blocks of six or more rows on average (the octree's 2x2x2-node aggregates):
// the lane-parallel block smoother (op_gs_blocks_coop) and restriction. Smaller blocks (a few
// rows, as on a quadtree with several nodes per cell) keep one thread per block: with
// kBlockLanes lanes each, most lanes would idle and the sweep would need more passes.
bool coop_blocks(const Level &lv) {
    return lv.nblocks > 0 && 6 * (int64_t)lv.nblocks <= (int64_t)lv.n;
}

bool is_reduction(const Op &op) {
    return op.kind == OP_MULTIDOT || op.kind == OP_SPMV_DOT || (op.kind == OP_UPDATE && !op.last);
}

// Walks Alg. 2 / Alg. 1 from a level and appends the ops to a program. The recursion stops
// at `stop_level`, where one OP_TAIL stands for B~ of that level (persistent program), or
// continues to the coarsest level (tail program, standalone execution).
struct Builder {
    amg_hierarchy *h;
    std::vector<Op> *out;
    int stop_level;  // >= nlev: never stop

    static Op mk(int kind, int level) {
        Op o;
        std::memset(&o, 0, sizeof o);
        o.kind = kind;
        o.level = level;
        o.red_pb = -1;
        o.fin_pb = -1;
        for (int k = 0; k < 4; k++) o.fin_dst[k] = -1;
        return o;
    }
    void emit(const Op &o) { out->push_back(o); }

    // first non-empty colour of level l (its point-GS first colour), [r0, r1)
    void first_colour(int l, int &r0, int &r1) const {
        const std::vector<int> &ranges = h->lev[l].color_rows;
        const int nc = (int)ranges.size() - 1;
        int c0 = 0;
        while (c0 < nc && ranges[c0 + 1] == ranges[c0]) c0++;
        r0 = c0 < nc ? ranges[c0] : 0;
        r1 = c0 < nc ? ranges[c0 + 1] : 0;
    }
    // does B~_l start with the point-GS first colour of B^_l (step 0) in this program?
    bool starts_with_first_colour(int l) const {
        return l >= 1 && l < h->nlev && l != stop_level && !h->lev[l].coarsest;
    }

    // the big blocks of colour c on the finest level go to whole CTAs (grid-wide programs)
    void big_range(int l, int c, Op &g) const {
        const Level &lv = h->lev[l];
        if (l != 0 || lv.nbig == 0) return;
        g.bb0 = lv.color_big[c];
        g.bbc = lv.color_bigc[c];
        g.bb1 = lv.color_big[c + 1];
    }

    // z = B^_l [f] (Alg. 2). first_done: the first colour of the pre-smoothing was already
    // done by the op before (a fused RESTRICT or UPDATE)
    void bhat(int l, int fsel, int zsel, bool first_done = false) {
        Level &lv = h->lev[l];
        const std::vector<int> &ranges = (l == 0) ? lv.color_blocks : lv.color_rows;
        const int nc = (int)ranges.size() - 1;
        int c0 = 0;  // pre-smoothing u1 = R_k f from zero, colours ascending
        if (l == 0) {
            Op z = mk(OP_ZERO, l);
            z.usel = zsel;
            emit(z);
        } else {  // first non-empty colour fused with the zero fill (point smoother)
            while (c0 < nc && ranges[c0 + 1] == ranges[c0]) c0++;
            if (!first_done) {
                Op g = mk(OP_GS_FIRST, l);
                g.i0 = c0 < nc ? ranges[c0] : 0;
                g.i1 = c0 < nc ? ranges[c0 + 1] : 0;
                g.fsel = fsel;
                g.usel = zsel;
                emit(g);
            }
            c0++;
        }
        // the first sweep's remaining colours, then nu_pre - 1 further forward sweeps
        for (int sw = 0; sw < h->opt.nu_pre; sw++)
            for (int c = sw == 0 ? c0 : 0; c < nc; c++) {
                if (ranges[c + 1] == ranges[c]) continue;
                Op g = mk(OP_GS, l);
                g.i0 = ranges[c];
                g.i1 = ranges[c + 1];
                g.fsel = fsel;
                g.usel = zsel;
                big_range(l, c, g);
                emit(g);
            }
        Op rs = mk(OP_RESTRICT, l);  // next.rhs = P^t (f - A u1)
        rs.fsel = fsel;
        rs.usel = zsel;
        if (l == 0 && lv.nbig > 0) rs.bb1 = lv.nbig;  // every big block, by whole CTAs
        const bool fuse = starts_with_first_colour(l + 1);
        if (fuse) {  // and the next level's first colour from zero
            rs.fuse = 1;
            first_colour(l + 1, rs.f0, rs.f1);
        }
        if (l >= 1 && lv.n >= kSplitRestrictRows) {
            // a large coarse level: the residual row by row into q_step, then the children
            // sums (coalesced slots instead of a gather over four colours' rows)
            Op rr = mk(OP_RESID, l);
            rr.fsel = fsel;
            rr.usel = zsel;
            rr.step = zsel - V_P0;
            emit(rr);
            rs.kind = OP_GATHER;
            rs.step = zsel - V_P0;
        }
        emit(rs);
        btilde(l + 1, fuse);         // next.e = B~_{k-1}[next.rhs]
        Op pr = mk(OP_PROLONG, l);   // u2 = u1 + P e
        pr.usel = zsel;
        emit(pr);
        for (int sw = 0; sw < h->opt.nu_post; sw++)  // post-smoothing: colours descending
            for (int c = nc - 1; c >= 0; c--) {
                if (ranges[c + 1] == ranges[c]) continue;
                Op g = mk(OP_GS, l);
                g.i0 = ranges[c];
                g.i1 = ranges[c + 1];
                g.backward = 1;
                g.fsel = fsel;
                g.usel = zsel;
                big_range(l, c, g);
                emit(g);
            }
    }

    // e = B~_l [rhs] (Alg. 1 with kcycle_n steps; exact on the coarsest level). first_done:
    // step 0's first colour was done by the restriction into this level
    void btilde(int l, bool first_done = false) {
        if (l == stop_level) {
            emit(mk(OP_TAIL, l));
            return;
        }
        Level &lv = h->lev[l];
        if (lv.coarsest) {
            emit(mk(OP_COARSE, l));
            return;
        }
        const int n = h->opt.kcycle_n;
        for (int i = 0; i < n; i++) {
            bhat(l, i == 0 ? V_RHS : V_R, V_P0 + i, i == 0 ? first_done : true);
            if (i > 0) {
                Op md = mk(OP_MULTIDOT, l);
                md.step = i;
                emit(md);
                Op ot = mk(OP_ORTH, l);
                ot.step = i;
                emit(ot);
            }
            Op sd = mk(OP_SPMV_DOT, l);
            sd.step = i;
            emit(sd);
            Op up = mk(OP_UPDATE, l);
            up.step = i;
            up.last = (i == n - 1);
            if (!up.last) {  // and the next step's first colour from zero, on r_{i+1}
                up.fuse = 1;
                first_colour(l, up.f0, up.f1);
            }
            emit(up);
        }
    }
};

// persistent program: reductions leave partials in alternating buffers; the next op sums
// them into the level's scalars
void annotate_reductions(std::vector<Op> &prog) {
    std::vector<Op> out;
    int pb = 0;
    bool pending = false;
    Op pend{};
    auto attach = [&](Op &op) {
        op.fin_pb = pend.red_pb;
        op.fin_level = pend.level;
        if (pend.kind == OP_MULTIDOT) {
            op.fin_n = pend.step;
            for (int j = 0; j < pend.step; j++) op.fin_dst[j] = SC_ZQ0 + j;
        } else if (pend.kind == OP_SPMV_DOT) {
            op.fin_n = 2;
            op.fin_dst[0] = SC_PQ0 + pend.step;
            op.fin_dst[1] = SC_RP0 + pend.step;
        } else {
            op.fin_n = 1;
            op.fin_dst[0] = SC_RR0 + pend.step;
        }
    };
    for (Op op : prog) {
        if (pending) {
            attach(op);
            pending = false;
        }
        if (is_reduction(op)) {
            op.red_pb = pb;
            pb ^= 1;
            pending = true;
            pend = op;
        }
        out.push_back(op);
    }
    if (pending) {
        Op nop = Builder::mk(OP_NOP, pend.level);
        attach(nop);
        out.push_back(nop);
    }
    prog.swap(out);
}

template <class T>
void table_image(amg_hierarchy *h, std::vector<GLev<T>> &tab) {
    tab.assign(h->nlev, GLev<T>());
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        GLev<T> &d = tab[l];
        std::memset(&d, 0, sizeof d);
        d.n = lv.n;
        d.fine = (l == 0) ? 1 : 0;
        // blocks of several rows (octree aggregates): a lane per row (op_gs_blocks_coop)
        d.bg = (l == 0 && coop_blocks(lv)) ? kBlockLanes : 0;
        d.w = lv.A.uw;
        d.sl = lv.A.sl_ptr;
        d.col = lv.A.col;
        if constexpr (sizeof(T) == 8) d.val = (const T *)lv.A.val;
        else d.val = (const T *)lv.A.val32;
        if constexpr (sizeof(T) == 8) d.dinv = (const T *)lv.dinv64;
        else d.dinv = (const T *)lv.dinv32;
        d.col16 = lv.col16;
        d.bptr = lv.bptr;
        d.big = (l == 0) ? lv.big_dev : nullptr;
        d.parent = lv.parent;
        d.children = (l + 1 < h->nlev) ? h->lev[l + 1].children : nullptr;
        d.children2 = (l + 1 < h->nlev) ? h->lev[l + 1].children2 : nullptr;
        d.Ainv = lv.Ainv;
        d.Ainv2 = lv.Ainv32;
        Vecs<T> &v = vecs<T>(lv);
        d.rhs = v.rhs;
        d.e = v.e;
        d.r = v.r;
        for (int i = 0; i < kMaxKcycle; i++) {
            d.p[i] = v.p[i];
            d.q[i] = v.q[i];
        }
        d.sc = lv.sc;
        d.nnext = (l + 1 < h->nlev) ? h->lev[l + 1].n : 0;
    }
}

template <class T>
void fill_tables(amg_hierarchy *h) {
    std::vector<GLev<T>> tab;
    table_image<T>(h, tab);
    void *&dst = (sizeof(T) == 8) ? h->lev_tab64 : h->lev_tab32;
    if (!dst) dst = halloc<GLev<T>>(h, h->nlev);
    AMG_CUDA(cudaMemcpyAsync(dst, tab.data(), sizeof(GLev<T>) * h->nlev, cudaMemcpyHostToDevice,
                             h->stream));
}

template <class T>
const GLev<T> *dtab(amg_hierarchy *h) {
    return (const GLev<T> *)((sizeof(T) == 8) ? h->lev_tab64 : h->lev_tab32);
}

// shared-memory image of levels l0..nlev-1; returns false if a level is too large
// widest slice (slots per row) of each level, from its slice pointers
std::vector<int> slice_widths(amg_hierarchy *h) {
    std::vector<int> w(h->nlev, 0);
    std::vector<std::vector<int>> sl(h->nlev);
    bool read = false;
    for (int l = 0; l < h->nlev; l++) {
        const Sell &A = h->lev[l].A;
        if (A.uw > 0) {  // one width, known here
            w[l] = A.uw;
            continue;
        }
        sl[l].resize(A.nslices + 1);
        AMG_CUDA(cudaMemcpyAsync(sl[l].data(), A.sl_ptr, sizeof(int) * sl[l].size(),
                                 cudaMemcpyDeviceToHost, h->stream));
        read = true;
    }
    if (read) AMG_CUDA(cudaStreamSynchronize(h->stream));
    for (int l = 0; l < h->nlev; l++)
        for (size_t k = 0; k + 1 < sl[l].size(); k++)
            w[l] = std::max(w[l], (sl[l][k + 1] - sl[l][k]) / kSliceH);
    return w;
}

// shared-memory image of the tail from level l0 down (value size `vb` bytes); the top level
// may stay in HBM (top_in_gmem). False if a level is too large or the tail too deep.
bool tail_layout(amg_hierarchy *h, int l0, int vb, bool top_in_gmem,
                 const std::vector<int> &widths, TailLayout &Y) {
    std::memset(&Y, 0, sizeof Y);
    Y.tl = l0;
    Y.nlev = h->nlev;
    Y.kc = h->opt.kcycle_n;
    Y.nu_pre = h->opt.nu_pre;
    Y.nu_post = h->opt.nu_post;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        int o = (int)off;
        off += align16(bytes);
        return o;
    };
    // colour ranges of every tail level, one block
    int words = 0;
    for (int l = l0; l < h->nlev; l++) words += (int)h->lev[l].color_rows.size();
    const int cbase = take(sizeof(int) * (size_t)words);
    int cw = 0;
    // one slice width for the staged levels: 9 (3x3-cell stencils) if every one fits
    bool w9 = true;
    for (int l = l0 + (top_in_gmem ? 1 : 0); l < h->nlev; l++) w9 = w9 && widths[l] <= 9;
    Y.W = w9 ? 9 : 0;
    const int kc = h->opt.kcycle_n;
    for (int l = l0; l < h->nlev; l++) {
        const Level &lv = h->lev[l];
        TailLevelLayout &y = Y.lv[l];
        y.n = lv.n;
        y.nslices = lv.A.nslices;
        y.padded = (int)lv.A.padded;
        y.colors = cbase + (int)sizeof(int) * cw;
        y.ncolors = (int)lv.color_rows.size() - 1;
        cw += (int)lv.color_rows.size();
        if (l == l0 && top_in_gmem) {
            if (lv.n > 65535 || lv.coarsest) return false;
            y.gmem = 1;
            y.w = 0;
            y.col = y.val = y.dinv = y.parent = y.children = y.children2 = y.Ainv = -1;
            y.rhs = y.e = y.r = -1;
            for (int k = 0; k < kMaxKcycle; k++) y.p[k] = y.q[k] = -1;
            continue;
        }
        if (lv.n > kTailRowsMax) return false;
        y.w = w9 ? 9 : std::max(1, widths[l]);
        const size_t img = (size_t)lv.A.nslices * kSliceH * y.w;
        y.col = take(2 * img);
        y.val = take((size_t)vb * img);
        y.dinv = lv.coarsest ? -1 : take((size_t)vb * lv.n);
        y.parent = lv.coarsest ? -1 : take(sizeof(int) * (size_t)lv.n);
        y.children = (l > l0) ? take(sizeof(int4) * (size_t)lv.n) : -1;
        y.children2 = (l > l0 && lv.children2) ? take(sizeof(int4) * (size_t)lv.n) : -1;
        y.Ainv = lv.coarsest ? take(sizeof(double) * lv.n * lv.n) : -1;
        y.rhs = take((size_t)vb * lv.n);
        y.e = take((size_t)vb * lv.n);
        y.r = lv.coarsest ? -1 : take((size_t)vb * lv.n);
        for (int k = 0; k < kMaxKcycle; k++) {
            y.p[k] = (!lv.coarsest && k < kc) ? take((size_t)vb * lv.n) : -1;
            y.q[k] = (!lv.coarsest && k < kc) ? take((size_t)vb * lv.n) : -1;
        }
        if (off > (size_t)INT32_MAX) return false;
    }
    // narrow group: about one thread per row of a colour of the largest staged level (a
    // quarter of its rows for the 2x2 colouring), whole warps, 128..1024 threads
    int nmax = 0;
    for (int l = l0; l < h->nlev; l++)
        if (!Y.lv[l].gmem) nmax = std::max(nmax, Y.lv[l].n);
    Y.narrow = std::min(vb == 8 ? kPThreads64 : kPThreads, std::max(128, (nmax / 4 + 31) / 32 * 32));
    if (const char *e = getenv("AMG_TAIL_NARROW")) {  // tuning knob: threads of the narrow group
        const int v = atoi(e);
        if (v >= 32 && v <= (vb == 8 ? kPThreads64 : kPThreads) && v % 32 == 0) Y.narrow = v;
    }
    Y.sc = take(sizeof(double) * SC_N * (size_t)(h->nlev - l0));
    Y.bytes = (int)off;
    return true;
}

template <class T>
EngineBase *&engine_slot(amg_hierarchy *h) {
    return (sizeof(T) == 8) ? h->eng64 : h->eng32;
}

int max_tail_bytes() {
    static int v = [] {
        const char *e = getenv("AMG_TAIL_SMEM");  // tuning knob: cap on the staged tail
        return e ? atoi(e) : INT32_MAX;
    }();
    return v;
}

template <class T>
void *cycle_kernel(int W, int B) {
    if (B) return W == 9 ? (void *)k_cycle<T, 9, 1> : (void *)k_cycle<T, 0, 1>;
    return W == 9 ? (void *)k_cycle<T, 9, 0> : (void *)k_cycle<T, 0, 0>;
}

template <class T>
void build_engine(amg_hierarchy *h) {
    EngineBase *&E = engine_slot<T>(h);
    if (!E) E = new EngineBase();
    cudaStream_t s = h->stream;
    int dev = h->device, optin = 0, nsm = 0;
    AMG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    AMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    size_t static_smem = 0;
    for (int W : {0, 9})
        for (int B : {0, 1}) {
            cudaFuncAttributes fa;
            AMG_CUDA(cudaFuncGetAttributes(&fa, cycle_kernel<T>(W, B)));
            static_smem = std::max(static_smem, fa.sharedSizeBytes);
        }
    E->coop = coop_blocks(h->lev[0]) ? 1 : 0;
    const long budget = std::min<long>((long)optin - (long)static_smem - 1024,
                                       (long)max_tail_bytes());
    // the tail: the finest coarse level from which everything fits in shared memory, or
    // fits once that top level is left in HBM/L2 (read in place by CTA 0)
    const std::vector<int> widths = slice_widths(h);
    int tl = h->nlev;
    for (int l = 1; l < h->nlev && tl == h->nlev; l++) {
        for (int top_gmem = 0; top_gmem <= 1; top_gmem++) {
            TailLayout Y;
            if (tail_layout(h, l, sizeof(T), top_gmem != 0, widths, Y) && Y.bytes <= budget) {
                tl = l;
                E->lay = Y;
                break;
            }
        }
    }
    if (tl < h->nlev && E->lay.lv[tl].gmem && !h->lev[tl].col16) {
        Level &lv = h->lev[tl];
        lv.col16 = halloc<unsigned short>(h, lv.A.padded);
        k_col16<<<nblocks_for(lv.A.padded, 256), 256, 0, h->stream>>>((int)lv.A.padded, lv.A.col, lv.col16);
        AMG_LAUNCH_CHECK();
        fill_tables<T>(h);
    }
    if (tl == h->nlev) {
        std::memset(&E->lay, 0, sizeof E->lay);
        E->lay.tl = h->nlev;
        E->lay.nlev = h->nlev;
    }
    h->tail_level = tl;
    E->hprog.clear();
    E->htail.clear();
    Builder b{h, &E->hprog, tl};
    b.bhat(0, V_RHS, V_E);
    annotate_reductions(E->hprog);
    E->tail_color_words = 0;
    if (tl < h->nlev) {
        Builder bt{h, &E->htail, h->nlev + 1};  // the tail's ops (traffic accounting only)
        bt.btilde(tl);
        std::vector<int> words;
        for (int l = tl; l < h->nlev; l++)
            words.insert(words.end(), h->lev[l].color_rows.begin(), h->lev[l].color_rows.end());
        E->tail_color_words = (int)words.size();
        E->tail_colors = halloc<int>(h, words.size());
        AMG_CUDA(cudaMemcpyAsync(E->tail_colors, words.data(), sizeof(int) * words.size(),
                                 cudaMemcpyHostToDevice, s));
        AMG_CUDA(cudaStreamSynchronize(s));  // words is a local
    }
    E->tail_bytes = 0;
    for (const Op &op : E->htail) E->tail_bytes += op_bytes(h, op, sizeof(T));
    E->cycle_bytes = 0;
    for (const Op &op : E->hprog)
        E->cycle_bytes += (op.kind == OP_TAIL) ? E->tail_bytes
                          : (op.kind == OP_NOP) ? 0.0 : op_bytes(h, op, sizeof(T));
    E->nops = (int)E->hprog.size();
    E->prog = halloc<Op>(h, E->hprog.size());
    AMG_CUDA(cudaMemcpyAsync(E->prog, E->hprog.data(), sizeof(Op) * E->hprog.size(),
                             cudaMemcpyHostToDevice, s));
    E->smem = tl < h->nlev ? (size_t)E->lay.bytes : 0;
    // Big blocks: swept in the shared memory of CTAs 1... A CTA-sized block needs as much as
    // the largest one that fits on the device; the warp-sized ones get a slice each on as
    // many warps per CTA as the most of them in one colour need (a block that does not fit
    // takes the global-memory sweep; the forward and backward schedules each count).
    E->big_smem = 0;
    E->big_wwarps = 0;
    E->big_wslice = 0;
    if (h->lev[0].nbig > 0 && nsm > 1) {
        const Level &F0 = h->lev[0];
        const int vsel = sizeof(T) == 8;
        const size_t avail = (size_t)std::max<long>(0, (long)optin - (long)static_smem - 1024);
        size_t big = 0;
        for (size_t need : F0.big_smem[vsel])
            if (need > 0 && need <= avail) big = std::max(big, need);
        const size_t wneed = F0.big_smem_warp[vsel];
        int wtasks = 0;  // warp-sized blocks of the fullest colour
        for (size_t c = 0; c < F0.color_bigc.size(); c++)
            wtasks = std::max(wtasks, F0.color_bigc[c] - F0.color_big[c]);
        if (wneed > 0 && wneed <= avail && wtasks > 0) {
            const int per_cta = (wtasks + nsm - 2) / (nsm - 1);
            E->big_wwarps = std::min({cycle_threads<T>() / 32, per_cta, (int)(avail / wneed)});
            E->big_wslice = (unsigned)wneed;
        }
        const size_t smem = std::max(big, (size_t)E->big_wwarps * E->big_wslice);
        if (smem > 0) {
            E->big_smem = 1;
            E->smem = std::max(E->smem, smem);
        }
    }
    void *kern = cycle_kernel<T>(E->lay.W, E->coop);
    // the kernel's dynamic shared-memory limit is a property of the function, shared by every
    // hierarchy of the process: set it to the device maximum (never lower it below what
    // another hierarchy's launches use); each launch passes its own size
    AMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)std::max<long>(0, (long)optin - (long)static_smem)));
    int per_sm = 0;
    AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, cycle_threads<T>(),
                                                           E->smem));
    if (per_sm < 1) throw Error{AMG_ERR_CUDA, "persistent cycle kernel cannot be resident"};
    E->grid = nsm;  // one CTA per SM (co-resident: cooperative launch)
    E->ts = halloc<unsigned long long>(h, E->hprog.size() + 1);
    E->tprof = halloc<unsigned long long>(h, 2 * kTprofCount);
    AMG_CUDA(cudaMemsetAsync(E->tprof, 0, 2 * kTprofCount * sizeof(unsigned long long), s));
}

template <class T>
void alloc_vecs(amg_hierarchy *h) {
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        Vecs<T> &v = vecs<T>(lv);
        int n = lv.n;
        if (l > 0) {
            if (!v.rhs) v.rhs = halloc<T>(h, n);
            if (!v.e) v.e = halloc<T>(h, n);
        }
        if (l > 0 && !lv.coarsest) {
            if (!v.r) v.r = halloc<T>(h, n);
            for (int i = 0; i < h->opt.kcycle_n; i++) {
                if (!v.p[i]) v.p[i] = halloc<T>(h, n);
                if (!v.q[i]) v.q[i] = halloc<T>(h, n);
            }
        }
    }
}

void ensure_fp32(amg_hierarchy *h) {
    if (h->fp32_ready) return;
    cudaStream_t s = h->stream;
    // every step keeps what an earlier, failed attempt already allocated (an allocation can
    // fail part-way; the next solve then completes the set)
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        if (lv.A.val32) continue;
        float *v = halloc<float>(h, lv.A.padded);
        k_convert<double, float><<<nblocks_for(lv.A.padded, 256), 256, 0, s>>>(
            (int)lv.A.padded, lv.A.val, v);
        AMG_LAUNCH_CHECK();
        lv.A.val32 = v;
    }
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        if (lv.dinv32) continue;
        float *d = halloc<float>(h, lv.n);
        k_inv_diag<float><<<nblocks_for(lv.n, 256), 256, 0, s>>>(lv.n, lv.A.sl_ptr, lv.A.val, d);
        AMG_LAUNCH_CHECK();
        lv.dinv32 = d;
    }
    alloc_vecs<float>(h);
    if (!h->r32) h->r32 = halloc<float>(h, h->N);
    if (!h->z32) h->z32 = halloc<float>(h, h->N);
    h->lev[0].v32.rhs = h->r32;
    h->lev[0].v32.e = h->z32;
    fill_tables<float>(h);
    build_engine<float>(h);
    h->fp32_ready = true;
}

// one launch of the persistent kernel: z = B^_0 [r] on level 0's table buffers
template <class T>
void launch_cycle(amg_hierarchy *h, T *rhs0 = nullptr, T *e0 = nullptr) {
    // hierarchies of a batched setup get their single-system engine on first use
    if (!engine_slot<T>(h)) build_engine<T>(h);
    EngineBase *E = engine_slot<T>(h);
    cudaStream_t s = h->stream;
    const bool prof = profiling(h);
    CycleArgs<T> a;
    a.tab = dtab<T>(h);
    a.rhs0 = rhs0;
    a.e0 = e0;
    a.prog = E->prog;
    a.nops = E->nops;
    a.tail_colors = E->tail_colors;
    a.tail_color_words = E->tail_color_words;
    a.lay = E->lay;
    a.partials = h->cyc_partials;
    a.bar = h->bar;
    a.err = h->err_flag;
    a.bar_limit_ns = h->dbg_bar_limit_ns > 0 ? (unsigned long long)h->dbg_bar_limit_ns
                                             : kBarrierLimitNs;
    a.bar_extra = h->dbg_bar_extra;
    a.big_smem = E->big_smem;
    a.big_wwarps = E->big_wwarps;
    a.big_wslice = E->big_wslice;
    AMG_CUDA(cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), s));
    a.ts = prof ? E->ts + 1 : nullptr;
    a.tprof = (prof && h->prof->tail_ops) ? E->tprof : nullptr;
    Profiler::Rec rec{};
    if (prof) {
        k_timestamp<<<1, 1, 0, s>>>(E->ts);
        AMG_LAUNCH_CHECK();
        rec = h->prof->begin(K_CYCLE, 0, E->cycle_bytes, s);
    }
    void *args[] = {&a};
    AMG_CUDA(cudaLaunchCooperativeKernel(cycle_kernel<T>(E->lay.W, E->coop), dim3(E->grid),
                                         dim3(cycle_threads<T>()), args, E->smem, s));
    AMG_LAUNCH_CHECK();
    if (prof) h->prof->end(rec, s);
}

// per-op durations of the last profiled launch, from the in-kernel timestamps (each op's
// time includes the grid barrier that ends it)
template <class T>
void harvest_cycle_timestamps(amg_hierarchy *h) {
    EngineBase *E = engine_slot<T>(h);
    std::vector<unsigned long long> t(E->hprog.size() + 1);
    AMG_CUDA(cudaMemcpy(t.data(), E->ts, sizeof(unsigned long long) * t.size(),
                        cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < E->hprog.size(); k++) {
        const Op &op = E->hprog[k];
        double ms = (double)(t[k + 1] - t[k]) * 1e-6;
        double bytes = (op.kind == OP_TAIL) ? E->tail_bytes
                       : (op.kind == OP_NOP) ? 0.0 : op_bytes(h, op, sizeof(T));
        h->prof->add(K_IN_CYCLE + op.kind, op.level, ms, bytes);
    }
    // inside the tail: SM cycles per op kind and level, reported at the nominal clock
    std::vector<unsigned long long> tp(2 * kTprofCount);
    AMG_CUDA(cudaMemcpy(tp.data(), E->tprof, sizeof(unsigned long long) * tp.size(),
                        cudaMemcpyDeviceToHost));
    AMG_CUDA(cudaMemset(E->tprof, 0, sizeof(unsigned long long) * tp.size()));
    int khz = 0;
    AMG_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, h->device));
    for (int slot = 0; slot < kTprofCount; slot++)
        if (tp[kTprofCount + slot])
            h->prof->add(K_IN_TAIL + (slot & 15), slot / 16, (double)tp[slot] / khz, 0.0,
                         (int64_t)tp[kTprofCount + slot]);
}

// standalone execution of B^_l (diagnostic path): one kernel per op, every level in HBM
template <class T>
void run_standalone(amg_hierarchy *h, int l, int fsel, int zsel) {
    cudaStream_t s = h->stream;
    std::vector<Op> prog;
    Builder b{h, &prog, h->nlev + 1};
    b.bhat(l, fsel, zsel);
    RedCtx rc{h->red_partials, h->red_counter};
    for (const Op &op : prog) {
        const Level &lv = h->lev[op.level];
        int grid;
        switch (op.kind) {
            case OP_GS: grid = nblocks_for(op.i1 - op.i0, kRedThreads); break;
            case OP_RESTRICT: grid = nblocks_for(h->lev[op.level + 1].n, kRedThreads); break;
            case OP_COARSE: grid = 1; break;
            case OP_MULTIDOT:
            case OP_SPMV_DOT:
            case OP_UPDATE: grid = red_grid(lv.n); break;
            default: grid = nblocks_for(lv.n, kRedThreads);
        }
        k_op<T><<<grid, kRedThreads, 0, s>>>(dtab<T>(h), op, rc);
        AMG_LAUNCH_CHECK();
    }
}

}  // namespace

// the cycle's level copies in its precision (FP32 copies are made once, on first use)
void prepare_cycle(amg_hierarchy *h) {
    if (h->opt.cycle_prec != AMG_FP32 || h->fp32_ready) return;
    if (h->nlev > 1) {
        ensure_fp32(h);
        return;
    }
    // one level: the cycle is the exact solve (high/low float inverse) on FP32 vectors
    h->r32 = halloc<float>(h, h->N);
    h->z32 = halloc<float>(h, h->N);
    h->lev[0].v32.rhs = h->r32;
    h->lev[0].v32.e = h->z32;
    fill_tables<float>(h);
    h->fp32_ready = true;
}

// device level table of the cycle precision (LevelDev<T, int>[nlev])
const void *level_table(const amg_hierarchy *h, bool fp32) {
    return fp32 ? h->lev_tab32 : h->lev_tab64;
}

void allocate_solve_workspace(amg_hierarchy *h) {
    const int n = (int)h->N;
    h->red_partials = halloc<double>(h, (size_t)kRedBlocks * std::max(8, h->opt.max_iters + 8));
    h->red_counter = halloc<unsigned int>(h, 1);
    AMG_CUDA(cudaMemsetAsync(h->red_counter, 0, sizeof(unsigned int), h->stream));
    h->cyc_partials = halloc<double>(h, 2 * 4 * 1024);
    h->bar = halloc<unsigned long long>(h, 32);
    AMG_CUDA(cudaMemsetAsync(h->bar, 0, 32 * sizeof(unsigned long long), h->stream));
    alloc_vecs<double>(h);
    // level-0 cycle input / output are the outer solver's r and z
    h->xo = halloc<double>(h, n);
    h->ro = halloc<double>(h, n);
    h->zo = halloc<double>(h, n);
    h->to = halloc<double>(h, n);
    h->bo = halloc<double>(h, n);
    h->lev[0].v64.rhs = h->ro;
    h->lev[0].v64.e = h->zo;
    h->osc = halloc<double>(h, outer_scalar_count(h->opt.max_iters));
    h->oit = halloc<int>(h, 1);
    h->dP = halloc<double *>(h, h->opt.max_iters);
    h->dQ = halloc<double *>(h, h->opt.max_iters);
    ensure_pinned(h);
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        lv.dinv64 = halloc<double>(h, lv.n);
        k_inv_diag<double><<<nblocks_for(lv.n, 256), 256, 0, h->stream>>>(lv.n, lv.A.sl_ptr, lv.A.val,
                                                                          lv.dinv64);
        AMG_LAUNCH_CHECK();
    }
    fill_tables<double>(h);
    // the FP64 cycle's engine now; an FP32-cycle hierarchy builds its FP32 engine on its first
    // solve (ensure_fp32), and an FP64 one only if the FP64 cycle is ever launched
    if (h->nlev > 1 && h->opt.cycle_prec != AMG_FP32) build_engine<double>(h);
}

int bounds_flags_solve() { return bounds_flag_read_clear(); }

size_t outer_scalar_count(int max_iters) { return OS_ZQ + 2 * (size_t)max_iters + 8; }

void ensure_pinned(amg_hierarchy *h) {
    if (!h->h_pinned)
        AMG_CUDA(cudaMallocHost(&h->h_pinned, (64 + 2 * (size_t)h->opt.max_iters) * sizeof(double)));
}

double cycle_application_bytes(amg_hierarchy *h, int value_bytes) {
    std::vector<Op> prog;
    Builder b{h, &prog, h->nlev + 1};  // every level's ops, down to the coarsest
    b.bhat(0, V_RHS, V_E);
    double s = 0.0;
    for (const Op &op : prog)
        if (op.kind != OP_NOP) s += op_bytes(h, op, value_bytes);
    return s;
}

size_t level_table_image(amg_hierarchy *h, bool fp32, std::vector<unsigned char> &out) {
    auto put = [&](const auto &tab) {
        const size_t b = sizeof(tab[0]) * tab.size();
        out.resize(b);
        std::memcpy(out.data(), tab.data(), b);
        return b;
    };
    if (fp32) {
        std::vector<GLev<float>> tab;
        table_image<float>(h, tab);
        return put(tab);
    }
    std::vector<GLev<double>> tab;
    table_image<double>(h, tab);
    return put(tab);
}

void free_engines(amg_hierarchy *h) {
    delete h->eng64;
    delete h->eng32;
    h->eng64 = h->eng32 = nullptr;
}

int ensure_directions(amg_hierarchy *h, int count) {
    const int n = (int)h->N;
    const int chunk = 16;
    int old = (int)h->P.size();
    if (count <= old) return old;
    int target = std::min(h->opt.max_iters, ((count + chunk - 1) / chunk) * chunk);
    // the new P and Q vectors in one allocation (each 256-byte aligned); if it fails, P and
    // Q keep their length
    const size_t stride = ((size_t)n + 31) & ~(size_t)31, m = (size_t)(target - old);
    double *slab = halloc<double>(h, 2 * m * stride);
    for (size_t j = 0; j < m; j++) {
        h->P.push_back(slab + j * stride);
        h->Q.push_back(slab + (m + j) * stride);
    }
    AMG_CUDA(cudaMemcpyAsync(h->dP, h->P.data(), sizeof(double *) * target, cudaMemcpyHostToDevice,
                             h->stream));
    AMG_CUDA(cudaMemcpyAsync(h->dQ, h->Q.data(), sizeof(double *) * target, cudaMemcpyHostToDevice,
                             h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));  // the tables are copied from host vectors
    return target;
}

static GLev<double> fine_view(amg_hierarchy *h) {
    GLev<double> L;
    std::memset(&L, 0, sizeof L);
    Level &lv = h->lev[0];
    L.n = lv.n;
    L.w = lv.A.uw;
    L.sl = lv.A.sl_ptr;
    L.col = lv.A.col;
    L.val = lv.A.val;
    return L;
}

// the cycle kernel's error flag, read by the caller
static void raise_device_error(amg_hierarchy *h, int err) {
    if (err & kErrTimeout) {
        // the kernel left its op loop: clear the flag and the barrier state for the next launch
        AMG_CUDA(cudaMemsetAsync(h->err_flag, 0, sizeof(int), h->stream));
        AMG_CUDA(cudaMemsetAsync(h->bar, 0, sizeof(unsigned long long), h->stream));
        AMG_CUDA(cudaStreamSynchronize(h->stream));
        throw Error{AMG_ERR_TIMEOUT, "a grid barrier of the cycle kernel timed out"};
    }
}

static void check_device_error(amg_hierarchy *h) {
    int err = 0;
    AMG_CUDA(cudaMemcpyAsync(&err, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));
    raise_device_error(h, err);
}

// one application of B^_0 to h->ro (FP64) into h->zo (FP64)
// out = B^_0 [in] (FP64 vectors; in = h->ro, out = h->zo unless given: the FGMRES basis
// passes its vectors directly)
static void apply_preconditioner(amg_hierarchy *h, const double *in = nullptr,
                                 double *out = nullptr) {
    cudaStream_t s = h->stream;
    const int n = (int)h->N;
    if (!in) in = h->ro;
    if (!out) out = h->zo;
    if (h->nlev == 1) {  // exact solve on the only level (table vectors ro -> zo)
        if (in != h->ro)
            AMG_CUDA(cudaMemcpyAsync(h->ro, in, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        Op op = Builder::mk(OP_COARSE, 0);
        RedCtx rc{h->red_partials, h->red_counter};
        k_op<double><<<1, kRedThreads, 0, s>>>(dtab<double>(h), op, rc);
        AMG_LAUNCH_CHECK();
        if (out != h->zo)
            AMG_CUDA(cudaMemcpyAsync(out, h->zo, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        return;
    }
    if (h->opt.cycle_prec == AMG_FP32) {
        k_convert<double, float><<<nblocks_for(n, 256), 256, 0, s>>>(n, in, h->r32);
        AMG_LAUNCH_CHECK();
        launch_cycle<float>(h);
        k_convert<float, double><<<nblocks_for(n, 256), 256, 0, s>>>(n, h->z32, out);
        AMG_LAUNCH_CHECK();
    } else {
        launch_cycle<double>(h, const_cast<double *>(in), out);
    }
}

static int solve_fgmres(amg_hierarchy *h, const double *b_nat, double tol, double *x_nat,
                        int *iters, double *relres);

int solve(amg_hierarchy *h, const double *b_nat, double tol, double *x_nat, int *iters,
          double *relres) {
    ensure_pinned(h);  // a hierarchy of the batched setup allocates it here
    if (h->opt.outer == AMG_OUTER_FGMRES) return solve_fgmres(h, b_nat, tol, x_nat, iters, relres);
    cudaStream_t s = h->stream;
    const int n = (int)h->N;
    const int maxit = h->opt.max_iters;
    Level &F = h->lev[0];
    RedCtx rc{h->red_partials, h->red_counter};
    const bool prof = profiling(h);
    if (h->opt.cycle_prec == AMG_FP32 && h->nlev > 1) ensure_fp32(h);
    // x = 0, r = b (pi order)
    k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, F.nat, b_nat, h->bo);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaMemcpyAsync(h->ro, h->bo, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    AMG_CUDA(cudaMemsetAsync(h->xo, 0, sizeof(double) * n, s));
    AMG_CUDA(cudaMemsetAsync(h->osc, 0, sizeof(double) * 8, s));
    AMG_CUDA(cudaMemsetAsync(h->oit, 0, sizeof(int), s));
    k_norm2<<<red_grid(n), kRedThreads, 0, s>>>(n, h->bo, h->osc + OS_BB, rc);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaMemcpyAsync(h->h_pinned, h->osc, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    const double bn = std::sqrt(h->h_pinned[OS_BB]);
    int status = AMG_ERR_NOT_CONVERGED;
    int it = 0;
    double rel = 1.0;
    if (!std::isfinite(bn)) throw Error{AMG_ERR_INVALID_ARG, "non-finite right-hand side"};
    if (bn == 0.0) {
        status = AMG_OK;
        rel = 0.0;
    } else {
        double *opq = h->osc + OS_ZQ + maxit;
        GLev<double> Lf = fine_view(h);
        const double nd = n, nnz = (double)F.A.stored;
        for (it = 0; it < maxit;) {
            ensure_directions(h, it + 1);
            apply_preconditioner(h);  // zo = B^[ro]
            Profiler::Rec rec{};
            if (prof) rec = h->prof->begin(K_OUTER_MULTIDOT, 0, 8.0 * nd * (1 + it), s);
            k_outer_multidot<<<red_grid(n), kRedThreads, 0, s>>>(n, h->zo, h->dQ, h->oit, h->osc, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s);
            if (prof) rec = h->prof->begin(K_OUTER_ORTH, 0, 8.0 * nd * (2 + it), s);
            k_outer_orth<<<nblocks_for(n, 256), 256, 0, s>>>(n, h->zo, h->dP, h->oit, h->osc, opq);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s);
            if (prof) rec = h->prof->begin(K_OUTER_SPMV_DOT, 0, 12.0 * nnz + 24.0 * nd, s);
            k_outer_spmv_dot<<<red_grid(n), kRedThreads, 0, s>>>(Lf, h->dP, h->dQ, h->oit, h->ro,
                                                                 h->osc, opq, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s);
            if (prof) rec = h->prof->begin(K_OUTER_UPDATE, 0, 48.0 * nd, s);
            k_outer_update<<<red_grid(n), kRedThreads, 0, s>>>(n, h->dP, h->dQ, h->oit, h->xo,
                                                               h->ro, h->osc, opq, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s);
            k_bump<<<1, 32, 0, s>>>(h->oit);
            AMG_LAUNCH_CHECK();
            AMG_CUDA(cudaMemcpyAsync(h->h_pinned, h->osc, sizeof(double) * 8,
                                     cudaMemcpyDeviceToHost, s));
            AMG_CUDA(cudaStreamSynchronize(s));
            if (h->nlev > 1) check_device_error(h);
            if (prof) {
                h->prof->harvest();
                if (h->nlev > 1) {
                    if (h->opt.cycle_prec == AMG_FP32) harvest_cycle_timestamps<float>(h);
                    else harvest_cycle_timestamps<double>(h);
                }
            }
            it++;
            if (h->h_pinned[OS_STOP] != 0.0) {
                status = AMG_ERR_BREAKDOWN;
                break;
            }
            rel = std::sqrt(h->h_pinned[OS_RR]) / bn;
            if (!std::isfinite(rel)) {
                status = AMG_ERR_BREAKDOWN;
                break;
            }
            if (rel <= tol) {
                k_true_residual<<<red_grid(n), kRedThreads, 0, s>>>(Lf, h->bo, h->xo, h->to,
                                                                    h->osc + OS_TT, rc);
                AMG_LAUNCH_CHECK();
                AMG_CUDA(cudaMemcpyAsync(h->h_pinned, h->osc, sizeof(double) * 8,
                                         cudaMemcpyDeviceToHost, s));
                AMG_CUDA(cudaStreamSynchronize(s));
                rel = std::sqrt(h->h_pinned[OS_TT]) / bn;
                if (rel <= tol) {
                    status = AMG_OK;
                    break;
                }
                AMG_CUDA(cudaMemcpyAsync(h->ro, h->to, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            }
        }
        if (status != AMG_OK) {
            k_true_residual<<<red_grid(n), kRedThreads, 0, s>>>(Lf, h->bo, h->xo, h->to,
                                                                h->osc + OS_TT, rc);
            AMG_LAUNCH_CHECK();
            AMG_CUDA(cudaMemcpyAsync(h->h_pinned, h->osc, sizeof(double) * 8,
                                     cudaMemcpyDeviceToHost, s));
            AMG_CUDA(cudaStreamSynchronize(s));
            rel = std::sqrt(h->h_pinned[OS_TT]) / bn;
        }
    }
    k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, F.nat, h->xo, x_nat);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = rel;
    return status;
}


// Restarted flexible GMRES(m) (right preconditioning, FP64 basis and Hessenberg matrix,
// classical Gram-Schmidt applied twice): the outer iteration for a preconditioner that
// varies between applications (the nonlinear AMLI-cycle, in FP32 or FP64). The host keeps the
// (m+1) x m Hessenberg matrix and its Givens rotations; each iteration reads m+2 scalars.
static int solve_fgmres(amg_hierarchy *h, const double *b_nat, double tol, double *x_nat,
                        int *iters, double *relres) {
    cudaStream_t s = h->stream;
    const int n = (int)h->N;
    const int maxit = h->opt.max_iters;
    const int m = std::max(1, std::min(h->opt.fgmres_restart, maxit));
    Level &F = h->lev[0];
    RedCtx rc{h->red_partials, h->red_counter};
    if (h->opt.cycle_prec == AMG_FP32 && h->nlev > 1) ensure_fp32(h);
    // basis V[0..m], preconditioned directions Z[0..m-1] (the outer direction store)
    ensure_directions(h, std::min(maxit, std::max(2 * m + 1, 1)));
    if ((int)h->P.size() < 2 * m + 1) throw Error{AMG_ERR_UNSUPPORTED, "max_iters too small for the restart length"};
    double **dV = h->dP;          // V[i] = P[i], i <= m
    double **dZ = h->dP + m + 1;  // Z[j] = P[m + 1 + j]
    double *w = h->to;
    double *dh = h->osc + OS_ZQ;           // first pass's dots and the norm: m + 2 scalars
    double *dh2 = h->osc + OS_ZQ + m + 2;  // second pass's dots: m + 1 (maxit >= 2m + 1)
    GLev<double> Lf = fine_view(h);
    k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, F.nat, b_nat, h->bo);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaMemsetAsync(h->xo, 0, sizeof(double) * n, s));
    k_norm2<<<red_grid(n), kRedThreads, 0, s>>>(n, h->bo, h->osc + OS_BB, rc);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaMemcpyAsync(h->h_pinned, h->osc, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    const double bn = std::sqrt(h->h_pinned[OS_BB]);
    if (!std::isfinite(bn)) throw Error{AMG_ERR_INVALID_ARG, "non-finite right-hand side"};
    int it = 0, status = AMG_ERR_NOT_CONVERGED;
    double rel = 1.0;
    const bool prof = profiling(h);
    const double nd = n, nnzf = (double)F.A.stored;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    std::vector<double> hv(std::max(m + 2, 8));
    double *dy = h->osc + OS_ZQ + maxit + 4;  // coefficients for the update (m <= maxit)
    auto read_scalars = [&](const double *d, int count, double *out) {
        AMG_CUDA(cudaMemcpyAsync(h->h_pinned, d, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < count; k++) out[k] = h->h_pinned[k];
    };
    if (bn == 0.0) {
        status = AMG_OK;
        rel = 0.0;
    }
    // r = b - A x (x = 0 at the start)
    AMG_CUDA(cudaMemcpyAsync(h->ro, h->bo, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double beta = bn;
    while (status != AMG_OK && it < maxit) {
        // V[0] = r / beta
        k_scale<<<nblocks_for(n, 256), 256, 0, s>>>(n, h->ro, 1.0 / beta, h->P[0]);
        AMG_LAUNCH_CHECK();
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        bool done = false;
        for (; j < m && it < maxit; j++) {
            // Z[j] = B^[V[j]]
            apply_preconditioner(h, h->P[j], h->P[m + 1 + j]);
            // w = A Z[j], orthogonalised twice against V[0..j]
            Profiler::Rec rec{};
            if (prof) rec = h->prof->begin(K_FGMRES_SPMV, 0, 12.0 * nnzf + 16.0 * nd, s);
            k_spmv<<<nblocks_for(n, 256), 256, 0, s>>>(Lf, h->P[m + 1 + j], w);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s);
            // classical Gram-Schmidt twice: h1 = V^t w, w -= V h1, h2 = V^t w, w -= V h2
            if (prof) rec = h->prof->begin(K_FGMRES_MDOT, 0, 8.0 * nd * (j + 2), s);
            k_mdot<<<red_grid(n), kRedThreads, 0, s>>>(n, w, dV, j + 1, dh, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s);
            if (prof) rec = h->prof->begin(K_FGMRES_ORTH, 0, 8.0 * nd * (j + 3), s);
            k_orth_mdot<<<red_grid(n), kRedThreads, 0, s>>>(n, w, dV, j + 1, dh, dh2, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s);
            if (prof) rec = h->prof->begin(K_FGMRES_ORTH, 0, 8.0 * nd * (j + 3), s);
            k_orth_sub<<<red_grid(n), kRedThreads, 0, s>>>(n, w, dV, j + 1, dh2, dh + j + 1, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s);
            {  // h1, the norm, h2 and the cycle's error flag: one round trip
                int err = 0;
                AMG_CUDA(cudaMemcpyAsync(h->h_pinned, dh, sizeof(double) * (j + 2),
                                         cudaMemcpyDeviceToHost, s));
                AMG_CUDA(cudaMemcpyAsync(h->h_pinned + m + 2, dh2, sizeof(double) * (j + 1),
                                         cudaMemcpyDeviceToHost, s));
                if (h->nlev > 1)
                    AMG_CUDA(cudaMemcpyAsync(&err, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
                AMG_CUDA(cudaStreamSynchronize(s));
                raise_device_error(h, err);
                for (int i = 0; i < j + 2; i++) hv[i] = h->h_pinned[i];
                for (int i = 0; i <= j; i++)
                    H[(size_t)i * m + j] = (0.0 + hv[i]) + h->h_pinned[m + 2 + i];
            }
            if (prof) {
                h->prof->harvest();
                if (h->nlev > 1) {
                    if (h->opt.cycle_prec == AMG_FP32) harvest_cycle_timestamps<float>(h);
                    else harvest_cycle_timestamps<double>(h);
                }
            }
            it++;
            const double hn = std::sqrt(hv[j + 1]);
            H[(size_t)(j + 1) * m + j] = hn;
            // apply the previous rotations to column j, then a new one
            for (int i = 0; i < j; i++) {
                double a = H[(size_t)i * m + j], b2 = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b2;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b2;
            }
            double a = H[(size_t)j * m + j], b2 = H[(size_t)(j + 1) * m + j];
            double r = std::hypot(a, b2);
            if (!(r > 0.0) || !std::isfinite(r)) {
                status = AMG_ERR_BREAKDOWN;
                done = true;
                break;
            }
            cs[j] = a / r;
            sn[j] = b2 / r;
            H[(size_t)j * m + j] = r;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            rel = std::fabs(g[j + 1]) / bn;
            if (rel <= tol) {
                j++;
                done = true;
                break;
            }
            if (hn > 0.0) {
                k_scale<<<nblocks_for(n, 256), 256, 0, s>>>(n, w, 1.0 / hn, h->P[j + 1]);
                AMG_LAUNCH_CHECK();
            } else {  // exact solution in the Krylov space
                j++;
                done = true;
                break;
            }
        }
        const int k = std::min(j, m);
        // y = H(0:k,0:k)^{-1} g(0:k); x += Z y
        for (int i = k - 1; i >= 0; i--) {
            double acc = g[i];
            for (int l = i + 1; l < k; l++) acc -= H[(size_t)i * m + l] * y[l];
            y[i] = acc / H[(size_t)i * m + i];
        }
        if (k > 0) {
            std::memcpy(h->h_pinned, y.data(), sizeof(double) * k);
            AMG_CUDA(cudaMemcpyAsync(dy, h->h_pinned, sizeof(double) * k, cudaMemcpyHostToDevice, s));
            k_lincomb<<<nblocks_for(n, 256), 256, 0, s>>>(n, h->xo, dZ, k, dy);
            AMG_LAUNCH_CHECK();
        }
        // true residual r = b - A x
        k_true_residual<<<red_grid(n), kRedThreads, 0, s>>>(Lf, h->bo, h->xo, h->ro, h->osc + OS_TT, rc);
        AMG_LAUNCH_CHECK();
        read_scalars(h->osc, 8, hv.data());
        beta = std::sqrt(hv[OS_TT]);
        rel = beta / bn;
        if (rel <= tol) status = AMG_OK;
        else if (status == AMG_ERR_BREAKDOWN) break;
        (void)done;
    }
    k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, F.nat, h->xo, x_nat);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = rel;
    return status;
}

// z = B^_level [f] in natural order (FP64). Level 0 runs the persistent kernel exactly as the
// solve does; coarser levels run the standalone executor (one kernel per op).
void apply_cycle_level(amg_hierarchy *h, int level, const double *f_nat, double *z_nat) {
    cudaStream_t s = h->stream;
    Level &lv = h->lev[level];
    const int n = lv.n;
    RedCtx rc{h->red_partials, h->red_counter};
    if (lv.coarsest) {
        double *fbuf = level == 0 ? h->ro : lv.v64.rhs;
        double *ebuf = level == 0 ? h->zo : lv.v64.e;
        k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, f_nat, fbuf);
        AMG_LAUNCH_CHECK();
        Op op = Builder::mk(OP_COARSE, level);
        k_op<double><<<1, kRedThreads, 0, s>>>(dtab<double>(h), op, rc);
        AMG_LAUNCH_CHECK();
        k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, ebuf, z_nat);
        AMG_LAUNCH_CHECK();
        AMG_CUDA(cudaStreamSynchronize(s));
        return;
    }
    if (level == 0) {  // the solve's preconditioner, in the configured cycle precision
        if (h->opt.cycle_prec == AMG_FP32) ensure_fp32(h);
        k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, f_nat, h->ro);
        AMG_LAUNCH_CHECK();
        apply_preconditioner(h);
        k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, h->zo, z_nat);
        AMG_LAUNCH_CHECK();
        AMG_CUDA(cudaStreamSynchronize(s));
        check_device_error(h);
        return;
    }
    k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, f_nat, lv.v64.rhs);
    AMG_LAUNCH_CHECK();
    run_standalone<double>(h, level, V_RHS, V_P0);
    k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, lv.v64.p[0], z_nat);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(s));
}

// one sweep of the coloured smoother on `level`, natural order in/out (FP64)
void smooth_level(amg_hierarchy *h, int level, int backward, const double *f_nat, double *u_nat) {
    cudaStream_t s = h->stream;
    Level &lv = h->lev[level];
    const int n = lv.n;
    double *fbuf = level == 0 ? h->ro : lv.v64.rhs;
    double *ubuf = level == 0 ? h->zo : lv.v64.e;
    k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, f_nat, fbuf);
    k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, u_nat, ubuf);
    AMG_LAUNCH_CHECK();
    const std::vector<int> &ranges = (level == 0) ? lv.color_blocks : lv.color_rows;
    const int nc = (int)ranges.size() - 1;
    RedCtx rc{h->red_partials, h->red_counter};
    for (int k = 0; k < nc; k++) {
        int c = backward ? nc - 1 - k : k;
        if (ranges[c + 1] == ranges[c]) continue;
        Op g = Builder::mk(OP_GS, level);
        g.i0 = ranges[c];
        g.i1 = ranges[c + 1];
        g.backward = backward;
        g.fsel = V_RHS;
        g.usel = V_E;
        Builder{h, nullptr, h->nlev}.big_range(level, c, g);
        k_op<double><<<nblocks_for(g.i1 - g.i0, kRedThreads), kRedThreads, 0, s>>>(dtab<double>(h), g, rc);
        AMG_LAUNCH_CHECK();
    }
    k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, ubuf, u_nat);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace amg
