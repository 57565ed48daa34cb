// Batched solves: many independent systems of uneven sizes, each with its own hierarchy
// (built by the single-system setup), solved by one persistent kernel.
//
// The paper solves one system at a time. A batch of small and mid-size systems would leave
// the GPU almost idle if each ran the grid-wide cycle kernel in turn (those solves are
// latency-bound: a few thousand dependent steps, each a grid barrier). Here every CTA takes
// the next slot from a queue (largest systems first) and runs that system's whole solve: the
// outer flexible CG (Alg. 1 on the finest level, FP64, full orthogonalisation, restarted
// after `cap` directions) and, every iteration, the AMLI-cycle B^_0 (Alg. 2, with Alg. 1 on
// the coarse levels and the exact coarsest solve) on levels that stay in HBM / L2. The cycle
// ops are the same device functions as the single-system kernel (cycle_ops.cuh) on the same
// level data, walked as a state machine over the levels.
//
// A system much larger than the batch's average work per CTA would alone set the batch's
// time, so it may be solved by a team of K CTAs (K slots in a row at the head of the queue):
// the team splits every op's rows, meets at a bounded barrier on a counter of its own, and
// reduces through per-rank partials summed in rank order (the same bits in every member).
// Team slots are at most half the grid and come first, so each is taken at once by a running
// CTA, and a CTA holds one slot at a time: no member waits for a CTA that is not running.
//
// Launch shape (threads per CTA, CTAs per SM) is chosen by a small autotuner that times the
// candidate shapes on the batch itself and keeps the fastest; the launch sequence of a solve
// is captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "cycle_ops.cuh"

namespace amg {

template <class T>
using BLev = LevelDev<T, int>;

constexpr int kBatchCap = 64;  // outer directions kept before a restart
constexpr int kMaxTeam = 8;    // CTAs of one team at most
constexpr int kTeamPart = 16 * kMaxTeam;  // doubles of partials per team

// one system of the batch
template <class T>
struct BatchProb {
    int n, nlev;
    int64_t off;                   // first row in the concatenated vectors
    const BLev<T> *tab;            // the system's level table (cycle precision)
    const int *colors;             // colour ranges of every level, concatenated
    int cofs[kMaxLevels];          // level l's ranges start at colors + cofs[l]
    int ncol[kMaxLevels];          // colours of level l (blocks on level 0, rows elsewhere)
    BLev<double> A0;               // finest matrix in FP64 (outer SpMV and true residual)
    const int *nat;                // finest pi-row -> row of the system
    double *bo, *xo, *ro, *zo, *to;  // outer vectors (pi order), FP64
    double *P, *Q;                 // kBatchCap directions and their images, n each
};

// ---------------------------------------------------------------------------------------
// the team of CTAs that solves the current system (a team of one is a single CTA)
struct Team {
    int K, rank;
    unsigned long long *bar;   // the team's barrier counter (zeroed before every launch)
    double *part;              // outer sums [2][4][K], then the cycle reductions [4][K]
    unsigned int *cnt;         // arrivals of the cycle's reductions (RM_TEAM)
    unsigned long long target;
    unsigned long long limit_ns;  // wait limit of the team barrier
    int parity;                // buffer of the next outer sum
    int abort;                 // a barrier wait ran out: no further waits
};
__shared__ Team bt_team;

// thread 0: arrive at the team's barrier and wait for the other members, bounded like the
// grid barrier (kBarrierLimitNs); out of line, as the one-CTA path never takes it
__device__ __noinline__ void team_wait() {
    if (bt_team.abort) return;
    bt_team.target += bt_team.K;
    red_release_add_u64(bt_team.bar, 1ull);
    unsigned long long t0 = 0;
    int spins = 0;
    while (ld_acquire_u64(bt_team.bar) < bt_team.target) {
        if ((++spins & 1023) == 0) {
            if (t0 == 0) {
                t0 = global_ns();
            } else if (global_ns() - t0 > bt_team.limit_ns) {
                bt_team.abort = 1;
                return;
            }
        }
    }
}

// every thread of every CTA of the team
__device__ __forceinline__ void team_sync() {
    __syncthreads();
    if (bt_team.K > 1) {
        if (threadIdx.x == 0) team_wait();
        __syncthreads();
    }
}

// r[k] = sum of v[k] over the team, returned to every thread: block sums, then (teams) the
// per-rank partials summed in rank order after the team barrier. Ends with a CTA barrier.
template <int NV>
__device__ __forceinline__ void team_sum(const double (&v)[NV], double (&r)[NV]) {
    __shared__ double bc[4];
    double s[NV];
    block_sum<NV, double>(v, s, BlockGroup{});
    if (bt_team.K == 1) {
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; k++) bc[k] = s[k];
        __syncthreads();
    } else {
        const int K = bt_team.K;
        double *part = bt_team.part + bt_team.parity * 4 * K;
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; k++) part[k * K + bt_team.rank] = s[k];
        team_sync();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < NV; k++) {
                double y = 0.0;
                for (int b = 0; b < K; b++) y += __ldcg(&part[k * K + b]);
                bc[k] = y;
            }
            bt_team.parity ^= 1;  // two buffers: a member may start the next sum at once
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < NV; k++) r[k] = bc[k];
    __syncthreads();  // bc and the reduction scratch are reused by the next call
}

__device__ __forceinline__ double team_sum1(double v) {
    const double a[1] = {v};
    double r[1];
    team_sum<1>(a, r);
    return r[0];
}

// this thread's row stride over the team, and the reduction context of the cycle's ops
__device__ __forceinline__ int team_tid() { return bt_team.rank * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int team_nth() { return bt_team.K * blockDim.x; }
__device__ __forceinline__ RedCtx team_rc() {
    RedCtx rc{bt_team.part + 8 * bt_team.K, bt_team.cnt};
    rc.rank = bt_team.rank;
    rc.size = bt_team.K;
    return rc;
}

__device__ __forceinline__ Op batch_op() {
    Op o;
    memset(&o, 0, sizeof o);
    o.red_pb = -1;
    o.fin_pb = -1;
    return o;
}

// ---------------------------------------------------------------------------------------
// the cycle on one system: z = B^_0 [rhs] on level 0's cycle vectors (tab[0].rhs -> tab[0].e)

template <class T>
struct BatchCycle {
    const BLev<T> *tab;  // shared-memory copy of the level table
    const int *colors;
    const int *cofs, *ncol;
    int nlev, kc;
    int nu_pre, nu_post;  // smoothing sweeps
};

// first non-empty colour [r0, r1) of level l >= 1
template <class T>
__device__ __forceinline__ void first_colour(const BatchCycle<T> &c, int l, int &r0, int &r1) {
    const int *cr = c.colors + c.cofs[l];
    const int nc = c.ncol[l];
    int k = 0;
    while (k < nc && cr[k + 1] == cr[k]) k++;
    r0 = k < nc ? cr[k] : 0;
    r1 = k < nc ? cr[k + 1] : 0;
}

// pre-smoothing and restriction of B^_l: level 0 from u = 0 (block smoother, all colours);
// coarse levels for z = p_i, f = rhs (i = 0) or r, the first non-empty colour as u = D^-1 f
template <class T>
__device__ __forceinline__ void bc_pre(const BatchCycle<T> &c, int l, int i) {
    const BLev<T> &L = c.tab[l];
    const int tid = team_tid(), nth = team_nth();
    const int *cr = c.colors + c.cofs[l];
    const int nc = c.ncol[l];
    const T *f = (l == 0 || i == 0) ? L.rhs : L.r;
    T *z = l == 0 ? L.e : pick(L.p, i);
    Op op = batch_op();
    int col = 0;
    if (l == 0) {
        op_zero(L, z, tid, nth);
        team_sync();
    } else {  // the first colour was done by the restriction into this level or the last UPDATE
        while (col < nc && cr[col + 1] == cr[col]) col++;
        col++;
    }
    // the first sweep's remaining colours, then nu_pre - 1 further forward sweeps
    for (int sw = 0, c1 = col; sw < c.nu_pre; sw++, c1 = 0)
        for (col = c1; col < nc; col++) {
            if (cr[col + 1] == cr[col]) continue;
            op.i0 = cr[col];
            op.i1 = cr[col + 1];
            op_gs(L, op, f, z, tid, nth);
            team_sync();
        }
    const BLev<T> &N = c.tab[l + 1];
    if (l + 1 < c.nlev - 1) {  // the next level smooths: its first colour from zero too
        int f0, f1;
        first_colour(c, l + 1, f0, f1);
        op_restrict(L, f, z, N.rhs, tid, nth, N.p[0], N.dinv, f0, f1);
    } else {
        op_restrict(L, f, z, N.rhs, tid, nth);
    }
    team_sync();
}

// prolongation and post-smoothing of B^_l; on coarse levels then Alg. 1 step i
template <class T>
__device__ __forceinline__ void bc_post(const BatchCycle<T> &c, int l, int i) {
    const BLev<T> &L = c.tab[l];
    const int tid = team_tid(), nth = team_nth();
    const int *cr = c.colors + c.cofs[l];
    const T *f = (l == 0 || i == 0) ? L.rhs : L.r;
    T *z = l == 0 ? L.e : pick(L.p, i);
    op_prolong(L, c.tab[l + 1].e, z, tid, nth);
    team_sync();
    Op op = batch_op();
    op.backward = 1;
    for (int sw = 0; sw < c.nu_post; sw++)
        for (int col = c.ncol[l] - 1; col >= 0; col--) {
            if (cr[col + 1] == cr[col]) continue;
            op.i0 = cr[col];
            op.i1 = cr[col + 1];
            op_gs(L, op, f, z, tid, nth);
            team_sync();
        }
    if (l == 0) return;
    const RedCtx rc = team_rc();
    op = batch_op();
    op.step = i;
    op.last = (i == c.kc - 1);
    if (!op.last) {  // the UPDATE also starts step i+1's pre-smoothing
        op.fuse = 1;
        first_colour(c, l, op.f0, op.f1);
    }
    if (i > 0) {
        op_multidot<BLev<T>, RM_TEAM>(L, op, rc, tid, nth, BlockGroup{});
        team_sync();
        op_orth(L, op, tid, nth, BlockGroup{});
        team_sync();
    }
    op_spmv_dot<BLev<T>, RM_TEAM>(L, op, rc, tid, nth, BlockGroup{});
    team_sync();
    op_update<BLev<T>, RM_TEAM>(L, op, rc, tid, nth, BlockGroup{});
    team_sync();
}

// B^_0 over the whole hierarchy: the recursion of Alg. 2 / Alg. 1 as a state machine (the
// same walk as the shared-memory tail of the single-system kernel, from level 0)
template <class T>
__device__ void batch_cycle(const BatchCycle<T> &c) {
    if (c.nlev == 1) {  // the only level is the coarsest: exact solve
        op_coarse(c.tab[0], team_tid(), team_nth());
        team_sync();
        return;
    }
    enum { ENTER, PRE, POST };
    int step[kMaxLevels] = {};
    int l = 0, ph = PRE;
    for (;;) {
        const bool coarsest = (l == c.nlev - 1);
        const int i = step[l];
        if (l > 0 && ph == ENTER && coarsest) {
            op_coarse(c.tab[l], team_tid(), team_nth());
            team_sync();
        } else if (ph == PRE) {
            bc_pre(c, l, i);
        } else if (ph == POST) {
            bc_post(c, l, i);
        }
        if (l == 0) {
            if (ph == POST) break;
            l = 1;  // PRE done: B~_1
            ph = ENTER;
            continue;
        }
        if (ph == ENTER && !coarsest) {
            step[l] = 0;
            ph = PRE;
            continue;
        }
        if (ph == PRE) {
            l++;
            ph = ENTER;
            continue;
        }
        if (ph == POST && i + 1 < c.kc) {
            step[l] = i + 1;
            ph = PRE;
            continue;
        }
        l--;  // B~_l done: back to B^_{l-1}
        ph = POST;
    }
}

// ---------------------------------------------------------------------------------------
// the outer iteration of one system (flexible CG with full orthogonalisation, FP64)

// t = b - A x on the team's rows, returns (t, t) over the system
__device__ __forceinline__ double true_residual(const BLev<double> &A, const double *b,
                                                const double *x, double *t) {
    double s = 0.0;
    for (int i = team_tid(), nth = team_nth(); i < A.n; i += nth) {
        const double ri = row_residual(A, i, b, x);
        t[i] = ri;
        s += ri * ri;
    }
    return team_sum1(s);
}

template <class T>
__device__ void solve_one(const BatchProb<T> &P, const BatchCycle<T> &cyc, const double *b,
                          double *x, double tol, int maxit, int *iters, double *relres,
                          int *status, int slot) {
    const int n = P.n;  // every row loop: from team_tid() in steps of team_nth()
    double *bo = P.bo, *xo = P.xo, *ro = P.ro, *zo = P.zo, *to = P.to;
    T *crhs = cyc.tab[0].rhs, *ce = cyc.tab[0].e;
    // (z, q_j) and (p_j, q_j) of the kept directions, held by every CTA of the team, and
    // their quotients (divided once per step, not per row: FP64 division is long here)
    __shared__ double zq[kBatchCap], pqh[kBatchCap], cq[kBatchCap];
    double bb = 0.0;
    for (int i = team_tid(), nth = team_nth(); i < n; i += nth) {
        const double v = b[P.off + P.nat[i]];
        bo[i] = v;
        ro[i] = v;
        xo[i] = 0.0;
        bb += v * v;
    }
    bb = team_sum1(bb);  // (its barrier also orders the writes above)
    const double bn = sqrt(bb);
    int st = AMG_ERR_NOT_CONVERGED, it = 0, k = 0;
    double rel = 1.0;
    if (!isfinite(bn)) {
        st = AMG_ERR_INVALID_ARG;
    } else if (bn == 0.0) {
        st = AMG_OK;
        rel = 0.0;
    } else {
        while (it < maxit) {
            // z = B^_0 [r] in the cycle precision
            if ((const void *)crhs != (const void *)ro)
                for (int i = team_tid(), nth = team_nth(); i < n; i += nth) crhs[i] = (T)ro[i];
            team_sync();
            batch_cycle(cyc);
            if ((const void *)ce != (const void *)zo)
                for (int i = team_tid(), nth = team_nth(); i < n; i += nth) zo[i] = (double)ce[i];
            team_sync();
            // (z, q_j), j < k
            double *pk = P.P + (size_t)k * n, *qk = P.Q + (size_t)k * n;
            for (int j0 = 0; j0 < k; j0 += 4) {
                double v[4] = {0.0, 0.0, 0.0, 0.0}, r[4];
                for (int i = team_tid(), nth = team_nth(); i < n; i += nth) {
                    const double zi = zo[i];
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if (j0 + j < k) v[j] += zi * P.Q[(size_t)(j0 + j) * n + i];
                }
                team_sum<4>(v, r);
                if (threadIdx.x == 0)
                    for (int j = 0; j < 4 && j0 + j < k; j++) zq[j0 + j] = r[j];
            }
            __syncthreads();
            for (int j = threadIdx.x; j < k; j += blockDim.x) cq[j] = zq[j] / pqh[j];
            __syncthreads();
            // p_k = z - sum_j (z, q_j) / (p_j, q_j) p_j
            for (int i = team_tid(), nth = team_nth(); i < n; i += nth) {
                double acc = zo[i];
                for (int j = 0; j < k; j++) acc -= cq[j] * P.P[(size_t)j * n + i];
                pk[i] = acc;
            }
            team_sync();
            // q_k = A p_k, (p_k, q_k), (r, p_k)
            double v2[2] = {0.0, 0.0}, r2[2];
            for (int i = team_tid(), nth = team_nth(); i < n; i += nth) {
                int base, width;
                row_span(P.A0, i, base, width);
                const double qi = row_dot(P.A0, base, 0, width, pk);
                qk[i] = qi;
                v2[0] += pk[i] * qi;
                v2[1] += ro[i] * pk[i];
            }
            team_sum<2>(v2, r2);
            const double pq = r2[0], rp = r2[1];
            if (threadIdx.x == 0) pqh[k] = pq;  // read after later barriers only
            if (!(pq > 0.0) || !isfinite(pq)) {
                st = AMG_ERR_BREAKDOWN;
                break;
            }
            const double alpha = rp / pq;
            double rr = 0.0;
            for (int i = team_tid(), nth = team_nth(); i < n; i += nth) {
                xo[i] += alpha * pk[i];
                const double rn = ro[i] - alpha * qk[i];
                ro[i] = rn;
                rr += rn * rn;
            }
            rr = team_sum1(rr);
            it++;
            k++;
            rel = sqrt(rr) / bn;
            if (!isfinite(rel)) {
                st = AMG_ERR_BREAKDOWN;
                break;
            }
            if (rel <= tol) {  // confirm with the true residual
                rel = sqrt(true_residual(P.A0, bo, xo, to)) / bn;
                if (rel <= tol) {
                    st = AMG_OK;
                    break;
                }
                for (int i = team_tid(), nth = team_nth(); i < n; i += nth) ro[i] = to[i];
                team_sync();
            }
            if (k == kBatchCap) {  // restart from the true residual
                true_residual(P.A0, bo, xo, ro);
                k = 0;
            }
            if (bt_team.abort) break;  // a member stopped answering: no result
        }
        if (st != AMG_OK && st != AMG_ERR_INVALID_ARG) rel = sqrt(true_residual(P.A0, bo, xo, to)) / bn;
    }
    for (int i = team_tid(), nth = team_nth(); i < n; i += nth) x[P.off + P.nat[i]] = xo[i];
    if (bt_team.abort) st = AMG_ERR_TIMEOUT;
    if (bt_team.rank == 0 && threadIdx.x == 0) {
        iters[slot] = it;
        relres[slot] = rel;
        status[slot] = st;
    }
    __syncthreads();
}

// every CTA: take the next slot from the queue (largest systems first; the K slots of a team
// in a row) and solve that system, alone or as rank s.y of a team of s.z CTAs
template <class T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_batch(const BatchProb<T> *__restrict__ probs, const int4 *__restrict__ slots, int nslots,
        int *next, int kc, int nu, const double *__restrict__ b, double *__restrict__ x,
        double tol, int maxit, int *iters, double *relres, int *status,
        unsigned long long *t_start, unsigned long long *t_end, unsigned long long *team_bar,
        double *team_part, unsigned int *team_cnt, unsigned long long bar_limit_ns,
        int bar_extra) {
    __shared__ BatchProb<T> sp;
    __shared__ BLev<T> stab[kMaxLevels];
    __shared__ int q;
    for (;;) {
        if (threadIdx.x == 0) q = atomicAdd(next, 1);
        __syncthreads();
        const int mine = q;
        if (mine >= nslots) break;
        const int4 sl = slots[mine];
        const int p = sl.x;
        if (threadIdx.x == 0) {
            bt_team.K = sl.z;
            bt_team.rank = sl.y;
            bt_team.bar = team_bar + p;
            bt_team.part = team_part + (size_t)p * kTeamPart;
            bt_team.cnt = team_cnt + p;
            bt_team.target = (unsigned long long)bar_extra;  // > 0 only under a host-set fault
            bt_team.limit_ns = bar_limit_ns;
            bt_team.parity = 0;
            bt_team.abort = 0;
        }
        {
            const int words = (int)(sizeof(BatchProb<T>) / sizeof(int));
            for (int i = threadIdx.x; i < words; i += blockDim.x)
                ((int *)&sp)[i] = ((const int *)&probs[p])[i];
        }
        __syncthreads();
        {
            const int words = sp.nlev * (int)(sizeof(BLev<T>) / sizeof(int));
            for (int i = threadIdx.x; i < words; i += blockDim.x)
                ((int *)stab)[i] = ((const int *)sp.tab)[i];
        }
        __syncthreads();
        // nu: nu_pre + 256 nu_post
        BatchCycle<T> cyc{stab, sp.colors, sp.cofs, sp.ncol, sp.nlev, kc, nu & 255, nu >> 8};
        if (threadIdx.x == 0 && sl.y == 0) t_start[p] = global_ns();
        solve_one(sp, cyc, b, x, tol, maxit, iters, relres, status, p);
        if (threadIdx.x == 0 && sl.y == 0) t_end[p] = global_ns();
        // (solve_one ends with a barrier: q and bt_team may be overwritten)
    }
}

// ---------------------------------------------------------------------------------------
// host side

struct BatchShape {
    int threads, per_sm;
};
static const BatchShape kShapes[] = {{1024, 1}, {512, 2}, {512, 1}, {256, 4}};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

template <class T>
void *batch_kernel(int shape) {
    switch (shape) {
        case 0: return (void *)k_batch<T, 1024, 1>;
        case 1: return (void *)k_batch<T, 512, 2>;
        case 2: return (void *)k_batch<T, 512, 1>;
        default: return (void *)k_batch<T, 256, 4>;
    }
}

struct BatchEngine {
    std::vector<amg_hierarchy *> hs;  // not owned
    std::vector<int64_t> row_off;
    int nprob = 0;
    int64_t N = 0;
    bool fp32 = false;
    int kc = 2, maxit = 200;
    int nu = 1 + 256;  // nu_pre + 256 nu_post
    // host-set team-barrier fault (amg_debug_batch_barrier_fault): 0 = none
    int64_t dbg_bar_limit_ns = 0;
    int dbg_bar_extra = 0;
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    void *probs = nullptr;  // BatchProb<T>[nprob]
    int *next = nullptr, *iters = nullptr, *status = nullptr;
    std::vector<int> ord;      // queue order: largest system first
    int max_team = 1;          // 0: sized per system; 1: no teams; k: at most k CTAs
    bool tuned = false;        // the shape was chosen by timing (re-timed when teams change)
    int4 *slots[kNumShapes] = {};  // per shape: (system, rank, team size, 0) per queue slot
    int nslots[kNumShapes] = {};
    std::vector<int> team[kNumShapes];  // per shape: team size of every system
    unsigned long long *team_bar = nullptr;  // per system: team barrier counter
    double *team_part = nullptr;             // per system: kTeamPart partials
    unsigned int *team_cnt = nullptr;        // per system: reduction arrivals
    double *relres = nullptr;
    unsigned long long *t_start = nullptr, *t_end = nullptr;  // per system, device clock (ns)
    int shape = -1;            // chosen launch shape (-1: not tuned yet)
    int grid[kNumShapes] = {};
    double tuned_ms[kNumShapes] = {};
    size_t bytes = 0;
    // the solve's launch sequence, captured once per (b, x, tol) binding
    cudaGraphExec_t graph = nullptr;
    const double *g_b = nullptr;
    double *g_x = nullptr;
    double g_tol = -1.0;
    int g_shape = -1;
};

template <class U>
U *balloc(BatchEngine *E, size_t count) {
    void *p = nullptr;
    device_alloc(&p, std::max<size_t>(16, count * sizeof(U)), E->stream);
    E->allocs.push_back(p);
    E->bytes += count * sizeof(U);
    return (U *)p;
}

// the hierarchy's batched-solve workspace, allocated (owned by the hierarchy) on first use
const BatchWs &batch_ws(amg_hierarchy *h) {
    BatchWs &w = h->bws;
    if (w.bo) return w;
    const size_t n = (size_t)h->N;
    w.cap = kBatchCap;
    w.bo = halloc<double>(h, n);
    w.xo = halloc<double>(h, n);
    w.to = halloc<double>(h, n);
    w.P = halloc<double>(h, (size_t)kBatchCap * n);
    w.Q = halloc<double>(h, (size_t)kBatchCap * n);
    std::vector<int> colors;
    for (int l = 0; l < h->nlev; l++) {
        const std::vector<int> &r = (l == 0) ? h->lev[0].color_blocks : h->lev[l].color_rows;
        w.cofs[l] = (int)colors.size();
        w.ncol[l] = std::max(0, (int)r.size() - 1);
        colors.insert(colors.end(), r.begin(), r.end());
    }
    w.colors = halloc<int>(h, colors.size());
    AMG_CUDA(cudaMemcpyAsync(w.colors, colors.data(), sizeof(int) * colors.size(),
                             cudaMemcpyHostToDevice, h->stream));
    AMG_CUDA(cudaStreamSynchronize(h->stream));  // colors is a local
    return w;
}

template <class T>
void build_probs(BatchEngine *E) {
    const int np = E->nprob;
    std::vector<BatchProb<T>> hp(np);
    for (int p = 0; p < np; p++) {
        amg_hierarchy *h = E->hs[p];
        const BatchWs &w = batch_ws(h);
        BatchProb<T> &B = hp[p];
        std::memset(&B, 0, sizeof B);
        B.n = (int)h->N;
        B.nlev = h->nlev;
        B.off = E->row_off[p];
        B.tab = (const BLev<T> *)level_table(h, sizeof(T) == 4);
        B.colors = w.colors;
        for (int l = 0; l < kMaxLevels; l++) {
            B.cofs[l] = w.cofs[l];
            B.ncol[l] = w.ncol[l];
        }
        const Level &F = h->lev[0];
        B.A0.n = F.n;
        B.A0.w = F.A.uw;
        B.A0.sl = F.A.sl_ptr;
        B.A0.col = F.A.col;
        B.A0.val = F.A.val;
        B.nat = F.nat;
        B.bo = w.bo;
        B.xo = w.xo;
        B.ro = h->ro;  // the FP64 cycle's level-0 input and output are the outer r and z
        B.zo = h->zo;
        B.to = w.to;
        B.P = w.P;
        B.Q = w.Q;
    }
    BatchProb<T> *dp = balloc<BatchProb<T>>(E, np);
    AMG_CUDA(cudaMemcpyAsync(dp, hp.data(), sizeof(BatchProb<T>) * np, cudaMemcpyHostToDevice,
                             E->stream));
    E->probs = dp;
    int nsm = 0;
    AMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, E->hs[0]->device));
    for (int s = 0; s < kNumShapes; s++) {
        int per = 0;
        AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<T>(s),
                                                               kShapes[s].threads, 0));
        E->grid[s] = nsm * std::min(per, kShapes[s].per_sm);  // surplus CTAs find no slot
    }
    AMG_CUDA(cudaStreamSynchronize(E->stream));  // hp is a local
}

// Team sizes and the queue of slots for launch shape s. A system gets about as many CTAs as
// its share of the batch's unknowns over the grid's CTAs (ceil(n / (N / grid)), at most
// max_team and kMaxTeam), largest systems first, while the team slots stay within half the
// grid; the other systems get one CTA. Team slots come first, in a row per team.
static void build_slots(BatchEngine *E, int s) {
    const int G = E->grid[s];
    const int cap = E->max_team == 0 ? kMaxTeam : std::min(E->max_team, kMaxTeam);
    std::vector<int> &team = E->team[s];
    team.assign(E->nprob, 1);
    if (cap > 1 && G >= 4) {
        const double share = (double)E->N / G;
        int used = 0;
        for (int p : E->ord) {
            const int64_t n = E->hs[p]->N;
            int K = (int)std::min<double>(cap, std::ceil((double)n / share - 1e-9));
            if (n < 4 * (int64_t)kShapes[s].threads) K = 1;  // a few rows per thread at most
            if (K < 2 || used + K > G / 2) break;  // sizes descend: the rest get one CTA
            team[p] = K;
            used += K;
        }
    }
    std::vector<int4> sl;
    for (int p : E->ord)
        for (int r = 0; r < team[p]; r++) sl.push_back(make_int4(p, r, team[p], 0));
    if (!E->slots[s]) E->slots[s] = balloc<int4>(E, (size_t)E->nprob + E->grid[s] / 2);
    E->nslots[s] = (int)sl.size();
    AMG_CUDA(cudaMemcpyAsync(E->slots[s], sl.data(), sizeof(int4) * sl.size(),
                             cudaMemcpyHostToDevice, E->stream));
    AMG_CUDA(cudaStreamSynchronize(E->stream));  // sl is a local
}

BatchEngine *batch_create(const std::vector<amg_hierarchy *> &hs, const std::vector<int64_t> &row_off,
                          cudaStream_t stream, int shape_threads) {
    BatchEngine *E = new BatchEngine();
    try {
        if (shape_threads == 1024) E->shape = 0;
        else if (shape_threads == 512) E->shape = 1;
        else if (shape_threads == 256) E->shape = 3;
        // teams follow the batch's composition: only where the shape is chosen by timing
        // (with a fixed shape a system's result does not depend on the other systems)
        E->max_team = E->shape < 0 ? 0 : 1;
        E->tuned = E->shape < 0;
        E->hs = hs;
        E->row_off = row_off;
        E->nprob = (int)hs.size();
        E->N = row_off.back();
        E->stream = stream;
        const amg_options &o = hs[0]->opt;
        E->fp32 = o.cycle_prec == AMG_FP32;
        E->kc = o.kcycle_n;
        E->nu = o.nu_pre + 256 * o.nu_post;
        E->maxit = o.max_iters;
        for (amg_hierarchy *h : hs) {
            AMG_CUDA(cudaStreamSynchronize(h->stream));
            if (E->fp32) prepare_cycle(h);
            AMG_CUDA(cudaStreamSynchronize(h->stream));
        }
        if (E->fp32) build_probs<float>(E);
        else build_probs<double>(E);
        // queue order: largest system first
        E->ord.resize(E->nprob);
        std::iota(E->ord.begin(), E->ord.end(), 0);
        std::stable_sort(E->ord.begin(), E->ord.end(),
                         [&](int a, int b) { return hs[a]->N > hs[b]->N; });
        for (int s = 0; s < kNumShapes; s++)
            if (E->grid[s] > 0) build_slots(E, s);
        E->team_bar = balloc<unsigned long long>(E, E->nprob);
        E->team_part = balloc<double>(E, (size_t)E->nprob * kTeamPart);
        E->team_cnt = balloc<unsigned int>(E, E->nprob);
        AMG_CUDA(cudaMemsetAsync(E->team_cnt, 0, sizeof(unsigned int) * E->nprob, E->stream));
        E->next = balloc<int>(E, 1);
        E->iters = balloc<int>(E, E->nprob);
        E->status = balloc<int>(E, E->nprob);
        E->relres = balloc<double>(E, E->nprob);
        E->t_start = balloc<unsigned long long>(E, E->nprob);
        E->t_end = balloc<unsigned long long>(E, E->nprob);
        AMG_CUDA(cudaStreamSynchronize(E->stream));
    } catch (...) {
        batch_destroy(E);
        throw;
    }
    return E;
}

void batch_destroy(BatchEngine *E) {
    if (!E) return;
    if (E->graph) cudaGraphExecDestroy(E->graph);
    for (void *p : E->allocs) cudaFreeAsync(p, E->stream);
    cudaStreamSynchronize(E->stream);
    delete E;
}

size_t batch_bytes(const BatchEngine *E) { return E->bytes; }

// queue and team counters reset + the persistent kernel, on E->stream
static void launch_batch(BatchEngine *E, int shape, const double *b, double *x, double tol) {
    AMG_CUDA(cudaMemsetAsync(E->next, 0, sizeof(int), E->stream));
    AMG_CUDA(cudaMemsetAsync(E->team_bar, 0, sizeof(unsigned long long) * E->nprob, E->stream));
    AMG_CUDA(cudaMemsetAsync(E->team_cnt, 0, sizeof(unsigned int) * E->nprob, E->stream));
    void *kern = E->fp32 ? batch_kernel<float>(shape) : batch_kernel<double>(shape);
    int nslots = E->nslots[shape], kc = E->kc, nu = E->nu, maxit = E->maxit;
    unsigned long long limit_ns =
        E->dbg_bar_limit_ns > 0 ? (unsigned long long)E->dbg_bar_limit_ns : kBarrierLimitNs;
    int extra = E->dbg_bar_extra;
    void *args[] = {&E->probs,  &E->slots[shape], &nslots,     &E->next,    &kc,  &nu,
                    &b,         &x,               &tol,        &maxit,      &E->iters,
                    &E->relres, &E->status,       &E->t_start, &E->t_end,   &E->team_bar,
                    &E->team_part, &E->team_cnt, &limit_ns, &extra};
    AMG_CUDA(cudaLaunchKernel(kern, dim3(E->grid[shape]), dim3(kShapes[shape].threads), args, 0,
                              E->stream));
    AMG_LAUNCH_CHECK();
}

// times every launch shape on this batch (each solve is complete and correct) and keeps the
// fastest
static void autotune(BatchEngine *E, const double *b, double *x, double tol) {
    cudaEvent_t e0, e1;
    AMG_CUDA(cudaEventCreate(&e0));
    AMG_CUDA(cudaEventCreate(&e1));
    int best = 0;
    for (int s = 0; s < kNumShapes; s++) {
        if (E->grid[s] < 1) {
            E->tuned_ms[s] = -1.0;
            continue;
        }
        launch_batch(E, s, b, x, tol);  // warm
        AMG_CUDA(cudaEventRecord(e0, E->stream));
        launch_batch(E, s, b, x, tol);
        AMG_CUDA(cudaEventRecord(e1, E->stream));
        AMG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        AMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        E->tuned_ms[s] = ms;
        if (E->tuned_ms[best] < 0.0 || ms < E->tuned_ms[best]) best = s;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    E->shape = best;
}

int batch_solve(BatchEngine *E, const double *b, double tol, double *x, int *iters, double *relres,
                int *status) {
    if (E->shape < 0) autotune(E, b, x, tol);
    if (!E->graph || E->g_b != b || E->g_x != x || E->g_tol != tol || E->g_shape != E->shape) {
        if (E->graph) {
            AMG_CUDA(cudaGraphExecDestroy(E->graph));
            E->graph = nullptr;
        }
        cudaGraph_t g;
        const int64_t counted = g_launches;  // capturing launches nothing
        AMG_CUDA(cudaStreamBeginCapture(E->stream, cudaStreamCaptureModeThreadLocal));
        launch_batch(E, E->shape, b, x, tol);
        AMG_CUDA(cudaStreamEndCapture(E->stream, &g));
        g_launches = counted;
        AMG_CUDA(cudaGraphInstantiate(&E->graph, g, 0));
        AMG_CUDA(cudaGraphDestroy(g));
        E->g_b = b;
        E->g_x = x;
        E->g_tol = tol;
        E->g_shape = E->shape;
    }
    AMG_CUDA(cudaGraphLaunch(E->graph, E->stream));
    g_launches += 1;  // the persistent kernel (after the counter resets)
    std::vector<int> it(E->nprob), st(E->nprob);
    std::vector<double> rr(E->nprob);
    AMG_CUDA(cudaMemcpyAsync(it.data(), E->iters, sizeof(int) * E->nprob, cudaMemcpyDeviceToHost, E->stream));
    AMG_CUDA(cudaMemcpyAsync(st.data(), E->status, sizeof(int) * E->nprob, cudaMemcpyDeviceToHost, E->stream));
    AMG_CUDA(cudaMemcpyAsync(rr.data(), E->relres, sizeof(double) * E->nprob, cudaMemcpyDeviceToHost, E->stream));
    AMG_CUDA(cudaStreamSynchronize(E->stream));
    int first_bad = AMG_OK;
    for (int p = 0; p < E->nprob; p++) {
        if (iters) iters[p] = it[p];
        if (relres) relres[p] = rr[p];
        if (status) status[p] = st[p];
        if (first_bad == AMG_OK && st[p] != AMG_OK) first_bad = st[p];
    }
    return first_bad;
}

// per-system start and end of the last solve, ns after the earliest start
void batch_timeline(const BatchEngine *E, int64_t *start_ns, int64_t *end_ns) {
    std::vector<unsigned long long> a(E->nprob), b(E->nprob);
    AMG_CUDA(cudaMemcpyAsync(a.data(), E->t_start, 8 * a.size(), cudaMemcpyDeviceToHost, E->stream));
    AMG_CUDA(cudaMemcpyAsync(b.data(), E->t_end, 8 * b.size(), cudaMemcpyDeviceToHost, E->stream));
    AMG_CUDA(cudaStreamSynchronize(E->stream));
    const unsigned long long t0 = *std::min_element(a.begin(), a.end());
    for (int p = 0; p < E->nprob; p++) {
        if (start_ns) start_ns[p] = (int64_t)(a[p] - t0);
        if (end_ns) end_ns[p] = (int64_t)(b[p] - t0);
    }
}

void batch_set_teams(BatchEngine *E, int max_team) {
    E->max_team = max_team;
    for (int s = 0; s < kNumShapes; s++)
        if (E->grid[s] > 0) build_slots(E, s);
    if (E->tuned) E->shape = -1;  // the shapes' times change with the teams
    E->g_shape = -1;              // recapture the launch
}

void batch_barrier_fault(BatchEngine *E, int64_t limit_ns, int extra) {
    E->dbg_bar_limit_ns = limit_ns;
    E->dbg_bar_extra = extra;
    E->g_shape = -1;  // recapture the launch with the new arguments
}

int bounds_flags_batch() { return bounds_flag_read_clear(); }

void batch_teams(const BatchEngine *E, int *team) {
    for (int p = 0; p < E->nprob; p++) team[p] = E->shape < 0 ? -1 : E->team[E->shape][p];
}

int batch_shape(const BatchEngine *E, int *threads, int *ctas, double *tuned_ms) {
    if (E->shape < 0) return -1;
    if (threads) *threads = kShapes[E->shape].threads;
    if (ctas) *ctas = E->grid[E->shape];
    if (tuned_ms)
        for (int s = 0; s < kNumShapes; s++) tuned_ms[s] = E->tuned_ms[s];
    return E->shape;
}

}  // namespace amg
