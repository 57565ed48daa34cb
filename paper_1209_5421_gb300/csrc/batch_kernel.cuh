// The batched solve's device code: the team of CTAs that solves one system, the AMLI-cycle
// walked over a system's levels, the outer flexible CG and the persistent kernel k_batch.
// Included by batch.cu (kernels for batches without big aggregates) and batch_graded.cu
// (BIG: the finest level's big aggregates swept by warps / CTAs in level order); the two
// translation units compile in parallel, and a batch without graded systems runs code
// without that phase.
#pragma once

#include "cycle_ops.cuh"

namespace amg {

template <class T>
using BLev = LevelDev<T, int>;

constexpr int kBatchChunk = 64;  // directions orthogonalised against per pass
constexpr int kBatchResume = 1000;  // status: the directions are full, the host adds more
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
    double *const *Pt;             // outer directions p_j (the hierarchy's table), n each
    double *const *Qt;             // their images q_j = A p_j
    double *pq;                    // (p_j, q_j)
    int cap;                       // directions allocated: p_j, q_j exist for j < cap
    const int4 *bigr;              // finest level's colours: big-block ranges, or NULL
    int nbig;                      // big blocks of the finest level
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
static __shared__ Team bt_team;

// thread 0: arrive at the team's barrier and wait for the other members, bounded like the
// grid barrier (kBarrierLimitNs); out of line, as the one-CTA path never takes it
static __device__ __noinline__ void team_wait() {
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

template <class T, bool BIG>
struct BatchCycle {
    const BLev<T> *tab;  // shared-memory copy of the level table
    const int *colors;
    const int *cofs, *ncol;
    int nlev, kc;
    int nu_pre, nu_post;  // smoothing sweeps
    const int4 *bigr;     // finest level's big-block ranges per colour, or NULL (BIG only)
    int nbig;
};

// first non-empty colour [r0, r1) of level l >= 1
template <class T, bool BIG>
__device__ __forceinline__ void first_colour(const BatchCycle<T, BIG> &c, int l, int &r0, int &r1) {
    const int *cr = c.colors + c.cofs[l];
    const int nc = c.ncol[l];
    int k = 0;
    while (k < nc && cr[k + 1] == cr[k]) k++;
    r0 = k < nc ? cr[k] : 0;
    r1 = k < nc ? cr[k + 1] : 0;
}

// one colour of a sweep on level l; on the finest level of a system with big blocks (BIG
// kernels only) the colour's big blocks go to the team's warps and CTAs in level order, as
// in the grid-wide program
template <class T, bool BIG>
__device__ __forceinline__ void bc_gs(const BatchCycle<T, BIG> &c, int l, const BLev<T> &L,
                                      Op &op, int col, const T *f, T *z, int tid, int nth) {
    if constexpr (BIG) {
        if (l == 0 && c.bigr) {
            const int4 r = c.bigr[col];
            op.bb0 = r.x;
            op.bbc = r.y;
            op.bb1 = r.z;
            op_gs<BLev<T>, true>(L, op, f, z, tid, nth, bt_team.rank, bt_team.K);
            op.bb0 = op.bbc = op.bb1 = 0;
            return;
        }
    }
    op_gs(L, op, f, z, tid, nth);
}

// pre-smoothing and restriction of B^_l: level 0 from u = 0 (block smoother, all colours);
// coarse levels for z = p_i, f = rhs (i = 0) or r, the first non-empty colour as u = D^-1 f
template <class T, bool BIG>
__device__ __forceinline__ void bc_pre(const BatchCycle<T, BIG> &c, int l, int i) {
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
            bc_gs(c, l, L, op, col, f, z, tid, nth);
            team_sync();
        }
    const BLev<T> &N = c.tab[l + 1];
    const bool big = BIG && l == 0 && c.nbig > 0;  // the finest level's big blocks: warps / CTAs
    if (l + 1 < c.nlev - 1) {  // the next level smooths: its first colour from zero too
        int f0, f1;
        first_colour(c, l + 1, f0, f1);
        op_restrict(L, f, z, N.rhs, tid, nth, N.p[0], N.dinv, f0, f1, big, bt_team.rank,
                    bt_team.K);
    } else {
        op_restrict(L, f, z, N.rhs, tid, nth, (T *)nullptr, (const T *)nullptr, 0, 0, big,
                    bt_team.rank, bt_team.K);
    }
    team_sync();
}

// prolongation and post-smoothing of B^_l; on coarse levels then Alg. 1 step i
template <class T, bool BIG>
__device__ __forceinline__ void bc_post(const BatchCycle<T, BIG> &c, int l, int i) {
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
            bc_gs(c, l, L, op, col, f, z, tid, nth);
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
template <class T, bool BIG>
__device__ void batch_cycle(const BatchCycle<T, BIG> &c) {
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

template <class T, bool BIG>
__device__ void solve_one(const BatchProb<T> &P, const BatchCycle<T, BIG> &cyc, const double *b,
                          double *x, double tol, int maxit, int *iters, double *relres,
                          int *status, int *resume, int slot) {
    const int n = P.n;  // every row loop: from team_tid() in steps of team_nth()
    double *bo = P.bo, *xo = P.xo, *ro = P.ro, *zo = P.zo, *to = P.to;
    T *crhs = cyc.tab[0].rhs, *ce = cyc.tab[0].e;
    // per chunk of kept directions, held by every CTA of the team: (z, q_j), its quotient by
    // (p_j, q_j) (divided once per step, not per row: FP64 division is long here), p_j, q_j
    __shared__ double zq[kBatchChunk], cq[kBatchChunk];
    __shared__ const double *sP[kBatchChunk], *sQ[kBatchChunk];
    // a resumed system (its directions were full) continues at step `it` from the x, r and
    // directions of the launch before; a fresh one starts from x = 0
    int it = resume[slot];
    double bb = 0.0;
    for (int i = team_tid(), nth = team_nth(); i < n; i += nth) {
        const double v = b[P.off + P.nat[i]];
        if (it == 0) {
            bo[i] = v;
            ro[i] = v;
            xo[i] = 0.0;
        }
        bb += v * v;
    }
    bb = team_sum1(bb);  // (its barrier also orders the writes above)
    const double bn = sqrt(bb);
    int st = AMG_ERR_NOT_CONVERGED;
    double rel = 1.0;
    if (!isfinite(bn)) {
        st = AMG_ERR_INVALID_ARG;
    } else if (bn == 0.0) {
        st = AMG_OK;
        rel = 0.0;
    } else {
        while (it < maxit) {
            if (it >= P.cap) {  // every allocated direction is in use: resumed with more
                st = kBatchResume;
                break;
            }
            // z = B^_0 [r] in the cycle precision
            if ((const void *)crhs != (const void *)ro)
                for (int i = team_tid(), nth = team_nth(); i < n; i += nth) crhs[i] = (T)ro[i];
            team_sync();
            batch_cycle(cyc);
            if ((const void *)ce != (const void *)zo)
                for (int i = team_tid(), nth = team_nth(); i < n; i += nth) zo[i] = (double)ce[i];
            team_sync();
            // p_k = z - sum_{j<k} (z, q_j) / (p_j, q_j) p_j (k = it: every direction is
            // kept), kBatchChunk directions per pass (the same operations in the same order)
            const int k = it;
            double *pk = P.Pt[k], *qk = P.Qt[k];
            for (int c0 = 0; c0 == 0 || c0 < k; c0 += kBatchChunk) {
                const int c1 = min(k, c0 + kBatchChunk);
                if (c0 > 0) __syncthreads();  // the last chunk's sP and cq are read no more
                for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
                    sP[j - c0] = P.Pt[j];
                    sQ[j - c0] = P.Qt[j];
                }
                __syncthreads();
                for (int j0 = c0; j0 < c1; j0 += 4) {  // (z, q_j)
                    double v[4] = {0.0, 0.0, 0.0, 0.0}, r[4];
                    for (int i = team_tid(), nth = team_nth(); i < n; i += nth) {
                        const double zi = zo[i];
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            if (j0 + j < c1) v[j] += zi * sQ[j0 + j - c0][i];
                    }
                    team_sum<4>(v, r);
                    if (threadIdx.x == 0)
                        for (int j = 0; j < 4 && j0 + j < c1; j++) zq[j0 + j - c0] = r[j];
                }
                __syncthreads();
                for (int j = c0 + threadIdx.x; j < c1; j += blockDim.x)
                    cq[j - c0] = zq[j - c0] / P.pq[j];
                __syncthreads();
                for (int i = team_tid(), nth = team_nth(); i < n; i += nth) {
                    double acc = c0 == 0 ? zo[i] : pk[i];
                    for (int j = c0; j < c1; j++) acc -= cq[j - c0] * sP[j - c0][i];
                    pk[i] = acc;
                }
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
            // read by the team's CTAs after later team barriers only
            if (bt_team.rank == 0 && threadIdx.x == 0) P.pq[k] = pq;
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
            if (bt_team.abort) break;  // a member stopped answering: no result
        }
        if (st != AMG_OK && st != AMG_ERR_INVALID_ARG && st != kBatchResume)
            rel = sqrt(true_residual(P.A0, bo, xo, to)) / bn;
    }
    if (bt_team.abort) st = AMG_ERR_TIMEOUT;
    if (st != kBatchResume)
        for (int i = team_tid(), nth = team_nth(); i < n; i += nth) x[P.off + P.nat[i]] = xo[i];
    if (bt_team.rank == 0 && threadIdx.x == 0) {
        iters[slot] = it;
        relres[slot] = rel;
        status[slot] = st;
        resume[slot] = st == kBatchResume ? it : 0;
    }
    __syncthreads();
}

// every CTA: take the next slot from the queue (largest systems first; the K slots of a team
// in a row) and solve that system, alone or as rank s.y of a team of s.z CTAs
template <class T, int NT, int MINB, bool BIG>
__global__ void __launch_bounds__(NT, MINB)
k_batch(const BatchProb<T> *__restrict__ probs, const int4 *__restrict__ slots, int nslots,
        int *next, int kc, int nu, const double *__restrict__ b, double *__restrict__ x,
        double tol, int maxit, int *iters, double *relres, int *status,
        unsigned long long *t_start, unsigned long long *t_end, unsigned long long *team_bar,
        double *team_part, unsigned int *team_cnt, unsigned long long bar_limit_ns,
        int bar_extra, int *resume) {
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
        BatchCycle<T, BIG> cyc{stab, sp.colors, sp.cofs,  sp.ncol, sp.nlev,
                               kc,   nu & 255,  nu >> 8, sp.bigr, sp.nbig};
        if (threadIdx.x == 0 && sl.y == 0 && resume[p] == 0) t_start[p] = global_ns();
        solve_one(sp, cyc, b, x, tol, maxit, iters, relres, status, resume, p);
        if (threadIdx.x == 0 && sl.y == 0) t_end[p] = global_ns();
        // (solve_one ends with a barrier: q and bt_team may be overwritten)
    }
}

template <class T, bool BIG>
void *batch_kernel_of(int shape) {
    switch (shape) {
        case 0: return (void *)k_batch<T, 1024, 1, BIG>;
        case 1: return (void *)k_batch<T, 512, 2, BIG>;
        case 2: return (void *)k_batch<T, 512, 1, BIG>;
        default: return (void *)k_batch<T, 256, 4, BIG>;
    }
}

// batch_graded.cu: the BIG kernels
void *batch_kernel_graded(bool fp32, int shape);

}  // namespace amg
