// Batched solves: many independent systems of uneven sizes, each with its own hierarchy
// (built by the single-system setup), solved by one persistent kernel.
//
// The paper solves one system at a time. A batch of small and mid-size systems would leave
// the GPU almost idle if each ran the grid-wide cycle kernel in turn (those solves are
// latency-bound: a few thousand dependent steps, each a grid barrier). Here every CTA takes
// the next unsolved system from a queue (largest first) and runs its whole solve alone: the
// outer flexible CG (Alg. 1 on the finest level, FP64, full orthogonalisation, restarted
// after `cap` directions) and, every iteration, the AMLI-cycle B^_0 (Alg. 2, with Alg. 1 on
// the coarse levels and the exact coarsest solve) on levels that stay in HBM / L2, with
// CTA-wide barriers only. The cycle ops are the same device functions as the single-system
// kernel (cycle_ops.cuh) on the same level data, walked as a state machine over the levels.
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
    double *osc;                   // outer scalars, kBatchOsc doubles
};

// outer scalars of one system
enum : int { BO_BB = 0, BO_ZQ = 8, BO_PQ = BO_ZQ + kBatchCap, kBatchOsc = BO_PQ + kBatchCap };

// ---------------------------------------------------------------------------------------
// CTA-wide helpers

// sum over the CTA, returned to every thread
__device__ __forceinline__ double cta_sum(double v) {
    __shared__ double bc;
    const double a[1] = {v};
    double r[1];
    block_sum<1, double>(a, r, BlockGroup{});
    if (threadIdx.x == 0) bc = r[0];
    __syncthreads();
    const double out = bc;
    __syncthreads();  // bc and the reduction scratch are reused by the next call
    return out;
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
    const int tid = threadIdx.x, nth = blockDim.x;
    const int *cr = c.colors + c.cofs[l];
    const int nc = c.ncol[l];
    const T *f = (l == 0 || i == 0) ? L.rhs : L.r;
    T *z = l == 0 ? L.e : pick(L.p, i);
    Op op = batch_op();
    int col = 0;
    if (l == 0) {
        op_zero(L, z, tid, nth);
        __syncthreads();
    } else {  // the first colour was done by the restriction into this level or the last UPDATE
        while (col < nc && cr[col + 1] == cr[col]) col++;
        col++;
    }
    for (; col < nc; col++) {
        if (cr[col + 1] == cr[col]) continue;
        op.i0 = cr[col];
        op.i1 = cr[col + 1];
        op_gs(L, op, f, z, tid, nth);
        __syncthreads();
    }
    const BLev<T> &N = c.tab[l + 1];
    if (l + 1 < c.nlev - 1) {  // the next level smooths: its first colour from zero too
        int f0, f1;
        first_colour(c, l + 1, f0, f1);
        op_restrict(L, f, z, N.rhs, tid, nth, N.p[0], N.dinv, f0, f1);
    } else {
        op_restrict(L, f, z, N.rhs, tid, nth);
    }
    __syncthreads();
}

// prolongation and post-smoothing of B^_l; on coarse levels then Alg. 1 step i
template <class T>
__device__ __forceinline__ void bc_post(const BatchCycle<T> &c, int l, int i) {
    const BLev<T> &L = c.tab[l];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int *cr = c.colors + c.cofs[l];
    const T *f = (l == 0 || i == 0) ? L.rhs : L.r;
    T *z = l == 0 ? L.e : pick(L.p, i);
    op_prolong(L, c.tab[l + 1].e, z, tid, nth);
    __syncthreads();
    Op op = batch_op();
    op.backward = 1;
    for (int col = c.ncol[l] - 1; col >= 0; col--) {
        if (cr[col + 1] == cr[col]) continue;
        op.i0 = cr[col];
        op.i1 = cr[col + 1];
        op_gs(L, op, f, z, tid, nth);
        __syncthreads();
    }
    if (l == 0) return;
    const RedCtx rc{nullptr, nullptr};
    op = batch_op();
    op.step = i;
    op.last = (i == c.kc - 1);
    if (!op.last) {  // the UPDATE also starts step i+1's pre-smoothing
        op.fuse = 1;
        first_colour(c, l, op.f0, op.f1);
    }
    if (i > 0) {
        op_multidot<BLev<T>, RM_BLOCK>(L, op, rc, tid, nth, BlockGroup{});
        __syncthreads();
        op_orth(L, op, tid, nth, BlockGroup{});
        __syncthreads();
    }
    op_spmv_dot<BLev<T>, RM_BLOCK>(L, op, rc, tid, nth, BlockGroup{});
    __syncthreads();
    op_update<BLev<T>, RM_BLOCK>(L, op, rc, tid, nth, BlockGroup{});
    __syncthreads();
}

// B^_0 over the whole hierarchy: the recursion of Alg. 2 / Alg. 1 as a state machine (the
// same walk as the shared-memory tail of the single-system kernel, from level 0)
template <class T>
__device__ void batch_cycle(const BatchCycle<T> &c) {
    if (c.nlev == 1) {  // the only level is the coarsest: exact solve
        op_coarse(c.tab[0], threadIdx.x, blockDim.x);
        __syncthreads();
        return;
    }
    enum { ENTER, PRE, POST };
    int step[kMaxLevels] = {};
    int l = 0, ph = PRE;
    for (;;) {
        const bool coarsest = (l == c.nlev - 1);
        const int i = step[l];
        if (l > 0 && ph == ENTER && coarsest) {
            op_coarse(c.tab[l], threadIdx.x, blockDim.x);
            __syncthreads();
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

// t = b - A x, returns (t, t)
__device__ __forceinline__ double true_residual(const BLev<double> &A, const double *b,
                                                const double *x, double *t) {
    double s = 0.0;
    for (int i = threadIdx.x; i < A.n; i += blockDim.x) {
        const double ri = row_residual(A, i, b, x);
        t[i] = ri;
        s += ri * ri;
    }
    return cta_sum(s);
}

template <class T>
__device__ void solve_one(const BatchProb<T> &P, const BatchCycle<T> &cyc, const double *b,
                          double *x, double tol, int maxit, int *iters, double *relres,
                          int *status, int slot) {
    const int n = P.n, tid = threadIdx.x, nth = blockDim.x;
    double *bo = P.bo, *xo = P.xo, *ro = P.ro, *zo = P.zo, *to = P.to, *osc = P.osc;
    T *crhs = cyc.tab[0].rhs, *ce = cyc.tab[0].e;
    double bb = 0.0;
    for (int i = tid; i < n; i += nth) {
        const double v = b[P.off + P.nat[i]];
        bo[i] = v;
        ro[i] = v;
        xo[i] = 0.0;
        bb += v * v;
    }
    bb = cta_sum(bb);  // (its barrier also orders the writes above)
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
                for (int i = tid; i < n; i += nth) crhs[i] = (T)ro[i];
            __syncthreads();
            batch_cycle(cyc);
            if ((const void *)ce != (const void *)zo)
                for (int i = tid; i < n; i += nth) zo[i] = (double)ce[i];
            __syncthreads();
            // (z, q_j), j < k
            double *pk = P.P + (size_t)k * n, *qk = P.Q + (size_t)k * n;
            for (int j0 = 0; j0 < k; j0 += 4) {
                double v[4] = {0.0, 0.0, 0.0, 0.0}, r[4];
                for (int i = tid; i < n; i += nth) {
                    const double zi = zo[i];
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if (j0 + j < k) v[j] += zi * P.Q[(size_t)(j0 + j) * n + i];
                }
                block_sum<4, double>(v, r, BlockGroup{});
                if (tid == 0)
                    for (int j = 0; j < 4 && j0 + j < k; j++) osc[BO_ZQ + j0 + j] = r[j];
                __syncthreads();
            }
            // p_k = z - sum_j (z, q_j) / (p_j, q_j) p_j
            for (int i = tid; i < n; i += nth) {
                double acc = zo[i];
                for (int j = 0; j < k; j++)
                    acc -= (osc[BO_ZQ + j] / osc[BO_PQ + j]) * P.P[(size_t)j * n + i];
                pk[i] = acc;
            }
            __syncthreads();
            // q_k = A p_k, (p_k, q_k), (r, p_k)
            double v2[2] = {0.0, 0.0}, r2[2];
            for (int i = tid; i < n; i += nth) {
                int base, width;
                row_span(P.A0, i, base, width);
                const double qi = row_dot(P.A0, base, 0, width, pk);
                qk[i] = qi;
                v2[0] += pk[i] * qi;
                v2[1] += ro[i] * pk[i];
            }
            block_sum<2, double>(v2, r2, BlockGroup{});
            __shared__ double pq_rp[2];
            if (tid == 0) {
                pq_rp[0] = r2[0];
                pq_rp[1] = r2[1];
                osc[BO_PQ + k] = r2[0];
            }
            __syncthreads();
            const double pq = pq_rp[0], rp = pq_rp[1];
            __syncthreads();
            if (!(pq > 0.0) || !isfinite(pq)) {
                st = AMG_ERR_BREAKDOWN;
                break;
            }
            const double alpha = rp / pq;
            double rr = 0.0;
            for (int i = tid; i < n; i += nth) {
                xo[i] += alpha * pk[i];
                const double rn = ro[i] - alpha * qk[i];
                ro[i] = rn;
                rr += rn * rn;
            }
            rr = cta_sum(rr);
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
                for (int i = tid; i < n; i += nth) ro[i] = to[i];
                __syncthreads();
            }
            if (k == kBatchCap) {  // restart from the true residual
                true_residual(P.A0, bo, xo, ro);
                k = 0;
            }
        }
        if (st != AMG_OK && st != AMG_ERR_INVALID_ARG) rel = sqrt(true_residual(P.A0, bo, xo, to)) / bn;
    }
    for (int i = tid; i < n; i += nth) x[P.off + P.nat[i]] = xo[i];
    if (tid == 0) {
        iters[slot] = it;
        relres[slot] = rel;
        status[slot] = st;
    }
    __syncthreads();
}

// every CTA: take the next system from the queue (largest first) and solve it alone
template <class T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_batch(const BatchProb<T> *__restrict__ probs, const int *__restrict__ order, int nprob,
        int *next, int kc, const double *__restrict__ b, double *__restrict__ x, double tol,
        int maxit, int *iters, double *relres, int *status, unsigned long long *t_start,
        unsigned long long *t_end) {
    __shared__ BatchProb<T> sp;
    __shared__ BLev<T> stab[kMaxLevels];
    __shared__ int q;
    for (;;) {
        if (threadIdx.x == 0) q = atomicAdd(next, 1);
        __syncthreads();
        const int mine = q;
        if (mine >= nprob) break;
        const int p = order[mine];
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
        BatchCycle<T> cyc{stab, sp.colors, sp.cofs, sp.ncol, sp.nlev, kc};
        if (threadIdx.x == 0) t_start[p] = global_ns();
        solve_one(sp, cyc, b, x, tol, maxit, iters, relres, status, p);
        if (threadIdx.x == 0) t_end[p] = global_ns();
        // (solve_one ends with a barrier: q may be overwritten)
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
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    void *probs = nullptr;  // BatchProb<T>[nprob]
    int *order = nullptr, *next = nullptr, *iters = nullptr, *status = nullptr;
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
    AMG_CUDA(cudaMallocAsync(&p, std::max<size_t>(16, count * sizeof(U)), E->stream));
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
    w.osc = halloc<double>(h, kBatchOsc);
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
        B.osc = w.osc;
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
        E->grid[s] = std::min(np, nsm * std::min(per, kShapes[s].per_sm));
    }
    AMG_CUDA(cudaStreamSynchronize(E->stream));  // hp is a local
}

BatchEngine *batch_create(const std::vector<amg_hierarchy *> &hs, const std::vector<int64_t> &row_off,
                          cudaStream_t stream, int shape_threads) {
    BatchEngine *E = new BatchEngine();
    try {
        if (shape_threads == 1024) E->shape = 0;
        else if (shape_threads == 512) E->shape = 1;
        else if (shape_threads == 256) E->shape = 3;
        E->hs = hs;
        E->row_off = row_off;
        E->nprob = (int)hs.size();
        E->N = row_off.back();
        E->stream = stream;
        const amg_options &o = hs[0]->opt;
        E->fp32 = o.cycle_prec == AMG_FP32;
        E->kc = o.kcycle_n;
        E->maxit = o.max_iters;
        for (amg_hierarchy *h : hs) {
            AMG_CUDA(cudaStreamSynchronize(h->stream));
            if (E->fp32) prepare_cycle(h);
            AMG_CUDA(cudaStreamSynchronize(h->stream));
        }
        if (E->fp32) build_probs<float>(E);
        else build_probs<double>(E);
        // queue order: largest system first
        std::vector<int> ord(E->nprob);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return hs[a]->N > hs[b]->N; });
        E->order = balloc<int>(E, E->nprob);
        AMG_CUDA(cudaMemcpyAsync(E->order, ord.data(), sizeof(int) * ord.size(),
                                 cudaMemcpyHostToDevice, E->stream));
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

// queue reset + the persistent kernel, on E->stream
static void launch_batch(BatchEngine *E, int shape, const double *b, double *x, double tol) {
    AMG_CUDA(cudaMemsetAsync(E->next, 0, sizeof(int), E->stream));
    void *kern = E->fp32 ? batch_kernel<float>(shape) : batch_kernel<double>(shape);
    int nprob = E->nprob, kc = E->kc, maxit = E->maxit;
    void *args[] = {&E->probs, &E->order, &nprob, &E->next, &kc,       &b,
                    &x,        &tol,      &maxit, &E->iters, &E->relres, &E->status,
                    &E->t_start, &E->t_end};
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
    g_launches += 1;  // the persistent kernel (after the queue-counter reset)
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

int batch_shape(const BatchEngine *E, int *threads, int *ctas, double *tuned_ms) {
    if (E->shape < 0) return -1;
    if (threads) *threads = kShapes[E->shape].threads;
    if (ctas) *ctas = E->grid[E->shape];
    if (tuned_ms)
        for (int s = 0; s < kNumShapes; s++) tuned_ms[s] = E->tuned_ms[s];
    return E->shape;
}

}  // namespace amg
