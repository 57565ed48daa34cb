// Solve phase on the GPU: the nonlinear AMLI-cycle (paper Alg. 2) with nonlinear PCG on
// the coarse levels (Alg. 1), the quadtree-coloured Gauss-Seidel smoother (Sec. 4.5),
// implicit prolongation / restriction (Sec. 4.3), and the outer Krylov iteration.
//
// Execution model. The cycle is a fixed sequence of operations ("ops") on device-resident
// data: a Gauss-Seidel sweep over one colour, a fused residual+restriction, a fused
// prolongation+correction, the exact coarsest solve, and the Alg. 1 pieces (A-orthogonal
// direction, SpMV with its two inner products, the update). Every scalar (alpha, beta, inner
// products) stays in device memory. The host walks the recursion once and either
//   * launches one multi-CTA kernel per op (large levels), or
//   * appends the op to a program that one CTA interprets with __syncthreads() between ops
//     (all levels from the "tail" level down: small levels are latency-bound, and one CTA
//     runs their whole recursive Alg. 1 / Alg. 2 without a kernel launch per op).
// The whole preconditioner application is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "amg_internal.cuh"

namespace amg {

enum OpKind : int {
    OP_ZERO = 0,      // u = 0
    OP_GS,            // one colour of a Gauss-Seidel sweep: rows/blocks [i0, i1)
    OP_RESTRICT,      // next.rhs = P^t (f - A u)
    OP_PROLONG,       // u += P next.e
    OP_COARSE,        // e = A^{-1} rhs (coarsest level)
    OP_MULTIDOT,      // sc[ZQ_j] = (p_i, q_j), j < i
    OP_ORTH,          // p_i -= sum_j (sc[ZQ_j] / sc[PQ_j]) p_j
    OP_SPMV_DOT,      // q_i = A p_i, sc[PQ_i] = (p_i, q_i), sc[RP_i] = (r_i, p_i)
    OP_UPDATE,        // alpha_i; e (+)= alpha_i p_i; r = r_i - alpha_i q_i; sc[RR] = (r, r)
};

struct Op {
    int kind;
    int level;
    int i0, i1;       // GS range
    int backward;     // GS direction
    int step;         // Alg. 1 step index i
    int last;         // Alg. 1: is this the last step
    int fsel, usel;   // vector selectors (see vec_of)
};

// vector selectors of a level
enum : int { V_RHS = 0, V_E, V_R, V_P0 };  // V_P0 + i = p_i

template <class T>
struct LevelDev {
    int n;
    int fine;                       // 1 on the finest level (block smoother, bptr)
    const int *sl, *col;
    const T *val;
    const int *bptr;
    const int *parent;
    const int4 *children;           // of the NEXT coarser level
    const T *Ainv;
    T *rhs, *e, *r;
    T *p[kMaxKcycle], *q[kMaxKcycle];
    double *sc;
    int nnext;                      // rows of the next coarser level
};

template <class T>
__device__ __forceinline__ T *vec_of(const LevelDev<T> &L, int sel) {
    return sel == V_RHS ? L.rhs : sel == V_E ? L.e : sel == V_R ? L.r : L.p[sel - V_P0];
}

// ---------------------------------------------------------------------------------------
// reductions: fixed-order trees, no floating-point atomics (bitwise reproducible)
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV]) {
    __shared__ double sm[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) sm[k][w] = v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) {
            v[k] = lane < nw ? sm[k][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
    __syncthreads();
}

struct RedCtx {
    double *partials;       // [NV * gridDim.x]
    unsigned int *counter;
};

// GRID: per-block partial, the last block to finish sums the partials in block order.
// !GRID (one CTA): the block sum. Thread 0 stores the results into out[k].
template <int NV, bool GRID>
__device__ __forceinline__ void reduce_store(double (&v)[NV], double *const (&out)[NV],
                                             const RedCtx &rc) {
    block_reduce<NV>(v);
    if (!GRID) {
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NV; k++)
                if (out[k]) *out[k] = v[k];
        __syncthreads();
        return;
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) rc.partials[k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        unsigned t = atomicAdd(rc.counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double w[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            w[k] = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
                w[k] += __ldcg(&rc.partials[k * gridDim.x + b]);
        }
        block_reduce<NV>(w);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < NV; k++)
                if (out[k]) *out[k] = w[k];
            *rc.counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------------------
// row kernels (sliced ELL, slot 0 = diagonal)
template <class T>
__device__ __forceinline__ T row_residual(const LevelDev<T> &L, int i, const T *f, const T *u) {
    const int s = i >> 5;
    const int base = L.sl[s] + (i & 31), width = (L.sl[s + 1] - L.sl[s]) >> 5;
    T acc = f[i];
    for (int k = 0; k < width; k++) {
        int c = L.col[base + 32 * k];
        if (c >= 0) acc -= L.val[base + 32 * k] * u[c];
    }
    return acc;
}

// Gauss-Seidel update of row i: u_i = (f_i - sum_{j != i} a_ij u_j) / a_ii
template <class T>
__device__ __forceinline__ void gs_row(const LevelDev<T> &L, int i, const T *f, T *u) {
    const int s = i >> 5;
    const int base = L.sl[s] + (i & 31), width = (L.sl[s + 1] - L.sl[s]) >> 5;
    T acc = f[i];
    const T d = L.val[base];
    for (int k = 1; k < width; k++) {
        int c = L.col[base + 32 * k];
        if (c >= 0) acc -= L.val[base + 32 * k] * u[c];
    }
    u[i] = acc / d;
}

// ---------------------------------------------------------------------------------------
// ops as row-parallel device functions: thread `tid` of `nth` (a grid or one CTA)
template <class T>
__device__ void op_zero(const LevelDev<T> &L, T *u, int tid, int nth) {
    for (int i = tid; i < L.n; i += nth) u[i] = T(0);
}

// one colour: independent blocks (finest level, rows of a block in sweep order) or rows
template <class T>
__device__ void op_gs(const LevelDev<T> &L, const Op &op, const T *f, T *u, int tid, int nth) {
    for (int b = op.i0 + tid; b < op.i1; b += nth) {
        if (L.fine) {
            const int r0 = L.bptr[b], r1 = L.bptr[b + 1];
            if (!op.backward)
                for (int i = r0; i < r1; i++) gs_row(L, i, f, u);
            else
                for (int i = r1 - 1; i >= r0; i--) gs_row(L, i, f, u);
        } else {
            gs_row(L, b, f, u);
        }
    }
}

// fc = P^t (f - A u): finest level sums the contiguous block of each aggregate; coarser
// levels the (up to four) children of each coarse cell (Sec. 4.3 explicit form)
template <class T>
__device__ void op_restrict(const LevelDev<T> &L, const T *f, const T *u, T *fc, int tid,
                            int nth) {
    for (int R = tid; R < L.nnext; R += nth) {
        T acc = T(0);
        if (L.fine) {
            for (int i = L.bptr[R]; i < L.bptr[R + 1]; i++) acc += row_residual(L, i, f, u);
        } else {
            const int4 ch = L.children[R];
            if (ch.x >= 0) acc += row_residual(L, ch.x, f, u);
            if (ch.y >= 0) acc += row_residual(L, ch.y, f, u);
            if (ch.z >= 0) acc += row_residual(L, ch.z, f, u);
            if (ch.w >= 0) acc += row_residual(L, ch.w, f, u);
        }
        fc[R] = acc;
    }
}

// u_i += e_{agg(i)} (Sec. 4.3 prolongation)
template <class T>
__device__ void op_prolong(const LevelDev<T> &L, const T *e, T *u, int tid, int nth) {
    for (int i = tid; i < L.n; i += nth) u[i] += e[L.parent[i]];
}

// e = A^{-1} rhs with the dense inverse of the coarsest level
template <class T>
__device__ void op_coarse(const LevelDev<T> &L, const T *f, T *e, int tid, int nth) {
    const int n = L.n;
    for (int i = tid; i < n; i += nth) {
        double s = 0.0;
        const T *a = L.Ainv + (size_t)i * n;
        for (int j = 0; j < n; j++) s += (double)a[j] * (double)f[j];
        e[i] = (T)s;
    }
}

template <class T, bool GRID>
__device__ void op_multidot(const LevelDev<T> &L, int i, const RedCtx &rc, int tid, int nth) {
    double v[kMaxKcycle] = {};
    const T *z = L.p[i];
    for (int r = tid; r < L.n; r += nth) {
        double zr = z[r];
#pragma unroll
        for (int j = 0; j < kMaxKcycle; j++)
            if (j < i) v[j] += zr * (double)L.q[j][r];
    }
    double *out[kMaxKcycle];
#pragma unroll
    for (int j = 0; j < kMaxKcycle; j++) out[j] = j < i ? &L.sc[SC_ZQ0 + j] : nullptr;
    reduce_store<kMaxKcycle, GRID>(v, out, rc);
}

// p_i = z + sum_j beta_ij p_j, beta_ij = -(z, p_j)_A / (p_j, p_j)_A  (Alg. 1, step 2)
template <class T>
__device__ void op_orth(const LevelDev<T> &L, int i, int tid, int nth) {
    double beta[kMaxKcycle];
#pragma unroll
    for (int j = 0; j < kMaxKcycle; j++) {
        double pq = L.sc[SC_PQ0 + j];
        beta[j] = (j < i && pq > 0.0) ? -L.sc[SC_ZQ0 + j] / pq : 0.0;
    }
    T *p = L.p[i];
    for (int r = tid; r < L.n; r += nth) {
        T acc = p[r];
#pragma unroll
        for (int j = 0; j < kMaxKcycle; j++)
            if (j < i) acc += (T)beta[j] * L.p[j][r];
        p[r] = acc;
    }
}

// q_i = A p_i; (p_i, q_i); (r_i, p_i) with r_0 = rhs
template <class T, bool GRID>
__device__ void op_spmv_dot(const LevelDev<T> &L, int i, const RedCtx &rc, int tid, int nth) {
    const T *p = L.p[i];
    T *q = L.q[i];
    const T *r = i == 0 ? L.rhs : L.r;
    double v[2] = {0.0, 0.0};
    for (int row = tid; row < L.n; row += nth) {
        const int s = row >> 5;
        const int base = L.sl[s] + (row & 31), width = (L.sl[s + 1] - L.sl[s]) >> 5;
        T acc = T(0);
        for (int k = 0; k < width; k++) {
            int c = L.col[base + 32 * k];
            if (c >= 0) acc += L.val[base + 32 * k] * p[c];
        }
        q[row] = acc;
        double pr = p[row];
        v[0] += pr * (double)acc;
        v[1] += (double)r[row] * pr;
    }
    double *out[2] = {&L.sc[SC_PQ0 + i], &L.sc[SC_RP0 + i]};
    reduce_store<2, GRID>(v, out, rc);
}

// alpha_i = (r_i, p_i) / (p_i, p_i)_A; u_{i+1} = u_i + alpha_i p_i; r_{i+1} = r_i - alpha_i q_i.
// Alg. 1 stops (alpha = 0 from then on) once (p_i, p_i)_A <= 0 or a residual is exactly zero.
template <class T, bool GRID>
__device__ void op_update(const LevelDev<T> &L, int i, int last, const RedCtx &rc, int tid,
                          int nth) {
    const double pq = L.sc[SC_PQ0 + i];
    const bool prev_stop =
        i > 0 && (L.sc[SC_STOP0 + i - 1] != 0.0 || L.sc[SC_RR0 + i - 1] == 0.0);
    const bool stopped = prev_stop || !(pq > 0.0) || !isfinite(pq);
    const double alpha = stopped ? 0.0 : L.sc[SC_RP0 + i] / pq;
    const T a = (T)alpha;
    const T *p = L.p[i];
    const T *q = L.q[i];
    const T *r_in = i == 0 ? L.rhs : L.r;
    T *e = L.e;
    double v[1] = {0.0};
    for (int row = tid; row < L.n; row += nth) {
        e[row] = (i == 0) ? a * p[row] : e[row] + a * p[row];
        if (!last) {
            T rn = r_in[row] - a * q[row];
            L.r[row] = rn;
            v[0] += (double)rn * (double)rn;
        }
    }
    if (!last) {
        double *out[1] = {&L.sc[SC_RR0 + i]};
        reduce_store<1, GRID>(v, out, rc);
    }
    if ((!GRID || blockIdx.x == 0) && threadIdx.x == 0) L.sc[SC_STOP0 + i] = stopped ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------------------
// multi-CTA kernels (one op per launch)
template <class T>
__global__ void k_zero(const LevelDev<T> *__restrict__ tab, Op op) {
    const LevelDev<T> &L = tab[op.level];
    op_zero(L, vec_of(L, op.usel), blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <class T>
__global__ void k_gs(const LevelDev<T> *__restrict__ tab, Op op) {
    const LevelDev<T> L = tab[op.level];
    op_gs(L, op, vec_of(L, op.fsel), vec_of(L, op.usel), blockIdx.x * blockDim.x + threadIdx.x,
          gridDim.x * blockDim.x);
}

template <class T>
__global__ void k_restrict(const LevelDev<T> *__restrict__ tab, Op op) {
    const LevelDev<T> L = tab[op.level];
    op_restrict(L, vec_of(L, op.fsel), vec_of(L, op.usel), tab[op.level + 1].rhs,
                blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <class T>
__global__ void k_prolong(const LevelDev<T> *__restrict__ tab, Op op) {
    const LevelDev<T> L = tab[op.level];
    op_prolong(L, tab[op.level + 1].e, vec_of(L, op.usel), blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x);
}

template <class T>
__global__ void k_coarse(const LevelDev<T> *__restrict__ tab, Op op) {
    const LevelDev<T> L = tab[op.level];
    op_coarse(L, L.rhs, L.e, threadIdx.x, blockDim.x);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const LevelDev<T> *__restrict__ tab,
                                                          Op op, RedCtx rc) {
    const LevelDev<T> L = tab[op.level];
    op_multidot<T, true>(L, op.step, rc, blockIdx.x * blockDim.x + threadIdx.x,
                         gridDim.x * blockDim.x);
}

template <class T>
__global__ void k_orth(const LevelDev<T> *__restrict__ tab, Op op) {
    const LevelDev<T> L = tab[op.level];
    op_orth(L, op.step, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads) k_spmv_dot(const LevelDev<T> *__restrict__ tab,
                                                          Op op, RedCtx rc) {
    const LevelDev<T> L = tab[op.level];
    op_spmv_dot<T, true>(L, op.step, rc, blockIdx.x * blockDim.x + threadIdx.x,
                         gridDim.x * blockDim.x);
}

template <class T>
__global__ void __launch_bounds__(kRedThreads) k_update(const LevelDev<T> *__restrict__ tab,
                                                        Op op, RedCtx rc) {
    const LevelDev<T> L = tab[op.level];
    op_update<T, true>(L, op.step, op.last, rc, blockIdx.x * blockDim.x + threadIdx.x,
                       gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------------------
// single-CTA interpreter of a program of ops (levels from the tail level down)
constexpr int kTailThreads = 512;

template <class T>
__global__ void __launch_bounds__(kTailThreads) k_tail(const LevelDev<T> *__restrict__ tab,
                                                       const Op *__restrict__ prog, int nops) {
    const int tid = threadIdx.x, nth = blockDim.x;
    RedCtx rc{nullptr, nullptr};
    for (int k = 0; k < nops; k++) {
        const Op op = prog[k];
        const LevelDev<T> &L = tab[op.level];
        switch (op.kind) {
            case OP_ZERO: op_zero(L, vec_of(L, op.usel), tid, nth); break;
            case OP_GS: op_gs(L, op, vec_of(L, op.fsel), vec_of(L, op.usel), tid, nth); break;
            case OP_RESTRICT:
                op_restrict(L, vec_of(L, op.fsel), vec_of(L, op.usel), tab[op.level + 1].rhs, tid, nth);
                break;
            case OP_PROLONG: op_prolong(L, tab[op.level + 1].e, vec_of(L, op.usel), tid, nth); break;
            case OP_COARSE: op_coarse(L, L.rhs, L.e, tid, nth); break;
            case OP_MULTIDOT: op_multidot<T, false>(L, op.step, rc, tid, nth); break;
            case OP_ORTH: op_orth(L, op.step, tid, nth); break;
            case OP_SPMV_DOT: op_spmv_dot<T, false>(L, op.step, rc, tid, nth); break;
            case OP_UPDATE: op_update<T, false>(L, op.step, op.last, rc, tid, nth); break;
        }
        __syncthreads();
    }
}

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
    reduce_store<1, true>(a, o, rc);
}

// t = b - A x, (t, t) -> out
__global__ void __launch_bounds__(kRedThreads) k_true_residual(LevelDev<double> L,
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
    reduce_store<1, true>(a, o, rc);
}

// outer scalars: osc[0] = (b,b), osc[1] = (r,r), osc[2] = stop flag, osc[3] = (p_i, A p_i),
// osc[4] = (r, p_i), osc[8 + j] = (z, A p_j), osc[8 + max_iters + j] = (p_j, A p_j)
enum : int { OS_BB = 0, OS_RR = 1, OS_STOP = 2, OS_PQ = 3, OS_RP = 4, OS_TT = 5, OS_ZQ = 8 };

// (z, q_j) for all j < it: each block loops over j; the last block reduces every j
__global__ void __launch_bounds__(kRedThreads) k_outer_multidot(int n, const double *__restrict__ z,
                                                                double *const *__restrict__ Q,
                                                                const int *__restrict__ it_ptr,
                                                                double *osc, RedCtx rc) {
    const int it = *it_ptr;
    __shared__ bool last;
    for (int j = 0; j < it; j++) {
        const double *q = Q[j];
        double a[1] = {0.0};
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
            a[0] += z[i] * q[i];
        block_reduce<1>(a);
        if (threadIdx.x == 0) rc.partials[(size_t)j * gridDim.x + blockIdx.x] = a[0];
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(rc.counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = 0; j < it; j++) {
        double w[1] = {0.0};
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            w[0] += __ldcg(&rc.partials[(size_t)j * gridDim.x + b]);
        block_reduce<1>(w);
        if (threadIdx.x == 0) osc[OS_ZQ + j] = w[0];
    }
    if (threadIdx.x == 0) *rc.counter = 0u;
}

// p_it = z - sum_j (z, q_j) / (p_j, q_j) p_j   (Alg. 1 step 2 on the finest level)
__global__ void k_outer_orth(int n, const double *__restrict__ z, double *const *__restrict__ P,
                             const int *__restrict__ it_ptr, const double *__restrict__ osc,
                             const double *__restrict__ opq) {
    const int it = *it_ptr;
    double *p = P[it];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = z[i];
        for (int j = 0; j < it; j++) acc += (-osc[OS_ZQ + j] / opq[j]) * P[j][i];
        p[i] = acc;
    }
}

// q = A p, (p, q) -> osc[PQ] and opq[it], (r, p) -> osc[RP]
__global__ void __launch_bounds__(kRedThreads) k_outer_spmv_dot(LevelDev<double> L,
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
        const int s = row >> 5;
        const int base = L.sl[s] + (row & 31), width = (L.sl[s + 1] - L.sl[s]) >> 5;
        double acc = 0.0;
        for (int k = 0; k < width; k++) {
            int c = L.col[base + 32 * k];
            if (c >= 0) acc += L.val[base + 32 * k] * p[c];
        }
        q[row] = acc;
        v[0] += p[row] * acc;
        v[1] += r[row] * p[row];
    }
    double *out[2] = {&opq[it], &osc[OS_RP]};
    reduce_store<2, true>(v, out, rc);
}

// alpha = (r, p) / (p, Ap); x += alpha p; r -= alpha q; (r, r); it++
__global__ void __launch_bounds__(kRedThreads) k_outer_update(int n, double *const *__restrict__ P,
                                                              double *const *__restrict__ Q,
                                                              int *it_ptr, double *__restrict__ x,
                                                              double *__restrict__ r, double *osc,
                                                              const double *__restrict__ opq,
                                                              RedCtx rc) {
    const int it = *it_ptr;
    const double pq = opq[it];
    const bool bad = !(pq > 0.0) || !isfinite(pq);
    const double alpha = bad ? 0.0 : osc[OS_RP] / pq;
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
    reduce_store<1, true>(v, out, rc);
    if (blockIdx.x == 0 && threadIdx.x == 0 && bad) osc[OS_STOP] = 1.0;
}

__global__ void k_bump(int *it_ptr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *it_ptr += 1;
}

// =======================================================================================
// diagnostics: CUDA-event timing of every op and its algorithmic bytes
thread_local int64_t g_launches = 0;

enum : int { K_TAIL = 9, K_OUTER_MULTIDOT, K_OUTER_ORTH, K_OUTER_SPMV_DOT, K_OUTER_UPDATE,
             K_TRUE_RESIDUAL, K_NUM };

const char *kernel_name(int kind) {
    static const char *names[K_NUM] = {"zero", "gs_colour", "resid_restrict", "prolong_correct",
                                       "coarse_solve", "alg1_multidot", "alg1_orth",
                                       "alg1_spmv_dot", "alg1_update", "tail_cta",
                                       "outer_multidot", "outer_orth", "outer_spmv_dot",
                                       "outer_update", "true_residual"};
    return (kind >= 0 && kind < K_NUM) ? names[kind] : "unknown";
}

struct Profiler {
    struct Rec {
        int kind, level;
        double bytes;
        cudaEvent_t a, b;
    };
    bool on = false;
    std::vector<Rec> graph_recs;  // event nodes inside the captured cycle graph
    std::vector<Rec> pending;     // direct launches not yet harvested
    std::vector<Rec> graph_old;   // records of superseded graphs (events freed at the end)
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
    Rec begin(int kind, int level, double bytes, cudaStream_t s) {
        Rec r{kind, level, bytes, nullptr, nullptr};
        AMG_CUDA(cudaEventCreate(&r.a));
        AMG_CUDA(cudaEventCreate(&r.b));
        // external event nodes inside a stream capture, plain records otherwise
        if (is_capturing(s)) AMG_CUDA(cudaEventRecordWithFlags(r.a, s, cudaEventRecordExternal));
        else AMG_CUDA(cudaEventRecord(r.a, s));
        return r;
    }
    void end(Rec &r, cudaStream_t s, bool capturing) {
        if (capturing) AMG_CUDA(cudaEventRecordWithFlags(r.b, s, cudaEventRecordExternal));
        else AMG_CUDA(cudaEventRecord(r.b, s));
        (capturing ? graph_recs : pending).push_back(r);
    }
    static bool is_capturing(cudaStream_t s) {
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
        return st == cudaStreamCaptureStatusActive;
    }
    void add(const Rec &r) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        Acc &a = slot(r.kind, r.level);
        a.launches++;
        a.ms += ms;
        a.bytes += r.bytes;
    }
    void harvest_graph() {
        for (auto &r : graph_recs) add(r);
    }
    void harvest_pending() {
        for (auto &r : pending) {
            add(r);
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        pending.clear();
    }
    ~Profiler() {
        for (auto *v : {&graph_recs, &pending, &graph_old})
            for (auto &r : *v) {
                cudaEventDestroy(r.a);
                cudaEventDestroy(r.b);
            }
    }
};

void profiler_enable(amg_hierarchy *h, bool on) {
    if (!h->prof) h->prof = new Profiler();
    h->prof->on = on;
    if (h->cycle_graph) {  // recapture so the graph carries (or drops) the event nodes
        cudaGraphExecDestroy(h->cycle_graph);
        h->cycle_graph = nullptr;
        for (auto &r : h->prof->graph_recs) h->prof->graph_old.push_back(r);
        h->prof->graph_recs.clear();
    }
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

static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st == cudaStreamCaptureStatusActive;
}

// algorithmic bytes of one op: every array the op must touch, once, at its width
// (w = value width, 4-byte column indices; padding of the sliced ELL is not counted)
static double op_bytes(const amg_hierarchy *h, const Op &op, int w) {
    const Level &lv = h->lev[op.level];
    const double n = lv.n, nnz = (double)lv.A.stored;
    const double nn = op.level + 1 < h->nlev ? h->lev[op.level + 1].n : 0;
    switch (op.kind) {
        case OP_ZERO: return w * n;
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
namespace {

template <class T>
Vecs<T> &vecs(Level &lv);
template <>
Vecs<double> &vecs<double>(Level &lv) { return lv.v64; }
template <>
Vecs<float> &vecs<float>(Level &lv) { return lv.v32; }

int red_grid(int64_t n) { return (int)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, (n + kRedThreads - 1) / kRedThreads)); }
int ew_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// Walks Alg. 1 / Alg. 2 and either launches or records each op.
template <class T>
struct Emitter {
    amg_hierarchy *h;
    const LevelDev<T> *tab;        // device table
    std::vector<Op> *record;       // non-null: record ops (tail program)
    int tail_level;                // levels >= tail_level are recorded into the tail program
    const Op *tail_prog = nullptr; // device program of the tail
    int tail_nops = 0;
    double tail_bytes = 0;
    RedCtx rc;

    void launch(const Op &op) {
        cudaStream_t s = h->stream;
        const Level &lv = h->lev[op.level];
        Profiler::Rec rec{};
        const bool prof = profiling(h);
        if (prof) rec = h->prof->begin(op.kind, op.level, op_bytes(h, op, sizeof(T)), s);
        switch (op.kind) {
            case OP_ZERO: k_zero<T><<<ew_grid(lv.n), 256, 0, s>>>(tab, op); break;
            case OP_GS: k_gs<T><<<ew_grid(op.i1 - op.i0), 256, 0, s>>>(tab, op); break;
            case OP_RESTRICT: k_restrict<T><<<ew_grid(h->lev[op.level + 1].n), 256, 0, s>>>(tab, op); break;
            case OP_PROLONG: k_prolong<T><<<ew_grid(lv.n), 256, 0, s>>>(tab, op); break;
            case OP_COARSE: k_coarse<T><<<1, 256, 0, s>>>(tab, op); break;
            case OP_MULTIDOT: k_multidot<T><<<red_grid(lv.n), kRedThreads, 0, s>>>(tab, op, rc); break;
            case OP_ORTH: k_orth<T><<<ew_grid(lv.n), 256, 0, s>>>(tab, op); break;
            case OP_SPMV_DOT: k_spmv_dot<T><<<red_grid(lv.n), kRedThreads, 0, s>>>(tab, op, rc); break;
            case OP_UPDATE: k_update<T><<<red_grid(lv.n), kRedThreads, 0, s>>>(tab, op, rc); break;
        }
        AMG_LAUNCH_CHECK();
        if (prof) h->prof->end(rec, s, capturing(s));
    }

    void emit(const Op &op) {
        if (record) {
            record->push_back(op);
            tail_bytes += op_bytes(h, op, sizeof(T));
        } else {
            launch(op);
        }
    }

    Op mk(int kind, int level) {
        Op o;
        std::memset(&o, 0, sizeof o);
        o.kind = kind;
        o.level = level;
        return o;
    }

    // z = B^_l [f] (Alg. 2)
    void bhat(int l, int fsel, int zsel) {
        Level &lv = h->lev[l];
        Op z = mk(OP_ZERO, l);
        z.usel = zsel;
        emit(z);
        const std::vector<int> &ranges = (l == 0) ? lv.color_blocks : lv.color_rows;
        const int nc = (int)ranges.size() - 1;
        for (int c = 0; c < nc; c++) {  // pre-smoothing u1 = R_k f, colours ascending
            if (ranges[c + 1] == ranges[c]) continue;
            Op g = mk(OP_GS, l);
            g.i0 = ranges[c];
            g.i1 = ranges[c + 1];
            g.backward = 0;
            g.fsel = fsel;
            g.usel = zsel;
            emit(g);
        }
        Op rs = mk(OP_RESTRICT, l);  // next.rhs = P^t (f - A u1)
        rs.fsel = fsel;
        rs.usel = zsel;
        emit(rs);
        btilde(l + 1);               // next.e = B~_{k-1}[next.rhs]
        Op pr = mk(OP_PROLONG, l);   // u2 = u1 + P e
        pr.usel = zsel;
        emit(pr);
        for (int c = nc - 1; c >= 0; c--) {  // post-smoothing: colours descending
            if (ranges[c + 1] == ranges[c]) continue;
            Op g = mk(OP_GS, l);
            g.i0 = ranges[c];
            g.i1 = ranges[c + 1];
            g.backward = 1;
            g.fsel = fsel;
            g.usel = zsel;
            emit(g);
        }
    }

    // e = B~_l [rhs] (Alg. 1 with kcycle_n steps; exact on the coarsest level)
    void btilde(int l) {
        if (!record && l == tail_level) {
            // the whole recursion from here runs in one CTA (the program is B~ of this level)
            Profiler::Rec rec{};
            const bool prof = profiling(h);
            if (prof) rec = h->prof->begin(K_TAIL, l, tail_bytes, h->stream);
            k_tail<T><<<1, kTailThreads, 0, h->stream>>>(tab, tail_prog, tail_nops);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, h->stream, capturing(h->stream));
            return;
        }
        Level &lv = h->lev[l];
        if (lv.coarsest) {
            emit(mk(OP_COARSE, l));
            return;
        }
        const int n = h->opt.kcycle_n;
        for (int i = 0; i < n; i++) {
            bhat(l, i == 0 ? V_RHS : V_R, V_P0 + i);
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
            emit(up);
        }
    }
};

template <class T>
void fill_tables(amg_hierarchy *h) {
    std::vector<LevelDev<T>> tab(h->nlev);
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        LevelDev<T> &d = tab[l];
        std::memset(&d, 0, sizeof d);
        d.n = lv.n;
        d.fine = (l == 0) ? 1 : 0;
        d.sl = lv.A.sl_ptr;
        d.col = lv.A.col;
        if constexpr (sizeof(T) == 8) d.val = (const T *)lv.A.val;
        else d.val = (const T *)lv.A.val32;
        d.bptr = lv.bptr;
        d.parent = lv.parent;
        d.children = (l + 1 < h->nlev) ? h->lev[l + 1].children : nullptr;
        if constexpr (sizeof(T) == 8) d.Ainv = (const T *)lv.Ainv;
        else d.Ainv = (const T *)lv.Ainv32;
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
    void *&dst = (sizeof(T) == 8) ? h->lev_tab64 : h->lev_tab32;
    if (!dst) dst = halloc<LevelDev<T>>(h, h->nlev);
    AMG_CUDA(cudaMemcpyAsync(dst, tab.data(), sizeof(LevelDev<T>) * h->nlev,
                             cudaMemcpyHostToDevice, h->stream));
}

int tail_rows() {
    static int v = [] {
        const char *e = getenv("AMG_TAIL_ROWS");
        return e ? atoi(e) : 4096;
    }();
    return v;
}

template <class T>
void build_tail(amg_hierarchy *h) {
    // the tail starts at the first coarse level (>= 1) with at most tail_rows() rows
    int tl = h->nlev;
    for (int l = 1; l < h->nlev; l++)
        if (h->lev[l].n <= tail_rows()) {
            tl = l;
            break;
        }
    h->tail_level = tl;
    if (tl >= h->nlev) return;
    std::vector<Op> prog;
    Emitter<T> em{h, nullptr, &prog, tl};
    em.btilde(tl);
    Op *d = halloc<Op>(h, prog.size());
    AMG_CUDA(cudaMemcpyAsync(d, prog.data(), sizeof(Op) * prog.size(), cudaMemcpyHostToDevice,
                             h->stream));
    if (sizeof(T) == 8) {
        h->tail_prog64 = d;
        h->tail_nops64 = (int)prog.size();
        h->tail_bytes64 = em.tail_bytes;
    } else {
        h->tail_prog32 = d;
        h->tail_nops32 = (int)prog.size();
        h->tail_bytes32 = em.tail_bytes;
    }
}

template <class T>
void alloc_vecs(amg_hierarchy *h) {
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        Vecs<T> &v = vecs<T>(lv);
        int n = lv.n;
        if (l > 0) {
            v.rhs = halloc<T>(h, n);
            v.e = halloc<T>(h, n);
        }
        if (l > 0 && !lv.coarsest) {
            v.r = halloc<T>(h, n);
            for (int i = 0; i < h->opt.kcycle_n; i++) {
                v.p[i] = halloc<T>(h, n);
                v.q[i] = halloc<T>(h, n);
            }
        }
    }
}

template <class T>
Emitter<T> make_emitter(amg_hierarchy *h) {
    Emitter<T> em{h, (const LevelDev<T> *)((sizeof(T) == 8) ? h->lev_tab64 : h->lev_tab32),
                  nullptr, h->tail_level};
    em.tail_prog = (const Op *)((sizeof(T) == 8) ? h->tail_prog64 : h->tail_prog32);
    em.tail_nops = (sizeof(T) == 8) ? h->tail_nops64 : h->tail_nops32;
    em.tail_bytes = (sizeof(T) == 8) ? h->tail_bytes64 : h->tail_bytes32;
    em.rc = RedCtx{h->red_partials, h->red_counter};
    return em;
}

void ensure_fp32(amg_hierarchy *h) {
    if (h->fp32_ready) return;
    cudaStream_t s = h->stream;
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        lv.A.val32 = halloc<float>(h, lv.A.padded);
        k_convert<double, float><<<nblocks_for(lv.A.padded, 256), 256, 0, s>>>(
            (int)lv.A.padded, lv.A.val, lv.A.val32);
        AMG_LAUNCH_CHECK();
    }
    alloc_vecs<float>(h);
    h->r32 = halloc<float>(h, h->N);
    h->z32 = halloc<float>(h, h->N);
    // the fine level's cycle vectors
    fill_tables<float>(h);
    build_tail<float>(h);
    h->fp32_ready = true;
}

// z (FP64, pi order) = B^_0 [r]; level-0 input/output buffers are set in the table
template <class T>
void record_cycle(amg_hierarchy *h) {
    Emitter<T> em = make_emitter<T>(h);
    em.bhat(0, V_RHS, V_E);
}

}  // namespace

// capture the preconditioner application B^_fine into a CUDA graph (once per precision)
static void ensure_cycle_graph(amg_hierarchy *h, int prec) {
    if (h->cycle_graph && h->cycle_graph_prec == prec) return;
    if (h->cycle_graph) {
        cudaGraphExecDestroy(h->cycle_graph);
        h->cycle_graph = nullptr;
    }
    cudaStream_t s = h->stream;
    AMG_CUDA(cudaStreamSynchronize(s));
    cudaGraph_t g;
    const int64_t launches_before = g_launches;
    AMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
        if (prec == AMG_FP32) record_cycle<float>(h);
        else record_cycle<double>(h);
    } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(s, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        throw;
    }
    AMG_CUDA(cudaStreamEndCapture(s, &g));
    h->graph_nodes = g_launches - launches_before;  // captured, not yet executed
    g_launches = launches_before;
    cudaError_t e = cudaGraphInstantiate(&h->cycle_graph, g, 0);
    cudaGraphDestroy(g);
    AMG_CUDA(e);
    h->cycle_graph_prec = prec;
}

void allocate_solve_workspace(amg_hierarchy *h) {
    const int n = (int)h->N;
    h->red_partials = halloc<double>(h, (size_t)kRedBlocks * std::max(8, h->opt.max_iters + 8));
    h->red_counter = halloc<unsigned int>(h, 1);
    AMG_CUDA(cudaMemsetAsync(h->red_counter, 0, sizeof(unsigned int), h->stream));
    alloc_vecs<double>(h);
    // level-0 cycle input / output live in the outer solver's vectors
    h->xo = halloc<double>(h, n);
    h->ro = halloc<double>(h, n);
    h->zo = halloc<double>(h, n);
    h->to = halloc<double>(h, n);
    h->bo = halloc<double>(h, n);
    h->lev[0].v64.rhs = h->ro;
    h->lev[0].v64.e = h->zo;
    h->osc = halloc<double>(h, OS_ZQ + 2 * (size_t)h->opt.max_iters + 8);
    h->oit = halloc<int>(h, 1);
    h->dP = halloc<double *>(h, h->opt.max_iters);
    h->dQ = halloc<double *>(h, h->opt.max_iters);
    AMG_CUDA(cudaMallocHost(&h->h_pinned, 64 * sizeof(double)));
    fill_tables<double>(h);
    build_tail<double>(h);
}

static void ensure_directions(amg_hierarchy *h, int count) {
    const int n = (int)h->N;
    const int chunk = 16;
    int old = (int)h->P.size();
    if (count <= old) return;
    int target = std::min(h->opt.max_iters, ((count + chunk - 1) / chunk) * chunk);
    for (int j = old; j < target; j++) {
        h->P.push_back(halloc<double>(h, n));
        h->Q.push_back(halloc<double>(h, n));
    }
    AMG_CUDA(cudaMemcpyAsync(h->dP, h->P.data(), sizeof(double *) * target, cudaMemcpyHostToDevice,
                             h->stream));
    AMG_CUDA(cudaMemcpyAsync(h->dQ, h->Q.data(), sizeof(double *) * target, cudaMemcpyHostToDevice,
                             h->stream));
}

static LevelDev<double> fine_view(amg_hierarchy *h) {
    LevelDev<double> L;
    std::memset(&L, 0, sizeof L);
    Level &lv = h->lev[0];
    L.n = lv.n;
    L.sl = lv.A.sl_ptr;
    L.col = lv.A.col;
    L.val = lv.A.val;
    return L;
}

// one application of B^_0 to h->ro (FP64) into h->zo (FP64)
static void apply_preconditioner(amg_hierarchy *h) {
    cudaStream_t s = h->stream;
    const int n = (int)h->N;
    if (h->nlev == 1) {  // exact solve
        LevelDev<double> L = fine_view(h);
        (void)L;
        Op op;
        std::memset(&op, 0, sizeof op);
        // rhs = ro, e = zo are the level-0 buffers of the table
        k_coarse<double><<<1, 256, 0, s>>>((const LevelDev<double> *)h->lev_tab64, op);
        AMG_LAUNCH_CHECK();
        return;
    }
    int prec = h->opt.cycle_prec;
    ensure_cycle_graph(h, prec);
    if (prec == AMG_FP32) {
        k_convert<double, float><<<nblocks_for(n, 256), 256, 0, s>>>(n, h->ro, h->r32);
        AMG_LAUNCH_CHECK();
    }
    AMG_CUDA(cudaGraphLaunch(h->cycle_graph, s));
    g_launches += h->graph_nodes;
    if (prec == AMG_FP32) {
        k_convert<float, double><<<nblocks_for(n, 256), 256, 0, s>>>(n, h->z32, h->zo);
        AMG_LAUNCH_CHECK();
    }
}

static void prepare_precision(amg_hierarchy *h) {
    if (h->opt.cycle_prec == AMG_FP32 && h->nlev > 1) {
        ensure_fp32(h);
        // FP32 level-0 in/out buffers are the conversion buffers
        h->lev[0].v32.rhs = h->r32;
        h->lev[0].v32.e = h->z32;
        fill_tables<float>(h);
    }
}

int solve(amg_hierarchy *h, const double *b_nat, double tol, double *x_nat, int *iters,
          double *relres) {
    cudaStream_t s = h->stream;
    const int n = (int)h->N;
    const int maxit = h->opt.max_iters;
    Level &F = h->lev[0];
    RedCtx rc{h->red_partials, h->red_counter};
    const bool prof = profiling(h);
    prepare_precision(h);
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
    if (!std::isfinite(bn)) {
        throw Error{AMG_ERR_INVALID_ARG, "non-finite right-hand side"};
    }
    if (bn == 0.0) {
        status = AMG_OK;
        rel = 0.0;
    } else {
        double *opq = h->osc + OS_ZQ + maxit;
        LevelDev<double> Lf = fine_view(h);
        for (it = 0; it < maxit;) {
            ensure_directions(h, it + 1);
            apply_preconditioner(h);  // zo = B^[ro]
            const double nd = n, nnz = (double)F.A.stored;
            Profiler::Rec rec{};
            if (prof) rec = h->prof->begin(K_OUTER_MULTIDOT, 0, 8.0 * nd * (1 + it), s);
            k_outer_multidot<<<red_grid(n), kRedThreads, 0, s>>>(n, h->zo, h->dQ, h->oit, h->osc, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s, false);
            if (prof) rec = h->prof->begin(K_OUTER_ORTH, 0, 8.0 * nd * (2 + it), s);
            k_outer_orth<<<ew_grid(n), 256, 0, s>>>(n, h->zo, h->dP, h->oit, h->osc, opq);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s, false);
            if (prof) rec = h->prof->begin(K_OUTER_SPMV_DOT, 0, 12.0 * nnz + 24.0 * nd, s);
            k_outer_spmv_dot<<<red_grid(n), kRedThreads, 0, s>>>(Lf, h->dP, h->dQ, h->oit, h->ro,
                                                                 h->osc, opq, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s, false);
            if (prof) rec = h->prof->begin(K_OUTER_UPDATE, 0, 48.0 * nd, s);
            k_outer_update<<<red_grid(n), kRedThreads, 0, s>>>(n, h->dP, h->dQ, h->oit, h->xo,
                                                               h->ro, h->osc, opq, rc);
            AMG_LAUNCH_CHECK();
            if (prof) h->prof->end(rec, s, false);
            k_bump<<<1, 32, 0, s>>>(h->oit);
            AMG_LAUNCH_CHECK();
            AMG_CUDA(cudaMemcpyAsync(h->h_pinned, h->osc, sizeof(double) * 8,
                                     cudaMemcpyDeviceToHost, s));
            AMG_CUDA(cudaStreamSynchronize(s));
            if (prof) {
                h->prof->harvest_graph();
                h->prof->harvest_pending();
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

// z = B^_level [f] in natural order (FP64), through the same ops as the solve
void apply_cycle_level(amg_hierarchy *h, int level, const double *f_nat, double *z_nat) {
    cudaStream_t s = h->stream;
    Level &lv = h->lev[level];
    const int n = lv.n;
    double *zbuf = level == 0 ? h->zo : lv.v64.p[0];
    double *fbuf = level == 0 ? h->ro : lv.v64.rhs;
    if (lv.coarsest) {
        // B^_1 = A_1^{-1}: on the coarsest level the cycle is the exact solve
        k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, f_nat, lv.v64.rhs ? lv.v64.rhs : h->ro);
        AMG_LAUNCH_CHECK();
        Op op;
        std::memset(&op, 0, sizeof op);
        op.level = level;
        k_coarse<double><<<1, 256, 0, s>>>((const LevelDev<double> *)h->lev_tab64, op);
        AMG_LAUNCH_CHECK();
        double *e = level == 0 ? h->zo : lv.v64.e;
        k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, e, z_nat);
        AMG_LAUNCH_CHECK();
        AMG_CUDA(cudaStreamSynchronize(s));
        return;
    }
    k_gather<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, f_nat, fbuf);
    AMG_LAUNCH_CHECK();
    Emitter<double> em = make_emitter<double>(h);
    if (level == 0) em.bhat(0, V_RHS, V_E);
    else em.bhat(level, V_RHS, V_P0);
    k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, zbuf, z_nat);
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
    Emitter<double> em = make_emitter<double>(h);
    const std::vector<int> &ranges = (level == 0) ? lv.color_blocks : lv.color_rows;
    const int nc = (int)ranges.size() - 1;
    for (int k = 0; k < nc; k++) {
        int c = backward ? nc - 1 - k : k;
        if (ranges[c + 1] == ranges[c]) continue;
        Op g = em.mk(OP_GS, level);
        g.i0 = ranges[c];
        g.i1 = ranges[c + 1];
        g.backward = backward;
        g.fsel = V_RHS;
        g.usel = V_E;
        em.launch(g);
    }
    k_scatter<<<nblocks_for(n, 256), 256, 0, s>>>(n, lv.nat, ubuf, u_nat);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace amg
