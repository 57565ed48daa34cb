// Batched solves: many independent systems of uneven sizes, each with its own hierarchy
// (built by the single-system setup), solved by one persistent kernel.
//
// The paper solves one system at a time. A batch of small and mid-size systems would leave
// the GPU almost idle if each ran the grid-wide cycle kernel in turn (those solves are
// latency-bound: a few thousand dependent steps, each a grid barrier). Here every CTA takes
// the next slot from a queue (largest systems first) and runs that system's whole solve: the
// outer flexible CG (Alg. 1 on the finest level, FP64, full orthogonalisation: a system whose
// allocated directions fill up is resumed with more in a further launch) and, every
// iteration, the AMLI-cycle B^_0 (Alg. 2, with Alg. 1 on the coarse levels and the exact
// coarsest solve) on levels that stay in HBM / L2. The cycle ops are the same device
// functions as the single-system kernel (cycle_ops.cuh) on the same level data, walked as a
// state machine over the levels. The device code is in batch_kernel.cuh.
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

#include "batch_kernel.cuh"

namespace amg {

// ---------------------------------------------------------------------------------------
// host side

struct BatchShape {
    int threads, per_sm;
};
static const BatchShape kShapes[] = {{1024, 1}, {512, 2}, {512, 1}, {256, 4}};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

// the kernel of launch shape `shape`, with the big-aggregate phase if `graded`
template <class T>
void *batch_kernel(int shape, bool graded) {
    return graded ? batch_kernel_graded(sizeof(T) == 4, shape) : batch_kernel_of<T, false>(shape);
}

struct BatchEngine {
    std::vector<amg_hierarchy *> hs;  // not owned
    std::vector<int64_t> row_off;
    int nprob = 0;
    int64_t N = 0;
    bool fp32 = false;
    bool graded = false;  // a system has big aggregates: the kernels with that phase
    int kc = 2, maxit = 200;
    int nu = 1 + 256;  // nu_pre + 256 nu_post
    // host-set team-barrier fault (amg_debug_batch_barrier_fault): 0 = none
    int64_t dbg_bar_limit_ns = 0;
    int dbg_bar_extra = 0;
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    void *probs = nullptr;  // BatchProb<T>[nprob]
    int *next = nullptr, *iters = nullptr, *status = nullptr;
    int *resume = nullptr;     // per system: the step a resumed solve continues at (0: fresh)
    int4 *rslots = nullptr;    // the queue of a resumed launch
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
    std::vector<int> last_iters;   // every system's outer steps in the last solve
    std::vector<double> cyc_bytes; // algorithmic bytes of one B^_0 per system (on demand)
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
    ensure_directions(h, std::min(h->opt.max_iters, kBatchDirs));
    w.pq = halloc<double>(h, h->opt.max_iters);
    w.bo = halloc<double>(h, n);
    w.xo = halloc<double>(h, n);
    w.to = halloc<double>(h, n);
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
    const Level &F = h->lev[0];
    std::vector<int4> bigr;
    if (F.nbig > 0) {  // the big blocks of every finest-level colour (as the grid's programs)
        for (size_t c = 0; c + 1 < F.color_big.size(); c++)
            bigr.push_back(make_int4(F.color_big[c], F.color_bigc[c], F.color_big[c + 1], 0));
        w.bigr = halloc<int4>(h, bigr.size());
        AMG_CUDA(cudaMemcpyAsync(w.bigr, bigr.data(), sizeof(int4) * bigr.size(),
                                 cudaMemcpyHostToDevice, h->stream));
    }
    AMG_CUDA(cudaStreamSynchronize(h->stream));  // colors and bigr are locals
    return w;
}

void batch_prepare(amg_hierarchy *h) {
    prepare_cycle(h);
    batch_ws(h);
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
        B.Pt = h->dP;
        B.Qt = h->dQ;
        B.pq = w.pq;
        B.cap = (int)h->P.size();
        B.bigr = w.bigr;
        B.nbig = F.nbig;
    }
    BatchProb<T> *dp = balloc<BatchProb<T>>(E, np);
    AMG_CUDA(cudaMemcpyAsync(dp, hp.data(), sizeof(BatchProb<T>) * np, cudaMemcpyHostToDevice,
                             E->stream));
    E->probs = dp;
    int nsm = 0;
    AMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, E->hs[0]->device));
    for (int s = 0; s < kNumShapes; s++) {
        int per = 0;
        AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<T>(s, E->graded),
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
            E->graded = E->graded || h->lev[0].nbig > 0;
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
        E->resume = balloc<int>(E, E->nprob);
        E->rslots = balloc<int4>(E, (size_t)E->nprob * kMaxTeam);
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

// queue and team counters reset + the persistent kernel, on E->stream. Without rslots: every
// system from the start; with rslots: the nr slots of the systems that are resumed.
static void launch_batch(BatchEngine *E, int shape, const double *b, double *x, double tol,
                         const int4 *rslots = nullptr, int nr = 0) {
    AMG_CUDA(cudaMemsetAsync(E->next, 0, sizeof(int), E->stream));
    AMG_CUDA(cudaMemsetAsync(E->team_bar, 0, sizeof(unsigned long long) * E->nprob, E->stream));
    AMG_CUDA(cudaMemsetAsync(E->team_cnt, 0, sizeof(unsigned int) * E->nprob, E->stream));
    if (!rslots) AMG_CUDA(cudaMemsetAsync(E->resume, 0, sizeof(int) * E->nprob, E->stream));
    void *kern = E->fp32 ? batch_kernel<float>(shape, E->graded)
                         : batch_kernel<double>(shape, E->graded);
    const int4 *sl = rslots ? rslots : E->slots[shape];
    int nslots = rslots ? nr : E->nslots[shape], kc = E->kc, nu = E->nu, maxit = E->maxit;
    unsigned long long limit_ns =
        E->dbg_bar_limit_ns > 0 ? (unsigned long long)E->dbg_bar_limit_ns : kBarrierLimitNs;
    int extra = E->dbg_bar_extra;
    void *args[] = {&E->probs,  &sl,         &nslots,     &E->next,    &kc,  &nu,
                    &b,         &x,          &tol,        &maxit,      &E->iters,
                    &E->relres, &E->status,  &E->t_start, &E->t_end,   &E->team_bar,
                    &E->team_part, &E->team_cnt, &limit_ns, &extra, &E->resume};
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

// Systems whose kept outer directions filled their allocation (status kBatchResume) get
// twice as many (at most max_iters) and continue in one more launch, with their teams: the
// flexible CG keeps every direction, as the single-system solver does. Returns whether a
// launch was made.
static bool resume_full(BatchEngine *E, const std::vector<int> &st, const double *b, double *x,
                        double tol) {
    std::vector<int4> sl;
    std::vector<int> caps;
    caps.reserve(E->nprob);  // (no reallocation: the copies below read from it)
    const int shape = E->shape;
    for (int p : E->ord) {
        if (st[p] != kBatchResume) continue;
        amg_hierarchy *h = E->hs[p];
        const int cap = (int)h->P.size();
        caps.push_back(ensure_directions(h, std::min(h->opt.max_iters, 2 * cap)));
        if (caps.back() <= cap) throw Error{AMG_ERR_UNSUPPORTED, "batched solve: no directions to add"};
        const int K = E->team[shape][p];
        for (int r = 0; r < K; r++) sl.push_back(make_int4(p, r, K, 0));
        // the system's capacity in its entry of the device table
        char *entry = (char *)E->probs + (size_t)p * (E->fp32 ? sizeof(BatchProb<float>)
                                                                : sizeof(BatchProb<double>));
        const size_t off = E->fp32 ? offsetof(BatchProb<float>, cap) : offsetof(BatchProb<double>, cap);
        AMG_CUDA(cudaMemcpyAsync(entry + off, &caps.back(), sizeof(int), cudaMemcpyHostToDevice,
                                 E->stream));
    }
    if (sl.empty()) return false;
    AMG_CUDA(cudaMemcpyAsync(E->rslots, sl.data(), sizeof(int4) * sl.size(),
                             cudaMemcpyHostToDevice, E->stream));
    AMG_CUDA(cudaStreamSynchronize(E->stream));  // caps and sl are locals
    launch_batch(E, shape, b, x, tol, E->rslots, (int)sl.size());
    g_launches += 1;
    return true;
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
    for (;;) {
        AMG_CUDA(cudaMemcpyAsync(it.data(), E->iters, sizeof(int) * E->nprob,
                                 cudaMemcpyDeviceToHost, E->stream));
        AMG_CUDA(cudaMemcpyAsync(st.data(), E->status, sizeof(int) * E->nprob,
                                 cudaMemcpyDeviceToHost, E->stream));
        AMG_CUDA(cudaMemcpyAsync(rr.data(), E->relres, sizeof(double) * E->nprob,
                                 cudaMemcpyDeviceToHost, E->stream));
        AMG_CUDA(cudaStreamSynchronize(E->stream));
        if (!resume_full(E, st, b, x, tol)) break;
    }
    int first_bad = AMG_OK;
    E->last_iters = it;
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

// Algorithmic bytes of a system's batched solve of `its` outer steps (solve_one, FP64 outer,
// 8-byte values, 4-byte indices): per step k (k = 0, 1, ...) one B^_0, the conversions to and
// from the cycle precision (FP32 cycle), the dots (z, q_j) of the k kept directions (z re-read
// per group of 4), p_k = z - sum c_j p_j (per chunk of 64: the running p_k read and written),
// q_k = A p_k with (p_k, q_k) and (r, p_k), and the x / r update; once per solve the gather of
// b (and bo, ro, xo written) and the true residual.
double batch_moved_bytes(BatchEngine *E) {
    if (E->last_iters.empty()) return 0.0;
    const int vb = E->fp32 ? 4 : 8;
    if (E->cyc_bytes.empty()) {
        E->cyc_bytes.resize(E->nprob);
        for (int p = 0; p < E->nprob; p++)
            E->cyc_bytes[p] = E->hs[p]->nlev > 1 ? cycle_application_bytes(E->hs[p], vb)
                                                 : (double)vb * ((double)E->hs[p]->N * E->hs[p]->N + 2.0 * E->hs[p]->N);
    }
    double total = 0.0;
    for (int p = 0; p < E->nprob; p++) {
        const double n = (double)E->hs[p]->N, nnz = (double)E->hs[p]->lev[0].A.stored;
        double s = 56.0 * n + 12.0 * nnz + 24.0 * n;  // gather of b; true residual
        for (int k = 0; k < E->last_iters[p]; k++) {
            s += E->cyc_bytes[p];
            if (E->fp32) s += 24.0 * n;
            s += 8.0 * n * (k + (k + 3) / 4);
            s += 16.0 * n * std::max(1, (k + 63) / 64) + 8.0 * n * k;
            s += 12.0 * nnz + 32.0 * n;
            s += 48.0 * n;
        }
        total += s;
    }
    return total;
}

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
