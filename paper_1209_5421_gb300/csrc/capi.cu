// C ABI of the library (include/amg.h): argument checks, host/device staging, ownership,
// status codes; no exception crosses the interface.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "amg_internal.cuh"

using amg::Error;
using amg::Scratch;

namespace {

thread_local std::string g_last_error;

int fail(int status, const std::string &what) {
    g_last_error = what;
    return status;
}

}  // namespace

namespace amg {
int set_last_error(int status, const char *what) { return fail(status, what); }

// host-set allocation fault: 0 = off, k > 0 = the k-th device allocation from now fails
static std::atomic<int64_t> g_fail_alloc_countdown{0};
bool fail_this_allocation() {
    int64_t k = g_fail_alloc_countdown.load(std::memory_order_relaxed);
    while (k > 0) {
        if (g_fail_alloc_countdown.compare_exchange_weak(k, k - 1, std::memory_order_relaxed))
            return k == 1;
    }
    return false;
}
}  // namespace amg

namespace {

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// device view of a device-or-host array (host data is copied into scratch)
template <class T>
const T *to_device(const T *p, size_t count, Scratch &tmp) {
    if (!p || count == 0 || is_device_ptr(p)) return p;
    T *d = tmp.get<T>(count);
    AMG_CUDA(cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, tmp.s));
    return d;
}

void init_pool_once(int dev) {
    static std::mutex m;
    static std::vector<int> done;
    std::lock_guard<std::mutex> g(m);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;  // keep freed blocks in this process's pool for reuse
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done.push_back(dev);
}

void destroy(amg_hierarchy *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    amg::free_engines(h);
    amg::profiler_free(h);
    for (void *p : h->allocs) cudaFreeAsync(p, h->stream);
    h->arena.s = h->stream;
    h->arena.release();
    cudaStreamSynchronize(h->stream);
    if (h->h_pinned) cudaFreeHost(h->h_pinned);
    if (h->order_ev) cudaEventDestroy(h->order_ev);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

#define AMG_CATCH                                                 \
    catch (const Error &e) {                                      \
        return fail(e.status, e.what);                            \
    }                                                             \
    catch (const std::bad_alloc &) {                              \
        return fail(AMG_ERR_OOM, "host allocation failed");       \
    }                                                             \
    catch (...) {                                                 \
        return fail(AMG_ERR_CUDA, "unexpected internal exception"); \
    }

__global__ void k_csr_to_ell(int rows, const int *__restrict__ rowptr, const int *__restrict__ col,
                             const double *__restrict__ val, int width, int diag_first,
                             int *__restrict__ Aj, double *__restrict__ Ax, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    int b = rowptr[i], e = rowptr[i + 1];
    if (e - b > width) {
        atomicOr(err, 1);
        return;
    }
    int k = 0;
    int dpos = -1;
    if (diag_first)
        for (int p = b; p < e; p++)
            if (col[p] == i) dpos = p;
    if (dpos >= 0) {
        Aj[i] = i;
        Ax[i] = val[dpos];
        k = 1;
    }
    for (int p = b; p < e; p++) {
        if (p == dpos) continue;
        Aj[(size_t)k * rows + i] = col[p];
        Ax[(size_t)k * rows + i] = val[p];
        k++;
    }
    for (; k < width; k++) {
        Aj[(size_t)k * rows + i] = -1;
        Ax[(size_t)k * rows + i] = 0.0;
    }
}

}  // namespace

extern "C" {

const char *amg_last_error(void) { return g_last_error.c_str(); }

void amg_options_default(amg_options *o) {
    if (!o) return;
    o->aux_level = 0;
    o->coarsest_max = 64;
    o->kcycle_n = 2;
    o->max_iters = 200;
    o->outer = AMG_OUTER_FCG;
    o->cycle_prec = AMG_FP64;
    o->fgmres_restart = 30;
    o->has_bbox = 0;
    o->bbox[0] = o->bbox[1] = o->bbox[2] = o->bbox[3] = 0.0;
    o->zbox[0] = o->zbox[1] = 0.0;
    o->nu_pre = 1;
    o->nu_post = 1;
}

const char *amg_status_string(int s) {
    switch (s) {
        case AMG_OK: return "ok";
        case AMG_ERR_INVALID_ARG: return "invalid argument";
        case AMG_ERR_BAD_MATRIX: return "matrix is not valid SPD CSR input";
        case AMG_ERR_OOM: return "out of device memory";
        case AMG_ERR_CUDA: return "CUDA error";
        case AMG_ERR_NOT_CONVERGED: return "not converged within max_iters";
        case AMG_ERR_BREAKDOWN: return "Krylov breakdown";
        case AMG_ERR_TIMEOUT: return "device wait timed out";
        case AMG_ERR_UNSUPPORTED: return "outside the library's limits";
        default: return "unknown status";
    }
}

namespace {

// option checks shared by amg_setup and amg_batch_setup
int check_options(const amg_options &o) {
    if (o.aux_level < 0 || o.aux_level > 14) return fail(AMG_ERR_UNSUPPORTED, "aux_level must be 0..14");
    if (o.coarsest_max < 1 || o.coarsest_max > amg::kMaxCoarsest)
        return fail(AMG_ERR_UNSUPPORTED, "coarsest_max must be 1..256");
    if (o.kcycle_n < 1 || o.kcycle_n > amg::kMaxKcycle)
        return fail(AMG_ERR_UNSUPPORTED, "kcycle_n must be 1..4");
    if (o.max_iters < 1 || o.max_iters > 100000) return fail(AMG_ERR_INVALID_ARG, "max_iters");
    if (o.outer == AMG_OUTER_FGMRES && 2 * o.fgmres_restart + 1 > o.max_iters)
        return fail(AMG_ERR_INVALID_ARG, "FGMRES needs max_iters >= 2 * fgmres_restart + 1");
    if (o.cycle_prec != AMG_FP64 && o.cycle_prec != AMG_FP32)
        return fail(AMG_ERR_INVALID_ARG, "cycle_prec");
    if (o.outer != AMG_OUTER_FCG && o.outer != AMG_OUTER_FGMRES)
        return fail(AMG_ERR_INVALID_ARG, "outer");
    if (o.outer == AMG_OUTER_FGMRES && (o.fgmres_restart < 1 || o.fgmres_restart > 1000))
        return fail(AMG_ERR_INVALID_ARG, "fgmres_restart");
    if (o.has_bbox && !(o.bbox[1] > o.bbox[0] && o.bbox[3] > o.bbox[2]))
        return fail(AMG_ERR_INVALID_ARG, "bbox must have b1 > a1 and b2 > a2");
    if (o.nu_pre < 0 || o.nu_pre > amg::kMaxSweeps || o.nu_post < 0 || o.nu_post > amg::kMaxSweeps)
        return fail(AMG_ERR_UNSUPPORTED, "nu_pre and nu_post must be 0..4 (0 = 1)");
    return AMG_OK;
}

// a hierarchy from device arrays (A's arrays, x, y on the device); throws amg::Error
amg_hierarchy *setup_device(const amg_csr &Ad, const double *xd, const double *yd,
                            const double *zd, const amg_options &o, void *stream) {
    amg_hierarchy *h = nullptr;
    try {
        h = new amg_hierarchy();
        h->opt = o;
        if (h->opt.nu_pre == 0) h->opt.nu_pre = 1;
        if (h->opt.nu_post == 0) h->opt.nu_post = 1;
        h->N = Ad.n;
        h->dim = zd ? 3 : 2;
        AMG_CUDA(cudaGetDevice(&h->device));
        init_pool_once(h->device);
        AMG_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        AMG_CUDA(cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming));
        amg::bind_stream(h, stream);
        const int64_t l0 = amg::g_launches;
        h->err_flag = amg::halloc<int>(h, 1);
        amg::build_hierarchy(h, Ad, xd, yd, zd);
        amg::allocate_solve_workspace(h);
        AMG_CUDA(cudaStreamSynchronize(h->stream));
        h->setup_launches = amg::g_launches - l0;
        return h;
    } catch (...) {
        destroy(h);
        throw;
    }
}

}  // namespace

int amg_setup(const amg_csr *A, const double *x, const double *y, const amg_options *opt,
              void *stream, amg_hierarchy **out) {
    if (!out) return fail(AMG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!A || !x || !y || !A->rowptr || !A->col || !A->val)
        return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    if (A->n <= 0) return fail(AMG_ERR_INVALID_ARG, "n must be positive");
    if (A->n >= INT32_MAX || A->nnz >= INT32_MAX)
        return fail(AMG_ERR_UNSUPPORTED, "n and nnz must be below 2^31");
    if (A->nnz < A->n) return fail(AMG_ERR_BAD_MATRIX, "every row needs its diagonal");
    amg_options o;
    if (opt) o = *opt;
    else amg_options_default(&o);
    if (int st = check_options(o)) return st;
    try {
        cudaStream_t us = (cudaStream_t)stream;
        Scratch tmp(us);
        const int n = (int)A->n;
        amg_csr Ad = *A;
        Ad.rowptr = to_device(A->rowptr, (size_t)n + 1, tmp);
        Ad.col = to_device(A->col, (size_t)A->nnz, tmp);
        Ad.val = to_device(A->val, (size_t)A->nnz, tmp);
        const double *xd = to_device(x, (size_t)n, tmp);
        const double *yd = to_device(y, (size_t)n, tmp);
        *out = setup_device(Ad, xd, yd, nullptr, o, stream);
        AMG_CUDA(cudaStreamSynchronize(us));  // the staging copies are read by the setup
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_setup3(const amg_csr *A, const double *x, const double *y, const double *z,
               const amg_options *opt, void *stream, amg_hierarchy **out) {
    if (!out) return fail(AMG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!A || !x || !y || !z || !A->rowptr || !A->col || !A->val)
        return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    if (A->n <= 0) return fail(AMG_ERR_INVALID_ARG, "n must be positive");
    if (A->n >= INT32_MAX || A->nnz >= INT32_MAX)
        return fail(AMG_ERR_UNSUPPORTED, "n and nnz must be below 2^31");
    if (A->nnz < A->n) return fail(AMG_ERR_BAD_MATRIX, "every row needs its diagonal");
    amg_options o;
    if (opt) o = *opt;
    else amg_options_default(&o);
    if (int st = check_options(o)) return st;
    if (o.aux_level > 10) return fail(AMG_ERR_UNSUPPORTED, "octree aux_level must be 0..10");
    if (o.has_bbox && !(o.zbox[1] > o.zbox[0]))
        return fail(AMG_ERR_INVALID_ARG, "zbox must have b3 > a3");
    try {
        cudaStream_t us = (cudaStream_t)stream;
        Scratch tmp(us);
        const int n = (int)A->n;
        amg_csr Ad = *A;
        Ad.rowptr = to_device(A->rowptr, (size_t)n + 1, tmp);
        Ad.col = to_device(A->col, (size_t)A->nnz, tmp);
        Ad.val = to_device(A->val, (size_t)A->nnz, tmp);
        const double *xd = to_device(x, (size_t)n, tmp);
        const double *yd = to_device(y, (size_t)n, tmp);
        const double *zd = to_device(z, (size_t)n, tmp);
        *out = setup_device(Ad, xd, yd, zd, o, stream);
        AMG_CUDA(cudaStreamSynchronize(us));
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_solve(amg_hierarchy *h, const double *b, double tol, double *x, int *iters,
              double *relres, void *stream) {
    if (!h || !b || !x) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    if (!(tol >= 0.0)) return fail(AMG_ERR_INVALID_ARG, "tol must be >= 0");
    try {
        amg::bind_stream(h, stream);
        const size_t n = (size_t)h->N;
        Scratch tmp(h->stream);
        const double *bd = to_device(b, n, tmp);
        bool xhost = !is_device_ptr(x);
        double *xd = xhost ? tmp.get<double>(n) : x;
        const int64_t l0 = amg::g_launches;
        int st = amg::solve(h, bd, tol, xd, iters, relres);
        h->solve_launches = amg::g_launches - l0;
        if (xhost) {
            AMG_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
            AMG_CUDA(cudaStreamSynchronize(h->stream));
        }
        if (st != AMG_OK) g_last_error = amg_status_string(st);
        return st;
    }
    AMG_CATCH
}

int amg_hierarchy_bytes(const amg_hierarchy *h, size_t *bytes) {
    if (!h || !bytes) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    *bytes = h->bytes;
    return AMG_OK;
}

void amg_free(amg_hierarchy *h) { destroy(h); }

// ---------------------------------------------------------------------------------------
// batched systems

struct amg_batch {
    std::vector<amg_hierarchy *> hs;
    bool owns = true;  // hierarchies built by amg_batch_setup (else borrowed)
    std::vector<int64_t> row_off;
    amg::BatchEngine *eng = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t order_ev = nullptr;
    int device = 0;
};

namespace {

void destroy_batch(amg_batch *bt) {
    if (!bt) return;
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    amg::batch_destroy(bt->eng);
    if (bt->owns)
        for (amg_hierarchy *h : bt->hs) destroy(h);
    if (bt->order_ev) cudaEventDestroy(bt->order_ev);
    if (bt->stream) cudaStreamDestroy(bt->stream);
    delete bt;
}

// rowptr[r0 + i] - nz0 and col[nz0 + k] - r0: the rows of one system, indexed locally
__global__ void k_localize_rows(int n, const int *__restrict__ rowptr, int nz0,
                                int *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) out[i] = rowptr[i] - nz0;
}
__global__ void k_localize_cols(int nnz, const int *__restrict__ col, int r0, int *__restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) out[k] = col[k] - r0;
}
// out[p] = rowptr[row_off[p]]: the first entry of every system
__global__ void k_gather_rowptr(int m, const int *__restrict__ rowptr,
                                const int64_t *__restrict__ row_off, int *__restrict__ out) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < m) out[p] = rowptr[row_off[p]];
}

}  // namespace

}  // extern "C"

namespace {

// the argument checks of amg_batch_setup and amg_setup_many
int check_systems(int32_t nprob, const int64_t *row_off, const amg_csr *A, const double *x,
                  const double *y) {
    if (nprob < 1 || !row_off || !A || !x || !y || !A->rowptr || !A->col || !A->val)
        return fail(AMG_ERR_INVALID_ARG, "NULL argument or no system");
    if (is_device_ptr(row_off)) return fail(AMG_ERR_INVALID_ARG, "row_off must be host memory");
    if (row_off[0] != 0 || row_off[nprob] != A->n)
        return fail(AMG_ERR_INVALID_ARG, "row_off must run from 0 to A->n");
    for (int p = 0; p < nprob; p++)
        if (row_off[p + 1] <= row_off[p]) return fail(AMG_ERR_INVALID_ARG, "every system needs a row");
    if (A->n >= INT32_MAX || A->nnz >= INT32_MAX)
        return fail(AMG_ERR_UNSUPPORTED, "n and nnz must be below 2^31");
    return AMG_OK;
}

// One hierarchy per system of the block-diagonal A (arguments checked), into hs (nprob
// entries; on a throw, hs holds what was built so far, for the caller to destroy). Systems
// of more than coarsest_max unknowns are set up together by one set of multi-system kernels
// on stream ws (setup_batch.cu); a system small enough to be its own coarsest level (one
// level, the exact solve) takes the single-system setup. batch_ws: also prepare every system
// for batched solves (as batch_prepare).
void setup_systems(int32_t nprob, const int64_t *row_off, const amg_csr *A, const double *x,
                   const double *y, const amg_options &o, cudaStream_t us, cudaStream_t ws,
                   bool batch_ws, std::vector<amg_hierarchy *> &hs) {
    hs.assign(nprob, nullptr);
    int dev = 0;
    AMG_CUDA(cudaGetDevice(&dev));
    init_pool_once(dev);
    Scratch tmp(us);
    const size_t N = (size_t)A->n;
    const int *rp = to_device(A->rowptr, N + 1, tmp);
    const int *cl = to_device(A->col, (size_t)A->nnz, tmp);
    const double *vl = to_device(A->val, (size_t)A->nnz, tmp);
    const double *xd = to_device(x, N, tmp);
    const double *yd = to_device(y, N, tmp);
    // nonzero offset of every system: rowptr[row_off[p]], gathered and read back at once
    std::vector<int> nz(nprob + 1);
    {
        int64_t *dro = tmp.get<int64_t>((size_t)nprob + 1);
        int *dnz = tmp.get<int>((size_t)nprob + 1);
        AMG_CUDA(cudaMemcpyAsync(dro, row_off, sizeof(int64_t) * (nprob + 1),
                                 cudaMemcpyHostToDevice, us));
        k_gather_rowptr<<<(nprob + 256) / 256, 256, 0, us>>>(nprob + 1, rp, dro, dnz);
        AMG_CUDA(cudaGetLastError());
        AMG_CUDA(cudaMemcpyAsync(nz.data(), dnz, sizeof(int) * (nprob + 1), cudaMemcpyDeviceToHost,
                                 us));
        AMG_CUDA(cudaStreamSynchronize(us));
    }
    if (nz[0] != 0 || nz[nprob] != A->nnz)
        throw Error{AMG_ERR_BAD_MATRIX, "rowptr does not run from 0 to nnz"};
    for (int p = 0; p < nprob; p++)
        if (nz[p + 1] - nz[p] < (int)(row_off[p + 1] - row_off[p]))
            throw Error{AMG_ERR_BAD_MATRIX, "every row needs its diagonal"};
    std::vector<int> multi;
    for (int p = 0; p < nprob; p++) {
        const int r0 = (int)row_off[p], n = (int)(row_off[p + 1] - row_off[p]);
        if (n > o.coarsest_max) {
            multi.push_back(p);
            continue;
        }
        const int z0 = nz[p], nnz = nz[p + 1] - nz[p];
        Scratch loc(us);
        int *lrp = loc.get<int>((size_t)n + 1), *lcl = loc.get<int>((size_t)nnz);
        k_localize_rows<<<(n + 256) / 256, 256, 0, us>>>(n, rp + r0, z0, lrp);
        k_localize_cols<<<(nnz + 255) / 256, 256, 0, us>>>(nnz, cl + z0, r0, lcl);
        AMG_CUDA(cudaGetLastError());
        amg_csr Ap{n, nnz, lrp, lcl, vl + z0};
        hs[p] = setup_device(Ap, xd + r0, yd + r0, nullptr, o, us);
        if (batch_ws) amg::batch_prepare(hs[p]);
    }
    if (multi.empty()) return;
    std::vector<amg_hierarchy *> mh;
    std::vector<amg::BatchRows> rows;
    cudaEvent_t ready;
    AMG_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaEventRecord(ready, us);  // the staged inputs
    cudaStreamWaitEvent(ws, ready, 0);
    cudaEventDestroy(ready);
    AMG_CUDA(cudaGetLastError());
    for (int p : multi) {
        amg_hierarchy *h = new amg_hierarchy();
        hs[p] = h;
        h->opt = o;
        if (h->opt.nu_pre == 0) h->opt.nu_pre = 1;
        if (h->opt.nu_post == 0) h->opt.nu_post = 1;
        h->N = row_off[p + 1] - row_off[p];
        h->dim = 2;
        h->device = dev;
        h->stream = ws;  // while the batched setup builds it
        mh.push_back(h);
        rows.push_back(amg::BatchRows{(int)row_off[p], (int)h->N, nz[p], nz[p + 1] - nz[p]});
    }
    const int64_t l0 = amg::g_launches;
    try {
        amg::build_batch(mh, amg_csr{A->n, A->nnz, rp, cl, vl}, xd, yd, rows, ws, batch_ws);
        for (amg_hierarchy *h : mh) {
            h->setup_launches = amg::g_launches - l0;  // the whole batched setup's launches
            h->stream = nullptr;
            AMG_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
            AMG_CUDA(cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming));
        }
        AMG_CUDA(cudaStreamSynchronize(ws));
    } catch (...) {
        cudaStreamSynchronize(ws);
        for (amg_hierarchy *h : mh)
            if (h->stream == ws) h->stream = nullptr;  // not the hierarchy's own
        throw;
    }
}

}  // namespace

extern "C" {

int amg_batch_setup(int32_t nprob, const int64_t *row_off, const amg_csr *A, const double *x,
                    const double *y, const amg_options *opt, void *stream, amg_batch **out) {
    if (!out) return fail(AMG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (int st = check_systems(nprob, row_off, A, x, y)) return st;
    amg_options o;
    if (opt) o = *opt;
    else amg_options_default(&o);
    if (int st = check_options(o)) return st;
    if (o.outer != AMG_OUTER_FCG)
        return fail(AMG_ERR_UNSUPPORTED, "batched systems use the flexible-CG outer iteration");
    amg_batch *bt = nullptr;
    try {
        bt = new amg_batch();
        AMG_CUDA(cudaGetDevice(&bt->device));
        AMG_CUDA(cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking));
        AMG_CUDA(cudaEventCreateWithFlags(&bt->order_ev, cudaEventDisableTiming));
        cudaStream_t us = (cudaStream_t)stream;
        bt->row_off.assign(row_off, row_off + nprob + 1);
        setup_systems(nprob, row_off, A, x, y, o, us, bt->stream, true, bt->hs);
        bt->eng = amg::batch_create(bt->hs, bt->row_off, bt->stream, 0);
        AMG_CUDA(cudaStreamSynchronize(us));
        *out = bt;
        return AMG_OK;
    } catch (const Error &e) {
        destroy_batch(bt);
        return fail(e.status, e.what);
    } catch (const std::bad_alloc &) {
        destroy_batch(bt);
        return fail(AMG_ERR_OOM, "host allocation failed");
    } catch (...) {
        destroy_batch(bt);
        return fail(AMG_ERR_CUDA, "unexpected internal exception");
    }
}

int amg_setup_many(int32_t nprob, const int64_t *row_off, const amg_csr *A, const double *x,
                   const double *y, const amg_options *opt, void *stream, amg_hierarchy **out) {
    if (!out) return fail(AMG_ERR_INVALID_ARG, "out is NULL");
    for (int p = 0; p < nprob; p++) out[p] = nullptr;
    if (int st = check_systems(nprob, row_off, A, x, y)) return st;
    amg_options o;
    if (opt) o = *opt;
    else amg_options_default(&o);
    if (int st = check_options(o)) return st;
    std::vector<amg_hierarchy *> hs;
    cudaStream_t ws = nullptr;
    int status = AMG_OK;
    std::string what;
    try {
        AMG_CUDA(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
        setup_systems(nprob, row_off, A, x, y, o, (cudaStream_t)stream, ws,
                      o.outer == AMG_OUTER_FCG, hs);
        AMG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    } catch (const Error &e) {
        status = e.status;
        what = e.what;
    } catch (const std::bad_alloc &) {
        status = AMG_ERR_OOM;
        what = "host allocation failed";
    } catch (...) {
        status = AMG_ERR_CUDA;
        what = "unexpected internal exception";
    }
    if (status != AMG_OK)
        for (amg_hierarchy *h : hs) destroy(h);
    if (ws) {
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    }
    if (status != AMG_OK) return fail(status, what);
    for (int p = 0; p < nprob; p++) out[p] = hs[p];
    return AMG_OK;
}

int amg_batch_create(int32_t nprob, amg_hierarchy *const *hs, int32_t threads, void *stream,
                     amg_batch **out) {
    if (!out) return fail(AMG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nprob < 1 || !hs) return fail(AMG_ERR_INVALID_ARG, "no system");
    if (threads != 0 && threads != 1024 && threads != 512 && threads != 256)
        return fail(AMG_ERR_INVALID_ARG, "threads must be 0, 1024, 512 or 256");
    for (int p = 0; p < nprob; p++) {
        if (!hs[p]) return fail(AMG_ERR_INVALID_ARG, "NULL hierarchy");
        if (hs[p]->opt.cycle_prec != hs[0]->opt.cycle_prec || hs[p]->opt.kcycle_n != hs[0]->opt.kcycle_n ||
            hs[p]->opt.nu_pre != hs[0]->opt.nu_pre || hs[p]->opt.nu_post != hs[0]->opt.nu_post ||
            hs[p]->opt.max_iters != hs[0]->opt.max_iters)
            return fail(AMG_ERR_INVALID_ARG,
                        "every hierarchy needs the same cycle_prec, kcycle_n, nu_pre and nu_post");
        for (int q = 0; q < p; q++)
            if (hs[q] == hs[p]) return fail(AMG_ERR_INVALID_ARG, "a hierarchy appears twice");
    }
    amg_batch *bt = nullptr;
    try {
        bt = new amg_batch();
        bt->owns = false;
        AMG_CUDA(cudaGetDevice(&bt->device));
        AMG_CUDA(cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking));
        AMG_CUDA(cudaEventCreateWithFlags(&bt->order_ev, cudaEventDisableTiming));
        AMG_CUDA(cudaEventRecord(bt->order_ev, (cudaStream_t)stream));
        AMG_CUDA(cudaStreamWaitEvent(bt->stream, bt->order_ev, 0));
        bt->hs.assign(hs, hs + nprob);
        bt->row_off.assign(1, 0);
        for (int p = 0; p < nprob; p++) bt->row_off.push_back(bt->row_off.back() + hs[p]->N);
        bt->eng = amg::batch_create(bt->hs, bt->row_off, bt->stream, threads);
        *out = bt;
        return AMG_OK;
    } catch (const Error &e) {
        destroy_batch(bt);
        return fail(e.status, e.what);
    } catch (const std::bad_alloc &) {
        destroy_batch(bt);
        return fail(AMG_ERR_OOM, "host allocation failed");
    } catch (...) {
        destroy_batch(bt);
        return fail(AMG_ERR_CUDA, "unexpected internal exception");
    }
}

int amg_batch_solve(amg_batch *bt, const double *b, double tol, double *x, int32_t *iters,
                    double *relres, int32_t *status, void *stream) {
    if (!bt || !b || !x) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    if (!(tol >= 0.0)) return fail(AMG_ERR_INVALID_ARG, "tol must be >= 0");
    try {
        AMG_CUDA(cudaEventRecord(bt->order_ev, (cudaStream_t)stream));
        AMG_CUDA(cudaStreamWaitEvent(bt->stream, bt->order_ev, 0));
        const size_t N = (size_t)bt->row_off.back();
        Scratch tmp(bt->stream);
        const double *bd = to_device(b, N, tmp);
        const bool xhost = !is_device_ptr(x);
        double *xd = xhost ? tmp.get<double>(N) : x;
        std::vector<int> it(bt->hs.size()), st(bt->hs.size());
        int r = amg::batch_solve(bt->eng, bd, tol, xd, it.data(), relres, st.data());
        if (xhost) {
            AMG_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * N, cudaMemcpyDeviceToHost, bt->stream));
            AMG_CUDA(cudaStreamSynchronize(bt->stream));
        }
        for (size_t p = 0; p < bt->hs.size(); p++) {
            if (iters) iters[p] = it[p];
            if (status) status[p] = st[p];
        }
        if (r != AMG_OK) g_last_error = amg_status_string(r);
        return r;
    }
    AMG_CATCH
}

int amg_batch_info(const amg_batch *bt, int32_t *nprob, int32_t *threads, int32_t *ctas,
                   double tuned_ms[4], size_t *bytes) {
    if (!bt) return fail(AMG_ERR_INVALID_ARG, "NULL batch");
    if (nprob) *nprob = (int32_t)bt->hs.size();
    int t = 0, c = 0;
    double ms[4] = {-1, -1, -1, -1};
    const int shape = amg::batch_shape(bt->eng, &t, &c, ms);
    if (threads) *threads = shape < 0 ? 0 : t;
    if (ctas) *ctas = shape < 0 ? 0 : c;
    if (tuned_ms)
        for (int k = 0; k < 4; k++) tuned_ms[k] = ms[k];
    if (bytes) {
        size_t s = amg::batch_bytes(bt->eng);
        for (amg_hierarchy *h : bt->hs) s += h->bytes;
        *bytes = s;
    }
    return AMG_OK;
}

int amg_batch_moved_bytes(amg_batch *bt, double *bytes) {
    if (!bt || !bytes) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    try {
        *bytes = amg::batch_moved_bytes(bt->eng);
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_batch_timeline(const amg_batch *bt, int64_t *start_ns, int64_t *end_ns) {
    if (!bt) return fail(AMG_ERR_INVALID_ARG, "NULL batch");
    try {
        amg::batch_timeline(bt->eng, start_ns, end_ns);
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_batch_set_teams(amg_batch *bt, int32_t max_team) {
    if (!bt) return fail(AMG_ERR_INVALID_ARG, "NULL batch");
    if (max_team < 0 || max_team > 8) return fail(AMG_ERR_INVALID_ARG, "max_team must be 0..8");
    try {
        amg::batch_set_teams(bt->eng, max_team);
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_debug_barrier_fault(amg_hierarchy *h, int64_t limit_ns, int32_t extra) {
    if (!h) return fail(AMG_ERR_INVALID_ARG, "NULL hierarchy");
    if (limit_ns < 0 || extra < 0) return fail(AMG_ERR_INVALID_ARG, "negative limit or arrivals");
    h->dbg_bar_limit_ns = limit_ns;
    h->dbg_bar_extra = extra;
    return AMG_OK;
}

int amg_debug_batch_barrier_fault(amg_batch *bt, int64_t limit_ns, int32_t extra) {
    if (!bt) return fail(AMG_ERR_INVALID_ARG, "NULL batch");
    if (limit_ns < 0 || extra < 0) return fail(AMG_ERR_INVALID_ARG, "negative limit or arrivals");
    amg::batch_barrier_fault(bt->eng, limit_ns, extra);
    return AMG_OK;
}

int amg_debug_fail_allocation(int64_t k) {
    if (k < 0) return fail(AMG_ERR_INVALID_ARG, "k must be >= 0");
    amg::g_fail_alloc_countdown.store(k);
    return AMG_OK;
}

int amg_debug_bounds_flags(int32_t *flags) {
    if (!flags) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    const int a = amg::bounds_flags_solve(), b = amg::bounds_flags_batch();
    if (a < 0 || b < 0) return fail(AMG_ERR_UNSUPPORTED, "built without index checks");
    *flags = a | b;
    return AMG_OK;
}

int amg_debug_pool_bytes_in_use(int32_t device, int64_t *bytes) {
    if (!bytes) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    cudaMemPool_t pool;
    cudaError_t e = cudaDeviceGetDefaultMemPool(&pool, device);
    uint64_t used = 0;
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(AMG_ERR_CUDA, cudaGetErrorString(e));
    }
    *bytes = (int64_t)used;
    return AMG_OK;
}

int amg_batch_teams(const amg_batch *bt, int32_t *team) {
    if (!bt || !team) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    std::vector<int> t(bt->hs.size());
    amg::batch_teams(bt->eng, t.data());
    for (size_t p = 0; p < t.size(); p++) team[p] = t[p];
    return AMG_OK;
}

amg_hierarchy *amg_batch_system(amg_batch *bt, int32_t p) {
    if (!bt || p < 0 || p >= (int32_t)bt->hs.size()) {
        fail(AMG_ERR_INVALID_ARG, "no such system");
        return nullptr;
    }
    return bt->hs[p];
}

void amg_batch_free(amg_batch *bt) { destroy_batch(bt); }

int amg_num_levels(const amg_hierarchy *h, int *num_levels, int *aux_level) {
    if (!h) return fail(AMG_ERR_INVALID_ARG, "NULL hierarchy");
    if (num_levels) *num_levels = h->nlev;
    if (aux_level) *aux_level = h->L;
    return AMG_OK;
}

int amg_get_bbox(const amg_hierarchy *h, double bbox[4]) {
    if (!h || !bbox) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < 4; k++) bbox[k] = h->bbox[k];
    return AMG_OK;
}

int amg_level_info(const amg_hierarchy *h, int level, int64_t info[8]) {
    if (!h || !info) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= h->nlev) return fail(AMG_ERR_INVALID_ARG, "level out of range");
    const amg::Level &lv = h->lev[level];
    info[0] = lv.n;
    info[1] = lv.A.stored;
    info[2] = lv.cellw;
    info[3] = lv.span;
    info[4] = lv.m;
    info[5] = lv.A.padded;
    info[6] = lv.coarsest ? 1 : 0;
    info[7] = (level == 0) ? lv.nblocks : 0;
    return AMG_OK;
}

int amg_level_t3(const amg_hierarchy *h, int level, int32_t *t3) {
    if (!h || !t3) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= h->nlev) return fail(AMG_ERR_INVALID_ARG, "level out of range");
    try {
        const amg::Level &lv = h->lev[level];
        const int n = lv.n;
        AMG_CUDA(cudaStreamSynchronize(h->stream));
        std::vector<int> c(n);
        AMG_CUDA(cudaMemcpy(c.data(), h->cell_nat[level], sizeof(int) * n, cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; i++) t3[i] = c[i] / lv.cellw / lv.cellw;
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_get_box3(const amg_hierarchy *h, int *dim, double box[6]) {
    if (!h) return fail(AMG_ERR_INVALID_ARG, "NULL hierarchy");
    if (dim) *dim = h->dim;
    if (box)
        for (int k = 0; k < 6; k++) box[k] = h->bbox[k];
    return AMG_OK;
}

int amg_level_export(const amg_hierarchy *h, int level, int32_t *agg, int32_t *color,
                     int32_t *t1, int32_t *t2, int32_t *rowptr, int32_t *col, double *val) {
    if (!h) return fail(AMG_ERR_INVALID_ARG, "NULL hierarchy");
    if (level < 0 || level >= h->nlev) return fail(AMG_ERR_INVALID_ARG, "level out of range");
    try {
        const amg::Level &lv = h->lev[level];
        cudaStream_t s = h->stream;
        const int n = lv.n;
        AMG_CUDA(cudaStreamSynchronize(s));
        if (agg) {
            if (lv.agg_nat) AMG_CUDA(cudaMemcpy(agg, lv.agg_nat, sizeof(int) * n, cudaMemcpyDeviceToHost));
            else std::fill(agg, agg + n, -1);
        }
        if (color) AMG_CUDA(cudaMemcpy(color, h->color_nat[level], sizeof(int) * n, cudaMemcpyDeviceToHost));
        if (t1 || t2) {
            std::vector<int> c(n);
            AMG_CUDA(cudaMemcpy(c.data(), h->cell_nat[level], sizeof(int) * n, cudaMemcpyDeviceToHost));
            for (int i = 0; i < n; i++) {  // cell = t1 + w (t2 + w t3)
                if (t1) t1[i] = c[i] % lv.cellw;
                if (t2) t2[i] = (c[i] / lv.cellw) % lv.cellw;
            }
        }
        if (rowptr || col || val) {
            std::vector<int> nat(n), sl(lv.A.nslices + 1), ac(lv.A.padded);
            std::vector<double> av(lv.A.padded);
            AMG_CUDA(cudaMemcpy(nat.data(), lv.nat, sizeof(int) * n, cudaMemcpyDeviceToHost));
            AMG_CUDA(cudaMemcpy(sl.data(), lv.A.sl_ptr, sizeof(int) * sl.size(), cudaMemcpyDeviceToHost));
            AMG_CUDA(cudaMemcpy(ac.data(), lv.A.col, sizeof(int) * ac.size(), cudaMemcpyDeviceToHost));
            AMG_CUDA(cudaMemcpy(av.data(), lv.A.val, sizeof(double) * av.size(), cudaMemcpyDeviceToHost));
            std::vector<int> inv(n);
            for (int p = 0; p < n; p++) inv[nat[p]] = p;
            std::vector<std::pair<int, double>> row;
            int64_t pos = 0;
            if (rowptr) rowptr[0] = 0;
            for (int R = 0; R < n; R++) {
                int p = inv[R];
                int sidx = p >> 5, lane = p & 31;
                int width = (sl[sidx + 1] - sl[sidx]) >> 5;
                row.clear();
                for (int k = 0; k < width; k++) {
                    int c = ac[sl[sidx] + 32 * k + lane];
                    if (c >= 0) row.push_back({nat[c], av[sl[sidx] + 32 * k + lane]});
                }
                std::sort(row.begin(), row.end(),
                          [](const std::pair<int, double> &a, const std::pair<int, double> &b) {
                              return a.first < b.first;
                          });
                for (auto &e : row) {
                    if (col) col[pos] = e.first;
                    if (val) val[pos] = e.second;
                    pos++;
                }
                if (rowptr) rowptr[R + 1] = (int32_t)pos;
            }
        }
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_apply_cycle(amg_hierarchy *h, int level, const double *f, double *z, void *stream) {
    if (!h || !f || !z) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= h->nlev) return fail(AMG_ERR_INVALID_ARG, "level out of range");
    try {
        amg::bind_stream(h, stream);
        const size_t n = (size_t)h->lev[level].n;
        Scratch tmp(h->stream);
        const double *fd = to_device(f, n, tmp);
        bool zhost = !is_device_ptr(z);
        double *zd = zhost ? tmp.get<double>(n) : z;
        amg::apply_cycle_level(h, level, fd, zd);
        if (zhost) {
            AMG_CUDA(cudaMemcpyAsync(z, zd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
            AMG_CUDA(cudaStreamSynchronize(h->stream));
        }
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_smooth(amg_hierarchy *h, int level, int backward, const double *f, double *u,
               void *stream) {
    if (!h || !f || !u) return fail(AMG_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= h->nlev) return fail(AMG_ERR_INVALID_ARG, "level out of range");
    if (h->lev[level].coarsest) return fail(AMG_ERR_INVALID_ARG, "the coarsest level is not smoothed");
    try {
        amg::bind_stream(h, stream);
        const size_t n = (size_t)h->lev[level].n;
        Scratch tmp(h->stream);
        const double *fd = to_device(f, n, tmp);
        bool uhost = !is_device_ptr(u);
        double *ud = u;
        if (uhost) {
            ud = tmp.get<double>(n);
            AMG_CUDA(cudaMemcpyAsync(ud, u, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
        }
        amg::smooth_level(h, level, backward ? 1 : 0, fd, ud);
        if (uhost) {
            AMG_CUDA(cudaMemcpyAsync(u, ud, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
            AMG_CUDA(cudaStreamSynchronize(h->stream));
        }
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_csr_to_ell(int32_t rows, const int32_t *rowptr, const int32_t *col, const double *val,
                   int32_t width, int diag_first, int32_t *Aj, double *Ax, void *stream) {
    if (rows <= 0 || width < 0 || !rowptr || !col || !val || !Aj || !Ax)
        return fail(AMG_ERR_INVALID_ARG, "bad argument");
    try {
        cudaStream_t s = (cudaStream_t)stream;
        Scratch tmp(s);
        std::vector<int32_t> hrp;
        const int32_t *rp = rowptr;
        int nnz;
        if (is_device_ptr(rowptr)) {
            AMG_CUDA(cudaMemcpyAsync(&nnz, rowptr + rows, sizeof(int), cudaMemcpyDeviceToHost, s));
            AMG_CUDA(cudaStreamSynchronize(s));
        } else {
            nnz = rowptr[rows];
        }
        rp = to_device(rowptr, (size_t)rows + 1, tmp);
        const int32_t *cd = to_device(col, (size_t)nnz, tmp);
        const double *vd = to_device(val, (size_t)nnz, tmp);
        bool host_out = !is_device_ptr(Aj) || !is_device_ptr(Ax);
        const size_t cells = (size_t)rows * width;
        int32_t *Ajd = host_out ? tmp.get<int32_t>(cells) : Aj;
        double *Axd = host_out ? tmp.get<double>(cells) : Ax;
        int *err = tmp.get<int>(1);
        AMG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        k_csr_to_ell<<<amg::nblocks_for(rows, 256), 256, 0, s>>>(rows, rp, cd, vd, width, diag_first,
                                                                  Ajd, Axd, err);
        AMG_LAUNCH_CHECK();
        int herr = 0;
        AMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        if (host_out) {
            AMG_CUDA(cudaMemcpyAsync(Aj, Ajd, sizeof(int32_t) * cells, cudaMemcpyDeviceToHost, s));
            AMG_CUDA(cudaMemcpyAsync(Ax, Axd, sizeof(double) * cells, cudaMemcpyDeviceToHost, s));
        }
        AMG_CUDA(cudaStreamSynchronize(s));
        if (herr) return fail(AMG_ERR_INVALID_ARG, "a row has more entries than width");
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_launch_counts(const amg_hierarchy *h, int64_t *setup_launches, int64_t *solve_launches) {
    if (!h) return fail(AMG_ERR_INVALID_ARG, "NULL hierarchy");
    if (setup_launches) *setup_launches = h->setup_launches;
    if (solve_launches) *solve_launches = h->solve_launches;
    return AMG_OK;
}

int amg_profile_enable(amg_hierarchy *h, int enable) {
    if (!h) return fail(AMG_ERR_INVALID_ARG, "NULL hierarchy");
    try {
        AMG_CUDA(cudaStreamSynchronize(h->stream));
        if (enable < 0 || enable > 2) return fail(AMG_ERR_INVALID_ARG, "profiling mode is 0, 1 or 2");
        amg::profiler_enable(h, enable);
        return AMG_OK;
    }
    AMG_CATCH
}

int amg_profile_read(const amg_hierarchy *h, int capacity, int32_t *kind, int32_t *level,
                     int64_t *launches, double *ms, double *bytes, int *count) {
    if (!h || !count || capacity < 0) return fail(AMG_ERR_INVALID_ARG, "bad argument");
    *count = amg::profiler_read(h, capacity, kind, level, launches, ms, bytes);
    return AMG_OK;
}

const char *amg_kernel_name(int kind) { return amg::kernel_name(kind); }

}  // extern "C"
