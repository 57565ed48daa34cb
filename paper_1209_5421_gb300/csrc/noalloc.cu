// amg_csr_to_ell_noalloc: the CSR -> ELL packer of amg_csr_to_ell without any allocation.
//
// Some callers cannot allocate device memory when they call into this library: a host
// application whose device memory is entirely owned by another allocator (a framework pool
// that reserved the whole GPU up front), or a latency-critical loop that forbids allocation
// calls. amg_csr_to_ell allocates a status word (and, for host arrays, staging buffers);
// this variant takes device arrays only and keeps its scratch -- one overflow count per
// 256-row block plus the combined count -- in the file-scope array below.
//
// The array lives in every GPU that loads this library, until the process exits. All calls
// on a device share it and it keeps the last call's contents: every block writes its own
// slot and the combining kernel overwrites the total, so nothing has to be cleared between
// calls, but calls whose kernels overlap on the GPU (different streams, or different host
// threads) race on it and must be ordered by the caller.
#include <stdio.h>

#include <mutex>

#include "amg_internal.cuh"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 16384;  // rows <= 16384 * 256 = 4,194,304
constexpr int kNoAllocMaxRows = kNoAllocMaxBlocks * kNoAllocThreads;

// [0, kNoAllocMaxBlocks): overflow count of each block; [kNoAllocMaxBlocks]: the total
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocMaxBlocks + 1];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
int *g_scratch_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// once per device, with that device current: the device address of the scratch array (in
// host code the array's name is only a host-side stand-in, never a device address)
int scratch_address(int dev, int **out) {
    if (dev < 0 || dev >= kMaxDevices) return AMG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return AMG_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (int *)p;
    }
    *out = g_scratch_ptr[dev];
    return AMG_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// one thread per row: ELL entries of the row (diagonal first if asked, padding -1 / 0), and
// the number of rows of this block longer than `width` into scratch[blockIdx.x]
__global__ void __launch_bounds__(kNoAllocThreads)
k_csr_to_ell_noalloc(int rows, const int *__restrict__ rowptr, const int *__restrict__ col,
                     const double *__restrict__ val, int width, int diag_first,
                     int *__restrict__ Aj, double *__restrict__ Ax, int *__restrict__ scratch) {
    __shared__ int over;
    if (threadIdx.x == 0) over = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < rows) {
        const int b = rowptr[i], e = rowptr[i + 1];
        if (e - b > width) {
            atomicAdd(&over, 1);
        } else {
            int k = 0, dpos = -1;
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
    }
    __syncthreads();
    if (threadIdx.x == 0) scratch[blockIdx.x] = over;
}

// scratch[kNoAllocMaxBlocks] = sum of the per-block counts (one block, fixed order)
__global__ void __launch_bounds__(kNoAllocThreads) k_noalloc_total(int nblocks, int *scratch) {
    __shared__ int part[kNoAllocThreads];
    int s = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += scratch[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = kNoAllocThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[kNoAllocMaxBlocks] = part[0];
}

// a CUDA error of this call: its text becomes amg_last_error's, the error is cleared
int cuda_fail(cudaError_t e, const char *where) {
    static thread_local char msg[192];
    snprintf(msg, sizeof msg, "%s: %s", where, cudaGetErrorString(e));
    cudaGetLastError();
    return amg::set_last_error(AMG_ERR_CUDA, msg);
}

}  // namespace

extern "C" int amg_csr_to_ell_noalloc(int32_t rows, const int32_t *rowptr, const int32_t *col,
                                      const double *val, int32_t width, int diag_first,
                                      int32_t *Aj, double *Ax, void *stream) {
    if (rows <= 0 || width < 0 || !rowptr || !col || !val || !Aj || !Ax)
        return amg::set_last_error(AMG_ERR_INVALID_ARG, "bad argument");
    if (rows > kNoAllocMaxRows)  // beyond the static scratch
        return amg::set_last_error(AMG_ERR_UNSUPPORTED,
                                   "rows above the allocation-free packer's limit (4,194,304)");
    cudaStream_t s = (cudaStream_t)stream;
    // the call reads its result back and waits on the stream, which a stream under capture
    // does not allow (and which would end the caller's capture): refuse it untouched
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return amg::set_last_error(AMG_ERR_UNSUPPORTED,
                                   "the allocation-free packer waits on its stream: not while "
                                   "the stream is capturing");
    if (!on_device(rowptr) || !on_device(col) || !on_device(val) || !on_device(Aj) ||
        !on_device(Ax))  // host arrays would need staging buffers
        return amg::set_last_error(AMG_ERR_INVALID_ARG,
                                   "the allocation-free packer takes device arrays only");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int *scratch = nullptr;
    int st = scratch_address(dev, &scratch);
    if (st == AMG_ERR_UNSUPPORTED)
        return amg::set_last_error(st, "device ordinal above the packer's device table");
    if (st != AMG_OK) return amg::set_last_error(st, "cudaGetSymbolAddress of the packer's scratch failed");
    const int nblocks = (rows + kNoAllocThreads - 1) / kNoAllocThreads;
    // cudaLaunchKernel returns the status of its own launch, so an error left pending on this
    // thread by other code is neither taken for this call's nor cleared here
    {
        int r = rows, w = width, df = diag_first;
        const int *rp = rowptr, *cl = col;
        const double *vl = val;
        int *aj = Aj, *sc = scratch;
        double *ax = Ax;
        void *args[] = {&r, &rp, &cl, &vl, &w, &df, &aj, &ax, &sc};
        e = cudaLaunchKernel((const void *)k_csr_to_ell_noalloc, dim3(nblocks),
                             dim3(kNoAllocThreads), args, 0, s);
        if (e != cudaSuccess) return cuda_fail(e, "packing kernel launch");
        int nb = nblocks;
        void *args2[] = {&nb, &sc};
        e = cudaLaunchKernel((const void *)k_noalloc_total, dim3(1), dim3(kNoAllocThreads), args2,
                             0, s);
        if (e != cudaSuccess) return cuda_fail(e, "count kernel launch");
    }
    int over = 0;
    e = cudaMemcpyAsync(&over, scratch + kNoAllocMaxBlocks, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the overflow count");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (over)  // some row has more than `width` entries
        return amg::set_last_error(AMG_ERR_INVALID_ARG, "a row has more entries than width");
    return AMG_OK;
}
