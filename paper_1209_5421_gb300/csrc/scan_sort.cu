// Deterministic device-wide exclusive scan and stable LSD radix sort (setup primitives:
// aggregate numbering by occupancy scan, paper Sec. 3.2 / 4.2, and the sweep-order
// permutation of Sec. 4.5).
#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;                       // items per thread
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// exclusive scan of one value per thread across the block; *total = block sum
__device__ int block_excl_scan(int v, int *smem, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = warp_incl_scan(v);
    if (lane == 31) smem[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? smem[lane] : 0;
        t = warp_incl_scan(t);
        smem[lane] = t;
    }
    __syncthreads();
    int wofs = w ? smem[w - 1] : 0;
    *total = smem[nw - 1];
    __syncthreads();
    return wofs + x - v;
}

__global__ void k_tile_sums(const int *__restrict__ in, int n, int *__restrict__ sums) {
    __shared__ int smem[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < n) s += in[base + k];
    int total;
    block_excl_scan(s, smem, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_tile_scan(const int *in, int n, int *out, const int *__restrict__ offs,
                            int *d_total) {
    __shared__ int smem[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int pre = block_excl_scan(s, smem, &total) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) out[base + k] = pre;
        pre += v[k];
    }
    if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *d_total = pre;
}

}  // namespace

void exclusive_scan(const int *in, int *out, int n, int *d_total, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) AMG_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int), s));
        return;
    }
    int tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_tile_scan<<<1, kScanThreads, 0, s>>>(in, n, out, nullptr, d_total);
        AMG_LAUNCH_CHECK();
        return;
    }
    Scratch tmp(s);
    int *sums = tmp.get<int>(tiles);
    k_tile_sums<<<tiles, kScanThreads, 0, s>>>(in, n, sums);
    AMG_LAUNCH_CHECK();
    exclusive_scan(sums, sums, tiles, nullptr, s);
    k_tile_scan<<<tiles, kScanThreads, 0, s>>>(in, n, out, sums, d_total);
    AMG_LAUNCH_CHECK();
}

// ---- stable radix sort ----------------------------------------------------------------
namespace {

constexpr int kSortThreads = 256;        // = number of digits
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kDigits = 256;

__global__ void k_digit_hist(const int *__restrict__ keys, int n, int shift, int ntiles,
                             int *__restrict__ cnt) {
    __shared__ int h[kDigits];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; r++) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    cnt[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];  // digit-major
}

__global__ void k_digit_scatter(const int *__restrict__ kin, const int *__restrict__ vin,
                                int n, int shift, int ntiles, const int *__restrict__ offs,
                                int *__restrict__ kout, int *__restrict__ vout) {
    __shared__ int running[kDigits];
    __shared__ int wcnt[kSortThreads / 32][kDigits];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    running[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; w++) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; r++) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        bool valid = i < n;
        int key = valid ? kin[i] : 0;
        int val = valid ? vin[i] : 0;
        int d = valid ? ((key >> shift) & 255) : kDigits;  // sentinel for missing items
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int before = 0;
            for (int w = 0; w < warp; w++) before += wcnt[w][d];
            int pos = running[d] + before + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; w++) {
            tot += wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = 0;
        }
        running[threadIdx.x] += tot;
        __syncthreads();
    }
}

}  // namespace

void stable_sort_pairs(int *keys, int *vals, int n, int key_bits, cudaStream_t s) {
    if (n <= 1) return;
    int ntiles = (n + kSortTile - 1) / kSortTile;
    Scratch tmp(s);
    int *k2 = tmp.get<int>(n);
    int *v2 = tmp.get<int>(n);
    int *cnt = tmp.get<int>((size_t)kDigits * ntiles);
    int *ka = keys, *va = vals, *kb = k2, *vb = v2;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_digit_hist<<<ntiles, kSortThreads, 0, s>>>(ka, n, shift, ntiles, cnt);
        AMG_LAUNCH_CHECK();
        exclusive_scan(cnt, cnt, kDigits * ntiles, nullptr, s);
        k_digit_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, n, shift, ntiles, cnt, kb, vb);
        AMG_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
        passes++;
    }
    if (passes & 1) {
        AMG_CUDA(cudaMemcpyAsync(keys, ka, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
        AMG_CUDA(cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace amg
