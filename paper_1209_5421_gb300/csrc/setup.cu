// Setup phase on the GPU (paper Sec. 3 and Sec. 4.2-4.5):
//   validation -> auxiliary box (eq. ab12) -> level-L cell of every unknown (Sec. 4.2 index
//   formula) -> aggregates of every level by occupancy scan over the quadtree cells
//   (eqs. agg_L, agg_k; empty cells skipped) -> span and quadtree colouring (Sec. 4.5) ->
//   sweep-order permutation -> sliced-ELL operators -> Galerkin operators by per-row
//   segmented reduction into stencil slots (eq. acsum / c-sum) -> coarsest exact inverse.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "amg_internal.cuh"
#include "setup_ops.cuh"

namespace amg {
namespace {

constexpr int kT = 256;

// ---------------------------------------------------------------------------------------
// validation: square CSR, sorted unique in-range columns, positive finite diagonal, finite
// values and coordinates. Bit 1 = bad matrix, bit 2 = bad coordinate.
__global__ void k_validate(int n, int64_t nnz, const int *__restrict__ rowptr,
                           const int *__restrict__ col, const double *__restrict__ val,
                           const double *__restrict__ x, const double *__restrict__ y,
                           const double *__restrict__ z, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int flags = validate_row(i, n, nnz, rowptr, 0, col, 0, val, x, y, z);
    if (flags) atomicOr(err, flags);
}

// ---------------------------------------------------------------------------------------
// eq. ab12: a1 = min x, b1 = max x, a2 = min y, b2 = max y (exact, order-independent)
__global__ void k_minmax_partial(int n, const double *__restrict__ x,
                                 const double *__restrict__ y, double *part) {
    __shared__ double s[4][kT];
    double a1 = INFINITY, b1 = -INFINITY, a2 = INFINITY, b2 = -INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xv = x[i], yv = y[i];
        a1 = fmin(a1, xv);
        b1 = fmax(b1, xv);
        a2 = fmin(a2, yv);
        b2 = fmax(b2, yv);
    }
    s[0][threadIdx.x] = a1;
    s[1][threadIdx.x] = b1;
    s[2][threadIdx.x] = a2;
    s[3][threadIdx.x] = b2;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + o]);
            s[1][threadIdx.x] = fmax(s[1][threadIdx.x], s[1][threadIdx.x + o]);
            s[2][threadIdx.x] = fmin(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}

// one warp: min / max of the per-block partials (exact in any order)
__global__ void k_minmax_final(int nb, const double *part, double *bbox) {
    double a1 = INFINITY, b1 = -INFINITY, a2 = INFINITY, b2 = -INFINITY;
    for (int b = threadIdx.x; b < nb; b += 32) {
        a1 = fmin(a1, part[4 * b]);
        b1 = fmax(b1, part[4 * b + 1]);
        a2 = fmin(a2, part[4 * b + 2]);
        b2 = fmax(b2, part[4 * b + 3]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a1 = fmin(a1, __shfl_xor_sync(0xffffffffu, a1, o));
        b1 = fmax(b1, __shfl_xor_sync(0xffffffffu, b1, o));
        a2 = fmin(a2, __shfl_xor_sync(0xffffffffu, a2, o));
        b2 = fmax(b2, __shfl_xor_sync(0xffffffffu, b2, o));
    }
    if (threadIdx.x == 0) {
        bbox[0] = a1;
        bbox[1] = b1;
        bbox[2] = a2;
        bbox[3] = b2;
    }
}

// level-L aggregate label of every unknown (eq. agg_L): i = ty * 2^L + tx
// Cells are indexed t1 + w (t2 + w t3), w = 2^level: t3 = 0 on the quadtree, so the same
// decoding serves both trees (cell_t1 / cell_t2 / cell_t3 below).
__global__ void k_bin(int n, const double *__restrict__ x, const double *__restrict__ y,
                      const double *__restrict__ z, const double *__restrict__ bbox, int L,
                      int *__restrict__ cell) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int tx = cell_1d(x[j], bbox[0], bbox[1], L);
    int ty = cell_1d(y[j], bbox[2], bbox[3], L);
    int tz = z ? cell_1d(z[j], bbox[4], bbox[5], L) : 0;
    cell[j] = (tz * (1 << L) + ty) * (1 << L) + tx;
}
// parent cell of a cell of a grid of width w (Sec. 4.2 coarse-level form):
// ((t2 / 2) * (w / 2) + t1 / 2)
__global__ void k_parent_cell(int n, const int *__restrict__ cell, int w, int *__restrict__ pc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pc[i] = parent_cell(cell[i], w);
}

__global__ void k_mark(int n, const int *__restrict__ cid, int *__restrict__ occ) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) occ[cid[i]] = 1;
}

__global__ void k_lookup(int n, const int *__restrict__ idx, const int *__restrict__ table,
                         int *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = table[idx[i]];
}

__global__ void k_cells_of_aggs(int64_t ncell, const int *__restrict__ occ,
                                const int *__restrict__ num, int *__restrict__ cellof) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell && occ[c]) cellof[num[c]] = (int)c;
}

__global__ void k_iota(int n, int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i;
}

__global__ void k_scatter_inv(int n, const int *__restrict__ nat, int *__restrict__ inv) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) inv[nat[p]] = p;
}

// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void block_max_atomic(int v, int *out) {
    __shared__ int sm[kT / 32];
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = sm[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = max(m, sm[w]);
        atomicMax(out, m);
    }
}

// fine level: cells = level-L cells of the unknowns (CSR input order)
__global__ void k_span_csr(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                           const int *__restrict__ cell, int w, int *span) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int s = 0;
    if (i < n) {
        int ci = cell[i];
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) s = max(s, cell_dist(ci, cell[col[p]], w));
    }
    block_max_atomic(s, span);
}

// span of the next coarser operator: offsets between the parent cells (width w/2) of the
// row and column of every entry of this level (sliced ELL, pi order)
__global__ void k_span_parent(int n, const int *__restrict__ sl, const int *__restrict__ col,
                              const int *__restrict__ cell, int w, int *span) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int s = 0;
    if (i < n) {
        const int base = sl[i >> 5] + (i & 31), width = (sl[(i >> 5) + 1] - sl[i >> 5]) >> 5;
        int pi = parent_cell(cell[i], w);
        for (int k = 0; k < width; k++) {
            int c = col[base + 32 * k];
            if (c < 0) continue;
            s = max(s, cell_dist(pi, parent_cell(cell[c], w), w >> 1));
        }
    }
    block_max_atomic(s, span);
}

// colour of a cell (Sec. 4.5, modulus m = max(2, s+1)): (t1 mod m) + m (t2 mod m)
__global__ void k_colors(int n, const int *__restrict__ cell, int w, int m,
                         int *__restrict__ color) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    color[i] = cell_color(cell[i], w, m);
}

// cnt[k] += number of i with key[i] == k, keys in [0, nbins): a shared-memory histogram per
// block, then one global add per bin and block (integer counts: exact in any order)
__global__ void k_count(int n, const int *__restrict__ key, int nbins, int *__restrict__ cnt) {
    extern __shared__ int hist[];
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&hist[key[i]], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < nbins; k += blockDim.x)
        if (hist[k]) atomicAdd(&cnt[k], hist[k]);
}

// block pointers from sorted block keys (every block non-empty)
__global__ void k_bptr(int n, int nb, const int *__restrict__ key, int *__restrict__ bptr) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && (p == 0 || key[p] != key[p - 1])) bptr[key[p]] = p;
    if (p == 0) bptr[nb] = n;
}

__global__ void k_gather_idx(int m, const int *__restrict__ idx, const int *__restrict__ src,
                             int *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = src[idx[i]];
}

// ---------------------------------------------------------------------------------------
// sliced ELL construction
__global__ void k_rowlen_csr(int n, const int *__restrict__ nat, const int *__restrict__ rowptr,
                             int *__restrict__ len) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) {
        int j = nat ? nat[p] : p;
        len[p] = rowptr[j + 1] - rowptr[j];
    }
}

// one warp per slice: 32 * (longest row of the slice)
__global__ void k_slice_width(int n, int nslices, const int *__restrict__ len, int *__restrict__ sw) {
    int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (s >= nslices) return;
    int r = s * 32 + lane;
    int v = r < n ? len[r] : 0;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sw[s] = 32 * v;
}

// out[0] = max of v[0..n) (one block)
// *out = max(*out, v[0..n)) for v >= 0 (*out zeroed by the caller): block maxima, then one
// integer atomicMax per block (exact in any order)
__global__ void k_max_int(int n, const int *__restrict__ v, int *__restrict__ out) {
    __shared__ int part[kT];
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, v[i]);
    part[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] = max(part[threadIdx.x], part[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && part[0] > 0) atomicMax(out, part[0]);
}

// sl[s] = s * slots for s <= nslices (every slice `slots` = 32 w entries)
__global__ void k_uniform_slices(int nslices, int slots, int *__restrict__ sl) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s <= nslices) sl[s] = s * slots;
}

// fine operator in pi order: row p <- input row nat[p], diagonal in slot 0, then the other
// entries in CSR order, columns renumbered to pi order
__global__ void k_fill_csr(int n, const int *__restrict__ nat, const int *__restrict__ inv,
                           const int *__restrict__ rowptr, const int *__restrict__ col,
                           const double *__restrict__ val, const int *__restrict__ sl,
                           int *__restrict__ ocol, double *__restrict__ oval) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int j = nat ? nat[p] : p;
    const int base = sl[p >> 5] + (p & 31), width = (sl[(p >> 5) + 1] - sl[p >> 5]) >> 5;
    int k = 1;
    for (int q = rowptr[j]; q < rowptr[j + 1]; q++) {
        int c = col[q];
        if (c == j) {
            ocol[base] = p;
            oval[base] = val[q];
        } else {
            ocol[base + 32 * k] = inv ? inv[c] : c;
            oval[base + 32 * k] = val[q];
            k++;
        }
    }
    for (; k < width; k++) {
        ocol[base + 32 * k] = -1;
        oval[base + 32 * k] = 0.0;
    }
}

// ---------------------------------------------------------------------------------------
// Galerkin operator by segmented reduction (eq. acsum, ELL form eq. c-sum): coarse row P
// gathers the rows of its aggregate (finest level: the contiguous block bptr[P]..bptr[P+1];
// coarser levels: up to four children by quadrant), maps every column to its coarse row C
// and adds the value into the stencil slot of the cell offset C - P (|offset| <= s). Fixed
// summation order (members ascending, slots ascending): deterministic, no atomics.
// COUNT pass writes the row lengths; FILL pass writes diagonal slot first, then the touched
// slots in ascending offset order (= ascending coarse aggregate number).
template <int SMAX, bool FINE, bool FILL, int DIM>
__global__ void k_rap(int nc, const int *__restrict__ bptr, const int4 *__restrict__ children,
                      const int4 *__restrict__ children2,
                      const int *__restrict__ fsl, const int *__restrict__ fcol,
                      const double *__restrict__ fval, const int *__restrict__ fparent,
                      const int *__restrict__ ccell, int cw, int s, const int *__restrict__ csl,
                      int *__restrict__ clen, int *__restrict__ ccol,
                      double *__restrict__ cval, int *err) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= nc) return;
    rap_row<SMAX, FINE, FILL, DIM>(P, bptr, children, children2, fsl, fcol, fval, fparent, ccell,
                                   cw, s, csl, clen, ccol, cval, err);
}

// stored entries per colour (rows of colour c are the range [cr[c], cr[c+1]))
// out[c] = sum of len over colour c's rows [cr[c], cr[c+1]) (rows are in colour order):
// block (c, j) sums chunk j of the range in shared memory and adds it once (integer sums:
// exact in any order)
__global__ void k_color_nnz(const int *__restrict__ len, const int *__restrict__ cr,
                            unsigned long long *__restrict__ out) {
    __shared__ unsigned long long part[kT];
    const int c = blockIdx.x;
    const int r0 = cr[c], r1 = cr[c + 1];
    unsigned long long acc = 0;
    for (int p = r0 + blockIdx.y * blockDim.x + threadIdx.x; p < r1; p += gridDim.y * blockDim.x)
        acc += (unsigned long long)len[p];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && part[0]) atomicAdd(&out[c], part[0]);
}

// parent pi-row of every pi-row: inv_next[agg_nat[nat[p]]]
__global__ void k_parent_pi(int n, const int *__restrict__ nat, const int *__restrict__ agg_nat,
                            const int *__restrict__ inv_next, int *__restrict__ parent) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) parent[p] = inv_next[agg_nat[nat[p]]];
}

// children of every coarse pi-row by quadrant q = (t1 & 1) + 2 (t2 & 1) of the child cell
// child of its parent by quadrant / octant q = (t1&1) + 2 (t2&1) + 4 (t3&1): q < 4 in
// children, q >= 4 (octree) in children2
__global__ void k_children(int n, const int *__restrict__ parent, const int *__restrict__ cell,
                           int cw, int4 *__restrict__ children, int4 *__restrict__ children2) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int c = cell[p];
    int q = (cell_t1(c, cw) & 1) + 2 * (cell_t2(c, cw) & 1) + 4 * (cell_t3(c, cw) & 1);
    int4 *dst = q < 4 ? children : children2;
    reinterpret_cast<int *>(dst + parent[p])[q & 3] = p;
}

// ---------------------------------------------------------------------------------------
// exact coarsest solve: dense A (pi order) -> Cholesky A = L L^t -> A^{-1} = L^{-t} L^{-1}.
// One CTA; n <= kMaxCoarsest. Bit 8 of err: not positive definite.
__global__ void k_dense_from_sell(int n, const int *__restrict__ sl, const int *__restrict__ col,
                                  const double *__restrict__ val, double *__restrict__ a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int base = sl[i >> 5] + (i & 31), width = (sl[(i >> 5) + 1] - sl[i >> 5]) >> 5;
    for (int k = 0; k < width; k++) {
        int c = col[base + 32 * k];
        if (c >= 0) a[(size_t)i * n + c] += val[base + 32 * k];
    }
}

__global__ void k_chol_inverse(int n, double *ga, double *gw, double *ainv, float *ainv32,
                               int *err) {
    extern __shared__ double smat[];
    chol_inverse_block(n, ga, gw, ainv, ainv32, err, smat);
}

// ---------------------------------------------------------------------------------------
// big blocks of the finest level: flag[b] = 1 for blocks of more than kBigBlockRows rows
__global__ void k_big_flag(int nb, const int *__restrict__ bptr, int *__restrict__ flag) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) flag[b] = (bptr[b + 1] - bptr[b] > kBigBlockRows) ? 1 : 0;
}
__global__ void k_big_compact(int nb, const int *__restrict__ flag, const int *__restrict__ pos,
                              const int *__restrict__ bptr, int *__restrict__ ids,
                              int2 *__restrict__ range) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb && flag[b]) {
        ids[pos[b]] = b;
        range[pos[b]] = make_int2(bptr[b], bptr[b + 1]);
    }
}

// sweep levels of one big block per CTA: lf(i) = 1 + max lf(j) over the coupled rows j < i of
// the block (0 if none), lb(i) the same over j > i. Monotone rounds from 0 until nothing
// changes reach the longest dependency path (the fixed point) in at most depth + 1 rounds;
// values read while others write in the same round only delay convergence. Bounded by the
// block's row count.
__global__ void k_big_levels(const int2 *__restrict__ range, const int *__restrict__ rofs,
                             const int *__restrict__ sl, const int *__restrict__ col,
                             int *lf, int *lb) {
    const int k = blockIdx.x;
    const int r0 = range[k].x, m = range[k].y - range[k].x, off = rofs[k];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        lf[off + i] = 0;
        lb[off + i] = 0;
    }
    __syncthreads();
    for (int round = 0; round <= m + 1; round++) {
        int changed = 0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const int row = r0 + i, a = sl[row >> 5], w = (sl[(row >> 5) + 1] - a) >> 5;
            int vf = 0, vb = 0;
            for (int t = 0; t < w; t++) {
                const int j = col[a + 32 * t + (row & 31)] - r0;
                if (j < 0 || j >= m || j == i) continue;
                if (j < i) vf = max(vf, ((volatile int *)lf)[off + j] + 1);
                else vb = max(vb, ((volatile int *)lb)[off + j] + 1);
            }
            if (vf != lf[off + i]) {
                lf[off + i] = vf;
                changed = 1;
            }
            if (vb != lb[off + i]) {
                lb[off + i] = vb;
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
}

int read_int(const int *d, cudaStream_t s) {
    int v = 0;
    AMG_CUDA(cudaMemcpyAsync(&v, d, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    return v;
}

std::vector<int> read_ints(const int *d, int n, cudaStream_t s) {
    std::vector<int> v(n);
    if (n) {
        AMG_CUDA(cudaMemcpyAsync(v.data(), d, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        AMG_CUDA(cudaStreamSynchronize(s));
    }
    return v;
}

// stored entries of each colour's rows into lv.d_color_nnz (read back by read_color_nnz)
void color_nnz(amg_hierarchy *h, Level &lv, const int *len) {
    cudaStream_t s = h->stream;
    const int nc = (int)lv.color_rows.size() - 1;
    Scratch tmp(s);
    int *cr = tmp.get<int>(nc + 1);
    lv.d_color_nnz = halloc<unsigned long long>(h, std::max(1, nc));
    AMG_CUDA(cudaMemcpyAsync(cr, lv.color_rows.data(), sizeof(int) * (nc + 1),
                             cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaMemsetAsync(lv.d_color_nnz, 0, sizeof(unsigned long long) * nc, s));
    const int per = std::max(1, std::min(64, nblocks_for(lv.n, kT) / std::max(1, nc)));
    k_color_nnz<<<dim3(nc, per), kT, 0, s>>>(len, cr, lv.d_color_nnz);
    AMG_LAUNCH_CHECK();
}

// every level's colour counts in one pass at the end of setup (one host round trip); a
// coarse level's stored entries are their sum
void read_color_nnz(amg_hierarchy *h) {
    cudaStream_t s = h->stream;
    std::vector<std::vector<unsigned long long>> v(h->nlev);
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        if (!lv.d_color_nnz) continue;
        v[l].resize(lv.color_rows.size() - 1);
        AMG_CUDA(cudaMemcpyAsync(v[l].data(), lv.d_color_nnz,
                                 sizeof(unsigned long long) * v[l].size(),
                                 cudaMemcpyDeviceToHost, s));
    }
    AMG_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l < h->nlev; l++) {
        Level &lv = h->lev[l];
        if (!lv.d_color_nnz) continue;
        lv.color_nnz.assign(v[l].begin(), v[l].end());
        if (l > 0) {
            int64_t tot = 0;
            for (unsigned long long c : v[l]) tot += (int64_t)c;
            lv.A.stored = tot;
        }
    }
}

int bits_for(int64_t maxval) {  // bits to hold values in [0, maxval]
    int b = 1;
    while (b < 31 && (1ll << b) <= maxval) b++;
    return b;
}

// sliced-ELL slice pointers from row lengths; returns padded size. With `uniform`, every
// slice gets the widest slice's width when that costs little (width <= 9, the 3x3-cell
// stencil of a span-1 coarse level, or <= 25% more slots): a row's first slot is then
// computed, not loaded, which takes one dependent memory round trip off every row kernel.
int64_t slice_pointers(amg_hierarchy *h, Sell &A, int n, const int *len, bool uniform) {
    cudaStream_t s = h->stream;
    A.n = n;
    A.nslices = (n + 31) / 32;
    A.sl_ptr = halloc<int>(h, A.nslices + 1);
    Scratch tmp(s);
    int *sw = tmp.get<int>(A.nslices);
    k_slice_width<<<nblocks_for((int64_t)A.nslices * 32, kT), kT, 0, s>>>(n, A.nslices, len, sw);
    AMG_LAUNCH_CHECK();
    exclusive_scan(sw, A.sl_ptr, A.nslices, A.sl_ptr + A.nslices, s);
    A.uw = 0;
    int wmax = 0;
    if (uniform) {  // the padded size and the widest slice in one read
        int *d_pw = tmp.get<int>(2);
        AMG_CUDA(cudaMemcpyAsync(d_pw, A.sl_ptr + A.nslices, sizeof(int),
                                 cudaMemcpyDeviceToDevice, s));
        AMG_CUDA(cudaMemsetAsync(d_pw + 1, 0, sizeof(int), s));
        k_max_int<<<std::min(nblocks_for(A.nslices, kT), 152), kT, 0, s>>>(A.nslices, sw, d_pw + 1);
        AMG_LAUNCH_CHECK();
        const std::vector<int> pw = read_ints(d_pw, 2, s);
        A.padded = pw[0];
        wmax = pw[1] / 32;
    } else {
        A.padded = read_int(A.sl_ptr + A.nslices, s);
    }
    if (uniform) {
        const int64_t up = (int64_t)A.nslices * 32 * wmax;
        if (wmax > 0 && up <= INT32_MAX && (wmax <= 9 || up * 4 <= A.padded * 5)) {
            k_uniform_slices<<<nblocks_for(A.nslices + 1, kT), kT, 0, s>>>(A.nslices, 32 * wmax,
                                                                         A.sl_ptr);
            AMG_LAUNCH_CHECK();
            A.padded = up;
            A.uw = wmax;
        }
    }
    A.col = halloc<int>(h, A.padded);
    A.val = halloc<double>(h, A.padded);
    return A.padded;
}

// colours + stable colour sort of a level given natural cells (width w): fills nat, inv,
// color_rows; returns natural colours (device, kept for export)
void order_level(amg_hierarchy *h, Level &lv, const int *cell_nat, int *color_nat) {
    cudaStream_t s = h->stream;
    int n = lv.n;
    lv.m = std::max(2, lv.span + 1);
    lv.ncolors = lv.m * lv.m * (h->dim == 3 ? lv.m : 1);
    k_colors<<<nblocks_for(n, kT), kT, 0, s>>>(n, cell_nat, lv.cellw, lv.m, color_nat);
    AMG_LAUNCH_CHECK();
    Scratch tmp(s);
    int *keys = tmp.get<int>(n);
    int *cnt = tmp.get<int>(lv.ncolors);
    AMG_CUDA(cudaMemcpyAsync(keys, color_nat, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    lv.nat = halloc<int>(h, n);
    lv.inv = halloc<int>(h, n);
    k_iota<<<nblocks_for(n, kT), kT, 0, s>>>(n, lv.nat);
    AMG_LAUNCH_CHECK();
    stable_sort_pairs(keys, lv.nat, n, bits_for(lv.ncolors - 1), s);
    k_scatter_inv<<<nblocks_for(n, kT), kT, 0, s>>>(n, lv.nat, lv.inv);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * lv.ncolors, s));
    k_count<<<std::min(nblocks_for(n, kT), 1216), kT, sizeof(int) * lv.ncolors, s>>>(
        n, color_nat, lv.ncolors, cnt);
    AMG_LAUNCH_CHECK();
    std::vector<int> c = read_ints(cnt, lv.ncolors, s);
    lv.color_rows.assign(lv.ncolors + 1, 0);
    for (int k = 0; k < lv.ncolors; k++) lv.color_rows[k + 1] = lv.color_rows[k] + c[k];
    lv.cell = halloc<int>(h, n);
    k_gather_idx<<<nblocks_for(n, kT), kT, 0, s>>>(n, lv.nat, cell_nat, lv.cell);
    AMG_LAUNCH_CHECK();
}

template <bool FINE>
void launch_rap(amg_hierarchy *h, Level &f, Level &c, bool fill, int *len) {
    cudaStream_t s = h->stream;
    int span = c.span;
    int nb = nblocks_for(c.n, 128);
#define AMG_RAP_CASE(SM, D)                                                                 \
    if (fill)                                                                               \
        k_rap<SM, FINE, true, D><<<nb, 128, 0, s>>>(c.n, f.bptr, c.children, c.children2,   \
                                                    f.A.sl_ptr, f.A.col, f.A.val, f.parent, \
                                                    c.cell, c.cellw, span, c.A.sl_ptr,      \
                                                    nullptr, c.A.col, c.A.val, h->err_flag); \
    else                                                                                    \
        k_rap<SM, FINE, false, D><<<nb, 128, 0, s>>>(c.n, f.bptr, c.children, c.children2,  \
                                                     f.A.sl_ptr, f.A.col, f.A.val, f.parent,\
                                                     c.cell, c.cellw, span, nullptr, len,   \
                                                     nullptr, nullptr, h->err_flag);
    if (h->dim == 3) {  // octree: spans up to 2 (build_hierarchy rejects wider ones)
        if (span <= 1) {
            AMG_RAP_CASE(1, 3)
        } else {
            AMG_RAP_CASE(2, 3)
        }
    } else if (span <= 1) {
        AMG_RAP_CASE(1, 2)
    } else if (span <= 2) {
        AMG_RAP_CASE(2, 2)
    } else if (span <= 4) {
        AMG_RAP_CASE(4, 2)
    } else {
        AMG_RAP_CASE(8, 2)
    }
#undef AMG_RAP_CASE
    AMG_LAUNCH_CHECK();
}

void galerkin(amg_hierarchy *h, Level &f, Level &c, bool fine) {
    cudaStream_t s = h->stream;
    Scratch tmp(s);
    int *len = tmp.get<int>(c.n);
    if (fine) launch_rap<true>(h, f, c, false, len);
    else launch_rap<false>(h, f, c, false, len);
    slice_pointers(h, c.A, c.n, len, true);  // (stored entries: read_color_nnz)
    color_nnz(h, c, len);
    if (fine) launch_rap<true>(h, f, c, true, nullptr);
    else launch_rap<false>(h, f, c, true, nullptr);
}

// the finest level's big blocks and their level-ordered sweep schedules (forward and
// backward); the levels come from the device, the orders are built here
void build_big_blocks(amg_hierarchy *h, Level &F) {
    cudaStream_t s = h->stream;
    const int nb = F.nblocks;
    const int ncol = (int)F.color_blocks.size() - 1;
    Scratch tmp(s);
    int *flag = tmp.get<int>(nb), *pos = tmp.get<int>(nb), *tot = tmp.get<int>(1);
    k_big_flag<<<nblocks_for(nb, 256), 256, 0, s>>>(nb, F.bptr, flag);
    AMG_LAUNCH_CHECK();
    exclusive_scan(flag, pos, nb, tot, s);
    const int nbig = read_int(tot, s);
    F.nbig = nbig;
    F.color_big.assign(ncol + 1, 0);
    F.color_bigc.assign(ncol, 0);
    if (nbig == 0) return;
    int *ids_asc = tmp.get<int>(nbig);
    int2 *range_asc = tmp.get<int2>(nbig);
    k_big_compact<<<nblocks_for(nb, 256), 256, 0, s>>>(nb, flag, pos, F.bptr, ids_asc, range_asc);
    AMG_LAUNCH_CHECK();
    std::vector<int> hid = read_ints(ids_asc, nbig, s);
    std::vector<int2> hra(nbig);
    AMG_CUDA(cudaMemcpyAsync(hra.data(), range_asc, sizeof(int2) * nbig, cudaMemcpyDeviceToHost, s));
    std::vector<int> sl = read_ints(F.A.sl_ptr, F.A.nslices + 1, s);
    // colour by colour (ids ascending: colours are block ranges), warp-sized blocks first
    std::vector<int> ord;
    ord.reserve(nbig);
    for (int c = 0; c < ncol; c++) {
        const int a = (int)(std::lower_bound(hid.begin(), hid.end(), F.color_blocks[c]) - hid.begin());
        const int b = (int)(std::lower_bound(hid.begin(), hid.end(), F.color_blocks[c + 1]) - hid.begin());
        F.color_big[c] = (int)ord.size();
        for (int k = a; k < b; k++)
            if (hra[k].y - hra[k].x <= kWarpBlockRows) ord.push_back(k);
        F.color_bigc[c] = (int)ord.size();
        for (int k = a; k < b; k++)
            if (hra[k].y - hra[k].x > kWarpBlockRows) ord.push_back(k);
    }
    F.color_big[ncol] = (int)ord.size();
    std::vector<int> ids(nbig), rofs(nbig + 1, 0);
    std::vector<int2> hr(nbig);
    for (int k = 0; k < nbig; k++) {
        ids[k] = hid[ord[k]];
        hr[k] = hra[ord[k]];
        rofs[k + 1] = rofs[k] + (hr[k].y - hr[k].x);
    }
    const int R = rofs[nbig];
    int2 *range = tmp.get<int2>(nbig);
    int *d_rofs = tmp.get<int>(nbig + 1), *lf = tmp.get<int>(R), *lb = tmp.get<int>(R);
    AMG_CUDA(cudaMemcpyAsync(range, hr.data(), sizeof(int2) * nbig, cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaMemcpyAsync(d_rofs, rofs.data(), sizeof(int) * (nbig + 1),
                             cudaMemcpyHostToDevice, s));
    k_big_levels<<<nbig, 256, 0, s>>>(range, d_rofs, F.A.sl_ptr, F.A.col, lf, lb);
    AMG_LAUNCH_CHECK();
    std::vector<int> hf = read_ints(lf, R, s), hb = read_ints(lb, R, s);
    // counting sort of each block's rows by level (rows ascending inside a level); an entry
    // carries the row's first slot and slot count, so the sweep reads no slice pointer
    std::vector<int4> ent_f(R), ent_b(R);
    std::vector<int> lofs_f(nbig + 1), lofs_b(nbig + 1), lp_f, lp_b;
    auto order = [&](const std::vector<int> &lv, std::vector<int4> &ent, std::vector<int> &lofs,
                     std::vector<int> &lp) {
        for (int k = 0; k < nbig; k++) {
            const int a = rofs[k], m = rofs[k + 1] - a, r0 = hr[k].x;
            int depth = 0;
            for (int i = 0; i < m; i++) depth = std::max(depth, lv[a + i] + 1);
            std::vector<int> cnt(depth + 1, 0);
            for (int i = 0; i < m; i++) cnt[lv[a + i] + 1]++;
            for (int j = 0; j < depth; j++) cnt[j + 1] += cnt[j];
            lofs[k] = (int)lp.size();
            for (int j = 0; j < depth; j++) lp.push_back(a + cnt[j]);
            std::vector<int> fill(cnt.begin(), cnt.end() - 1);
            for (int i = 0; i < m; i++) {
                const int row = r0 + i, sa = sl[row >> 5];
                ent[a + fill[lv[a + i]]++] =
                    make_int4(row, sa + (row & 31), (sl[(row >> 5) + 1] - sa) >> 5, 0);
            }
            int ns = 0;  // the rows' off-diagonal slots, numbered in level order
            for (int i = 0; i < m; i++) {
                ent[a + i].w = ns;
                ns += ent[a + i].z - 1;
            }
            for (int vb : {4, 8}) {
                const size_t need = big_smem_bytes(m, depth, ns, vb);
                if (m > kWarpBlockRows) {
                    F.big_smem[vb == 8].push_back(need);
                } else {
                    size_t &w = F.big_smem_warp[vb == 8];
                    w = std::max(w, need);
                }
            }
        }
        lofs[nbig] = (int)lp.size();
        lp.push_back(R);
    };
    order(hf, ent_f, lofs_f, lp_f);
    order(hb, ent_b, lofs_b, lp_b);
    auto up = [&](const auto &v) {
        using E = typename std::decay_t<decltype(v)>::value_type;
        E *d = halloc<E>(h, v.size());
        AMG_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(E) * v.size(), cudaMemcpyHostToDevice, s));
        return (const E *)d;
    };
    BigSched S;
    S.nbig = nbig;
    S.ids = up(ids);
    S.lofs_f = up(lofs_f);
    S.lofs_b = up(lofs_b);
    S.lp_f = up(lp_f);
    S.lp_b = up(lp_b);
    S.ent_f = up(ent_f);
    S.ent_b = up(ent_b);
    BigSched *d = halloc<BigSched>(h, 1);
    AMG_CUDA(cudaMemcpyAsync(d, &S, sizeof S, cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaStreamSynchronize(s));  // the host vectors above are locals
    F.big_dev = d;
}

void coarsest_inverse(amg_hierarchy *h, Level &lv) {
    cudaStream_t s = h->stream;
    int n = lv.n;
    Scratch tmp(s);
    lv.Ainv = halloc<double>(h, (size_t)n * n);
    lv.Ainv32 = halloc<float>(h, 2 * (size_t)n * n);
    const size_t smem = 2 * sizeof(double) * (size_t)n * n;  // factor + inverse factor
    if (smem <= 160 * 1024) {  // n <= 102: everything in shared memory; the matrix via Ainv
        AMG_CUDA(cudaMemsetAsync(lv.Ainv, 0, sizeof(double) * n * n, s));
        k_dense_from_sell<<<nblocks_for(n, kT), kT, 0, s>>>(n, lv.A.sl_ptr, lv.A.col, lv.A.val,
                                                          lv.Ainv);
        AMG_LAUNCH_CHECK();
        // opt in to more than 48 KB once per process (thread-safe: setups may run in parallel)
        static const bool attr = [] {
            AMG_CUDA(cudaFuncSetAttribute(k_chol_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          160 * 1024));
            return true;
        }();
        (void)attr;
        k_chol_inverse<<<1, 1024, smem, s>>>(n, nullptr, nullptr, lv.Ainv, lv.Ainv32, h->err_flag);
    } else {
        double *a = tmp.get<double>((size_t)n * n);
        double *w = tmp.get<double>((size_t)n * n);
        AMG_CUDA(cudaMemsetAsync(a, 0, sizeof(double) * n * n, s));
        k_dense_from_sell<<<nblocks_for(n, kT), kT, 0, s>>>(n, lv.A.sl_ptr, lv.A.col, lv.A.val, a);
        AMG_LAUNCH_CHECK();
        k_chol_inverse<<<1, 1024, 0, s>>>(n, a, w, lv.Ainv, lv.Ainv32, h->err_flag);
    }
    AMG_LAUNCH_CHECK();
}

}  // namespace

void build_fine_big_blocks(amg_hierarchy *h) { build_big_blocks(h, h->lev[0]); }

// =======================================================================================
void build_hierarchy(amg_hierarchy *h, const amg_csr &Ain, const double *x, const double *y,
                     const double *z) {
    cudaStream_t s = h->stream;
    const int n = (int)Ain.n;
    const amg_options &o = h->opt;

    // ---- validation
    AMG_CUDA(cudaMemsetAsync(h->err_flag, 0, sizeof(int), s));
    k_validate<<<nblocks_for(n, kT), kT, 0, s>>>(n, Ain.nnz, Ain.rowptr, Ain.col, Ain.val, x, y,
                                                z, h->err_flag);
    AMG_LAUNCH_CHECK();
    int err = read_int(h->err_flag, s);
    if (err & 1) throw Error{AMG_ERR_BAD_MATRIX, "matrix is not valid SPD CSR input"};
    if (err & 2) throw Error{AMG_ERR_INVALID_ARG, "non-finite coordinate"};

    Scratch tmp(s);
    // ---- auxiliary box (eq. ab12; the octree adds [a3, b3] from z)
    const int dim = h->dim;
    double *d_bbox = tmp.get<double>(6);
    if (o.has_bbox) {
        for (int k = 0; k < 4; k++) h->bbox[k] = o.bbox[k];
        h->bbox[4] = o.zbox[0];
        h->bbox[5] = o.zbox[1];
        AMG_CUDA(cudaMemcpyAsync(d_bbox, h->bbox, sizeof(double) * 6, cudaMemcpyHostToDevice, s));
    } else {
        int nb = std::min(nblocks_for(n, kT), 1024);
        double *part = tmp.get<double>(4 * nb);
        k_minmax_partial<<<nb, kT, 0, s>>>(n, x, y, part);
        AMG_LAUNCH_CHECK();
        k_minmax_final<<<1, 32, 0, s>>>(nb, part, d_bbox);
        AMG_LAUNCH_CHECK();
        if (dim == 3) {  // (z, z): a3, b3 twice, into d_bbox[4..7]
            double *zb = tmp.get<double>(4);
            k_minmax_partial<<<nb, kT, 0, s>>>(n, z, z, part);
            AMG_LAUNCH_CHECK();
            k_minmax_final<<<1, 32, 0, s>>>(nb, part, zb);
            AMG_LAUNCH_CHECK();
            AMG_CUDA(cudaMemcpyAsync(d_bbox + 4, zb, sizeof(double) * 2, cudaMemcpyDeviceToDevice, s));
        }
        AMG_CUDA(cudaMemcpyAsync(h->bbox, d_bbox, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
    }
    // ---- depth L (Sec. 3.1): the largest L with 4^L <= n (octree: 8^L <= n)
    int L = o.aux_level;
    if (L == 0)
        while ((int64_t)1 << (dim * (L + 1)) <= (int64_t)n) L++;
    h->L = L;

    // ---- level-L cells of the unknowns
    int *cellL = tmp.get<int>(n);
    k_bin<<<nblocks_for(n, kT), kT, 0, s>>>(n, x, y, dim == 3 ? z : nullptr, d_bbox, L, cellL);
    AMG_LAUNCH_CHECK();

    // ---- aggregates of every level, natural numbering (ascending cell index)
    struct Nat {
        int n;
        int w;       // width of the grid `cell` refers to
        int *cell;   // natural cells
        int *agg;    // natural aggregate in the next level
    };
    std::vector<Nat> nat;
    nat.push_back({n, 1 << L, cellL, nullptr});
    int k = L;
    while (nat.back().n > o.coarsest_max) {
        Nat &cur = nat.back();
        const int w = 1 << k;
        const int64_t ncell = (int64_t)w * w * (dim == 3 ? w : 1);
        int *cid;
        if (nat.size() == 1) {
            cid = cur.cell;
        } else {
            cid = tmp.get<int>(cur.n);
            k_parent_cell<<<nblocks_for(cur.n, kT), kT, 0, s>>>(cur.n, cur.cell, cur.w, cid);
            AMG_LAUNCH_CHECK();
        }
        int *occ = tmp.get<int>(ncell);
        int *num = tmp.get<int>(ncell + 1);
        AMG_CUDA(cudaMemsetAsync(occ, 0, sizeof(int) * ncell, s));
        k_mark<<<nblocks_for(cur.n, kT), kT, 0, s>>>(cur.n, cid, occ);
        AMG_LAUNCH_CHECK();
        exclusive_scan(occ, num, (int)ncell, num + ncell, s);
        int nc = read_int(num + ncell, s);
        cur.agg = halloc<int>(h, cur.n);
        k_lookup<<<nblocks_for(cur.n, kT), kT, 0, s>>>(cur.n, cid, num, cur.agg);
        AMG_LAUNCH_CHECK();
        int *cellof = halloc<int>(h, nc);
        k_cells_of_aggs<<<nblocks_for(ncell, kT), kT, 0, s>>>(ncell, occ, num, cellof);
        AMG_LAUNCH_CHECK();
        nat.push_back({nc, w, cellof, nullptr});
        if (k == 0) break;
        k--;
    }
    const int nlev = (int)nat.size();
    h->nlev = nlev;
    h->lev.assign(nlev, Level());
    for (int l = 0; l < nlev; l++) {
        h->lev[l].n = nat[l].n;
        h->lev[l].cellw = nat[l].w;
        h->lev[l].agg_nat = nat[l].agg;
    }
    h->lev[nlev - 1].coarsest = true;

    // keep natural cells and colours of every level for inspection
    // (level 0's cells are the level-L cells of the unknowns)
    std::vector<int *> cell_nat(nlev), color_nat(nlev);
    cell_nat[0] = halloc<int>(h, n);
    AMG_CUDA(cudaMemcpyAsync(cell_nat[0], cellL, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    for (int l = 1; l < nlev; l++) cell_nat[l] = nat[l].cell;
    for (int l = 0; l < nlev; l++) color_nat[l] = halloc<int>(h, nat[l].n);

    // ---- span of the fine operator in level-L cells
    int *d_span = tmp.get<int>(1);
    AMG_CUDA(cudaMemsetAsync(d_span, 0, sizeof(int), s));
    k_span_csr<<<nblocks_for(n, kT), kT, 0, s>>>(n, Ain.rowptr, Ain.col, cellL, 1 << L, d_span);
    AMG_LAUNCH_CHECK();
    int span0 = read_int(d_span, s);
    if (span0 > 8) throw Error{AMG_ERR_UNSUPPORTED, "fine couplings span more than 8 auxiliary cells"};
    if (dim == 3 && span0 > 2)
        throw Error{AMG_ERR_UNSUPPORTED, "octree: fine couplings span more than 2 auxiliary cells"};

    Level &F = h->lev[0];
    F.span = span0;
    if (nlev == 1) {
        // the fine level is the coarsest: natural order, exact inverse only
        F.m = std::max(2, span0 + 1);
        F.ncolors = F.m * F.m * (dim == 3 ? F.m : 1);
        k_colors<<<nblocks_for(n, kT), kT, 0, s>>>(n, cellL, 1 << L, F.m, color_nat[0]);
        AMG_LAUNCH_CHECK();
        F.nat = halloc<int>(h, n);
        F.inv = halloc<int>(h, n);
        k_iota<<<nblocks_for(n, kT), kT, 0, s>>>(n, F.nat);
        k_iota<<<nblocks_for(n, kT), kT, 0, s>>>(n, F.inv);
        AMG_LAUNCH_CHECK();
        F.cell = cell_nat[0];
        int *len = tmp.get<int>(n);
        k_rowlen_csr<<<nblocks_for(n, kT), kT, 0, s>>>(n, nullptr, Ain.rowptr, len);
        AMG_LAUNCH_CHECK();
        slice_pointers(h, F.A, n, len, false);
        k_fill_csr<<<nblocks_for(n, kT), kT, 0, s>>>(n, nullptr, nullptr, Ain.rowptr, Ain.col,
                                                     Ain.val, F.A.sl_ptr, F.A.col, F.A.val);
        AMG_LAUNCH_CHECK();
        F.A.stored = Ain.nnz;
        F.color_rows = {0, n};
        coarsest_inverse(h, F);
    } else {
        // ---- level 1 (auxiliary level L): colours with the fine span, pi order
        Level &C1 = h->lev[1];
        C1.span = span0;  // pattern of P^t A P = cell pairs of the fine couplings
        order_level(h, C1, cell_nat[1], color_nat[1]);
        F.m = C1.m;
        F.ncolors = C1.ncolors;
        k_colors<<<nblocks_for(n, kT), kT, 0, s>>>(n, cellL, 1 << L, F.m, color_nat[0]);
        AMG_LAUNCH_CHECK();

        // ---- fine pi order: blocks = level-1 pi rows, stable in the unknown index
        int *keys = tmp.get<int>(n);
        k_lookup<<<nblocks_for(n, kT), kT, 0, s>>>(n, F.agg_nat, C1.inv, keys);
        AMG_LAUNCH_CHECK();
        F.nat = halloc<int>(h, n);
        F.inv = halloc<int>(h, n);
        k_iota<<<nblocks_for(n, kT), kT, 0, s>>>(n, F.nat);
        AMG_LAUNCH_CHECK();
        stable_sort_pairs(keys, F.nat, n, bits_for(C1.n - 1), s);
        k_scatter_inv<<<nblocks_for(n, kT), kT, 0, s>>>(n, F.nat, F.inv);
        AMG_LAUNCH_CHECK();
        F.parent = halloc<int>(h, n);
        AMG_CUDA(cudaMemcpyAsync(F.parent, keys, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
        F.nblocks = C1.n;
        F.bptr = halloc<int>(h, C1.n + 1);
        k_bptr<<<nblocks_for(n, kT), kT, 0, s>>>(n, C1.n, keys, F.bptr);
        AMG_LAUNCH_CHECK();
        F.cell = halloc<int>(h, n);
        k_gather_idx<<<nblocks_for(n, kT), kT, 0, s>>>(n, F.nat, cellL, F.cell);
        AMG_LAUNCH_CHECK();
        F.color_blocks = C1.color_rows;
        {
            int *idx = tmp.get<int>(C1.ncolors + 1);
            int *out = tmp.get<int>(C1.ncolors + 1);
            AMG_CUDA(cudaMemcpyAsync(idx, C1.color_rows.data(), sizeof(int) * (C1.ncolors + 1),
                                     cudaMemcpyHostToDevice, s));
            k_gather_idx<<<1, 256, 0, s>>>(C1.ncolors + 1, idx, F.bptr, out);
            AMG_LAUNCH_CHECK();
            F.color_rows = read_ints(out, C1.ncolors + 1, s);
        }

        // ---- fine operator in pi order
        int *len = tmp.get<int>(n);
        k_rowlen_csr<<<nblocks_for(n, kT), kT, 0, s>>>(n, F.nat, Ain.rowptr, len);
        AMG_LAUNCH_CHECK();
        slice_pointers(h, F.A, n, len, true);  // interior P1 rows: one length
        k_fill_csr<<<nblocks_for(n, kT), kT, 0, s>>>(n, F.nat, F.inv, Ain.rowptr, Ain.col, Ain.val,
                                                     F.A.sl_ptr, F.A.col, F.A.val);
        AMG_LAUNCH_CHECK();
        F.A.stored = Ain.nnz;
        color_nnz(h, F, len);
        build_big_blocks(h, F);

        // ---- A_1 = P^t A P
        galerkin(h, F, C1, true);

        // ---- coarser levels
        for (int l = 2; l < nlev; l++) {
            Level &f = h->lev[l - 1];
            Level &c = h->lev[l];
            AMG_CUDA(cudaMemsetAsync(d_span, 0, sizeof(int), s));
            k_span_parent<<<nblocks_for(f.n, kT), kT, 0, s>>>(f.n, f.A.sl_ptr, f.A.col, f.cell,
                                                              f.cellw, d_span);
            AMG_LAUNCH_CHECK();
            c.span = read_int(d_span, s);
            if (dim == 3 && c.span > 2)
                throw Error{AMG_ERR_UNSUPPORTED, "octree: a coarse operator spans more than 2 cells"};
            order_level(h, c, cell_nat[l], color_nat[l]);
            f.parent = halloc<int>(h, f.n);
            k_parent_pi<<<nblocks_for(f.n, kT), kT, 0, s>>>(f.n, f.nat, f.agg_nat, c.inv, f.parent);
            AMG_LAUNCH_CHECK();
            c.children = halloc<int4>(h, c.n);
            AMG_CUDA(cudaMemsetAsync(c.children, 0xff, sizeof(int4) * c.n, s));
            if (dim == 3) {
                c.children2 = halloc<int4>(h, c.n);
                AMG_CUDA(cudaMemsetAsync(c.children2, 0xff, sizeof(int4) * c.n, s));
            }
            k_children<<<nblocks_for(f.n, kT), kT, 0, s>>>(f.n, f.parent, f.cell, f.cellw,
                                                           c.children, c.children2);
            AMG_LAUNCH_CHECK();
            galerkin(h, f, c, false);
        }
        coarsest_inverse(h, h->lev[nlev - 1]);
    }
    read_color_nnz(h);
    err = read_int(h->err_flag, s);
    if (err & 8) throw Error{AMG_ERR_BAD_MATRIX, "coarsest operator is not positive definite"};
    if (err & 4) throw Error{AMG_ERR_CUDA, "internal error: stencil offset beyond the span"};
    // natural cells / colours for inspection live as long as the hierarchy
    for (int l = 0; l < nlev; l++) {
        h->lev[l].sc = halloc<double>(h, SC_N);
    }
    h->cell_nat = cell_nat;
    h->color_nat = color_nat;
    AMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace amg
