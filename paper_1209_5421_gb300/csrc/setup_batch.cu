// Batched setup (amg_batch_setup): the hierarchies of many independent systems built together.
//
// Every step of the single-system setup (setup.cu) runs once for all systems of the batch. A
// multi-system launch covers every participating system: system k of the launch owns a range
// of blocks and finds its own arguments in a device table (one entry per system), so the
// launch does what one launch per system would. Scans and stable sorts run once over the
// systems' data laid end to end, with keys offset per system so that every system's part of
// the result is exactly its own scan or sort. The per-element work is the functions the
// single-system setup runs (setup_ops.cuh), and the integer steps compute the same values, so
// each system's hierarchy is the one amg_setup builds, bit for bit.
//
// What changes is the host side: the setup of one system is a chain of about 240 small
// launches with a host round trip at every step that sizes the next arrays; here every step
// is one launch and one round trip for the whole batch, and the many small arrays of a
// hierarchy come from a few large allocations of its own (its Arena).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "amg_internal.cuh"
#include "setup_ops.cuh"

namespace amg {
namespace {

constexpr int kB = 256;          // threads of a multi-system launch
constexpr int kMaxColors = 81;   // m <= 9 (span <= 8): at most 81 colours on a quadtree level

int pad_rows(int n) { return (n + kB - 1) / kB * kB; }  // a system's rows: whole blocks
int blocks_of(int64_t n) { return (int)std::max<int64_t>(1, (n + kB - 1) / kB); }
int bits_of(int64_t maxval) {  // bits to hold values in [0, maxval]
    int b = 1;
    while (b < 31 && (1ll << b) <= maxval) b++;
    return b;
}

// participant of block b (vb: the first block of each of np participants, then the total)
__device__ __forceinline__ int part_of(const int *__restrict__ vb, int np, int b) {
    int lo = 0, hi = np;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (vb[mid] <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

// thread's participant k and its element index i inside that participant's range
#define MULTI_INDEX(vb, np)                                  \
    const int k_ = part_of(vb, np, (int)blockIdx.x);         \
    const int i = ((int)blockIdx.x - vb[k_]) * kB + (int)threadIdx.x

// ---------------------------------------------------------------------------------------
// Host staging: uploads of the launch tables (pinned buffer -> device buffer, both bump
// allocated, never reused before a stream synchronisation) and readbacks into pinned memory.
struct Stage {
    cudaStream_t s;
    char *hbuf = nullptr, *dbuf = nullptr, *rbuf = nullptr;
    size_t cap, used = 0, rcap, rused = 0;
    Stage(cudaStream_t s_, size_t cap_, size_t rcap_) : s(s_), cap(cap_), rcap(rcap_) {
        AMG_CUDA(cudaMallocHost(&hbuf, cap));
        AMG_CUDA(cudaMallocHost(&rbuf, rcap));
        device_alloc((void **)&dbuf, cap, s);
    }
    std::vector<std::pair<void *, void *>> extra;  // one-off buffers of tables above cap
    ~Stage() {
        cudaStreamSynchronize(s);
        if (dbuf) cudaFreeAsync(dbuf, s);
        for (auto &e : extra)
            if (e.second) cudaFreeAsync(e.second, s);
        cudaStreamSynchronize(s);
        if (hbuf) cudaFreeHost(hbuf);
        if (rbuf) cudaFreeHost(rbuf);
        for (auto &e : extra) cudaFreeHost(e.first);
    }
    // device copy of count T's (valid for kernels launched on s afterwards)
    template <class T>
    T *put(const T *src, size_t count) {
        const size_t b = (std::max<size_t>(count * sizeof(T), 1) + 255) & ~size_t(255);
        if (b > cap) {  // a table of its own (very large batches)
            void *h = nullptr, *d = nullptr;
            AMG_CUDA(cudaMallocHost(&h, b));
            extra.emplace_back(h, nullptr);
            device_alloc(&d, b, s);
            extra.back().second = d;
            std::memcpy(h, src, count * sizeof(T));
            AMG_CUDA(cudaMemcpyAsync(d, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
            return (T *)d;
        }
        if (used + b > cap) {  // every earlier upload has been read once s is idle
            AMG_CUDA(cudaStreamSynchronize(s));
            used = 0;
        }
        std::memcpy(hbuf + used, src, count * sizeof(T));
        AMG_CUDA(cudaMemcpyAsync(dbuf + used, hbuf + used, count * sizeof(T),
                                 cudaMemcpyHostToDevice, s));
        T *d = (T *)(dbuf + used);
        used += b;
        return d;
    }
    // host copy of count T's of device memory, valid after sync()
    template <class T>
    T *get(const T *dsrc, size_t count) {
        const size_t b = (std::max<size_t>(count * sizeof(T), 1) + 15) & ~size_t(15);
        if (rused + b > rcap) throw Error{AMG_ERR_UNSUPPORTED, "batched setup: readback too large"};
        T *h = (T *)(rbuf + rused);
        rused += b;
        if (count) AMG_CUDA(cudaMemcpyAsync(h, dsrc, count * sizeof(T), cudaMemcpyDeviceToHost, s));
        return h;
    }
    void sync() { AMG_CUDA(cudaStreamSynchronize(s)); }
    void reset_readbacks() { rused = 0; }  // after the values read back have been used
};

// one multi-system launch: per-participant arguments and block ranges
template <class D>
struct Multi {
    std::vector<D> d;
    std::vector<int> vb{0};
    void add(const D &x, int64_t elems) {
        d.push_back(x);
        vb.push_back(vb.back() + blocks_of(elems));
    }
    int np() const { return (int)d.size(); }
    int nblocks() const { return vb.back(); }
};

template <class D, class K>
void launch(Stage &st, const Multi<D> &m, K kern, size_t smem = 0) {
    if (m.d.empty()) return;
    const D *dd = st.put(m.d.data(), m.d.size());
    const int *dv = st.put(m.vb.data(), m.vb.size());
    kern<<<m.nblocks(), kB, smem, st.s>>>(dd, dv, m.np());
    AMG_LAUNCH_CHECK();
}

// a piece of h's arena (h is charged the arena's chunks at the end of the setup)
template <class T>
T *aget(amg_hierarchy *h, size_t count) {
    return (T *)h->arena.get(std::max<size_t>(count * sizeof(T), 16));
}

// ---------------------------------------------------------------------------------------
// kernels (one entry of the argument table per participating system)

struct DValidate {
    int n, nz0, r0;
    int64_t nnz;
    const int *rowptr, *col;  // rowptr at the system's first row; col, val at its first entry
    const double *val, *x, *y;
    int *err;
};
__global__ void kb_validate(const DValidate *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DValidate &a = D[k_];
    if (i >= a.n) return;
    const int f = validate_row(i, a.n, a.nnz, a.rowptr, a.nz0, a.col, a.r0, a.val, a.x, a.y,
                               nullptr);
    if (f) atomicOr(a.err, f);
}

// eq. ab12 per system: block partials (min / max are exact in any order), then one warp per
// system over its blocks' partials
struct DMinmax {
    int n;
    const double *x, *y;
    double *part;  // 4 per block of the launch
    double *box;   // 6 per system
};
__global__ void kb_minmax_partial(const DMinmax *__restrict__ D, const int *__restrict__ vb, int np) {
    __shared__ double s[4][kB];
    MULTI_INDEX(vb, np);
    const DMinmax &a = D[k_];
    double a1 = INFINITY, b1 = -INFINITY, a2 = INFINITY, b2 = -INFINITY;
    if (i < a.n) {
        a1 = b1 = a.x[i];
        a2 = b2 = a.y[i];
    }
    s[0][threadIdx.x] = a1;
    s[1][threadIdx.x] = b1;
    s[2][threadIdx.x] = a2;
    s[3][threadIdx.x] = b2;
    __syncthreads();
    for (int o = kB / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s[0][threadIdx.x] = fmin(s[0][threadIdx.x], s[0][threadIdx.x + o]);
            s[1][threadIdx.x] = fmax(s[1][threadIdx.x], s[1][threadIdx.x + o]);
            s[2][threadIdx.x] = fmin(s[2][threadIdx.x], s[2][threadIdx.x + o]);
            s[3][threadIdx.x] = fmax(s[3][threadIdx.x], s[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) a.part[blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}
__global__ void kb_minmax_final(const DMinmax *__restrict__ D, const int *__restrict__ vb, int np) {
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= np) return;
    const DMinmax &a = D[k];
    double a1 = INFINITY, b1 = -INFINITY, a2 = INFINITY, b2 = -INFINITY;
    for (int b = vb[k] + lane; b < vb[k + 1]; b += 32) {
        a1 = fmin(a1, a.part[4 * b]);
        b1 = fmax(b1, a.part[4 * b + 1]);
        a2 = fmin(a2, a.part[4 * b + 2]);
        b2 = fmax(b2, a.part[4 * b + 3]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a1 = fmin(a1, __shfl_xor_sync(0xffffffffu, a1, o));
        b1 = fmax(b1, __shfl_xor_sync(0xffffffffu, b1, o));
        a2 = fmin(a2, __shfl_xor_sync(0xffffffffu, a2, o));
        b2 = fmax(b2, __shfl_xor_sync(0xffffffffu, b2, o));
    }
    if (lane == 0) {
        a.box[0] = a1;
        a.box[1] = b1;
        a.box[2] = a2;
        a.box[3] = b2;
        a.box[4] = 0.0;
        a.box[5] = 0.0;
    }
}

struct DBin {
    int n, L;
    const double *x, *y, *box;
    int *cell;
};
__global__ void kb_bin(const DBin *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DBin &a = D[k_];
    if (i >= a.n) return;
    const int tx = cell_1d(a.x[i], a.box[0], a.box[1], a.L);
    const int ty = cell_1d(a.y[i], a.box[2], a.box[3], a.L);
    a.cell[i] = ty * (1 << a.L) + tx;
}

// block maximum (every thread of a block belongs to one system), then one atomicMax
__device__ __forceinline__ void block_max_to(int v, int *out) {
    __shared__ int sm[kB / 32];
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = sm[0];
        for (int w = 1; w < kB / 32; w++) m = max(m, sm[w]);
        if (m > 0) atomicMax(out, m);
    }
}

// fine-level span in level-L cells (CSR input)
struct DSpanCsr {
    int n, nz0, r0, w;
    const int *rowptr, *col, *cell;
    int *span;
};
__global__ void kb_span_csr(const DSpanCsr *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DSpanCsr &a = D[k_];
    int s = 0;
    if (i < a.n) {
        const int ci = a.cell[i];
        for (int p = a.rowptr[i] - a.nz0; p < a.rowptr[i + 1] - a.nz0; p++)
            s = max(s, cell_dist(ci, a.cell[a.col[p] - a.r0], a.w));
    }
    block_max_to(s, a.span);
}

// span of the next coarser operator from this level's sliced ELL (pi order)
struct DSpanPar {
    int n, w;
    const int *sl, *col, *cell;
    int *span;
};
__global__ void kb_span_parent(const DSpanPar *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DSpanPar &a = D[k_];
    int s = 0;
    if (i < a.n) {
        const int base = a.sl[i >> 5] + (i & 31), width = (a.sl[(i >> 5) + 1] - a.sl[i >> 5]) >> 5;
        const int pi = parent_cell(a.cell[i], a.w);
        for (int t = 0; t < width; t++) {
            const int c = a.col[base + 32 * t];
            if (c < 0) continue;
            s = max(s, cell_dist(pi, parent_cell(a.cell[c], a.w), a.w >> 1));
        }
    }
    block_max_to(s, a.span);
}

// aggregation step: cell id (this step's grid, offset by the system's cell range) and
// occupancy
struct DMark {
    int n, wprev;     // wprev = 0: the rows' cells are this step's cells (the level-L step)
    int64_t cofs;     // first cell of the system in the step's concatenated cell range
    const int *cell;  // cells of the rows (grid of width wprev, or this step's grid)
    int *cid, *occ;
};
__global__ void kb_mark(const DMark *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DMark &a = D[k_];
    if (i >= a.n) return;
    const int c = a.wprev ? parent_cell(a.cell[i], a.wprev) : a.cell[i];
    const int g = (int)(a.cofs + c);
    a.cid[i] = g;
    a.occ[g] = 1;
}
// aggregates of the step per system: num[cofs + ncell] - num[cofs]
struct DCount {
    int64_t cofs, ncell;
    const int *num;
    int *out;
};
__global__ void kb_count_aggs(const DCount *__restrict__ D, int np) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < np) *D[k].out = D[k].num[D[k].cofs + D[k].ncell] - D[k].num[D[k].cofs];
}
struct DAgg {
    int n;
    int64_t cofs;
    const int *cid, *num;
    int *agg;
};
__global__ void kb_agg(const DAgg *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DAgg &a = D[k_];
    if (i < a.n) a.agg[i] = a.num[a.cid[i]] - a.num[a.cofs];
}
struct DCellOf {
    int ncell;
    int64_t cofs;
    const int *occ, *num;
    int *cellof;
};
__global__ void kb_cellof(const DCellOf *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DCellOf &a = D[k_];
    if (i < a.ncell && a.occ[a.cofs + i]) a.cellof[a.num[a.cofs + i] - a.num[a.cofs]] = i;
}

struct DColors {
    int n, w, m;
    const int *cell;
    int *color;
};
__global__ void kb_colors(const DColors *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DColors &a = D[k_];
    if (i < a.n) a.color[i] = cell_color(a.cell[i], a.w, a.m);
}

// keys of the colour sort (system key offset + colour; padding rows after every colour of
// their system) and the per-colour counts
struct DColorKeys {
    int n, ncolors, kofs;
    const int *color;
    int *keys, *vals, *cnt;  // keys, vals at the system's rows of the concatenation
};
__global__ void kb_color_keys(const DColorKeys *__restrict__ D, const int *__restrict__ vb, int np) {
    __shared__ int hist[kMaxColors];
    MULTI_INDEX(vb, np);
    const DColorKeys &a = D[k_];
    for (int c = threadIdx.x; c < a.ncolors; c += kB) hist[c] = 0;
    __syncthreads();
    if (i < a.n) {
        const int c = a.color[i];
        a.keys[i] = a.kofs + c;
        a.vals[i] = i;
        atomicAdd(&hist[c], 1);
    } else {
        a.keys[i] = a.kofs + a.ncolors;
        a.vals[i] = -1;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < a.ncolors; c += kB)
        if (hist[c]) atomicAdd(&a.cnt[c], hist[c]);
}
// the sorted rows of a system: nat (pi row -> natural row) and its inverse
struct DPerm {
    int n;
    const int *vals;
    int *nat, *inv;
};
__global__ void kb_perm(const DPerm *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DPerm &a = D[k_];
    if (i >= a.n) return;
    const int v = a.vals[i];
    a.nat[i] = v;
    a.inv[v] = i;
}
struct DGather {
    int n;
    const int *idx, *src;
    int *out;
};
__global__ void kb_gather(const DGather *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DGather &a = D[k_];
    if (i < a.n) a.out[i] = a.src[a.idx[i]];
}

// finest level in pi order: keys = the level-1 pi row of each unknown's aggregate
struct DFineKeys {
    int n, nb, kofs;
    const int *agg, *inv1;
    int *keys, *vals;
};
__global__ void kb_fine_keys(const DFineKeys *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DFineKeys &a = D[k_];
    if (i < a.n) {
        a.keys[i] = a.kofs + a.inv1[a.agg[i]];
        a.vals[i] = i;
    } else {
        a.keys[i] = a.kofs + a.nb;
        a.vals[i] = -1;
    }
}
struct DFineUnpack {
    int n, nb, kofs;
    const int *keys, *vals;
    int *nat, *inv, *parent, *bptr;
};
__global__ void kb_fine_unpack(const DFineUnpack *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DFineUnpack &a = D[k_];
    if (i >= a.n) return;
    const int v = a.vals[i], key = a.keys[i] - a.kofs;
    a.nat[i] = v;
    a.inv[v] = i;
    a.parent[i] = key;
    if (i == 0 || a.keys[i] != a.keys[i - 1]) a.bptr[key] = i;
    if (i == 0) a.bptr[a.nb] = a.n;
}
// out[j] = *(ptr[j]) for a list of single values (colour ranges of the finest level)
__global__ void kb_gather_items(const int *const *__restrict__ ptr, int m, int *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) out[j] = *ptr[j];
}

// sliced ELL
struct DRowlen {
    int n, nz0;
    const int *nat, *rowptr;
    int *len;
};
__global__ void kb_rowlen(const DRowlen *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DRowlen &a = D[k_];
    if (i < a.n) {
        const int j = a.nat[i];
        a.len[i] = a.rowptr[j + 1] - a.rowptr[j];
    }
}
struct DSliceW {
    int n, nslices;
    const int *len;
    int *sw, *wmax;
};
__global__ void kb_slice_width(const DSliceW *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DSliceW &a = D[k_];
    const int s = i >> 5, lane = threadIdx.x & 31;
    if (s >= a.nslices) return;  // whole warps
    const int r = s * 32 + lane;
    int v = r < a.n ? a.len[r] : 0;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) {
        a.sw[s] = 32 * v;
        if (a.wmax && v > 0) atomicMax(a.wmax, v);
    }
}
struct DSlicePtr {
    int nslices;
    const int *gsl;  // the concatenation's exclusive scan at the system's first slice
    int *sl, *padded;
};
__global__ void kb_slice_ptr(const DSlicePtr *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DSlicePtr &a = D[k_];
    if (i > a.nslices) return;
    const int v = a.gsl[i] - a.gsl[0];
    a.sl[i] = v;
    if (i == a.nslices) *a.padded = v;
}
struct DUniform {
    int nslices, slots;
    int *sl;
};
__global__ void kb_uniform(const DUniform *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DUniform &a = D[k_];
    if (i <= a.nslices) a.sl[i] = i * a.slots;
}
// fine operator in pi order: row p <- input row nat[p] (diagonal in slot 0, then the other
// entries in CSR order, columns renumbered to pi order)
struct DFill {
    int n, nz0, r0;
    const int *nat, *inv, *rowptr, *col;
    const double *val;
    const int *sl;
    int *ocol;
    double *oval;
};
__global__ void kb_fill_csr(const DFill *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DFill &a = D[k_];
    if (i >= a.n) return;
    const int j = a.nat[i];
    const int base = a.sl[i >> 5] + (i & 31), width = (a.sl[(i >> 5) + 1] - a.sl[i >> 5]) >> 5;
    int t = 1;
    for (int q = a.rowptr[j] - a.nz0; q < a.rowptr[j + 1] - a.nz0; q++) {
        const int c = a.col[q] - a.r0;
        if (c == j) {
            a.ocol[base] = i;
            a.oval[base] = a.val[q];
        } else {
            a.ocol[base + 32 * t] = a.inv[c];
            a.oval[base + 32 * t] = a.val[q];
            t++;
        }
    }
    for (; t < width; t++) {
        a.ocol[base + 32 * t] = -1;
        a.oval[base + 32 * t] = 0.0;
    }
}

// stored entries of one colour of one system: one block per (system, colour) item
struct DColorNnz {
    int r0, r1;
    const int *len;
    unsigned long long *out;
};
__global__ void kb_color_nnz(const DColorNnz *__restrict__ D, int m,
                             unsigned long long *__restrict__ mirror) {
    __shared__ unsigned long long part[kB];
    const int j = blockIdx.x;
    if (j >= m) return;
    const DColorNnz &a = D[j];
    unsigned long long acc = 0;
    for (int p = a.r0 + threadIdx.x; p < a.r1; p += kB) acc += (unsigned long long)a.len[p];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kB / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *a.out = part[0];
        mirror[j] = part[0];  // every item of the launch in one array, for one readback
    }
}

// finest-level blocks of more than kBigBlockRows rows, counted per system
struct DBigCount {
    int nb;
    const int *bptr;
    int *cnt;
};
__global__ void kb_big_count(const DBigCount *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DBigCount &a = D[k_];
    const int big = (i < a.nb && a.bptr[i + 1] - a.bptr[i] > kBigBlockRows) ? 1 : 0;
    const int c = __syncthreads_count(big);
    if (threadIdx.x == 0 && c) atomicAdd(a.cnt, c);
}

// Galerkin rows (rap_row) of every system of one stencil-width group
struct DRap {
    int nc, cw, s;
    const int *bptr;
    const int4 *children;
    const int *fsl, *fcol;
    const double *fval;
    const int *fparent, *ccell, *csl;
    int *clen, *ccol;
    double *cval;
    int *err;
};
template <int SMAX, bool FINE, bool FILL>
__global__ void kb_rap(const DRap *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DRap &a = D[k_];
    if (i >= a.nc) return;
    rap_row<SMAX, FINE, FILL, 2>(i, a.bptr, a.children, nullptr, a.fsl, a.fcol, a.fval, a.fparent,
                                 a.ccell, a.cw, a.s, a.csl, a.clen, a.ccol, a.cval, a.err);
}

struct DParentPi {
    int n;
    const int *nat, *agg, *inv_next;
    int *parent;
};
__global__ void kb_parent_pi(const DParentPi *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DParentPi &a = D[k_];
    if (i < a.n) a.parent[i] = a.inv_next[a.agg[a.nat[i]]];
}
struct DChildren {
    int n, cw;
    const int *parent, *cell;
    int4 *children;
};
__global__ void kb_children_clear(const DChildren *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DChildren &a = D[k_];  // here n = coarse rows
    if (i < a.n) a.children[i] = make_int4(-1, -1, -1, -1);
}
__global__ void kb_children(const DChildren *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DChildren &a = D[k_];
    if (i >= a.n) return;
    const int c = a.cell[i];
    const int q = (cell_t1(c, a.cw) & 1) + 2 * (cell_t2(c, a.cw) & 1);
    reinterpret_cast<int *>(a.children + a.parent[i])[q] = i;
}

// coarsest level: dense matrix (zeroed first), then one CTA per system
struct DDense {
    int n;
    const int *sl, *col;
    const double *val;
    double *a;
};
__global__ void kb_zero_dense(const DDense *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DDense &a = D[k_];
    if (i < a.n * a.n) a.a[i] = 0.0;
}
__global__ void kb_dense(const DDense *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DDense &a = D[k_];
    if (i >= a.n) return;
    const int base = a.sl[i >> 5] + (i & 31), width = (a.sl[(i >> 5) + 1] - a.sl[i >> 5]) >> 5;
    for (int t = 0; t < width; t++) {
        const int c = a.col[base + 32 * t];
        if (c >= 0) a.a[(size_t)i * a.n + c] += a.val[base + 32 * t];
    }
}
struct DChol {
    int n;
    double *ga, *gw, *ainv;
    float *ainv32;
    int *err;
};
constexpr int kCholThreads = 1024;
__global__ void __launch_bounds__(kCholThreads) kb_chol(const DChol *__restrict__ D, int np) {
    extern __shared__ double smat[];
    const DChol &a = D[blockIdx.x];
    chol_inverse_block(a.n, a.ga, a.gw, a.ainv, a.ainv32, a.err, smat);
}

// solve preparation: reciprocal diagonals and FP32 copies
struct DDiag {
    int n;
    const int *sl;
    const double *val;
    double *d64;
    float *d32;
};
__global__ void kb_inv_diag(const DDiag *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DDiag &a = D[k_];
    if (i >= a.n) return;
    const double v = a.val[a.sl[i >> 5] + (i & 31)];
    a.d64[i] = (double)(1.0 / v);
    if (a.d32) a.d32[i] = (float)(1.0 / v);
}
struct DConvert {
    int n;
    const double *src;
    float *dst;
};
__global__ void kb_convert(const DConvert *__restrict__ D, const int *__restrict__ vb, int np) {
    MULTI_INDEX(vb, np);
    const DConvert &a = D[k_];
    if (i < a.n) a.dst[i] = (float)a.src[i];
}
// byte copies from the upload buffer to every hierarchy's tables, or zeros where the source
// is null (one block per item)
struct DCopy {
    const unsigned char *src;
    unsigned char *dst;
    int64_t bytes;
};
__global__ void kb_copy(const DCopy *__restrict__ D, int m) {
    const DCopy &a = D[blockIdx.x];
    for (int64_t b = threadIdx.x; b < a.bytes; b += blockDim.x) a.dst[b] = a.src ? a.src[b] : 0;
}

// ---------------------------------------------------------------------------------------
// host side

struct Sys {
    amg_hierarchy *h;
    int n, r0, nz0, nnz, L;
    int k;  // quadtree depth of the next aggregation step
    bool done = false;
    std::vector<int> ln, lw;      // rows and cell-grid width of every level
    std::vector<int *> cellnat;   // natural cells of every level
    std::vector<int *> agg;       // natural aggregate in the next level (all but the last)
    int span0 = 0;
};

int span_case(int span) { return span <= 1 ? 1 : span <= 2 ? 2 : span <= 4 ? 4 : 8; }

template <int SM>
void launch_rap_group(Stage &st, const Multi<DRap> &m, bool fine, bool fill) {
    if (m.d.empty()) return;
    if (fine) {
        if (fill) launch(st, m, kb_rap<SM, true, true>);
        else launch(st, m, kb_rap<SM, true, false>);
    } else {
        if (fill) launch(st, m, kb_rap<SM, false, true>);
        else launch(st, m, kb_rap<SM, false, false>);
    }
}

// the RAP pass of level c from level f = c - 1 for the systems `ps` (grouped by span)
void rap_pass(Stage &st, const std::vector<Sys *> &ps, int lc, bool fill,
              const std::vector<int *> &len) {
    Multi<DRap> g[4];
    for (size_t k = 0; k < ps.size(); k++) {
        amg_hierarchy *h = ps[k]->h;
        Level &f = h->lev[lc - 1], &c = h->lev[lc];
        DRap d{};
        d.nc = c.n;
        d.cw = c.cellw;
        d.s = c.span;
        d.bptr = f.bptr;
        d.children = c.children;
        d.fsl = f.A.sl_ptr;
        d.fcol = f.A.col;
        d.fval = f.A.val;
        d.fparent = f.parent;
        d.ccell = c.cell;
        d.csl = fill ? c.A.sl_ptr : nullptr;
        d.clen = fill ? nullptr : len[k];
        d.ccol = fill ? c.A.col : nullptr;
        d.cval = fill ? c.A.val : nullptr;
        d.err = h->err_flag;
        const int sc = span_case(c.span);
        g[sc == 1 ? 0 : sc == 2 ? 1 : sc == 4 ? 2 : 3].add(d, c.n);
    }
    const bool fine = (lc == 1);
    launch_rap_group<1>(st, g[0], fine, fill);
    launch_rap_group<2>(st, g[1], fine, fill);
    launch_rap_group<4>(st, g[2], fine, fill);
    launch_rap_group<8>(st, g[3], fine, fill);
}

// sliced-ELL slice pointers of level l of the systems ps from their row lengths len[k]
// (uniform: one slice width where it costs little, as the single-system setup decides);
// allocates col / val. One host round trip.
void slice_pointers_multi(Stage &st, Scratch &tmp, const std::vector<Sys *> &ps, int l,
                          const std::vector<int *> &len, bool uniform) {
    const int np = (int)ps.size();
    std::vector<int64_t> so(np + 1, 0);
    for (int k = 0; k < np; k++) so[k + 1] = so[k] + pad_rows(ps[k]->h->lev[l].n) / 32;
    if (so[np] >= INT32_MAX) throw Error{AMG_ERR_UNSUPPORTED, "batched setup: too many slices"};
    const int S = (int)so[np];
    int *sw = tmp.get<int>((size_t)S + 1);
    int *gsl = tmp.get<int>((size_t)S + 1);
    int *small = tmp.get<int>(2 * (size_t)np);  // padded, widest row
    AMG_CUDA(cudaMemsetAsync(sw, 0, sizeof(int) * ((size_t)S + 1), st.s));
    AMG_CUDA(cudaMemsetAsync(small, 0, sizeof(int) * 2 * (size_t)np, st.s));
    Multi<DSliceW> mw;
    Multi<DSlicePtr> mp;
    for (int k = 0; k < np; k++) {
        amg_hierarchy *h = ps[k]->h;
        Level &lv = h->lev[l];
        Sell &A = lv.A;
        A.n = lv.n;
        A.nslices = (lv.n + 31) / 32;
        A.uw = 0;
        A.sl_ptr = aget<int>(h, (size_t)A.nslices + 1);
        mw.add(DSliceW{lv.n, A.nslices, len[k], sw + so[k], uniform ? small + np + k : nullptr},
               (int64_t)A.nslices * 32);
        mp.add(DSlicePtr{A.nslices, gsl + so[k], A.sl_ptr, small + k}, (int64_t)A.nslices + 1);
    }
    launch(st, mw, kb_slice_width);
    exclusive_scan(sw, gsl, S + 1, nullptr, st.s);
    launch(st, mp, kb_slice_ptr);
    const int *hs = st.get(small, 2 * (size_t)np);
    st.sync();
    Multi<DUniform> mu;
    for (int k = 0; k < np; k++) {
        amg_hierarchy *h = ps[k]->h;
        Sell &A = h->lev[l].A;
        A.padded = hs[k];
        if (uniform) {
            const int wmax = hs[np + k];
            const int64_t up = (int64_t)A.nslices * 32 * wmax;
            if (wmax > 0 && up <= INT32_MAX && (wmax <= 9 || up * 4 <= A.padded * 5)) {
                mu.add(DUniform{A.nslices, 32 * wmax, A.sl_ptr}, (int64_t)A.nslices + 1);
                A.padded = up;
                A.uw = wmax;
            }
        }
        A.col = aget<int>(h, (size_t)A.padded);
        A.val = aget<double>(h, (size_t)A.padded);
    }
    st.reset_readbacks();
    launch(st, mu, kb_uniform);
}

// colour counts still on the device: where they go on the host, read back at the end
struct NnzRead {
    std::vector<Level *> lv;  // the level of every count, in the launch's item order
    unsigned long long *mirror;
};

// stored entries of every colour of level l (its colour ranges must be on the host)
void color_nnz_multi(Stage &st, Scratch &tmp, const std::vector<Sys *> &ps, int l,
                     const std::vector<int *> &len, std::vector<NnzRead> &reads) {
    std::vector<DColorNnz> items;
    NnzRead rd;
    for (size_t k = 0; k < ps.size(); k++) {
        amg_hierarchy *h = ps[k]->h;
        Level &lv = h->lev[l];
        const int nc = (int)lv.color_rows.size() - 1;
        lv.d_color_nnz = aget<unsigned long long>(h, std::max(1, nc));
        for (int c = 0; c < nc; c++) {
            items.push_back(DColorNnz{lv.color_rows[c], lv.color_rows[c + 1], len[k], lv.d_color_nnz + c});
            rd.lv.push_back(&lv);
        }
    }
    if (items.empty()) return;
    rd.mirror = tmp.get<unsigned long long>(items.size());
    const DColorNnz *d = st.put(items.data(), items.size());
    kb_color_nnz<<<(int)items.size(), kB, 0, st.s>>>(d, (int)items.size(), rd.mirror);
    AMG_LAUNCH_CHECK();
    reads.push_back(std::move(rd));
}

void galerkin_multi(Stage &st, Scratch &tmp, const std::vector<Sys *> &ps, int lc,
                    std::vector<NnzRead> &reads) {
    std::vector<int *> len(ps.size());
    for (size_t k = 0; k < ps.size(); k++) len[k] = tmp.get<int>(ps[k]->h->lev[lc].n);
    rap_pass(st, ps, lc, false, len);
    slice_pointers_multi(st, tmp, ps, lc, len, true);
    color_nnz_multi(st, tmp, ps, lc, len, reads);
    rap_pass(st, ps, lc, true, len);
}

// colours, stable colour sort (pi order), colour ranges and cells of level l >= 1 of ps
// (spans set). One host round trip.
void order_level_multi(Stage &st, Scratch &tmp, const std::vector<Sys *> &ps, int l) {
    const int np = (int)ps.size();
    std::vector<int64_t> vo(np + 1, 0);
    std::vector<int> kofs(np + 1, 0);
    for (int k = 0; k < np; k++) {
        Level &lv = ps[k]->h->lev[l];
        lv.m = std::max(2, lv.span + 1);
        lv.ncolors = lv.m * lv.m;
        if (lv.ncolors > kMaxColors) throw Error{AMG_ERR_UNSUPPORTED, "batched setup: too many colours"};
        vo[k + 1] = vo[k] + pad_rows(lv.n);
        kofs[k + 1] = kofs[k] + lv.ncolors + 1;
    }
    const int64_t R = vo[np];
    int *keys = tmp.get<int>((size_t)R), *vals = tmp.get<int>((size_t)R);
    int *cnt = tmp.get<int>((size_t)kofs[np]);
    AMG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)kofs[np], st.s));
    Multi<DColors> mc;
    Multi<DColorKeys> mk;
    Multi<DPerm> mp;
    Multi<DGather> mg;
    for (int k = 0; k < np; k++) {
        amg_hierarchy *h = ps[k]->h;
        Level &lv = h->lev[l];
        int *color = h->color_nat[l];
        mc.add(DColors{lv.n, lv.cellw, lv.m, h->cell_nat[l], color}, lv.n);
        mk.add(DColorKeys{lv.n, lv.ncolors, kofs[k], color, keys + vo[k], vals + vo[k], cnt + kofs[k]},
               pad_rows(lv.n));
        lv.nat = aget<int>(h, lv.n);
        lv.inv = aget<int>(h, lv.n);
        lv.cell = aget<int>(h, lv.n);
        mp.add(DPerm{lv.n, vals + vo[k], lv.nat, lv.inv}, lv.n);
        mg.add(DGather{lv.n, lv.nat, h->cell_nat[l], lv.cell}, lv.n);
    }
    launch(st, mc, kb_colors);
    launch(st, mk, kb_color_keys);
    stable_sort_pairs(keys, vals, (int)R, bits_of(kofs[np] - 1), st.s);
    launch(st, mp, kb_perm);
    launch(st, mg, kb_gather);
    const int *hc = st.get(cnt, (size_t)kofs[np]);
    st.sync();
    for (int k = 0; k < np; k++) {
        Level &lv = ps[k]->h->lev[l];
        lv.color_rows.assign(lv.ncolors + 1, 0);
        for (int c = 0; c < lv.ncolors; c++) lv.color_rows[c + 1] = lv.color_rows[c] + hc[kofs[k] + c];
    }
    st.reset_readbacks();
}

}  // namespace

void build_batch(const std::vector<amg_hierarchy *> &hs, const amg_csr &A, const double *x,
                 const double *y, const std::vector<BatchRows> &rows, cudaStream_t s,
                 bool batch_ws) {
    const int P = (int)hs.size();
    const amg_options &o = hs[0]->opt;
    Stage st(s, std::min<size_t>(std::max<size_t>((size_t)P << 13, size_t(1) << 20), size_t(16) << 20),
             ((size_t)P << 14) + (size_t(64) << 10));
    Scratch tmp(s);
    std::vector<NnzRead> reads;
    std::vector<Sys> sys(P);
    std::vector<Sys *> all(P);
    for (int p = 0; p < P; p++) {
        Sys &S = sys[p];
        S.h = hs[p];
        S.r0 = rows[p].r0;
        S.n = rows[p].n;
        S.nz0 = rows[p].nz0;
        S.nnz = rows[p].nnz;
        all[p] = &S;
        // the arena's first chunk: about 450 bytes per unknown for the levels and the solve
        // workspace, 540 more for a batched solve's workspace (most of it the 32 outer
        // directions), 1.2 MB of fixed buffers
        hs[p]->arena.s = s;
        hs[p]->arena.chunk = (size_t(5) << 18) + (size_t)S.n * (batch_ws ? 990 : 450);
    }
    // every hierarchy's error flag, reduction counter and grid-barrier words (zeroed)
    constexpr size_t kSmall = 512;  // bytes: err (int), counter (uint), bar[32] at 256
    std::vector<DCopy> zero(P);
    std::vector<const int *> errp(P);
    for (int p = 0; p < P; p++) {
        amg_hierarchy *h = hs[p];
        char *small = (char *)h->arena.get(kSmall);
        h->err_flag = (int *)small;
        h->red_counter = (unsigned int *)(small + 4);
        h->bar = (unsigned long long *)(small + 256);
        zero[p] = DCopy{nullptr, (unsigned char *)small, (int64_t)kSmall};
        errp[p] = h->err_flag;
    }
    {
        const DCopy *d = st.put(zero.data(), zero.size());
        kb_copy<<<P, kB, 0, s>>>(d, P);  // a null source writes zeros
        AMG_LAUNCH_CHECK();
    }
    const int *const *d_errp = st.put(errp.data(), errp.size());
    int *errs = tmp.get<int>((size_t)P);

    // ---- validation and auxiliary boxes (eq. ab12); one round trip
    double *box = tmp.get<double>(6 * (size_t)P);
    {
        Multi<DValidate> mv;
        Multi<DMinmax> mm;
        for (Sys *S : all) {
            mv.add(DValidate{S->n, S->nz0, S->r0, S->nnz, A.rowptr + S->r0, A.col + S->nz0,
                             A.val + S->nz0, x + S->r0, y + S->r0, S->h->err_flag},
                   S->n);
            mm.add(DMinmax{S->n, x + S->r0, y + S->r0, nullptr, box + 6 * (S - sys.data())}, S->n);
        }
        launch(st, mv, kb_validate);
        if (o.has_bbox) {
            std::vector<double> b(6 * (size_t)P);
            for (int p = 0; p < P; p++) {
                for (int t = 0; t < 4; t++) b[6 * p + t] = o.bbox[t];
                b[6 * p + 4] = b[6 * p + 5] = 0.0;
            }
            const double *d = st.put(b.data(), b.size());
            AMG_CUDA(cudaMemcpyAsync(box, d, sizeof(double) * b.size(), cudaMemcpyDeviceToDevice, s));
        } else {
            double *part = tmp.get<double>(4 * (size_t)mm.nblocks());
            for (DMinmax &d : mm.d) d.part = part;
            launch(st, mm, kb_minmax_partial);
            const DMinmax *dd = st.put(mm.d.data(), mm.d.size());
            const int *dv = st.put(mm.vb.data(), mm.vb.size());
            kb_minmax_final<<<(P + 7) / 8, kB, 0, s>>>(dd, dv, P);
            AMG_LAUNCH_CHECK();
        }
        const double *hb = st.get(box, 6 * (size_t)P);
        kb_gather_items<<<blocks_of(P), kB, 0, s>>>(d_errp, P, errs);
        AMG_LAUNCH_CHECK();
        const int *ef = st.get(errs, (size_t)P);
        st.sync();
        for (int p = 0; p < P; p++) {
            if (ef[p] & 1) throw Error{AMG_ERR_BAD_MATRIX, "matrix is not valid SPD CSR input"};
            if (ef[p] & 2) throw Error{AMG_ERR_INVALID_ARG, "non-finite coordinate"};
        }
        for (int p = 0; p < P; p++) {
            amg_hierarchy *h = hs[p];
            for (int t = 0; t < 6; t++) h->bbox[t] = hb[6 * p + t];
            int L = o.aux_level;
            if (L == 0)
                while ((int64_t)1 << (2 * (L + 1)) <= (int64_t)sys[p].n) L++;
            h->L = L;
            sys[p].L = L;
            sys[p].k = L;
        }
        st.reset_readbacks();
    }

    // ---- level-L cells, the fine span, and the aggregates of every level (one round trip
    // per quadtree step for the whole batch)
    int *spans = tmp.get<int>((size_t)P);
    AMG_CUDA(cudaMemsetAsync(spans, 0, sizeof(int) * P, s));
    {
        Multi<DBin> mb;
        Multi<DSpanCsr> ms;
        for (Sys *S : all) {
            amg_hierarchy *h = S->h;
            int *cell = aget<int>(h, S->n);
            S->ln.push_back(S->n);
            S->lw.push_back(1 << S->L);
            S->cellnat.push_back(cell);
            const int p = (int)(S - sys.data());
            mb.add(DBin{S->n, S->L, x + S->r0, y + S->r0, box + 6 * p, cell}, S->n);
            ms.add(DSpanCsr{S->n, S->nz0, S->r0, 1 << S->L, A.rowptr + S->r0, A.col + S->nz0, cell,
                            spans + p},
                   S->n);
        }
        launch(st, mb, kb_bin);
        launch(st, ms, kb_span_csr);
    }
    const int *hspan = nullptr;
    for (int step = 0;; step++) {
        std::vector<Sys *> act;
        for (Sys *S : all)
            if (!S->done && S->ln.back() > o.coarsest_max) act.push_back(S);
            else S->done = true;
        if (act.empty()) break;
        const int na = (int)act.size();
        std::vector<int64_t> co(na + 1, 0), ro(na + 1, 0);
        for (int k = 0; k < na; k++) {
            const int w = 1 << act[k]->k;
            co[k + 1] = co[k] + (int64_t)w * w;
            ro[k + 1] = ro[k] + act[k]->ln.back();
        }
        if (co[na] >= INT32_MAX) throw Error{AMG_ERR_UNSUPPORTED, "batched setup: too many cells"};
        const int T = (int)co[na];
        int *occ = tmp.get<int>((size_t)T + 1), *num = tmp.get<int>((size_t)T + 1);
        int *cid = tmp.get<int>((size_t)ro[na]), *nc = tmp.get<int>((size_t)na);
        AMG_CUDA(cudaMemsetAsync(occ, 0, sizeof(int) * ((size_t)T + 1), s));
        Multi<DMark> mm;
        std::vector<DCount> cnt(na);
        for (int k = 0; k < na; k++) {
            Sys *S = act[k];
            const int w = 1 << S->k;
            mm.add(DMark{S->ln.back(), step == 0 ? 0 : S->lw.back(), co[k], S->cellnat.back(),
                         cid + ro[k], occ},
                   S->ln.back());
            cnt[k] = DCount{co[k], (int64_t)w * w, num, nc + k};
        }
        launch(st, mm, kb_mark);
        exclusive_scan(occ, num, T + 1, nullptr, s);
        {
            const DCount *d = st.put(cnt.data(), cnt.size());
            kb_count_aggs<<<blocks_of(na), kB, 0, s>>>(d, na);
            AMG_LAUNCH_CHECK();
        }
        const int *hn = st.get(nc, (size_t)na);
        if (step == 0) hspan = st.get(spans, (size_t)P);
        st.sync();
        if (step == 0)
            for (int p = 0; p < P; p++) sys[p].span0 = hspan[p];
        Multi<DAgg> ma;
        Multi<DCellOf> mo;
        for (int k = 0; k < na; k++) {
            Sys *S = act[k];
            amg_hierarchy *h = S->h;
            const int w = 1 << S->k, ncl = hn[k];
            int *agg = aget<int>(h, S->ln.back());
            int *cellof = aget<int>(h, ncl);
            ma.add(DAgg{S->ln.back(), co[k], cid + ro[k], num, agg}, S->ln.back());
            mo.add(DCellOf{w * w, co[k], occ, num, cellof}, (int64_t)w * w);
            S->agg.push_back(agg);
            S->ln.push_back(ncl);
            S->lw.push_back(w);
            S->cellnat.push_back(cellof);
            if (S->k == 0) S->done = true;
            else S->k--;
        }
        st.reset_readbacks();
        launch(st, ma, kb_agg);
        launch(st, mo, kb_cellof);
    }

    // ---- the levels of every hierarchy
    int maxlev = 0;
    for (Sys *S : all) {
        amg_hierarchy *h = S->h;
        if (S->span0 > 8)
            throw Error{AMG_ERR_UNSUPPORTED, "fine couplings span more than 8 auxiliary cells"};
        const int nlev = (int)S->ln.size();
        if (nlev < 2) throw Error{AMG_ERR_CUDA, "internal error: batched setup of a one-level system"};
        h->nlev = nlev;
        h->lev.assign(nlev, Level());
        h->cell_nat.assign(nlev, nullptr);
        h->color_nat.assign(nlev, nullptr);
        for (int l = 0; l < nlev; l++) {
            Level &lv = h->lev[l];
            lv.n = S->ln[l];
            lv.cellw = S->lw[l];
            lv.agg_nat = l + 1 < nlev ? S->agg[l] : nullptr;
            h->cell_nat[l] = S->cellnat[l];
            h->color_nat[l] = aget<int>(h, lv.n);
        }
        h->lev[nlev - 1].coarsest = true;
        h->lev[0].span = S->span0;
        h->lev[1].span = S->span0;
        maxlev = std::max(maxlev, nlev);
    }

    // ---- level 1 (auxiliary level L): colours with the fine span, pi order
    order_level_multi(st, tmp, all, 1);

    // ---- finest level: colours, pi order (blocks = level-1 pi rows), operator, big blocks
    {
        std::vector<int64_t> vo(P + 1, 0);
        std::vector<int> kofs(P + 1, 0);
        for (int p = 0; p < P; p++) {
            vo[p + 1] = vo[p] + pad_rows(sys[p].n);
            kofs[p + 1] = kofs[p] + hs[p]->lev[1].n + 1;
        }
        const int64_t R = vo[P];
        int *keys = tmp.get<int>((size_t)R), *vals = tmp.get<int>((size_t)R);
        Multi<DColors> mc;
        Multi<DFineKeys> mk;
        Multi<DFineUnpack> mu;
        Multi<DGather> mg;
        for (int p = 0; p < P; p++) {
            amg_hierarchy *h = hs[p];
            Level &F = h->lev[0], &C1 = h->lev[1];
            F.m = C1.m;
            F.ncolors = C1.ncolors;
            mc.add(DColors{F.n, 1 << h->L, F.m, h->cell_nat[0], h->color_nat[0]}, F.n);
            mk.add(DFineKeys{F.n, C1.n, kofs[p], F.agg_nat, C1.inv, keys + vo[p], vals + vo[p]},
                   pad_rows(F.n));
            F.nat = aget<int>(h, F.n);
            F.inv = aget<int>(h, F.n);
            F.parent = aget<int>(h, F.n);
            F.nblocks = C1.n;
            F.bptr = aget<int>(h, (size_t)C1.n + 1);
            F.cell = aget<int>(h, F.n);
            mu.add(DFineUnpack{F.n, C1.n, kofs[p], keys + vo[p], vals + vo[p], F.nat, F.inv, F.parent,
                               F.bptr},
                   F.n);
            mg.add(DGather{F.n, F.nat, h->cell_nat[0], F.cell}, F.n);
            F.color_blocks = C1.color_rows;
        }
        launch(st, mc, kb_colors);
        launch(st, mk, kb_fine_keys);
        stable_sort_pairs(keys, vals, (int)R, bits_of(kofs[P] - 1), s);
        launch(st, mu, kb_fine_unpack);
        launch(st, mg, kb_gather);
        // colour row ranges (block boundaries), row lengths, big-block counts
        std::vector<const int *> items;
        for (int p = 0; p < P; p++) {
            const Level &F = hs[p]->lev[0];
            for (int b : F.color_blocks) items.push_back(F.bptr + b);
        }
        int *crow = tmp.get<int>(items.size());
        {
            const int *const *d = st.put(items.data(), items.size());
            kb_gather_items<<<blocks_of((int64_t)items.size()), kB, 0, s>>>(d, (int)items.size(), crow);
            AMG_LAUNCH_CHECK();
        }
        int *bigc = tmp.get<int>((size_t)P);
        AMG_CUDA(cudaMemsetAsync(bigc, 0, sizeof(int) * P, s));
        Multi<DBigCount> mb;
        Multi<DRowlen> mr;
        std::vector<int *> len(P);
        for (int p = 0; p < P; p++) {
            Level &F = hs[p]->lev[0];
            len[p] = tmp.get<int>(F.n);
            mb.add(DBigCount{F.nblocks, F.bptr, bigc + p}, F.nblocks);
            mr.add(DRowlen{F.n, sys[p].nz0, F.nat, A.rowptr + sys[p].r0, len[p]}, F.n);
        }
        launch(st, mb, kb_big_count);
        launch(st, mr, kb_rowlen);
        const int *hcr = st.get(crow, items.size());
        const int *hbig = st.get(bigc, (size_t)P);
        st.sync();
        std::vector<int> nbig(P);
        for (int p = 0, j = 0; p < P; p++) {
            Level &F = hs[p]->lev[0];
            F.color_rows.assign(hcr + j, hcr + j + F.color_blocks.size());
            j += (int)F.color_blocks.size();
            nbig[p] = hbig[p];
        }
        st.reset_readbacks();
        slice_pointers_multi(st, tmp, all, 0, len, true);
        Multi<DFill> mf;
        for (int p = 0; p < P; p++) {
            Level &F = hs[p]->lev[0];
            F.A.stored = sys[p].nnz;
            mf.add(DFill{F.n, sys[p].nz0, sys[p].r0, F.nat, F.inv, A.rowptr + sys[p].r0,
                         A.col + sys[p].nz0, A.val + sys[p].nz0, F.A.sl_ptr, F.A.col, F.A.val},
                   F.n);
        }
        launch(st, mf, kb_fill_csr);
        color_nnz_multi(st, tmp, all, 0, len, reads);
        for (int p = 0; p < P; p++) {
            Level &F = hs[p]->lev[0];
            if (nbig[p] > 0) {
                build_fine_big_blocks(hs[p]);  // the single-system code (its own round trips)
            } else {
                const int ncol = (int)F.color_blocks.size() - 1;
                F.nbig = 0;
                F.color_big.assign(ncol + 1, 0);
                F.color_bigc.assign(ncol, 0);
            }
        }
    }

    // ---- A_1 = P^t A P, then the coarser levels
    galerkin_multi(st, tmp, all, 1, reads);
    for (int l = 2; l < maxlev; l++) {
        std::vector<Sys *> ps;
        for (Sys *S : all)
            if (S->h->nlev > l) ps.push_back(S);
        const int np = (int)ps.size();
        AMG_CUDA(cudaMemsetAsync(spans, 0, sizeof(int) * np, s));
        Multi<DSpanPar> msp;
        for (int k = 0; k < np; k++) {
            Level &f = ps[k]->h->lev[l - 1];
            msp.add(DSpanPar{f.n, f.cellw, f.A.sl_ptr, f.A.col, f.cell, spans + k}, f.n);
        }
        launch(st, msp, kb_span_parent);
        const int *hsp = st.get(spans, (size_t)np);
        st.sync();
        for (int k = 0; k < np; k++) ps[k]->h->lev[l].span = hsp[k];
        st.reset_readbacks();
        order_level_multi(st, tmp, ps, l);
        Multi<DParentPi> mpp;
        Multi<DChildren> mcc, mch;
        for (int k = 0; k < np; k++) {
            amg_hierarchy *h = ps[k]->h;
            Level &f = h->lev[l - 1], &c = h->lev[l];
            f.parent = aget<int>(h, f.n);
            c.children = aget<int4>(h, c.n);
            mpp.add(DParentPi{f.n, f.nat, f.agg_nat, c.inv, f.parent}, f.n);
            mcc.add(DChildren{c.n, 0, nullptr, nullptr, c.children}, c.n);
            mch.add(DChildren{f.n, f.cellw, f.parent, f.cell, c.children}, f.n);
        }
        launch(st, mpp, kb_parent_pi);
        launch(st, mcc, kb_children_clear);
        launch(st, mch, kb_children);
        galerkin_multi(st, tmp, ps, l, reads);
    }

    // ---- coarsest levels: dense Cholesky and explicit inverse, one CTA per system
    {
        Multi<DDense> mz, md;
        std::vector<DChol> ch(P);
        size_t smem = 0;
        for (int p = 0; p < P; p++) {
            amg_hierarchy *h = hs[p];
            Level &lv = h->lev[h->nlev - 1];
            const int n = lv.n;
            lv.Ainv = aget<double>(h, (size_t)n * n);
            lv.Ainv32 = aget<float>(h, 2 * (size_t)n * n);
            const size_t need = 2 * sizeof(double) * (size_t)n * n;
            double *a = lv.Ainv, *w = nullptr;
            if (need > 160 * 1024) {  // factor and inverse factor in global scratch
                a = tmp.get<double>((size_t)n * n);
                w = tmp.get<double>((size_t)n * n);
                ch[p] = DChol{n, a, w, lv.Ainv, lv.Ainv32, h->err_flag};
            } else {
                smem = std::max(smem, need);
                ch[p] = DChol{n, nullptr, nullptr, lv.Ainv, lv.Ainv32, h->err_flag};
            }
            mz.add(DDense{n, nullptr, nullptr, nullptr, a}, (int64_t)n * n);
            md.add(DDense{n, lv.A.sl_ptr, lv.A.col, lv.A.val, a}, n);
        }
        launch(st, mz, kb_zero_dense);
        launch(st, md, kb_dense);
        static const bool attr = [] {
            AMG_CUDA(cudaFuncSetAttribute(kb_chol, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          160 * 1024));
            return true;
        }();
        (void)attr;
        const DChol *d = st.put(ch.data(), ch.size());
        kb_chol<<<P, kCholThreads, smem, s>>>(d, P);
        AMG_LAUNCH_CHECK();
    }

    // ---- every level's colour counts and the error flags (one round trip)
    {
        std::vector<const unsigned long long *> hr(reads.size());
        for (size_t r = 0; r < reads.size(); r++) hr[r] = st.get(reads[r].mirror, reads[r].lv.size());
        kb_gather_items<<<blocks_of(P), kB, 0, s>>>(d_errp, P, errs);
        AMG_LAUNCH_CHECK();
        const int *ef = st.get(errs, (size_t)P);
        st.sync();
        for (size_t r = 0; r < reads.size(); r++)
            for (size_t j = 0; j < reads[r].lv.size(); j++)
                reads[r].lv[j]->color_nnz.push_back((int64_t)hr[r][j]);
        for (int p = 0; p < P; p++) {
            amg_hierarchy *h = hs[p];
            for (int l = 1; l < h->nlev; l++) {
                Level &lv = h->lev[l];
                int64_t tot = 0;
                for (int64_t c : lv.color_nnz) tot += c;
                lv.A.stored = tot;
            }
            if (ef[p] & 8) throw Error{AMG_ERR_BAD_MATRIX, "coarsest operator is not positive definite"};
            if (ef[p] & 4) throw Error{AMG_ERR_CUDA, "internal error: stencil offset beyond the span"};
        }
        st.reset_readbacks();
    }

    // ---- what amg_setup's solve workspace and a batched solve's preparation hold
    const bool fp32 = (o.cycle_prec == AMG_FP32);
    const int kc = o.kcycle_n, maxit = o.max_iters;
    Multi<DDiag> mdg;
    Multi<DConvert> mcv;
    std::vector<DCopy> copies;
    std::vector<unsigned char> up;  // bytes to upload: level tables, direction tables, colours
    struct Pending {
        size_t off, bytes;
        void *dst;
    };
    std::vector<Pending> pend;
    auto stage = [&](void *dst, const void *src, size_t bytes) {
        const size_t off = (up.size() + 15) & ~size_t(15);
        up.resize(off + bytes);
        std::memcpy(up.data() + off, src, bytes);
        pend.push_back(Pending{off, bytes, dst});
    };
    for (int p = 0; p < P; p++) {
        amg_hierarchy *h = hs[p];
        const size_t n = (size_t)h->N;
        h->red_partials = aget<double>(h, (size_t)kRedBlocks * std::max(8, maxit + 8));
        h->cyc_partials = aget<double>(h, 2 * 4 * 1024);
        h->xo = aget<double>(h, n);
        h->ro = aget<double>(h, n);
        h->zo = aget<double>(h, n);
        h->to = aget<double>(h, n);
        h->bo = aget<double>(h, n);
        h->osc = aget<double>(h, outer_scalar_count(maxit));
        h->oit = aget<int>(h, 1);
        h->dP = aget<double *>(h, maxit);
        h->dQ = aget<double *>(h, maxit);
        for (int l = 0; l < h->nlev; l++) {
            Level &lv = h->lev[l];
            for (int prec = 0; prec < (fp32 ? 2 : 1); prec++) {
                if (l > 0) {
                    if (prec == 0) {
                        lv.v64.rhs = aget<double>(h, lv.n);
                        lv.v64.e = aget<double>(h, lv.n);
                    } else {
                        lv.v32.rhs = aget<float>(h, lv.n);
                        lv.v32.e = aget<float>(h, lv.n);
                    }
                }
                if (l > 0 && !lv.coarsest) {
                    for (int i = -1; i < kc; i++) {
                        if (prec == 0) {
                            if (i < 0) lv.v64.r = aget<double>(h, lv.n);
                            else {
                                lv.v64.p[i] = aget<double>(h, lv.n);
                                lv.v64.q[i] = aget<double>(h, lv.n);
                            }
                        } else {
                            if (i < 0) lv.v32.r = aget<float>(h, lv.n);
                            else {
                                lv.v32.p[i] = aget<float>(h, lv.n);
                                lv.v32.q[i] = aget<float>(h, lv.n);
                            }
                        }
                    }
                }
            }
            lv.dinv64 = aget<double>(h, lv.n);
            if (fp32) {
                lv.dinv32 = aget<float>(h, lv.n);
                lv.A.val32 = aget<float>(h, (size_t)lv.A.padded);
                mcv.add(DConvert{(int)lv.A.padded, lv.A.val, lv.A.val32}, lv.A.padded);
            }
            mdg.add(DDiag{lv.n, lv.A.sl_ptr, lv.A.val, lv.dinv64, fp32 ? lv.dinv32 : nullptr}, lv.n);
            lv.sc = aget<double>(h, SC_N);
        }
        h->lev[0].v64.rhs = h->ro;
        h->lev[0].v64.e = h->zo;
        if (fp32) {
            h->r32 = aget<float>(h, n);
            h->z32 = aget<float>(h, n);
            h->lev[0].v32.rhs = h->r32;
            h->lev[0].v32.e = h->z32;
        }
        // level tables (the solve's and the batch kernel's view of the levels)
        std::vector<unsigned char> img;
        for (int prec = 0; prec < (fp32 ? 2 : 1); prec++) {
            const size_t b = level_table_image(h, prec == 1, img);
            void *dst = h->arena.get(b);
            (prec == 1 ? h->lev_tab32 : h->lev_tab64) = dst;
            stage(dst, img.data(), b);
        }
        if (batch_ws) {
            // outer directions of a batched solve (as ensure_directions: in chunks of 16, each
            // vector 256-byte aligned) and the batched-solve workspace (as batch_ws)
            const int target = std::min(maxit, ((std::min(maxit, kBatchDirs) + 15) / 16) * 16);
            const size_t stride = (n + 31) & ~size_t(31);
            double *slab = aget<double>(h, 2 * (size_t)target * stride);
            for (int j = 0; j < target; j++) {
                h->P.push_back(slab + j * stride);
                h->Q.push_back(slab + (target + j) * stride);
            }
            stage(h->dP, h->P.data(), sizeof(double *) * target);
            stage(h->dQ, h->Q.data(), sizeof(double *) * target);
            BatchWs &w = h->bws;
            w.pq = aget<double>(h, maxit);
            w.bo = aget<double>(h, n);
            w.xo = aget<double>(h, n);
            w.to = aget<double>(h, n);
            std::vector<int> colors;
            for (int l = 0; l < h->nlev; l++) {
                const std::vector<int> &r = (l == 0) ? h->lev[0].color_blocks : h->lev[l].color_rows;
                w.cofs[l] = (int)colors.size();
                w.ncol[l] = std::max(0, (int)r.size() - 1);
                colors.insert(colors.end(), r.begin(), r.end());
            }
            w.colors = aget<int>(h, colors.size());
            stage(w.colors, colors.data(), sizeof(int) * colors.size());
            const Level &F = h->lev[0];
            if (F.nbig > 0) {
                std::vector<int4> bigr;
                for (size_t c = 0; c + 1 < F.color_big.size(); c++)
                    bigr.push_back(make_int4(F.color_big[c], F.color_bigc[c], F.color_big[c + 1], 0));
                w.bigr = aget<int4>(h, bigr.size());
                stage(w.bigr, bigr.data(), sizeof(int4) * bigr.size());
            }
        }
        if (fp32) h->fp32_ready = true;
    }
    launch(st, mdg, kb_inv_diag);
    launch(st, mcv, kb_convert);
    if (!up.empty()) {
        unsigned char *dup = (unsigned char *)tmp.get<unsigned char>(up.size());
        unsigned char *hup = nullptr;
        AMG_CUDA(cudaMallocHost(&hup, up.size()));
        std::memcpy(hup, up.data(), up.size());
        AMG_CUDA(cudaMemcpyAsync(dup, hup, up.size(), cudaMemcpyHostToDevice, s));
        for (const Pending &q : pend)
            copies.push_back(DCopy{dup + q.off, (unsigned char *)q.dst, (int64_t)q.bytes});
        const DCopy *d = st.put(copies.data(), copies.size());
        kb_copy<<<(int)copies.size(), kB, 0, s>>>(d, (int)copies.size());
        AMG_LAUNCH_CHECK();
        st.sync();
        cudaFreeHost(hup);
    }
    st.sync();
    for (amg_hierarchy *h : hs) h->bytes += h->arena.bytes;  // the hierarchy's chunks
}

}  // namespace amg
