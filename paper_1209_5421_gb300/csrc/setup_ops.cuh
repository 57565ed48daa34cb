// Per-element steps of the setup phase shared by the single-system setup (setup.cu) and
// the batched setup (setup_batch.cu): both run exactly these functions, so a system's
// hierarchy is the same bit for bit whichever builds it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace amg {

// ---------------------------------------------------------------------------------------
// validation of row i: square CSR, sorted unique in-range columns, positive finite diagonal,
// finite values and coordinates. Bit 1 = bad matrix, bit 2 = bad coordinate. rowptr and col
// may be those of a larger matrix: row i's entries are rowptr[i] - nz0 .. rowptr[i+1] - nz0
// of col / val, and its columns are col - r0 (0, 0 for a matrix of its own).
__device__ __forceinline__ int validate_row(int i, int n, int64_t nnz,
                                            const int *__restrict__ rowptr, int nz0,
                                            const int *__restrict__ col, int r0,
                                            const double *__restrict__ val,
                                            const double *__restrict__ x,
                                            const double *__restrict__ y,
                                            const double *__restrict__ z) {
    int flags = 0;
    int64_t b = (int64_t)rowptr[i] - nz0, e = (int64_t)rowptr[i + 1] - nz0;
    if (i == 0 && b != 0) flags |= 1;
    if (i == n - 1 && e != nnz) flags |= 1;
    if (b < 0 || e < b || e > nnz) {
        flags |= 1;
    } else {
        bool diag = false;
        int prev = -1;
        for (int64_t p = b; p < e; p++) {
            int c = col[p] - r0;
            double v = val[p];
            if (c < 0 || c >= n || c <= prev) flags |= 1;
            prev = c;
            if (!isfinite(v)) flags |= 1;
            if (c == i) {
                diag = true;
                if (!(v > 0.0)) flags |= 1;
            }
        }
        if (!diag) flags |= 1;
    }
    if (!isfinite(x[i]) || !isfinite(y[i]) || (z && !isfinite(z[i]))) flags |= 2;
    return flags;
}

// ---------------------------------------------------------------------------------------
// Sec. 4.2 index formula, one coordinate: floor((v - lo) / (hi - lo) * 2^L). Operation order
// subtract, IEEE round-to-nearest divide, exact multiply by 2^L, floor; the closed upper
// edge of the box belongs to the last cell and points outside are clamped into it.
__device__ __forceinline__ int cell_1d(double v, double lo, double hi, int L) {
    const int w = 1 << L;
    if (!(hi > lo)) return 0;
    double q = __ddiv_rn(__dsub_rn(v, lo), __dsub_rn(hi, lo));
    double s = __dmul_rn(q, (double)w);
    if (!(s >= 0.0)) return 0;
    if (s >= (double)w) return w - 1;
    return (int)floor(s);
}

// Cells are indexed t1 + w (t2 + w t3), w = 2^level: t3 = 0 on the quadtree, so the same
// decoding serves both trees.
__device__ __forceinline__ int cell_t1(int c, int w) { return c % w; }
__device__ __forceinline__ int cell_t2(int c, int w) { return (c / w) % w; }
__device__ __forceinline__ int cell_t3(int c, int w) { return c / w / w; }
// parent cell on the grid of width w/2: every coordinate halved (eq. agg_k, both trees)
__device__ __forceinline__ int parent_cell(int c, int w) {
    const int h = w >> 1;
    return ((cell_t3(c, w) >> 1) * h + (cell_t2(c, w) >> 1)) * h + (cell_t1(c, w) >> 1);
}

// span s: the largest |dt1|, |dt2| between the cells of the row and column of an entry
__device__ __forceinline__ int cell_dist(int a, int b, int w) {
    int d1 = abs(cell_t1(a, w) - cell_t1(b, w)), d2 = abs(cell_t2(a, w) - cell_t2(b, w));
    int d3 = abs(cell_t3(a, w) - cell_t3(b, w));
    return max(max(d1, d2), d3);
}

// colour of a cell (Sec. 4.5, modulus m = max(2, s+1)): (t1 mod m) + m (t2 mod m)
__device__ __forceinline__ int cell_color(int c, int w, int m) {
    return cell_t1(c, w) % m + m * (cell_t2(c, w) % m) + m * m * (cell_t3(c, w) % m);
}

// ---------------------------------------------------------------------------------------
// Galerkin operator, coarse row P, by segmented reduction (eq. acsum, ELL form eq. c-sum):
// P gathers the rows of its aggregate (finest level: the contiguous block bptr[P]..bptr[P+1];
// coarser levels: up to four children by quadrant), maps every column to its coarse row C
// and adds the value into the stencil slot of the cell offset C - P (|offset| <= s). Fixed
// summation order (members ascending, slots ascending): deterministic, no atomics.
// COUNT pass (FILL = false) writes the row length; FILL pass writes the diagonal slot first,
// then the touched slots in ascending offset order (= ascending coarse aggregate number).
template <int SMAX, bool FINE, bool FILL, int DIM>
__device__ __forceinline__ void rap_row(int P, const int *__restrict__ bptr,
                                        const int4 *__restrict__ children,
                                        const int4 *__restrict__ children2,
                                        const int *__restrict__ fsl, const int *__restrict__ fcol,
                                        const double *__restrict__ fval,
                                        const int *__restrict__ fparent,
                                        const int *__restrict__ ccell, int cw, int s,
                                        const int *__restrict__ csl, int *__restrict__ clen,
                                        int *__restrict__ ccol, double *__restrict__ cval,
                                        int *err) {
    constexpr int WMAX = 2 * SMAX + 1;
    constexpr int NS = DIM == 3 ? WMAX * WMAX * WMAX : WMAX * WMAX;
    constexpr int NKIDS = DIM == 3 ? 8 : 4;
    const int W = 2 * s + 1;
    double acc[FILL ? NS : 1];
    int cof[FILL ? NS : 1];
    unsigned long long bits[(NS + 63) / 64];
#pragma unroll
    for (int t = 0; t < (NS + 63) / 64; t++) bits[t] = 0ull;
    if (FILL) {
        for (int t = 0; t < NS; t++) acc[t] = 0.0;
    }
    const int cP = ccell[P];
    const int p1 = cell_t1(cP, cw), p2 = cell_t2(cP, cw), p3 = cell_t3(cP, cw);
    int rbeg, rend;
    int kids[NKIDS];
    if (FINE) {
        rbeg = bptr[P];
        rend = bptr[P + 1];
    } else {
        int4 ch = children[P];
        kids[0] = ch.x;
        kids[1] = ch.y;
        kids[2] = ch.z;
        kids[3] = ch.w;
        if constexpr (DIM == 3) {
            int4 c2 = children2[P];
            kids[4] = c2.x;
            kids[5] = c2.y;
            kids[6] = c2.z;
            kids[7] = c2.w;
        }
        rbeg = 0;
        rend = NKIDS;
    }
    for (int it = rbeg; it < rend; it++) {
        int i = FINE ? it : kids[it];
        if (i < 0) continue;
        const int base = fsl[i >> 5] + (i & 31), width = (fsl[(i >> 5) + 1] - fsl[i >> 5]) >> 5;
        for (int k = 0; k < width; k++) {
            int c = fcol[base + 32 * k];
            if (c < 0) continue;
            int C = fparent[c];
            int cC = ccell[C];
            int d1 = cell_t1(cC, cw) - p1, d2 = cell_t2(cC, cw) - p2, d3 = cell_t3(cC, cw) - p3;
            if (d1 < -s || d1 > s || d2 < -s || d2 > s || d3 < -s || d3 > s) {
                atomicOr(err, 4);
                continue;
            }
            // slots in ascending offset order (d3, d2, d1) = ascending coarse cell index
            int t = ((DIM == 3 ? (d3 + s) * W : 0) + (d2 + s)) * W + (d1 + s);
            bits[t >> 6] |= 1ull << (t & 63);
            if (FILL) {
                acc[t] += fval[base + 32 * k];
                cof[t] = C;
            }
        }
    }
    const int center = DIM == 3 ? (s * W + s) * W + s : s * W + s;
    const int nslot = DIM == 3 ? W * W * W : W * W;
    if (!FILL) {
        int cnt = 0;
#pragma unroll
        for (int t = 0; t < (NS + 63) / 64; t++) cnt += __popcll(bits[t]);
        if (!((bits[center >> 6] >> (center & 63)) & 1ull)) cnt++;  // diagonal always stored
        clen[P] = cnt;
        return;
    }
    const int base = csl[P >> 5] + (P & 31), width = (csl[(P >> 5) + 1] - csl[P >> 5]) >> 5;
    ccol[base] = P;
    cval[base] = acc[center];
    int k = 1;
    for (int t = 0; t < nslot; t++) {
        if (t == center || !((bits[t >> 6] >> (t & 63)) & 1ull)) continue;
        ccol[base + 32 * k] = cof[t];
        cval[base + 32 * k] = acc[t];
        k++;
    }
    for (; k < width; k++) {
        ccol[base + 32 * k] = -1;
        cval[base + 32 * k] = 0.0;
    }
}


// ---------------------------------------------------------------------------------------
// exact coarsest solve, one CTA: dense A -> Cholesky A = L L^t -> A^{-1} = L^{-t} L^{-1}.
// The factor and the inverse factor live in shared memory (smat, 2 n^2 doubles) when ga is
// null -- the dense matrix then arrives in ainv --, else in the global scratch ga, gw. Bit 8
// of err: not positive definite. ainv32 receives the inverse as float high parts, then low
// parts.
__device__ __forceinline__ void chol_inverse_block(int n, double *ga, double *gw, double *ainv,
                                                   float *ainv32, int *err, double *smat) {
    // the factor and the inverse factor live in shared memory when they fit (every access
    // of the n^3 loops is then a shared-memory access), else in the global scratch
    const bool in_smem = (ga == nullptr);
    double *a = in_smem ? smat : ga;
    double *w = in_smem ? smat + (size_t)n * n : gw;
    __shared__ int bad;
    const int t = threadIdx.x, T = blockDim.x;
    if (t == 0) bad = 0;
    if (in_smem)
        for (int e = t; e < n * n; e += T) a[e] = ainv[e];  // the dense matrix arrives in ainv
    __syncthreads();
    const int lane = t & 31, warp = t >> 5, nwarp = T >> 5;
    for (int j = 0; j < n; j++) {
        if (t == 0) {
            double d = a[(size_t)j * n + j];
            if (!(d > 0.0) || !isfinite(d)) bad = 1;
            a[(size_t)j * n + j] = sqrt(fabs(d));
        }
        __syncthreads();
        if (bad) break;
        double djj = a[(size_t)j * n + j];
        for (int i = j + 1 + t; i < n; i += T) a[(size_t)i * n + j] /= djj;
        __syncthreads();
        // trailing update of the lower triangle, a warp per row (each entry once per j)
        for (int i = j + 1 + warp; i < n; i += nwarp) {
            const double lij = a[(size_t)i * n + j];
            for (int k = j + 1 + lane; k <= i; k += 32) a[(size_t)i * n + k] -= lij * a[(size_t)k * n + j];
        }
        __syncthreads();
    }
    if (bad) {
        if (t == 0) atomicOr(err, 8);
        return;
    }
    // W = L^{-1} (lower), one column per thread
    for (int c = t; c < n; c += T) {
        for (int i = 0; i < c; i++) w[(size_t)i * n + c] = 0.0;
        for (int i = c; i < n; i++) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; k++) s -= a[(size_t)i * n + k] * w[(size_t)k * n + c];
            w[(size_t)i * n + c] = s / a[(size_t)i * n + i];
        }
    }
    __syncthreads();
    // A^{-1} = W^t W: entry (i, j), i >= j, and its mirror (the same sum: products commute)
    const int tri = n * (n + 1) / 2;
    for (int q = t; q < tri; q += T) {
        int i = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);  // q = i (i+1) / 2 + j
        while (i * (i + 1) / 2 > q) i--;
        while ((i + 1) * (i + 2) / 2 <= q) i++;
        const int j = q - i * (i + 1) / 2;
        double s = 0.0;
        for (int k = i; k < n; k++) s += w[(size_t)k * n + i] * w[(size_t)k * n + j];
        const float hi = (float)s;  // FP32 cycle: high and low parts, s ~ hi + lo
        const float lo = (float)(s - (double)hi);
        for (int m = 0; m < (i == j ? 1 : 2); m++) {
            const size_t e = m == 0 ? (size_t)i * n + j : (size_t)j * n + i;
            ainv[e] = s;
            ainv32[e] = hi;
            ainv32[(size_t)n * n + e] = lo;
        }
    }
}

}  // namespace amg
