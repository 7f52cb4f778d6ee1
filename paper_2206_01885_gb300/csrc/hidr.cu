// hidr.cu -- hierarchical data reduction (section 3, Algorithm 1 of
// arXiv 2206.01885) with the volume-based DataReduct of section 3.3.
//
// DataReduct(S, g^d): S itself (sorted) when |S| <= g^d; otherwise, for each
// of the g^d cell-centred points q of a tensor grid on the bounding box of S,
// the point of S nearest to q (float64 squared distance evaluated in a fixed
// order without contraction; ties to the smaller Morton position), then the
// distinct winners sorted.  One CTA reduces one node's set; all nodes of a
// level run in one launch.
#include <climits>

#include <mutex>

#include "h2_internal.cuh"

namespace h2 {
namespace {

constexpr int DR_THREADS = 256;
constexpr int DR_TILE = 256;  // points staged in shared memory per pass
constexpr int DR_GPT = 4;     // grid points per thread per sweep
constexpr int DR_MAX_GRID = 16384;

// ---------------------------------------------------------------- sizes
// |S_i|: the leaf's points, or the sum of the children's |X_c*|
__global__ void k_size_up(int lb, int nl, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                          const int32_t *end, const int32_t *xcnt, int g, int d, int64_t *sz, int64_t *cap) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nl) return;
    int i = lb + a;
    int64_t s = 0;
    if (nchild[i] == 0) s = end[i] - begin[i];
    else
        for (int c = fchild[i]; c < fchild[i] + nchild[i]; c++) s += xcnt[c];
    int64_t G = 1;
    for (int k = 0; k < d; k++) G *= g;
    sz[a] = s;
    cap[a] = s < G ? s : G;
}

// |T_i| = |Y_p*| + sum over j in IL(i) of |X_j*|; one warp per node.  With
// szl (the interaction-list reduction), szl[a] = the interaction-list part's
// size, capl[a] its reduced set's capacity, and cap[a] holds both reductions.
// psz[a] (when given) = |Y_p*|.
__global__ void k_size_down(int lb, int nl, const int32_t *parent, const int64_t *far_ptr, const int32_t *far_idx,
                            const int32_t *xcnt, const int32_t *ycnt, int g, int d, int64_t *sz, int64_t *cap,
                            int64_t *szl, int64_t *capl, int64_t *psz) {
    int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (a >= nl) return;
    int i = lb + a;
    int64_t s = 0;
    for (int64_t e = far_ptr[i] + lane; e < far_ptr[i + 1]; e += 32) s += xcnt[far_idx[e]];
    s = warp_sum(s);
    if (lane == 0) {
        const int64_t sl = s;
        s += ycnt[parent[i]];
        if (psz) psz[a] = ycnt[parent[i]];
        int64_t G = 1;
        for (int k = 0; k < d; k++) G *= g;
        sz[a] = s;
        cap[a] = s < G ? s : G;
        if (szl) {
            const int64_t cl = sl < G ? sl : G;
            szl[a] = sl;
            capl[a] = cl;
            cap[a] += cl;
        }
    }
}

// --------------------------------------------------------------- gathers
// Bounding boxes are kept as order-preserving integer keys of the float64
// coordinates (see dkey): box[6 * i + k] = min key, box[6 * i + 3 + k] = max
// key of coordinate k; an empty set has (LLONG_MAX, LLONG_MIN).  The box of a
// union is the componentwise min / max of its parts' boxes, exactly.
__device__ __forceinline__ long long dkey(double x) {
    long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dkey_inv(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// block-wide min of lo[0..2] and max of hi[0..2]; thread 0 writes box[0..5]
__device__ void block_box_write(long long lo[3], long long hi[3], long long *box) {
    __shared__ long long red[2][3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; k++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < 3; k++) { red[0][k][warp] = lo[k]; red[1][k][warp] = hi[k]; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; k++) {
            long long mn = red[0][k][0], mx = red[1][k][0];
            for (int w = 1; w < nw; w++) { mn = min(mn, red[0][k][w]); mx = max(mx, red[1][k][w]); }
            box[k] = mn;
            box[3 + k] = mx;
        }
}

__device__ __forceinline__ void box_merge(long long lo[3], long long hi[3], const long long *b) {
#pragma unroll
    for (int k = 0; k < 3; k++) { lo[k] = min(lo[k], b[k]); hi[k] = max(hi[k], b[3 + k]); }
}

// float32 offset of coordinate k of point s from the box corner, from the
// packed {hi, lo} root-relative pair: (xh - lh) + (xl - ll)
__device__ __forceinline__ float dr_offset(const float4 *xq, int32_t s, int k, float lh, float ll) {
    const float4 qa = xq[2 * (int64_t)s];
    if (k == 0) return (qa.x - lh) + (qa.w - ll);
    const float4 qb = xq[2 * (int64_t)s + 1];
    return k == 1 ? (qa.y - lh) + (qb.x - ll) : (qa.z - lh) + (qb.y - ll);
}

// T_i = S_i: the leaf's points, or the children's X_c* in child order; tbox[a]
// its bounding box (the leaf's points, or the union of the children's boxes)
__global__ void k_gather_up(int lb, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                            const int32_t *end, int32_t *const *xptr, const int32_t *xcnt, const int64_t *toff,
                            int32_t *tdata, const double *x0, const double *x1, const double *x2, int d,
                            const long long *xbox, long long *tbox) {
    int a = blockIdx.x;
    int i = lb + a;
    int32_t *dst = tdata + toff[a];
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    if (nchild[i] == 0) {
        int32_t b0 = begin[i], n = end[i] - begin[i];
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            dst[r] = b0 + r;
            const long long k0 = dkey(x0[b0 + r]);
            lo[0] = min(lo[0], k0);
            hi[0] = max(hi[0], k0);
            if (d > 1) {
                const long long k1 = dkey(x1[b0 + r]);
                lo[1] = min(lo[1], k1);
                hi[1] = max(hi[1], k1);
            }
            if (d > 2) {
                const long long k2 = dkey(x2[b0 + r]);
                lo[2] = min(lo[2], k2);
                hi[2] = max(hi[2], k2);
            }
        }
    } else {
        int64_t w = 0;
        for (int c = fchild[i]; c < fchild[i] + nchild[i]; c++) {
            const int32_t *src = xptr[c];
            int n = xcnt[c];
            for (int r = threadIdx.x; r < n; r += blockDim.x) dst[w + r] = src[r];
            w += n;
            if (threadIdx.x == 0) box_merge(lo, hi, xbox + 6 * (int64_t)c);
        }
    }
    block_box_write(lo, hi, tbox + 6 * (int64_t)a);
}

// T_i = Y_p* followed by X_j* for j in IL(i); tbox[a] the union of their boxes.
// The interaction list is taken in tiles of GD_TILE entries: a block scan of
// the X_j* sizes gives each segment's place, then one warp copies each segment
// (no chain of dependent loads along the list).  blockDim.x must be
// GD_TILE / GD_ITEMS.
constexpr int GD_ITEMS = 4;
constexpr int GD_THREADS = 256;
constexpr int GD_TILE = GD_ITEMS * GD_THREADS;

__global__ void __launch_bounds__(GD_THREADS) k_gather_down(int lb, const int32_t *parent, const int64_t *far_ptr,
                                                            const int32_t *far_idx, int32_t *const *xptr,
                                                            const int32_t *xcnt, int32_t *const *yptr,
                                                            const int32_t *ycnt, const int64_t *toff,
                                                            int32_t *tdata, const long long *xbox,
                                                            const long long *ybox, long long *tbox) {
    __shared__ int32_t s_j[GD_TILE], s_off[GD_TILE + 1];
    __shared__ int32_t s_wsum[GD_THREADS / 32];
    const int a = blockIdx.x, i = lb + a;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int32_t *dst = tdata + toff[a];
    const int p = parent[i];
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    int64_t base;
    {
        const int32_t *src = yptr[p];
        const int n = ycnt[p];
        for (int r = threadIdx.x; r < n; r += blockDim.x) dst[r] = src[r];
        base = n;
        if (threadIdx.x == 0 && n > 0) box_merge(lo, hi, ybox + 6 * (int64_t)p);
    }
    const int64_t f0 = far_ptr[i], f1 = far_ptr[i + 1];
    for (int64_t e = f0 + threadIdx.x; e < f1; e += blockDim.x) box_merge(lo, hi, xbox + 6 * (int64_t)far_idx[e]);
    for (int64_t t0 = f0; t0 < f1; t0 += GD_TILE) {
        const int nt = (int)min((int64_t)GD_TILE, f1 - t0);
        // this thread's GD_ITEMS consecutive entries: sizes, then an exclusive block scan
        int len[GD_ITEMS], tot = 0;
#pragma unroll
        for (int q = 0; q < GD_ITEMS; q++) {
            const int e = threadIdx.x * GD_ITEMS + q;
            int j = 0, n = 0;
            if (e < nt) { j = far_idx[t0 + e]; n = xcnt[j]; s_j[e] = j; }
            len[q] = n;
            tot += n;
        }
        int inc = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) s_wsum[warp] = inc;
        __syncthreads();
        int wbase = 0;
        for (int w = 0; w < warp; w++) wbase += s_wsum[w];
        int run = wbase + inc - tot;
#pragma unroll
        for (int q = 0; q < GD_ITEMS; q++) {
            const int e = threadIdx.x * GD_ITEMS + q;
            if (e < nt) s_off[e] = run;
            run += len[q];
        }
        if (threadIdx.x == blockDim.x - 1) s_off[nt] = run;  // (entries past nt add 0)
        __syncthreads();
        for (int e = warp; e < nt; e += nwarps) {
            const int32_t *src = xptr[s_j[e]];
            const int n = s_off[e + 1] - s_off[e];
            int32_t *d = dst + base + s_off[e];
            for (int r = lane; r < n; r += 32) d[r] = src[r];
        }
        base += s_off[nt];
        __syncthreads();
    }
    block_box_write(lo, hi, tbox + 6 * (int64_t)a);
}

// The interaction-list part of T_i (what follows Y_p* there) copied to its own
// segment tl[loff[a] .. loff[a+1]), and its box, the union of the X_j* boxes
// over j in IL(i), to lbox[a]
__global__ void k_gather_il(int lb, const int32_t *parent, const int64_t *far_ptr, const int32_t *far_idx,
                            const int32_t *ycnt, const int64_t *toff, const int32_t *tdata, const int64_t *loff,
                            int32_t *tl, const long long *xbox, long long *lbox) {
    const int a = blockIdx.x, i = lb + a;
    const int64_t src = toff[a] + ycnt[parent[i]], dst = loff[a], n = loff[a + 1] - loff[a];
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) tl[dst + r] = tdata[src + r];
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (int64_t e = far_ptr[i] + threadIdx.x; e < far_ptr[i + 1]; e += blockDim.x)
        box_merge(lo, hi, xbox + 6 * (int64_t)far_idx[e]);
    block_box_write(lo, hi, lbox + 6 * (int64_t)a);
}

__global__ void k_set_ptrs(int lb, int nl, int32_t *base, const int64_t *off, int32_t **ptr) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < nl) ptr[lb + a] = base + off[a];
}

// ----------------------------------------------------------- DataReduct
__device__ void block_bitonic_sort(int32_t *v, int P) {
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool asc = (i & k) == 0;
                    int32_t x = v[i], y = v[ixj];
                    if ((x > y) == asc) { v[i] = y; v[ixj] = x; }
                }
            }
            __syncthreads();
        }
}

// writes the distinct values of sorted v[0..P) (INT_MAX = padding) to out,
// returns their number (valid in every thread)
__device__ int block_unique_write(const int32_t *v, int P, int32_t *out, int *scratch) {
    int chunk = (P + blockDim.x - 1) / blockDim.x;
    int s0 = threadIdx.x * chunk, s1 = min(P, s0 + chunk);
    int cnt = 0;
    for (int i = s0; i < s1; i++)
        if (v[i] != INT_MAX && (i == 0 || v[i] != v[i - 1])) cnt++;
    // exclusive scan of cnt over the block
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? scratch[lane] : 0, wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) scratch[lane] = wi - w;
        if (lane == nw - 1) scratch[32] = wi;
    }
    __syncthreads();
    int w = scratch[warp] + inc - cnt;
    for (int i = s0; i < s1; i++)
        if (v[i] != INT_MAX && (i == 0 || v[i] != v[i - 1])) out[w++] = v[i];
    int total = scratch[32];
    __syncthreads();
    return total;
}

// Y_i* u (the interaction-list part's reduced set lptr[a]): both sorted and
// free of repeats; their union, sorted, replaces Y_i* in place (its buffer
// holds both capacities), and Y_i*'s box takes the union of the two boxes.
// A node with an empty interaction list (common at levels 1-2) has an empty
// second part whose box is DataReduct's empty-set sentinel (LLONG_MAX lows,
// LLONG_MIN highs), so the min/max below leave Y_i*'s box unchanged.
// Dynamic shared memory: the next power of two >= |Y_i*| + |lptr[a]| int32.
__global__ void k_merge_il(int lb, int32_t *const *yptr, int32_t *ycnt, long long *ybox, int32_t *const *lptr,
                           const int32_t *lcnt, const long long *lobox) {
    extern __shared__ int32_t mv[];
    __shared__ int scratch[33];
    const int a = blockIdx.x, i = lb + a;
    const int na = ycnt[i], nb = lcnt[a];
    int32_t *y = yptr[i];
    const int32_t *b = lptr[a];
    int P = 1;
    while (P < na + nb) P <<= 1;
    for (int r = threadIdx.x; r < P; r += blockDim.x) mv[r] = r < na ? y[r] : (r < na + nb ? b[r - na] : INT_MAX);
    __syncthreads();
    block_bitonic_sort(mv, P);
    const int m = block_unique_write(mv, P, y, scratch);
    if (threadIdx.x == 0) ycnt[i] = m;
    if (threadIdx.x < 3) {
        const int k = threadIdx.x;
        ybox[6 * (int64_t)i + k] = min(ybox[6 * (int64_t)i + k], lobox[6 * (int64_t)a + k]);
        ybox[6 * (int64_t)i + 3 + k] = max(ybox[6 * (int64_t)i + 3 + k], lobox[6 * (int64_t)a + 3 + k]);
    }
}

// in-place inclusive scan of v[0..n) in shared memory by the whole block
__device__ void block_scan_inclusive(int *v, int n, int *scratch) {
    int chunk = (n + blockDim.x - 1) / blockDim.x;
    int s0 = threadIdx.x * chunk, s1 = min(n, s0 + chunk);
    int sum = 0;
    for (int i = s0; i < s1; i++) sum += v[i];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = sum;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? scratch[lane] : 0, wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) scratch[lane] = wi - w;
    }
    __syncthreads();
    int run = scratch[warp] + inc - sum;
    for (int i = s0; i < s1; i++) {
        run += v[i];
        v[i] = run;
    }
    __syncthreads();
}

// order-preserving map of a float64 to a signed 64-bit integer and back
__device__ __forceinline__ double dmin_(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ double dmax_(double a, double b) { return a > b ? a : b; }

__device__ __forceinline__ float warp_minf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Cell e of the (2r+1)^d block of cells around cell cid (flat dimensions
// collapsed): whether it lies inside the grid at Chebyshev distance exactly r,
// its bin, and a float32 lower bound lb of the squared distance from the grid
// point (offset qf from the box corner) to the cell widened by delf per side.
__device__ __forceinline__ bool dr_ring_cell(int e, int r, int d, int g, const int *cid, const bool *flat,
                                             const float *hf, const float *qf, float delf, int &bin, float &lb) {
    const int side = 2 * r + 1;
    int rem = e, stride = 1, cheb = 0;
    bool ok = true;
    bin = 0;
    lb = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k >= d) break;
        int o = 0;
        if (!flat[k]) {
            // rem / side: rings 0 and 1 (side 1, 3; rem < 27) by multiply-shift
            const int qd = side == 1 ? rem : (side == 3 && rem < 32 ? (rem * 11) >> 5 : rem / side);
            o = rem - qd * side - r;
            rem = qd;
        }
        const int ck = cid[k] + o;
        ok = ok && ck >= 0 && ck < g;
        cheb = max(cheb, abs(o));
        bin += ck * stride;
        stride *= g;
        if (!flat[k]) {
            const float lo = (float)ck * hf[k] - delf, hi = (float)(ck + 1) * hf[k] + delf;
            const float gap = fmaxf(0.f, fmaxf(lo - qf[k], qf[k] - hi));
            lb = fmaf(gap, gap, lb);
        }
    }
    return ok && cheb == r;
}

constexpr int DR_BIN_MAX = 4096;    // largest grid binned in shared memory
constexpr int DR_QTAB = 1024;       // largest grid tabulated in shared memory

// dynamic shared memory of k_datareduct: win (grid-point winners, padded to a
// power of two), then the bin starts (G + 1 ints) and the list of non-empty
// cells (G ints), then, 8-byte aligned, the grid-point table (3G doubles and 3G
// floats) when G <= DR_QTAB
__host__ __device__ __forceinline__ size_t dr_win_bytes(int G) {
    size_t p2 = 1;
    while (p2 < (size_t)G) p2 <<= 1;
    size_t a = p2 * 4, b = (size_t)((G + 31) & ~31) * 8;
    return a > b ? a : b;
}
__host__ __device__ __forceinline__ size_t dr_bins_offset(int G) { return dr_win_bytes(G); }
__host__ __device__ __forceinline__ size_t dr_qtab_offset(int G) {
    return (dr_bins_offset(G) + (size_t)(2 * G + 1) * 4 + 7) & ~(size_t)7;
}
__host__ __device__ __forceinline__ size_t dr_smem_bytes(int G) {
    if (G > DR_BIN_MAX) return dr_win_bytes(G);  // no binned search above DR_BIN_MAX
    return dr_qtab_offset(G) + (G <= DR_QTAB ? (size_t)G * 3 * (8 + 4) : 0);
}




// A non-empty cell in the search list: its bin in bits 0..11 and its index
// along coordinate k in bits 12 + 6k .. 17 + 6k (the binned search has
// g^d <= 4096, so g <= 64).
__device__ __forceinline__ int dr_pack_cell(int bin, int d, int g) {
    int v = bin, rem = bin;
    for (int k = 0; k < d; k++) {
        v |= (rem % g) << (12 + 6 * k);
        rem /= g;
    }
    return v;
}

// Lower bound of the squared distance from the grid point (offset qf) to the
// packed cell widened by delf per side, and the cell's Chebyshev distance from cid.
__device__ __forceinline__ float dr_cell_lb(int packed, int d, const int *cid, const bool *flat, const float *hf,
                                            const float *qf, float delf, int &cheb) {
    float lb = 0.f;
    cheb = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k >= d) break;
        const int ck = (packed >> (12 + 6 * k)) & 63;
        if (!flat[k]) {
            cheb = max(cheb, abs(ck - cid[k]));
            const float lo = (float)ck * hf[k] - delf, hi = (float)(ck + 1) * hf[k] + delf;
            const float gap = fmaxf(0.f, fmaxf(lo - qf[k], qf[k] - hi));
            lb = fmaf(gap, gap, lb);
        }
    }
    return lb;
}

// Float32 top-two over the points of the cells the lanes selected (lane c's
// cell `bin` when ok), walked as one flat range across the warp: lane c's cell
// is [cs, cs + cn) at offset exc of the warp's prefix sum of the counts.  l1 is
// the label of the lane's smallest.
__device__ __forceinline__ void dr_scan_top2(bool ok, int bin, const int *bstart, const float4 *pq, const float *qf,
                                             float &b1, float &b2, int32_t &l1, int lane) {
    if (__ballot_sync(0xffffffffu, ok) == 0u) return;
    int cs = 0, cn = 0;
    if (ok) {
        cs = bstart[bin];
        cn = bstart[bin + 1] - cs;
    }
    int inc = cn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    const int exc = inc - cn;
    // one selected cell (ring 0 always): its range directly, no lane search
    const unsigned sel = __ballot_sync(0xffffffffu, cn > 0);
    const bool one = (sel & (sel - 1)) == 0u;
    const int cs1 = one && sel ? __shfl_sync(0xffffffffu, cs, __ffs(sel) - 1) : 0;
    for (int f0 = 0; f0 < total; f0 += 32) {
        const int f = f0 + lane;
        int p;
        if (one) {
            p = cs1 + f;
        } else {
            int src = 0;  // last lane whose range starts at or before f
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int ex = __shfl_sync(0xffffffffu, exc, src + st);
                if (ex <= f) src += st;
            }
            p = __shfl_sync(0xffffffffu, cs, src) + f - __shfl_sync(0xffffffffu, exc, src);
        }
        if (f < total) {
            const float4 e = pq[p];
            const float e0f = e.x - qf[0], e1f = e.y - qf[1], e2f = e.z - qf[2];
            const float d32 = fmaf(e2f, e2f, fmaf(e1f, e1f, e0f * e0f));
            if (d32 < b2) {
                if (d32 < b1) {
                    b2 = b1;
                    b1 = d32;
                    l1 = __float_as_int(e.w);
                } else {
                    b2 = d32;
                }
            }
        }
    }
}

// Near ties: every point of the selected cells whose float32 distance is at
// most limx, compared in float64 (non-negative doubles order as their bit
// patterns), the smaller label taking ties; (bk, bl) is the warp's best.
__device__ __forceinline__ void dr_scan_exact(bool ok, int bin, const int *bstart, const float4 *pq, const float *qf,
                                              float limx, int d, const double *x0, const double *x1, const double *x2,
                                              const double *q, long long &bk, int32_t &bl, int lane) {
    unsigned cm = __ballot_sync(0xffffffffu, ok);
    while (cm) {
        const int b = __shfl_sync(0xffffffffu, bin, __ffs(cm) - 1);
        cm &= cm - 1;
        const int pe = bstart[b + 1];
        for (int p0 = bstart[b]; p0 < pe; p0 += 32) {
            const int p = p0 + lane;
            bool c = false;
            int32_t id = INT_MAX;
            if (p < pe) {
                const float4 e = pq[p];
                const float e0f = e.x - qf[0], e1f = e.y - qf[1], e2f = e.z - qf[2];
                c = fmaf(e2f, e2f, fmaf(e1f, e1f, e0f * e0f)) <= limx;
                id = __float_as_int(e.w);
            }
            unsigned pm = __ballot_sync(0xffffffffu, c);
            if (pm == 0u) continue;
            long long kk = LLONG_MAX;
            if (!c) id = INT_MAX;
            if (c)
                kk = __double_as_longlong(h2_dist2(d, x0[id], d > 1 ? x1[id] : 0.0, d > 2 ? x2[id] : 0.0, q[0], q[1],
                                                   q[2]));
            while (pm) {
                const int s2 = __ffs(pm) - 1;
                pm &= pm - 1;
                const long long kv = __shfl_sync(0xffffffffu, kk, s2);
                const int32_t iv = __shfl_sync(0xffffffffu, id, s2);
                if (kv < bk || (kv == bk && iv < bl)) {
                    bk = kv;
                    bl = iv;
                }
            }
        }
    }
}

// One CTA per node.  tdata[toff[a] .. toff[a+1]) are the labels of S (T),
// tbox[a] its bounding box; coordinates of label s are (x0[s], x1[s], x2[s]).
// The box of the result goes to outbox[node].
__global__ void __launch_bounds__(DR_THREADS, 5) k_datareduct(const int64_t *toff, const int32_t *tdata, int g, int d,
                                                           DRPoints PT, int32_t *const *outptr, int32_t *outcnt, int lb,
                                                           int2 *bin_base, float4 *pq_base, const long long *tbox,
                                                           long long *outbox) {
    const double *x0 = PT.x[0], *x1 = PT.x[1], *x2 = PT.x[2];
    extern __shared__ unsigned char smem_raw[];
    int32_t *win = reinterpret_cast<int32_t *>(smem_raw);  // [P]
    __shared__ int32_t tid_s[DR_TILE];
    __shared__ float tf_s[3][DR_TILE];
    __shared__ int scratch[33];
    const int a = blockIdx.x;
    const int node = lb + a;
    const int64_t t0 = toff[a], nt = toff[a + 1] - toff[a];
    const int32_t *T = tdata + t0;
    int32_t *out = outptr[node];
    int G = 1;
    for (int k = 0; k < d; k++) G *= g;
    if (nt <= G) {  // DataReduct returns S itself
        int P = 1;
        while (P < nt) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) win[i] = i < nt ? T[i] : INT_MAX;
        __syncthreads();
        block_bitonic_sort(win, P);
        for (int i = threadIdx.x; i < nt; i += blockDim.x) out[i] = win[i];
        if (threadIdx.x < 6) outbox[6 * (int64_t)node + threadIdx.x] = tbox[6 * (int64_t)a + threadIdx.x];
        if (threadIdx.x == 0) outcnt[node] = (int32_t)nt;
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double l[3] = {0.0, 0.0, 0.0}, h[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k >= d) break;
        l[k] = dkey_inv(tbox[6 * (int64_t)a + k]);
        h[k] = __ddiv_rn(__dsub_rn(dkey_inv(tbox[6 * (int64_t)a + 3 + k]), l[k]), (double)g);
    }
    // Both searches below stage float32 offsets from the box corner l,
    //   x - l = (xh - lh) + (xl - ll),
    // from the {hi, lo} split of the root-relative coordinates (xh + xl and
    // lh + ll within 2^-47 R of x - ref and l - ref, R the root extent).  Per
    // coordinate the offset is within 2 u W + 8 u^2 R of exact (u = 2^-24, W the
    // largest box extent), the grid point's within u W, so a float32 squared
    // distance is within E = 30 u W^2 + 48 u^2 W R of the float64 one.  With
    // M = 8e-6 W^2 + 1e-12 W R > 2E + 3u (3 W^2): when a point's float32
    // distance exceeds the smallest one by more than M, its float64 distance
    // exceeds the float64 distance of the float32 winner, which is then the
    // float64 winner; otherwise the float64 distances of every point within M
    // of the smallest decide, the smaller label taking ties.
    double W = 0.0, hmin = INFINITY;
    float ihf[3] = {0.f, 0.f, 0.f}, hf[3] = {0.f, 0.f, 0.f}, lh[3] = {0.f, 0.f, 0.f}, ll[3] = {0.f, 0.f, 0.f};
    bool flat[3] = {true, true, true};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k >= d) break;
        W = dmax_(W, __dmul_rn(h[k], (double)g));
        flat[k] = !(h[k] > 0.0);
        if (!flat[k]) {
            hmin = dmin_(hmin, h[k]);
            ihf[k] = (float)(1.0 / h[k]);
            hf[k] = (float)h[k];
        }
        const double Lk = l[k] - PT.ref[k];
        lh[k] = (float)Lk;
        ll[k] = (float)(Lk - (double)lh[k]);
    }
    const float M = (float)(8e-6 * W * W + 1e-12 * W * PT.R);
    if (G <= DR_BIN_MAX && bin_base != nullptr) {
        // Binned search.  The points of S are binned into the g^d cells of the
        // reference grid itself (grid point q is the centre of its cell) by a
        // counting sort in shared memory, their float32 offsets stored in bin
        // order.  For each grid point a warp scans its own cell, then the
        // Chebyshev rings of cells around it, each lane keeping the two
        // smallest float32 distances it has seen.  A cell whose widened box
        // bound exceeds the warp's smallest distance plus M is skipped, and the
        // search stops after ring r once that sum is below the square of
        // (r + 1/2) h_min - delta, a lower bound for every point in a farther
        // cell (delta = 1e-5 W + 1e-12 R covers the float32 binning error).
        int2 *bidx = bin_base + t0;     // bin of each entry and its rank in the bin
        float4 *pq = pq_base + t0;      // in bin order: float32 offsets and the label (as bits)
        int *bstart = reinterpret_cast<int *>(smem_raw + dr_bins_offset(G));
        const float delf = (float)(1e-5 * W + 1e-12 * PT.R);
        const float hminf = (float)hmin;
        for (int b = threadIdx.x; b <= G; b += blockDim.x) bstart[b] = 0;
        __syncthreads();
        // counting sort into cells.  Consecutive labels are Morton-coherent and
        // mostly share a cell, so the atomics are warp-aggregated: lanes with the
        // same cell elect one leader that adds the group's count, and each lane
        // takes the old count + its rank in the group as its rank in the bin.
        const unsigned lt = (1u << lane) - 1u;
        for (int64_t p0 = (int64_t)warp * 32; p0 < nt; p0 += blockDim.x) {
            const int64_t p = p0 + lane;
            int bi = -1;
            if (p < nt) {
                const int32_t sid = T[p];
                int stride = 1;
                bi = 0;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if (k >= d) break;
                    int cidx = 0;
                    if (!flat[k]) {
                        const float f = dr_offset(PT.xq, sid, k, lh[k], ll[k]);
                        cidx = min(max((int)(f * ihf[k]), 0), g - 1);
                    }
                    bi += cidx * stride;
                    stride *= g;
                }
            }
            const unsigned peers = __match_any_sync(0xffffffffu, bi);
            const int leader = __ffs(peers) - 1;
            int base = 0;
            if (bi >= 0 && lane == leader) base = atomicAdd(&bstart[bi + 1], __popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (bi >= 0) bidx[p] = make_int2(bi, base + __popc(peers & lt));
        }
        __syncthreads();
        block_scan_inclusive(bstart, G + 1, scratch);  // bstart[b]: first position of bin b
        __syncthreads();
        for (int64_t p = threadIdx.x; p < nt; p += blockDim.x) {
            const int2 bo = bidx[p];
            const int pos = bstart[bo.x] + bo.y;
            const int32_t sid = T[p];
            const float4 qa = PT.xq[2 * (int64_t)sid], qb = PT.xq[2 * (int64_t)sid + 1];
            const float f0 = (qa.x - lh[0]) + (qa.w - ll[0]);
            const float f1 = d > 1 ? (qa.y - lh[1]) + (qb.x - ll[1]) : 0.f;
            const float f2 = d > 2 ? (qa.z - lh[2]) + (qb.y - ll[2]) : 0.f;
            pq[pos] = make_float4(f0, f1, f2, __int_as_float(sid));
        }
        // grid points: float64 q and its float32 offset qf, computed once each
        double *qtab = reinterpret_cast<double *>(smem_raw + dr_qtab_offset(G));
        float *qftab = reinterpret_cast<float *>(qtab + 3 * G);
        const bool table = G <= DR_QTAB;
        if (table)
            for (int gi = threadIdx.x; gi < G; gi += blockDim.x) {
                int rem = gi;
                #pragma unroll
                for (int k = 0; k < 3; k++) {
                    if (k >= d) break;
                    const int idx = rem % g;
                    rem /= g;
                    const double qk = __dadd_rn(l[k], __dmul_rn(__dadd_rn((double)idx, 0.5), h[k]));
                    qtab[3 * gi + k] = qk;
                    qftab[3 * gi + k] = (float)__dsub_rn(qk, l[k]);
                }
            }
        // the non-empty cells, for searches that go past ring 1 (the cursor
        // area of the bins is free after the scatter; order does not matter)
        int *nel = bstart + G + 1;
        __shared__ int s_nne;
        if (threadIdx.x == 0) s_nne = 0;
        __syncthreads();
        for (int b = threadIdx.x; b < G; b += blockDim.x)
            if (bstart[b + 1] > bstart[b]) nel[atomicAdd(&s_nne, 1)] = dr_pack_cell(b, d, g);
        __syncthreads();
        const int nne = s_nne;
        for (int gi = warp; gi < G; gi += nw) {
            double q[3] = {0.0, 0.0, 0.0};
            float qf[3] = {0.f, 0.f, 0.f};
            int cid[3] = {0, 0, 0};
            int rmax = 0;
            {
                int rem = gi;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if (k >= d) break;
                    const int idx = rem % g;
                    rem /= g;
                    if (table) {
                        q[k] = qtab[3 * gi + k];
                        qf[k] = qftab[3 * gi + k];
                    } else {
                        q[k] = __dadd_rn(l[k], __dmul_rn(__dadd_rn((double)idx, 0.5), h[k]));
                        qf[k] = (float)__dsub_rn(q[k], l[k]);
                    }
                    cid[k] = flat[k] ? 0 : idx;
                    if (!flat[k]) rmax = max(rmax, max(cid[k], g - 1 - cid[k]));
                }
            }
            float b1 = INFINITY, b2 = INFINITY;  // this lane's two smallest float32 distances
            int32_t l1 = INT_MAX;                // the label of its smallest
            float lim = INFINITY;                // the warp's smallest distance + M
            // rings 0 and 1 with the stop test; a search still open after ring 1
            // (sparse or empty surroundings) scans the non-empty cells instead
            const int rA = min(rmax, 1);
            int stage = 2;  // 0 or 1: stopped after that ring; 2: the non-empty cells were scanned
            for (int r = 0; r <= rA; r++) {
                const int side = 2 * r + 1;
                int total = 1;
#pragma unroll
                for (int k = 0; k < 3; k++)
                    if (k < d) total *= flat[k] ? 1 : side;
                for (int e0 = 0; e0 < total; e0 += 32) {
                    int bin = 0;
                    float lb = 0.f;
                    bool ok = e0 + lane < total && dr_ring_cell(e0 + lane, r, d, g, cid, flat, hf, qf, delf, bin, lb);
                    ok = ok && lb <= lim;
                    dr_scan_top2(ok, bin, bstart, pq, qf, b1, b2, l1, lane);
                    lim = warp_minf(b1) + M;
                }
                // (r + 1/2) h_min - delta and its square rounded down in float32
                const float rr = ((float)r + 0.5f) * hminf * 0.9999996f - delf;
                if (rr > 0.f && lim < rr * rr * 0.9999996f) {
                    stage = r;
                    break;
                }
            }
            if (stage == 2 && rmax <= 1) stage = rA;  // rings 0..rmax held every cell
            if (stage == 2) {
                // the non-empty cell with the smallest bound first (it sets lim when
                // rings 0 and 1 were empty), then the others whose bound passes
                float blb = INFINITY;
                int bbin = -1;
                for (int e0 = lane; e0 < nne; e0 += 32) {
                    const int pk = nel[e0];
                    int cheb;
                    const float lb = dr_cell_lb(pk, d, cid, flat, hf, qf, delf, cheb);
                    if (cheb >= 2 && lb < blb) {
                        blb = lb;
                        bbin = pk & 4095;
                    }
                }
                const float mlb = warp_minf(blb);
                const int b0 = __shfl_sync(0xffffffffu, bbin, __ffs(__ballot_sync(0xffffffffu, blb == mlb)) - 1);
                if (b0 >= 0 && mlb <= lim) {
                    dr_scan_top2(lane == 0, b0, bstart, pq, qf, b1, b2, l1, lane);
                    lim = warp_minf(b1) + M;
                }
                for (int e0 = 0; e0 < nne; e0 += 32) {
                    bool ok = false;
                    int bin = 0;
                    if (e0 + lane < nne) {
                        const int pk = nel[e0 + lane];
                        bin = pk & 4095;
                        int cheb;
                        const float lb = dr_cell_lb(pk, d, cid, flat, hf, qf, delf, cheb);
                        ok = cheb >= 2 && lb <= lim && bin != b0;
                    }
                    dr_scan_top2(ok, bin, bstart, pq, qf, b1, b2, l1, lane);
                    lim = warp_minf(b1) + M;
                }
            }
            const float m1 = warp_minf(b1);
            const int w = __ffs(__ballot_sync(0xffffffffu, b1 == m1)) - 1;
            const float sec = warp_minf(lane == w ? b2 : b1);
            const float limx = m1 + M;
            int32_t winner;
            if (sec > limx) {
                winner = __shfl_sync(0xffffffffu, l1, w);
            } else {
                // near tie: every point within M of the smallest in float64, over
                // the cells the search visited
                long long bk = LLONG_MAX;
                int32_t bl = INT_MAX;
                const int rB = stage == 2 ? rA : stage;
                for (int r = 0; r <= rB; r++) {
                    const int side = 2 * r + 1;
                    int total = 1;
#pragma unroll
                    for (int k = 0; k < 3; k++)
                        if (k < d) total *= flat[k] ? 1 : side;
                    for (int e0 = 0; e0 < total; e0 += 32) {
                        int bin = 0;
                        float lb = 0.f;
                        bool ok =
                            e0 + lane < total && dr_ring_cell(e0 + lane, r, d, g, cid, flat, hf, qf, delf, bin, lb);
                        ok = ok && lb <= limx && bstart[bin + 1] > bstart[bin];
                        dr_scan_exact(ok, bin, bstart, pq, qf, limx, d, x0, x1, x2, q, bk, bl, lane);
                    }
                }
                if (stage == 2)
                    for (int e0 = 0; e0 < nne; e0 += 32) {
                        bool ok = false;
                        int bin = 0;
                        if (e0 + lane < nne) {
                            const int pk = nel[e0 + lane];
                            bin = pk & 4095;
                            int cheb;
                            const float lb = dr_cell_lb(pk, d, cid, flat, hf, qf, delf, cheb);
                            ok = cheb >= 2 && lb <= limx;
                        }
                        dr_scan_exact(ok, bin, bstart, pq, qf, limx, d, x0, x1, x2, q, bk, bl, lane);
                    }
                winner = bl;
            }
            if (lane == 0) win[gi] = winner;
        }
    } else {
        // Brute force (grids above DR_BIN_MAX): DR_GPT grid points per thread
        // per sweep over S staged in shared memory, each keeping its two
        // smallest float32 distances; a grid point without a gap of more than M
        // between them takes a second sweep that compares every point within M
        // of the smallest in float64.
        for (int gbase = 0; gbase < G; gbase += DR_THREADS * DR_GPT) {
            float qf[DR_GPT][3], b1[DR_GPT], b2[DR_GPT];
            int32_t i1[DR_GPT];
#pragma unroll
            for (int j = 0; j < DR_GPT; j++) {
                int rem = gbase + j * DR_THREADS + threadIdx.x;
                for (int k = 0; k < 3; k++) {
                    int idx = 0;
                    if (k < d) {
                        idx = rem % g;
                        rem /= g;
                    }
                    qf[j][k] = k < d ? (float)__dsub_rn(
                                           __dadd_rn(l[k], __dmul_rn(__dadd_rn((double)idx, 0.5), h[k])), l[k])
                                     : 0.0f;
                }
                b1[j] = INFINITY;
                b2[j] = INFINITY;
                i1[j] = INT_MAX;
            }
            for (int64_t tb = 0; tb < nt; tb += DR_TILE) {
                const int cnt = (int)(nt - tb < DR_TILE ? nt - tb : DR_TILE);
                __syncthreads();
                for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
                    const int32_t s = T[tb + r];
                    tid_s[r] = s;
#pragma unroll
                    for (int k = 0; k < 3; k++) tf_s[k][r] = k < d ? dr_offset(PT.xq, s, k, lh[k], ll[k]) : 0.f;
                }
                __syncthreads();
                for (int r = 0; r < cnt; r++) {
                    const float f0 = tf_s[0][r], f1 = tf_s[1][r], f2 = tf_s[2][r];
#pragma unroll
                    for (int j = 0; j < DR_GPT; j++) {
                        const float e0 = f0 - qf[j][0], e1 = f1 - qf[j][1], e2 = f2 - qf[j][2];
                        const float d32 = fmaf(e2, e2, fmaf(e1, e1, e0 * e0));
                        if (d32 < b2[j]) {
                            if (d32 < b1[j]) {
                                b2[j] = b1[j];
                                b1[j] = d32;
                                i1[j] = tid_s[r];
                            } else {
                                b2[j] = d32;
                            }
                        }
                    }
                }
            }
            // near ties, one grid-point slot at a time
#pragma unroll
            for (int j = 0; j < DR_GPT; j++) {
                const int gi = gbase + j * DR_THREADS + threadIdx.x;
                const float limx = b1[j] + M;
                const bool need = gi < G && !(b2[j] > limx);
                if (!__syncthreads_or(need)) continue;
                double q[3] = {0.0, 0.0, 0.0};
                {
                    int rem = gi;
                    #pragma unroll
                    for (int k = 0; k < 3; k++) {
                        if (k >= d) break;
                        const int idx = rem % g;
                        rem /= g;
                        q[k] = __dadd_rn(l[k], __dmul_rn(__dadd_rn((double)idx, 0.5), h[k]));
                    }
                }
                long long bk = LLONG_MAX;
                int32_t bl = INT_MAX;
                for (int64_t tb = 0; tb < nt; tb += DR_TILE) {
                    const int cnt = (int)(nt - tb < DR_TILE ? nt - tb : DR_TILE);
                    __syncthreads();
                    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
                        const int32_t s = T[tb + r];
                        tid_s[r] = s;
#pragma unroll
                        for (int k = 0; k < 3; k++) tf_s[k][r] = k < d ? dr_offset(PT.xq, s, k, lh[k], ll[k]) : 0.f;
                    }
                    __syncthreads();
                    if (need)
                        for (int r = 0; r < cnt; r++) {
                            const float e0 = tf_s[0][r] - qf[j][0], e1 = tf_s[1][r] - qf[j][1],
                                        e2 = tf_s[2][r] - qf[j][2];
                            if (fmaf(e2, e2, fmaf(e1, e1, e0 * e0)) <= limx) {
                                const int32_t s = tid_s[r];
                                const long long kk = __double_as_longlong(
                                    h2_dist2(d, x0[s], d > 1 ? x1[s] : 0.0, d > 2 ? x2[s] : 0.0, q[0], q[1], q[2]));
                                if (kk < bk || (kk == bk && s < bl)) {
                                    bk = kk;
                                    bl = s;
                                }
                            }
                        }
                }
                if (need) i1[j] = bl;
            }
#pragma unroll
            for (int j = 0; j < DR_GPT; j++) {
                const int gi = gbase + j * DR_THREADS + threadIdx.x;
                if (gi < G) win[gi] = i1[j];
            }
        }
    }
    __syncthreads();
    {  // bounding box of the winners
        long long blo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, bhi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        for (int gi = threadIdx.x; gi < G; gi += blockDim.x) {
            const int32_t sid = win[gi];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k >= d) break;
                const long long kv = dkey((k == 0 ? x0 : (k == 1 ? x1 : x2))[sid]);
                blo[k] = min(blo[k], kv);
                bhi[k] = max(bhi[k], kv);
            }
        }
        block_box_write(blo, bhi, outbox + 6 * (int64_t)node);
    }
    int P = 1;
    while (P < G) P <<= 1;
    for (int i = G + threadIdx.x; i < P; i += blockDim.x) win[i] = INT_MAX;
    __syncthreads();
    block_bitonic_sort(win, P);
    int m = block_unique_write(win, P, out, scratch);
    if (threadIdx.x == 0) outcnt[node] = m;
}

// ------------------------------------- DataReduct over a union of reduced sets
// A top-down set is a union, S = Y_p* (when given) u X_j* over j in IL(i).
// The X_j* are many (hundreds per node at tau = 1/2) and each one recurs in
// the sets of many nodes of its level, so copying S out and binning every
// entry dominated HiDR.  This form reads the X_j* in place.  Each X_j*
// (sorted labels, so Morton-coherent) is cut into chunks of DM_CHUNK
// consecutive labels; the box of every chunk and of every member is computed
// once per build, in the hi parts of the float32 root-relative split
// (xh = fl32(fl64(x - corner)), monotone in x, so these boxes bound the hi
// parts exactly).  Per node the members are entered in every cell of the
// reference grid their box overlaps (mode A) or, when the member-cell pairs
// exceed the list's capacity, in the cell of their box centre only, with every
// cell bound and the stopping radius widened by the largest half extent E
// (mode B).  A grid point's search walks the cells as the binned search of
// k_datareduct does; in each cell it scans Y_p*'s points (binned point by
// point, as there) and, for every member this warp has not yet visited whose
// box bound passes, the chunks whose box bound passes, lane k taking entry k
// of a chunk.  The float32 top-two, the stopping rule and the float64
// decision of near ties are the binned search's, so the result is the same
// set: for every grid point the float64-nearest point of S, ties to the
// smaller label.
//
// Offsets in a node's frame: a point's offset f = (xh - lh) + (xl - ll) has
// |fl32(xl - ll)| <= 2u R (1 + u) (u = 2^-24, R the root extent), so xh in
// [a, b] puts f in [fl32(a - lh) - cR, fl32(b - lh) + cR] for cR = 2.5 u R;
// the boxes are moved to the frame with cw = 2e-7 R + delf per side, delf
// being the binned search's widening (it absorbs the rounding of the bound
// itself).
constexpr int DM_CHUNK = 32;
constexpr int DM_MAX_MEMBERS = 16384;  // longest interaction list the member search takes

__global__ void k_chunk_counts(int nn, const int32_t *xcnt, int64_t *nch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nn) nch[i] = (xcnt[i] + DM_CHUNK - 1) / DM_CHUNK;
}

// chunk boxes cbox[2 (choff[i] + c)], [.. + 1] (low, high corner of the hi
// parts) and member boxes mbox[2 i], [2 i + 1] of X_i* for nodes [n0, nn),
// and the packed coordinates of X_i*'s entry r copied to xqm[2 (32 choff[i] +
// r)], [.. + 1] (xq's two float4, the label in the second's .z as int bits),
// so that a chunk is read with one coalesced load; one warp a node
__global__ void k_member_boxes(int n0, int nn, int32_t *const *xptr, const int32_t *xcnt, const int64_t *choff,
                               const float4 *xq, float4 *cbox, float4 *mbox, float4 *xqm) {
    const int i = n0 + (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nn) return;
    const int cnt = xcnt[i];
    const int32_t *lab = xptr[i];
    float mlo[3] = {INFINITY, INFINITY, INFINITY}, mhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int c = 0; c * DM_CHUNK < cnt; c++) {
        const int r = c * DM_CHUNK + lane;
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        if (r < cnt) {
            const int32_t sid = lab[r];
            const float4 qa = xq[2 * (int64_t)sid], qb = xq[2 * (int64_t)sid + 1];
            const int64_t o = 2 * (DM_CHUNK * choff[i] + r);
            xqm[o] = qa;
            xqm[o + 1] = make_float4(qb.x, qb.y, __int_as_float(sid), 0.f);
            lo[0] = hi[0] = qa.x;
            lo[1] = hi[1] = qa.y;
            lo[2] = hi[2] = qa.z;
        }
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        if (lane == 0) {
            const int64_t cc = choff[i] + c;
            cbox[2 * cc] = make_float4(lo[0], lo[1], lo[2], 0.f);
            cbox[2 * cc + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            mlo[k] = fminf(mlo[k], lo[k]);
            mhi[k] = fmaxf(mhi[k], hi[k]);
        }
    }
    if (lane == 0) {
        mbox[2 * (int64_t)i] = make_float4(mlo[0], mlo[1], mlo[2], 0.f);
        mbox[2 * (int64_t)i + 1] = make_float4(mhi[0], mhi[1], mhi[2], 0.f);
    }
}

// Lower bound of the float32 squared distance from the grid point (offset qf)
// to any point whose hi parts lie in the box (lo, hi), in this node's frame
// (corner hi parts lh) with cw added per side; flat coordinates add nothing.
__device__ __forceinline__ float dm_box_lb(float4 lo, float4 hi, const float *lh, const float *qf,
                                           const bool *flat, float cw, int d) {
    const float l3[3] = {lo.x, lo.y, lo.z}, h3[3] = {hi.x, hi.y, hi.z};
    float lb = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k >= d) break;
        if (flat[k]) continue;
        const float a = (l3[k] - lh[k]) - cw, b = (h3[k] - lh[k]) + cw;
        const float gap = fmaxf(0.f, fmaxf(a - qf[k], qf[k] - b));
        lb = fmaf(gap, gap, lb);
    }
    return lb;
}

struct DMArgs {
    int lb;        // first node of the level; node lb + a is CTA a's
    int outlb;     // the result of CTA a goes to outptr / outcnt / outbox [outlb + a]
    int g, d;
    int mcap;      // capacity of the member-cell list (entries)
    int vwords;    // 32-bit words of a warp's visited-member bitmask
    const int64_t *toff;   // |S| of CTA a's set = toff[a + 1] - toff[a]
    const int32_t *parent;  // null: the set has no Y_p* part
    int32_t *const *yptr;
    const int32_t *ycnt;
    const long long *ybox;
    const int64_t *poff;    // staging of CTA a's Y_p* part: pbin / pq [poff[a] ..)
    int2 *pbin;
    float4 *pq;
    const int64_t *far_ptr;
    const int32_t *far_idx;
    int32_t *const *xptr;
    const int32_t *xcnt;
    const long long *xbox;
    const int64_t *choff;
    const float4 *cbox, *mbox, *xqm;
    int32_t *const *outptr;
    int32_t *outcnt;
    long long *outbox;
};

// the grid point's frame, shared by the scans of one warp
struct DMFrame {
    const float4 *xq, *xqm;
    const double *x0, *x1, *x2;
    float lh[3], ll[3], qf[3];
    double q[3];
    bool flat[3];
    float cw, M;
    int d;
};

__device__ __forceinline__ float dm_entry_d32(const DMFrame &F, float4 qa, float4 qb) {
    const float e0 = ((qa.x - F.lh[0]) + (qa.w - F.ll[0])) - F.qf[0];
    const float e1 = F.d > 1 ? ((qa.y - F.lh[1]) + (qb.x - F.ll[1])) - F.qf[1] : 0.f;
    const float e2 = F.d > 2 ? ((qa.z - F.lh[2]) + (qb.y - F.ll[2])) - F.qf[2] : 0.f;
    return fmaf(e2, e2, fmaf(e1, e1, e0 * e0));
}

// The first lane still a candidate, or -1; its candidacy is cleared.
__device__ __forceinline__ int dm_next_any(bool &cand, int lane) {
    const unsigned cm = __ballot_sync(0xffffffffu, cand);
    if (cm == 0u) return -1;
    const int s = __ffs(cm) - 1;
    if (lane == s) cand = false;
    return s;
}

// The lane holding the smallest bound among the candidates (cand), or -1
// when there is none or that bound exceeds lim; its candidacy is cleared.
__device__ __forceinline__ int dm_next_nearest(bool &cand, float bound, float lim, int lane) {
    if (__ballot_sync(0xffffffffu, cand) == 0u) return -1;
    const float mb = warp_minf(cand ? bound : INFINITY);
    if (mb > lim) return -1;
    const int s = __ffs(__ballot_sync(0xffffffffu, cand && bound == mb)) - 1;
    if (lane == s) cand = false;
    return s;
}

// The chunks of member j whose box bound is at most lim, nearest bound first:
// float32 top-two of the lane (entry k of a chunk on lane k, l1 the label of
// its smallest), lim = the warp's smallest + M after each chunk.
__device__ __forceinline__ void dm_scan_member(const DMArgs &A, const DMFrame &F, int j, float &b1, float &b2,
                                               int32_t &l1, float &lim, int lane) {
    const int cnt = A.xcnt[j];
    const int64_t ch = A.choff[j];
    const float4 *cb = A.cbox + 2 * ch, *xm = F.xqm + 2 * DM_CHUNK * ch;
    const int nc = (cnt + DM_CHUNK - 1) / DM_CHUNK;
    for (int c0 = 0; c0 < nc; c0 += 32) {
        float lbc = INFINITY;
        bool cand = false;
        if (c0 + lane < nc) {
            lbc = dm_box_lb(cb[2 * (c0 + lane)], cb[2 * (c0 + lane) + 1], F.lh, F.qf, F.flat, F.cw, F.d);
            cand = lbc <= lim;
        }
        for (int s; (s = dm_next_nearest(cand, lbc, lim, lane)) >= 0;) {
            const int r = (c0 + s) * DM_CHUNK + lane;
            if (r < cnt) {
                const float4 qa = xm[2 * r], qb = xm[2 * r + 1];
                const int32_t sid = __float_as_int(qb.z);
                const float d32 = dm_entry_d32(F, qa, qb);
                if (d32 < b2) {
                    if (d32 < b1) {
                        b2 = b1;
                        b1 = d32;
                        l1 = sid;
                    } else {
                        b2 = d32;
                    }
                }
            }
            lim = warp_minf(b1) + F.M;
        }
    }
}

// Near ties over member j: every point of its chunks whose float32 distance is
// at most limx, compared in float64 (the lane's best key bk and label bl; the
// caller reduces over the warp).
__device__ __forceinline__ void dm_exact_member(const DMArgs &A, const DMFrame &F, int j, float limx,
                                                long long &bk, int32_t &bl, int lane) {
    const int cnt = A.xcnt[j];
    const int64_t ch = A.choff[j];
    const float4 *cb = A.cbox + 2 * ch, *xm = F.xqm + 2 * DM_CHUNK * ch;
    const int nc = (cnt + DM_CHUNK - 1) / DM_CHUNK;
    for (int c0 = 0; c0 < nc; c0 += 32) {
        bool pass = false;
        if (c0 + lane < nc)
            pass = dm_box_lb(cb[2 * (c0 + lane)], cb[2 * (c0 + lane) + 1], F.lh, F.qf, F.flat, F.cw, F.d) <= limx;
        unsigned pc = __ballot_sync(0xffffffffu, pass);
        while (pc) {
            const int s = __ffs(pc) - 1;
            pc &= pc - 1;
            const int r = (c0 + s) * DM_CHUNK + lane;
            if (r < cnt) {
                const float4 qa = xm[2 * r], qb = xm[2 * r + 1];
                const int32_t sid = __float_as_int(qb.z);
                if (dm_entry_d32(F, qa, qb) <= limx) {
                    const long long kk = __double_as_longlong(h2_dist2(F.d, F.x0[sid], F.d > 1 ? F.x1[sid] : 0.0,
                                                                       F.d > 2 ? F.x2[sid] : 0.0, F.q[0], F.q[1],
                                                                       F.q[2]));
                    if (kk < bk || (kk == bk && sid < bl)) {
                        bk = kk;
                        bl = sid;
                    }
                }
            }
        }
    }
}

// The members listed in the cells the lanes selected (lane c's cell `bin`
// when ok), walked as one flat range across the warp as dr_scan_top2 walks
// points.  A member not yet in the warp's visited bitmask whose box bound is
// at most lim (limx, exact) is marked and scanned, nearest bound first.
template <bool EXACT>
__device__ __forceinline__ void dm_visit(bool ok, int bin, const int *mstart, const uint16_t *mlist, uint32_t *vis,
                                         int64_t f0, const DMArgs &A, const DMFrame &F, float &b1, float &b2,
                                         int32_t &l1, float &lim, long long &bk, int32_t &bl, int lane) {
    if (__ballot_sync(0xffffffffu, ok) == 0u) return;
    int cs = 0, cn = 0;
    if (ok) {
        cs = mstart[bin];
        cn = mstart[bin + 1] - cs;
    }
    int inc = cn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    const int exc = inc - cn;
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int f = t0 + lane;
        int src = 0;  // last lane whose range starts at or before f
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int ex = __shfl_sync(0xffffffffu, exc, src + st);
            if (ex <= f) src += st;
        }
        const int pos = __shfl_sync(0xffffffffu, cs, src) + f - __shfl_sync(0xffffffffu, exc, src);
        int e = -1;
        float lbm = INFINITY;
        bool cand = false;  // (explicit: lim starts infinite, and INF <= INF)
        if (f < total) {
            e = mlist[pos];
            if (!((vis[e >> 5] >> (e & 31)) & 1u)) {
                const int j = A.far_idx[f0 + e];
                lbm = dm_box_lb(A.mbox[2 * (int64_t)j], A.mbox[2 * (int64_t)j + 1], F.lh, F.qf, F.flat, F.cw, F.d);
                cand = lbm <= lim;
            }
        }
        // nearest bound first (the exact pass takes them in any order)
        for (int s; (s = EXACT ? dm_next_any(cand, lane) : dm_next_nearest(cand, lbm, lim, lane)) >= 0;) {
            const int es = __shfl_sync(0xffffffffu, e, s);
            const uint32_t bit = 1u << (es & 31);
            uint32_t was = 0u;  // mark it; lane 0's test decides for the warp
            if (lane == 0) was = atomicOr(&vis[es >> 5], bit);
            if (__shfl_sync(0xffffffffu, was, 0) & bit) continue;  // listed twice among these cells
            const int j = A.far_idx[f0 + es];
            if (EXACT) dm_exact_member(A, F, j, lim, bk, bl, lane);
            else dm_scan_member(A, F, j, b1, b2, l1, lim, lane);
        }
    }
}

// dynamic shared memory of k_dr_members (G <= DR_BIN_MAX): the winners,
// Y_p*'s bin starts and the non-empty cells as k_datareduct lays them out,
// the grid points' float32 offsets (3 G floats), then the member cells' starts
// (G + 2 ints), the warps' visited bitmasks (vwords words each) and the
// member-cell list (mcap 16-bit member indices)
__host__ __device__ inline size_t dm_qf_offset(int G) {
    return (dr_bins_offset(G) + (size_t)(2 * G + 1) * 4 + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t dm_mstart_offset(int G) { return dm_qf_offset(G) + (size_t)G * 12; }
__host__ __device__ inline size_t dm_vis_offset(int G) {
    return (dm_mstart_offset(G) + (size_t)(G + 2) * 4 + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t dm_mlist_offset(int G, int vwords) {
    return dm_vis_offset(G) + (size_t)(DR_THREADS / 32) * vwords * 4;
}
__host__ __device__ inline size_t dm_smem_bytes(int G, int vwords, int mcap) {
    return dm_mlist_offset(G, vwords) + (size_t)mcap * 2;
}

// cell range [c0, c1] per coordinate of a member box (hi parts lo, hi) moved
// to this node's frame and widened by cw; flat coordinates take cell 0
__device__ __forceinline__ void dm_cell_range(float4 lo4, float4 hi4, const float *lh, const bool *flat,
                                              const float *ihf, float cw, int d, int g, int *c0, int *c1,
                                              float &ext) {
    const float l3[3] = {lo4.x, lo4.y, lo4.z}, h3[3] = {hi4.x, hi4.y, hi4.z};
    ext = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        c0[k] = c1[k] = 0;
        if (k >= d || flat[k]) continue;
        const float a = (l3[k] - lh[k]) - cw, b = (h3[k] - lh[k]) + cw;
        c0[k] = min(max((int)(a * ihf[k]), 0), g - 1);
        c1[k] = min(max((int)(b * ihf[k]), 0), g - 1);
        ext = fmaxf(ext, b - a);
    }
}

// bin of the cell holding the centre of a member box (as dm_cell_range moves it)
__device__ __forceinline__ int dm_centre_bin(float4 lo4, float4 hi4, const float *lh, const bool *flat,
                                             const float *ihf, float cw, int d, int g) {
    const float l3[3] = {lo4.x, lo4.y, lo4.z}, h3[3] = {hi4.x, hi4.y, hi4.z};
    int bin = 0, stride = 1;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k >= d) break;
        int c = 0;
        if (!flat[k]) {
            const float a = (l3[k] - lh[k]) - cw, b = (h3[k] - lh[k]) + cw;
            c = min(max((int)(0.5f * (a + b) * ihf[k]), 0), g - 1);
        }
        bin += c * stride;
        stride *= g;
    }
    return bin;
}

// One CTA per node: DataReduct(S, g^d) for S = Y_p* (when A.parent) u X_j*
// over j in IL(i), read in place.  Result as k_datareduct's: the distinct
// winners sorted to outptr[outlb + a], their number and box.
__global__ void __launch_bounds__(DR_THREADS, 5) k_dr_members(DMArgs A, DRPoints PT) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int scratch[33];
    __shared__ long long s_box[6];
    __shared__ int s_cnt, s_nne;
    __shared__ unsigned s_ext;
    const int a = blockIdx.x, i = A.lb + a;
    const int d = A.d, g = A.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int G = 1;
    for (int k = 0; k < d; k++) G *= g;
    const int64_t nt = A.toff[a + 1] - A.toff[a];
    const int64_t f0 = A.far_ptr[i];
    const int m = (int)(A.far_ptr[i + 1] - f0);
    const int p = A.parent ? A.parent[i] : -1;
    const int np = p >= 0 ? A.ycnt[p] : 0;
    const int32_t *Yp = np > 0 ? A.yptr[p] : nullptr;
    int32_t *out = A.outptr[A.outlb + a];
    int32_t *win = reinterpret_cast<int32_t *>(smem_raw);
    {  // the box of S: the union of its parts' boxes
        long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        for (int e = threadIdx.x; e < m; e += blockDim.x) box_merge(lo, hi, A.xbox + 6 * (int64_t)A.far_idx[f0 + e]);
        if (threadIdx.x == 0 && np > 0) box_merge(lo, hi, A.ybox + 6 * (int64_t)p);
        block_box_write(lo, hi, s_box);
        __syncthreads();
    }
    if (nt <= G) {  // DataReduct returns S itself
        int P = 1;
        while (P < nt) P <<= 1;
        for (int r = threadIdx.x; r < P; r += blockDim.x) win[r] = r < np ? Yp[r] : INT_MAX;
        if (threadIdx.x == 0) s_cnt = np;
        __syncthreads();
        for (int e = warp; e < m; e += nw) {
            const int j = A.far_idx[f0 + e];
            const int c = A.xcnt[j];
            int base = 0;
            if (lane == 0) base = atomicAdd(&s_cnt, c);
            base = __shfl_sync(0xffffffffu, base, 0);
            const int32_t *src = A.xptr[j];
            for (int r = lane; r < c; r += 32) win[base + r] = src[r];
        }
        __syncthreads();
        block_bitonic_sort(win, P);
        for (int r = threadIdx.x; r < nt; r += blockDim.x) out[r] = win[r];
        if (threadIdx.x < 6) A.outbox[6 * (int64_t)(A.outlb + a) + threadIdx.x] = s_box[threadIdx.x];
        if (threadIdx.x == 0) A.outcnt[A.outlb + a] = (int32_t)nt;
        return;
    }
    DMFrame F;
    F.xq = PT.xq;
    F.xqm = A.xqm;
    F.x0 = PT.x[0];
    F.x1 = PT.x[1];
    F.x2 = PT.x[2];
    F.d = d;
    double l[3] = {0.0, 0.0, 0.0}, h[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k >= d) break;
        l[k] = dkey_inv(s_box[k]);
        h[k] = __ddiv_rn(__dsub_rn(dkey_inv(s_box[3 + k]), l[k]), (double)g);
    }
    double W = 0.0, hmin = INFINITY;
    float ihf[3] = {0.f, 0.f, 0.f}, hf[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        F.flat[k] = true;
        F.lh[k] = F.ll[k] = F.qf[k] = 0.f;
        F.q[k] = 0.0;
        if (k >= d) continue;
        W = dmax_(W, __dmul_rn(h[k], (double)g));
        F.flat[k] = !(h[k] > 0.0);
        if (!F.flat[k]) {
            hmin = dmin_(hmin, h[k]);
            ihf[k] = (float)(1.0 / h[k]);
            hf[k] = (float)h[k];
        }
        const double Lk = l[k] - PT.ref[k];
        F.lh[k] = (float)Lk;
        F.ll[k] = (float)(Lk - (double)F.lh[k]);
    }
    // M and delf as in k_datareduct; cw widens the member and chunk boxes
    F.M = (float)(8e-6 * W * W + 1e-12 * W * PT.R);
    const float delf = (float)(1e-5 * W + 1e-12 * PT.R);
    F.cw = (float)(2e-7 * PT.R) + delf;
    const float hminf = (float)hmin;
    int *bstart = reinterpret_cast<int *>(smem_raw + dr_bins_offset(G));
    int *mstart = reinterpret_cast<int *>(smem_raw + dm_mstart_offset(G));
    uint32_t *vis = reinterpret_cast<uint32_t *>(smem_raw + dm_vis_offset(G)) + warp * A.vwords;
    uint16_t *mlist = reinterpret_cast<uint16_t *>(smem_raw + dm_mlist_offset(G, A.vwords));
    for (int b = threadIdx.x; b <= G; b += blockDim.x) bstart[b] = 0;
    for (int b = threadIdx.x; b < G + 2; b += blockDim.x) mstart[b] = 0;
    if (threadIdx.x == 0) {
        s_cnt = 0;
        s_ext = 0u;
    }
    __syncthreads();
    // Y_p*: counting sort into the cells, as k_datareduct bins its set
    int2 *bidx = A.pbin + (np > 0 ? A.poff[a] : 0);
    float4 *pq = A.pq + (np > 0 ? A.poff[a] : 0);
    const unsigned lt = (1u << lane) - 1u;
    for (int p0 = warp * 32; p0 < np; p0 += blockDim.x) {
        const int pp = p0 + lane;
        int bi = -1;
        if (pp < np) {
            const int32_t sid = Yp[pp];
            int stride = 1;
            bi = 0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k >= d) break;
                int cidx = 0;
                if (!F.flat[k]) {
                    const float f = dr_offset(PT.xq, sid, k, F.lh[k], F.ll[k]);
                    cidx = min(max((int)(f * ihf[k]), 0), g - 1);
                }
                bi += cidx * stride;
                stride *= g;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, bi);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (bi >= 0 && lane == leader) base = atomicAdd(&bstart[bi + 1], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (bi >= 0) bidx[pp] = make_int2(bi, base + __popc(peers & lt));
    }
    // members: count the member-cell pairs (mode A)
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
        const int j = A.far_idx[f0 + e];
        int c0[3], c1[3];
        float ext;
        dm_cell_range(A.mbox[2 * (int64_t)j], A.mbox[2 * (int64_t)j + 1], F.lh, F.flat, ihf, F.cw, d, g, c0, c1, ext);
        atomicAdd(&s_cnt, (c1[0] - c0[0] + 1) * (c1[1] - c0[1] + 1) * (c1[2] - c0[2] + 1));
        for (int z = c0[2]; z <= c1[2]; z++)
            for (int y = c0[1]; y <= c1[1]; y++)
                for (int x = c0[0]; x <= c1[0]; x++) atomicAdd(&mstart[x + g * (y + g * z) + 2], 1);
    }
    __syncthreads();
    const bool modeB = s_cnt > A.mcap;
    if (modeB) {  // too many pairs: each member in the cell of its box centre
        for (int b = threadIdx.x; b < G + 2; b += blockDim.x) mstart[b] = 0;
        __syncthreads();
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const int j = A.far_idx[f0 + e];
            int c0[3], c1[3];
            float ext;
            const float4 lo4 = A.mbox[2 * (int64_t)j], hi4 = A.mbox[2 * (int64_t)j + 1];
            dm_cell_range(lo4, hi4, F.lh, F.flat, ihf, F.cw, d, g, c0, c1, ext);
            atomicMax(&s_ext, __float_as_uint(ext));  // non-negative floats order as their bits
            atomicAdd(&mstart[dm_centre_bin(lo4, hi4, F.lh, F.flat, ihf, F.cw, d, g) + 2], 1);
        }
    }
    __syncthreads();
    block_scan_inclusive(bstart, G + 1, scratch);  // bstart[b]: first position of bin b
    block_scan_inclusive(mstart, G + 2, scratch);  // mstart[b + 1]: first position of bin b
    for (int pp = threadIdx.x; pp < np; pp += blockDim.x) {
        const int2 bo = bidx[pp];
        const int pos = bstart[bo.x] + bo.y;
        const int32_t sid = Yp[pp];
        const float4 qa = PT.xq[2 * (int64_t)sid], qb = PT.xq[2 * (int64_t)sid + 1];
        const float p0f = (qa.x - F.lh[0]) + (qa.w - F.ll[0]);
        const float p1f = d > 1 ? (qa.y - F.lh[1]) + (qb.x - F.ll[1]) : 0.f;
        const float p2f = d > 2 ? (qa.z - F.lh[2]) + (qb.y - F.ll[2]) : 0.f;
        pq[pos] = make_float4(p0f, p1f, p2f, __int_as_float(sid));
    }
    for (int e = threadIdx.x; e < m; e += blockDim.x) {  // the member-cell list, bin by bin
        const int j = A.far_idx[f0 + e];
        const float4 lo4 = A.mbox[2 * (int64_t)j], hi4 = A.mbox[2 * (int64_t)j + 1];
        if (modeB) {
            mlist[atomicAdd(&mstart[dm_centre_bin(lo4, hi4, F.lh, F.flat, ihf, F.cw, d, g) + 1], 1)] = (uint16_t)e;
        } else {
            int c0[3], c1[3];
            float ext;
            dm_cell_range(lo4, hi4, F.lh, F.flat, ihf, F.cw, d, g, c0, c1, ext);
            for (int z = c0[2]; z <= c1[2]; z++)
                for (int y = c0[1]; y <= c1[1]; y++)
                    for (int x = c0[0]; x <= c1[0]; x++)
                        mlist[atomicAdd(&mstart[x + g * (y + g * z) + 1], 1)] = (uint16_t)e;
        }
    }
    // grid points' float32 offsets qf, computed once each (the float64 point
    // itself is formed again only for a near tie)
    float *qftab = reinterpret_cast<float *>(smem_raw + dm_qf_offset(G));
    for (int gi = threadIdx.x; gi < G; gi += blockDim.x) {
        int rem = gi;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (k >= d) break;
            const int idx = rem % g;
            rem /= g;
            qftab[3 * gi + k] =
                (float)__dsub_rn(__dadd_rn(l[k], __dmul_rn(__dadd_rn((double)idx, 0.5), h[k])), l[k]);
        }
    }
    __syncthreads();  // mstart[b] is now the first position of bin b
    int *nel = bstart + G + 1;
    if (threadIdx.x == 0) s_nne = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < G; b += blockDim.x)
        if (bstart[b + 1] > bstart[b] || mstart[b + 1] > mstart[b]) nel[atomicAdd(&s_nne, 1)] = dr_pack_cell(b, d, g);
    __syncthreads();
    const int nne = s_nne;
    // mode B widens every cell bound and the stopping radius by the largest
    // half extent of a member box (plus its rounding)
    const float delc = modeB ? delf + fmaf(0.5f, __uint_as_float(s_ext), 1e-6f * __uint_as_float(s_ext)) + delf : delf;
    const bool havep = np > 0;  // a Y_p* part to scan
    // gi / g through a float reciprocal: (gi + 1/2) / g lies at least 1 / (2 g)
    // from an integer, far above the product's rounding for gi < 2^21
    const float invg = 1.0f / (float)g;
    for (int gi = warp; gi < G; gi += nw) {
        int cid[3] = {0, 0, 0}, gidx[3] = {0, 0, 0};
        int rmax = 0;
        {
            int rem = gi;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k >= d) break;
                const int qd = (int)(((float)rem + 0.5f) * invg);
                const int idx = rem - qd * g;
                rem = qd;
                gidx[k] = idx;
                F.qf[k] = qftab[3 * gi + k];
                cid[k] = F.flat[k] ? 0 : idx;
                if (!F.flat[k]) rmax = max(rmax, max(cid[k], g - 1 - cid[k]));
            }
        }
        for (int w = lane; w < A.vwords; w += 32) vis[w] = 0u;
        __syncwarp();
        float b1 = INFINITY, b2 = INFINITY;  // this lane's two smallest float32 distances
        int32_t l1 = INT_MAX;                // the label of its smallest
        float lim = INFINITY;                // the warp's smallest distance + M
        long long bk = LLONG_MAX;            // (near ties) the best float64 key and its label
        int32_t bl = INT_MAX;
        // rings 0 and 1 with the stop test; a search still open after ring 1
        // scans the non-empty cells instead
        const int rA = min(rmax, 1);
        int stage = 2;  // 0 or 1: stopped after that ring; 2: the non-empty cells were scanned
        for (int r = 0; r <= rA; r++) {
            const int side = 2 * r + 1;
            int total = 1;
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (k < d) total *= F.flat[k] ? 1 : side;
            for (int e0 = 0; e0 < total; e0 += 32) {
                int bin = 0;
                float lb = 0.f;
                bool ok = e0 + lane < total && dr_ring_cell(e0 + lane, r, d, g, cid, F.flat, hf, F.qf, delc, bin, lb);
                ok = ok && lb <= lim;
                dr_scan_top2(havep && ok, bin, bstart, pq, F.qf, b1, b2, l1, lane);
                lim = warp_minf(b1) + F.M;
                dm_visit<false>(ok, bin, mstart, mlist, vis, f0, A, F, b1, b2, l1, lim, bk, bl, lane);
            }
            // (r + 1/2) h_min - delta and its square rounded down in float32
            const float rr = ((float)r + 0.5f) * hminf * 0.9999996f - delc;
            if (rr > 0.f && lim < rr * rr * 0.9999996f) {
                stage = r;
                break;
            }
        }
        if (stage == 2 && rmax <= 1) stage = rA;  // rings 0..rmax held every cell
        if (stage == 2) {
            // the non-empty cell with the smallest bound first, then the
            // others whose bound passes
            float blb = INFINITY;
            int bbin = -1;
            for (int e0 = lane; e0 < nne; e0 += 32) {
                const int pk = nel[e0];
                int cheb;
                const float lb = dr_cell_lb(pk, d, cid, F.flat, hf, F.qf, delc, cheb);
                if (cheb >= 2 && lb < blb) {
                    blb = lb;
                    bbin = pk & 4095;
                }
            }
            const float mlb = warp_minf(blb);
            const int b0 = __shfl_sync(0xffffffffu, bbin, __ffs(__ballot_sync(0xffffffffu, blb == mlb)) - 1);
            if (b0 >= 0 && mlb <= lim) {
                dr_scan_top2(havep && lane == 0, b0, bstart, pq, F.qf, b1, b2, l1, lane);
                lim = warp_minf(b1) + F.M;
                dm_visit<false>(lane == 0, b0, mstart, mlist, vis, f0, A, F, b1, b2, l1, lim, bk, bl, lane);
            }
            for (int e0 = 0; e0 < nne; e0 += 32) {
                bool ok = false;
                int bin = 0;
                if (e0 + lane < nne) {
                    const int pk = nel[e0 + lane];
                    bin = pk & 4095;
                    int cheb;
                    const float lb = dr_cell_lb(pk, d, cid, F.flat, hf, F.qf, delc, cheb);
                    ok = cheb >= 2 && lb <= lim && bin != b0;
                }
                dr_scan_top2(havep && ok, bin, bstart, pq, F.qf, b1, b2, l1, lane);
                lim = warp_minf(b1) + F.M;
                dm_visit<false>(ok, bin, mstart, mlist, vis, f0, A, F, b1, b2, l1, lim, bk, bl, lane);
            }
        }
        const float m1 = warp_minf(b1);
        const int w = __ffs(__ballot_sync(0xffffffffu, b1 == m1)) - 1;
        const float sec = warp_minf(lane == w ? b2 : b1);
        float limx = m1 + F.M;
        int32_t winner;
        if (sec > limx) {
            winner = __shfl_sync(0xffffffffu, l1, w);
        } else if (!__any_sync(0xffffffffu, b2 <= limx)) {
            // near tie, but no lane holds two points within limx: every point
            // within limx was scanned (the bounds prune only farther ones) and
            // went to one lane (each point is scanned once, on one lane), where
            // it is the smallest, so those lanes' points are all the
            // candidates.  Float64 distances, the smaller label taking ties.
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (k < d) F.q[k] = __dadd_rn(l[k], __dmul_rn(__dadd_rn((double)gidx[k], 0.5), h[k]));
            long long bk2 = LLONG_MAX;
            int32_t bl2 = INT_MAX;
            if (b1 <= limx) {
                bk2 = __double_as_longlong(h2_dist2(d, F.x0[l1], d > 1 ? F.x1[l1] : 0.0, d > 2 ? F.x2[l1] : 0.0,
                                                    F.q[0], F.q[1], F.q[2]));
                bl2 = l1;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long kk = __shfl_xor_sync(0xffffffffu, bk2, o);
                const int32_t kl = __shfl_xor_sync(0xffffffffu, bl2, o);
                if (kk < bk2 || (kk == bk2 && kl < bl2)) {
                    bk2 = kk;
                    bl2 = kl;
                }
            }
            winner = bl2;
        } else {
            // near tie: every point within M of the smallest in float64, over
            // the cells the search visited
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (k < d) F.q[k] = __dadd_rn(l[k], __dmul_rn(__dadd_rn((double)gidx[k], 0.5), h[k]));
            for (int v = lane; v < A.vwords; v += 32) vis[v] = 0u;
            __syncwarp();
            const int rB = stage == 2 ? rA : stage;
            for (int r = 0; r <= rB; r++) {
                const int side = 2 * r + 1;
                int total = 1;
#pragma unroll
                for (int k = 0; k < 3; k++)
                    if (k < d) total *= F.flat[k] ? 1 : side;
                for (int e0 = 0; e0 < total; e0 += 32) {
                    int bin = 0;
                    float lb = 0.f;
                    bool ok =
                        e0 + lane < total && dr_ring_cell(e0 + lane, r, d, g, cid, F.flat, hf, F.qf, delc, bin, lb);
                    ok = ok && lb <= limx;
                    dr_scan_exact(havep && ok && bstart[bin + 1] > bstart[bin], bin, bstart, pq, F.qf, limx, d, F.x0, F.x1,
                                  F.x2, F.q, bk, bl, lane);
                    dm_visit<true>(ok, bin, mstart, mlist, vis, f0, A, F, b1, b2, l1, limx, bk, bl, lane);
                }
            }
            if (stage == 2)
                for (int e0 = 0; e0 < nne; e0 += 32) {
                    bool ok = false;
                    int bin = 0;
                    if (e0 + lane < nne) {
                        const int pk = nel[e0 + lane];
                        bin = pk & 4095;
                        int cheb;
                        const float lb = dr_cell_lb(pk, d, cid, F.flat, hf, F.qf, delc, cheb);
                        ok = cheb >= 2 && lb <= limx;
                    }
                    dr_scan_exact(havep && ok && bstart[bin + 1] > bstart[bin], bin, bstart, pq, F.qf, limx, d, F.x0, F.x1,
                                  F.x2, F.q, bk, bl, lane);
                    dm_visit<true>(ok, bin, mstart, mlist, vis, f0, A, F, b1, b2, l1, limx, bk, bl, lane);
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long kk = __shfl_xor_sync(0xffffffffu, bk, o);
                const int32_t kl = __shfl_xor_sync(0xffffffffu, bl, o);
                if (kk < bk || (kk == bk && kl < bl)) {
                    bk = kk;
                    bl = kl;
                }
            }
            winner = bl;
        }
        if (lane == 0) win[gi] = winner;
    }
    __syncthreads();
    {  // bounding box of the winners
        long long blo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, bhi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        for (int gi = threadIdx.x; gi < G; gi += blockDim.x) {
            const int32_t sid = win[gi];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k >= d) break;
                const long long kv = dkey((k == 0 ? F.x0 : (k == 1 ? F.x1 : F.x2))[sid]);
                blo[k] = min(blo[k], kv);
                bhi[k] = max(bhi[k], kv);
            }
        }
        block_box_write(blo, bhi, A.outbox + 6 * (int64_t)(A.outlb + a));
    }
    int P = 1;
    while (P < G) P <<= 1;
    for (int r = G + threadIdx.x; r < P; r += blockDim.x) win[r] = INT_MAX;
    __syncthreads();
    block_bitonic_sort(win, P);
    const int mm = block_unique_write(win, P, out, scratch);
    if (threadIdx.x == 0) A.outcnt[A.outlb + a] = mm;
}

// Surface-based DataReduct (section 3.3): the reference set is ne points on
// each of three ellipsoids centred at the centre c of the set's box [l, u],
// semi-axes gamma (u - l) for gamma = 0.3, 0.6, 1.2 (q = c + (gamma (u - l)) *
// dir_j per coordinate, each operation explicitly rounded in that order; the
// unit directions dir_j come precomputed from the host); every reference point
// takes its nearest point of the set (float64 squared distance, ties to the
// smaller label), the winners deduplicated and sorted.  The search is the
// brute-force sweep of k_datareduct with float32 top-two distances and a
// float64 re-scan on near ties; the reference points reach 1.7 box widths from
// the corner, so M takes twice the box's extent.
constexpr int DS_THREADS = 256;
constexpr int DS_QPT = 4;

__global__ void __launch_bounds__(DS_THREADS)
    k_datareduct_surface(const int64_t *toff, const int32_t *tdata, int g, int d, DRPoints PT, const double *dirs,
                         int ne, int32_t *const *outptr, int32_t *outcnt, int lb, const long long *tbox,
                         long long *outbox) {
    const double *x0 = PT.x[0], *x1 = PT.x[1], *x2 = PT.x[2];
    extern __shared__ unsigned char smem_raw[];
    int32_t *win = reinterpret_cast<int32_t *>(smem_raw);  // [P]
    __shared__ int32_t tid_s[DR_TILE];
    __shared__ float tf_s[3][DR_TILE];
    __shared__ int scratch[33];
    const int a = blockIdx.x;
    const int node = lb + a;
    const int64_t t0 = toff[a], nt = toff[a + 1] - toff[a];
    const int32_t *T = tdata + t0;
    int32_t *out = outptr[node];
    int G = 1;
    for (int k = 0; k < d; k++) G *= g;
    if (nt <= G) {  // DataReduct returns S itself
        int P = 1;
        while (P < nt) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) win[i] = i < nt ? T[i] : INT_MAX;
        __syncthreads();
        block_bitonic_sort(win, P);
        for (int i = threadIdx.x; i < nt; i += blockDim.x) out[i] = win[i];
        if (threadIdx.x < 6) outbox[6 * (int64_t)node + threadIdx.x] = tbox[6 * (int64_t)a + threadIdx.x];
        if (threadIdx.x == 0) outcnt[node] = (int32_t)nt;
        return;
    }
    const int NQ = 3 * ne;
    double l[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0}, w[3] = {0.0, 0.0, 0.0};
    float lh[3] = {0.f, 0.f, 0.f}, ll[3] = {0.f, 0.f, 0.f};
    double W = 0.0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (k >= d) break;
        l[k] = dkey_inv(tbox[6 * (int64_t)a + k]);
        const double u = dkey_inv(tbox[6 * (int64_t)a + 3 + k]);
        c[k] = __dmul_rn(__dadd_rn(l[k], u), 0.5);
        w[k] = __dsub_rn(u, l[k]);
        W = dmax_(W, w[k]);
        const double Lk = l[k] - PT.ref[k];
        lh[k] = (float)Lk;
        ll[k] = (float)(Lk - (double)lh[k]);
    }
    const double E = 2.0 * W;
    const float M = (float)(8e-6 * E * E + 1e-12 * E * PT.R);
    auto refpt = [&](int qi, double *q) {
        const int e = qi / ne, j = qi - e * ne;
        const double ge = e == 0 ? 0.3 : (e == 1 ? 0.6 : 1.2);
#pragma unroll
        for (int k = 0; k < 3; k++)
            q[k] = k < d ? __dadd_rn(c[k], __dmul_rn(__dmul_rn(ge, w[k]), dirs[3 * j + k])) : 0.0;
    };
    for (int qbase = 0; qbase < NQ; qbase += DS_THREADS * DS_QPT) {
        float qf[DS_QPT][3], b1[DS_QPT], b2[DS_QPT];
        int32_t i1[DS_QPT];
#pragma unroll
        for (int j = 0; j < DS_QPT; j++) {
            const int qi = qbase + j * DS_THREADS + threadIdx.x;
            double q[3] = {0.0, 0.0, 0.0};
            if (qi < NQ) refpt(qi, q);
#pragma unroll
            for (int k = 0; k < 3; k++) qf[j][k] = k < d ? (float)__dsub_rn(q[k], l[k]) : 0.0f;
            b1[j] = INFINITY;
            b2[j] = INFINITY;
            i1[j] = INT_MAX;
        }
        for (int64_t tb = 0; tb < nt; tb += DR_TILE) {
            const int cnt = (int)(nt - tb < DR_TILE ? nt - tb : DR_TILE);
            __syncthreads();
            for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
                const int32_t sid = T[tb + r];
                tid_s[r] = sid;
#pragma unroll
                for (int k = 0; k < 3; k++) tf_s[k][r] = k < d ? dr_offset(PT.xq, sid, k, lh[k], ll[k]) : 0.f;
            }
            __syncthreads();
            for (int r = 0; r < cnt; r++) {
                const float f0 = tf_s[0][r], f1 = tf_s[1][r], f2 = tf_s[2][r];
#pragma unroll
                for (int j = 0; j < DS_QPT; j++) {
                    const float e0 = f0 - qf[j][0], e1 = f1 - qf[j][1], e2 = f2 - qf[j][2];
                    const float d32 = fmaf(e2, e2, fmaf(e1, e1, e0 * e0));
                    if (d32 < b2[j]) {
                        if (d32 < b1[j]) {
                            b2[j] = b1[j];
                            b1[j] = d32;
                            i1[j] = tid_s[r];
                        } else {
                            b2[j] = d32;
                        }
                    }
                }
            }
        }
        // near ties: every point within M of the smallest, in float64
#pragma unroll
        for (int j = 0; j < DS_QPT; j++) {
            const int qi = qbase + j * DS_THREADS + threadIdx.x;
            const float limx = b1[j] + M;
            const bool need = qi < NQ && !(b2[j] > limx);
            if (!__syncthreads_or(need)) continue;
            double q[3] = {0.0, 0.0, 0.0};
            if (qi < NQ) refpt(qi, q);
            long long bk = LLONG_MAX;
            int32_t bl = INT_MAX;
            for (int64_t tb = 0; tb < nt; tb += DR_TILE) {
                const int cnt = (int)(nt - tb < DR_TILE ? nt - tb : DR_TILE);
                __syncthreads();
                for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
                    const int32_t sid = T[tb + r];
                    tid_s[r] = sid;
#pragma unroll
                    for (int k = 0; k < 3; k++) tf_s[k][r] = k < d ? dr_offset(PT.xq, sid, k, lh[k], ll[k]) : 0.f;
                }
                __syncthreads();
                if (need)
                    for (int r = 0; r < cnt; r++) {
                        const float e0 = tf_s[0][r] - qf[j][0], e1 = tf_s[1][r] - qf[j][1], e2 = tf_s[2][r] - qf[j][2];
                        if (fmaf(e2, e2, fmaf(e1, e1, e0 * e0)) <= limx) {
                            const int32_t sid = tid_s[r];
                            const long long kk = __double_as_longlong(
                                h2_dist2(d, x0[sid], d > 1 ? x1[sid] : 0.0, d > 2 ? x2[sid] : 0.0, q[0], q[1], q[2]));
                            if (kk < bk || (kk == bk && sid < bl)) {
                                bk = kk;
                                bl = sid;
                            }
                        }
                    }
            }
            if (need) i1[j] = bl;
        }
#pragma unroll
        for (int j = 0; j < DS_QPT; j++) {
            const int qi = qbase + j * DS_THREADS + threadIdx.x;
            if (qi < NQ) win[qi] = i1[j];
        }
    }
    __syncthreads();
    {  // bounding box of the winners
        long long blo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, bhi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        for (int qi = threadIdx.x; qi < NQ; qi += blockDim.x) {
            const int32_t sid = win[qi];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k >= d) break;
                const long long kv = dkey((k == 0 ? x0 : (k == 1 ? x1 : x2))[sid]);
                blo[k] = min(blo[k], kv);
                bhi[k] = max(bhi[k], kv);
            }
        }
        block_box_write(blo, bhi, outbox + 6 * (int64_t)node);
    }
    int P = 1;
    while (P < NQ) P <<= 1;
    for (int i = NQ + threadIdx.x; i < P; i += blockDim.x) win[i] = INT_MAX;
    __syncthreads();
    block_bitonic_sort(win, P);
    int m = block_unique_write(win, P, out, scratch);
    if (threadIdx.x == 0) outcnt[node] = m;
}

// DataReduct by farthest point sampling (section 3.3): X* starts with the
// point of smallest label and grows by the point farthest from X* (largest
// float64 squared distance to its nearest member, ties to the smaller label)
// until it holds g^d points; sorted on output.  One CTA a node; md holds each
// point's squared distance to X* (negative once the point is in X*).  g^d
// rounds of a block-wide update and argmax over the set: exact, but costly on
// large sets by its sequential nature.
constexpr int FPS_THREADS = 512;

__device__ __forceinline__ void fps_better(long long &k, int32_t &lab, int &pos, long long k2, int32_t lab2,
                                           int pos2) {
    if (k2 > k || (k2 == k && lab2 < lab)) { k = k2; lab = lab2; pos = pos2; }
}

__global__ void __launch_bounds__(FPS_THREADS)
    k_datareduct_fps(const int64_t *toff, const int32_t *tdata, int g, int d, DRPoints PT, double *mdbase,
                     int32_t *const *outptr, int32_t *outcnt, int lb, const long long *tbox, long long *outbox) {
    const double *x0 = PT.x[0], *x1 = PT.x[1], *x2 = PT.x[2];
    extern __shared__ unsigned char smem_raw[];
    int32_t *win = reinterpret_cast<int32_t *>(smem_raw);  // [P]
    __shared__ long long s_key[FPS_THREADS / 32];
    __shared__ int32_t s_lab[FPS_THREADS / 32];
    __shared__ int s_pos[FPS_THREADS / 32];
    __shared__ int s_f;
    __shared__ int scratch[33];
    const int a = blockIdx.x;
    const int node = lb + a;
    const int64_t t0 = toff[a], nt64 = toff[a + 1] - toff[a];
    const int32_t *T = tdata + t0;
    int32_t *out = outptr[node];
    int G = 1;
    for (int k = 0; k < d; k++) G *= g;
    if (nt64 <= G) {  // DataReduct returns S itself
        int P = 1;
        while (P < nt64) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) win[i] = i < nt64 ? T[i] : INT_MAX;
        __syncthreads();
        block_bitonic_sort(win, P);
        for (int i = threadIdx.x; i < nt64; i += blockDim.x) out[i] = win[i];
        if (threadIdx.x < 6) outbox[6 * (int64_t)node + threadIdx.x] = tbox[6 * (int64_t)a + threadIdx.x];
        if (threadIdx.x == 0) outcnt[node] = (int32_t)nt64;
        return;
    }
    const int nt = (int)nt64;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double *md = mdbase + t0;
    // the first point: the smallest label
    {
        long long bk = LLONG_MIN;
        int32_t bl = INT_MAX;
        int bp = -1;
        for (int p = threadIdx.x; p < nt; p += blockDim.x) {
            md[p] = INFINITY;
            fps_better(bk, bl, bp, 0, T[p], p);  // equal keys: the label decides
        }
        for (int o = 16; o > 0; o >>= 1)
            fps_better(bk, bl, bp, __shfl_xor_sync(0xffffffffu, bk, o), __shfl_xor_sync(0xffffffffu, bl, o),
                       __shfl_xor_sync(0xffffffffu, bp, o));
        if (lane == 0) { s_key[warp] = bk; s_lab[warp] = bl; s_pos[warp] = bp; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; w++) fps_better(bk, bl, bp, s_key[w], s_lab[w], s_pos[w]);
            s_f = bp;
        }
        __syncthreads();
    }
    for (int m = 0; m < G; m++) {
        const int f = s_f;
        const int32_t fl = T[f];
        if (threadIdx.x == 0) {
            win[m] = fl;
            md[f] = -1.0;
        }
        if (m + 1 == G) break;
        __syncthreads();
        const double f0 = x0[fl], f1 = d > 1 ? x1[fl] : 0.0, f2 = d > 2 ? x2[fl] : 0.0;
        long long bk = LLONG_MIN;
        int32_t bl = INT_MAX;
        int bp = -1;
        for (int p = threadIdx.x; p < nt; p += blockDim.x) {
            double v = md[p];
            if (v < 0.0) continue;
            const int32_t sid = T[p];
            const double dd = h2_dist2(d, x0[sid], d > 1 ? x1[sid] : 0.0, d > 2 ? x2[sid] : 0.0, f0, f1, f2);
            if (dd < v) {
                v = dd;
                md[p] = v;
            }
            fps_better(bk, bl, bp, __double_as_longlong(v), sid, p);
        }
        for (int o = 16; o > 0; o >>= 1)
            fps_better(bk, bl, bp, __shfl_xor_sync(0xffffffffu, bk, o), __shfl_xor_sync(0xffffffffu, bl, o),
                       __shfl_xor_sync(0xffffffffu, bp, o));
        if (lane == 0) { s_key[warp] = bk; s_lab[warp] = bl; s_pos[warp] = bp; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; w++) fps_better(bk, bl, bp, s_key[w], s_lab[w], s_pos[w]);
            s_f = bp;
        }
        __syncthreads();
    }
    __syncthreads();
    {  // bounding box of the picked points
        long long blo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, bhi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
        for (int i = threadIdx.x; i < G; i += blockDim.x) {
            const int32_t sid = win[i];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k >= d) break;
                const long long kv = dkey((k == 0 ? x0 : (k == 1 ? x1 : x2))[sid]);
                blo[k] = min(blo[k], kv);
                bhi[k] = max(bhi[k], kv);
            }
        }
        block_box_write(blo, bhi, outbox + 6 * (int64_t)node);
    }
    int P = 1;
    while (P < G) P <<= 1;
    for (int i = G + threadIdx.x; i < P; i += blockDim.x) win[i] = INT_MAX;
    __syncthreads();
    block_bitonic_sort(win, P);
    int m = block_unique_write(win, P, out, scratch);
    if (threadIdx.x == 0) outcnt[node] = m;
}

// unit directions of the surface reference points: the Fibonacci lattice in
// 3D (z_j = 1 - (2j + 1) / ne, rho = sqrt(1 - z^2), phi_j = j pi (3 - sqrt 5)),
// equal angles 2 pi (j + 1/2) / ne in 2D; host arithmetic without contraction
std::vector<double> surface_dirs(int d, int ne) {
    const double pi = 3.14159265358979323846;
    std::vector<double> v((size_t)3 * std::max(ne, 1), 0.0);
    for (int j = 0; j < ne; j++) {
        if (d == 3) {
            const double z = 1.0 - (2.0 * j + 1.0) / ne;
            const double rho = std::sqrt(1.0 - z * z);
            const double phi = j * (pi * (3.0 - std::sqrt(5.0)));
            v[3 * j] = rho * std::cos(phi);
            v[3 * j + 1] = rho * std::sin(phi);
            v[3 * j + 2] = z;
        } else {
            const double th = 2.0 * pi * (j + 0.5) / ne;
            v[3 * j] = std::cos(th);
            v[3 * j + 1] = std::sin(th);
        }
    }
    return v;
}

int64_t gridsize(int g, int d) {
    int64_t G = 1;
    for (int k = 0; k < d; k++) G *= g;
    return G;
}

void launch_datareduct(const int64_t *toff, const int32_t *tdata, int64_t ttot, int nl, int g, int d,
                       const DRPoints &pts, int32_t *const *outptr, int32_t *outcnt, int lb, const long long *tbox,
                       long long *outbox, cudaStream_t s, int method = 0) {
    if (nl <= 0) return;
    int G = (int)gridsize(g, d);
    if (method == 2) {  // farthest point sampling
        static std::once_flag fattr;
        std::call_once(fattr, [] {
            H2_CUDA(cudaFuncSetAttribute(k_datareduct_fps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(DR_MAX_GRID * sizeof(int32_t))));
        });
        DevBuf<double> md;
        md.alloc((size_t)std::max<int64_t>(ttot, 1), s);
        int P = 1;
        while (P < G) P <<= 1;
        ProfScope ps(KT_DATAREDUCT, s);
        k_datareduct_fps<<<nl, FPS_THREADS, (size_t)P * sizeof(int32_t), s>>>(toff, tdata, g, d, pts, md.p, outptr,
                                                                              outcnt, lb, tbox, outbox);
        H2_LAUNCH("k_datareduct_fps");
        return;
    }
    if (method == 1) {  // surface-based
        static std::once_flag sattr;
        std::call_once(sattr, [] {
            H2_CUDA(cudaFuncSetAttribute(k_datareduct_surface, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(DR_MAX_GRID * sizeof(int32_t))));
        });
        const int ne = d >= 2 ? G / 3 : 0;
        const std::vector<double> hd = surface_dirs(d, ne);
        DevBuf<double> dirs;
        dirs.alloc(hd.size(), s);
        H2_CUDA(cudaMemcpyAsync(dirs.p, hd.data(), hd.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        int P = 1;
        while (P < G) P <<= 1;
        ProfScope ps(KT_DATAREDUCT, s);
        k_datareduct_surface<<<nl, DS_THREADS, (size_t)P * sizeof(int32_t), s>>>(toff, tdata, g, d, pts, dirs.p, ne,
                                                                                 outptr, outcnt, lb, tbox, outbox);
        H2_LAUNCH("k_datareduct_surface");  // (a pageable-source copy has read hd when it returns)
        return;
    }
    size_t sm = dr_smem_bytes(G);
    static std::once_flag attr;
    std::call_once(attr, [] {
        size_t mx = std::max(dr_smem_bytes(DR_MAX_GRID), dr_smem_bytes(DR_BIN_MAX));
        H2_CUDA(cudaFuncSetAttribute(k_datareduct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    });
    DevBuf<int2> bins;
    DevBuf<float4> pq;
    bins.alloc((size_t)std::max<int64_t>(ttot, 1), s);
    pq.alloc((size_t)std::max<int64_t>(ttot, 1), s);
    ProfScope ps(KT_DATAREDUCT, s);
    k_datareduct<<<nl, DR_THREADS, sm, s>>>(toff, tdata, g, d, pts, outptr, outcnt, lb, bins.p, pq.p, tbox, outbox);
    H2_LAUNCH("k_datareduct");
}

constexpr int DM_MCAP_MAX = 32768;         // member-cell list entries at most
constexpr size_t DM_SMEM_MAX = 200 * 1024;  // dynamic shared memory of k_dr_members at most

// DataReduct of the nl sets A describes by the search over members; ilmax is
// the longest interaction list among them
void launch_members(DMArgs A, const DRPoints &pts, int nl, int G, int ilmax, cudaStream_t s) {
    if (nl <= 0) return;
    A.vwords = std::max(1, (ilmax + 31) / 32);
    // about five cells a member (boxes near a cell's size overlap two cells per
    // coordinate at most); a node needing more takes mode B
    A.mcap = std::max(ilmax, std::min(5 * ilmax + G, DM_MCAP_MAX));
    const size_t sm = dm_smem_bytes(G, A.vwords, A.mcap);
    H2_REQUIRE(sm <= DM_SMEM_MAX, "DataReduct over members: shared memory");
    static std::once_flag attr;
    std::call_once(attr, [] {
        H2_CUDA(cudaFuncSetAttribute(k_dr_members, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DM_SMEM_MAX));
    });
    ProfScope ps(KT_DATAREDUCT, s);
    k_dr_members<<<nl, DR_THREADS, sm, s>>>(A, pts);
    H2_LAUNCH("k_dr_members");
}

}  // namespace

void hidr_impl(h2_hidr_s *h) {
    h2_tree_s *t = h->tree;
    cudaStream_t s = h->stream;
    const int nn = t->nnodes, d = t->d;
    H2_REQUIRE(gridsize(h->g1, d) <= DR_MAX_GRID && gridsize(h->g2, d) <= DR_MAX_GRID,
               "g^dim must be at most 16384");
    h->xcnt.alloc(nn, s);
    h->ycnt.alloc(nn, s);
    h->xptr.alloc(nn, s);
    h->yptr.alloc(nn, s);
    H2_CUDA(cudaMemsetAsync(h->xcnt.p, 0, nn * sizeof(int32_t), s));
    H2_CUDA(cudaMemsetAsync(h->ycnt.p, 0, nn * sizeof(int32_t), s));
    H2_CUDA(cudaMemsetAsync(h->xptr.p, 0, nn * sizeof(int32_t *), s));
    H2_CUDA(cudaMemsetAsync(h->yptr.p, 0, nn * sizeof(int32_t *), s));
    DRPoints pts;
    pts.xq = t->xq.p;
    for (int k = 0; k < 3; k++) {
        pts.x[k] = t->xs[k].p;
        pts.ref[k] = t->geom.lo[k];
    }
    h->xbox.alloc((size_t)nn * 6, s);
    h->ybox.alloc((size_t)nn * 6, s);
    pts.R = t->geom.side;
    h->xbufs.resize(t->nlevels);
    h->ybufs.resize(t->nlevels);
    h->xmax_level.assign(t->nlevels, 0);
    h->ymax_level.assign(t->nlevels, 0);
    DevBuf<int64_t> sz, cap, toff, coff;
    DevBuf<int32_t> tdata;
    DevBuf<long long> tbox;
    cudaEvent_t e0, e1, e2;
    H2_CUDA(cudaEventCreate(&e0));
    H2_CUDA(cudaEventCreate(&e1));
    H2_CUDA(cudaEventCreate(&e2));
    H2_CUDA(cudaEventRecord(e0, s));
    // bottom-up: X_i* = DataReduct(S_i, g1^d), deepest level first
    for (int l = t->nlevels - 1; l >= 1; l--) {
        int lb = t->lptr[l], nl = t->lptr[l + 1] - lb;
        sz.alloc(nl, s); cap.alloc(nl, s); toff.alloc(nl + 1, s); coff.alloc(nl + 1, s);
        k_size_up<<<blocks_for(nl, 128), 128, 0, s>>>(lb, nl, t->nchild.p, t->fchild.p, t->begin.p, t->end.p,
                                                       h->xcnt.p, h->g1, d, sz.p, cap.p);
        H2_LAUNCH("k_size_up");
        scan_exclusive(sz.p, toff.p, nl, s);
        scan_exclusive(cap.p, coff.p, nl, s);
        int64_t ttot = read_scalar(toff.p + nl, s), ctot = read_scalar(coff.p + nl, s);
        h->tmax = std::max(h->tmax, ttot);
        h->ttotal += ttot;
        tdata.alloc(ttot > 0 ? ttot : 1, s);
        h->xbufs[l].alloc(ctot > 0 ? ctot : 1, s);
        k_set_ptrs<<<blocks_for(nl, 128), 128, 0, s>>>(lb, nl, h->xbufs[l].p, coff.p, h->xptr.p);
        H2_LAUNCH("k_set_ptrs");
        tbox.alloc((size_t)nl * 6, s);
        k_gather_up<<<nl, 256, 0, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, t->end.p, h->xptr.p, h->xcnt.p,
                                       toff.p, tdata.p, t->xs[0].p, t->xs[1].p, t->xs[2].p, d, h->xbox.p, tbox.p);
        H2_LAUNCH("k_gather_up");
        launch_datareduct(toff.p, tdata.p, ttot, nl, h->g1, d, pts, h->xptr.p, h->xcnt.p, lb, tbox.p, h->xbox.p, s,
                          h->method);
    }
    H2_CUDA(cudaEventRecord(e1, s));
    // top-down: Y_i* = DataReduct(Y_p* u X_j* (j in IL(i)), g2^d), level 1 first;
    // with the interaction-list reduction, u DataReduct(X_j* (j in IL(i)), g2^d)
    const bool il = h->il_reduce;
    const int G2 = (int)gridsize(h->g2, d);
    // The volume method on a grid binned in shared memory reads the X_j* in
    // place (k_dr_members) on levels whose interaction lists are at most
    // DM_MAX_MEMBERS long; other levels and methods copy each set out first.
    const bool members = h->method == 0 && G2 <= DR_BIN_MAX && !h->copy_sets;
    std::vector<int> ilmax(t->nlevels, 0);
    DevBuf<int64_t> nch, choff, psz, poff;
    DevBuf<float4> cbox, mbox, xqm;
    DevBuf<int2> pbin;
    DevBuf<float4> ppq;
    if (members) {
        const std::vector<int64_t> fp = read_vec(t->far_ptr.p, (size_t)nn + 1, s);
        for (int l = 1; l < t->nlevels; l++)
            for (int i = t->lptr[l]; i < t->lptr[l + 1]; i++)
                ilmax[l] = std::max(ilmax[l], (int)std::min<int64_t>(fp[i + 1] - fp[i], INT_MAX));
        nch.alloc(nn, s);
        choff.alloc(nn + 1, s);
        k_chunk_counts<<<blocks_for(nn, 256), 256, 0, s>>>(nn, h->xcnt.p, nch.p);
        H2_LAUNCH("k_chunk_counts");
        scan_exclusive(nch.p, choff.p, nn, s);
        const int64_t nchunks = read_scalar(choff.p + nn, s);
        cbox.alloc((size_t)std::max<int64_t>(2 * nchunks, 2), s);
        mbox.alloc((size_t)2 * nn, s);
        xqm.alloc((size_t)std::max<int64_t>(2 * DM_CHUNK * nchunks, 2), s);
        if (nn > 1) {
            k_member_boxes<<<blocks_for((int64_t)(nn - 1) * 32, 256), 256, 0, s>>>(1, nn, h->xptr.p, h->xcnt.p,
                                                                                   choff.p, t->xq.p, cbox.p, mbox.p, xqm.p);
            H2_LAUNCH("k_member_boxes");
        }
    }
    DevBuf<int64_t> szl, capl, loff, lcoff;
    DevBuf<int32_t> tl, lbuf, lcnt;
    DevBuf<int32_t *> lptr;
    DevBuf<long long> lbox, lobox;
    size_t merge_smem = 0;
    if (il) {
        int P = 1;
        while (P < 2 * gridsize(h->g2, d)) P <<= 1;
        merge_smem = (size_t)P * sizeof(int32_t);
        H2_REQUIRE(merge_smem <= 48 * 1024, "the interaction-list reduction needs g2^dim <= 4096");
    }
    h->members_levels = 0;
    for (int l = 1; l < t->nlevels; l++) {
        int lb = t->lptr[l], nl = t->lptr[l + 1] - lb;
        const bool mem_l = members && ilmax[l] <= DM_MAX_MEMBERS;
        sz.alloc(nl, s); cap.alloc(nl, s); toff.alloc(nl + 1, s); coff.alloc(nl + 1, s);
        if (il) { szl.alloc(nl, s); capl.alloc(nl, s); loff.alloc(nl + 1, s); lcoff.alloc(nl + 1, s); }
        if (mem_l) { psz.alloc(nl, s); poff.alloc(nl + 1, s); }
        k_size_down<<<blocks_for((int64_t)nl * 32, 256), 256, 0, s>>>(lb, nl, t->parent.p, t->far_ptr.p,
                                                                       t->far_idx.p, h->xcnt.p, h->ycnt.p, h->g2, d,
                                                                       sz.p, cap.p, il ? szl.p : nullptr,
                                                                       il ? capl.p : nullptr, mem_l ? psz.p : nullptr);
        H2_LAUNCH("k_size_down");
        scan_exclusive(sz.p, toff.p, nl, s);
        scan_exclusive(cap.p, coff.p, nl, s);
        int64_t ttot = read_scalar(toff.p + nl, s), ctot = read_scalar(coff.p + nl, s);
        h->tmax = std::max(h->tmax, ttot);
        h->ttotal += ttot;
        h->ybufs[l].alloc(ctot > 0 ? ctot : 1, s);
        k_set_ptrs<<<blocks_for(nl, 128), 128, 0, s>>>(lb, nl, h->ybufs[l].p, coff.p, h->yptr.p);
        H2_LAUNCH("k_set_ptrs");
        DMArgs A{};
        if (mem_l) {
            h->members_levels++;
            scan_exclusive(psz.p, poff.p, nl, s);
            const int64_t ptot = read_scalar(poff.p + nl, s);
            pbin.alloc((size_t)std::max<int64_t>(ptot, 1), s);
            ppq.alloc((size_t)std::max<int64_t>(ptot, 1), s);
            A.lb = lb;
            A.outlb = lb;
            A.g = h->g2;
            A.d = d;
            A.toff = toff.p;
            A.parent = t->parent.p;
            A.yptr = h->yptr.p;
            A.ycnt = h->ycnt.p;
            A.ybox = h->ybox.p;
            A.poff = poff.p;
            A.pbin = pbin.p;
            A.pq = ppq.p;
            A.far_ptr = t->far_ptr.p;
            A.far_idx = t->far_idx.p;
            A.xptr = h->xptr.p;
            A.xcnt = h->xcnt.p;
            A.xbox = h->xbox.p;
            A.choff = choff.p;
            A.cbox = cbox.p;
            A.mbox = mbox.p;
            A.xqm = xqm.p;
            A.outptr = h->yptr.p;
            A.outcnt = h->ycnt.p;
            A.outbox = h->ybox.p;
            launch_members(A, pts, nl, G2, ilmax[l], s);
        } else {
            tdata.alloc(ttot > 0 ? ttot : 1, s);
            tbox.alloc((size_t)nl * 6, s);
            k_gather_down<<<nl, GD_THREADS, 0, s>>>(lb, t->parent.p, t->far_ptr.p, t->far_idx.p, h->xptr.p,
                                                    h->xcnt.p, h->yptr.p, h->ycnt.p, toff.p, tdata.p, h->xbox.p,
                                                    h->ybox.p, tbox.p);
            H2_LAUNCH("k_gather_down");
            launch_datareduct(toff.p, tdata.p, ttot, nl, h->g2, d, pts, h->yptr.p, h->ycnt.p, lb, tbox.p,
                              h->ybox.p, s, h->method);
        }
        if (il) {
            scan_exclusive(szl.p, loff.p, nl, s);
            scan_exclusive(capl.p, lcoff.p, nl, s);
            const int64_t ltot = read_scalar(loff.p + nl, s), lctot = read_scalar(lcoff.p + nl, s);
            h->iltotal += ltot;
            lbuf.alloc(lctot > 0 ? lctot : 1, s);
            lptr.alloc(nl, s);
            lcnt.alloc(nl, s);
            lobox.alloc((size_t)nl * 6, s);
            k_set_ptrs<<<blocks_for(nl, 128), 128, 0, s>>>(0, nl, lbuf.p, lcoff.p, lptr.p);
            H2_LAUNCH("k_set_ptrs");
            // outputs indexed from 0: lptr, lcnt and lobox hold this level's nodes only
            if (mem_l) {
                DMArgs B = A;
                B.outlb = 0;
                B.toff = loff.p;
                B.parent = nullptr;
                B.outptr = lptr.p;
                B.outcnt = lcnt.p;
                B.outbox = lobox.p;
                launch_members(B, pts, nl, G2, ilmax[l], s);
            } else {
                tl.alloc(ltot > 0 ? ltot : 1, s);
                lbox.alloc((size_t)nl * 6, s);
                k_gather_il<<<nl, 256, 0, s>>>(lb, t->parent.p, t->far_ptr.p, t->far_idx.p, h->ycnt.p, toff.p,
                                               tdata.p, loff.p, tl.p, h->xbox.p, lbox.p);
                H2_LAUNCH("k_gather_il");
                launch_datareduct(loff.p, tl.p, ltot, nl, h->g2, d, pts, lptr.p, lcnt.p, 0, lbox.p, lobox.p, s,
                                  h->method);
            }
            k_merge_il<<<nl, 256, merge_smem, s>>>(lb, h->yptr.p, h->ycnt.p, h->ybox.p, lptr.p, lcnt.p, lobox.p);
            H2_LAUNCH("k_merge_il");
        }
    }
    H2_CUDA(cudaEventRecord(e2, s));
    H2_CUDA(cudaEventSynchronize(e2));
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, e0, e1);
    cudaEventElapsedTime(&b, e1, e2);
    h->ms_up = a;
    h->ms_down = b;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    // per-level maxima of |X*| and |Y*| for later launch sizing, and the
    // totals of the sets as built (the buffers' capacities can be larger:
    // DataReduct deduplicates, and the interaction-list merge drops repeats)
    std::vector<int32_t> xc = read_vec(h->xcnt.p, nn, s), yc = read_vec(h->ycnt.p, nn, s);
    h->xtotal = h->ytotal = 0;
    for (int l = 0; l < t->nlevels; l++)
        for (int i = t->lptr[l]; i < t->lptr[l + 1]; i++) {
            h->xmax_level[l] = std::max(h->xmax_level[l], (int)xc[i]);
            h->ymax_level[l] = std::max(h->ymax_level[l], (int)yc[i]);
            h->xtotal += xc[i];
            h->ytotal += yc[i];
        }
}

int64_t datareduct_one(const DRPoints &pts, int d, int64_t n, int g, const long long *box_keys, int32_t *out_dev,
                       cudaStream_t s) {
    // one node whose set is the labels 0..n-1
    DevBuf<int64_t> toff;
    DevBuf<int32_t> tdata, cnt;
    DevBuf<int32_t *> optr;
    DevBuf<long long> box;
    box.alloc(12, s);  // the set's box, then the result's
    H2_CUDA(cudaMemcpyAsync(box.p, box_keys, 6 * sizeof(long long), cudaMemcpyHostToDevice, s));
    toff.alloc(2, s);
    tdata.alloc(n, s);
    cnt.alloc(1, s);
    optr.alloc(1, s);
    std::vector<int32_t> ids(n);
    for (int64_t i = 0; i < n; i++) ids[i] = (int32_t)i;
    int64_t offs[2] = {0, n};
    H2_CUDA(cudaMemcpyAsync(toff.p, offs, sizeof offs, cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaMemcpyAsync(tdata.p, ids.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaMemcpyAsync(optr.p, &out_dev, sizeof(int32_t *), cudaMemcpyHostToDevice, s));
    launch_datareduct(toff.p, tdata.p, n, 1, g, d, pts, optr.p, cnt.p, 0, box.p, box.p + 6, s);
    return read_scalar(cnt.p, s);
}

}  // namespace h2
