// matvec.cu -- the O(n) H^2 matrix-vector product (section 2.1 of
// arXiv 2206.01885) and the exact sampled rows of the section 6 error.
//
//   upward    xh_i = U_i^T x_i (leaf), xh_p = U_p^T [xh_c1; ...] (parent)
//   coupling  zh_i = sum_{j far from i} K(Xhat_i, Xhat_j) xh_j  (B_ij is a
//             kernel submatrix, evaluated on the fly)
//   downward  [zh_c1; ...] += U_p zh_p (parent), y_i = U_i zh_i (leaf)
//   near      y_i += K(X_i, X_j) x_j over near leaf pairs (on the fly)
// Vectors live in Morton order inside; x and y are permuted at the ends.
#include <mutex>

#include <cfloat>

#include "h2_internal.cuh"
#include "kappa_fast.cuh"

// Scratch of h2_exact_rows_noalloc: the right-hand side permuted to Morton
// order.  It lives in the library image, so every GPU that loads the library
// holds these H2_NOALLOC_MAX_N doubles (8 MiB) until the process exits.
#define H2_NOALLOC_MAX_N (1 << 20)
static __device__ __align__(256) double g_noalloc_zm[H2_NOALLOC_MAX_N];

namespace h2 {
namespace {

constexpr int MV_THREADS = 256;
constexpr int NB_WARPS = 8;   // warps of an N-body CTA, each taking every 8th source block

__global__ void k_perm_in(const double *x, const int32_t *perm, int64_t n, double *xm) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) xm[p] = x[perm[p]];
}

__global__ void k_to_float(const double *a, int64_t n, float *b) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) b[p] = (float)a[p];
}

// xh_i[a] = sum_r U_i[r, a] in[r]; one CTA per node, one warp per column,
// float64 accumulation (U is float64 or float32)
template <class UT>
__global__ void k_upward(int lb, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                         const int32_t *kk, const int32_t *cc, void *const *uptr, const int64_t *sk_off,
                         const double *xm, double *xh) {
    extern __shared__ double sin_[];
    int i = lb + blockIdx.x;
    int k = kk[i], c = cc[i];
    if (k == 0) return;
    const double *in = nchild[i] == 0 ? xm + begin[i] : xh + sk_off[fchild[i]];
    for (int r = threadIdx.x; r < c; r += blockDim.x) sin_[r] = in[r];
    __syncthreads();
    const UT *U = static_cast<const UT *>(uptr[i]);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = warp; a < k; a += nw) {
        const UT *col = U + (int64_t)a * c;
        double s = 0.0;
        for (int r = lane; r < c; r += 32) s += (double)col[r] * sin_[r];
        s = warp_sum(s);
        if (lane == 0) xh[sk_off[i] + a] = s;
    }
}

// out = U_i zh_i, added to the children's zh (parent) or to y (leaf)
template <class UT>
__global__ void k_downward(int lb, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                           const int32_t *kk, const int32_t *cc, void *const *uptr, const int64_t *sk_off,
                           double *zh, double *ym) {
    extern __shared__ double sz_[];
    int i = lb + blockIdx.x;
    int k = kk[i], c = cc[i];
    if (k == 0) return;
    const double *z = zh + sk_off[i];
    for (int a = threadIdx.x; a < k; a += blockDim.x) sz_[a] = z[a];
    __syncthreads();
    const UT *U = static_cast<const UT *>(uptr[i]);
    double *out = nchild[i] == 0 ? ym + begin[i] : zh + sk_off[fchild[i]];
    for (int r = threadIdx.x; r < c; r += blockDim.x) {
        double s = 0.0;
        for (int a = 0; a < k; a++) s += (double)U[r + (int64_t)a * c] * sz_[a];
        out[r] += s;
    }
}

// out[r] = sum_q kappa(x_s, x_q) z_q for s = rows[r]; one CTA per row (kpar:
// the kernel parameter as h2_kappa_param gives it)
__global__ void k_exact_rows(const int64_t *rows, int64_t nrows, const int32_t *iperm, const double *x0,
                             const double *x1, const double *x2, const double *zm, int64_t n, int d, int kid,
                             double kpar, double *out) {
    __shared__ double red[32];
    int64_t r = blockIdx.x;
    if (r >= nrows) return;
    int64_t row = rows[r];
    if (row < 0 || row >= n) {  // out-of-range row: NaN instead of an out-of-bounds read
        if (threadIdx.x == 0) out[r] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    int64_t p = iperm[row];
    double a0 = x0[p], a1 = d > 1 ? x1[p] : 0.0, a2 = d > 2 ? x2[p] : 0.0;
    double s = 0.0;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x)
        s += h2_kxy_fast(kid, kpar, a0, a1, a2, x0[q], d > 1 ? x1[q] : 0.0, d > 2 ? x2[q] : 0.0) * zm[q];
    s = warp_sum(s);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        out[r] = t;
    }
}

// Chunked form of k_exact_rows: CTA (r, c) sums chunk c (ER_CHUNK points) of
// row r into part[r * nch + c]; k_exact_sum adds a row's chunks in order.
// Short CTAs let other streams' kernels take SMs as they retire.
constexpr int ER_CHUNK = 1 << 14;
constexpr int ER_THREADS = 256;

__global__ void __launch_bounds__(ER_THREADS)
    k_exact_part(const int64_t *rows, int64_t nrows, const int32_t *iperm, const double *x0, const double *x1,
                 const double *x2, const double *zm, int64_t n, int d, int kid, double kpar, int nch, double *part) {
    __shared__ double red[ER_THREADS / 32];
    const int64_t r = blockIdx.y;
    const int c = blockIdx.x;
    const int64_t row = rows[r];
    if (row < 0 || row >= n) {  // out-of-range row: NaN instead of an out-of-bounds read
        if (threadIdx.x == 0) part[r * nch + c] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const int64_t p = iperm[row];
    const double a0 = x0[p], a1 = d > 1 ? x1[p] : 0.0, a2 = d > 2 ? x2[p] : 0.0;
    const int64_t q0 = (int64_t)c * ER_CHUNK, q1 = min(n, q0 + ER_CHUNK);
    double s = 0.0;
    for (int64_t q = q0 + threadIdx.x; q < q1; q += ER_THREADS)
        s += h2_kxy_fast(kid, kpar, a0, a1, a2, x0[q], d > 1 ? x1[q] : 0.0, d > 2 ? x2[q] : 0.0) * zm[q];
    s = warp_sum(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < ER_THREADS / 32; w++) t += red[w];
        part[r * nch + c] = t;
    }
}

__global__ void k_exact_sum(const double *part, int64_t nrows, int nch, double *out) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    double t = 0.0;
    for (int c = 0; c < nch; c++) t += part[r * nch + c];
    out[r] = t;
}

// err = ||exact - approx[rows]|| / ||exact||, one CTA, fixed reduction order
__global__ void k_sampled_error(const double *exact, const double *approx, const int64_t *rows, int64_t nrows,
                                int64_t n, double *err) {
    __shared__ double red[2][32];
    double sn = 0.0, sd = 0.0;
    for (int64_t r = threadIdx.x; r < nrows; r += blockDim.x) {
        int64_t row = rows[r];
        double a = (row >= 0 && row < n) ? approx[row] : __longlong_as_double(0x7ff8000000000000ll);
        double e = exact[r] - a;
        sn += e * e;
        sd += exact[r] * exact[r];
    }
    sn = warp_sum(sn);
    sd = warp_sum(sd);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = sn; red[1][warp] = sd; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tn = 0.0, td = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { tn += red[0][w]; td += red[1][w]; }
        *err = td > 0.0 ? sqrt(tn / td) : sqrt(tn);
    }
}

// (node, first target) tiles for every node with targets and a non-empty list
void build_tiles(const std::vector<int32_t> &cnt, const std::vector<int64_t> &lptr, int per_tile,
                 DevBuf<int2> &tiles, cudaStream_t s) {
    std::vector<int2> v;
    for (size_t i = 0; i < cnt.size(); i++) {
        if (cnt[i] <= 0 || lptr[i + 1] == lptr[i]) continue;
        for (int a = 0; a < cnt[i]; a += per_tile) v.push_back(make_int2((int)i, a));
    }
    tiles.alloc(std::max<size_t>(v.size(), 1), s);
    if (!v.empty()) H2_CUDA(cudaMemcpyAsync(tiles.p, v.data(), v.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaStreamSynchronize(s));
    tiles.n = v.size();
}

// ------------------------------------------------------------ several RHS
// Inside, R right-hand sides are stored point-major: entry (p, j) at p*R + j.

template <class T>
__global__ void k_perm_in_multi(const T *x, int64_t ld, const int32_t *perm, int64_t n, int R, double *xm) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    int64_t p = t / R;
    int j = (int)(t - p * R);
    xm[t] = (double)x[perm[p] + j * ld];
}

template <class T>
__global__ void k_perm_out_multi(const double *ym, const int32_t *perm, int64_t n, int R, T *y, int64_t ld) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    int64_t p = t / R;
    int j = (int)(t - p * R);
    y[perm[p] + j * ld] = (T)ym[t];
}

// xh_i[a, j] = sum_r U_i[r, a] in[r, j]; one CTA per node, a thread per (a, j)
template <class UT>
__global__ void k_upward_multi(int lb, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                               const int32_t *kk, const int32_t *cc, void *const *uptr, const int64_t *sk_off,
                               const double *xm, double *xh, int R) {
    const int i = lb + blockIdx.x;
    const int k = kk[i], c = cc[i];
    if (k == 0) return;
    const double *in = nchild[i] == 0 ? xm + (int64_t)begin[i] * R : xh + sk_off[fchild[i]] * R;
    const UT *U = static_cast<const UT *>(uptr[i]);
    double *o = xh + sk_off[i] * R;
    for (int t = threadIdx.x; t < k * R; t += blockDim.x) {
        const int a = t / R, j = t - a * R;
        const UT *col = U + (int64_t)a * c;
        double s = 0.0;
        for (int r = 0; r < c; r++) s += (double)col[r] * in[(int64_t)r * R + j];
        o[t] = s;
    }
}

// out[r, j] += sum_a U_i[r, a] zh_i[a, j], into the children's zh (parent) or y (leaf)
template <class UT>
__global__ void k_downward_multi(int lb, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                                 const int32_t *kk, const int32_t *cc, void *const *uptr, const int64_t *sk_off,
                                 double *zh, double *ym, int R) {
    const int i = lb + blockIdx.x;
    const int k = kk[i], c = cc[i];
    if (k == 0) return;
    const double *z = zh + sk_off[i] * R;
    const UT *U = static_cast<const UT *>(uptr[i]);
    double *out = nchild[i] == 0 ? ym + (int64_t)begin[i] * R : zh + sk_off[fchild[i]] * R;
    for (int t = threadIdx.x; t < c * R; t += blockDim.x) {
        const int r = t / R, j = t - r * R;
        double s = 0.0;
        for (int a = 0; a < k; a++) s += (double)U[r + (int64_t)a * c] * z[(int64_t)a * R + j];
        out[t] += s;
    }
}

// Error-free sum of a + b (Knuth's TwoSum); the rounding error goes into e.
__device__ __forceinline__ void two_sum_acc(float &a, float &e, float b) {
    const float s = a + b, bp = s - a;
    e += (a - (s - bp)) + (b - bp);
    a = s;
}

// Tiled N-body accumulation for R right-hand sides at once:
//   out[t, j] += sum_s kappa(x_t, x_s) w[s, j]
// (w and out with row strides ws and os).  The point set of node i is
// [start[i], start[i] + count[i]) of the coordinate arrays.  One CTA takes a
// tile of 32 * TPT targets of node i (TPT per lane); its warps split the source
// blocks j of the list lidx[lptr[i] .. lptr[i+1]), and each warp stages 32
// source points at a time (coordinates and R weights) in shared memory, read
// back as broadcasts, so one kernel evaluation feeds R fused multiply-adds.
// Real = double: absolute float64 coordinates, float64 sums.  Real = float:
// coordinates relative to each node's cell centre, the centre offset added per
// block pair from the centres' float32 {hi, lo} splits, each block's float32
// sums folded into compensated float32 accumulators.
template <class Real, int KID, int R, int TPT>
__global__ void __launch_bounds__(NB_WARPS * 32)
    k_nbody(const int2 *tiles, const int64_t *start, const int32_t *count, const Real *X0, const Real *X1,
            const Real *X2, const float2 *F0, const float2 *F1, const float2 *F2, const Real *w, int ws, double *out,
            int os, const int64_t *lptr, const int32_t *lidx, int d, double kpar) {
    constexpr int RW = (int)((((4 + R) * sizeof(Real) + 15) / 16 * 16) / sizeof(Real));
    constexpr size_t STG = sizeof(Real) * NB_WARPS * 32 * RW, PART = sizeof(double) * NB_WARPS * 32 * TPT * R;
    __shared__ __align__(16) unsigned char sraw[STG > PART ? STG : PART];
    Real(*stg)[32][RW] = reinterpret_cast<Real(*)[32][RW]>(sraw);
    double(*part)[32 * TPT][R] = reinterpret_cast<double(*)[32 * TPT][R]>(sraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 tl = tiles[blockIdx.x];
    const int i = tl.x;
    const int64_t ts = start[i];
    const int tn = count[i];
    const Real p = (Real)kpar;
    Real tx[TPT][3], acc[TPT][R], cmp[TPT][R];
#pragma unroll
    for (int u = 0; u < TPT; u++) {
        const int a = tl.y + u * 32 + lane;
        const bool ok = a < tn;
        tx[u][0] = ok ? X0[ts + a] : (Real)0;
        tx[u][1] = ok && d > 1 ? X1[ts + a] : (Real)0;
        tx[u][2] = ok && d > 2 ? X2[ts + a] : (Real)0;
#pragma unroll
        for (int j = 0; j < R; j++) { acc[u][j] = (Real)0; cmp[u][j] = (Real)0; }
    }
    for (int64_t e = lptr[i] + warp; e < lptr[i + 1]; e += NB_WARPS) {
        const int jn = lidx[e];
        const int64_t ss = start[jn];
        const int sn = count[jn];
        Real o0 = (Real)0, o1 = (Real)0, o2 = (Real)0;
        if constexpr (sizeof(Real) == 4) {  // target coordinates in node jn's frame
            const float2 a0 = F0[i], b0 = F0[jn];
            o0 = (a0.x - b0.x) + (a0.y - b0.y);
            if (d > 1) {
                const float2 a1 = F1[i], b1 = F1[jn];
                o1 = (a1.x - b1.x) + (a1.y - b1.y);
            }
            if (d > 2) {
                const float2 a2 = F2[i], b2 = F2[jn];
                o2 = (a2.x - b2.x) + (a2.y - b2.y);
            }
        }
        Real sh[TPT][3], blk[TPT][R];
#pragma unroll
        for (int u = 0; u < TPT; u++) {
            sh[u][0] = tx[u][0] + o0;
            sh[u][1] = tx[u][1] + o1;
            sh[u][2] = tx[u][2] + o2;
#pragma unroll
            for (int j = 0; j < R; j++) blk[u][j] = (Real)0;
        }
        for (int q0 = 0; q0 < sn; q0 += 32) {
            const int cnt = min(32, sn - q0);
            __syncwarp();
            if (lane < cnt) {
                const int64_t sp = ss + q0 + lane;
                stg[warp][lane][0] = X0[sp];
                stg[warp][lane][1] = d > 1 ? X1[sp] : (Real)0;
                stg[warp][lane][2] = d > 2 ? X2[sp] : (Real)0;
            }
            for (int e2 = lane; e2 < cnt * R; e2 += 32) {
                const int r = e2 / R, c = e2 - r * R;
                stg[warp][r][4 + c] = w[(ss + q0 + r) * (int64_t)ws + c];
            }
            __syncwarp();
            for (int q = 0; q < cnt; q++) {
                const Real *row = stg[warp][q];
                const Real a0 = row[0], a1 = row[1], a2 = row[2];
#pragma unroll
                for (int u = 0; u < TPT; u++) {
                    const Real kv = kap_pt<KID, false>(sh[u][0], sh[u][1], sh[u][2], a0, a1, a2, p);
#pragma unroll
                    for (int j = 0; j < R; j++) blk[u][j] += kv * row[4 + j];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < TPT; u++)
#pragma unroll
            for (int j = 0; j < R; j++) {
                if constexpr (sizeof(Real) == 8) acc[u][j] += blk[u][j];
                else two_sum_acc(acc[u][j], cmp[u][j], blk[u][j]);
            }
    }
    __syncthreads();  // every warp is done with its staging area before it becomes part[]
#pragma unroll
    for (int u = 0; u < TPT; u++)
#pragma unroll
        for (int j = 0; j < R; j++) part[warp][u * 32 + lane][j] = (double)acc[u][j] + (double)cmp[u][j];
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * TPT * R; t += blockDim.x) {
        const int l = t / R, j = t - l * R;
        const int aa = tl.y + l;
        if (aa < tn) {
            double sum = 0.0;
            for (int wv = 0; wv < NB_WARPS; wv++) sum += part[wv][l][j];
            out[(ts + aa) * (int64_t)os + j] += sum;
        }
    }
}

// Symmetric tiled N-body for one right-hand side.  kappa is symmetric, so the
// list of node i is walked only from its first entry j >= i: a pair j > i is
// evaluated once for both out_i += K(X_i, X_j) w_j and out_j += K(X_j, X_i) w_i,
// and j == i (a leaf's own block) gives the first term only.  A CTA takes a
// tile of 32 targets of i (one a lane), its warps split the pairs; sources
// are staged 32 at a time and at step q lane l evaluates source (l + q) mod 32,
// so every lane meets every staged source once.  The row sum stays in the
// lane; the column sum of source (l + q) mod 32 rides in lane l and moves one
// lane down after each step, so after 32 steps lane l holds source l's column
// sum.  Row sums (per CTA) and column sums (per warp and 32 sources) are
// added to out with float64 atomics: other CTAs add to the same entries.
// Padding is skipped where it would dominate: a block's short last chunk of
// sources is read by broadcast with one warp sum per source's column, and a
// node's short last tile of targets runs with lanes over the sources and the
// targets broadcast by shuffles (see the thresholds below).

// a staged source point: coordinates and weight in one 16-byte (float) or
// 32-byte (double) record, one shared-memory load per evaluation
template <class Real>
struct alignas(4 * sizeof(Real)) SrcPt {
    Real x, y, z, w;
};

template <class Real, int KID>
__global__ void __launch_bounds__(NB_WARPS * 32)
    k_nbody_sym(const int2 *tiles, const int64_t *start, const int32_t *count, const Real *X0, const Real *X1,
                const Real *X2, const float2 *F0, const float2 *F1, const float2 *F2, const Real *w, double *out,
                const int64_t *lptr, const int64_t *lfirst, const int32_t *lidx, int d, double kpar) {
    // staged sources of each warp, stored twice (s and s + 32) so that lane l
    // reads source (l + q) mod 32 at a fixed base plus q
    __shared__ SrcPt<Real> stg[NB_WARPS][64];
    __shared__ double part[NB_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 tl = tiles[blockIdx.x];
    const int i = tl.x;
    const int64_t ts = start[i];
    const int tn = count[i];
    const int a = tl.y + lane;
    const bool act = a < tn;
    const Real p = (Real)kpar;
    // lanes past the tile's end and sources past a block's end sit at far,
    // distinct sentinels with weight 0: every pair evaluated below has r2 > 0
    // and contributes exactly 0 when either side is padding (cos(x . y) needs
    // no distinct points: its padding sits at the origin)
    const Real far_t = KID == H2_K_COSDOT ? (Real)0 : (Real)1e18;
    const Real tx0 = act ? X0[ts + a] : far_t, tx1 = act && d > 1 ? X1[ts + a] : (Real)0,
               tx2 = act && d > 2 ? X2[ts + a] : (Real)0;
    const Real tw = act ? w[ts + a] : (Real)0;
    // a short tile (the last of a node, e.g. 11 of a 43-point skeleton) turns
    // the roles around: lanes take sources, targets are broadcast, so no lane
    // evaluates a padding target (cheaper than the rotation up to about 24
    // targets in float64, 12 in float32)
    const int tcount = min(32, tn - tl.y);
    constexpr int SHORT_T = sizeof(Real) == 8 ? 24 : 12;
    const bool short_tile = tcount <= SHORT_T;
    Real acc = (Real)0, cmp = (Real)0;
    for (int64_t e = lfirst[i] + warp; e < lptr[i + 1]; e += NB_WARPS) {
        const int jn = lidx[e];
        const bool sym = jn != i;
        const int64_t ss = start[jn];
        const int sn = count[jn];
        Real s0 = tx0, s1 = tx1, s2 = tx2;
        if constexpr (sizeof(Real) == 4) {  // target coordinates in node jn's frame
            const float2 a0 = F0[i], b0 = F0[jn];
            s0 += (a0.x - b0.x) + (a0.y - b0.y);
            if (d > 1) {
                const float2 a1 = F1[i], b1 = F1[jn];
                s1 += (a1.x - b1.x) + (a1.y - b1.y);
            }
            if (d > 2) {
                const float2 a2 = F2[i], b2 = F2[jn];
                s2 += (a2.x - b2.x) + (a2.y - b2.y);
            }
        }
        Real blk = (Real)0;
        for (int q0 = 0; q0 < sn; q0 += 32) {
            const int cnt = min(32, sn - q0);
            __syncwarp();
            {  // sources past the end: a far sentinel with weight 0 (their terms vanish)
                const bool ok = lane < cnt;
                const int64_t sp = ss + q0 + lane;
                SrcPt<Real> v;
                v.x = ok ? X0[sp] : -far_t;
                v.y = ok && d > 1 ? X1[sp] : (Real)0;
                v.z = ok && d > 2 ? X2[sp] : (Real)0;
                v.w = ok ? w[sp] : (Real)0;
                stg[warp][lane] = v;
                stg[warp][lane + 32] = v;
            }
            __syncwarp();
            Real col = (Real)0;
            // a short last chunk skips the rotation's padding steps: its cnt
            // sources are read as broadcasts and each one's column sum is
            // reduced across the warp (cheaper than 32 rotation steps up to
            // about 24 sources in float64, 16 in float32)
            constexpr int ROT_MIN = sizeof(Real) == 8 ? 24 : 16;
            if (sym && short_tile) {
                const SrcPt<Real> sv = stg[warp][lane];  // (lanes past cnt: the weight-0 sentinel)
                for (int t = 0; t < tcount; t++) {      // (tcount is the same in every lane)
                    const Real a0 = __shfl_sync(0xffffffffu, s0, t), a1 = __shfl_sync(0xffffffffu, s1, t),
                               a2 = __shfl_sync(0xffffffffu, s2, t), aw = __shfl_sync(0xffffffffu, tw, t);
                    const Real kv = kap_pt<KID, true>(a0, a1, a2, sv.x, sv.y, sv.z, p);
                    col += kv * aw;
                    const Real r = warp_sum(kv * sv.w);
                    if (lane == t) blk += r;
                }
                if (lane < cnt) atomicAdd(out + ss + q0 + lane, (double)col);
            } else if (sym && cnt > ROT_MIN) {
                const SrcPt<Real> *row = &stg[warp][lane];
#pragma unroll 8
                for (int q = 0; q < 32; q++) {
                    const SrcPt<Real> sv = row[q];
                    const Real kv = kap_pt<KID, true>(s0, s1, s2, sv.x, sv.y, sv.z, p);
                    blk += kv * sv.w;
                    col += kv * tw;
                    col = __shfl_sync(0xffffffffu, col, (lane + 1) & 31);
                }
                if (lane < cnt) atomicAdd(out + ss + q0 + lane, (double)col);
            } else if (sym) {
                for (int q = 0; q < cnt; q++) {  // (cnt is the same in every lane)
                    const SrcPt<Real> sv = stg[warp][q];
                    const Real kv = kap_pt<KID, true>(s0, s1, s2, sv.x, sv.y, sv.z, p);
                    blk += kv * sv.w;
                    const Real c = warp_sum(kv * tw);
                    if (lane == 0) atomicAdd(out + ss + q0 + q, (double)c);
                }
            } else {
                for (int q = 0; q < cnt; q++) {
                    const SrcPt<Real> sv = stg[warp][q];
                    blk += kap_pt<KID, false>(s0, s1, s2, sv.x, sv.y, sv.z, p) * sv.w;
                }
            }
        }
        if constexpr (sizeof(Real) == 8) acc += blk;
        else two_sum_acc(acc, cmp, blk);
    }
    part[warp][lane] = (double)acc + (double)cmp;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int aa = tl.y + threadIdx.x;
        if (aa < tn) {
            double sum = 0.0;
            for (int wv = 0; wv < NB_WARPS; wv++) sum += part[wv][threadIdx.x];
            atomicAdd(out + ts + aa, sum);
        }
    }
}

// first entry of each node's (sorted) list whose index is >= the node's own
__global__ void k_list_first(const int64_t *ptr, const int32_t *idx, int nn, int64_t *first) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int64_t lo = ptr[i], hi = ptr[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (idx[mid] < i) lo = mid + 1;
        else hi = mid;
    }
    first[i] = lo;
}

template <class Real>
void nbody_sym(int kid, const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count, const Real *X0,
               const Real *X1, const Real *X2, const float2 *F0, const float2 *F1, const float2 *F2, const Real *w,
               double *out, const int64_t *lptr, const int64_t *lfirst, const int32_t *lidx, int d, double kp0,
               cudaStream_t s) {
    if (tiles.n == 0) return;
    const unsigned nb = (unsigned)tiles.n;
    const double p = kap_param(kid, kp0);
#define H2_SYM(K)                                                                                                  \
    k_nbody_sym<Real, K><<<nb, NB_WARPS * 32, 0, s>>>(tiles.p, start, count, X0, X1, X2, F0, F1, F2, w, out, lptr, \
                                                      lfirst, lidx, d, p)
    switch (kid) {
    case H2_K_COULOMB: H2_SYM(H2_K_COULOMB); break;
    case H2_K_GAUSSIAN: H2_SYM(H2_K_GAUSSIAN); break;
    case H2_K_EXPONENTIAL: H2_SYM(H2_K_EXPONENTIAL); break;
    case H2_K_BUMP: H2_SYM(H2_K_BUMP); break;
    case H2_K_POWER: H2_SYM(H2_K_POWER); break;
    case H2_K_COSDOT: H2_SYM(H2_K_COSDOT); break;
    default: H2_SYM(H2_K_MULTIQUADRIC);
    }
#undef H2_SYM
    H2_LAUNCH("k_nbody_sym");
}

template <class Real, int R, int TPT>
void nbody_kid(int kid, const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count, const Real *X0,
               const Real *X1, const Real *X2, const float2 *F0, const float2 *F1, const float2 *F2, const Real *w,
               int ws, double *out, int os, const int64_t *lptr, const int32_t *lidx, int d, double kp0,
               cudaStream_t s) {
    const unsigned nb = (unsigned)tiles.n;
    const double p = kap_param(kid, kp0);
#define H2_NB(K)                                                                                                   \
    k_nbody<Real, K, R, TPT><<<nb, NB_WARPS * 32, 0, s>>>(tiles.p, start, count, X0, X1, X2, F0, F1, F2, w, ws, out, \
                                                          os, lptr, lidx, d, p)
    switch (kid) {
    case H2_K_COULOMB: H2_NB(H2_K_COULOMB); break;
    case H2_K_GAUSSIAN: H2_NB(H2_K_GAUSSIAN); break;
    case H2_K_EXPONENTIAL: H2_NB(H2_K_EXPONENTIAL); break;
    case H2_K_BUMP: H2_NB(H2_K_BUMP); break;
    case H2_K_POWER: H2_NB(H2_K_POWER); break;
    case H2_K_COSDOT: H2_NB(H2_K_COSDOT); break;
    default: H2_NB(H2_K_MULTIQUADRIC);
    }
#undef H2_NB
    H2_LAUNCH("k_nbody");
}

// all nrhs columns, in launches of 16, 8, 4, 2 and 1 columns; tiles hold 32
// targets (one a lane: skeletons of a few dozen points fill whole tiles)
template <class Real>
void nbody(int kid, const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count, const Real *X0,
           const Real *X1, const Real *X2, const float2 *F0, const float2 *F1, const float2 *F2, const Real *w,
           double *out, int nrhs, const int64_t *lptr, const int32_t *lidx, int d, double kp0, cudaStream_t s,
           int cbegin = 0) {
    if (tiles.n == 0) return;
    for (int c0 = cbegin; c0 < nrhs;) {
        const int left = nrhs - c0;
        const Real *wc = w + c0;
        double *oc = out + c0;
        if (left >= 16) {
            nbody_kid<Real, 16, 1>(kid, tiles, start, count, X0, X1, X2, F0, F1, F2, wc, nrhs, oc, nrhs, lptr, lidx,
                                   d, kp0, s);
            c0 += 16;
        } else if (left >= 8) {
            nbody_kid<Real, 8, 1>(kid, tiles, start, count, X0, X1, X2, F0, F1, F2, wc, nrhs, oc, nrhs, lptr, lidx, d,
                                  kp0, s);
            c0 += 8;
        } else if (left >= 4) {
            nbody_kid<Real, 4, 1>(kid, tiles, start, count, X0, X1, X2, F0, F1, F2, wc, nrhs, oc, nrhs, lptr, lidx, d,
                                  kp0, s);
            c0 += 4;
        } else if (left >= 2) {
            nbody_kid<Real, 2, 1>(kid, tiles, start, count, X0, X1, X2, F0, F1, F2, wc, nrhs, oc, nrhs, lptr, lidx, d,
                                  kp0, s);
            c0 += 2;
        } else {
            nbody_kid<Real, 1, 1>(kid, tiles, start, count, X0, X1, X2, F0, F1, F2, wc, nrhs, oc, nrhs, lptr, lidx, d,
                                  kp0, s);
            c0 += 1;
        }
    }
}

// tiles of 128 targets of every leaf with a near list (the tensor-core
// nearfield), and its timeout flag, built on first use
void prepare_tc_tiles(h2_tree_s *t, cudaStream_t s) {
    if (t->near_tiles_tc_ready) return;
    const int nn = t->nnodes;
    std::vector<int32_t> b = read_vec(t->begin.p, nn, s), e = read_vec(t->end.p, nn, s),
                         nc = read_vec(t->nchild.p, nn, s);
    std::vector<int64_t> np = read_vec(t->near_ptr.p, nn + 1, s);
    std::vector<int32_t> cnt(nn);
    for (int i = 0; i < nn; i++) cnt[i] = nc[i] == 0 ? e[i] - b[i] : 0;
    DevBuf<int> st;
    st.alloc(1, s);
    H2_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), s));
    build_tiles(cnt, np, 128, t->near_tiles_tc, s);
    t->tc_status = std::move(st);
    t->near_tiles_tc_ready = true;
}

// the upward/downward kernels' shared-memory opt-in, once per process
void set_matvec_attrs() {
    static std::once_flag attr;
    std::call_once(attr, [] {
        for (auto f : {(const void *)k_upward<double>, (const void *)k_upward<float>, (const void *)k_downward<double>,
                       (const void *)k_downward<float>})
            H2_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    });
}

// tiles of the coupling (per matrix) and nearfield (per tree) kernels for
// 32 * tpt targets a tile, built on first use and rebuilt when tpt changes
void prepare_tiles(h2_matrix_s *A, int tpt, cudaStream_t s) {
    h2_tree_s *t = A->tree;
    const int nn = t->nnodes;
    if (A->far_tile_tpt != tpt) {
        A->far_tile_tpt = 0;  // set again only once the tiles exist
        std::vector<int32_t> kh = read_vec(A->k.p, nn, s);
        std::vector<int64_t> fp = read_vec(t->far_ptr.p, nn + 1, s);
        build_tiles(kh, fp, 32 * tpt, A->far_tiles, s);
        A->far_tile_tpt = tpt;
    }
    if (t->near_tile_tpt != tpt) {
        t->near_tile_tpt = 0;
        std::vector<int32_t> b = read_vec(t->begin.p, nn, s), e = read_vec(t->end.p, nn, s),
                             nc = read_vec(t->nchild.p, nn, s);
        std::vector<int64_t> np = read_vec(t->near_ptr.p, nn + 1, s);
        std::vector<int32_t> cnt(nn);
        for (int i = 0; i < nn; i++) cnt[i] = nc[i] == 0 ? e[i] - b[i] : 0;
        if (!t->leaf_start.p || !t->leaf_count.p) {  // int64 starts of every node's points (nearfield point sets)
            std::vector<int64_t> st(b.begin(), b.end());
            std::vector<int32_t> ct(nn);
            for (int i = 0; i < nn; i++) ct[i] = e[i] - b[i];
            DevBuf<int64_t> ls;
            DevBuf<int32_t> lc;
            ls.alloc(nn, s);
            lc.alloc(nn, s);
            H2_CUDA(cudaMemcpyAsync(ls.p, st.data(), nn * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            H2_CUDA(cudaMemcpyAsync(lc.p, ct.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            H2_CUDA(cudaStreamSynchronize(s));
            t->leaf_start = std::move(ls);
            t->leaf_count = std::move(lc);
        }
        build_tiles(cnt, np, 32 * tpt, t->near_tiles, s);
        t->near_tile_tpt = tpt;  // last: a failure above leaves the tiles to be rebuilt
    }
}

}  // namespace

void matvec_impl(h2_matrix_s *A, const double *x, double *y, cudaStream_t s) {
    matvec_multi_impl(A, x, y, 1, H2_DTYPE_F64, A->tree->n, s);
}

void matvec_multi_impl(h2_matrix_s *A, const void *x, void *y, int R, int dtype, int64_t ld, cudaStream_t s) {
    h2_tree_s *t = A->tree;
    const int d = t->d;
    const int64_t n = t->n, nr = n * R;
    const bool f64 = A->prec == H2_PREC_FP64;
    if (R == 1) {  // one column: the single-CTA shared-memory upward and downward kernels
        set_matvec_attrs();
        for (int l = 1; l < t->nlevels; l++)
            if ((size_t)A->cmax_level[l] * sizeof(double) > 200 * 1024)
                fail(H2_ERR_UNIMPLEMENTED, "candidate set too large for the single-CTA upward pass");
    }
    prepare_tiles(A, 1, s);
    // one right-hand side: each unordered block pair is evaluated once
    const bool sym = R == 1;
    if (sym && (!t->near_first.p || !t->far_first.p)) {
        const int nn = t->nnodes;
        DevBuf<int64_t> nf, ff;  // both exist before either is kept
        nf.alloc(nn, s);
        ff.alloc(nn, s);
        k_list_first<<<blocks_for(nn, 256), 256, 0, s>>>(t->near_ptr.p, t->near_idx.p, nn, nf.p);
        k_list_first<<<blocks_for(nn, 256), 256, 0, s>>>(t->far_ptr.p, t->far_idx.p, nn, ff.p);
        note_launches(1);  // (two launches above)
        H2_LAUNCH("k_list_first");
        t->near_first = std::move(nf);
        t->far_first = std::move(ff);
    }
    const int64_t kt = std::max<int64_t>(A->ktotal, 1);
    DevBuf<double> xm, ym, xh, zh;
    xm.alloc(nr, s);
    ym.alloc(nr, s);
    xh.alloc(kt * R, s);
    zh.alloc(kt * R, s);
    H2_CUDA(cudaMemsetAsync(ym.p, 0, nr * sizeof(double), s));
    H2_CUDA(cudaMemsetAsync(zh.p, 0, kt * R * sizeof(double), s));
    if (dtype == H2_DTYPE_F64)
        k_perm_in_multi<double><<<blocks_for(nr, 256), 256, 0, s>>>(static_cast<const double *>(x), ld, t->perm.p,
                                                                     n, R, xm.p);
    else
        k_perm_in_multi<float><<<blocks_for(nr, 256), 256, 0, s>>>(static_cast<const float *>(x), ld, t->perm.p, n,
                                                                    R, xm.p);
    H2_LAUNCH("k_perm_in_multi");
    // upward, deepest level first
    for (int l = t->nlevels - 1; l >= 1; l--) {
        int lb = t->lptr[l], nl = t->lptr[l + 1] - lb;
        if (A->kmax_level[l] == 0) continue;
        ProfScope ps(KT_UPWARD, s);
        if (R == 1) {
            size_t sm = (size_t)A->cmax_level[l] * sizeof(double);
            if (f64)
                k_upward<double><<<nl, MV_THREADS, sm, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p, A->c.p,
                                                            A->uptr.p, A->sk_off.p, xm.p, xh.p);
            else
                k_upward<float><<<nl, MV_THREADS, sm, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p, A->c.p,
                                                           A->uptr.p, A->sk_off.p, xm.p, xh.p);
        } else if (f64) {
            k_upward_multi<double><<<nl, MV_THREADS, 0, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p,
                                                             A->c.p, A->uptr.p, A->sk_off.p, xm.p, xh.p, R);
        } else {
            k_upward_multi<float><<<nl, MV_THREADS, 0, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p, A->c.p,
                                                            A->uptr.p, A->sk_off.p, xm.p, xh.p, R);
        }
        H2_LAUNCH("k_upward");
    }
    // float-pair copies of the weights for the float64 form's float-float
    // Coulomb products (3D, one right-hand side, blocks not stored)
    const bool df = f64 && sym && !A->stored && !A->fp64_products && A->kid == H2_K_COULOMB && d == 3;
    DevBuf<float2> xm2, xh2;
    if (df) {
        ensure_df_matrix(A, s);
        xm2.alloc(n, s);
        xh2.alloc(kt, s);
        split_vector(xm.p, n, xm2.p, s);
        split_vector(xh.p, kt, xh2.p, s);
    }
    // float32 copies of the weights for the float32 N-body kernels
    DevBuf<float> xmf, xhf;
    if (!f64) {
        xmf.alloc(nr, s);
        xhf.alloc(kt * R, s);
        k_to_float<<<blocks_for(nr, 256), 256, 0, s>>>(xm.p, nr, xmf.p);
        k_to_float<<<blocks_for(kt * R, 256), 256, 0, s>>>(xh.p, kt * R, xhf.p);
        note_launches(1);
        H2_LAUNCH("k_to_float");
    }
    // float32 point coordinates and centre splits of the N-body kernels: the
    // tree's node-relative ones, or for cos(x . y) absolute coordinates and
    // zero centres (the skeletons' are absolute already)
    const float *PX[3] = {t->xr[0].p, t->xr[1].p, t->xr[2].p};
    const float2 *CF[3] = {t->cenf[0].p, t->cenf[1].p, t->cenf[2].p};
    DevBuf<float> xabs[3];
    DevBuf<float2> czero;
    if (!f64 && A->kid == H2_K_COSDOT) {
        for (int k = 0; k < d; k++) {
            xabs[k].alloc(n, s);
            k_to_float<<<blocks_for(n, 256), 256, 0, s>>>(t->xs[k].p, n, xabs[k].p);
            PX[k] = xabs[k].p;
        }
        note_launches(d - 1);
        H2_LAUNCH("k_to_float");
        czero.alloc(t->nnodes, s);
        H2_CUDA(cudaMemsetAsync(czero.p, 0, t->nnodes * sizeof(float2), s));
        CF[0] = CF[1] = CF[2] = czero.p;
    }
    // coupling over far pairs: B_ij = K(Xhat_i, Xhat_j), stored or on the fly
    const bool st = sym && A->stored;
    if (st) {
        ProfScope ps(KT_COUPLING_ST, s);
        if (f64)
            stored_product<double>(A->far_tiles, A->sk_off.p, A->k.p, A->far_blk.p, A->far_boff.p, xh.p, zh.p,
                                   t->far_ptr.p, t->far_first.p, t->far_idx.p, s);
        else
            stored_product<float>(A->far_tiles, A->sk_off.p, A->k.p, A->far_blk.p, A->far_boff.p, xhf.p, zh.p,
                                  t->far_ptr.p, t->far_first.p, t->far_idx.p, s);
    } else {
        ProfScope ps(KT_COUPLING, s);
        if (df)
            nbody_sym_df(t, A->far_tiles, A->sk_off.p, A->k.p, A->skdf, xh2.p, zh.p, t->far_ptr.p, t->far_first.p,
                         t->far_idx.p, s);
        else if (sym && f64)
            nbody_sym<double>(A->kid, A->far_tiles, A->sk_off.p, A->k.p, A->skc[0].p, A->skc[1].p, A->skc[2].p,
                              nullptr, nullptr, nullptr, xh.p, zh.p, t->far_ptr.p, t->far_first.p, t->far_idx.p, d,
                              A->kp[0], s);
        else if (sym)
            nbody_sym<float>(A->kid, A->far_tiles, A->sk_off.p, A->k.p, A->skr[0].p, A->skr[1].p, A->skr[2].p, CF[0],
                             CF[1], CF[2], xhf.p, zh.p, t->far_ptr.p, t->far_first.p, t->far_idx.p, d, A->kp[0], s);
        else if (f64)
            nbody<double>(A->kid, A->far_tiles, A->sk_off.p, A->k.p, A->skc[0].p, A->skc[1].p, A->skc[2].p, nullptr,
                          nullptr, nullptr, xh.p, zh.p, R, t->far_ptr.p, t->far_idx.p, d, A->kp[0], s);
        else
            nbody<float>(A->kid, A->far_tiles, A->sk_off.p, A->k.p, A->skr[0].p, A->skr[1].p, A->skr[2].p, CF[0],
                         CF[1], CF[2], xhf.p, zh.p, R, t->far_ptr.p, t->far_idx.p, d, A->kp[0], s);
    }
    // downward, level 1 first
    for (int l = 1; l < t->nlevels; l++) {
        int lb = t->lptr[l], nl = t->lptr[l + 1] - lb;
        if (A->kmax_level[l] == 0) continue;
        ProfScope ps(KT_DOWNWARD, s);
        if (R == 1) {
            size_t sm = (size_t)A->kmax_level[l] * sizeof(double);
            if (f64)
                k_downward<double><<<nl, MV_THREADS, sm, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p,
                                                              A->c.p, A->uptr.p, A->sk_off.p, zh.p, ym.p);
            else
                k_downward<float><<<nl, MV_THREADS, sm, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p,
                                                             A->c.p, A->uptr.p, A->sk_off.p, zh.p, ym.p);
        } else if (f64) {
            k_downward_multi<double><<<nl, MV_THREADS, 0, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p,
                                                               A->c.p, A->uptr.p, A->sk_off.p, zh.p, ym.p, R);
        } else {
            k_downward_multi<float><<<nl, MV_THREADS, 0, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p,
                                                              A->c.p, A->uptr.p, A->sk_off.p, zh.p, ym.p, R);
        }
        H2_LAUNCH("k_downward");
    }
    // nearfield over near leaf pairs: K(X_i, X_j), stored or on the fly
    if (st) {
        ProfScope ps(KT_NEAR_ST, s);
        if (f64)
            stored_product<double>(t->near_tiles, t->leaf_start.p, t->leaf_count.p, A->near_blk.p, A->near_boff.p,
                                   xm.p, ym.p, t->near_ptr.p, t->near_first.p, t->near_idx.p, s);
        else
            stored_product<float>(t->near_tiles, t->leaf_start.p, t->leaf_count.p, A->near_blk.p, A->near_boff.p,
                                  xmf.p, ym.p, t->near_ptr.p, t->near_first.p, t->near_idx.p, s);
    } else {
        ProfScope ps(KT_NEAR, s);
        if (df)
            nbody_sym_df(t, t->near_tiles, t->leaf_start.p, t->leaf_count.p, nullptr, xm2.p, ym.p, t->near_ptr.p,
                         t->near_first.p, t->near_idx.p, s);
        else if (sym && f64)
            nbody_sym<double>(A->kid, t->near_tiles, t->leaf_start.p, t->leaf_count.p, t->xs[0].p, t->xs[1].p,
                              t->xs[2].p, nullptr, nullptr, nullptr, xm.p, ym.p, t->near_ptr.p, t->near_first.p,
                              t->near_idx.p, d, A->kp[0], s);
        else if (sym)
            nbody_sym<float>(A->kid, t->near_tiles, t->leaf_start.p, t->leaf_count.p, PX[0], PX[1], PX[2], CF[0],
                             CF[1], CF[2], xmf.p, ym.p, t->near_ptr.p, t->near_first.p, t->near_idx.p, d, A->kp[0], s);
        else if (f64)
            nbody<double>(A->kid, t->near_tiles, t->leaf_start.p, t->leaf_count.p, t->xs[0].p, t->xs[1].p,
                          t->xs[2].p, nullptr, nullptr, nullptr, xm.p, ym.p, R, t->near_ptr.p, t->near_idx.p, d,
                          A->kp[0], s);
        else {
            // 16 columns at a time on the tensor cores, the rest on the CUDA cores
            const int rtc = A->tensor_core_products ? R / 16 * 16 : 0;
            if (rtc > 0) {
                prepare_tc_tiles(t, s);
                for (int c0 = 0; c0 < rtc; c0 += 16)
                    nbody_tc16(A->kid, t->near_tiles_tc, t->leaf_start.p, t->leaf_count.p, PX[0], PX[1], PX[2],
                               CF[0], CF[1], CF[2], xmf.p + c0, R, ym.p + c0, R, t->near_ptr.p, t->near_idx.p, d,
                               A->kp[0], t->tc_status.p, s);
            }
            nbody<float>(A->kid, t->near_tiles, t->leaf_start.p, t->leaf_count.p, PX[0], PX[1], PX[2], CF[0], CF[1],
                         CF[2], xmf.p, ym.p, R, t->near_ptr.p, t->near_idx.p, d, A->kp[0], s, rtc);
        }
    }
    if (dtype == H2_DTYPE_F64)
        k_perm_out_multi<double><<<blocks_for(nr, 256), 256, 0, s>>>(ym.p, t->perm.p, n, R, static_cast<double *>(y),
                                                                      ld);
    else
        k_perm_out_multi<float><<<blocks_for(nr, 256), 256, 0, s>>>(ym.p, t->perm.p, n, R, static_cast<float *>(y),
                                                                     ld);
    H2_LAUNCH("k_perm_out_multi");
}

void exact_rows_impl(h2_tree_s *t, int kid, const double *kp, const double *z, const int64_t *rows, int64_t nrows,
                     double *out, cudaStream_t s) {
    const int64_t n = t->n;
    DevBuf<double> zm;
    zm.alloc(n, s);
    k_perm_in<<<blocks_for(n, 256), 256, 0, s>>>(z, t->perm.p, n, zm.p);
    H2_LAUNCH("k_perm_in");
    if (nrows > 0 && kid == H2_K_COULOMB && t->d == 3) {
        // 3D Coulomb: float-float terms and sums (nbody_df.cu), eight rows a CTA
        const int nch = (int)((n + ER_CHUNK - 1) / ER_CHUNK);
        const int64_t rb = std::min<int64_t>(nrows, 65536);
        DevBuf<double> part;
        part.alloc((size_t)rb * nch, s);
        ProfScope ps(KT_EXACT, s);
        for (int64_t r0 = 0; r0 < nrows; r0 += rb) {
            const int64_t nr = std::min<int64_t>(rb, nrows - r0);
            exact_rows_df_parts(t, zm.p, rows + r0, nr, ER_CHUNK, nch, part.p, s);
            k_exact_sum<<<blocks_for(nr, 256), 256, 0, s>>>(part.p, nr, nch, out + r0);
            H2_LAUNCH("k_exact_sum");
        }
    } else if (nrows > 0) {
        const int nch = (int)((n + ER_CHUNK - 1) / ER_CHUNK);
        const int64_t rb = std::min<int64_t>(nrows, 65535);  // rows per launch (grid y limit)
        DevBuf<double> part;
        part.alloc((size_t)rb * nch, s);
        ProfScope ps(KT_EXACT, s);
        for (int64_t r0 = 0; r0 < nrows; r0 += rb) {
            const int64_t nr = std::min<int64_t>(rb, nrows - r0);
            k_exact_part<<<dim3((unsigned)nch, (unsigned)nr), ER_THREADS, 0, s>>>(
                rows + r0, nr, t->iperm.p, t->xs[0].p, t->xs[1].p, t->xs[2].p, zm.p, n, t->d, kid,
                h2_kappa_param(kid, kp[0]), nch, part.p);
            k_exact_sum<<<blocks_for(nr, 256), 256, 0, s>>>(part.p, nr, nch, out + r0);
            note_launches(1);
            H2_LAUNCH("k_exact_part");
        }
    }
}

void sampled_error_impl(const double *exact, const double *approx, const int64_t *rows, int64_t nrows, int64_t n,
                        double *err_out, cudaStream_t s) {
    k_sampled_error<<<1, 1024, 0, s>>>(exact, approx, rows, nrows, n, err_out);
    H2_LAUNCH("k_sampled_error");
}

// Device address of g_noalloc_zm on the current device.  Host code cannot use
// the symbol's name as a device pointer, so it is looked up once per device
// (with that device current) and cached.
static double *noalloc_scratch_for_current_device() {
    static std::mutex mu;
    static double *addr[256] = {};
    int dev = 0;
    H2_CUDA(cudaGetDevice(&dev));
    H2_REQUIRE(dev >= 0 && dev < 256, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        H2_CUDA(cudaGetSymbolAddress(&p, g_noalloc_zm));
        addr[dev] = static_cast<double *>(p);
    }
    return addr[dev];
}

void exact_rows_noalloc_impl(h2_tree_s *t, int kid, const double *kp, const double *z, const int64_t *rows,
                             int64_t nrows, double *out, cudaStream_t s) {
    const int64_t n = t->n;
    if (n > H2_NOALLOC_MAX_N)
        fail(H2_ERR_INVALID_ARG, "h2_exact_rows_noalloc supports at most 1048576 points (tree has " +
                                     std::to_string(n) + ")");
    double *zm = noalloc_scratch_for_current_device();
    // zm[0..n) is fully overwritten below; nothing needs clearing first
    k_perm_in<<<blocks_for(n, 256), 256, 0, s>>>(z, t->perm.p, n, zm);
    H2_LAUNCH("k_perm_in (noalloc)");
    if (nrows > 0) {
        k_exact_rows<<<(unsigned)nrows, 512, 0, s>>>(rows, nrows, t->iperm.p, t->xs[0].p, t->xs[1].p, t->xs[2].p,
                                                     zm, n, t->d, kid, h2_kappa_param(kid, kp[0]), out);
        H2_LAUNCH("k_exact_rows (noalloc)");
    }
}

}  // namespace h2
