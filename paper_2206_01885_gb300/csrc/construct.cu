// construct.cu -- Algorithm 2 of arXiv 2206.01885: for every level from the
// deepest to 1, the kernel block A_i = K(Y_i*, Xbar_i) of every node, its
// column-pivoted QR interpolative decomposition (section 4.1, eqs. (3)-(5)),
// the skeleton Xhat_i and the nested basis U_i = P [I; (R11^{-1} R12)^T].
//
// One CTA factors one node's block; all nodes of a level run in one launch.
// The float64 path evaluates the block and the Householder updates in
// float64.  Column norms are downdated as in LAPACK's xLAQP2 and recomputed
// once the downdated value has lost about half its digits.
#include <climits>

#include <mutex>

#include <cooperative_groups.h>

#include "h2_internal.cuh"
#include "df.cuh"

namespace h2 {
namespace {

constexpr int QR_THREADS = 512;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr size_t SMEM_LIMIT = 220 * 1024;

// c_i, m_i and the block / candidate sizes of each node of a level
__global__ void k_cand_sizes(int lb, int nl, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                             const int32_t *end, const int32_t *kk, const int32_t *ycnt, int32_t *cc,
                             int64_t *szc, int64_t *sza) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nl) return;
    int i = lb + a;
    int c = 0;
    if (nchild[i] == 0) c = end[i] - begin[i];
    else
        for (int ch = fchild[i]; ch < fchild[i] + nchild[i]; ch++) c += kk[ch];
    int m = ycnt[i];
    if (m == 0) c = 0;  // no farfield: no basis, the node is skipped
    cc[i] = c;
    szc[a] = c;
    sza[a] = (int64_t)m * c;
}

// Xbar_i: the leaf's points, or the children's skeletons in child order
__global__ void k_gather_cand(int lb, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                              const int32_t *cc, const int32_t *kk, int32_t *const *skptr, const int64_t *coff,
                              int32_t *cand) {
    int a = blockIdx.x, i = lb + a;
    int c = cc[i];
    if (c == 0) return;
    int32_t *dst = cand + coff[a];
    if (nchild[i] == 0) {
        for (int r = threadIdx.x; r < c; r += blockDim.x) dst[r] = begin[i] + r;
        return;
    }
    int w = 0;
    for (int ch = fchild[i]; ch < fchild[i] + nchild[i]; ch++) {
        int n = kk[ch];
        const int32_t *src = skptr[ch];
        for (int r = threadIdx.x; r < n; r += blockDim.x) dst[w + r] = src[r];
        w += n;
    }
}

// A_i[r + l m] = kappa(y_r, xbar_l), column-major m x c, float64: every entry
// evaluated exactly as the plain IEEE formula (bit-identical to a CPU
// evaluation for Coulomb).
__global__ void k_keval_f64(int lb, const int32_t *ycnt, const int32_t *cc, int32_t *const *yptr,
                            const int32_t *cand, const int64_t *coff, const int64_t *aoff, const double *x0,
                            const double *x1, const double *x2, int d, int kid, double kp0, double *Abase) {
    int a = blockIdx.x, i = lb + a;
    int m = ycnt[i], c = cc[i];
    if (m == 0 || c == 0) return;
    const int32_t *Y = yptr[i];
    const int32_t *X = cand + coff[a];
    double *A = Abase + aoff[a];
    // columns split over the CTAs of the node, rows over the threads (no
    // per-element index division)
    for (int l = blockIdx.y; l < c; l += gridDim.y) {
        const int32_t x = X[l];
        const double b0 = x0[x], b1 = d > 1 ? x1[x] : 0.0, b2 = d > 2 ? x2[x] : 0.0;
        double *Acol = A + (int64_t)l * m;
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            const int32_t y = Y[r];
            Acol[r] = h2_kxy(kid, kp0, d, x0[y], d > 1 ? x1[y] : 0.0, d > 2 ? x2[y] : 0.0, b0, b1, b2);
        }
    }
}

// float32 block: the node's Y_i* and Xbar_i points, relative to the node's
// cell centre, are staged once in shared memory as float32.
__global__ void k_keval_f32(int lb, const int32_t *ycnt, const int32_t *cc, int32_t *const *yptr,
                            const int32_t *cand, const int64_t *coff, const int64_t *aoff, const double *x0,
                            const double *x1, const double *x2, const double *cen0, const double *cen1,
                            const double *cen2, int d, int kid, double kp0, float *Abase) {
    extern __shared__ float sp_[];
    int a = blockIdx.x, i = lb + a;
    int m = ycnt[i], c = cc[i];
    if (m == 0 || c == 0) return;
    const int32_t *Y = yptr[i];
    const int32_t *X = cand + coff[a];
    float *ys = sp_, *xs = sp_ + 3 * m;
    // (cos(x . y) takes absolute coordinates; every other kernel relative ones)
    const bool cosdot = kid == H2_K_COSDOT;
    const double o0 = cosdot ? 0.0 : cen0[i], o1 = d > 1 && !cosdot ? cen1[i] : 0.0,
                 o2 = d > 2 && !cosdot ? cen2[i] : 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        int32_t y = Y[r];
        ys[3 * r] = (float)(x0[y] - o0);
        ys[3 * r + 1] = d > 1 ? (float)(x1[y] - o1) : 0.f;
        ys[3 * r + 2] = d > 2 ? (float)(x2[y] - o2) : 0.f;
    }
    for (int l = threadIdx.x; l < c; l += blockDim.x) {
        int32_t x = X[l];
        xs[3 * l] = (float)(x0[x] - o0);
        xs[3 * l + 1] = d > 1 ? (float)(x1[x] - o1) : 0.f;
        xs[3 * l + 2] = d > 2 ? (float)(x2[x] - o2) : 0.f;
    }
    __syncthreads();
    float *A = Abase + aoff[a];
    const float k0 = (float)kp0;
    // one warp per column, lanes over its rows (no index division)
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = blockIdx.y * nw + (threadIdx.x >> 5); l < c; l += gridDim.y * nw) {
        const float bx = xs[3 * l], by = xs[3 * l + 1], bz = xs[3 * l + 2];
        float *Acol = A + (int64_t)l * m;
        if (cosdot) {
            for (int r = lane; r < m; r += 32)
                Acol[r] = __cosf(fmaf(ys[3 * r + 2], bz, fmaf(ys[3 * r + 1], by, ys[3 * r] * bx)));
        } else {
            for (int r = lane; r < m; r += 32) {
                float dx = ys[3 * r] - bx, dy = ys[3 * r + 1] - by, dz = ys[3 * r + 2] - bz;
                float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                Acol[r] = h2_kappa_f(kid, k0, r2);
            }
        }
    }
}

// (value, index) max with ties to the smaller index
// (key, index) max with ties to the smaller index; keys are the bit patterns
// of non-negative doubles, which order like the values (integer compares, no
// float64 instruction)
__device__ __forceinline__ void argmax_key(long long &k, int &i, long long k2, int i2) {
    if (k2 > k || (k2 == k && i2 < i)) { k = k2; i = i2; }
}

// Column-pivoted Householder QR of each node's block, stopped at the first
// step whose pivot norm is <= tol * |r_11|.  On exit A holds R (upper
// triangle of the first k columns and rows 0..k-1 of the others), kout[i] = k
// and piv[0..c) is the column order.  Real = double: everything float64.
// Real = float: the block, the reflector and the trailing update are float32,
// and so are the per-lane partial sums of squares; the cross-lane sums, the
// column norms, their downdating, the pivot choice and the stop test are
// float64.  This form keeps squared norms and downdates them as nu^2 - r^2
// (one float64 fma instead of two divisions and a square root: float64 runs
// at 1/64 of the float32 rate on this GPU), recomputing once the downdated
// value falls below sqrt(2^-24) of its last recomputed value, the float32
// analogue of LAPACK's sqrt(eps).
template <class Real, int RPL>
__global__ void __launch_bounds__(QR_THREADS, 2) k_cpqr(int lb, const int32_t *ycnt, const int32_t *cc,
                                                     const int64_t *aoff, Real *Abase, double tol, int32_t *kout,
                                                     const int64_t *coff, int32_t *pivbase) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int a = blockIdx.x, node = lb + a;
    const int m = ycnt[node], c = cc[node];
    if (m == 0 || c == 0) {
        if (threadIdx.x == 0) kout[node] = 0;
        return;
    }
    double *nrm = reinterpret_cast<double *>(smem_raw);
    double *nrm0 = nrm + c;
    Real *rowj = reinterpret_cast<Real *>(nrm0 + c);  // row j of the updated trailing columns
    Real *v = rowj + c;
    int32_t *pv = reinterpret_cast<int32_t *>(v + m);
    unsigned char *flag = reinterpret_cast<unsigned char *>(pv + c);
    __shared__ double red[QR_WARPS];
    __shared__ long long bkey[QR_WARPS];
    __shared__ int bidx[QR_WARPS];
    __shared__ int s_p, s_stop;
    __shared__ Real s_tau, s_beta, s_sc;
    __shared__ int s_has;
    Real *A = Abase + aoff[a];
    int32_t *piv = pivbase + coff[a];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const double tol3z = sqrt(ldexp(1.0, sizeof(Real) == 8 ? -53 : -24));

    for (int l = threadIdx.x; l < c; l += blockDim.x) pv[l] = l;
    // per-lane partial sums in the block's type, reduced across lanes in float64
    // float64 form: nrm holds column norms (LAPACK downdating); float32 form:
    // nrm holds squared column norms, downdated as nu^2 - r^2 in float64
    constexpr bool SQ = sizeof(Real) == 4;
    for (int l = warp; l < c; l += nwarps) {
        const Real *col = A + (int64_t)l * m;
        Real sp = 0;
        for (int r = lane; r < m; r += 32) sp += col[r] * col[r];
        const double s = (double)warp_sum(sp);
        if (lane == 0) { nrm[l] = SQ ? s : sqrt(s); nrm0[l] = nrm[l]; }
    }
    __syncthreads();
    const int kmax = min(m, c);
    int k = 0;
    double r11 = 0.0;
    for (int j = 0; j < kmax; j++) {
        // pivot: largest downdated norm among columns j..c-1
        long long bk = -1;
        int bi = INT_MAX;
        for (int l = j + threadIdx.x; l < c; l += blockDim.x) argmax_key(bk, bi, __double_as_longlong(nrm[l]), l);
        for (int o = 16; o > 0; o >>= 1) {
            long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
            int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            argmax_key(bk, bi, k2, i2);
        }
        if (lane == 0) { bkey[warp] = bk; bidx[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long kk2 = bkey[0];
            int ii = bidx[0];
            for (int w = 1; w < nwarps; w++) argmax_key(kk2, ii, bkey[w], bidx[w]);
            const double vv = __longlong_as_double(kk2);
            if (j == 0) r11 = vv;
            s_p = ii;
            // float32 form compares squared norms: nu^2 <= tol^2 r11^2
            s_stop = (!(vv > (SQ ? tol * tol : tol) * r11) || vv == 0.0) ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p;
        if (p != j) {
            Real *cj = A + (int64_t)j * m, *cp = A + (int64_t)p * m;
            for (int r = threadIdx.x; r < m; r += blockDim.x) {
                Real t = cj[r]; cj[r] = cp[r]; cp[r] = t;
            }
            if (threadIdx.x == 0) {
                double t = nrm[j]; nrm[j] = nrm[p]; nrm[p] = t;
                t = nrm0[j]; nrm0[j] = nrm0[p]; nrm0[p] = t;
                int ti = pv[j]; pv[j] = pv[p]; pv[p] = ti;
            }
        }
        __syncthreads();
        // Householder reflector for A[j:m, j]
        // (per-lane and per-warp partial sums in the block's type, the warps'
        // sums added in order by thread 0, which also forms the reflector's
        // scalars once and broadcasts them)
        Real *aj = A + (int64_t)j * m;
        Real part = 0;
        for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) part += aj[r] * aj[r];
        part = warp_sum(part);
        if (lane == 0) red[warp] = (double)part;
        __syncthreads();
        if (threadIdx.x == 0) {  // in the block's type
            Real sigma = 0;
            for (int w = 0; w < nwarps; w++) sigma += (Real)red[w];
            const Real alpha = aj[j];
            Real tau = 0, beta = alpha, sc = 0;
            if (sigma != (Real)0) {
                Real xn = sqrt(alpha * alpha + sigma);
                beta = alpha >= (Real)0 ? -xn : xn;
                tau = (beta - alpha) / beta;
                sc = (Real)1 / (alpha - beta);
            }
            s_tau = tau;
            s_beta = beta;
            s_sc = sc;
            s_has = tau != (Real)0;
            s_stop = (alpha == (Real)0 && sigma == (Real)0) ? 1 : 0;  // exactly zero pivot column
        }
        __syncthreads();
        if (s_stop) break;
        const bool has_tau = s_has != 0;
        const Real scR = s_sc;
        for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) v[r] = aj[r] * scR;
        __syncthreads();
        if (threadIdx.x == 0) aj[j] = s_beta;
        const Real tauR = s_tau;
        // apply to the trailing columns (one warp per column); row j of the
        // result goes to shared memory for the norm downdate.  With RPL > 0 a
        // lane keeps its RPL rows in registers and a warp takes two columns at
        // a time: all their loads are issued together (twice the loads in
        // flight), each reflector entry is read once for both, and the update
        // reuses the registers.
        if constexpr (RPL > 0 && RPL <= 12) {
            for (int l = j + 1 + warp; l < c; l += 2 * nwarps) {
                const int l2 = l + nwarps;
                const bool two = l2 < c;  // (warp-uniform)
                Real *al = A + (int64_t)l * m;
                Real *bl = A + (int64_t)(two ? l2 : l) * m;
                Real ajl = al[j], bjl = two ? bl[j] : (Real)0;
                Real a2[RPL], b2[RPL];
#pragma unroll
                for (int u = 0; u < RPL; u++) {
                    const int r = j + 1 + lane + 32 * u;
                    a2[u] = r < m ? al[r] : (Real)0;
                    b2[u] = two && r < m ? bl[r] : (Real)0;
                }
                if (has_tau) {
                    Real wa = 0, wb = 0;
#pragma unroll
                    for (int u = 0; u < RPL; u++) {
                        const int r = j + 1 + lane + 32 * u;
                        if (r < m) {
                            const Real vr = v[r];
                            wa += vr * a2[u];
                            wb += vr * b2[u];
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        wa += __shfl_xor_sync(0xffffffffu, wa, o);
                        wb += __shfl_xor_sync(0xffffffffu, wb, o);
                    }
                    wa = (wa + ajl) * tauR;
                    wb = (wb + bjl) * tauR;
#pragma unroll
                    for (int u = 0; u < RPL; u++) {
                        const int r = j + 1 + lane + 32 * u;
                        if (r < m) {
                            const Real vr = v[r];
                            al[r] = a2[u] - wa * vr;
                            if (two) bl[r] = b2[u] - wb * vr;
                        }
                    }
                    ajl = ajl - wa;
                    bjl = bjl - wb;
                    if (lane == 0) {
                        al[j] = ajl;
                        if (two) bl[j] = bjl;
                    }
                }
                if (lane == 0) {
                    rowj[l] = ajl;
                    if (two) rowj[l2] = bjl;
                }
            }
        } else if constexpr (RPL > 0) {  // longer slices: one column a warp (registers)
            for (int l = j + 1 + warp; l < c; l += nwarps) {
                Real *al = A + (int64_t)l * m;
                Real ajl = al[j];
                Real a1[RPL];
#pragma unroll
                for (int u = 0; u < RPL; u++) {
                    const int r = j + 1 + lane + 32 * u;
                    a1[u] = r < m ? al[r] : (Real)0;
                }
                if (has_tau) {
                    Real w = 0;
#pragma unroll
                    for (int u = 0; u < RPL; u++) {
                        const int r = j + 1 + lane + 32 * u;
                        if (r < m) w += v[r] * a1[u];
                    }
                    w = warp_sum(w) + ajl;
                    w = w * tauR;
#pragma unroll
                    for (int u = 0; u < RPL; u++) {
                        const int r = j + 1 + lane + 32 * u;
                        if (r < m) al[r] = a1[u] - w * v[r];
                    }
                    ajl = ajl - w;
                    if (lane == 0) al[j] = ajl;
                }
                if (lane == 0) rowj[l] = ajl;
            }
        } else {
            for (int l = j + 1 + warp; l < c; l += nwarps) {
                Real *al = A + (int64_t)l * m;
                Real ajl = al[j];
                if (has_tau) {
                    Real w = 0;
                    for (int r = j + 1 + lane; r < m; r += 32) w += v[r] * al[r];
                    w = warp_sum(w) + ajl;
                    w = w * tauR;
                    for (int r = j + 1 + lane; r < m; r += 32) al[r] = al[r] - w * v[r];
                    ajl = ajl - w;
                    if (lane == 0) al[j] = ajl;
                }
                if (lane == 0) rowj[l] = ajl;
            }
        }
        __syncthreads();
        // downdate the norms, one thread per column; flag the ones that have
        // lost about half their digits for recomputation
        for (int l = j + 1 + threadIdx.x; l < c; l += blockDim.x) {
            double nl = nrm[l];
            flag[l] = 0;
            if (nl != 0.0) {
                const double rj = (double)rowj[l];
                if constexpr (SQ) {  // nu^2 - r^2, recomputed once below sqrt(2^-24) nu0^2
                    double n2 = fma(-rj, rj, nl);
                    if (!(n2 > tol3z * nrm0[l])) flag[l] = 1;
                    else nrm[l] = n2;
                } else {
                    double tt = fabs(rj) / nl;
                    tt = 1.0 - tt * tt;
                    if (tt < 0.0) tt = 0.0;
                    double t2 = nl / nrm0[l];
                    t2 = tt * t2 * t2;
                    if (t2 <= tol3z) flag[l] = 1;
                    else nrm[l] = nl * sqrt(tt);
                }
            }
        }
        __syncthreads();
        for (int l = j + 1 + warp; l < c; l += nwarps) {
            if (!flag[l]) continue;
            const Real *al = A + (int64_t)l * m;
            Real sp = 0;
            if constexpr (RPL > 0) {
                Real a[RPL];
#pragma unroll
                for (int u = 0; u < RPL; u++) {
                    int r = j + 1 + lane + 32 * u;
                    a[u] = r < m ? al[r] : (Real)0;
                }
#pragma unroll
                for (int u = 0; u < RPL; u++) sp += a[u] * a[u];
            } else {
                for (int r = j + 1 + lane; r < m; r += 32) sp += al[r] * al[r];
            }
            const double s = (double)warp_sum(sp);
            if (lane == 0) { nrm[l] = SQ ? s : sqrt(s); nrm0[l] = nrm[l]; }
        }
        __syncthreads();
        k = j + 1;
    }
    for (int l = threadIdx.x; l < c; l += blockDim.x) piv[l] = pv[l];
    if (threadIdx.x == 0) kout[node] = k;
}

// Float64 form, float-float arithmetic: the same column-pivoted Householder
// QR as k_cpqr<double, 0> (right-looking, one warp per trailing column, the
// same pivots, downdates, recomputation and stop test in float64), with the
// block held as float pairs hi + lo (about 48 bits) and the reflector, its
// products with the trailing columns and their rank-1 updates computed in
// float-float arithmetic on the float32 units (float64 runs at 1/74 of the
// float32 rate on this GPU).  A float64 block is converted in place on entry
// (each element keeps its 8 bytes; split = 1: the block already holds float
// pairs); on exit rows 0..k-1 of every column -- R, what the solve reads --
// are converted back to float64 in place.  The reflector's scalars (one
// square root, two divisions) and the column norms stay float64.
__global__ void __launch_bounds__(QR_THREADS, 2) k_cpqr_df(int lb, const int32_t *ycnt, const int32_t *cc,
                                                         const int64_t *aoff, double *Abase, double tol,
                                                         int32_t *kout, const int64_t *coff, int32_t *pivbase,
                                                         int split) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int a = blockIdx.x, node = lb + a;
    const int m = ycnt[node], c = cc[node];
    if (m == 0 || c == 0) {
        if (threadIdx.x == 0) kout[node] = 0;
        return;
    }
    double *nrm = reinterpret_cast<double *>(smem_raw);
    double *nrm0 = nrm + c;
    double *rowj = nrm0 + c;                            // row j of the updated trailing columns
    float2 *v = reinterpret_cast<float2 *>(rowj + c);  // the reflector, rows j..m-1
    int32_t *pv = reinterpret_cast<int32_t *>(v + m);
    unsigned char *flag = reinterpret_cast<unsigned char *>(pv + c);
    __shared__ double red[QR_WARPS];
    __shared__ long long bkey[QR_WARPS];
    __shared__ int bidx[QR_WARPS];
    __shared__ int s_p, s_stop;
    __shared__ float2 s_tau, s_beta, s_sc;
    __shared__ int s_has;
    double *Ad = Abase + aoff[a];
    float2 *A = reinterpret_cast<float2 *>(Ad);  // the same 8 bytes per element
    int32_t *piv = pivbase + coff[a];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const double tol3z = sqrt(ldexp(1.0, -53));
    const int64_t mc = (int64_t)m * c;
    if (!split)
        for (int64_t e = threadIdx.x; e < mc; e += blockDim.x) A[e] = df::from_double(Ad[e]);
    for (int l = threadIdx.x; l < c; l += blockDim.x) pv[l] = l;
    __syncthreads();
    for (int l = warp; l < c; l += nwarps) {
        const float2 *col = A + (int64_t)l * m;
        float sh = 0.f, sl = 0.f;
        for (int r = lane; r < m; r += 32) df::mac(sh, sl, col[r], col[r]);
        const double s = df::to_double(df::warp_sum(sh, sl));
        if (lane == 0) { nrm[l] = sqrt(s); nrm0[l] = nrm[l]; }
    }
    __syncthreads();
    const int kmax = min(m, c);
    int k = 0;
    double r11 = 0.0;
    for (int j = 0; j < kmax; j++) {
        // pivot: largest downdated norm among columns j..c-1
        long long bk = -1;
        int bi = INT_MAX;
        for (int l = j + threadIdx.x; l < c; l += blockDim.x) argmax_key(bk, bi, __double_as_longlong(nrm[l]), l);
        for (int o = 16; o > 0; o >>= 1) {
            long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
            int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            argmax_key(bk, bi, k2, i2);
        }
        if (lane == 0) { bkey[warp] = bk; bidx[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long kk2 = bkey[0];
            int ii = bidx[0];
            for (int w = 1; w < nwarps; w++) argmax_key(kk2, ii, bkey[w], bidx[w]);
            const double vv = __longlong_as_double(kk2);
            if (j == 0) r11 = vv;
            s_p = ii;
            s_stop = (!(vv > tol * r11) || vv == 0.0) ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p;
        if (p != j) {
            float2 *cj = A + (int64_t)j * m, *cp = A + (int64_t)p * m;
            for (int r = threadIdx.x; r < m; r += blockDim.x) {
                float2 t = cj[r]; cj[r] = cp[r]; cp[r] = t;
            }
            if (threadIdx.x == 0) {
                double t = nrm[j]; nrm[j] = nrm[p]; nrm[p] = t;
                t = nrm0[j]; nrm0[j] = nrm0[p]; nrm0[p] = t;
                int ti = pv[j]; pv[j] = pv[p]; pv[p] = ti;
            }
        }
        __syncthreads();
        // Householder reflector for A[j:m, j]: sum of squares in float-float,
        // the warps' sums added in float64 by thread 0, which forms the
        // scalars in float64 and broadcasts them as float pairs
        float2 *aj = A + (int64_t)j * m;
        {
            float sh = 0.f, sl = 0.f;
            for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) df::mac(sh, sl, aj[r], aj[r]);
            const float2 ws = df::warp_sum(sh, sl);
            if (lane == 0) red[warp] = df::to_double(ws);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sigma = 0;
            for (int w = 0; w < nwarps; w++) sigma += red[w];
            const double alpha = df::to_double(aj[j]);
            double tau = 0, beta = alpha, sc = 0;
            if (sigma != 0.0) {
                const double xn = sqrt(alpha * alpha + sigma);
                beta = alpha >= 0.0 ? -xn : xn;
                tau = (beta - alpha) / beta;
                sc = 1.0 / (alpha - beta);
            }
            s_tau = df::from_double(tau);
            s_beta = df::from_double(beta);
            s_sc = df::from_double(sc);
            s_has = tau != 0.0;
            s_stop = (alpha == 0.0 && sigma == 0.0) ? 1 : 0;  // exactly zero pivot column
        }
        __syncthreads();
        if (s_stop) break;
        const bool has_tau = s_has != 0;
        const float2 scD = s_sc, tauD = s_tau;
        for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) v[r] = df::mul(aj[r], scD);
        __syncthreads();
        if (threadIdx.x == 0) aj[j] = s_beta;
        // apply to the trailing columns, one warp per column: w = tau (v^T a),
        // a -= w v, all in float-float; row j of the result (float64) feeds the
        // norm downdate
        for (int l = j + 1 + warp; l < c; l += nwarps) {
            float2 *al = A + (int64_t)l * m;
            float2 ajl = al[j];
            if (has_tau) {
                // eight (then four) rows a lane in flight, two accumulators (the
                // loads are independent; the float-float sums chain)
                float sh = 0.f, sl = 0.f, th = 0.f, tl = 0.f;
                int r = j + 1 + lane;
                for (; r + 224 < m; r += 256) {
                    float2 a[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) a[u] = al[r + 32 * u];
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        df::mac(sh, sl, v[r + 32 * u], a[u]);
                        df::mac(th, tl, v[r + 32 * u + 32], a[u + 1]);
                    }
                }
                for (; r + 96 < m; r += 128) {
                    const float2 a0 = al[r], a1 = al[r + 32], a2 = al[r + 64], a3 = al[r + 96];
                    df::mac(sh, sl, v[r], a0);
                    df::mac(th, tl, v[r + 32], a1);
                    df::mac(sh, sl, v[r + 64], a2);
                    df::mac(th, tl, v[r + 96], a3);
                }
                for (; r < m; r += 32) df::mac(sh, sl, v[r], al[r]);
                const float2 s2 = df::add(df::norm(sh, sl), df::norm(th, tl));
                float2 w = df::add(df::warp_sum(s2.x, s2.y), ajl);
                w = df::mul(w, tauD);
                r = j + 1 + lane;
                for (; r + 224 < m; r += 256) {
                    float2 a[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) a[u] = al[r + 32 * u];
#pragma unroll
                    for (int u = 0; u < 8; u++) al[r + 32 * u] = df::fms(a[u], w, v[r + 32 * u]);
                }
                for (; r + 96 < m; r += 128) {
                    const float2 a0 = al[r], a1 = al[r + 32], a2 = al[r + 64], a3 = al[r + 96];
                    al[r] = df::fms(a0, w, v[r]);
                    al[r + 32] = df::fms(a1, w, v[r + 32]);
                    al[r + 64] = df::fms(a2, w, v[r + 64]);
                    al[r + 96] = df::fms(a3, w, v[r + 96]);
                }
                for (; r < m; r += 32) al[r] = df::fms(al[r], w, v[r]);
                ajl = df::sub(ajl, w);
                if (lane == 0) al[j] = ajl;
            }
            if (lane == 0) rowj[l] = df::to_double(ajl);
        }
        __syncthreads();
        // downdate the norms (float64, LAPACK's rule), one thread per column;
        // flag the ones that have lost about half their digits
        for (int l = j + 1 + threadIdx.x; l < c; l += blockDim.x) {
            double nl = nrm[l];
            flag[l] = 0;
            if (nl != 0.0) {
                const double rj = rowj[l];
                double tt = fabs(rj) / nl;
                tt = 1.0 - tt * tt;
                if (tt < 0.0) tt = 0.0;
                double t2 = nl / nrm0[l];
                t2 = tt * t2 * t2;
                if (t2 <= tol3z) flag[l] = 1;
                else nrm[l] = nl * sqrt(tt);
            }
        }
        __syncthreads();
        for (int l = j + 1 + warp; l < c; l += nwarps) {
            if (!flag[l]) continue;
            const float2 *al = A + (int64_t)l * m;
            float sh = 0.f, sl = 0.f;
            for (int r = j + 1 + lane; r < m; r += 32) df::mac(sh, sl, al[r], al[r]);
            const double s = df::to_double(df::warp_sum(sh, sl));
            if (lane == 0) { nrm[l] = sqrt(s); nrm0[l] = nrm[l]; }
        }
        __syncthreads();
        k = j + 1;
    }
    // R (rows 0..k-1 of every column) back to float64, in place
    __syncthreads();
    for (int l = warp; l < c; l += nwarps)
        for (int r = lane; r < k; r += 32) {
            const int64_t e = r + (int64_t)l * m;
            Ad[e] = df::to_double(A[e]);
        }
    for (int l = threadIdx.x; l < c; l += blockDim.x) piv[l] = pv[l];
    if (threadIdx.x == 0) kout[node] = k;
}

// Float64 form, float-float arithmetic, one node per cluster of QR_CL CTAs.
// The factorization is k_cpqr_df's: the same per-column arithmetic, the same
// pivots with the same ties (largest downdated norm, then smallest position),
// the same stop tests, and so the same R, rank and pivot order.  The node's
// candidate columns are shared out over the cluster's CTAs, so a level with
// fewer nodes than SMs still fills the GPU, and one block is in flight per
// cluster rather than per CTA.  Columns stay where they are: CTA r owns the
// columns l = r mod QR_CL.  perm maps positions to columns and pos maps them
// back; every CTA keeps both, updated identically.  A step runs as follows:
//  - every CTA offers the best (norm, position) among its own columns that are
//    not yet pivoted;
//  - one cluster barrier (it also publishes the previous step's updates);
//  - every CTA reads all the offers from the others' shared memory and takes
//    the same pivot;
//  - every CTA forms the same reflector from the pivot column, read from L2;
//  - each CTA updates, downdates and, where needed, renormalises its own
//    columns.
// R(j, j) is kept in the pivot column's norm slot (the other CTAs may still be
// reading row j of that column).  On exit rows 0..k-1 of every column go,
// as float64 and in pivot order, to Rbase, whose layout is the block's.
// piv = perm.  Every exit and break depends only on data that all CTAs of the
// cluster read alike (the offers, the pivot column after the barrier), so
// every CTA reaches every cluster barrier.
constexpr int QR_CL = 8;

__global__ void __cluster_dims__(QR_CL, 1, 1) __launch_bounds__(QR_THREADS, 2)
    k_cpqr_df_cl(int lb, const int32_t *ycnt, const int32_t *cc, const int64_t *aoff, double *Abase,
                 double *Rbase, double tol, int32_t *kout, const int64_t *coff, int32_t *pivbase, int split) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rank = (int)cl.block_rank();
    const int a = blockIdx.x / QR_CL, node = lb + a;
    const int m = ycnt[node], c = cc[node];
    if (m == 0 || c == 0) {  // (the same for every CTA of the cluster: no barrier is left waiting)
        if (rank == 0 && threadIdx.x == 0) kout[node] = 0;
        return;
    }
    double *nrm = reinterpret_cast<double *>(smem_raw);  // by column (own columns only)
    double *nrm0 = nrm + c;
    double *rowj = nrm0 + c;
    float2 *v = reinterpret_cast<float2 *>(rowj + c);
    int32_t *perm = reinterpret_cast<int32_t *>(v + m);  // position -> column
    int32_t *pos = perm + c;                              // column -> position
    unsigned char *flag = reinterpret_cast<unsigned char *>(pos + c);
    __shared__ long long off_key[2];  // this CTA's offer, by step parity
    __shared__ int off_pos[2];
    __shared__ double red[QR_WARPS];
    __shared__ long long bkey[QR_WARPS];
    __shared__ int bidx[QR_WARPS];
    __shared__ int s_p, s_stop;
    __shared__ float2 s_tau, s_beta, s_sc;
    __shared__ int s_has;
    double *Ad = Abase + aoff[a];
    float2 *A = reinterpret_cast<float2 *>(Ad);
    double *Rd = Rbase + aoff[a];
    int32_t *piv = pivbase + coff[a];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const double tol3z = sqrt(ldexp(1.0, -53));
    // own columns: l = rank + QR_CL * u, u = 0, 1, ...
    const int nown = c > rank ? (c - rank + QR_CL - 1) / QR_CL : 0;
    if (!split)
        for (int u = warp; u < nown; u += nwarps) {
            float2 *col = A + (int64_t)(rank + QR_CL * u) * m;
            const double *cd = Ad + (int64_t)(rank + QR_CL * u) * m;
            for (int r = lane; r < m; r += 32) col[r] = df::from_double(cd[r]);
        }
    for (int l = threadIdx.x; l < c; l += blockDim.x) { perm[l] = l; pos[l] = l; }
    for (int u = warp; u < nown; u += nwarps) {
        const int l = rank + QR_CL * u;
        const float2 *col = A + (int64_t)l * m;
        float sh = 0.f, sl = 0.f;
        for (int r = lane; r < m; r += 32) df::mac(sh, sl, col[r], col[r]);
        const double s = df::to_double(df::warp_sum(sh, sl));
        if (lane == 0) { nrm[l] = sqrt(s); nrm0[l] = nrm[l]; }
    }
    __syncthreads();
    const int kmax = min(m, c);
    int k = 0;
    double r11 = 0.0;
    for (int j = 0; j < kmax; j++) {
        // this CTA's offer: its best (norm, position) at positions >= j
        long long bk = -1;
        int bi = INT_MAX;
        for (int u = threadIdx.x; u < nown; u += blockDim.x) {
            const int l = rank + QR_CL * u;
            if (pos[l] >= j) argmax_key(bk, bi, __double_as_longlong(nrm[l]), pos[l]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
            int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            argmax_key(bk, bi, k2, i2);
        }
        if (lane == 0) { bkey[warp] = bk; bidx[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long kk2 = bkey[0];
            int ii = bidx[0];
            for (int w = 1; w < nwarps; w++) argmax_key(kk2, ii, bkey[w], bidx[w]);
            off_key[j & 1] = kk2;
            off_pos[j & 1] = ii;
        }
        cl.sync();  // the offers, and every CTA's column updates of the previous step
        if (threadIdx.x == 0) {
            long long kk2 = -1;
            int ii = INT_MAX;
            for (int r = 0; r < QR_CL; r++)
                argmax_key(kk2, ii, *cl.map_shared_rank(&off_key[j & 1], r), *cl.map_shared_rank(&off_pos[j & 1], r));
            const double vv = __longlong_as_double(kk2);
            if (j == 0) r11 = vv;
            s_p = ii;
            s_stop = (!(vv > tol * r11) || vv == 0.0) ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p;
        if (threadIdx.x == 0 && p != j) {
            const int cj = perm[j], cp = perm[p];
            perm[j] = cp; perm[p] = cj;
            pos[cp] = j; pos[cj] = p;
        }
        __syncthreads();
        const int jc = perm[j];  // the pivot column
        const bool own_pivot = jc % QR_CL == rank;
        // the reflector, in every CTA alike; the pivot column is read from L2
        // (its owner wrote it before the barrier)
        const float2 *aj = A + (int64_t)jc * m;
        {
            float sh = 0.f, sl = 0.f;
            for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) {
                const float2 x = __ldcg(aj + r);
                df::mac(sh, sl, x, x);
            }
            const float2 ws = df::warp_sum(sh, sl);
            if (lane == 0) red[warp] = df::to_double(ws);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sigma = 0;
            for (int w = 0; w < nwarps; w++) sigma += red[w];
            const double alpha = df::to_double(__ldcg(aj + j));
            double tau = 0, beta = alpha, sc = 0;
            if (sigma != 0.0) {
                const double xn = sqrt(alpha * alpha + sigma);
                beta = alpha >= 0.0 ? -xn : xn;
                tau = (beta - alpha) / beta;
                sc = 1.0 / (alpha - beta);
            }
            s_tau = df::from_double(tau);
            s_beta = df::from_double(beta);
            s_sc = df::from_double(sc);
            s_has = tau != 0.0;
            s_stop = (alpha == 0.0 && sigma == 0.0) ? 1 : 0;  // exactly zero pivot column
        }
        __syncthreads();
        if (s_stop) break;
        const bool has_tau = s_has != 0;
        const float2 scD = s_sc, tauD = s_tau;
        for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) v[r] = df::mul(__ldcg(aj + r), scD);
        __syncthreads();
        if (threadIdx.x == 0 && own_pivot) nrm[jc] = df::to_double(s_beta);  // R(j, j), written out on exit
        // own trailing columns, one warp a column (k_cpqr_df's arithmetic)
        for (int u = warp; u < nown; u += nwarps) {
            const int l = rank + QR_CL * u;
            if (pos[l] <= j) continue;
            float2 *al = A + (int64_t)l * m;
            float2 ajl = al[j];
            if (has_tau) {
                float sh = 0.f, sl = 0.f, th = 0.f, tl = 0.f;
                int r = j + 1 + lane;
                for (; r + 224 < m; r += 256) {
                    float2 x[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) x[q] = al[r + 32 * q];
#pragma unroll
                    for (int q = 0; q < 8; q += 2) {
                        df::mac(sh, sl, v[r + 32 * q], x[q]);
                        df::mac(th, tl, v[r + 32 * q + 32], x[q + 1]);
                    }
                }
                for (; r + 96 < m; r += 128) {
                    const float2 a0 = al[r], a1 = al[r + 32], a2 = al[r + 64], a3 = al[r + 96];
                    df::mac(sh, sl, v[r], a0);
                    df::mac(th, tl, v[r + 32], a1);
                    df::mac(sh, sl, v[r + 64], a2);
                    df::mac(th, tl, v[r + 96], a3);
                }
                for (; r < m; r += 32) df::mac(sh, sl, v[r], al[r]);
                const float2 s2 = df::add(df::norm(sh, sl), df::norm(th, tl));
                float2 w = df::add(df::warp_sum(s2.x, s2.y), ajl);
                w = df::mul(w, tauD);
                r = j + 1 + lane;
                for (; r + 224 < m; r += 256) {
                    float2 x[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) x[q] = al[r + 32 * q];
#pragma unroll
                    for (int q = 0; q < 8; q++) al[r + 32 * q] = df::fms(x[q], w, v[r + 32 * q]);
                }
                for (; r + 96 < m; r += 128) {
                    const float2 a0 = al[r], a1 = al[r + 32], a2 = al[r + 64], a3 = al[r + 96];
                    al[r] = df::fms(a0, w, v[r]);
                    al[r + 32] = df::fms(a1, w, v[r + 32]);
                    al[r + 64] = df::fms(a2, w, v[r + 64]);
                    al[r + 96] = df::fms(a3, w, v[r + 96]);
                }
                for (; r < m; r += 32) al[r] = df::fms(al[r], w, v[r]);
                ajl = df::sub(ajl, w);
                if (lane == 0) al[j] = ajl;
            }
            if (lane == 0) rowj[l] = df::to_double(ajl);
        }
        __syncthreads();
        for (int u = threadIdx.x; u < nown; u += blockDim.x) {
            const int l = rank + QR_CL * u;
            if (pos[l] <= j) continue;
            double nl = nrm[l];
            flag[l] = 0;
            if (nl != 0.0) {
                const double rj = rowj[l];
                double tt = fabs(rj) / nl;
                tt = 1.0 - tt * tt;
                if (tt < 0.0) tt = 0.0;
                double t2 = nl / nrm0[l];
                t2 = tt * t2 * t2;
                if (t2 <= tol3z) flag[l] = 1;
                else nrm[l] = nl * sqrt(tt);
            }
        }
        __syncthreads();
        for (int u = warp; u < nown; u += nwarps) {
            const int l = rank + QR_CL * u;
            if (pos[l] <= j || !flag[l]) continue;
            const float2 *al = A + (int64_t)l * m;
            float sh = 0.f, sl = 0.f;
            for (int r = j + 1 + lane; r < m; r += 32) df::mac(sh, sl, al[r], al[r]);
            const double s = df::to_double(df::warp_sum(sh, sl));
            if (lane == 0) { nrm[l] = sqrt(s); nrm0[l] = nrm[l]; }
        }
        __syncthreads();
        k = j + 1;
    }
    // R in pivot order: rows 0..k-1 of each own column, as float64, at its
    // position; a pivoted column's diagonal entry is the kept R(j, j)
    for (int u = warp; u < nown; u += nwarps) {
        const int l = rank + QR_CL * u, q = pos[l];
        const float2 *al = A + (int64_t)l * m;
        double *rq = Rd + (int64_t)q * m;
        for (int r = lane; r < k; r += 32) rq[r] = (r == q) ? nrm[l] : df::to_double(al[r]);
    }
    if (rank == 0) {
        for (int l = threadIdx.x; l < c; l += blockDim.x) piv[l] = perm[l];
        if (threadIdx.x == 0) kout[node] = k;
    }
    cl.sync();  // no CTA leaves while another may still read its offers
}

// shared memory of the loop-form solve for ranks up to kmax: the reciprocals
// of R11's diagonal and the skeleton sort (a power of two >= kmax)
size_t loop_solve_smem(int kmax) {
    size_t P = 1;
    while (P < (size_t)kmax) P <<= 1;
    return (size_t)kmax * sizeof(double) + P * sizeof(int32_t);
}

__device__ void bitonic_sort_i32(int32_t *v, int P) {
    for (int kk = 2; kk <= P; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool asc = (i & kk) == 0;
                    int32_t x = v[i], y = v[ixj];
                    if ((x > y) == asc) { v[i] = y; v[ixj] = x; }
                }
            }
            __syncthreads();
        }
}

// U_i = P [I; G] from G^T = W[p + (k + l) m] (p < k, l < c - k) and the pivot
// order piv: the skeleton sorted by Morton position (its candidates' labels
// cd[.] go to skel), U's column for pivot p the position of piv[p] among the
// sorted skeleton; the largest |G| entry goes to *gmax_bits (non-negative
// doubles order as their bit patterns).  sk: shared scratch of a power of two
// >= k entries.  Called by every thread of the CTA.
template <class Real>
__device__ void id_write_u(int m, int c, int k, const double *W, const int32_t *piv, const int32_t *cd, Real *U,
                           int32_t *skel, int32_t *sk, unsigned long long *gmax_bits) {
    const int nr = c - k;
    int P = 1;
    while (P < k) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) sk[i] = i < k ? piv[i] : INT_MAX;
    __syncthreads();
    bitonic_sort_i32(sk, P);
    for (int64_t e = threadIdx.x; e < (int64_t)c * k; e += blockDim.x) U[e] = (Real)0;
    for (int q = threadIdx.x; q < k; q += blockDim.x) skel[q] = cd[sk[q]];
    __syncthreads();
    // column of U for pivot p: position of piv[p] in the sorted skeleton;
    // the largest |G| entry goes to *gmax_bits (non-negative doubles order as
    // their bit patterns)
    unsigned long long gm = 0;
    for (int l = threadIdx.x >> 5; l <= nr; l += blockDim.x >> 5) {  // l == 0: identity rows, else T column l-1
        for (int p = threadIdx.x & 31; p < k; p += 32) {
            int lo = 0, hi = k - 1, key = piv[p];
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (sk[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            if (l == 0) {
                U[piv[p] + (int64_t)lo * c] = (Real)1;
            } else {
                const double gv = W[p + (int64_t)(k + l - 1) * m];
                U[piv[k + l - 1] + (int64_t)lo * c] = (Real)gv;
                gm = max(gm, (unsigned long long)__double_as_longlong(fabs(gv)));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if ((threadIdx.x & 31) == 0 && gm) atomicMax(gmax_bits, gm);
}

// T = R11^{-1} R12 in float64 (right-looking back substitution in the
// workspace W, which for a float64 block is the block itself), then, with
// write_u, U_i (c x k, column-major, columns in sorted-skeleton order, stored as
// Real) and the sorted skeleton's Morton positions.
template <class Real>
__global__ void __launch_bounds__(QR_THREADS) k_id_solve(int lb, const int32_t *ycnt, const int32_t *cc,
                                                         const int32_t *kk, const int64_t *aoff, const Real *Abase,
                                                         double *Wbase, const int64_t *coff, const int32_t *pivbase,
                                                         const int32_t *cand, void *const *uptr,
                                                         int32_t *const *skptr, unsigned long long *gmax_bits,
                                                         bool write_u) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int a = blockIdx.x, node = lb + a;
    const int m = ycnt[node], c = cc[node], k = kk[node];
    if (k == 0) return;
    double *rinv = reinterpret_cast<double *>(smem_raw);  // 1 / r_ii, one division per row of R11
    int32_t *sk = reinterpret_cast<int32_t *>(rinv + k);
    const Real *A = Abase + aoff[a];
    double *W = Wbase + aoff[a];
    const int32_t *piv = pivbase + coff[a];
    const int32_t *cd = cand + coff[a];
    const int nr = c - k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) rinv[i] = 1.0 / (double)A[i + (int64_t)i * m];
    if ((const void *)A != (const void *)W) {  // float32 block: R12 into the float64 workspace
        for (int l = threadIdx.x >> 5; l < nr; l += blockDim.x >> 5)
            for (int p = threadIdx.x & 31; p < k; p += 32)
                W[p + (int64_t)(k + l) * m] = (double)A[p + (int64_t)(k + l) * m];
    }
    __syncthreads();
    for (int i = k - 1; i >= 0; i--) {
        const double ri = rinv[i];
        for (int l = threadIdx.x; l < nr; l += blockDim.x) {
            double *e = W + i + (int64_t)(k + l) * m;
            *e = *e * ri;
        }
        __syncthreads();
        // the i x nr entries above row i, packed over the threads: (p, l) walks
        // by blockDim.x entries with one division per row, not per entry
        if (i > 0 && (int)threadIdx.x < i * nr) {
            const int dq = blockDim.x / i, dr = blockDim.x % i;
            int p = threadIdx.x % i, l = threadIdx.x / i;
            const Real *ai = A + (int64_t)i * m;
            for (; l < nr; l += dq, p += dr) {
                if (p >= i) { p -= i; l++; if (l >= nr) break; }
                double *wl = W + (int64_t)(k + l) * m;
                wl[p] -= (double)ai[p] * wl[i];
            }
        }
        __syncthreads();
    }
    if (write_u) id_write_u<Real>(m, c, k, W, piv, cd, static_cast<Real *>(uptr[node]), skptr[node], sk, gmax_bits);
}

// eq. (3)'s bound ||G||_max <= f, on G^T = W[p + (k + l) m] as k_id_solve
// leaves it: while some |G[p, l]| > f (the largest, ties to the first in the
// order p + l k), skeleton candidate piv[p] and non-skeleton candidate
// piv[k + l] trade places by a Gauss-Jordan pivot on G.  With g = G[p, l]:
// G'[p, m] = G[p, m] / g and G'[q, m] = G[q, m] - G[q, l] G'[p, m] for m != l,
// G'[q, l] = -(G[q, l] / g) for q != p, G'[p, l] = 1 / g, each operation
// explicitly rounded in this order.  Each exchange multiplies the skeleton
// columns' volume by |g| > f; at most 8k exchanges.  Then U_i from the final
// G and pivot order as k_id_solve writes it, and the count adds to *nex_total.
constexpr int EX_THREADS = 256;

template <class Real>
__global__ void __launch_bounds__(EX_THREADS) k_id_exchange(int lb, const int32_t *ycnt, const int32_t *cc,
                                                            const int32_t *kk, const int64_t *aoff, double *Wbase,
                                                            const int64_t *coff, int32_t *pivbase,
                                                            const int32_t *cand, void *const *uptr,
                                                            int32_t *const *skptr, unsigned long long *gmax_bits,
                                                            double f, unsigned long long *nex_total) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t *sk = reinterpret_cast<int32_t *>(smem_raw);
    __shared__ long long s_key[EX_THREADS / 32];
    __shared__ int s_idx[EX_THREADS / 32];
    __shared__ int s_p, s_l;
    __shared__ double s_g;
    const int a = blockIdx.x, node = lb + a;
    const int m = ycnt[node], c = cc[node], k = kk[node];
    if (k == 0) return;
    double *W = Wbase + aoff[a];
    int32_t *piv = pivbase + coff[a];
    const int nr = c - k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int nex = 0;
    while (nr > 0 && nex < 8 * k) {
        long long bk = -1;
        int bi = INT_MAX;
        for (int l = warp; l < nr; l += nwarps)
            for (int p = lane; p < k; p += 32)
                argmax_key(bk, bi, __double_as_longlong(fabs(W[p + (int64_t)(k + l) * m])), p + l * k);
        for (int o = 16; o > 0; o >>= 1) {
            const long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            argmax_key(bk, bi, k2, i2);
        }
        if (lane == 0) { s_key[warp] = bk; s_idx[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nwarps; w++) argmax_key(bk, bi, s_key[w], s_idx[w]);
            s_p = -1;
            if (__longlong_as_double(bk) > f) {
                s_p = bi % k;
                s_l = bi / k;
                s_g = W[s_p + (int64_t)(k + s_l) * m];
            }
        }
        __syncthreads();
        const int p = s_p, l = s_l;
        const double g = s_g;
        if (p < 0) break;
        double *gl = W + (int64_t)(k + l) * m;  // column l of G^T
        for (int mm = threadIdx.x; mm < nr; mm += blockDim.x)
            if (mm != l) W[p + (int64_t)(k + mm) * m] = __ddiv_rn(W[p + (int64_t)(k + mm) * m], g);
        __syncthreads();
        for (int mm = warp; mm < nr; mm += nwarps) {
            if (mm == l) continue;
            double *gm = W + (int64_t)(k + mm) * m;
            const double tp = gm[p];
            for (int q = lane; q < k; q += 32)
                if (q != p) gm[q] = __dsub_rn(gm[q], __dmul_rn(gl[q], tp));
        }
        __syncthreads();
        for (int q = threadIdx.x; q < k; q += blockDim.x)
            if (q != p) gl[q] = -__ddiv_rn(gl[q], g);
        if (threadIdx.x == 0) {
            gl[p] = __ddiv_rn(1.0, g);
            const int32_t t = piv[p];
            piv[p] = piv[k + l];
            piv[k + l] = t;
        }
        __syncthreads();
        nex++;
    }
    if (threadIdx.x == 0 && nex > 0) atomicAdd(nex_total, (unsigned long long)nex);
    id_write_u<Real>(m, c, k, W, piv, cand + coff[a], static_cast<Real *>(uptr[node]), skptr[node], sk, gmax_bits);
}

// The same solve and U for a float32 block of rank up to 128, one lane per
// column of R12: a warp takes 32 columns and runs the back substitution on all
// of them at once (a node's columns are split over several CTAs, so the few
// wide nodes of the upper levels do not run on a handful of SMs).  The
// multiplier r_pi is the same for every lane and comes from R11's strict upper
// triangle, staged once per node in float64 (a shared-memory broadcast, with no
// per-lane conversion); the columns stay in shared memory (entry p of a lane's
// column at p * 32 + lane, so a warp's accesses never conflict).  Every lane
// of every float64 instruction does useful work (float64 runs at 1/64 of the
// float32 rate on this GPU), and no block barrier sits inside the solve.  Each
// entry takes the operations of the loop form in the same order (subtract
// r_pi * t_i for i descending, then scale by 1 / r_pp at its own row), so the
// results are bit-identical.  The column of U that each pivot lands in is its
// rank among the skeleton labels (no sort).
constexpr int SOLVE_WARPS = 4;
constexpr int SOLVE_KMAX = 128;

size_t solve_cols_smem(int kcap) {
    const size_t tri = (size_t)kcap * (kcap - 1) / 2;
    return (tri + kcap + (size_t)SOLVE_WARPS * 32 * kcap) * sizeof(double) + 2 * (size_t)kcap * sizeof(int32_t);
}

__global__ void __launch_bounds__(SOLVE_WARPS * 32) k_id_solve_cols(int kcap, int lb, const int32_t *ycnt,
                                                                    const int32_t *cc, const int32_t *kk,
                                                                    const int64_t *aoff, const float *Abase,
                                                                    const int64_t *coff, const int32_t *pivbase,
                                                                    const int32_t *cand, void *const *uptr,
                                                                    int32_t *const *skptr,
                                                                    unsigned long long *gmax_bits) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *W = reinterpret_cast<double *>(smem_raw);   // SOLVE_WARPS x kcap x 32
    double *tri = W + (size_t)SOLVE_WARPS * 32 * kcap;  // r_pi (p < i) at i (i - 1) / 2 + p
    double *rinv = tri + (size_t)kcap * (kcap - 1) / 2;
    int32_t *pv = reinterpret_cast<int32_t *>(rinv + kcap), *pos = pv + kcap;
    const int a = blockIdx.x, node = lb + a;
    const int m = ycnt[node], c = cc[node], k = kk[node];
    if (k == 0) return;
    const float *A = Abase + aoff[a];
    const int32_t *piv = pivbase + coff[a];
    const int32_t *cd = cand + coff[a];
    const int nr = c - k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // the node's columns are split over gridDim.y CTAs of nwarps * 32 columns;
    // slice 0 also writes the skeleton and U's identity rows
    const int slice = blockIdx.y, width = nwarps * 32;
    if (slice > 0 && slice * width >= nr) return;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        rinv[i] = 1.0 / (double)A[i + (int64_t)i * m];
        pv[i] = piv[i];
    }
    for (int i = warp; i < k; i += nwarps)
        for (int p = lane; p < i; p += 32) tri[i * (i - 1) / 2 + p] = (double)A[p + (int64_t)i * m];
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const int key = pv[i];
        int r = 0;
        for (int q = 0; q < k; q++) r += pv[q] < key;
        pos[i] = r;
    }
    __syncthreads();
    float *U = static_cast<float *>(uptr[node]);
    if (slice == 0) {
        int32_t *skel = skptr[node];
        for (int i = threadIdx.x; i < k; i += blockDim.x) skel[pos[i]] = cd[pv[i]];
        for (int i = warp; i < k; i += nwarps)  // identity row of skeleton point i, in full
            for (int q = lane; q < k; q += 32) U[pv[i] + (int64_t)q * c] = q == pos[i] ? 1.0f : 0.0f;
    }
    double *w = W + (size_t)warp * 32 * kcap + lane;
    unsigned long long gm = 0;
    for (int l0 = slice * width + warp * 32; l0 < nr; l0 += gridDim.y * width) {  // (warp-uniform)
        const int l = l0 + lane;
        const bool act = l < nr;
        const float *r12 = A + (int64_t)(k + (act ? l : 0)) * m;
        for (int p = 0; p < k; p++) w[p * 32] = act ? (double)r12[p] : 0.0;
        for (int i = k - 1; i >= 0; i--) {
            const double wi = w[i * 32] * rinv[i];
            w[i * 32] = wi;
            const double *ri = tri + i * (i - 1) / 2;
            for (int p = 0; p < i; p++) w[p * 32] -= ri[p] * wi;
        }
        if (act) {
            const int64_t row = piv[k + l];
            for (int p = 0; p < k; p++) {
                const double g = w[p * 32];
                U[row + (int64_t)pos[p] * c] = (float)g;
                gm = max(gm, (unsigned long long)__double_as_longlong(fabs(g)));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if (lane == 0 && gm) atomicMax(gmax_bits, gm);
}

__global__ void k_ku_sizes(int lb, int nl, const int32_t *kk, const int32_t *cc, int64_t *szk, int64_t *szu) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nl) return;
    int i = lb + a;
    szk[a] = kk[i];
    szu[a] = (int64_t)kk[i] * cc[i];
}

__global__ void k_set_ptrs2(int lb, int nl, int32_t *kbase, const int64_t *koff, int32_t **skptr,
                            unsigned char *ubase, const int64_t *uoff, int esize, void **uptr) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nl) return;
    skptr[lb + a] = kbase + koff[a];
    uptr[lb + a] = ubase + uoff[a] * esize;
}

// contiguous skeletons (node order) and their coordinates (float32: relative
// to the node's centre c, or absolute when c is null)
__global__ void k_compact_skel(int nn, const int32_t *kk, const int64_t *off, int32_t *const *skptr, int32_t *skel,
                               const double *x0, const double *x1, const double *x2, int d, double *s0, double *s1,
                               double *s2, const double *c0, const double *c1, const double *c2, float *r0,
                               float *r1, float *r2) {
    int i = blockIdx.x;
    if (i >= nn) return;
    int k = kk[i];
    const int32_t *src = skptr[i];
    const double o0 = c0 ? c0[i] : 0.0, o1 = c1 && d > 1 ? c1[i] : 0.0, o2 = c2 && d > 2 ? c2[i] : 0.0;
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
        int32_t p = src[q];
        int64_t o = off[i] + q;
        skel[o] = p;
        s0[o] = x0[p];
        r0[o] = (float)(x0[p] - o0);
        if (d > 1) { s1[o] = x1[p]; r1[o] = (float)(x1[p] - o1); }
        if (d > 2) { s2[o] = x2[p]; r2[o] = (float)(x2[p] - o2); }
    }
}

// launch the QR with the smallest register slice that holds the level's tallest
// block (rows per lane = ceil(mmax / 32)), or the loop form above 1024 rows
// threads of a k_cpqr CTA for a level with at most cmax columns: a QR step is
// a chain of block barriers and one-thread scalar work, so narrow blocks run
// in small CTAs, several to a SM, which hide each other's chains (measured:
// 128 threads up to 128 columns beat 256 or 512)
int qr_threads(int cmax) { return cmax <= 128 ? 128 : QR_THREADS; }

template <class Real>
void launch_cpqr(int nl, size_t smem, int mmax, int lb, const int32_t *ycnt, const int32_t *cc, const int64_t *aoff,
                 Real *A, double tol, int32_t *kout, const int64_t *coff, int32_t *piv, cudaStream_t s,
                 int cmax = 1 << 30) {
    const int nthr = qr_threads(cmax);
#define H2_QR(R) k_cpqr<Real, R><<<nl, nthr, smem, s>>>(lb, ycnt, cc, aoff, A, tol, kout, coff, piv)
    int rpl = (mmax + 31) / 32;
    // the float64 form is bound by the float64 pipe, not by load latency: the
    // loop form keeps its register count (and occupancy) low
    if (sizeof(Real) == 8) H2_QR(0);
    else if (rpl <= 4) H2_QR(4);
    else if (rpl <= 8) H2_QR(8);
    else if (rpl <= 12) H2_QR(12);
    else if (rpl <= 16) H2_QR(16);
    else if (rpl <= 24) H2_QR(24);
    else if (rpl <= 32) H2_QR(32);
    else H2_QR(0);
#undef H2_QR
}

template <class Real>
void set_qr_attrs() {
    for (const void *f : {(const void *)k_cpqr<Real, 4>, (const void *)k_cpqr<Real, 8>, (const void *)k_cpqr<Real, 12>,
                          (const void *)k_cpqr<Real, 16>, (const void *)k_cpqr<Real, 24>,
                          (const void *)k_cpqr<Real, 32>, (const void *)k_cpqr<Real, 0>})
        // (all variants are instantiated; the float64 form launches the loop variant)
        H2_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_LIMIT));
}

size_t qr_smem(int cmax, int mmax, size_t esize = sizeof(double)) {
    return (size_t)cmax * (3 * sizeof(double) + sizeof(int32_t) + 1) + (size_t)mmax * esize + 64;
}

// k_cpqr_df_cl: three float64 arrays, two int32 maps and a flag by column, the reflector
size_t qr_smem_cl(int cmax, int mmax) {
    return (size_t)cmax * (3 * sizeof(double) + 2 * sizeof(int32_t) + 1) + (size_t)mmax * sizeof(float2) + 64;
}

}  // namespace

void construct_impl(h2_matrix_s *A, h2_hidr_s *h) {
    h2_tree_s *t = A->tree;
    cudaStream_t s = A->stream;
    const int nn = t->nnodes, d = t->d;
    const bool f64 = A->prec == H2_PREC_FP64;
    const size_t esize = f64 ? sizeof(double) : sizeof(float);
    // float64 form, 3D Coulomb, float-float QR: the blocks are evaluated in
    // float-float arithmetic too and handed to the QR as float pairs
    const bool dfblocks = f64 && !A->fp64_qr && A->kid == H2_K_COULOMB && d == 3;
    A->k.alloc(nn, s);
    A->c.alloc(nn, s);
    DevBuf<unsigned long long> gmax, nexd;  // largest |G| entry over all nodes (float64 bits); exchanges
    gmax.alloc(1, s);
    nexd.alloc(1, s);
    H2_CUDA(cudaMemsetAsync(gmax.p, 0, sizeof(unsigned long long), s));
    H2_CUDA(cudaMemsetAsync(nexd.p, 0, sizeof(unsigned long long), s));
    H2_CUDA(cudaMemsetAsync(A->k.p, 0, nn * sizeof(int32_t), s));
    H2_CUDA(cudaMemsetAsync(A->c.p, 0, nn * sizeof(int32_t), s));
    DevBuf<int32_t *> skptr;
    skptr.alloc(nn, s);
    A->uptr.alloc(nn, s);
    H2_CUDA(cudaMemsetAsync(skptr.p, 0, nn * sizeof(int32_t *), s));
    H2_CUDA(cudaMemsetAsync(A->uptr.p, 0, nn * sizeof(void *), s));
    int dev = 0, sm_count = 0;
    H2_CUDA(cudaGetDevice(&dev));
    H2_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
    std::vector<DevBuf<int32_t>> skbufs(t->nlevels);
    A->ubufs.resize(t->nlevels);
    A->kmax_level.assign(t->nlevels, 0);
    A->cmax_level.assign(t->nlevels, 0);
    static std::once_flag attr;
    std::call_once(attr, [] {
        set_qr_attrs<double>();
        set_qr_attrs<float>();
        H2_CUDA(cudaFuncSetAttribute(k_cpqr_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_LIMIT));
        H2_CUDA(cudaFuncSetAttribute(k_cpqr_df_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_LIMIT));
        H2_CUDA(cudaFuncSetAttribute(k_id_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_LIMIT));
        H2_CUDA(cudaFuncSetAttribute(k_id_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_LIMIT));
        H2_CUDA(cudaFuncSetAttribute(k_keval_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_LIMIT));
        H2_CUDA(cudaFuncSetAttribute(k_id_solve_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)solve_cols_smem(SOLVE_KMAX)));
    });
    cudaEvent_t e0, e1;
    H2_CUDA(cudaEventCreate(&e0));
    H2_CUDA(cudaEventCreate(&e1));
    H2_CUDA(cudaEventRecord(e0, s));
    const std::vector<int32_t> yc = read_vec(h->ycnt.p, nn, s);
    DevBuf<int64_t> szc, sza, coff, aoff, szk, szu, koff, uoff;
    DevBuf<int32_t> cand, piv;
    DevBuf<unsigned char> Ablk;
    DevBuf<double> Wf;  // float64 workspace of the solve when the block is float32
    DevBuf<double> Rq;  // R in pivot order, from the cluster QR
    for (int l = t->nlevels - 1; l >= 1; l--) {
        const int lb = t->lptr[l], nl = t->lptr[l + 1] - lb;
        szc.alloc(nl, s); sza.alloc(nl, s); coff.alloc(nl + 1, s); aoff.alloc(nl + 1, s);
        k_cand_sizes<<<blocks_for(nl, 128), 128, 0, s>>>(lb, nl, t->nchild.p, t->fchild.p, t->begin.p, t->end.p,
                                                          A->k.p, h->ycnt.p, A->c.p, szc.p, sza.p);
        H2_LAUNCH("k_cand_sizes");
        scan_exclusive(szc.p, coff.p, nl, s);
        scan_exclusive(sza.p, aoff.p, nl, s);
        std::vector<int64_t> cs = read_vec(szc.p, nl, s);
        int64_t ctot = read_scalar(coff.p + nl, s), atot = read_scalar(aoff.p + nl, s);
        int cmax = 0;
        for (int64_t v : cs) cmax = std::max<int>(cmax, (int)v);
        A->cmax_level[l] = cmax;
        if (ctot == 0) continue;
        const int mmax = h->ymax_level[l];
        if (qr_smem(cmax, mmax, esize) > SMEM_LIMIT)
            fail(H2_ERR_UNIMPLEMENTED, "kernel block too large for the single-CTA QR (candidates " +
                                           std::to_string(cmax) + ", rows " + std::to_string(mmax) + ")");
        cand.alloc(ctot, s);
        piv.alloc(ctot, s);
        Ablk.alloc((size_t)atot * esize, s);
        k_gather_cand<<<nl, 128, 0, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->c.p, A->k.p, skptr.p, coff.p,
                                         cand.p);
        H2_LAUNCH("k_gather_cand");
        dim3 kg(nl, std::max(1, std::min(16, (int)((int64_t)cmax * mmax / (256 * 64)))));
        {
            ProfScope ps(KT_KEVAL, s);
            if (dfblocks) {
                ensure_df_tree(t, s);
                keval_df(t, nl, (int)kg.y, lb, h->ycnt.p, A->c.p, h->yptr.p, cand.p, coff.p, aoff.p,
                         reinterpret_cast<float2 *>(Ablk.p), s);
            } else if (f64) {
                k_keval_f64<<<kg, 256, 0, s>>>(lb, h->ycnt.p, A->c.p, h->yptr.p, cand.p, coff.p, aoff.p, t->xs[0].p,
                                               t->xs[1].p, t->xs[2].p, d, A->kid, A->kp[0],
                                               reinterpret_cast<double *>(Ablk.p));
            } else {
                size_t sm = (size_t)(cmax + mmax) * 3 * sizeof(float);
                if (sm > SMEM_LIMIT) fail(H2_ERR_UNIMPLEMENTED, "kernel block too large for the float32 evaluation");
                k_keval_f32<<<kg, 256, sm, s>>>(lb, h->ycnt.p, A->c.p, h->yptr.p, cand.p, coff.p, aoff.p, t->xs[0].p,
                                                t->xs[1].p, t->xs[2].p, t->cen[0].p, t->cen[1].p, t->cen[2].p, d,
                                                A->kid, A->kp[0], reinterpret_cast<float *>(Ablk.p));
            }
            H2_LAUNCH("k_keval");
        }
        A->evals_block += (double)atot;
        // where R goes (float64 form): the block itself, or Rq from the cluster QR
        double *Rb = reinterpret_cast<double *>(Ablk.p);
        {
            ProfScope ps(KT_CPQR, s);
            // float-float QR: one node a CTA; a wide level with fewer nodes than
            // SMs takes one node per cluster of QR_CL CTAs, which puts every SM
            // to work.  (On levels with many nodes the cluster form measured
            // slower: with a few columns a warp per step, its per-step barriers
            // outweigh the blocks staying in L2.)
            if (f64 && !A->fp64_qr && qr_threads(cmax) == QR_THREADS && nl < sm_count) {
                if (qr_smem_cl(cmax, mmax) > SMEM_LIMIT)
                    fail(H2_ERR_UNIMPLEMENTED, "kernel block too large for the cluster QR");
                Rq.alloc(atot, s);
                Rb = Rq.p;
                k_cpqr_df_cl<<<(unsigned)nl * QR_CL, QR_THREADS, qr_smem_cl(cmax, mmax), s>>>(
                    lb, h->ycnt.p, A->c.p, aoff.p, reinterpret_cast<double *>(Ablk.p), Rb, A->id_tol, A->k.p,
                    coff.p, piv.p, dfblocks ? 1 : 0);
            } else if (f64 && !A->fp64_qr)
                k_cpqr_df<<<nl, qr_threads(cmax), qr_smem(cmax, mmax, esize), s>>>(
                    lb, h->ycnt.p, A->c.p, aoff.p, reinterpret_cast<double *>(Ablk.p), A->id_tol, A->k.p, coff.p,
                    piv.p, dfblocks ? 1 : 0);
            else if (f64)
                launch_cpqr<double>(nl, qr_smem(cmax, mmax, esize), mmax, lb, h->ycnt.p, A->c.p, aoff.p,
                                    reinterpret_cast<double *>(Ablk.p), A->id_tol, A->k.p, coff.p, piv.p, s, cmax);
            else
                launch_cpqr<float>(nl, qr_smem(cmax, mmax, esize), mmax, lb, h->ycnt.p, A->c.p, aoff.p,
                                   reinterpret_cast<float *>(Ablk.p), A->id_tol, A->k.p, coff.p, piv.p, s, cmax);
            H2_LAUNCH("k_cpqr");
        }
        szk.alloc(nl, s); szu.alloc(nl, s); koff.alloc(nl + 1, s); uoff.alloc(nl + 1, s);
        k_ku_sizes<<<blocks_for(nl, 128), 128, 0, s>>>(lb, nl, A->k.p, A->c.p, szk.p, szu.p);
        H2_LAUNCH("k_ku_sizes");
        scan_exclusive(szk.p, koff.p, nl, s);
        scan_exclusive(szu.p, uoff.p, nl, s);
        std::vector<int64_t> ks = read_vec(szk.p, nl, s);
        int64_t ktot = read_scalar(koff.p + nl, s), utot = read_scalar(uoff.p + nl, s);
        int kmax = 0;
        for (int64_t v : ks) kmax = std::max<int>(kmax, (int)v);
        A->kmax_level[l] = kmax;
        A->kmax = std::max(A->kmax, kmax);
        for (int a = 0; a < nl; a++) {  // Householder QR flops of an m x c block stopped at rank k
            double kk = (double)ks[a], cc = (double)cs[a], mm = (double)yc[lb + a];
            if (kk > 0) A->flops_qr += 4 * mm * cc * kk - 2 * kk * kk * (mm + cc) + 4.0 / 3.0 * kk * kk * kk;
        }
        skbufs[l].alloc(ktot > 0 ? ktot : 1, s);
        A->ubufs[l].alloc((size_t)(utot > 0 ? utot : 1) * esize, s);
        k_set_ptrs2<<<blocks_for(nl, 128), 128, 0, s>>>(lb, nl, skbufs[l].p, koff.p, skptr.p, A->ubufs[l].p,
                                                         uoff.p, (int)esize, A->uptr.p);
        H2_LAUNCH("k_set_ptrs2");
        {
            ProfScope ps(KT_SOLVE, s);
            // float32 blocks: one lane per column; float64 blocks (and larger
            // ranks): the loop form, whose 512-thread CTAs hold their share of
            // the float64 pipe beside the other float64 kernels (measured at
            // 1M: 16.8 ms against 21.8 for the column form)
            const bool cols = !f64 && kmax <= SOLVE_KMAX && A->g_bound == 0.0;
            const bool bound = A->g_bound > 0.0;  // exchanges, then U (k_id_exchange)
            int nrmax = 0;  // most columns of R12 in a node of the level
            for (int a = 0; a < nl; a++) nrmax = std::max(nrmax, (int)(cs[a] - ks[a]));
            const dim3 sg(nl, std::max(1, (nrmax + SOLVE_WARPS * 32 - 1) / (SOLVE_WARPS * 32)));
            if (cols) {
                k_id_solve_cols<<<sg, SOLVE_WARPS * 32, solve_cols_smem(kmax), s>>>(
                    kmax, lb, h->ycnt.p, A->c.p, A->k.p, aoff.p, reinterpret_cast<const float *>(Ablk.p), coff.p,
                    piv.p, cand.p, A->uptr.p, skptr.p, gmax.p);
            } else if (f64) {
                k_id_solve<double><<<nl, qr_threads(cmax), loop_solve_smem(kmax), s>>>(
                    lb, h->ycnt.p, A->c.p, A->k.p, aoff.p, Rb, Rb, coff.p, piv.p, cand.p, A->uptr.p, skptr.p, gmax.p,
                    !bound);
            } else {
                Wf.alloc(atot, s);
                k_id_solve<float><<<nl, qr_threads(cmax), loop_solve_smem(kmax), s>>>(
                    lb, h->ycnt.p, A->c.p, A->k.p, aoff.p, reinterpret_cast<float *>(Ablk.p), Wf.p, coff.p, piv.p,
                    cand.p, A->uptr.p, skptr.p, gmax.p, !bound);
            }
            H2_LAUNCH("k_id_solve");
            if (bound) {
                const size_t sm = loop_solve_smem(kmax) - (size_t)kmax * sizeof(double);  // the sort scratch
                if (f64)
                    k_id_exchange<double><<<nl, EX_THREADS, sm, s>>>(
                        lb, h->ycnt.p, A->c.p, A->k.p, aoff.p, Rb, coff.p, piv.p,
                        cand.p, A->uptr.p, skptr.p, gmax.p, A->g_bound, nexd.p);
                else
                    k_id_exchange<float><<<nl, EX_THREADS, sm, s>>>(lb, h->ycnt.p, A->c.p, A->k.p, aoff.p, Wf.p,
                                                                    coff.p, piv.p, cand.p, A->uptr.p, skptr.p,
                                                                    gmax.p, A->g_bound, nexd.p);
                H2_LAUNCH("k_id_exchange");
            }
        }
        A->ktotal += ktot;
        A->utotal += utot;
    }
    // skeletons contiguous in node order, with coordinates for the matvec
    A->sk_off.alloc(nn + 1, s);
    scan_exclusive_i32(A->k.p, A->sk_off.p, nn, s);
    int64_t kt = read_scalar(A->sk_off.p + nn, s);
    A->skel.alloc(kt > 0 ? kt : 1, s);
    for (int k = 0; k < 3; k++) {
        A->skc[k].alloc(kt > 0 ? kt : 1, s);
        A->skr[k].alloc(kt > 0 ? kt : 1, s);
    }
    // float32 skeleton coordinates: relative to the node's centre, or absolute
    // for cos(x . y)
    const bool rel = A->kid != H2_K_COSDOT;
    k_compact_skel<<<std::max(1, nn), 128, 0, s>>>(
        nn, A->k.p, A->sk_off.p, skptr.p, A->skel.p, t->xs[0].p, t->xs[1].p, t->xs[2].p, d, A->skc[0].p,
        A->skc[1].p, A->skc[2].p, rel ? t->cen[0].p : nullptr, rel ? t->cen[1].p : nullptr,
        rel ? t->cen[2].p : nullptr, A->skr[0].p, A->skr[1].p, A->skr[2].p);
    H2_LAUNCH("k_compact_skel");
    H2_CUDA(cudaEventRecord(e1, s));
    H2_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    A->ms_construct = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const unsigned long long gb = read_scalar(gmax.p, s);
    double gv;
    memcpy(&gv, &gb, sizeof gv);
    A->g_max = gv;
    A->exchanges = (int64_t)read_scalar(nexd.p, s);
}

namespace {
// A[r + l m] = kappa(y_{ids[r]}, x_l) for the calibration block K(Z2*, Z1)
__global__ void k_calib_block(const int32_t *ids, int m, int c, const double *y0, const double *y1, const double *y2,
                              const double *x0, const double *x1, const double *x2, int d, int kid, double kp0,
                              double *A) {
    int64_t total = (int64_t)m * c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int r = (int)(e % m), l = (int)(e / m);
        int32_t y = ids[r];
        A[e] = h2_kxy(kid, kp0, d, y0[y], d > 1 ? y1[y] : 0.0, d > 2 ? y2[y] : 0.0, x0[l], d > 1 ? x1[l] : 0.0,
                      d > 2 ? x2[l] : 0.0);
    }
}

// per candidate l (block): num_l = sum_b (kappa(z1[piv l], z2 b) - sum_p T[p, l] kappa(z1[piv p], z2 b))^2
// for l >= k (0 for skeleton columns), den_l = sum_b kappa(z1[piv l], z2 b)^2
__global__ void k_calib_err(const double *A, int m, int c, int k, const int32_t *piv, const double *a0,
                            const double *a1, const double *a2, int n1, const double *b0, const double *b1,
                            const double *b2, int n2, int d, int kid, double kp0, double *num, double *den) {
    __shared__ double red[2][32];
    int l = blockIdx.x;
    if (l >= c) return;
    int pl = piv[l];
    double sn = 0.0, sd = 0.0;
    for (int b = threadIdx.x; b < n2; b += blockDim.x) {
        double zb0 = b0[b], zb1 = d > 1 ? b1[b] : 0.0, zb2 = d > 2 ? b2[b] : 0.0;
        double kv = h2_kxy(kid, kp0, d, a0[pl], d > 1 ? a1[pl] : 0.0, d > 2 ? a2[pl] : 0.0, zb0, zb1, zb2);
        sd += kv * kv;
        if (l >= k) {
            double s = 0.0;
            for (int p = 0; p < k; p++) {
                int pp = piv[p];
                s += A[p + (int64_t)l * m] *
                     h2_kxy(kid, kp0, d, a0[pp], d > 1 ? a1[pp] : 0.0, d > 2 ? a2[pp] : 0.0, zb0, zb1, zb2);
            }
            double e = kv - s;
            sn += e * e;
        }
    }
    sn = warp_sum(sn);
    sd = warp_sum(sd);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = sn; red[1][warp] = sd; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tn = 0.0, td = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { tn += red[0][w]; td += red[1][w]; }
        num[l] = tn;
        den[l] = td;
    }
    (void)n1;
}
}  // namespace

double calib_error_gpu(int d, int kid, double kp0, double id_tol, const double *const z1s[3], int n1,
                       const DRPoints &z2, const long long *z2_box, int n2, int g, int *k_out, int *m_out,
                       cudaStream_t s) {
    const double *const *z2s = z2.x;
    DevBuf<int32_t> ids;
    ids.alloc(n2, s);
    int m = (int)datareduct_one(z2, d, n2, g, z2_box, ids.p, s);
    const int c = n1;
    DevBuf<double> A;
    A.alloc((size_t)m * c, s);
    k_calib_block<<<blocks_for((int64_t)m * c, 256), 256, 0, s>>>(ids.p, m, c, z2s[0], z2s[1], z2s[2], z1s[0],
                                                                   z1s[1], z1s[2], d, kid, kp0, A.p);
    H2_LAUNCH("k_calib_block");
    // one-node level: ycnt = m, c, offsets 0
    int32_t hv[2] = {m, c};
    int64_t offs[4] = {0, (int64_t)m * c, 0, c};
    DevBuf<int32_t> mc, kk, piv, skel;
    DevBuf<int64_t> off;
    DevBuf<double> U;
    DevBuf<void *> up;
    DevBuf<int32_t *> sp;
    mc.alloc(2, s); kk.alloc(1, s); piv.alloc(c, s); off.alloc(4, s);
    H2_CUDA(cudaMemcpyAsync(mc.p, hv, sizeof hv, cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaMemcpyAsync(off.p, offs, sizeof offs, cudaMemcpyHostToDevice, s));
    static std::once_flag attr;
    std::call_once(attr, [] {
        set_qr_attrs<double>();
        H2_CUDA(cudaFuncSetAttribute(k_id_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_LIMIT));
    });
    if (qr_smem(c, m) > SMEM_LIMIT) fail(H2_ERR_UNIMPLEMENTED, "calibration block too large");
    launch_cpqr<double>(1, qr_smem(c, m), m, 0, mc.p, mc.p + 1, off.p, A.p, id_tol, kk.p, off.p + 2, piv.p, s);
    H2_LAUNCH("k_cpqr (calibration)");
    int k = read_scalar(kk.p, s);
    U.alloc((size_t)std::max(1, k) * c, s);
    skel.alloc(std::max(1, k), s);
    up.alloc(1, s);
    sp.alloc(1, s);
    H2_CUDA(cudaMemcpyAsync(up.p, &U.p, sizeof(double *), cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaMemcpyAsync(sp.p, &skel.p, sizeof(int32_t *), cudaMemcpyHostToDevice, s));
    DevBuf<int32_t> cand;
    cand.alloc(c, s);
    std::vector<int32_t> iota(c);
    for (int i = 0; i < c; i++) iota[i] = i;
    H2_CUDA(cudaMemcpyAsync(cand.p, iota.data(), c * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (k > 0) {
        DevBuf<unsigned long long> gm;
        gm.alloc(1, s);
        H2_CUDA(cudaMemsetAsync(gm.p, 0, sizeof(unsigned long long), s));
        k_id_solve<double><<<1, QR_THREADS, loop_solve_smem(k), s>>>(
            0, mc.p, mc.p + 1, kk.p, off.p, A.p, A.p, off.p + 2, piv.p, cand.p, up.p, sp.p, gm.p, true);
        H2_LAUNCH("k_id_solve (calibration)");
    }
    DevBuf<double> num, den;
    num.alloc(c, s);
    den.alloc(c, s);
    k_calib_err<<<c, 256, 0, s>>>(A.p, m, c, k, piv.p, z1s[0], z1s[1], z1s[2], n1, z2s[0], z2s[1], z2s[2], n2, d,
                                  kid, kp0, num.p, den.p);
    H2_LAUNCH("k_calib_err");
    std::vector<double> nv = read_vec(num.p, c, s), dv = read_vec(den.p, c, s);
    double tn = 0.0, td = 0.0;
    for (int l = 0; l < c; l++) { tn += nv[l]; td += dv[l]; }
    if (k_out) *k_out = k;
    if (m_out) *m_out = m;
    return td > 0.0 ? sqrt(tn / td) : 0.0;
}

void matrix_rebind(h2_matrix_s *A, cudaStream_t s) {
    A->stream = s;
    A->k.rebind(s);
    A->c.rebind(s);
    A->sk_off.rebind(s);
    A->skel.rebind(s);
    for (int k = 0; k < 3; k++) {
        A->skc[k].rebind(s);
        A->skr[k].rebind(s);
    }
    A->uptr.rebind(s);
    for (auto &b : A->ubufs) b.rebind(s);
    A->far_tiles.rebind(s);
    A->far_blk.rebind(s);
    A->near_blk.rebind(s);
    A->far_boff.rebind(s);
    A->near_boff.rebind(s);
    for (int k = 0; k < 3; k++) A->skdf[k].rebind(s);
}

}  // namespace h2
