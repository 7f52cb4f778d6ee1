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

#include "h2_internal.cuh"

// Scratch of h2_exact_rows_noalloc: the right-hand side permuted to Morton
// order.  It lives in the library image, so every GPU that loads the library
// holds these H2_NOALLOC_MAX_N doubles (8 MiB) until the process exits.
#define H2_NOALLOC_MAX_N (1 << 20)
static __device__ __align__(256) double g_noalloc_zm[H2_NOALLOC_MAX_N];

namespace h2 {
namespace {

constexpr int MV_THREADS = 256;
constexpr int NB_TILE = 256;  // source points staged per pass in the N-body kernels
constexpr int MAX_TPT = 8;    // targets per thread in the N-body kernels

__global__ void k_perm_in(const double *x, const int32_t *perm, int64_t n, double *xm) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) xm[p] = x[perm[p]];
}

__global__ void k_perm_out(const double *ym, const int32_t *perm, int64_t n, double *y) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) y[perm[p]] = ym[p];
}

// xh_i[a] = sum_r U_i[r, a] in[r]; one CTA per node, one warp per column
__global__ void k_upward(int lb, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                         const int32_t *kk, const int32_t *cc, double *const *uptr, const int64_t *sk_off,
                         const double *xm, double *xh) {
    extern __shared__ double sin_[];
    int i = lb + blockIdx.x;
    int k = kk[i], c = cc[i];
    if (k == 0) return;
    const double *in = nchild[i] == 0 ? xm + begin[i] : xh + sk_off[fchild[i]];
    for (int r = threadIdx.x; r < c; r += blockDim.x) sin_[r] = in[r];
    __syncthreads();
    const double *U = uptr[i];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = warp; a < k; a += nw) {
        const double *col = U + (int64_t)a * c;
        double s = 0.0;
        for (int r = lane; r < c; r += 32) s += col[r] * sin_[r];
        s = warp_sum(s);
        if (lane == 0) xh[sk_off[i] + a] = s;
    }
}

// out = U_i zh_i, added to the children's zh (parent) or to y (leaf)
__global__ void k_downward(int lb, const int32_t *nchild, const int32_t *fchild, const int32_t *begin,
                           const int32_t *kk, const int32_t *cc, double *const *uptr, const int64_t *sk_off,
                           double *zh, double *ym) {
    extern __shared__ double sz_[];
    int i = lb + blockIdx.x;
    int k = kk[i], c = cc[i];
    if (k == 0) return;
    const double *z = zh + sk_off[i];
    for (int a = threadIdx.x; a < k; a += blockDim.x) sz_[a] = z[a];
    __syncthreads();
    const double *U = uptr[i];
    double *out = nchild[i] == 0 ? ym + begin[i] : zh + sk_off[fchild[i]];
    for (int r = threadIdx.x; r < c; r += blockDim.x) {
        double s = 0.0;
        for (int a = 0; a < k; a++) s += U[r + (int64_t)a * c] * sz_[a];
        out[r] += s;
    }
}

// N-body accumulation: targets t (owned by this CTA) += sum_s kappa(t, s) w_s
// over a list of source blocks.  kind 0: coupling (sources = far skeletons),
// kind 1: nearfield (sources = near leaves' points).
template <int TPT>
__global__ void __launch_bounds__(MV_THREADS) k_nbody(int kind, const int32_t *kk, const int64_t *sk_off,
                                                      const double *s0, const double *s1, const double *s2,
                                                      const double *xh, double *zh, const int32_t *begin,
                                                      const int32_t *end, const double *x0, const double *x1,
                                                      const double *x2, const double *xm, double *ym,
                                                      const int64_t *lptr, const int32_t *lidx,
                                                      const int32_t *nodes, int d, int kid, double kp0) {
    __shared__ double sx[3][NB_TILE], sw[NB_TILE];
    const int i = nodes[blockIdx.x];
    // target range of this CTA
    int64_t tb, nt;
    const double *tx0, *tx1, *tx2;
    if (kind == 0) { tb = sk_off[i]; nt = kk[i]; tx0 = s0; tx1 = s1; tx2 = s2; }
    else { tb = begin[i]; nt = end[i] - begin[i]; tx0 = x0; tx1 = x1; tx2 = x2; }
    for (int64_t chunk = 0; chunk < nt; chunk += (int64_t)MV_THREADS * TPT) {
        double t[TPT][3], acc[TPT];
#pragma unroll
        for (int u = 0; u < TPT; u++) {
            int64_t a = chunk + u * MV_THREADS + threadIdx.x;
            bool ok = a < nt;
            t[u][0] = ok ? tx0[tb + a] : 0.0;
            t[u][1] = ok && d > 1 ? tx1[tb + a] : 0.0;
            t[u][2] = ok && d > 2 ? tx2[tb + a] : 0.0;
            acc[u] = 0.0;
        }
        for (int64_t e = lptr[i]; e < lptr[i + 1]; e++) {
            int j = lidx[e];
            int64_t sb, ns;
            const double *q0, *q1, *q2, *w;
            if (kind == 0) { sb = sk_off[j]; ns = kk[j]; q0 = s0; q1 = s1; q2 = s2; w = xh; }
            else { sb = begin[j]; ns = end[j] - begin[j]; q0 = x0; q1 = x1; q2 = x2; w = xm; }
            for (int64_t p0 = 0; p0 < ns; p0 += NB_TILE) {
                int cnt = (int)(ns - p0 < NB_TILE ? ns - p0 : NB_TILE);
                __syncthreads();
                for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
                    sx[0][r] = q0[sb + p0 + r];
                    sx[1][r] = d > 1 ? q1[sb + p0 + r] : 0.0;
                    sx[2][r] = d > 2 ? q2[sb + p0 + r] : 0.0;
                    sw[r] = w[sb + p0 + r];
                }
                __syncthreads();
                for (int r = 0; r < cnt; r++) {
                    double a0 = sx[0][r], a1 = sx[1][r], a2 = sx[2][r], ww = sw[r];
#pragma unroll
                    for (int u = 0; u < TPT; u++) {
                        double r2 = h2_dist2(d, t[u][0], t[u][1], t[u][2], a0, a1, a2);
                        acc[u] += h2_kappa(kid, kp0, r2) * ww;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < TPT; u++) {
            int64_t a = chunk + u * MV_THREADS + threadIdx.x;
            if (a < nt) {
                if (kind == 0) zh[tb + a] += acc[u];
                else ym[tb + a] += acc[u];
            }
        }
        __syncthreads();
    }
}

// out[r] = sum_q kappa(x_s, x_q) z_q for s = rows[r]; one CTA per row
__global__ void k_exact_rows(const int64_t *rows, int64_t nrows, const int32_t *iperm, const double *x0,
                             const double *x1, const double *x2, const double *zm, int64_t n, int d, int kid,
                             double kp0, double *out) {
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
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
        double r2 = h2_dist2(d, a0, a1, a2, x0[q], d > 1 ? x1[q] : 0.0, d > 2 ? x2[q] : 0.0);
        s += h2_kappa(kid, kp0, r2) * zm[q];
    }
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

__global__ void k_active_nodes(const int32_t *kk, const int64_t *lptr, int nn, int32_t *list, int32_t *cnt,
                               const int32_t *nchild, int kind) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    bool act = kind == 0 ? (kk[i] > 0 && lptr[i + 1] > lptr[i]) : (nchild[i] == 0 && lptr[i + 1] > lptr[i]);
    if (act) list[atomicAdd(cnt, 1)] = i;
}

}  // namespace

void matvec_impl(h2_matrix_s *A, const double *x, double *y, cudaStream_t s) {
    h2_tree_s *t = A->tree;
    const int nn = t->nnodes, d = t->d;
    const int64_t n = t->n;
    static bool attr = false;
    if (!attr) {
        H2_CUDA(cudaFuncSetAttribute(k_upward, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        H2_CUDA(cudaFuncSetAttribute(k_downward, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    for (int l = 1; l < t->nlevels; l++)
        if ((size_t)A->cmax_level[l] * sizeof(double) > 200 * 1024)
            fail(H2_ERR_UNIMPLEMENTED, "candidate set too large for the single-CTA upward pass");
    DevBuf<double> xm, ym, xh, zh;
    xm.alloc(n, s);
    ym.alloc(n, s);
    int64_t kt = std::max<int64_t>(A->ktotal, 1);
    xh.alloc(kt, s);
    zh.alloc(kt, s);
    H2_CUDA(cudaMemsetAsync(ym.p, 0, n * sizeof(double), s));
    H2_CUDA(cudaMemsetAsync(zh.p, 0, kt * sizeof(double), s));
    k_perm_in<<<blocks_for(n, 256), 256, 0, s>>>(x, t->perm.p, n, xm.p);
    H2_LAUNCH("k_perm_in");
    // upward, deepest level first
    for (int l = t->nlevels - 1; l >= 1; l--) {
        int lb = t->lptr[l], nl = t->lptr[l + 1] - lb;
        if (A->kmax_level[l] == 0) continue;
        size_t sm = (size_t)A->cmax_level[l] * sizeof(double);
        ProfScope ps(KT_UPWARD, s);
        k_upward<<<nl, MV_THREADS, sm, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p, A->c.p, A->uptr.p,
                                            A->sk_off.p, xm.p, xh.p);
        H2_LAUNCH("k_upward");
    }
    // coupling over far pairs
    DevBuf<int32_t> list, cnt;
    list.alloc(std::max(nn, 1), s);
    cnt.alloc(1, s);
    H2_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t), s));
    k_active_nodes<<<blocks_for(nn, 256), 256, 0, s>>>(A->k.p, t->far_ptr.p, nn, list.p, cnt.p, t->nchild.p, 0);
    H2_LAUNCH("k_active_nodes far");
    int nact = read_scalar(cnt.p, s);
    int tpt = 1;
    while (tpt < MAX_TPT && (int64_t)tpt * MV_THREADS < A->kmax) tpt *= 2;
    auto launch_nbody = [&](int kind, int nblocks, int tp, const int64_t *lp, const int32_t *li) {
        if (nblocks <= 0) return;
#define H2_NB(T)                                                                                                   \
    k_nbody<T><<<nblocks, MV_THREADS, 0, s>>>(kind, A->k.p, A->sk_off.p, A->skc[0].p, A->skc[1].p, A->skc[2].p,    \
                                              xh.p, zh.p, t->begin.p, t->end.p, t->xs[0].p, t->xs[1].p,            \
                                              t->xs[2].p, xm.p, ym.p, lp, li, list.p, d, A->kid, A->kp[0])
        ProfScope ps(kind == 0 ? KT_COUPLING : KT_NEAR, s);
        switch (tp) {
        case 1: H2_NB(1); break;
        case 2: H2_NB(2); break;
        case 4: H2_NB(4); break;
        default: H2_NB(8); break;
        }
#undef H2_NB
        H2_LAUNCH("k_nbody");
    };
    launch_nbody(0, nact, tpt, t->far_ptr.p, t->far_idx.p);
    // downward, level 1 first
    for (int l = 1; l < t->nlevels; l++) {
        int lb = t->lptr[l], nl = t->lptr[l + 1] - lb;
        if (A->kmax_level[l] == 0) continue;
        size_t sm = (size_t)A->kmax_level[l] * sizeof(double);
        ProfScope ps(KT_DOWNWARD, s);
        k_downward<<<nl, MV_THREADS, sm, s>>>(lb, t->nchild.p, t->fchild.p, t->begin.p, A->k.p, A->c.p, A->uptr.p,
                                              A->sk_off.p, zh.p, ym.p);
        H2_LAUNCH("k_downward");
    }
    // nearfield over near leaf pairs
    H2_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t), s));
    k_active_nodes<<<blocks_for(nn, 256), 256, 0, s>>>(A->k.p, t->near_ptr.p, nn, list.p, cnt.p, t->nchild.p, 1);
    H2_LAUNCH("k_active_nodes near");
    int nleaf = read_scalar(cnt.p, s);
    int tpn = 1;
    while (tpn < MAX_TPT && (int64_t)tpn * MV_THREADS < t->max_leaf) tpn *= 2;
    launch_nbody(1, nleaf, tpn, t->near_ptr.p, t->near_idx.p);
    k_perm_out<<<blocks_for(n, 256), 256, 0, s>>>(ym.p, t->perm.p, n, y);
    H2_LAUNCH("k_perm_out");
}

void exact_rows_impl(h2_tree_s *t, int kid, const double *kp, const double *z, const int64_t *rows, int64_t nrows,
                     double *out, cudaStream_t s) {
    const int64_t n = t->n;
    DevBuf<double> zm;
    zm.alloc(n, s);
    k_perm_in<<<blocks_for(n, 256), 256, 0, s>>>(z, t->perm.p, n, zm.p);
    H2_LAUNCH("k_perm_in");
    if (nrows > 0) {
        ProfScope ps(KT_EXACT, s);
        k_exact_rows<<<(unsigned)nrows, 512, 0, s>>>(rows, nrows, t->iperm.p, t->xs[0].p, t->xs[1].p, t->xs[2].p,
                                                     zm.p, n, t->d, kid, kp[0], out);
        H2_LAUNCH("k_exact_rows");
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
                                                     zm, n, t->d, kid, kp[0], out);
        H2_LAUNCH("k_exact_rows (noalloc)");
    }
}

}  // namespace h2
