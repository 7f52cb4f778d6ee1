// tree.cu -- adaptive Morton cluster tree and near/far interaction lists
// (section 2.1 and eq. (1) of arXiv 2206.01885; Algorithm 2 step 1).
//
// Bit-exact with a plain IEEE evaluation: quantisation uses explicitly rounded
// float64 operations, everything after it is integer work.
#include "h2_internal.cuh"

namespace h2 {
namespace {

constexpr int BBOX_THREADS = 256;

// per-block min/max of each coordinate and whether any is non-finite;
// pts row-major n x d; part holds 7 values per block
__global__ void k_bbox_partial(const double *pts, int64_t n, int d, double *part) {
    __shared__ double smin[3][BBOX_THREADS], smax[3][BBOX_THREADS];
    double mn[3], mx[3];
    bool bad = false;
    for (int k = 0; k < 3; k++) { mn[k] = INFINITY; mx[k] = -INFINITY; }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < d; k++) {
            double v = pts[i * d + k];
            bad = bad || !isfinite(v);
            mn[k] = fmin(mn[k], v);
            mx[k] = fmax(mx[k], v);
        }
    for (int k = 0; k < 3; k++) { smin[k][threadIdx.x] = mn[k]; smax[k][threadIdx.x] = mx[k]; }
    bad = __syncthreads_or(bad);
    for (int o = BBOX_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; k++) {
                smin[k][threadIdx.x] = fmin(smin[k][threadIdx.x], smin[k][threadIdx.x + o]);
                smax[k][threadIdx.x] = fmax(smax[k][threadIdx.x], smax[k][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; k++) { part[blockIdx.x * 7 + k] = smin[k][0]; part[blockIdx.x * 7 + 3 + k] = smax[k][0]; }
        part[blockIdx.x * 7 + 6] = bad ? 1.0 : 0.0;
    }
}

// root cube: lo = componentwise min, side = max_k (hi_k - lo_k), scale = 2^B / side
__global__ void k_bbox_final(const double *part, int nblk, int d, int B, Geom *g) {
    if (threadIdx.x != 0) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    for (int b = 0; b < nblk; b++) {
        for (int k = 0; k < 3; k++) { lo[k] = fmin(lo[k], part[b * 7 + k]); hi[k] = fmax(hi[k], part[b * 7 + 3 + k]); }
        bad |= part[b * 7 + 6] != 0.0;
    }
    double side = 0.0;
    for (int k = 0; k < 3; k++) {
        g->lo[k] = k < d ? lo[k] : 0.0;
        g->hi[k] = k < d ? hi[k] : 0.0;
        if (k < d) {
            double w = __dsub_rn(hi[k], lo[k]);
            if (w > side) side = w;
        }
    }
    g->side = side;
    g->scale = side > 0.0 ? __ddiv_rn(ldexp(1.0, B), side) : 0.0;
    g->nonfinite = bad;
}

// quantise c = min(floor((x - lo) * scale), 2^B - 1) and interleave the bits,
// coordinate k's bit b at key bit d*b + k
__global__ void k_morton(const double *pts, int64_t n, int d, int B, const Geom *g, uint64_t *key, int32_t *idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double top = ldexp(1.0, B);
    uint64_t c[3] = {0, 0, 0};
    if (g->side > 0.0)
        for (int k = 0; k < d; k++) {
            double t = __dmul_rn(__dsub_rn(pts[i * d + k], g->lo[k]), g->scale);
            c[k] = (t < top) ? (uint64_t)t : ((1ull << B) - 1ull);
        }
    uint64_t kk = 0;
    for (int b = 0; b < B; b++)
        for (int k = 0; k < d; k++) kk |= ((c[k] >> b) & 1ull) << (d * b + k);
    key[i] = kk;
    idx[i] = (int32_t)i;
}

__global__ void k_gather_coords(const double *pts, int64_t n, int d, const int32_t *perm, double *x0, double *x1,
                                double *x2, int32_t *iperm) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t o = perm[p];
    x0[p] = pts[o * d];
    if (d > 1) x1[p] = pts[o * d + 1];
    if (d > 2) x2[p] = pts[o * d + 2];
    iperm[o] = (int32_t)p;
}

__global__ void k_root(int32_t *level, int32_t *parent, int32_t *fchild, int32_t *nchild, int32_t *begin,
                       int32_t *end, uint64_t *prefix, int32_t n) {
    level[0] = 0; parent[0] = -1; fchild[0] = -1; nchild[0] = 0; begin[0] = 0; end[0] = n; prefix[0] = 0;
}

// first position p in [lo, hi) whose orthant digit >= o (digits ascend in the range)
__device__ __forceinline__ int32_t orthant_start(const uint64_t *key, int32_t lo, int32_t hi, int shift, uint64_t mask,
                                                 uint64_t o) {
    while (lo < hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (((key[mid] >> shift) & mask) < o) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// number of non-empty children of each node of level l (0 if it is a leaf)
__global__ void k_split_count(const int32_t *begin, const int32_t *end, int lb, int nl, const uint64_t *key, int q,
                              int l, int B, int d, int can_split, int32_t *cnt) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nl) return;
    int i = lb + a;
    int32_t b0 = begin[i], e0 = end[i];
    int c = 0;
    if (can_split && (e0 - b0) > q && l < B) {
        int shift = d * (B - l - 1);
        uint64_t mask = (1ull << d) - 1ull;
        int32_t s = b0;
        for (uint64_t o = 0; o <= mask; o++) {
            int32_t e = orthant_start(key, s, e0, shift, mask, o + 1);
            if (e > s) c++;
            s = e;
        }
    }
    cnt[a] = c;
}

__global__ void k_split_write(int32_t *level, int32_t *parent, int32_t *fchild, int32_t *nchild, int32_t *begin,
                              int32_t *end, uint64_t *prefix, int lb, int nl, const int64_t *off, const uint64_t *key,
                              int l, int B, int d) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nl) return;
    int i = lb + a;
    int64_t c0 = off[a], c1 = off[a + 1];
    int first = lb + nl + (int)c0;
    nchild[i] = (int)(c1 - c0);
    fchild[i] = c1 > c0 ? first : -1;
    if (c1 == c0) return;
    int shift = d * (B - l - 1);
    uint64_t mask = (1ull << d) - 1ull;
    int32_t s = begin[i], e0 = end[i];
    int w = first;
    for (uint64_t o = 0; o <= mask; o++) {
        int32_t e = orthant_start(key, s, e0, shift, mask, o + 1);
        if (e > s) {
            level[w] = l + 1; parent[w] = i; fchild[w] = -1; nchild[w] = 0;
            begin[w] = s; end[w] = e; prefix[w] = key[s] >> shift;
            w++;
        }
        s = e;
    }
}

// centre of each node's cell in real coordinates: lo + (c + 1/2) side / 2^level
__global__ void k_node_centres(const int32_t *level, const uint64_t *prefix, int nn, int d, const Geom *g, double *c0,
                               double *c1, double *c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int l = level[i];
    uint64_t c[3] = {0, 0, 0};
    for (int b = 0; b < l; b++)
        for (int k = 0; k < d; k++) c[k] |= ((prefix[i] >> (d * b + k)) & 1ull) << b;
    double w = ldexp(g->side, -l);
    double *out[3] = {c0, c1, c2};
    for (int k = 0; k < d; k++) out[k][i] = g->lo[k] + ((double)c[k] + 0.5) * w;
}

// float32 coordinates of each point relative to the centre of its leaf (one CTA per node, leaves only)
__global__ void k_rel_coords(const int32_t *nchild, const int32_t *begin, const int32_t *end, const double *c0,
                             const double *c1, const double *c2, const double *x0, const double *x1,
                             const double *x2, int d, float *r0, float *r1, float *r2) {
    int i = blockIdx.x;
    if (nchild[i] != 0) return;
    for (int p = begin[i] + threadIdx.x; p < end[i]; p += blockDim.x) {
        r0[p] = (float)(x0[p] - c0[i]);
        if (d > 1) r1[p] = (float)(x1[p] - c1[i]);
        if (d > 2) r2[p] = (float)(x2[p] - c2[i]);
    }
}

// coordinates relative to the root box corner as float32 {hi, lo} pairs:
// hi = fl32(x - lo), lo = fl32((x - lo) - hi) (DataReduct's float32 search)
__device__ __forceinline__ float2 h2_split(double v) {
    float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

__global__ void k_root_coords(const double *x0, const double *x1, const double *x2, int64_t n, int d, const Geom *g,
                              float4 *xq) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float2 a = h2_split(x0[p] - g->lo[0]);
    const float2 b = d > 1 ? h2_split(x1[p] - g->lo[1]) : make_float2(0.f, 0.f);
    const float2 c = d > 2 ? h2_split(x2[p] - g->lo[2]) : make_float2(0.f, 0.f);
    xq[2 * p] = make_float4(a.x, b.x, c.x, a.y);
    xq[2 * p + 1] = make_float4(b.y, c.y, 0.f, 0.f);
}

__global__ void k_centre_split(const double *c0, const double *c1, const double *c2, int nn, int d, const Geom *g,
                               float2 *f0, float2 *f1, float2 *f2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    f0[i] = h2_split(c0[i] - g->lo[0]);
    if (d > 1) f1[i] = h2_split(c1[i] - g->lo[1]);
    if (d > 2) f2[i] = h2_split(c2[i] - g->lo[2]);
}

__global__ void k_max_leaf(const int32_t *nchild, const int32_t *begin, const int32_t *end, int nn, int32_t *mx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nn && nchild[i] == 0) atomicMax(mx, end[i] - begin[i]);
}

// ------------------------------------------------------------------ lists
// eq. (1) with the cells' diameters sqrt(d) e and centres; A = 2 * centre =
// e (2c + 1) in quantised units:
//   den^2 d (e_i + e_j)^2 <= num^2 |A_i - A_j|^2
__device__ __forceinline__ void cell_of(uint64_t prefix, int l, int d, uint64_t *c) {
    c[0] = c[1] = c[2] = 0;
    for (int b = 0; b < l; b++)
        for (int k = 0; k < d; k++) c[k] |= ((prefix >> (d * b + k)) & 1ull) << b;
}

__device__ bool admissible(int i, int j, const int32_t *level, const uint64_t *prefix, int d, int B, int tnum,
                           int tden) {
    uint64_t ci[3], cj[3];
    int li = level[i], lj = level[j];
    cell_of(prefix[i], li, d, ci);
    cell_of(prefix[j], lj, d, cj);
    uint64_t ei = 1ull << (B - li), ej = 1ull << (B - lj);
    unsigned __int128 dist = 0;
    for (int k = 0; k < d; k++) {
        uint64_t ai = ei * (2 * ci[k] + 1), aj = ej * (2 * cj[k] + 1);
        uint64_t df = ai > aj ? ai - aj : aj - ai;
        dist += (unsigned __int128)df * df;
    }
    unsigned __int128 es = (unsigned __int128)(ei + ej) * (ei + ej);
    unsigned __int128 lhs = (unsigned __int128)((uint64_t)tden * (uint64_t)tden) * (unsigned __int128)d * es;
    unsigned __int128 rhs = (unsigned __int128)((uint64_t)tnum * (uint64_t)tnum) * dist;
    return lhs <= rhs;
}

// classify each frontier pair: 0 far, 1 near, 2 expand into children pairs
__global__ void k_pairs_classify(const int2 *F, int64_t nf, const int32_t *level, const uint64_t *prefix,
                                 const int32_t *nchild, int d, int B, int tnum, int tden, int8_t *cls,
                                 int64_t *nexp, unsigned long long *rc) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nf) return;
    int i = F[a].x, j = F[a].y;
    int8_t c;
    int64_t ne = 0;
    if (admissible(i, j, level, prefix, d, B, tnum, tden)) {
        c = 0;
        atomicAdd(&rc[0], 1ull);
    } else if (nchild[i] == 0 && nchild[j] == 0) {
        c = 1;
        atomicAdd(&rc[1], 1ull);
    } else {
        c = 2;
        int ni = nchild[i] ? nchild[i] : 1, nj = nchild[j] ? nchild[j] : 1;
        ne = (int64_t)ni * nj;
    }
    cls[a] = c;
    nexp[a] = ne;
}

__global__ void k_pairs_emit(const int2 *F, int64_t nf, const int8_t *cls, const int64_t *off, const int32_t *fchild,
                             const int32_t *nchild, int nn, uint64_t *farbuf, uint64_t *nearbuf,
                             unsigned long long *cursor, int2 *Fn) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nf) return;
    int i = F[a].x, j = F[a].y;
    int8_t c = cls[a];
    if (c == 0) {
        unsigned long long p = atomicAdd(&cursor[0], 1ull);
        farbuf[p] = (uint64_t)i * (uint64_t)nn + (uint64_t)j;
    } else if (c == 1) {
        unsigned long long p = atomicAdd(&cursor[1], 1ull);
        nearbuf[p] = (uint64_t)i * (uint64_t)nn + (uint64_t)j;
    } else {
        int a0 = nchild[i] ? fchild[i] : i, a1 = nchild[i] ? fchild[i] + nchild[i] : i + 1;
        int b0 = nchild[j] ? fchild[j] : j, b1 = nchild[j] ? fchild[j] + nchild[j] : j + 1;
        int64_t w = off[a];
        for (int x = a0; x < a1; x++)
            for (int y = b0; y < b1; y++) Fn[w++] = make_int2(x, y);
    }
}

// CSR from pair keys sorted by (i, j): ptr[i] = first key >= i * nn
__global__ void k_csr(const uint64_t *keys, int64_t m, int nn, int64_t *ptr, int32_t *idx) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= nn) {
        uint64_t target = (uint64_t)t * (uint64_t)nn;
        int64_t lo = 0, hi = m;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        ptr[t] = lo;
    }
    if (t < m) idx[t] = (int32_t)(keys[t] % (uint64_t)nn);
}

template <class T>
void grow(DevBuf<T> &b, size_t need, size_t keep, cudaStream_t s) {
    if (b.n >= need) return;
    size_t cap = b.n ? b.n : 1024;
    while (cap < need) cap *= 2;
    DevBuf<T> nb;
    nb.alloc(cap, s);
    if (keep) H2_CUDA(cudaMemcpyAsync(nb.p, b.p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s));
    b = std::move(nb);
}

int bits_needed(uint64_t v) {
    int b = 0;
    while (b < 64 && (v >> b) != 0) b++;
    return b;
}

}  // namespace

void tree_build_impl(h2_tree_s *t, const double *pts) {
    cudaStream_t s = t->stream;
    const int64_t n = t->n;
    const int d = t->d, B = t->B;
    // root box
    int nblk = (int)std::min<int64_t>(1024, (n + BBOX_THREADS - 1) / BBOX_THREADS);
    DevBuf<double> part;
    part.alloc((size_t)nblk * 7, s);
    DevBuf<Geom> g;
    g.alloc(1, s);
    k_bbox_partial<<<nblk, BBOX_THREADS, 0, s>>>(pts, n, d, part.p);
    H2_LAUNCH("k_bbox_partial");
    k_bbox_final<<<1, 32, 0, s>>>(part.p, nblk, d, B, g.p);
    H2_LAUNCH("k_bbox_final");
    // keys, stable sort by (key, index)
    t->key.alloc(n, s);
    t->perm.alloc(n, s);
    k_morton<<<blocks_for(n, 256), 256, 0, s>>>(pts, n, d, B, g.p, t->key.p, t->perm.p);
    H2_LAUNCH("k_morton");
    {
        ProfScope ps(KT_SORT, s);
        radix_sort(t->key.p, t->perm.p, n, d * B, s);
    }
    for (int k = 0; k < 3; k++) t->xs[k].alloc(k < d ? n : 1, s);
    t->iperm.alloc(n, s);
    k_gather_coords<<<blocks_for(n, 256), 256, 0, s>>>(pts, n, d, t->perm.p, t->xs[0].p, t->xs[1].p, t->xs[2].p,
                                                        t->iperm.p);
    H2_LAUNCH("k_gather_coords");
    t->geom = read_scalar(g.p, s);
    if (t->geom.nonfinite) fail(H2_ERR_NUMERIC, "point coordinates must be finite");
    // levels: split every node holding more than q points into its non-empty orthants
    size_t cap = 1024;
    t->level.alloc(cap, s); t->parent.alloc(cap, s); t->fchild.alloc(cap, s); t->nchild.alloc(cap, s);
    t->begin.alloc(cap, s); t->end.alloc(cap, s); t->prefix.alloc(cap, s);
    k_root<<<1, 1, 0, s>>>(t->level.p, t->parent.p, t->fchild.p, t->nchild.p, t->begin.p, t->end.p, t->prefix.p,
                          (int32_t)n);
    H2_LAUNCH("k_root");
    t->lptr = {0, 1};
    const int can_split = t->geom.side > 0.0 ? 1 : 0;
    DevBuf<int32_t> cnt;
    DevBuf<int64_t> off;
    for (int l = 0;; l++) {
        int lb = t->lptr[l], le = t->lptr[l + 1], nl = le - lb;
        cnt.alloc(nl, s);
        off.alloc(nl + 1, s);
        k_split_count<<<blocks_for(nl, 128), 128, 0, s>>>(t->begin.p, t->end.p, lb, nl, t->key.p, t->q, l, B, d,
                                                           can_split, cnt.p);
        H2_LAUNCH("k_split_count");
        scan_exclusive_i32(cnt.p, off.p, nl, s);
        int64_t total = read_scalar(off.p + nl, s);
        if (total == 0) break;
        size_t need = (size_t)le + (size_t)total;
        grow(t->level, need, le, s); grow(t->parent, need, le, s); grow(t->fchild, need, le, s);
        grow(t->nchild, need, le, s); grow(t->begin, need, le, s); grow(t->end, need, le, s);
        grow(t->prefix, need, le, s);
        k_split_write<<<blocks_for(nl, 128), 128, 0, s>>>(t->level.p, t->parent.p, t->fchild.p, t->nchild.p,
                                                           t->begin.p, t->end.p, t->prefix.p, lb, nl, off.p,
                                                           t->key.p, l, B, d);
        H2_LAUNCH("k_split_write");
        t->lptr.push_back((int)need);
    }
    t->nnodes = t->lptr.back();
    t->nlevels = (int)t->lptr.size() - 1;
    // cell centres and leaf-relative float32 coordinates (float32 kernels)
    for (int k = 0; k < 3; k++) {
        t->cen[k].alloc(k < d ? t->nnodes : 1, s);
        t->xr[k].alloc(k < d ? n : 1, s);
    }
    k_node_centres<<<blocks_for(t->nnodes, 256), 256, 0, s>>>(t->level.p, t->prefix.p, t->nnodes, d, g.p,
                                                              t->cen[0].p, t->cen[1].p, t->cen[2].p);
    H2_LAUNCH("k_node_centres");
    k_rel_coords<<<t->nnodes, 128, 0, s>>>(t->nchild.p, t->begin.p, t->end.p, t->cen[0].p, t->cen[1].p, t->cen[2].p,
                                          t->xs[0].p, t->xs[1].p, t->xs[2].p, d, t->xr[0].p, t->xr[1].p, t->xr[2].p);
    H2_LAUNCH("k_rel_coords");
    t->xq.alloc(2 * n, s);
    k_root_coords<<<blocks_for(n, 256), 256, 0, s>>>(t->xs[0].p, t->xs[1].p, t->xs[2].p, n, d, g.p, t->xq.p);
    H2_LAUNCH("k_root_coords");
    for (int k = 0; k < 3; k++) t->cenf[k].alloc(k < d ? t->nnodes : 1, s);
    k_centre_split<<<blocks_for(t->nnodes, 256), 256, 0, s>>>(t->cen[0].p, t->cen[1].p, t->cen[2].p, t->nnodes, d,
                                                              g.p, t->cenf[0].p, t->cenf[1].p, t->cenf[2].p);
    H2_LAUNCH("k_centre_split");
    DevBuf<int32_t> mx;
    mx.alloc(1, s);
    H2_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(int32_t), s));
    k_max_leaf<<<blocks_for(t->nnodes, 256), 256, 0, s>>>(t->nchild.p, t->begin.p, t->end.p, t->nnodes, mx.p);
    H2_LAUNCH("k_max_leaf");
    t->max_leaf = read_scalar(mx.p, s);
}

void lists_build_impl(h2_tree_s *t) {
    cudaStream_t s = t->stream;
    ProfScope ps(KT_LISTS, s);
    const int nn = t->nnodes;
    DevBuf<int2> F, Fn;
    DevBuf<int8_t> cls;
    DevBuf<int64_t> nexp, off;
    DevBuf<uint64_t> farbuf, nearbuf;
    DevBuf<unsigned long long> ctr;  // [0..1] this traversal step's far/near counts, [2..3] cursors
    ctr.alloc(4, s);
    H2_CUDA(cudaMemsetAsync(ctr.p, 0, 4 * sizeof(unsigned long long), s));
    F.alloc(1024, s);
    int2 root = make_int2(0, 0);
    H2_CUDA(cudaMemcpyAsync(F.p, &root, sizeof(int2), cudaMemcpyHostToDevice, s));
    int64_t nf = 1, nfar = 0, nnear = 0;
    while (nf > 0) {
        cls.alloc(nf, s);
        nexp.alloc(nf, s);
        off.alloc(nf + 1, s);
        H2_CUDA(cudaMemsetAsync(ctr.p, 0, 2 * sizeof(unsigned long long), s));
        k_pairs_classify<<<blocks_for(nf, 256), 256, 0, s>>>(F.p, nf, t->level.p, t->prefix.p, t->nchild.p, t->d,
                                                             t->B, t->tau_num, t->tau_den, cls.p, nexp.p, ctr.p);
        H2_LAUNCH("k_pairs_classify");
        scan_exclusive(nexp.p, off.p, nf, s);
        int64_t next = read_scalar(off.p + nf, s);
        unsigned long long rc[2];
        H2_CUDA(cudaMemcpyAsync(rc, ctr.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        H2_CUDA(cudaStreamSynchronize(s));
        grow(farbuf, (size_t)(nfar + rc[0]), (size_t)nfar, s);
        grow(nearbuf, (size_t)(nnear + rc[1]), (size_t)nnear, s);
        Fn.alloc(next > 0 ? next : 1, s);
        k_pairs_emit<<<blocks_for(nf, 256), 256, 0, s>>>(F.p, nf, cls.p, off.p, t->fchild.p, t->nchild.p, nn,
                                                         farbuf.p, nearbuf.p, ctr.p + 2, Fn.p);
        H2_LAUNCH("k_pairs_emit");
        nfar += (int64_t)rc[0];
        nnear += (int64_t)rc[1];
        std::swap(F, Fn);
        nf = next;
    }
    int nbits = bits_needed((uint64_t)nn * (uint64_t)nn);
    t->nfar = nfar;
    t->nnear = nnear;
    t->far_ptr.alloc(nn + 1, s);
    t->near_ptr.alloc(nn + 1, s);
    t->far_idx.alloc(nfar > 0 ? nfar : 1, s);
    t->near_idx.alloc(nnear > 0 ? nnear : 1, s);
    if (nfar > 0) radix_sort(farbuf.p, nullptr, nfar, nbits, s);
    if (nnear > 0) radix_sort(nearbuf.p, nullptr, nnear, nbits, s);
    k_csr<<<blocks_for(std::max<int64_t>(nfar, nn + 1), 256), 256, 0, s>>>(farbuf.p, nfar, nn, t->far_ptr.p,
                                                                            t->far_idx.p);
    H2_LAUNCH("k_csr far");
    k_csr<<<blocks_for(std::max<int64_t>(nnear, nn + 1), 256), 256, 0, s>>>(nearbuf.p, nnear, nn, t->near_ptr.p,
                                                                             t->near_idx.p);
    H2_LAUNCH("k_csr near");
    H2_CUDA(cudaStreamSynchronize(s));
}

}  // namespace h2
