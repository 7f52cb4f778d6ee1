// blocks.cu -- stored coupling and nearfield blocks (Algorithm 2 of arXiv
// 2206.01885 forms B_ij = K(Xhat_i, Xhat_j) for every far pair and
// K(X_i, X_j) for every near leaf pair).  By default the matvec evaluates
// these kernel submatrices on the fly; with the STORE memory mode the
// construction evaluates each block once and keeps it, and every later
// single-vector product reads it instead.
//
// Layout: kappa is symmetric, so only the entries e of node i's list with
// j = idx[e] >= i are stored, as the row-major block K(targets of i, sources
// of j) (rows = skeleton or points of i, columns = those of j) at element
// offset boff[e] of one buffer per list; boff[e] = -1 for j < i.  The product
// reads each block once and uses it both ways: y_i += B x_j and, for j != i,
// y_j += B^T x_i.
#include <cfloat>

#include "h2_internal.cuh"
#include "kappa_fast.cuh"

namespace h2 {
namespace {

constexpr int BF_THREADS = 256;  // block fill: 8 warps, a warp per row, lanes over columns
constexpr int SB_WARPS = 8;      // stored-block product: warps of a CTA

// The stored entries of one list: entry e (a CSR position), its node pair
// and the block's element offset.
struct StoredList {
    const int32_t *row;   // node i of each stored entry
    const int32_t *col;   // node j
    const int64_t *off;   // element offset of the block
};

// Fill the stored blocks of one list: CTA b takes stored entry b.  Target
// and source coordinates are those the on-the-fly N-body uses (absolute
// float64 in the float64 form; node-relative float32 plus the pair's centre
// offset from float32 {hi, lo} splits in the float32 form), evaluated with
// the same kappa, so a stored entry equals the on-the-fly value bit for bit.
template <class Real, int KID>
__global__ void __launch_bounds__(BF_THREADS)
    k_fill_blocks(StoredList L, const int64_t *start, const int32_t *count, const Real *X0, const Real *X1,
                  const Real *X2, const float2 *F0, const float2 *F1, const float2 *F2, int d, double kpar,
                  Real *blk) {
    const int b = blockIdx.x;
    const int i = L.row[b], j = L.col[b];
    const int64_t ts = start[i], ss = start[j];
    const int tn = count[i], sn = count[j];
    Real *B = blk + L.off[b];
    const Real p = (Real)kpar;
    Real o0 = 0, o1 = 0, o2 = 0;
    if constexpr (sizeof(Real) == 4) {
        if (F0) {
            const float2 a0 = F0[i], b0 = F0[j];
            o0 = (a0.x - b0.x) + (a0.y - b0.y);
            if (d > 1) {
                const float2 a1 = F1[i], b1 = F1[j];
                o1 = (a1.x - b1.x) + (a1.y - b1.y);
            }
            if (d > 2) {
                const float2 a2 = F2[i], b2 = F2[j];
                o2 = (a2.x - b2.x) + (a2.y - b2.y);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < tn; r += BF_THREADS / 32) {
        const Real t0 = X0[ts + r] + o0, t1 = (d > 1 ? X1[ts + r] : (Real)0) + o1,
                   t2 = (d > 2 ? X2[ts + r] : (Real)0) + o2;
        Real *row = B + (int64_t)r * sn;
        for (int c = lane; c < sn; c += 32)
            row[c] = kap_pt<KID, false>(t0, t1, t2, X0[ss + c], d > 1 ? X1[ss + c] : (Real)0,
                                        d > 2 ? X2[ss + c] : (Real)0, p);
    }
}

// v[u] (u < 32) in every lane -> lane l returns the sum over the warp's lanes
// of v[l] (recursive halving: 31 shuffles instead of 32 full warp sums)
template <class Real>
__device__ __forceinline__ Real reduce_scatter32(Real (&v)[32], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int u = 0; u < o; u++) {
            const Real send = up ? v[u] : v[u + o];
            const Real keep = up ? v[u + o] : v[u];
            v[u] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

__device__ __forceinline__ void two_sum_add(float &a, float &e, float b) {
    const float s = a + b, bp = s - a;
    e += (a - (s - bp)) + (b - bp);
    a = s;
}

// Product with the stored blocks of one list, one right-hand side:
//   out_i += B_e w_j, and out_j += B_e^T w_i for j != i,
// over the stored entries e of node i's list.  A CTA takes a tile of 32
// targets of i (rows a0 .. a0 + 31 of every block of i); its warps split the
// entries.  Per 32-column chunk of a block each lane loads its column of the
// tile's 32 rows (32 coalesced row segments in flight), adds B[u, c] w_j[c]
// to its partial of row u and B[u, c] w_i[u] to its column sum, which goes to
// out_j with one float64 atomic.  The row partials are summed across lanes
// by a reduce-scatter (lane l gets row l): once per CTA in float64, once per
// block in float32 (then folded into a compensated float32 accumulator, as
// the on-the-fly kernels do).  Row sums meet other CTAs' in float64 atomics.
template <class Real>
__global__ void __launch_bounds__(SB_WARPS * 32)
    k_stored_sym(const int2 *tiles, const int64_t *start, const int32_t *count, const Real *blk,
                 const int64_t *boff, const Real *w, double *out, const int64_t *lptr, const int64_t *lfirst,
                 const int32_t *lidx) {
    __shared__ Real wt[32];
    __shared__ double part[SB_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 tl = tiles[blockIdx.x];
    const int i = tl.x, a0 = tl.y;
    const int64_t ts = start[i];
    const int tn = count[i];
    const int tcount = min(32, tn - a0);
    if (threadIdx.x < 32) wt[threadIdx.x] = threadIdx.x < tcount ? w[ts + a0 + threadIdx.x] : (Real)0;
    __syncthreads();
    Real v[32];
#pragma unroll
    for (int u = 0; u < 32; u++) v[u] = (Real)0;
    float acc = 0.f, cmp = 0.f;  // float32 form: this lane's row, compensated
    for (int64_t e = lfirst[i] + warp; e < lptr[i + 1]; e += SB_WARPS) {
        const int j = lidx[e];
        const int64_t bo = boff[e];
        if (bo < 0) continue;  // an empty block (a node without skeleton)
        const bool sym = j != i;
        const int64_t ss = start[j];
        const int sn = count[j];
        const Real *B = blk + bo + (int64_t)a0 * sn;
        for (int c0 = 0; c0 < sn; c0 += 32) {
            const int c = c0 + lane;
            const bool okc = c < sn;
            const Real ws = okc ? w[ss + c] : (Real)0;
            Real col = (Real)0;
#pragma unroll
            for (int u = 0; u < 32; u++) {
                const Real bv = okc && u < tcount ? B[(int64_t)u * sn + c] : (Real)0;
                v[u] += bv * ws;
                col += bv * wt[u];
            }
            if (sym && okc) atomicAdd(out + ss + c, (double)col);
        }
        if constexpr (sizeof(Real) == 4) {
            two_sum_add(acc, cmp, reduce_scatter32(v, lane));
#pragma unroll
            for (int u = 0; u < 32; u++) v[u] = 0.f;
        }
    }
    double mine;
    if constexpr (sizeof(Real) == 8) mine = reduce_scatter32(v, lane);
    else mine = (double)acc + (double)cmp;
    part[warp][lane] = mine;
    __syncthreads();
    if (threadIdx.x < tcount) {
        double sum = 0.0;
        for (int wv = 0; wv < SB_WARPS; wv++) sum += part[wv][threadIdx.x];
        atomicAdd(out + ts + a0 + threadIdx.x, sum);
    }
}

template <class Real>
void fill_list(int kid, const StoredList &L, int64_t nstored, const int64_t *start, const int32_t *count,
               const Real *X0, const Real *X1, const Real *X2, const float2 *F0, const float2 *F1, const float2 *F2,
               int d, double kp0, Real *blk, cudaStream_t s) {
    if (nstored == 0) return;
    const double p = kap_param(kid, kp0);
#define H2_FILL(K)                                                                                              \
    k_fill_blocks<Real, K><<<(unsigned)nstored, BF_THREADS, 0, s>>>(L, start, count, X0, X1, X2, F0, F1, F2, d, \
                                                                     p, blk)
    switch (kid) {
    case H2_K_COULOMB: H2_FILL(H2_K_COULOMB); break;
    case H2_K_GAUSSIAN: H2_FILL(H2_K_GAUSSIAN); break;
    case H2_K_EXPONENTIAL: H2_FILL(H2_K_EXPONENTIAL); break;
    case H2_K_BUMP: H2_FILL(H2_K_BUMP); break;
    case H2_K_POWER: H2_FILL(H2_K_POWER); break;
    case H2_K_COSDOT: H2_FILL(H2_K_COSDOT); break;
    default: H2_FILL(H2_K_MULTIQUADRIC);
    }
#undef H2_FILL
    H2_LAUNCH("k_fill_blocks");
}

__global__ void k_to_float_abs(const double *a, int64_t n, float *b) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) b[p] = (float)a[p];
}

// Host plan of one list: offsets of the stored entries (j >= i) and their
// node pairs, for blocks of rows[i] x rows[j] elements.
struct ListPlan {
    std::vector<int64_t> boff;           // per CSR entry, -1 where not stored
    std::vector<int32_t> row, col;       // per stored entry
    std::vector<int64_t> off;            // per stored entry
    int64_t elems = 0;
};

ListPlan plan_list(const std::vector<int64_t> &ptr, const std::vector<int32_t> &idx,
                   const std::vector<int32_t> &rows) {
    ListPlan P;
    const int nn = (int)rows.size();
    P.boff.assign(idx.size(), -1);
    for (int i = 0; i < nn; i++)
        for (int64_t e = ptr[i]; e < ptr[i + 1]; e++) {
            const int j = idx[e];
            if (j < i || rows[i] == 0 || rows[j] == 0) continue;
            P.boff[e] = P.elems;
            P.row.push_back(i);
            P.col.push_back(j);
            P.off.push_back(P.elems);
            P.elems += (int64_t)rows[i] * rows[j];
        }
    return P;
}

}  // namespace

void store_blocks_impl(h2_matrix_s *A, int mode, double fraction) {
    h2_tree_s *t = A->tree;
    cudaStream_t s = A->stream;
    const int nn = t->nnodes, d = t->d;
    const bool f64 = A->prec == H2_PREC_FP64;
    const size_t esz = f64 ? sizeof(double) : sizeof(float);
    std::vector<int32_t> kh = read_vec(A->k.p, nn, s);
    std::vector<int32_t> b = read_vec(t->begin.p, nn, s), e = read_vec(t->end.p, nn, s),
                         nc = read_vec(t->nchild.p, nn, s);
    std::vector<int32_t> pts(nn);
    for (int i = 0; i < nn; i++) pts[i] = nc[i] == 0 ? e[i] - b[i] : 0;
    ListPlan far = plan_list(read_vec(t->far_ptr.p, nn + 1, s), read_vec(t->far_idx.p, t->nfar, s), kh);
    ListPlan near = plan_list(read_vec(t->near_ptr.p, nn + 1, s), read_vec(t->near_idx.p, t->nnear, s), pts);
    const double bytes = (double)(far.elems + near.elems) * (double)esz;
    // free device memory: what the device reports plus what the stream-ordered
    // pool holds without using (the library keeps freed memory in the pool)
    size_t fr = 0, tot = 0;
    H2_CUDA(cudaMemGetInfo(&fr, &tot));
    {
        int dev = 0;
        cudaMemPool_t pool;
        uint64_t reserved = 0, used = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            fr += (size_t)(reserved - used);
        cudaGetLastError();
    }
    const double budget = fraction * (double)fr;
    A->stored_bytes_plan = (int64_t)bytes;
    if (bytes > budget) {
        if (mode == H2_MEM_STORE) {
            char buf[200];
            snprintf(buf, sizeof buf,
                     "stored blocks need %.3g bytes, above mem_fraction %.3g of the %.3g bytes free", bytes, fraction,
                     (double)fr);
            fail(H2_ERR_OOM, buf);
        }
        return;  // AUTO: on the fly
    }
    cudaEvent_t e0, e1;
    H2_CUDA(cudaEventCreate(&e0));
    H2_CUDA(cudaEventCreate(&e1));
    H2_CUDA(cudaEventRecord(e0, s));
    DevBuf<unsigned char> fblk, nblk;
    DevBuf<int64_t> fboff, nboff;
    fblk.alloc(std::max<int64_t>(far.elems, 1) * esz, s);
    nblk.alloc(std::max<int64_t>(near.elems, 1) * esz, s);
    fboff.alloc(std::max<size_t>(far.boff.size(), 1), s);
    nboff.alloc(std::max<size_t>(near.boff.size(), 1), s);
    if (!far.boff.empty())
        H2_CUDA(cudaMemcpyAsync(fboff.p, far.boff.data(), far.boff.size() * 8, cudaMemcpyHostToDevice, s));
    if (!near.boff.empty())
        H2_CUDA(cudaMemcpyAsync(nboff.p, near.boff.data(), near.boff.size() * 8, cudaMemcpyHostToDevice, s));
    // per stored entry: i, j, offset
    auto upload = [&](const ListPlan &P, DevBuf<int32_t> &r, DevBuf<int32_t> &c, DevBuf<int64_t> &o) {
        const size_t ns = std::max<size_t>(P.row.size(), 1);
        r.alloc(ns, s);
        c.alloc(ns, s);
        o.alloc(ns, s);
        if (P.row.empty()) return;
        H2_CUDA(cudaMemcpyAsync(r.p, P.row.data(), P.row.size() * 4, cudaMemcpyHostToDevice, s));
        H2_CUDA(cudaMemcpyAsync(c.p, P.col.data(), P.col.size() * 4, cudaMemcpyHostToDevice, s));
        H2_CUDA(cudaMemcpyAsync(o.p, P.off.data(), P.off.size() * 8, cudaMemcpyHostToDevice, s));
    };
    DevBuf<int32_t> fr_, fc_, nr_, nc_;
    DevBuf<int64_t> fo_, no_;
    upload(far, fr_, fc_, fo_);
    upload(near, nr_, nc_, no_);
    // point sets of the leaves (int64 starts, counts) as the N-body uses them
    DevBuf<int64_t> lstart;
    DevBuf<int32_t> lcount;
    {
        std::vector<int64_t> st(b.begin(), b.end());
        std::vector<int32_t> ct(nn);
        for (int i = 0; i < nn; i++) ct[i] = e[i] - b[i];
        lstart.alloc(nn, s);
        lcount.alloc(nn, s);
        H2_CUDA(cudaMemcpyAsync(lstart.p, st.data(), nn * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        H2_CUDA(cudaMemcpyAsync(lcount.p, ct.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    {
        ProfScope ps(KT_FILL, s);
        const StoredList FL{fr_.p, fc_.p, fo_.p}, NL{nr_.p, nc_.p, no_.p};
        if (f64) {
            fill_list<double>(A->kid, FL, (int64_t)far.row.size(), A->sk_off.p, A->k.p, A->skc[0].p, A->skc[1].p,
                              A->skc[2].p, nullptr, nullptr, nullptr, d, A->kp[0],
                              reinterpret_cast<double *>(fblk.p), s);
            fill_list<double>(A->kid, NL, (int64_t)near.row.size(), lstart.p, lcount.p, t->xs[0].p, t->xs[1].p,
                              t->xs[2].p, nullptr, nullptr, nullptr, d, A->kp[0],
                              reinterpret_cast<double *>(nblk.p), s);
        } else {
            // float32 coordinates as the on-the-fly kernels take them: node-relative
            // with centre splits, or absolute with zero offsets for cos(x . y)
            const bool cosd = A->kid == H2_K_COSDOT;
            const float2 *CF[3] = {cosd ? nullptr : t->cenf[0].p, t->cenf[1].p, t->cenf[2].p};
            DevBuf<float> xabs[3];
            const float *PX[3] = {t->xr[0].p, t->xr[1].p, t->xr[2].p};
            if (cosd) {
                for (int k = 0; k < d; k++) {
                    xabs[k].alloc(t->n, s);
                    k_to_float_abs<<<blocks_for(t->n, 256), 256, 0, s>>>(t->xs[k].p, t->n, xabs[k].p);
                    H2_LAUNCH("k_to_float_abs");
                    PX[k] = xabs[k].p;
                }
            }
            fill_list<float>(A->kid, FL, (int64_t)far.row.size(), A->sk_off.p, A->k.p, A->skr[0].p, A->skr[1].p,
                             A->skr[2].p, CF[0], CF[1], CF[2], d, A->kp[0], reinterpret_cast<float *>(fblk.p), s);
            fill_list<float>(A->kid, NL, (int64_t)near.row.size(), lstart.p, lcount.p, PX[0], PX[1], PX[2], CF[0],
                             CF[1], CF[2], d, A->kp[0], reinterpret_cast<float *>(nblk.p), s);
        }
    }
    H2_CUDA(cudaEventRecord(e1, s));
    H2_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    A->far_blk = std::move(fblk);
    A->near_blk = std::move(nblk);
    A->far_boff = std::move(fboff);
    A->near_boff = std::move(nboff);
    A->stored = true;
    A->stored_far_bytes = far.elems * (int64_t)esz;
    A->stored_near_bytes = near.elems * (int64_t)esz;
    A->ms_blocks = ms;
}

// coupling or nearfield with the stored blocks, one right-hand side (w in
// the block's type, out float64)
template <class Real>
void stored_product(const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count, const void *blk,
                    const int64_t *boff, const Real *w, double *out, const int64_t *lptr, const int64_t *lfirst,
                    const int32_t *lidx, cudaStream_t s) {
    if (tiles.n == 0) return;
    k_stored_sym<Real><<<(unsigned)tiles.n, SB_WARPS * 32, 0, s>>>(tiles.p, start, count,
                                                                   static_cast<const Real *>(blk), boff, w, out,
                                                                   lptr, lfirst, lidx);
    H2_LAUNCH("k_stored_sym");
}
template void stored_product<double>(const DevBuf<int2> &, const int64_t *, const int32_t *, const void *,
                                     const int64_t *, const double *, double *, const int64_t *, const int64_t *,
                                     const int32_t *, cudaStream_t);
template void stored_product<float>(const DevBuf<int2> &, const int64_t *, const int32_t *, const void *,
                                    const int64_t *, const float *, double *, const int64_t *, const int64_t *,
                                    const int32_t *, cudaStream_t);

}  // namespace h2
