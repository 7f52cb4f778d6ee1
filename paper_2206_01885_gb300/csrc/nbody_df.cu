// nbody_df.cu -- the float64 form's Coulomb coupling and nearfield products
// (section 2.1's H^2 matvec: sum_j K(X_i, X_j) w_j over far skeleton pairs and
// near leaf pairs) in float-float arithmetic on the float32 units.
//
// On this GPU float64 runs at about 1/74 of the float32 rate (measured FMA
// throughput 1.06 against 78.4 TFLOP/s), and an on-the-fly float64 Coulomb
// evaluation costs ~14 float64 instructions.  Here every quantity is an
// unevaluated sum hi + lo of two float32 numbers (about 48 significant bits):
// differences by TwoSum, squares by FMA-exact products, 1/sqrt(r^2) by the
// float32 approximation refined with one second-order correction computed
// from an exact residual, products and sums accumulated with their rounding
// errors.  One evaluation is ~80-100 float32 instructions; its relative error
// is below 2^-43 (far below the 1e-8 the float64 form is built for).  Row sums
// are folded into float64 once per block pair, column sums once per 32
// sources (float64 atomics, as in the float64 kernels).
//
// Coordinates.  Coupling (skeleton points of well-separated nodes): offsets
// from each node's cell centre as float pairs, the target moved into the
// source node's frame once per pair; x - y is then exact to ~2^-48 of a cell
// width, well below 2^-46 of |x - y| for admissible pairs.  Nearfield
// (neighbouring leaves, where two points can be much closer than a cell): an
// exact integer cell index K along each coordinate (a float32 integer) plus
// the residual in cells as a float pair, in units of a power of two u' near
// side / 2^B; x - y = (K_x - K_y) + (r_x - r_y) has an exact integer part, so
// its error is ~2^-48 of |x - y| itself, as in float64; the sums are scaled by
// 1/u' (exact) when they are folded into float64.
#include <mutex>

#include "h2_internal.cuh"

namespace h2 {
namespace {

constexpr int DF_WARPS = 8;

// s + e = a + b exactly (Knuth's TwoSum); explicitly rounded operations, never
// contracted into fused multiply-adds
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// t + m u as a float pair, m an integer (|m| < 2^23, exact in float32) and
// u = uh + ul: the product m uh is exact as p + fma(m, uh, -p)
__device__ __forceinline__ float2 df_shift(float2 t, int m, float uh, float ul) {
    const float mf = (float)m;
    const float dh = __fmul_rn(mf, uh);
    const float dl = fmaf(mf, ul, fmaf(mf, uh, -dh));
    float s, e;
    two_sum(t.x, dh, s, e);
    e = __fadd_rn(e, __fadd_rn(t.y, dl));
    float h, l;
    two_sum(s, e, h, l);
    return make_float2(h, l);
}

// (a, lo) with a + lo = t - s to ~2^-48 of the operands; then (a + lo)^2 as
// p + e (p = a^2 rounded, e = its exact error + (2a + lo) lo)
__device__ __forceinline__ void df_sq_diff(float th, float tl, float sh, float sl, float &p, float &e) {
    float a, ea;
    two_sum(th, -sh, a, ea);
    const float lo = __fadd_rn(ea, __fsub_rn(tl, sl));
    p = __fmul_rn(a, a);
    e = fmaf(fmaf(2.f, a, lo), lo, fmaf(a, a, -p));
}

// the same for points given as an exact integer cell index K (a float32
// integer) plus a residual rh + rl in cells: (Kt - Ks) is exact, the residuals'
// difference is taken by TwoSum, and their sum by another
__device__ __forceinline__ void df_sq_diff_int(float kt, float rth, float rtl, float ks, float rsh, float rsl,
                                               float &p, float &e) {
    float d, ed;
    two_sum(rth, -rsh, d, ed);
    const float dl = __fadd_rn(ed, __fsub_rn(rtl, rsl));
    float a, ea;
    two_sum(__fsub_rn(kt, ks), d, a, ea);
    const float lo = __fadd_rn(ea, dl);
    p = __fmul_rn(a, a);
    e = fmaf(fmaf(2.f, a, lo), lo, fmaf(a, a, -p));
}

// 1/r from r^2 = p_k + e_k summed over k (float pairs): kh + kl; r2 > 0
// unless ZERO_OK and the points coincide (then 0)
template <bool ZERO_OK>
__device__ __forceinline__ void df_rsqrt_sum(float p0, float e0, float p1, float e1, float p2, float e2, float &kh,
                                             float &kl) {
    float s01, r01, s, r2;
    two_sum(p0, p1, s01, r01);
    two_sum(s01, p2, s, r2);
    const float low = __fadd_rn(__fadd_rn(__fadd_rn(r01, r2), __fadd_rn(e0, e1)), e2);
    const float rh = __fadd_rn(s, low);  // s >= 0 dominates low: Fast2Sum
    const float rl = __fsub_rn(low, __fsub_rn(rh, s));
    float y0;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(y0) : "f"(rh));  // relative error below 2^-22
    // residual e = 1 - r2 y0^2 from exact pieces: y0^2 = q + eq, rh q = m + em,
    // 1 - m exact (m is within 2^-21 of 1); the correction y0 (e/2 + 3e^2/8)
    // leaves an O(e^3) error, below 2^-60
    const float q = __fmul_rn(y0, y0);
    const float eq = fmaf(y0, y0, -q);
    const float m = __fmul_rn(rh, q);
    const float em = fmaf(rh, q, -m);
    const float tt = fmaf(rl, q, fmaf(rh, eq, em));
    const float ee = __fsub_rn(__fsub_rn(1.f, m), tt);
    const float c = __fmul_rn(__fmul_rn(y0, ee), fmaf(0.375f, ee, 0.5f));
    if (ZERO_OK && !(rh > 0.f)) {  // kappa(x, x) = 0 (a leaf's own block)
        kh = 0.f;
        kl = 0.f;
    } else {
        kh = y0;
        kl = c;
    }
}

// 1/|t - s| for points as float pairs (t in the source node's frame)
template <bool ZERO_OK>
__device__ __forceinline__ void df_coulomb(const float2 (&t)[3], float4 sh, float4 sl, float &kh, float &kl) {
    float p0, e0, p1, e1, p2, e2;
    df_sq_diff(t[0].x, t[0].y, sh.x, sl.x, p0, e0);
    df_sq_diff(t[1].x, t[1].y, sh.y, sl.y, p1, e1);
    df_sq_diff(t[2].x, t[2].y, sh.z, sl.z, p2, e2);
    df_rsqrt_sum<ZERO_OK>(p0, e0, p1, e1, p2, e2, kh, kl);
}

// 1/|t - s| in cells for points as integer cells + residuals: t = (K, rh, rl)
// per coordinate; s: sk (K, weight hi), sh (residual hi, weight lo), sl
// (residual lo)
template <bool ZERO_OK>
__device__ __forceinline__ void df_coulomb_int(const float (&t)[3][3], float4 sk, float4 sh, float4 sl, float &kh,
                                               float &kl) {
    float p0, e0, p1, e1, p2, e2;
    df_sq_diff_int(t[0][0], t[0][1], t[0][2], sk.x, sh.x, sl.x, p0, e0);
    df_sq_diff_int(t[1][0], t[1][1], t[1][2], sk.y, sh.y, sl.y, p1, e1);
    df_sq_diff_int(t[2][0], t[2][1], t[2][2], sk.z, sh.z, sl.z, p2, e2);
    df_rsqrt_sum<ZERO_OK>(p0, e0, p1, e1, p2, e2, kh, kl);
}

// (ah, al) += (kh + kl) (wh + wl), the product's rounding error kept
__device__ __forceinline__ void df_mac(float &ah, float &al, float kh, float kl, float wh, float wl) {
    const float p = __fmul_rn(kh, wh);
    const float lo = fmaf(kh, wl, fmaf(kl, wh, fmaf(kh, wh, -p)));
    float s, e;
    two_sum(ah, p, s, e);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(e, lo));
}

// Symmetric tiled N-body for the float64 form's Coulomb products (one
// right-hand side), the structure of the float64/float32 symmetric kernel:
// node i's list walked from its first entry j >= i, a CTA per tile of 32
// targets (a lane each), warps over the pairs, 32 sources staged at a time
// (stored twice) and rotated so that lane l meets source (l + q) mod 32 at
// step q while the column sum rides one lane down per step.  Weights are
// float pairs.  Padding: far sentinels with weight 0.
//   NEAR = false (coupling): X0..X2 are float pairs relative to each node's
//     cell centre lo + A u (A the integer doubled centre, u = side / 2^(B+1));
//     the target moves into the source node's frame by (A_i - A_j) u once per
//     pair; scale = 1.
//   NEAR = true (nearfield): P holds three float4 per point, (K, 0), (rh, 0),
//     (rl, 0): integer cells and residuals in units of u'; sums are in 1/cells
//     and scale = 1/u'.
template <bool NEAR>
__global__ void __launch_bounds__(DF_WARPS * 32)
    k_nbody_sym_df(const int2 *tiles, const int64_t *start, const int32_t *count, const float2 *X0,
                   const float2 *X1, const float2 *X2, const int32_t *A0, const int32_t *A1, const int32_t *A2,
                   float uh, float ul, const float4 *P, double scale, const float2 *w, double *out,
                   const int64_t *lptr, const int64_t *lfirst, const int32_t *lidx) {
    constexpr int NV = NEAR ? 3 : 2;  // float4 words per staged source
    __shared__ float4 stg[DF_WARPS][64][NV];
    __shared__ double part[DF_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 tl = tiles[blockIdx.x];
    const int i = tl.x;
    const int64_t ts = start[i];
    const int tn = count[i];
    const int a = tl.y + lane;
    const bool act = a < tn;
    const float2 zero2 = make_float2(0.f, 0.f);
    const float2 tw = act ? w[ts + a] : zero2;
    // the target: NEAR (K, rh, rl) per coordinate; otherwise float pairs
    float tk[3][3] = {{1e18f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float2 t0 = make_float2(1e18f, 0.f), t1 = zero2, t2 = zero2;
    int ai0 = 0, ai1 = 0, ai2 = 0;
    if constexpr (NEAR) {
        if (act) {
            const float4 k = P[3 * (ts + a)], rh = P[3 * (ts + a) + 1], rl = P[3 * (ts + a) + 2];
            tk[0][0] = k.x; tk[1][0] = k.y; tk[2][0] = k.z;
            tk[0][1] = rh.x; tk[1][1] = rh.y; tk[2][1] = rh.z;
            tk[0][2] = rl.x; tk[1][2] = rl.y; tk[2][2] = rl.z;
        }
    } else {
        if (act) {
            t0 = X0[ts + a];
            t1 = X1[ts + a];
            t2 = X2[ts + a];
        }
        ai0 = A0[i];
        ai1 = A1[i];
        ai2 = A2[i];
    }
    double acc = 0.0;
    for (int64_t e = lfirst[i] + warp; e < lptr[i + 1]; e += DF_WARPS) {
        const int jn = lidx[e];
        const bool sym = jn != i;
        const int64_t ss = start[jn];
        const int sn = count[jn];
        float2 tp[3];
        if constexpr (!NEAR) {
            tp[0] = df_shift(t0, ai0 - A0[jn], uh, ul);
            tp[1] = df_shift(t1, ai1 - A1[jn], uh, ul);
            tp[2] = df_shift(t2, ai2 - A2[jn], uh, ul);
        }
        float bh = 0.f, bl = 0.f;
        for (int q0 = 0; q0 < sn; q0 += 32) {
            const int cnt = min(32, sn - q0);
            __syncwarp();
            {
                const bool ok = lane < cnt;
                const int64_t sp = ss + q0 + lane;
                const float2 sw = ok ? w[sp] : zero2;
                float4 v[NV];
                if constexpr (NEAR) {
                    v[0] = ok ? P[3 * sp] : make_float4(-1e18f, 0.f, 0.f, 0.f);
                    v[1] = ok ? P[3 * sp + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                    v[2] = ok ? P[3 * sp + 2] : make_float4(0.f, 0.f, 0.f, 0.f);
                    v[0].w = sw.x;
                    v[1].w = sw.y;
                } else {
                    const float2 s0 = ok ? X0[sp] : make_float2(-1e18f, 0.f), s1 = ok ? X1[sp] : zero2,
                                 s2 = ok ? X2[sp] : zero2;
                    v[0] = make_float4(s0.x, s1.x, s2.x, sw.x);
                    v[1] = make_float4(s0.y, s1.y, s2.y, sw.y);
                }
#pragma unroll
                for (int c = 0; c < NV; c++) {
                    stg[warp][lane][c] = v[c];
                    stg[warp][lane + 32][c] = v[c];
                }
            }
            __syncwarp();
            if (sym) {
                float ch = 0.f, cl = 0.f;
#pragma unroll 4
                for (int q = 0; q < 32; q++) {
                    float kh, kl, wh, wl;
                    if constexpr (NEAR) {
                        const float4 v0 = stg[warp][lane + q][0], v1 = stg[warp][lane + q][1],
                                     v2 = stg[warp][lane + q][2];
                        df_coulomb_int<false>(tk, v0, v1, v2, kh, kl);
                        wh = v0.w;
                        wl = v1.w;
                    } else {
                        const float4 vh = stg[warp][lane + q][0], vl = stg[warp][lane + q][1];
                        df_coulomb<false>(tp, vh, vl, kh, kl);
                        wh = vh.w;
                        wl = vl.w;
                    }
                    df_mac(bh, bl, kh, kl, wh, wl);
                    df_mac(ch, cl, kh, kl, tw.x, tw.y);
                    ch = __shfl_sync(0xffffffffu, ch, (lane + 1) & 31);
                    cl = __shfl_sync(0xffffffffu, cl, (lane + 1) & 31);
                }
                if (lane < cnt) atomicAdd(out + ss + q0 + lane, ((double)ch + (double)cl) * scale);
            } else {
                for (int q = 0; q < cnt; q++) {  // (cnt is the same in every lane)
                    float kh, kl, wh, wl;
                    if constexpr (NEAR) {
                        const float4 v0 = stg[warp][q][0], v1 = stg[warp][q][1], v2 = stg[warp][q][2];
                        df_coulomb_int<true>(tk, v0, v1, v2, kh, kl);
                        wh = v0.w;
                        wl = v1.w;
                    } else {
                        const float4 vh = stg[warp][q][0], vl = stg[warp][q][1];
                        df_coulomb<true>(tp, vh, vl, kh, kl);
                        wh = vh.w;
                        wl = vl.w;
                    }
                    df_mac(bh, bl, kh, kl, wh, wl);
                }
            }
        }
        acc += ((double)bh + (double)bl) * scale;
    }
    part[warp][lane] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int aa = tl.y + threadIdx.x;
        if (aa < tn) {
            double sum = 0.0;
            for (int wv = 0; wv < DF_WARPS; wv++) sum += part[wv][threadIdx.x];
            atomicAdd(out + ts + aa, sum);
        }
    }
}

// the integer doubled cell centre A = (2c + 1) 2^(B - level) per coordinate
// (the centre is lo + A u, u = side / 2^(B+1))
__global__ void k_cell_ints(const int32_t *level, const uint64_t *prefix, int nn, int B, int32_t *A0, int32_t *A1,
                            int32_t *A2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const int l = level[i];
    uint32_t c[3] = {0, 0, 0};
    for (int b = 0; b < l; b++)
        for (int k = 0; k < 3; k++) c[k] |= (uint32_t)((prefix[i] >> (3 * b + k)) & 1ull) << b;
    A0[i] = (int32_t)((2u * c[0] + 1u) << (B - l));
    A1[i] = (int32_t)((2u * c[1] + 1u) << (B - l));
    A2[i] = (int32_t)((2u * c[2] + 1u) << (B - l));
}

__device__ __forceinline__ float2 df_split(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// every point as integer cells K and a residual r (float pair) in units of
// u' (a power of two): x - lo = (K + r) u' with x - lo kept exact as a
// double pair, so r is exact to float64 rounding before its split
__global__ void k_df_cells(const double *x0, const double *x1, const double *x2, int64_t n, double lo0, double lo1,
                           double lo2, double inv_u, float4 *P) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double x[3] = {x0[p], x1[p], x2[p]}, lo[3] = {lo0, lo1, lo2};
    float kf[3], rh[3], rl[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double dh = x[k] - lo[k];              // x - lo = dh + de exactly (TwoSum)
        const double bb = dh - x[k];
        const double de = (x[k] - (dh - bb)) + (-lo[k] - bb);
        const double vh = dh * inv_u, ve = de * inv_u;  // exact: inv_u is a power of two
        const double K = floor(vh);
        const double r = (vh - K) + ve;              // vh - K is exact
        kf[k] = (float)K;                            // exact: K < 2^24
        const float h = (float)r;
        rh[k] = h;
        rl[k] = (float)(r - (double)h);
    }
    P[3 * p] = make_float4(kf[0], kf[1], kf[2], 0.f);
    P[3 * p + 1] = make_float4(rh[0], rh[1], rh[2], 0.f);
    P[3 * p + 2] = make_float4(rl[0], rl[1], rl[2], 0.f);
}

// the same for the skeleton points of every node (skeleton coordinates in
// node order, node i's at sk_off[i] .. sk_off[i] + k_i)
__global__ void k_df_skel(int nn, const int32_t *kk, const int64_t *off, const double *s0, const double *s1,
                          const double *s2, const int32_t *A0, const int32_t *A1, const int32_t *A2, double lo0,
                          double lo1, double lo2, double u, float2 *r0, float2 *r1, float2 *r2) {
    const int i = blockIdx.x;
    if (i >= nn) return;
    const double c0 = (double)A0[i], c1 = (double)A1[i], c2 = (double)A2[i];
    for (int q = threadIdx.x; q < kk[i]; q += blockDim.x) {
        const int64_t o = off[i] + q;
        r0[o] = df_split(fma(-c0, u, s0[o] - lo0));
        r1[o] = df_split(fma(-c1, u, s1[o] - lo1));
        r2[o] = df_split(fma(-c2, u, s2[o] - lo2));
    }
}

__global__ void k_split_vec(const double *v, int64_t n, float2 *out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) out[p] = df_split(v[p]);
}

double df_unit(const h2_tree_s *t) { return ldexp(t->geom.side, -(t->B + 1)); }

// u' = the largest power of two <= side / 2^B (1 when side = 0): at most
// 2^(B+1) cells per coordinate, exact in float32 for B = 21
double df_cell(const h2_tree_s *t) {
    const double c = ldexp(t->geom.side, -t->B);
    if (!(c > 0.0)) return 1.0;
    int ex = 0;
    frexp(c, &ex);  // c = f 2^ex, f in [0.5, 1)
    return ldexp(1.0, ex - 1);
}

// The float64 form's Coulomb kernel blocks A_i = K(Y_i*, Xbar_i) (Algorithm 2)
// in float-float arithmetic: each entry 1/|y - x| from the points' integer
// cells and residuals (exact integer part, so full relative accuracy at any
// distance), scaled by the power of two 1/u' (exact) and stored as the float
// pair hi + lo in the entry's 8 bytes, the layout the float-float QR works
// in.  Columns split over the node's CTAs, rows over the threads, as
// k_keval_f64.
__global__ void k_keval_df(int lb, const int32_t *ycnt, const int32_t *cc, int32_t *const *yptr,
                           const int32_t *cand, const int64_t *coff, const int64_t *aoff, const float4 *P,
                           float scale, float2 *Abase) {
    const int a = blockIdx.x, i = lb + a;
    const int m = ycnt[i], c = cc[i];
    if (m == 0 || c == 0) return;
    const int32_t *Y = yptr[i];
    const int32_t *X = cand + coff[a];
    float2 *A = Abase + aoff[a];
    for (int l = blockIdx.y; l < c; l += gridDim.y) {
        const int32_t x = X[l];
        const float4 sk = P[3 * (int64_t)x], sh = P[3 * (int64_t)x + 1], sl = P[3 * (int64_t)x + 2];
        float2 *Acol = A + (int64_t)l * m;
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            const int64_t y = Y[r];
            const float4 tk = P[3 * y], th = P[3 * y + 1], tl = P[3 * y + 2];
            const float t[3][3] = {{tk.x, th.x, tl.x}, {tk.y, th.y, tl.y}, {tk.z, th.z, tl.z}};
            float kh, kl;
            df_coulomb_int<true>(t, sk, sh, sl, kh, kl);
            Acol[r] = make_float2(__fmul_rn(kh, scale), __fmul_rn(kl, scale));
        }
    }
}

// The exact sampled-row sums of the section 6 metric, (K z)_s = sum_q
// 1/|x_s - x_q| z_q, for 3D Coulomb in float-float arithmetic: every term from
// the points' integer cells and residuals (full relative accuracy at any
// distance, ~2^-43 a term), z as float pairs, float-pair accumulators.  CTA
// (chunk c, group of XD_ROWS rows) sums chunk c (ER_CHUNK points) for its
// rows, each point's coordinates and weight loaded once for all of them; the
// row's sum is reduced in a fixed order and written in float64 (scaled by
// 1/u', a power of two) to part[r * nch + c].  A row index outside [0, n)
// gives NaN, as in the float64 kernels.  p = iperm[row] is its tree position.
constexpr int XD_ROWS = 8;
constexpr int XD_THREADS = 256;

__global__ void __launch_bounds__(XD_THREADS)
    k_exact_part_df(const int64_t *rows, int64_t nrows, const int32_t *iperm, const float4 *P, const float2 *zf,
                    int64_t n, int64_t chunk, int nch, double inv_u, double *part) {
    __shared__ float2 red[XD_ROWS][XD_THREADS / 32];
    const int64_t r0 = (int64_t)blockIdx.y * XD_ROWS;
    const int c = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float t[XD_ROWS][3][3];
    bool ok[XD_ROWS];
#pragma unroll
    for (int i = 0; i < XD_ROWS; i++) {
        const int64_t r = r0 + i;
        const int64_t row = r < nrows ? rows[r] : -1;
        ok[i] = row >= 0 && row < n;
        const int64_t p = ok[i] ? iperm[row] : 0;
        const float4 k4 = P[3 * p], h4 = P[3 * p + 1], l4 = P[3 * p + 2];
        t[i][0][0] = k4.x; t[i][0][1] = h4.x; t[i][0][2] = l4.x;
        t[i][1][0] = k4.y; t[i][1][1] = h4.y; t[i][1][2] = l4.y;
        t[i][2][0] = k4.z; t[i][2][1] = h4.z; t[i][2][2] = l4.z;
    }
    float ah[XD_ROWS], al[XD_ROWS];
#pragma unroll
    for (int i = 0; i < XD_ROWS; i++) ah[i] = al[i] = 0.f;
    const int64_t q0 = (int64_t)c * chunk, q1 = min(n, q0 + chunk);
    for (int64_t q = q0 + threadIdx.x; q < q1; q += XD_THREADS) {
        const float4 sk = P[3 * q], sh = P[3 * q + 1], sl = P[3 * q + 2];
        const float2 w = zf[q];
#pragma unroll
        for (int i = 0; i < XD_ROWS; i++) {
            float kh, kl;
            df_coulomb_int<true>(t[i], sk, sh, sl, kh, kl);
            df_mac(ah[i], al[i], kh, kl, w.x, w.y);
        }
    }
    // each row: warp sums in float-float (fixed shuffle order), then the
    // warps' sums added in order in float64 by one thread
#pragma unroll
    for (int i = 0; i < XD_ROWS; i++) {
        float h = ah[i], l = al[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
            float s, e;
            two_sum(h, oh, s, e);
            e = __fadd_rn(e, __fadd_rn(l, ol));
            two_sum(s, e, h, l);
        }
        if (lane == 0) red[i][warp] = make_float2(h, l);
    }
    __syncthreads();
    if (threadIdx.x < XD_ROWS) {
        const int i = threadIdx.x;
        const int64_t r = r0 + i;
        if (r < nrows) {
            double acc = 0.0;
            for (int w = 0; w < XD_THREADS / 32; w++) acc += (double)red[i][w].x + (double)red[i][w].y;
            part[r * nch + c] = ok[i] ? acc * inv_u : __longlong_as_double(0x7ff8000000000000ll);
        }
    }
}

}  // namespace

// exact rows of a 3D Coulomb tree in float-float arithmetic (k_exact_part_df):
// zm is z in tree order (float64, device); part holds nrows x nch partial
// sums, nch = ceil(n / chunk)
void exact_rows_df_parts(h2_tree_s *t, const double *zm, const int64_t *rows, int64_t nrows, int64_t chunk,
                         int nch, double *part, cudaStream_t s) {
    ensure_df_tree(t, s);
    const int64_t n = t->n;
    DevBuf<float2> zf;
    zf.alloc((size_t)std::max<int64_t>(n, 1), s);
    split_vector(zm, n, zf.p, s);
    for (int64_t r0 = 0; r0 < nrows; r0 += (int64_t)65535 * XD_ROWS) {
        const int64_t nr = std::min<int64_t>((int64_t)65535 * XD_ROWS, nrows - r0);
        k_exact_part_df<<<dim3((unsigned)nch, (unsigned)((nr + XD_ROWS - 1) / XD_ROWS)), XD_THREADS, 0, s>>>(
            rows + r0, nr, t->iperm.p, t->xcell.p, zf.p, n, chunk, nch, 1.0 / df_cell(t), part + r0 * nch);
        H2_LAUNCH("k_exact_part_df");
    }
}

void keval_df(const h2_tree_s *t, int nl, int ysplit, int lb, const int32_t *ycnt, const int32_t *cc,
              int32_t *const *yptr, const int32_t *cand, const int64_t *coff, const int64_t *aoff, float2 *A,
              cudaStream_t s) {
    if (nl <= 0) return;
    k_keval_df<<<dim3(nl, ysplit), 256, 0, s>>>(lb, ycnt, cc, yptr, cand, coff, aoff, t->xcell.p,
                                                (float)(1.0 / df_cell(t)), A);
    H2_LAUNCH("k_keval_df");
}

// the tree's float-pair point coordinates and integer cell centres, built on
// first use (3D trees).  Several host threads may construct on one tree at
// once (h2_construct_batched): the first builds under a lock and waits for
// its stream before publishing, so no other stream reads a half-built buffer.
static std::mutex df_tree_mutex;

void ensure_df_tree(h2_tree_s *t, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(df_tree_mutex);
    if (t->df_ready) return;
    const int nn = t->nnodes;
    const int64_t n = t->n;
    DevBuf<int32_t> A[3];
    DevBuf<float4> P;
    for (int k = 0; k < 3; k++) A[k].alloc(nn, s);
    P.alloc((size_t)3 * n, s);
    k_cell_ints<<<blocks_for(nn, 256), 256, 0, s>>>(t->level.p, t->prefix.p, nn, t->B, A[0].p, A[1].p, A[2].p);
    H2_LAUNCH("k_cell_ints");
    k_df_cells<<<blocks_for(n, 256), 256, 0, s>>>(t->xs[0].p, t->xs[1].p, t->xs[2].p, n, t->geom.lo[0],
                                                   t->geom.lo[1], t->geom.lo[2], 1.0 / df_cell(t), P.p);
    H2_LAUNCH("k_df_cells");
    H2_CUDA(cudaStreamSynchronize(s));
    // the tree frees them on its own stream (s may be a batched call's
    // internal stream, gone when the tree is freed)
    for (int k = 0; k < 3; k++) {
        A[k].rebind(t->stream);
        t->cellA[k] = std::move(A[k]);
    }
    P.rebind(t->stream);
    t->xcell = std::move(P);
    t->df_ready = true;
}

void ensure_df_matrix(h2_matrix_s *A, cudaStream_t s) {
    if (A->df_ready) return;
    h2_tree_s *t = A->tree;
    ensure_df_tree(t, s);
    const int64_t kt = std::max<int64_t>(A->ktotal, 1);
    DevBuf<float2> X[3];
    for (int k = 0; k < 3; k++) X[k].alloc(kt, s);
    k_df_skel<<<std::max(1, t->nnodes), 128, 0, s>>>(t->nnodes, A->k.p, A->sk_off.p, A->skc[0].p, A->skc[1].p,
                                                     A->skc[2].p, t->cellA[0].p, t->cellA[1].p, t->cellA[2].p,
                                                     t->geom.lo[0], t->geom.lo[1], t->geom.lo[2], df_unit(t),
                                                     X[0].p, X[1].p, X[2].p);
    H2_LAUNCH("k_df_skel");
    for (int k = 0; k < 3; k++) A->skdf[k] = std::move(X[k]);
    A->df_ready = true;
}

void split_vector(const double *v, int64_t n, float2 *out, cudaStream_t s) {
    k_split_vec<<<blocks_for(n, 256), 256, 0, s>>>(v, n, out);
    H2_LAUNCH("k_split_vec");
}

void nbody_sym_df(const h2_tree_s *t, const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count,
                  const DevBuf<float2> *X, const float2 *w, double *out, const int64_t *lptr, const int64_t *lfirst,
                  const int32_t *lidx, cudaStream_t s) {
    if (tiles.n == 0) return;
    if (X == nullptr) {  // nearfield: integer cells + residuals of the tree's points
        k_nbody_sym_df<true><<<(unsigned)tiles.n, DF_WARPS * 32, 0, s>>>(
            tiles.p, start, count, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f, 0.f, t->xcell.p,
            1.0 / df_cell(t), w, out, lptr, lfirst, lidx);
    } else {  // coupling: offsets of skeleton points from their node's centre
        const double u = df_unit(t);
        const float uh = (float)u, ul = (float)(u - (double)uh);
        k_nbody_sym_df<false><<<(unsigned)tiles.n, DF_WARPS * 32, 0, s>>>(
            tiles.p, start, count, X[0].p, X[1].p, X[2].p, t->cellA[0].p, t->cellA[1].p, t->cellA[2].p, uh, ul,
            nullptr, 1.0, w, out, lptr, lfirst, lidx);
    }
    H2_LAUNCH("k_nbody_sym_df");
}

}  // namespace h2
