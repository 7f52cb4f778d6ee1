// h2_internal.cuh -- shared declarations of the sm_103a H^2 library.
//
// Host orchestration is C++ with exceptions internally; every C-ABI entry
// point catches them and turns them into an h2_status plus a thread-local
// message.  Device memory comes from the stream-ordered allocator
// (cudaMallocAsync) on the caller's stream.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/h2.h"

namespace h2 {

// ------------------------------------------------------------------ errors
struct Error {
    h2_status st;
    std::string msg;
};

[[noreturn]] void fail(h2_status st, const std::string &msg);
void cuda_check(cudaError_t e, const char *what, const char *file, int line);
void note_launches(int k);  // adds to the library's count of kernel launches
long long launches_total();
#define H2_CUDA(call) ::h2::cuda_check((call), #call, __FILE__, __LINE__)
// after each kernel launch: count it and surface a launch error
#define H2_LAUNCH(what) (::h2::note_launches(1), ::h2::cuda_check(cudaGetLastError(), what, __FILE__, __LINE__))
#define H2_REQUIRE(cond, msg)                                             \
    do {                                                                  \
        if (!(cond)) ::h2::fail(H2_ERR_INVALID_ARG, std::string(msg));    \
    } while (0)

// ----------------------------------------------------------- device memory
void *dmalloc_bytes(size_t bytes, cudaStream_t s);
void dfree_bytes(void *p, cudaStream_t s);
int64_t debug_fail_alloc(int64_t k);
// measured float64 / float32 fused multiply-add throughput of this device (TFLOP/s)
void fma_peaks(double *fp64_tflops, double *fp32_tflops, cudaStream_t s);  // arm the k-th allocation to fail; returns the count since the last arming

// Owning device array, released on the stream it was allocated on.
template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        if (count) p = static_cast<T *>(dmalloc_bytes(count * sizeof(T), st));  // throws on failure
        n = count;  // only once the memory exists: a failed alloc leaves an empty buffer
    }
    void release() {
        if (p) dfree_bytes(p, s);
        p = nullptr;
        n = 0;
    }
    T *get() const { return p; }
    // release on st from now on (st must be ordered after every use so far)
    void rebind(cudaStream_t st) { s = st; }
};

// copy helpers (synchronous on the stream)
template <class T>
T read_scalar(const T *dptr, cudaStream_t s) {
    T v;
    H2_CUDA(cudaMemcpyAsync(&v, dptr, sizeof(T), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    return v;
}
template <class T>
std::vector<T> read_vec(const T *dptr, size_t n, cudaStream_t s) {
    std::vector<T> v(n);
    if (n) {
        H2_CUDA(cudaMemcpyAsync(v.data(), dptr, n * sizeof(T), cudaMemcpyDeviceToHost, s));
        H2_CUDA(cudaStreamSynchronize(s));
    }
    return v;
}

// ----------------------------------------------------------- primitives
// out[i] = sum_{j<i} in[j] for i in [0, n]; out has n+1 entries (out[n] = total).
void scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
void scan_exclusive_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of 64-bit keys on their low `nbits` bits; `vals`
// (may be null) are permuted alongside.  Buffers are sorted in place.
void radix_sort(uint64_t *keys, int32_t *vals, int64_t n, int nbits, cudaStream_t s);

// ------------------------------------------------------------- profiling
// Optional CUDA-event timing of the main kernels, on the stream each kernel is
// launched on; totals are read through h2_get_stats(NULL, ...).
enum KernelKind {
    KT_DATAREDUCT = 0, KT_KEVAL, KT_CPQR, KT_SOLVE, KT_UPWARD, KT_COUPLING, KT_DOWNWARD, KT_NEAR, KT_EXACT,
    KT_SORT, KT_LISTS, KT_FILL, KT_COUPLING_ST, KT_NEAR_ST, KT_COUNT
};
extern const char *const kernel_kind_names[KT_COUNT];
bool profiling_enabled();
void profile_set(bool on, bool reset);
std::string profile_json();
struct ProfScope {
    int kind;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr;
    ProfScope(int k, cudaStream_t st);
    ~ProfScope();
};

inline int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 2147483647 ? 2147483647 : b));
}

// ---------------------------------------------------------------- handles
enum : uint32_t {
    TAG_TREE = 0x48325452u,
    TAG_HIDR = 0x48324844u,
    TAG_MATRIX = 0x48324d58u,
    TAG_GRAPH = 0x48324750u,
    TAG_DEAD = 0xdeadbeefu
};

struct Geom {
    double lo[3];
    double hi[3];
    double side;
    double scale;  // 2^B / side, 0 when side == 0
    int nonfinite;  // 1 when some coordinate is NaN or infinite
};

struct PhaseTimes {
    double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

}  // namespace h2

struct h2_tree_s {
    uint32_t tag = h2::TAG_TREE;
    int refs = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    int d = 0, B = 0, q = 0, tau_num = 7, tau_den = 10;
    h2::Geom geom{};
    h2::DevBuf<double> xs[3];     // coordinates in Morton order, one array per dimension
    h2::DevBuf<uint64_t> key;     // sorted Morton keys
    h2::DevBuf<int32_t> perm;     // Morton position -> original index
    h2::DevBuf<int32_t> iperm;    // original index -> Morton position
    int nnodes = 0, nlevels = 0;
    std::vector<int> lptr;        // host: nodes of level l are [lptr[l], lptr[l+1])
    h2::DevBuf<int32_t> level, parent, fchild, nchild, begin, end;
    h2::DevBuf<uint64_t> prefix;
    h2::DevBuf<int64_t> near_ptr, far_ptr;
    h2::DevBuf<int32_t> near_idx, far_idx;
    int64_t nnear = 0, nfar = 0;
    int max_leaf = 0;             // largest leaf population
    double ms_tree = 0, ms_lists = 0;
    h2::DevBuf<double> cen[3];    // cell centre of every node
    h2::DevBuf<float> xr[3];      // point coordinates relative to their leaf's centre (float32 kernels)
    h2::DevBuf<float4> xq;        // x - root corner as float32 hi + lo, two float4 per point (see DRPoints)
    h2::DevBuf<float2> cenf[3];   // cell centre - root corner split into float32 hi + lo (float32 N-body)
    h2::DevBuf<int2> near_tiles;  // (leaf, first target) tiles of the nearfield kernel, built on first use
    int near_tile_tpt = 0;
    h2::DevBuf<int64_t> near_first, far_first;  // first list entry of each node with index >= its own
    h2::DevBuf<int64_t> leaf_start;  // begin of every node as int64 (nearfield point sets)
    h2::DevBuf<int32_t> leaf_count;  // end - begin of every node
    // coordinates of the float64 form's float-float Coulomb products (3D, built
    // on first use): integer doubled cell centres A of the nodes (centre =
    // lo + A u, u = side / 2^(B+1)), and every point as integer cells K and a
    // float-pair residual in units of a power of two u' (three float4 a point)
    bool df_ready = false;
    h2::DevBuf<int32_t> cellA[3];
    h2::DevBuf<float4> xcell;
    // tiles of 128 targets of the tensor-core nearfield (several right-hand
    // sides, mixed form), built on first use; the kernel's timeout flag
    h2::DevBuf<int2> near_tiles_tc;
    bool near_tiles_tc_ready = false;
    h2::DevBuf<int> tc_status;
};

struct h2_hidr_s {
    uint32_t tag = h2::TAG_HIDR;
    int refs = 0;
    h2_tree_s *tree = nullptr;
    cudaStream_t stream = nullptr;
    int g1 = 0, g2 = 0;
    int method = 0;  // DataReduct: 0 volume-based, 1 surface-based, 2 farthest point sampling
    bool il_reduce = false;  // Y_i* also takes the reduction of its interaction-list part alone
    bool copy_sets = false;  // top-down sets copied out and binned entry by entry (H2_HIDR_COPY_SETS)
    // per node: count and device pointer into one of the per-level buffers
    h2::DevBuf<int32_t> xcnt, ycnt;
    h2::DevBuf<int32_t *> xptr, yptr;
    std::vector<h2::DevBuf<int32_t>> xbufs, ybufs;
    h2::DevBuf<long long> xbox, ybox;  // per node: bounding box of X_i*, Y_i* (6 integer keys)
    std::vector<int> xmax_level, ymax_level;  // host: largest set per level
    int64_t xtotal = 0, ytotal = 0, tmax = 0, ttotal = 0;
    int64_t iltotal = 0;  // entries of the interaction-list parts (interaction-list reduction only)
    double ms_up = 0, ms_down = 0;
    int members_levels = 0;  // top-down levels reduced by the search over members (hidr.cu)
};

struct h2_matrix_s {
    uint32_t tag = h2::TAG_MATRIX;
    int refs = 0;
    h2_tree_s *tree = nullptr;
    cudaStream_t stream = nullptr;
    int kid = 1;
    double kp[4] = {0, 0, 0, 0};
    double id_tol = 0;
    int prec = H2_PREC_FP64;
    h2::DevBuf<int32_t> k, c;          // rank and candidate count per node
    h2::DevBuf<int64_t> sk_off;        // exclusive scan of k over nodes (nnodes + 1)
    h2::DevBuf<int32_t> skel;          // skeletons, node order, each sorted
    h2::DevBuf<double> skc[3];         // skeleton coordinates, aligned with skel
    h2::DevBuf<float> skr[3];          // skeleton coordinates relative to their node's centre (float32)
    h2::DevBuf<void *> uptr;           // per node U_i (c_i x k_i, column-major; double or float)
    std::vector<h2::DevBuf<unsigned char>> ubufs;
    h2::DevBuf<int2> far_tiles;        // (node, first target) tiles of the coupling kernel
    int far_tile_tpt = 0;
    std::vector<int> kmax_level, cmax_level;  // host
    int64_t ktotal = 0, utotal = 0;
    int kmax = 0;
    double ms_construct = 0;
    double flops_qr = 0, evals_block = 0;
    double g_max = 0;  // largest |G| = |(R11^{-1} R12)^T| entry over all nodes (what strong RRQR would bound)
    double g_bound = 0;       // f of the exchanges bounding ||G||_max (0: none)
    int64_t exchanges = 0;    // exchanges made
    // stored coupling and nearfield blocks (memory mode STORE, or AUTO when
    // they fit): per list entry e with j >= i the row-major block K(i, j) at
    // element offset *_boff[e] (-1: not stored)
    int mem_mode = 0;                  // requested: H2_MEM_ON_THE_FLY / STORE / AUTO
    double mem_fraction = 0.5;         // share of the free device memory the blocks may take
    bool stored = false;               // blocks stored (the products read them)
    h2::DevBuf<unsigned char> far_blk, near_blk;
    h2::DevBuf<int64_t> far_boff, near_boff;
    int64_t stored_far_bytes = 0, stored_near_bytes = 0, stored_bytes_plan = 0;
    double ms_blocks = 0;
    // float64 form: Coulomb products in float-float arithmetic unless
    // fp64_products is set (then plain float64); skeleton offsets from their
    // node's centre as hi + lo, built on first use
    bool fp64_products = false;
    bool fp64_qr = false;  // float64 form: the QR's trailing updates in float64 (else float-float)
    bool tensor_core_products = false;  // mixed form: the 16-column nearfield on the tensor cores
    bool df_ready = false;
    h2::DevBuf<float2> skdf[3];
};

// a matvec recorded as a CUDA graph (h2_matvec_graph_create)
struct h2_graph_s {
    uint32_t tag = h2::TAG_GRAPH;
    h2_matrix_s *A = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~h2_graph_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

namespace h2 {

h2_tree_s *as_tree(void *h);
h2_hidr_s *as_hidr(void *h);
h2_matrix_s *as_matrix(void *h);

// phases (host orchestration, defined in the per-phase .cu files)
void tree_build_impl(h2_tree_s *t, const double *pts_dev_rowmajor);
void lists_build_impl(h2_tree_s *t);
void hidr_impl(h2_hidr_s *h);
void construct_impl(h2_matrix_s *A, h2_hidr_s *h);
// release every buffer of A on s from now on (s ordered after A's construction)
void matrix_rebind(h2_matrix_s *A, cudaStream_t s);
void matvec_impl(h2_matrix_s *A, const double *x_dev, double *y_dev, cudaStream_t s);
// nrhs columns, x and y column-major with leading dimension ld (device)
void matvec_multi_impl(h2_matrix_s *A, const void *x_dev, void *y_dev, int nrhs, int dtype, int64_t ld,
                       cudaStream_t s);
void exact_rows_impl(h2_tree_s *t, int kid, const double *kp, const double *z_dev, const int64_t *rows_dev,
                     int64_t nrows, double *out_dev, cudaStream_t s);
// float-float Coulomb products of the float64 form (3D)
void ensure_df_tree(h2_tree_s *t, cudaStream_t s);
// exact rows of a 3D Coulomb tree in float-float arithmetic: part[r * nch + c]
// = the sum over chunk c (chunk points) of row r (nbody_df.cu)
void exact_rows_df_parts(h2_tree_s *t, const double *zm, const int64_t *rows, int64_t nrows, int64_t chunk,
                         int nch, double *part, cudaStream_t s);
// float64 form, 3D Coulomb: kernel blocks of a level in float-float
// arithmetic, each entry a float pair hi + lo in its 8 bytes (nbody_df.cu)
void keval_df(const h2_tree_s *t, int nl, int ysplit, int lb, const int32_t *ycnt, const int32_t *cc,
              int32_t *const *yptr, const int32_t *cand, const int64_t *coff, const int64_t *aoff, float2 *A,
              cudaStream_t s);
void ensure_df_matrix(h2_matrix_s *A, cudaStream_t s);
void split_vector(const double *v, int64_t n, float2 *out, cudaStream_t s);
void nbody_sym_df(const h2_tree_s *t, const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count,
                  const DevBuf<float2> *X, const float2 *w, double *out, const int64_t *lptr, const int64_t *lfirst,
                  const int32_t *lidx, cudaStream_t s);
// the mixed form's nearfield for 16 right-hand sides on the tensor cores
void nbody_tc16(int kid, const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count, const float *X0,
                const float *X1, const float *X2, const float2 *F0, const float2 *F1, const float2 *F2,
                const float *w, int ws, double *out, int os, const int64_t *lptr, const int32_t *lidx, int d,
                double kp0, int *status, cudaStream_t s);
// evaluate and keep the coupling and nearfield blocks (mode H2_MEM_STORE:
// H2_ERR_OOM above `fraction` of the free memory; H2_MEM_AUTO: keep them
// only when they fit)
void store_blocks_impl(h2_matrix_s *A, int mode, double fraction);
// y += stored-block product of one list (one right-hand side)
template <class Real>
void stored_product(const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count, const void *blk,
                    const int64_t *boff, const Real *w, double *out, const int64_t *lptr, const int64_t *lfirst,
                    const int32_t *lidx, cudaStream_t s);

void exact_rows_noalloc_impl(h2_tree_s *t, int kid, const double *kp, const double *z_dev, const int64_t *rows_dev,
                             int64_t nrows, double *out_dev, cudaStream_t s);
void sampled_error_impl(const double *exact, const double *approx, const int64_t *rows, int64_t nrows, int64_t n,
                        double *err_out, cudaStream_t s);

// Coordinates DataReduct reads: float64 x (exact distances) and xq, the
// float64 difference x - ref (|x - ref| <= R per coordinate) split into float32
// pairs {hi, lo} with hi + lo equal to it within 2^-47 R, packed in one
// 32-byte record per point: xq[2s] = {hi0, hi1, hi2, lo0}, xq[2s+1] = {lo1, lo2, 0, 0}.
struct DRPoints {
    const double *x[3];
    const float4 *xq;
    double ref[3];
    double R;
};
// one DataReduct over an explicit point set (used by the calibration); ids
// are labels 0..n-1 of the points, box_keys their bounding box as 6
// order-preserving keys (host).  Output sorted labels.
int64_t datareduct_one(const DRPoints &pts, int d, int64_t n, int g, const long long *box_keys, int32_t *out_dev,
                       cudaStream_t s);
// order-preserving integer key of a float64 (host copy of the device form)
inline long long dkey_host(double x) {
    long long b;
    memcpy(&b, &x, sizeof b);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// Section 4.2 test problem at grid size g: relative Frobenius error of
// K(Z1, Z2) ~= U K(Zhat1, Z2) where U comes from the ID (tolerance id_tol) of
// K(DataReduct(Z2, g), Z1).  z1s, z2s: device SoA coordinates.
double calib_error_gpu(int d, int kid, double kp0, double id_tol, const double *const z1s[3], int n1,
                       const DRPoints &z2, const long long *z2_box, int n2, int g, int *k_out, int *m_out,
                       cudaStream_t s);

}  // namespace h2

// ----------------------------------------------------------- device math
// Squared distance ((x0-y0)^2 + (x1-y1)^2) + (x2-y2)^2 with explicitly rounded
// operations (no contraction), so that it is bit-identical to a plain IEEE
// evaluation in this order.
__device__ __forceinline__ double h2_dist2(int d, double a0, double a1, double a2, double b0, double b1,
                                           double b2) {
    double t = __dsub_rn(a0, b0);
    double s = __dmul_rn(t, t);
    if (d > 1) {
        t = __dsub_rn(a1, b1);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    if (d > 2) {
        t = __dsub_rn(a2, b2);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// kappa(x, y) as a function of r^2 = |x - y|^2, float64 (Table 1 and section 2):
// Coulomb 1/r with kappa(x, x) = 0; Gaussian exp(-r^2/h^2); exponential
// exp(-r/l); multiquadric sqrt(1 + r^2); bump (Table 1's kappa_4)
// exp(-1/(1 - a r^2)), 0 where a r^2 >= 1; power r^p (section 5.2).
__device__ __forceinline__ double h2_kappa(int kid, double kp0, double r2) {
    switch (kid) {
    case H2_K_COULOMB: return r2 > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(r2)) : 0.0;
    case H2_K_GAUSSIAN: return exp(-__ddiv_rn(r2, __dmul_rn(kp0, kp0)));
    case H2_K_EXPONENTIAL: return exp(-__ddiv_rn(__dsqrt_rn(r2), kp0));
    case H2_K_MULTIQUADRIC: return __dsqrt_rn(__dadd_rn(1.0, r2));
    case H2_K_BUMP: {
        const double t = __dmul_rn(kp0, r2);
        return t < 1.0 ? exp(-__ddiv_rn(1.0, __dadd_rn(1.0, -t))) : 0.0;
    }
    case H2_K_POWER: return r2 > 0.0 ? pow(r2, 0.5 * kp0) : 0.0;
    default: return 0.0;
    }
}

// float64 kappa in its fast forms (rsqrt: within 1 ulp of 1/sqrt) for
// products that are compared with a tolerance rather than bit for bit
// 1/sqrt(r2) for r2 >= 0, and 0 at r2 = 0 (Coulomb's kappa(x, x) = 0): the PTX
// approximation rsqrt.approx.ftz.f64 (relative error below 2^-20) refined by
// one third-order step of the series (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + ...,
// e = 1 - r2 y0^2, which leaves an O(e^3) error below float64 rounding;
// measured within 1 ulp of rsqrt() over r2 in [1e-300, 1e300].  Subnormal r2
// (outside the approximation's range) takes rsqrt().
__device__ __forceinline__ double h2_rsqrt64(double r2) {
    const long long bits = __double_as_longlong(r2);
    if (bits < 0x0010000000000000LL) return bits == 0 ? 0.0 : rsqrt(r2);
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(r2));
    const double t = r2 * y0;
    const double e = fma(-t, y0, 1.0);
    const double p = fma(e, 0.375, 0.5);
    return fma(y0 * e, p, y0);
}

// p: the kernel parameter in the form h2_kappa_param gives (a reciprocal
// formed once per launch instead of a float64 division per evaluation)
__device__ __forceinline__ double h2_kappa_fast(int kid, double p, double r2) {
    switch (kid) {
    case H2_K_COULOMB: return h2_rsqrt64(r2);
    case H2_K_GAUSSIAN: return exp(-r2 * p);
    case H2_K_EXPONENTIAL: return exp(-sqrt(r2) * p);
    case H2_K_MULTIQUADRIC: return sqrt(1.0 + r2);
    case H2_K_BUMP: {
        const double t = p * r2;
        return t < 1.0 ? exp(-1.0 / (1.0 - t)) : 0.0;
    }
    case H2_K_POWER: return r2 > 0.0 ? pow(r2, p) : 0.0;
    default: return 0.0;
    }
}

// kparams[0] in the form the fast kernels take: 1/h^2 (Gaussian), 1/l
// (exponential), a (bump), p/2 (power), unused otherwise
inline double h2_kappa_param(int kid, double kp0) {
    switch (kid) {
    case H2_K_GAUSSIAN: return 1.0 / (kp0 * kp0);
    case H2_K_EXPONENTIAL: return 1.0 / kp0;
    case H2_K_BUMP: return kp0;
    case H2_K_POWER: return 0.5 * kp0;
    default: return 0.0;
    }
}

// x . y with explicitly rounded operations in the order x0 y0 + x1 y1 + x2 y2
// (bit-identical to a plain IEEE evaluation in this order)
__device__ __forceinline__ double h2_dot(int d, double a0, double a1, double a2, double b0, double b1, double b2) {
    double s = __dmul_rn(a0, b0);
    if (d > 1) s = __dadd_rn(s, __dmul_rn(a1, b1));
    if (d > 2) s = __dadd_rn(s, __dmul_rn(a2, b2));
    return s;
}

// kappa of two points, float64: Table 1's kappa_3 = cos(x . y) from the points,
// every other kernel from their squared distance (h2_kappa)
__device__ __forceinline__ double h2_kxy(int kid, double kp0, int d, double a0, double a1, double a2, double b0,
                                         double b1, double b2) {
    if (kid == H2_K_COSDOT) return cos(h2_dot(d, a0, a1, a2, b0, b1, b2));
    return h2_kappa(kid, kp0, h2_dist2(d, a0, a1, a2, b0, b1, b2));
}

// the same in the fast forms of h2_kappa_fast (contracted arithmetic; p as
// h2_kappa_param gives it)
__device__ __forceinline__ double h2_kxy_fast(int kid, double p, double a0, double a1, double a2, double b0,
                                              double b1, double b2) {
    if (kid == H2_K_COSDOT) return cos(a0 * b0 + a1 * b1 + a2 * b2);
    const double dx = a0 - b0, dy = a1 - b1, dz = a2 - b2;
    return h2_kappa_fast(kid, p, dx * dx + dy * dy + dz * dz);
}

// float32 kappa for the mixed-precision path
__device__ __forceinline__ float h2_kappa_f(int kid, float kp0, float r2) {
    switch (kid) {
    case H2_K_COULOMB: return r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    case H2_K_GAUSSIAN: return __expf(-r2 / (kp0 * kp0));
    case H2_K_EXPONENTIAL: return __expf(-sqrtf(r2) / kp0);
    case H2_K_MULTIQUADRIC: return sqrtf(1.0f + r2);
    case H2_K_BUMP: {
        const float t = kp0 * r2;
        return t < 1.0f ? __expf(__fdividef(-1.0f, 1.0f - t)) : 0.0f;
    }
    case H2_K_POWER: return r2 > 0.0f ? __powf(r2, 0.5f * kp0) : 0.0f;
    default: return 0.0f;
    }
}

// ----------------------------------------------------- block reductions
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
