/*
 * h2.h -- C ABI of the GB300 (sm_103a) library for the data-driven H^2
 * construction of Cai, Huang, Chow and Xi, "Data-Driven Construction of
 * Hierarchical Matrices with Nested Bases" (arXiv 2206.01885).
 *
 * Pipeline (each call consumes the previous call's handle):
 *   h2_tree_build   adaptive Morton cluster tree + near/far interaction lists
 *                   (section 2.1, eq. (1); Algorithm 2 step 1)
 *   h2_calibrate    grid size g with r1 = r2 = g^d from epsilon (section 4.2;
 *                   Algorithm 2 step 2)
 *   h2_hidr_reduce  hierarchical data reduction X_i*, Y_i* (section 3,
 *                   Algorithm 1; Algorithm 2 step 3)
 *   h2_construct    level-by-level kernel blocks K(Y_i*, Xbar_i) and pivoted-QR
 *                   interpolative decompositions giving skeletons Xhat_i and
 *                   nested bases U_i (section 4.1 eqs. (3)-(5); Algorithm 2
 *                   steps 4-14)
 *   h2_matvec       y = K~ x, the O(n) H^2 product (section 2.1)
 *   h2_exact_rows   exact (K z)_s on sampled rows, for the section 6 error
 *
 * Conventions shared by every call:
 *   - Points are float64, row-major n x dim (point i at pts[i*dim + k]), in
 *     the caller's original order.  dim is 2 or 3.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     queued on it; calls that must learn sizes (tree levels, list lengths,
 *     per-level ranks) synchronise that stream internally.  A handle's later
 *     calls may use another stream only after the first stream is synchronised.
 *   - Pointers flagged `*_on_device` are device pointers of the current CUDA
 *     device; otherwise host pointers (pageable or pinned).  The caller owns
 *     every buffer it passes; the library copies what it keeps.
 *   - Handles are opaque, owned by the library and released only by h2_free.
 *     A tree must outlive every hidr and matrix built on it (h2_free of a tree
 *     with live dependents returns H2_ERR_STATE and frees nothing).
 *   - No call aborts the process.  Errors return a status and set a
 *     thread-local message read by h2_last_error().  Device-side faults
 *     surface as H2_ERR_CUDA at the next synchronising call.
 *   - There is no CPU fallback: every step runs in this library's kernels.
 */
#ifndef H2_GB300_H
#define H2_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    H2_OK = 0,
    H2_ERR_INVALID_ARG = 1,   /* bad pointer, size, kernel id, parameter      */
    H2_ERR_OOM = 2,           /* device allocation failed                      */
    H2_ERR_CUDA = 3,          /* a CUDA runtime call or kernel failed          */
    H2_ERR_TIMEOUT = 4,       /* a bounded device wait gave up                 */
    H2_ERR_NUMERIC = 5,       /* non-finite value met                          */
    H2_ERR_UNIMPLEMENTED = 6, /* option not built                              */
    H2_ERR_STATE = 7          /* handle in the wrong state / has dependents    */
} h2_status;

/* kernel functions kappa(x, y) (section 2, Table 1): functions of r = |x - y|,
   except H2_K_COSDOT */
typedef enum {
    H2_K_COULOMB = 1,      /* 1/r, and kappa(x, x) = 0 (Table 1 caption)       */
    H2_K_GAUSSIAN = 2,     /* exp(-r^2 / h^2), kparams[0] = h                  */
    H2_K_EXPONENTIAL = 3,  /* exp(-r / l), kparams[0] = l                      */
    H2_K_MULTIQUADRIC = 4, /* sqrt(1 + r^2)                                    */
    H2_K_BUMP = 5,         /* Table 1's kappa_4: exp(-1 / (1 - a r^2)),
                              kparams[0] = a (0.1 in Table 1); 0 where
                              a r^2 >= 1 (the formula's limit there)          */
    H2_K_POWER = 6,        /* r^p, kparams[0] = p > 0 (11 in section 5.2)      */
    H2_K_COSDOT = 7        /* Table 1's kappa_3: cos(x . y), of the points
                              themselves (not of r); no kparams                */
} h2_kernel_id;

/* arithmetic of h2_construct / h2_matvec */
typedef enum {
    H2_PREC_FP64 = 0,  /* everything in float64                                */
    H2_PREC_MIXED = 1  /* float32 kernel blocks and QR updates; float64 column
                          norms, pivots and R11^{-1} R12 solve                  */
} h2_precision;

typedef struct h2_tree_s *h2_tree;
typedef struct h2_hidr_s *h2_hidr;
typedef struct h2_matrix_s *h2_matrix;
typedef struct h2_graph_s *h2_graph;

/* Algorithm 2 inputs "separation ratio tau" and "leaf size q".  tau is the
 * rational tau_num / tau_den so that eq. (1) is decided exactly in integers
 * (default 7/10, the top of the paper's range [0, 0.7]). */
typedef struct {
    int leaf_size; /* q >= 1: a node holding more than q points is split      */
    int tau_num;   /* >= 0                                                     */
    int tau_den;   /* >= 1                                                     */
} h2_tree_params;

/* ---------------------------------------------------------------- tree --- */
/* Section 2.1 ("recursively partitioning X spatially until no more than m
 * points are contained in each subset"), eq. (1) admissibility, and the
 * interaction list; Algorithm 2 step 1.
 * pts: n x dim float64 (device if pts_on_device, else host), n >= 1,
 * n < 2^31.  The root box is the cube of side max_k(max x_k - min x_k) at the
 * componentwise minimum; coordinates are quantised to 21 (dim 3) or 31
 * (dim 2) bits and Morton-interleaved (coordinate 0 in the lowest bit); points
 * are stably sorted by key.  A node splits while it holds more than q points;
 * children are its non-empty orthants in key order; nodes are numbered level by
 * level, then by key.  Near/far lists come from a dual traversal from
 * (root, root): an admissible pair is far, a pair of leaves is near, otherwise
 * every non-leaf side is split.  Errors: H2_ERR_INVALID_ARG (null pointers,
 * n < 1, dim not 2/3, q < 1, bad tau), H2_ERR_NUMERIC (a coordinate is NaN or
 * infinite), H2_ERR_OOM, H2_ERR_CUDA. */
h2_status h2_tree_build(const double *pts, int64_t n, int dim, int pts_on_device,
                        const h2_tree_params *params, void *stream, h2_tree *out);

/* Trees of nprob independent point sets (the batched configuration; no
 * counterpart in the paper beyond its independent problems): tree p is exactly
 * what h2_tree_build(pts[p], ns[p], dim, pts_on_device, &params[p]) returns,
 * but the builds run concurrently, each on one of up to eight internal
 * streams driven by host threads.  The work starts after the work already
 * queued on `stream`; on return `stream` is ordered after every build and
 * every tree belongs to it.  pts: nprob pointers to n x dim float64 arrays
 * (all device or all host, as pts_on_device says); ns, params: nprob entries.
 * Errors: as h2_tree_build; on any error no tree is returned (out[] all NULL)
 * and the message names the first failing problem. */
h2_status h2_tree_build_batched(int nprob, const double *const *pts, const int64_t *ns, int dim, int pts_on_device,
                                const h2_tree_params *params, void *stream, h2_tree *out);

/* what for h2_tree_get (element type, length):
 *   H2_TREE_PERM      int64 [n]          Morton position -> original index
 *   H2_TREE_KEYS      uint64 [n]         sorted Morton keys
 *   H2_TREE_LEVEL, H2_TREE_PARENT, H2_TREE_FCHILD, H2_TREE_NCHILD  int32 [nnodes]
 *                                        (parent of root = -1, fchild of leaf = -1)
 *   H2_TREE_BEGIN, H2_TREE_END  int64 [nnodes]  point range in Morton order
 *   H2_TREE_PREFIX    uint64 [nnodes]    key >> dim*(B - level)
 *   H2_TREE_LPTR      int32 [nlevels+1]  nodes of level l: [lptr[l], lptr[l+1])
 *   H2_TREE_NEAR_PTR, H2_TREE_FAR_PTR   int64 [nnodes+1]  CSR row pointers
 *   H2_TREE_NEAR_IDX, H2_TREE_FAR_IDX   int32 [nnear] / [nfar], rows sorted
 *   H2_TREE_INFO      int64 [8]: n, dim, B, nnodes, nlevels, nnear, nfar, q
 *   H2_TREE_GEOM      float64 [4]: lo[0..2] (unused entries 0), side
 * host_buf may be NULL to query *len (in elements).  Synchronises the tree's
 * stream.  Errors: H2_ERR_INVALID_ARG (unknown what, cap too small). */
enum {
    H2_TREE_PERM = 0, H2_TREE_KEYS = 1, H2_TREE_LEVEL = 2, H2_TREE_PARENT = 3,
    H2_TREE_FCHILD = 4, H2_TREE_NCHILD = 5, H2_TREE_BEGIN = 6, H2_TREE_END = 7,
    H2_TREE_PREFIX = 8, H2_TREE_LPTR = 9, H2_TREE_NEAR_PTR = 10, H2_TREE_FAR_PTR = 11,
    H2_TREE_NEAR_IDX = 12, H2_TREE_FAR_IDX = 13, H2_TREE_INFO = 14, H2_TREE_GEOM = 15
};
h2_status h2_tree_get(h2_tree t, int what, void *host_buf, int64_t cap, int64_t *len);

/* ----------------------------------------------------------- calibrate --- */
/* Section 4.2: r1 = r2 = g^dim is raised from g = 1 until the interpolative
 * decomposition of the artificial block K(Z2*, Z1), Z2* = DataReduct(Z2, g),
 * reproduces K(Z1, Z2) with relative Frobenius error < 1e-2 * eps; the ID in
 * this test is itself truncated at 1e-2 * eps.  z1 (n1 x dim) and z2
 * (n2 x dim) are host float64 point sets that the caller draws well separated
 * in the sense of eq. (1).  Runs on the GPU with the library's own DataReduct,
 * kernel-block and ID kernels.  *g_out = the smallest g <= gmax that passes, or
 * gmax + 1 if none does; *err_out (may be NULL) = that g's error.
 * Synchronises `stream`.  Errors: H2_ERR_INVALID_ARG, H2_ERR_OOM, H2_ERR_CUDA. */
h2_status h2_calibrate(int dim, int kernel, const double *kparams, double eps,
                       const double *z1, int n1, const double *z2, int n2, int gmax,
                       void *stream, int *g_out, double *err_out);

/* ---------------------------------------------------------------- HiDR --- */
/* Section 3.1-3.3 and Algorithm 1.  Bottom-up from the deepest level:
 * S_i = X_i for a leaf, the union of the children's X_c* otherwise, and
 * X_i* = DataReduct(S_i, g1^dim).  Top-down from level 1:
 * T_i = Y_p* union X_j* over j in the interaction (far) list of i, and
 * Y_i* = DataReduct(T_i, g2^dim) (empty when T_i is).  DataReduct(S, g^d) is the
 * volume-based variant used in section 6: S itself when |S| <= g^d; otherwise
 * the nearest point of S (float64 squared distance, ties to the smaller
 * Morton position) to each cell-centred point of a g^d tensor grid on the
 * bounding box of S, deduplicated.  Sets are stored as sorted Morton
 * positions.  Kernel-independent: one hidr serves every kernel.
 * g1, g2 >= 1 (g^dim <= 16384).  Errors: H2_ERR_INVALID_ARG, H2_ERR_OOM,
 * H2_ERR_CUDA. */
h2_status h2_hidr_reduce(h2_tree t, int g1, int g2, void *stream, h2_hidr *out);

/* DataReduct variants of section 3.3 for h2_hidr_reduce_ex */
typedef enum {
    H2_DR_VOLUME = 0, /* h2_hidr_reduce's: nearest points to a g^d tensor grid */
    H2_DR_SURFACE = 1, /* nearest points to floor(g^d / 3) reference points on
                         each of three ellipsoids centred at the centre c of
                         the set's bounding box [l, u], semi-axes gamma (u - l)
                         for gamma = 0.3, 0.6, 1.2: q = c + (gamma (u - l)) *
                         dir_j, dir_j the Fibonacci-lattice unit directions
                         in 3D (z_j = 1 - (2j + 1) / ne, rho_j = sqrt(1 -
                         z_j^2), phi_j = j pi (3 - sqrt 5)) and the equal
                         angles 2 pi (j + 1/2) / ne in 2D; same nearest-point
                         rule, deduplicated and sorted                       */
    H2_DR_FPS = 2     /* farthest point sampling: start at the smallest label,
                         add the point farthest from the chosen ones (float64
                         squared distance to the nearest of them, ties to the
                         smaller label) until g^d are chosen; sequential by
                         nature (g^d rounds over the set per node), so meant
                         for small problems                                  */
} h2_datareduct;

/* Flag ORed into h2_hidr_reduce_ex's method: each Y_i* also takes the
 * reduction of its interaction-list part alone, on that part's own bounding
 * box: Y_i* = DataReduct(T_i, g2^d) u DataReduct(union of X_j* over j in IL(i),
 * g2^d), deduplicated and sorted, at most 2 g2^d points (a variant of
 * Algorithm 1's top-down step).  The grid over all of T_i spans nearly the
 * whole domain at every depth, because Y_p* covers the parent's farfield; the
 * second grid scales with the node, so deep nodes' closest far nodes keep
 * their samples.  Requires g2^dim <= 4096. */
#define H2_HIDR_IL_REDUCE 0x100

/* Flag ORed into h2_hidr_reduce_ex's method: the top-down sets T_i are copied
 * into one array each and binned entry by entry, instead of the default volume
 * search that reads the X_j* in place (with chunk and member boxes).  Both
 * give the same X_i*, Y_i*; this form is slower and serves comparisons. */
#define H2_HIDR_COPY_SETS 0x200

/* h2_hidr_reduce with the DataReduct variant `method` (h2_datareduct),
 * optionally ORed with H2_HIDR_IL_REDUCE and H2_HIDR_COPY_SETS.
 * Errors: as h2_hidr_reduce; H2_ERR_INVALID_ARG for an unknown method or flag,
 * or for H2_HIDR_IL_REDUCE with g2^dim > 4096. */
h2_status h2_hidr_reduce_ex(h2_tree t, int g1, int g2, int method, void *stream, h2_hidr *out);

/* HiDR of nprob trees at once (the batched configuration): hidr p is exactly
 * h2_hidr_reduce_ex(trees[p], g1[p], g2[p], methods[p]) (methods may be NULL:
 * H2_DR_VOLUME for all), the reductions running concurrently on up to eight
 * internal streams driven by host threads.  Stream and error conventions as
 * h2_tree_build_batched.  A tree may appear more than once. */
h2_status h2_hidr_reduce_batched(int nprob, const h2_tree *trees, const int *g1, const int *g2, const int *methods,
                                 void *stream, h2_hidr *out);

/* which: 0 = X_i*, 1 = Y_i*.  Fills counts (int32 [nnodes], may be NULL) and,
 * if data is not NULL, the concatenation over nodes in node order of the
 * sorted Morton positions (int32, cap elements).  *total = sum of counts.
 * Synchronises. */
h2_status h2_hidr_get(h2_hidr h, int which, int32_t *counts, int32_t *data, int64_t cap,
                      int64_t *total);

/* ----------------------------------------------------------- construct --- */
/* Section 4.1 eqs. (3)-(5) and Algorithm 2 steps 4-14.  For levels from the
 * deepest to 1 and every node i with Y_i* non-empty: Xbar_i = X_i for a leaf,
 * the concatenation of the children's skeletons (child order, each sorted) for a
 * parent; A_i = K(Y_i*, Xbar_i) (|Y_i*| x |Xbar_i|); column-pivoted Householder
 * QR of A_i (pivot = largest downdated column norm, ties to the first column;
 * LAPACK-style downdating with recomputation); stop at the first step j whose
 * pivot norm <= id_tol * |r_11|, so k_i = j; G^T = R11^{-1} R12; skeleton
 * Xhat_i = the k_i pivoted candidates, stored sorted by Morton position;
 * U_i = P [I; G] (|Xbar_i| x k_i, columns in skeleton order).  For a leaf U_i
 * is the leaf basis, for a parent it stacks the transfer matrices R_c.
 * Coupling blocks B_ij = K(Xhat_i, Xhat_j) and nearfield blocks K(X_i, X_j)
 * are kernel submatrices and are evaluated inside h2_matvec.
 * kparams: 4 float64 (host; may be NULL for Coulomb / multiquadric).
 * precision: H2_PREC_FP64 or H2_PREC_MIXED.  id_tol >= 0.
 * Errors: H2_ERR_INVALID_ARG, H2_ERR_OOM, H2_ERR_CUDA, H2_ERR_UNIMPLEMENTED. */
h2_status h2_construct(h2_tree t, h2_hidr h, int kernel, const double *kparams, double id_tol,
                       int precision, void *stream, h2_matrix *out);

/* Memory mode of the coupling blocks B_ij = K(Xhat_i, Xhat_j) (far pairs)
 * and nearfield blocks K(X_i, X_j) (near leaf pairs) that Algorithm 2 forms
 * after the bases.  ON_THE_FLY evaluates them inside every h2_matvec;
 * STORE evaluates each once at construction and keeps it on the device
 * (kappa is symmetric: one block per unordered pair, row-major, in the
 * matrix's precision -- float64, or float32 in the mixed form), and every
 * later single-right-hand-side product reads the stored blocks; AUTO stores
 * them when they fit (as STORE's budget below) and the form is float64, the
 * one whose on-the-fly evaluation costs more than reading a stored entry. */
enum { H2_MEM_ON_THE_FLY = 0, H2_MEM_STORE = 1, H2_MEM_AUTO = 2 };

/* Options of h2_construct_ex; zero-initialised options are h2_construct's. */
typedef struct {
    double g_bound;      /* f > 1: bound ||G||_max by f as below; 0: no exchanges */
    int mem_mode;        /* H2_MEM_ON_THE_FLY (0), H2_MEM_STORE or H2_MEM_AUTO       */
    double mem_fraction; /* share of the device's free memory (cudaMemGetInfo at
                            construction) the stored blocks may take, in (0, 1];
                            0 means 0.5.  STORE above it fails with H2_ERR_OOM;
                            AUTO above it stays on the fly                      */
    int fp64_products;   /* float64 form, 3D Coulomb, one right-hand side: 0 (default)
                            evaluates the on-the-fly coupling and nearfield
                            products in float-float arithmetic on the float32
                            units (values hi + lo of two float32, relative error
                            of an evaluation below 2^-43, offsets from the cell
                            centres carried to ~2^-48 of a cell width); 1 keeps
                            them in float64 arithmetic.  The construction, the
                            stored blocks and every other product are float64
                            either way                                          */
    int tensor_core_products; /* mixed form, several right-hand sides: 1 runs the
                            nearfield 16 columns at a time on the tensor cores
                            (kernel values and weights split as tf32 hi + lo,
                            three tcgen05 products per 32-source chunk, float32
                            accumulation folded per chunk, error per term ~2^-21
                            relative); 0 (default) keeps every column on the CUDA
                            cores, which measure faster (the kernel values, not
                            the products, bound this step).  A tensor-core wait
                            that gives up (never expected) makes a synchronising
                            h2_matvec return H2_ERR_TIMEOUT                    */
    int fp64_qr;         /* float64 form: 0 (default) runs the column-pivoted QR's
                            reflectors and trailing updates in float-float
                            arithmetic on the float32 units (the block held as
                            float pairs of ~48 bits; norms, downdates, pivots,
                            the stop test and the reflector's scalars stay
                            float64; R is returned to float64 for the solve);
                            with it, for 3D Coulomb, the kernel blocks are
                            evaluated in float-float arithmetic as well and
                            handed to the QR as float pairs.  1 keeps the
                            blocks and the QR in float64 arithmetic throughout
                            (blocks bit-identical to a plain float64
                            evaluation).  The solve is float64 either way     */
} h2_construct_opts;

/* h2_construct with options (opts may be NULL: exactly h2_construct).
 * Eq. (3) asks for an ID whose ||G||_max is bounded by a prescribed constant
 * (the property strong RRQR provides).  With g_bound = f > 1, after each
 * node's column-pivoted QR and solve, while some |G[p, l]| > f (the largest;
 * ties to the first in column-major order of G^T, p + l k), skeleton candidate
 * p and non-skeleton candidate l trade places by a Gauss-Jordan pivot on G:
 * with g = G[p, l], G'[p, m] = G[p, m] / g and G'[q, m] = G[q, m] -
 * G[q, l] G'[p, m] (m != l), G'[q, l] = -G[q, l] / g (q != p), G'[p, l] = 1 / g.
 * Each exchange grows the skeleton columns' volume by a factor |g| > f, so the
 * loop ends; it is cut at 8 k exchanges per node in any case.  The count is
 * the matrix statistic "exchanges".  The parent's candidates are the
 * children's final skeletons, so the bound holds at every level.
 * mem_mode (Algorithm 2's coupling and nearfield blocks, stored or not):
 * with the blocks stored, h2_matvec with nrhs = 1 reads them (several
 * right-hand sides still evaluate on the fly); the product equals the
 * on-the-fly one to rounding (the stored entries are the values the
 * on-the-fly kernels compute).  The matrix statistics report "mem_mode",
 * "stored_bytes" and the fill time "ms_blocks".
 * Errors: as h2_construct; H2_ERR_INVALID_ARG if g_bound is neither 0 nor a
 * finite number > 1, for an unknown mem_mode or a mem_fraction outside
 * [0, 1]; H2_ERR_OOM when STORE's blocks exceed the budget. */
h2_status h2_construct_ex(h2_tree t, h2_hidr h, int kernel, const double *kparams, double id_tol,
                          int precision, const h2_construct_opts *opts, void *stream, h2_matrix *out);

/* Construction of nprob independent problems (configuration 4 of the
 * benchmark plan): matrix p is exactly what h2_construct(trees[p], hidrs[p],
 * kernels[p], kparams + 4p, id_tols[p], precisions[p]) returns, but the
 * problems run concurrently, each level-synchronous on one of up to eight
 * internal streams driven by host threads, so small problems fill the GPU
 * together.  The work starts after the work already queued on `stream`; on
 * return `stream` is ordered after every construction and every matrix
 * belongs to it (its buffers are released on it).  kparams: 4 float64 per
 * problem, or NULL when no problem needs parameters.  A tree or hidr may
 * appear in several problems (e.g. one HiDR reused across kernels).
 * Errors: as h2_construct; on any error no matrix is returned (out[] all
 * NULL) and the message names the first failing problem. */
h2_status h2_construct_batched(int nprob, const h2_tree *trees, const h2_hidr *hidrs, const int *kernels,
                               const double *kparams, const double *id_tols, const int *precisions,
                               void *stream, h2_matrix *out);

/* what for h2_matrix_get:
 *   H2_MAT_RANK   int32 [nnodes]  k_i (0 where Y_i* is empty; 0 for the root)
 *   H2_MAT_NCAND  int32 [nnodes]  |Xbar_i|
 *   H2_MAT_SKEL   int32 [sum k_i] skeletons in node order, each sorted
 *   H2_MAT_U      float64 [sum |Xbar_i| k_i] U_i in node order, each column-major
 *   H2_MAT_INFO   int64 [4]: sum k_i, sum |Xbar_i| k_i, max k_i, levels
 * Synchronises. */
enum { H2_MAT_RANK = 0, H2_MAT_NCAND = 1, H2_MAT_SKEL = 2, H2_MAT_U = 3, H2_MAT_INFO = 4 };
h2_status h2_matrix_get(h2_matrix A, int what, void *host_buf, int64_t cap, int64_t *len);

/* -------------------------------------------------------------- matvec --- */
/* element type of h2_matvec's vectors */
enum { H2_DTYPE_F64 = 0, H2_DTYPE_F32 = 1 };

/* Y = K~ X for nrhs right-hand sides with the H^2 representation (section
 * 2.1): upward pass xh_i = U_i^T x_i (leaves) and xh_p = U_p^T [xh_c ...]
 * (parents); coupling zh_i = sum_{j far from i} K(Xhat_i, Xhat_j) xh_j;
 * downward pass [zh_c ...] += U_p zh_p and y_i = U_i zh_i; nearfield
 * y_i += K(X_i, X_j) x_j over near leaf pairs.  Every kernel evaluation serves
 * all right-hand sides.
 *   x, y   column-major n x nrhs in the original point order: entry (i, j) at
 *          x[i + j * ld]; elements of `dtype` (H2_DTYPE_F64 or H2_DTYPE_F32);
 *          device pointers if on_device, else host (then copied in and out
 *          on `stream` and the call synchronises; entries of y between
 *          columns are left untouched).  x and y must not overlap.
 *   nrhs   >= 1; ld >= n.
 * The arithmetic follows the matrix's precision (float64, or float32 kernel
 * evaluations with float64 or compensated float32 accumulation); dtype only
 * sets the element type of x and y.
 * Errors: H2_ERR_INVALID_ARG, H2_ERR_OOM, H2_ERR_CUDA, H2_ERR_UNIMPLEMENTED. */
h2_status h2_matvec(h2_matrix A, const void *x, void *y, int nrhs, int dtype, int64_t ld, int on_device,
                    void *stream);

/* Repeated products through a CUDA graph (no counterpart in the paper: it
 * serves callers that apply one matrix many times, e.g. iterative solvers).
 * h2_matvec_graph_create runs h2_matvec(A, x, y, nrhs, dtype, ld, on_device
 * = 1, stream) once, waits for it, then records the same product on device
 * buffers x and y (same meaning and checks as h2_matvec) into a CUDA graph
 * with its own scratch.  h2_matvec_graph_launch replays it on `stream`: fill
 * x, launch, read y once the stream reaches that point.  Each replay computes
 * y = K~ x for x's contents at that time, like a fresh h2_matvec call (the
 * float64 atomics make two products agree to rounding, not bit for bit).
 * While a graph lives, h2_free of its matrix fails with H2_ERR_STATE; free
 * the graph (h2_free) first.  Errors: as h2_matvec; H2_ERR_CUDA if the
 * capture or instantiation fails. */
h2_status h2_matvec_graph_create(h2_matrix A, void *x, void *y, int nrhs, int dtype, int64_t ld, void *stream,
                                 h2_graph *out);
h2_status h2_matvec_graph_launch(h2_graph g, void *stream);

/* ---------------------------------------------------------- exact rows --- */
/* The reference of the section 6 error ||K z - K~ z|| / ||K z||: for each
 * row s in rows (original indices), out[s'] = sum_j kappa(x_s, x_j) z_j over
 * all n points, by direct summation (kappa(x, x) = 0 for Coulomb): in float64,
 * and for 3D Coulomb in float-float arithmetic (each term within about 2^-43
 * of exact, float-pair sums, a float64 result), which frees the float64 units
 * for the path it runs beside.  z: n float64,
 * rows: nrows int64, out: nrows float64; all device if on_device, else host
 * (then the call synchronises).  Errors: H2_ERR_INVALID_ARG, H2_ERR_CUDA. */
h2_status h2_exact_rows(h2_tree t, int kernel, const double *kparams, const double *z,
                        const int64_t *rows, int64_t nrows, double *out, int on_device,
                        void *stream);

/* Allocation-free variant of h2_exact_rows, for callers that must not
 * allocate device memory during the call: code running while a CUDA graph is
 * being captured on another stream of the same device, applications whose
 * memory is fully reserved up front by another allocator, or real-time loops
 * that forbid allocator calls (cudaMalloc can synchronise the device and fail
 * under memory pressure).  The paper has no counterpart; it computes exactly
 * what h2_exact_rows computes.  Differences from h2_exact_rows:
 *   - z, rows and out must be device (or managed) memory of the current
 *     device (no host staging); a host pointer is refused with
 *     H2_ERR_INVALID_ARG before anything is launched;
 *   - the tree may hold at most 1,048,576 points: the permuted right-hand side
 *     is kept in a fixed 8 MiB array inside the library image, which every GPU
 *     that loads the library holds until the process exits; larger trees are
 *     rejected with H2_ERR_INVALID_ARG;
 *   - no cudaMalloc, cudaFree or other allocating call is made; the first call
 *     on a device looks up the array's device address (cudaGetSymbolAddress),
 *     so make that first call before any stream capture begins;
 *   - every call shares the one array (it is fully overwritten on each call),
 *     so calls that may overlap on the GPU -- on different streams without
 *     ordering between them -- race and must not be issued.
 * Errors: H2_ERR_INVALID_ARG, H2_ERR_CUDA. */
h2_status h2_exact_rows_noalloc(h2_tree t, int kernel, const double *kparams, const double *z,
                                const int64_t *rows, int64_t nrows, double *out, void *stream);

/* The section 6 error on sampled rows: *err_out = ||exact - approx[rows]||_2
 * / ||exact||_2, with exact[r] = (K z)_{rows[r]} from h2_exact_rows and approx
 * the full H^2 product (n entries, original order).  Device pointers if
 * on_device (err_out then a device scalar), else host (the call then
 * synchronises).  Errors: H2_ERR_INVALID_ARG, H2_ERR_CUDA. */
h2_status h2_sampled_error(const double *exact, const double *approx, const int64_t *rows, int64_t nrows,
                           int64_t n, double *err_out, int on_device, void *stream);

/* ----------------------------------------------------------- autotune --- */
/* Leaf-size autotuner (leaf sizes of batched problems "chosen by the
 * autotuner"; the paper fixes q by hand): for each of the ncand leaf sizes
 * cands[c] (>= 1), builds the tree (tau 7/10), the HiDR (g1 = g2 = g), the
 * construction (kernel, kparams, id_tol, precision) and one float64 matvec on
 * pts, reps times (>= 1), and keeps the least device time (CUDA events on
 * stream) of tree + HiDR + construction + matvec in times[c] (ms, host, may
 * be NULL).  *best = the fastest candidate's leaf size (ties to the first).
 * pts: n x dim float64 row-major, on the device if pts_on_device else on the
 * host; pass a subsample to keep the search cheap (the costs per point vary
 * little with n above ~1e5).  Synchronises.
 * Errors: those of the calls it makes, and H2_ERR_INVALID_ARG. */
h2_status h2_autotune_leaf(const double *pts, int64_t n, int dim, int pts_on_device, const int *cands,
                           int ncand, int g, int kernel, const double *kparams, double id_tol, int precision,
                           int reps, void *stream, int *best, double *times);

/* ------------------------------------------------------- fault testing --- */
/* Host-side allocation-failure injection, for testing the error paths (the
 * paper has no counterpart).  Resets the library's count of device
 * allocations to 0 and arms the k-th allocation from now on (k >= 1) to fail
 * as if the device were out of memory: the call making it returns H2_ERR_OOM,
 * hands out no handle (*out = NULL), releases what it had allocated, and
 * leaves every existing handle and the CUDA context usable.  k = 0 disarms.
 * *allocs_since_last (may be NULL) receives the number of device allocations
 * made since the previous h2_debug_fail_alloc call.  The count is process-wide:
 * concurrent calls on other threads draw from it too.
 * Errors: H2_ERR_INVALID_ARG (k < 0). */
h2_status h2_debug_fail_alloc(int64_t k, int64_t *allocs_since_last);

/* ------------------------------------------------------------- common --- */
/* Release any handle returned above (NULL is a no-op).  Device memory is
 * returned on the handle's stream, which must still exist. */
h2_status h2_free(void *handle);

/* Thread-local text of the last error on this thread ("" if none). */
const char *h2_last_error(void);

/* JSON object with counters and per-phase device times (ms) of a tree, hidr
 * or matrix handle, written to json (cap bytes, NUL-terminated).  A hidr
 * reports its DataReduct "method" ("volume", "surface" or "fps"), the sizes
 * of the reduced sets ("x_total", "y_total"), of the sets reduced ("t_total":
 * the top-down sets T_i; "t_il_total": their interaction-list parts, reduced a
 * second time with H2_HIDR_IL_REDUCE) and the bottom-up and top-down device
 * times ("ms_up", "ms_down").  A matrix reports,
 * among others, its total and largest rank, QR flops and g_max, the largest
 * |G| entry of the interpolation matrices U_i = P [I; G] (the quantity strong
 * RRQR, which the paper names, bounds), and "g_bound" and "exchanges" of
 * h2_construct_ex (0 for h2_construct).  With handle == NULL: the per-kernel
 * totals {"name": {"ms", "launches"}} collected while profiling is enabled. */
h2_status h2_get_stats(const void *handle, char *json, int64_t cap);

/* Per-kernel timing: when enabled, the main kernels are bracketed by CUDA
 * events on the stream they are launched on; `reset` zeroes the totals.
 * Off by default. */
h2_status h2_profile(int enable, int reset);

/* Measured arithmetic peaks of the current device, the denominators of the
 * roofline fractions of ALU-bound kernels (the paper has no counterpart): a
 * kernel of 8 independent fused multiply-add chains per thread, 8 CTAs of
 * 256 threads per SM, timed with CUDA events after a warm-up launch; a
 * multiply-add counts as 2 flops.  Either output may be NULL (not both).
 * Synchronises `stream`.  Errors: H2_ERR_INVALID_ARG, H2_ERR_OOM, H2_ERR_CUDA. */
h2_status h2_fma_peak(double *fp64_tflops, double *fp32_tflops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* H2_GB300_H */
