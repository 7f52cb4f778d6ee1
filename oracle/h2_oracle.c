/*
 * h2_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the data-driven H^2 construction of
 * Cai, Huang, Chow and Xi, "Data-Driven Construction of Hierarchical Matrices
 * with Nested Bases" (arXiv 2206.01885).  It exists to check the CUDA library
 * against; nothing in the product path may call it.  It shares no source with
 * the CUDA path.  Built with -O2 -ffp-contract=off so that every floating-point
 * expression below is evaluated exactly as written (no fused multiply-adds).
 * OpenMP, when enabled, only runs independent nodes of one tree level at once.
 *
 * Steps, in the paper's order:
 *   tree       section 2.1 (adaptive partition), Algorithm 2 step 1
 *   lists      section 2.1, eq. (1) admissibility and the interaction list
 *   DataReduct section 3.3, volume-based reduction (the variant of section 6)
 *   HiDR       Algorithm 1 (bottom-up X_i*, top-down Y_i*)
 *   getBasis   section 4.1, eqs. (3)-(5), as a column-pivoted QR ID
 *   construct  Algorithm 2 steps 4-14 (nested bases, coupling, nearfield)
 *   matvec     the O(n) H^2 product of section 2.1
 *   calibrate  section 4.2 (r1 = r2 chosen from epsilon)
 *   error      section 6 relative matvec error (dense / exact sampled rows)
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - root box: a cube of side max_k(hi_k - lo_k) at the componentwise minimum;
 *     coordinates quantised to B = 21 (d = 3) or 31 (d = 1, 2) bits;
 *   - a node splits when it holds more than q points and its level is < B;
 *     children are the non-empty orthants, in Morton (key) order;
 *   - diam and centre in eq. (1) are those of the node's cell (a cube), so the
 *     test is done exactly in integers; tau is the rational tau_num / tau_den;
 *   - interaction lists come from the dual traversal starting at (root, root),
 *     which reproduces the paper's 1D example IL(4) = {6,7}, IL(10) = {8,12,13};
 *   - DataReduct(S, g): S itself when |S| <= g^d, otherwise the nearest point of
 *     S to each of the g^d cell-centred points of a tensor grid over the
 *     bounding box of S (ties to the smaller Morton position), deduplicated;
 *   - getBasis: Businger-Golub column pivoting, LAPACK-style norm downdating,
 *     stop at the first step whose pivot norm is <= eps * |r_11|;
 *   - optionally (il_reduce), Y_i* also takes the reduction of its
 *     interaction-list part on that part's own box (a variant, off by default).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;
typedef uint64_t u64;
typedef unsigned __int128 u128;

enum { K_COULOMB = 1, K_GAUSSIAN = 2, K_EXPONENTIAL = 3, K_MULTIQUADRIC = 4, K_BUMP = 5, K_POWER = 6, K_COSDOT = 7 };

/* ------------------------------------------------------------------------ */
/* Kernel functions (section 2, Table 1).                                    */
/* ------------------------------------------------------------------------ */

/* squared distance ((x0-y0)^2 + (x1-y1)^2) + (x2-y2)^2, left to right */
static double dist2(const double *a, const double *b, int d) {
    double s = 0.0;
    for (int k = 0; k < d; k++) {
        double t = a[k] - b[k];
        s = s + t * t;
    }
    return s;
}

/* kappa as a function of the squared distance.  Coulomb: 1/|x-y| with
 * kappa(x,x) = 0 (Table 1 caption).  Gaussian exp(-|x-y|^2 / h^2), exponential
 * exp(-|x-y| / l), multiquadric sqrt(1 + |x-y|^2).  Bump: Table 1's kappa_4,
 * exp(-1 / (1 - a |x-y|^2)) with a = kp[0] (0.1 there), taken as 0 where
 * a |x-y|^2 >= 1 (the formula's limit there, so the kernel is the smooth
 * compactly supported bump).  Power: |x-y|^p with p = kp[0] (11 in the data
 * reduction comparison of section 5.2). */
static double kfun(int kid, const double *kp, double r2) {
    switch (kid) {
    case K_COULOMB: return r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
    case K_GAUSSIAN: return exp(-(r2 / (kp[0] * kp[0])));
    case K_EXPONENTIAL: return exp(-(sqrt(r2) / kp[0]));
    case K_MULTIQUADRIC: return sqrt(1.0 + r2);
    case K_BUMP: {
        double t = kp[0] * r2;
        return t < 1.0 ? exp(-(1.0 / (1.0 - t))) : 0.0;
    }
    case K_POWER: return r2 > 0.0 ? pow(r2, 0.5 * kp[0]) : 0.0;
    default: return NAN;
    }
}

/* kappa(a, b) for two points: Table 1's kappa_3 = cos(a . b) from the points
 * themselves (it is not a function of |a - b|), every other kernel from
 * |a - b|^2. */
static double kxy(int kid, const double *kp, const double *a, const double *b, int d) {
    if (kid == K_COSDOT) {
        double s = 0.0;
        for (int k = 0; k < d; k++) s = s + a[k] * b[k];
        return cos(s);
    }
    return kfun(kid, kp, dist2(a, b, d));
}

/* ------------------------------------------------------------------------ */
/* Tree (section 2.1; Algorithm 2 step 1).                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    i64 n;
    int d, B, q;
    i64 tau_num, tau_den;
    double lo[3], side;
    u64 *key;      /* Morton keys, sorted                              */
    i64 *perm;     /* Morton position -> original index                */
    double *x;     /* coordinates in Morton order, n x d row-major     */
    int nnodes, nlevels;
    int *lptr;     /* nodes of level l are [lptr[l], lptr[l+1])        */
    int *level, *parent, *fchild, *nchild;
    i64 *begin, *end;
    u64 *prefix;   /* key >> d*(B - level)                             */
    /* interaction lists, CSR over nodes, rows sorted by column node id */
    i64 *near_ptr, *far_ptr;
    int *near_idx, *far_idx;
    i64 nnear, nfar;
} otree;

typedef struct { u64 key; i64 idx; } keyidx;

static int cmp_keyidx(const void *a, const void *b) {
    const keyidx *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int bits_for_dim(int d) { return d == 3 ? 21 : 31; }

/* quantise one coordinate: c = min(floor((x - lo) * s), 2^B - 1) */
static u64 quantise(double x, double lo, double s, int B) {
    double t = (x - lo) * s;
    double top = ldexp(1.0, B);
    if (!(t < top)) return (((u64)1) << B) - 1;
    return (u64)t; /* t >= 0, so truncation is floor */
}

/* interleave: bit b of coordinate k goes to key bit d*b + k */
static u64 interleave(const u64 *c, int d, int B) {
    u64 key = 0;
    for (int b = 0; b < B; b++)
        for (int k = 0; k < d; k++) key |= ((c[k] >> b) & 1ull) << (d * b + k);
    return key;
}

/* de-interleave the level-l prefix into integer cell coordinates */
static void cell_coords(u64 prefix, int d, int l, u64 *c) {
    for (int k = 0; k < d; k++) c[k] = 0;
    for (int b = 0; b < l; b++)
        for (int k = 0; k < d; k++) c[k] |= ((prefix >> (d * b + k)) & 1ull) << b;
}

otree *or_tree_build(const double *pts, i64 n, int d, int q, i64 tau_num, i64 tau_den) {
    if (n <= 0 || d < 1 || d > 3 || q < 1 || tau_num < 0 || tau_den < 1) return NULL;
    otree *t = calloc(1, sizeof(otree));
    t->n = n; t->d = d; t->q = q; t->B = bits_for_dim(d);
    t->tau_num = tau_num; t->tau_den = tau_den;
    int B = t->B;
    double hi[3];
    for (int k = 0; k < d; k++) { t->lo[k] = pts[k]; hi[k] = pts[k]; }
    for (i64 i = 1; i < n; i++)
        for (int k = 0; k < d; k++) {
            double v = pts[i * d + k];
            if (v < t->lo[k]) t->lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    t->side = 0.0;
    for (int k = 0; k < d; k++) {
        double w = hi[k] - t->lo[k];
        if (w > t->side) t->side = w;
    }
    keyidx *ki = malloc(sizeof(keyidx) * n);
    double s = t->side > 0.0 ? ldexp(1.0, B) / t->side : 0.0;
    for (i64 i = 0; i < n; i++) {
        u64 c[3] = {0, 0, 0};
        if (t->side > 0.0)
            for (int k = 0; k < d; k++) c[k] = quantise(pts[i * d + k], t->lo[k], s, B);
        ki[i].key = interleave(c, d, B);
        ki[i].idx = i;
    }
    qsort(ki, n, sizeof(keyidx), cmp_keyidx); /* (key, index): a stable order */
    t->key = malloc(sizeof(u64) * n);
    t->perm = malloc(sizeof(i64) * n);
    t->x = malloc(sizeof(double) * n * d);
    for (i64 p = 0; p < n; p++) {
        t->key[p] = ki[p].key;
        t->perm[p] = ki[p].idx;
        for (int k = 0; k < d; k++) t->x[p * d + k] = pts[ki[p].idx * d + k];
    }
    free(ki);

    /* level-by-level construction; nodes numbered by level, then key order */
    int cap = 64;
    t->level = malloc(sizeof(int) * cap); t->parent = malloc(sizeof(int) * cap);
    t->fchild = malloc(sizeof(int) * cap); t->nchild = malloc(sizeof(int) * cap);
    t->begin = malloc(sizeof(i64) * cap); t->end = malloc(sizeof(i64) * cap);
    t->prefix = malloc(sizeof(u64) * cap);
    t->lptr = malloc(sizeof(int) * (B + 2));
    int nn = 1;
    t->level[0] = 0; t->parent[0] = -1; t->fchild[0] = -1; t->nchild[0] = 0;
    t->begin[0] = 0; t->end[0] = n; t->prefix[0] = 0;
    t->lptr[0] = 0; t->lptr[1] = 1;
    int l = 0;
    const int C = 1 << d;
    for (;;) {
        int lb = t->lptr[l], le = t->lptr[l + 1];
        int before = nn;
        for (int i = lb; i < le; i++) {
            i64 cnt = t->end[i] - t->begin[i];
            if (!(cnt > q && l < B && t->side > 0.0)) continue;
            int shift = d * (B - l - 1);
            i64 p = t->begin[i];
            int first = nn;
            for (int o = 0; o < C; o++) {
                i64 s0 = p;
                while (p < t->end[i] && (int)((t->key[p] >> shift) & (u64)(C - 1)) == o) p++;
                if (p == s0) continue;
                if (nn == cap) {
                    cap *= 2;
                    t->level = realloc(t->level, sizeof(int) * cap);
                    t->parent = realloc(t->parent, sizeof(int) * cap);
                    t->fchild = realloc(t->fchild, sizeof(int) * cap);
                    t->nchild = realloc(t->nchild, sizeof(int) * cap);
                    t->begin = realloc(t->begin, sizeof(i64) * cap);
                    t->end = realloc(t->end, sizeof(i64) * cap);
                    t->prefix = realloc(t->prefix, sizeof(u64) * cap);
                }
                t->level[nn] = l + 1; t->parent[nn] = i; t->fchild[nn] = -1; t->nchild[nn] = 0;
                t->begin[nn] = s0; t->end[nn] = p;
                t->prefix[nn] = t->key[s0] >> shift;
                nn++;
            }
            t->fchild[i] = first;
            t->nchild[i] = nn - first;
        }
        if (nn == before) break;
        l++;
        t->lptr[l + 1] = nn;
    }
    t->nnodes = nn;
    t->nlevels = l + 1;
    return t;
}

/* eq. (1) with cell diameters and centres, exactly in integers:
 * sqrt(d)(e_i + e_j) <= 2 tau |a_i - a_j|  <=>
 * den^2 d (e_i + e_j)^2 <= num^2 |A_i - A_j|^2,  A = 2 * centre = e (2c + 1). */
static int admissible(const otree *t, int i, int j) {
    int d = t->d, B = t->B;
    u64 ci[3], cj[3];
    cell_coords(t->prefix[i], d, t->level[i], ci);
    cell_coords(t->prefix[j], d, t->level[j], cj);
    u64 ei = 1ull << (B - t->level[i]), ej = 1ull << (B - t->level[j]);
    u128 dist = 0;
    for (int k = 0; k < d; k++) {
        u64 ai = ei * (2 * ci[k] + 1), aj = ej * (2 * cj[k] + 1);
        u64 df = ai > aj ? ai - aj : aj - ai;
        dist += (u128)df * df;
    }
    u128 es = (u128)(ei + ej) * (ei + ej);
    u128 lhs = (u128)(t->tau_den * t->tau_den) * (u128)d * es;
    u128 rhs = (u128)(t->tau_num * t->tau_num) * dist;
    return lhs <= rhs;
}

typedef struct { int i, j; } pair_t;
typedef struct { pair_t *a; i64 n, cap; } pairvec;

static void pv_push(pairvec *v, int i, int j) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->a = realloc(v->a, sizeof(pair_t) * v->cap);
    }
    v->a[v->n].i = i; v->a[v->n].j = j; v->n++;
}

static int cmp_pair(const void *a, const void *b) {
    const pair_t *x = a, *y = b;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    return x->j < y->j ? -1 : (x->j > y->j);
}

/* dual traversal: admissible -> far; two leaves -> near; else split every
 * non-leaf side and visit all child pairs */
static void traverse(const otree *t, int i, int j, pairvec *nearv, pairvec *farv) {
    if (admissible(t, i, j)) { pv_push(farv, i, j); return; }
    int li = t->nchild[i] == 0, lj = t->nchild[j] == 0;
    if (li && lj) { pv_push(nearv, i, j); return; }
    int a0 = li ? i : t->fchild[i], a1 = li ? i + 1 : t->fchild[i] + t->nchild[i];
    int b0 = lj ? j : t->fchild[j], b1 = lj ? j + 1 : t->fchild[j] + t->nchild[j];
    for (int a = a0; a < a1; a++)
        for (int b = b0; b < b1; b++) traverse(t, a, b, nearv, farv);
}

static void to_csr(const pairvec *v, int nnodes, i64 **ptr, int **idx) {
    qsort(v->a, v->n, sizeof(pair_t), cmp_pair);
    *ptr = calloc(nnodes + 1, sizeof(i64));
    *idx = malloc(sizeof(int) * (v->n > 0 ? v->n : 1));
    for (i64 e = 0; e < v->n; e++) { (*ptr)[v->a[e].i + 1]++; (*idx)[e] = v->a[e].j; }
    for (int i = 0; i < nnodes; i++) (*ptr)[i + 1] += (*ptr)[i];
}

void or_tree_lists(otree *t) {
    pairvec nv = {0}, fv = {0};
    traverse(t, 0, 0, &nv, &fv);
    to_csr(&nv, t->nnodes, &t->near_ptr, &t->near_idx);
    to_csr(&fv, t->nnodes, &t->far_ptr, &t->far_idx);
    t->nnear = nv.n; t->nfar = fv.n;
    free(nv.a); free(fv.a);
}

/* info[0..9] = n, d, B, nnodes, nlevels, nnear, nfar, side(bits), -, - */
void or_tree_info(const otree *t, i64 *info, double *geom) {
    info[0] = t->n; info[1] = t->d; info[2] = t->B; info[3] = t->nnodes;
    info[4] = t->nlevels; info[5] = t->nnear; info[6] = t->nfar;
    for (int k = 0; k < 3; k++) geom[k] = k < t->d ? t->lo[k] : 0.0;
    geom[3] = t->side;
}

/* copy out: which = 0 perm(i64 n) 1 key(u64 n) 2 level 3 parent 4 fchild
 * 5 nchild (int nnodes) 6 begin 7 end (i64 nnodes) 8 prefix (u64 nnodes)
 * 9 lptr (int nlevels+1) 10 near_ptr 11 far_ptr (i64 nnodes+1)
 * 12 near_idx (int nnear) 13 far_idx (int nfar) 14 x (double n*d) */
void or_tree_get(const otree *t, int which, void *out) {
    i64 n = t->n; int nn = t->nnodes;
    switch (which) {
    case 0: memcpy(out, t->perm, sizeof(i64) * n); break;
    case 1: memcpy(out, t->key, sizeof(u64) * n); break;
    case 2: memcpy(out, t->level, sizeof(int) * nn); break;
    case 3: memcpy(out, t->parent, sizeof(int) * nn); break;
    case 4: memcpy(out, t->fchild, sizeof(int) * nn); break;
    case 5: memcpy(out, t->nchild, sizeof(int) * nn); break;
    case 6: memcpy(out, t->begin, sizeof(i64) * nn); break;
    case 7: memcpy(out, t->end, sizeof(i64) * nn); break;
    case 8: memcpy(out, t->prefix, sizeof(u64) * nn); break;
    case 9: memcpy(out, t->lptr, sizeof(int) * (t->nlevels + 1)); break;
    case 10: memcpy(out, t->near_ptr, sizeof(i64) * (nn + 1)); break;
    case 11: memcpy(out, t->far_ptr, sizeof(i64) * (nn + 1)); break;
    case 12: memcpy(out, t->near_idx, sizeof(int) * t->nnear); break;
    case 13: memcpy(out, t->far_idx, sizeof(int) * t->nfar); break;
    case 14: memcpy(out, t->x, sizeof(double) * n * t->d); break;
    }
}

int or_admissible(const otree *t, int i, int j) { return admissible(t, i, j); }

void or_tree_free(otree *t) {
    if (!t) return;
    free(t->key); free(t->perm); free(t->x); free(t->lptr);
    free(t->level); free(t->parent); free(t->fchild); free(t->nchild);
    free(t->begin); free(t->end); free(t->prefix);
    free(t->near_ptr); free(t->far_ptr); free(t->near_idx); free(t->far_idx);
    free(t);
}

/* ------------------------------------------------------------------------ */
/* DataReduct, volume-based (section 3.3).                                   */
/* ------------------------------------------------------------------------ */

static int cmp_i64(const void *a, const void *b) {
    i64 x = *(const i64 *)a, y = *(const i64 *)b;
    return x < y ? -1 : (x > y);
}

static i64 ipow(i64 g, int d) { i64 r = 1; for (int k = 0; k < d; k++) r *= g; return r; }

/* S: ns labels (Morton positions, distinct); coords of label s at xs[s*d].
 * Writes the reduced set, sorted, to out (capacity >= min(ns, g^d)); returns its size. */
i64 or_datareduct(const double *xs, int d, const i64 *S, i64 ns, int g, i64 *out) {
    i64 r = ipow(g, d);
    if (ns <= r) {
        memcpy(out, S, sizeof(i64) * ns);
        qsort(out, ns, sizeof(i64), cmp_i64);
        return ns;
    }
    double l[3], u[3], h[3];
    for (int k = 0; k < d; k++) { l[k] = xs[S[0] * d + k]; u[k] = l[k]; }
    for (i64 a = 1; a < ns; a++)
        for (int k = 0; k < d; k++) {
            double v = xs[S[a] * d + k];
            if (v < l[k]) l[k] = v;
            if (v > u[k]) u[k] = v;
        }
    for (int k = 0; k < d; k++) h[k] = (u[k] - l[k]) / (double)g;
    i64 m = 0;
    for (i64 gi = 0; gi < r; gi++) {
        double qp[3];
        i64 rem = gi;
        for (int k = 0; k < d; k++) {
            i64 idx = rem % g; rem /= g;
            qp[k] = l[k] + ((double)idx + 0.5) * h[k];
        }
        i64 best = -1; double bd = 0.0;
        for (i64 a = 0; a < ns; a++) {
            double dd = dist2(xs + S[a] * d, qp, d);
            if (best < 0 || dd < bd || (dd == bd && S[a] < best)) { bd = dd; best = S[a]; }
        }
        out[m++] = best;
    }
    qsort(out, m, sizeof(i64), cmp_i64);
    i64 w = 0;
    for (i64 a = 0; a < m; a++)
        if (w == 0 || out[a] != out[w - 1]) out[w++] = out[a];
    return w;
}

/* DataReduct, surface-based (section 3.3): the reference set Q lies on three
 * ellipsoids centred at the centre c of S's bounding box [l, u], with
 * semi-axes gamma (u_k - l_k) for gamma = 0.3, 0.6, 1.2, ne = floor(g^d / 3)
 * points on each; every q takes its nearest point of S (float64 squared
 * distance, ties to the smaller label), and the winners, deduplicated and
 * sorted, form X*.  The paper leaves the points on the ellipsoids open; here
 * they are the unit directions of the Fibonacci lattice in 3D,
 *   z_j = 1 - (2j + 1) / ne, rho_j = sqrt(1 - z_j^2), phi_j = j pi (3 - sqrt 5),
 *   u_j = (rho_j cos phi_j, rho_j sin phi_j, z_j),
 * and equal angles theta_j = 2 pi (j + 1/2) / ne in 2D, u_j = (cos, sin), so
 * q = c + (gamma (u - l)) * u_j per coordinate.  |S| <= g^d returns S. */
static const double SURF_GAMMA[3] = {0.3, 0.6, 1.2};
static const double SURF_PI = 3.14159265358979323846;

static void surf_dir(int d, int ne, int j, double *u) {
    if (d == 3) {
        double z = 1.0 - (2.0 * j + 1.0) / ne;
        double rho = sqrt(1.0 - z * z);
        double phi = j * (SURF_PI * (3.0 - sqrt(5.0)));
        u[0] = rho * cos(phi); u[1] = rho * sin(phi); u[2] = z;
    } else {
        double th = 2.0 * SURF_PI * (j + 0.5) / ne;
        u[0] = cos(th); u[1] = sin(th); u[2] = 0.0;
    }
}

i64 or_datareduct_surface(const double *xs, int d, const i64 *S, i64 ns, int g, i64 *out) {
    i64 r = ipow(g, d);
    if (ns <= r || d < 2) {
        memcpy(out, S, sizeof(i64) * ns);
        qsort(out, ns, sizeof(i64), cmp_i64);
        return ns;
    }
    double l[3], u[3];
    for (int k = 0; k < d; k++) { l[k] = xs[S[0] * d + k]; u[k] = l[k]; }
    for (i64 a = 1; a < ns; a++)
        for (int k = 0; k < d; k++) {
            double v = xs[S[a] * d + k];
            if (v < l[k]) l[k] = v;
            if (v > u[k]) u[k] = v;
        }
    int ne = (int)(r / 3);
    i64 m = 0;
    for (int e = 0; e < 3; e++)
        for (int j = 0; j < ne; j++) {
            double dir[3], qp[3];
            surf_dir(d, ne, j, dir);
            for (int k = 0; k < d; k++) {
                double c = (l[k] + u[k]) * 0.5;
                double a = SURF_GAMMA[e] * (u[k] - l[k]);
                qp[k] = c + a * dir[k];
            }
            i64 best = -1; double bd = 0.0;
            for (i64 b = 0; b < ns; b++) {
                double dd = dist2(xs + S[b] * d, qp, d);
                if (best < 0 || dd < bd || (dd == bd && S[b] < best)) { bd = dd; best = S[b]; }
            }
            out[m++] = best;
        }
    qsort(out, m, sizeof(i64), cmp_i64);
    i64 w = 0;
    for (i64 a = 0; a < m; a++)
        if (w == 0 || out[a] != out[w - 1]) out[w++] = out[a];
    return w;
}

/* DataReduct by farthest point sampling (section 3.3): X* starts with the
 * point of S of smallest label and grows by the point of S farthest from X*
 * (largest float64 squared distance to its nearest member of X*, ties to the
 * smaller label) until it holds g^d points; returned sorted.  The paper leaves
 * the first point open; it is read here as the smallest label.  |S| <= g^d
 * returns S. */
i64 or_datareduct_fps(const double *xs, int d, const i64 *S, i64 ns, int g, i64 *out) {
    i64 r = ipow(g, d);
    if (ns <= r) {
        memcpy(out, S, sizeof(i64) * ns);
        qsort(out, ns, sizeof(i64), cmp_i64);
        return ns;
    }
    double *md = malloc(sizeof(double) * ns);      /* squared distance to X* */
    unsigned char *in = calloc((size_t)ns, 1);      /* member of X* */
    i64 f = 0;
    for (i64 a = 0; a < ns; a++) {
        md[a] = INFINITY;
        if (S[a] < S[f]) f = a;
    }
    for (i64 m = 0; m < r; m++) {
        out[m] = S[f];
        in[f] = 1;
        if (m + 1 == r) break;
        i64 b = -1;
        for (i64 a = 0; a < ns; a++) {
            if (in[a]) continue;
            double dd = dist2(xs + S[a] * d, xs + S[f] * d, d);
            if (dd < md[a]) md[a] = dd;
            if (b < 0 || md[a] > md[b] || (md[a] == md[b] && S[a] < S[b])) b = a;
        }
        f = b;
    }
    free(md);
    free(in);
    qsort(out, r, sizeof(i64), cmp_i64);
    return r;
}

/* the DataReduct of HiDR: method 0 volume-based, 1 surface-based, 2 farthest
 * point sampling */
static i64 datareduct_m(int method, const double *xs, int d, const i64 *S, i64 ns, int g, i64 *out) {
    if (method == 2) return or_datareduct_fps(xs, d, S, ns, g, out);
    return method == 1 ? or_datareduct_surface(xs, d, S, ns, g, out) : or_datareduct(xs, d, S, ns, g, out);
}

/* ------------------------------------------------------------------------ */
/* HiDR, Algorithm 1.                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nnodes, g1, g2;
    i64 **xs, **ys;     /* X_i*, Y_i* per node (sorted Morton positions) */
    i64 *nx, *ny;       /* sizes; -1 = not computed                     */
} ohidr;

/* a and b sorted and free of repeats: writes their union, sorted, to out and
 * returns its size */
static i64 union_sorted(const i64 *a, i64 na, const i64 *b, i64 nb, i64 *out) {
    i64 u = 0, v = 0, w = 0;
    while (u < na || v < nb) {
        i64 x;
        if (v == nb || (u < na && a[u] < b[v])) x = a[u++];
        else if (u == na || b[v] < a[u]) x = b[v++];
        else { x = a[u++]; v++; }
        out[w++] = x;
    }
    return w;
}

/* need_y: per-node flag (NULL = all) of nodes whose Y* is wanted; Y* is then
 * also computed for every ancestor of a flagged node.  X* is computed for all
 * non-root nodes.
 *
 * il_reduce = 0 is Algorithm 1 as printed.  il_reduce = 1 adds to each Y_i* the
 * reduction of the interaction-list part alone, DataReduct(union of X_j* over
 * j in IL(i), r2), whose reference grid spans only the box of those nearby
 * nodes: Y_i* = DataReduct(T_i, r2) u DataReduct(IL part, r2), at most 2 r2
 * points.  The grid over all of T_i spans nearly the whole domain at every
 * depth (Y_p* covers the parent's farfield), so on deep trees it leaves the
 * closest far nodes with a few samples or none; the second grid scales with
 * the node. */
ohidr *or_hidr(const otree *t, int g1, int g2, const unsigned char *need_y, int method, int il_reduce) {
    int nn = t->nnodes, d = t->d;
    ohidr *h = calloc(1, sizeof(ohidr));
    h->nnodes = nn; h->g1 = g1; h->g2 = g2;
    h->xs = calloc(nn, sizeof(i64 *)); h->ys = calloc(nn, sizeof(i64 *));
    h->nx = malloc(sizeof(i64) * nn); h->ny = malloc(sizeof(i64) * nn);
    unsigned char *want = malloc(nn);
    for (int i = 0; i < nn; i++) { h->nx[i] = -1; h->ny[i] = -1; want[i] = need_y ? need_y[i] : 1; }
    for (int i = nn - 1; i > 0; i--)
        if (want[i]) want[t->parent[i]] = 1;
    /* bottom-up: S_i = X_i for a leaf, union of children's X_c* otherwise */
    for (int l = t->nlevels - 1; l >= 1; l--) {
        int lb = t->lptr[l], le = t->lptr[l + 1];
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = lb; i < le; i++) {
            i64 ns = 0;
            i64 *S;
            if (t->nchild[i] == 0) {
                ns = t->end[i] - t->begin[i];
                S = malloc(sizeof(i64) * ns);
                for (i64 a = 0; a < ns; a++) S[a] = t->begin[i] + a;
            } else {
                for (int c = t->fchild[i]; c < t->fchild[i] + t->nchild[i]; c++) ns += h->nx[c];
                S = malloc(sizeof(i64) * (ns > 0 ? ns : 1));
                i64 w = 0;
                for (int c = t->fchild[i]; c < t->fchild[i] + t->nchild[i]; c++) {
                    memcpy(S + w, h->xs[c], sizeof(i64) * h->nx[c]);
                    w += h->nx[c];
                }
            }
            i64 cap = ns < ipow(g1, d) ? ns : ipow(g1, d);
            h->xs[i] = malloc(sizeof(i64) * (cap > 0 ? cap : 1));
            h->nx[i] = datareduct_m(method, t->x, d, S, ns, g1, h->xs[i]);
            free(S);
        }
    }
    /* top-down: T_i = Y_p* union X_j* over j in IL(i) */
    h->ny[0] = 0; h->ys[0] = malloc(sizeof(i64));
    for (int l = 1; l < t->nlevels; l++) {
        int lb = t->lptr[l], le = t->lptr[l + 1];
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = lb; i < le; i++) {
            if (!want[i]) continue;
            int p = t->parent[i];
            i64 nt = h->ny[p];
            for (i64 e = t->far_ptr[i]; e < t->far_ptr[i + 1]; e++) nt += h->nx[t->far_idx[e]];
            if (nt == 0) { h->ny[i] = 0; h->ys[i] = malloc(sizeof(i64)); continue; }
            i64 *T = malloc(sizeof(i64) * nt);
            i64 w = 0;
            memcpy(T, h->ys[p], sizeof(i64) * h->ny[p]); w += h->ny[p];
            for (i64 e = t->far_ptr[i]; e < t->far_ptr[i + 1]; e++) {
                int j = t->far_idx[e];
                memcpy(T + w, h->xs[j], sizeof(i64) * h->nx[j]);
                w += h->nx[j];
            }
            i64 gd = ipow(g2, d), nil = nt - h->ny[p];
            i64 cap = nt < gd ? nt : gd;
            i64 capl = il_reduce && nil > 0 ? (nil < gd ? nil : gd) : 0;
            h->ys[i] = malloc(sizeof(i64) * (cap + capl));
            h->ny[i] = datareduct_m(method, t->x, d, T, nt, g2, h->ys[i]);
            if (capl > 0) {
                i64 *A = malloc(sizeof(i64) * cap), *B = malloc(sizeof(i64) * capl);
                i64 na = h->ny[i];
                memcpy(A, h->ys[i], sizeof(i64) * na);
                i64 nb = datareduct_m(method, t->x, d, T + h->ny[p], nil, g2, B);
                h->ny[i] = union_sorted(A, na, B, nb, h->ys[i]);
                free(A); free(B);
            }
            free(T);
        }
    }
    free(want);
    return h;
}

/* which = 0: X_i*, 1: Y_i*.  Returns the size (-1 if not computed); copies if out. */
i64 or_hidr_get(const ohidr *h, int node, int which, i64 *out) {
    i64 n = which ? h->ny[node] : h->nx[node];
    if (n > 0 && out) memcpy(out, which ? h->ys[node] : h->xs[node], sizeof(i64) * n);
    return n;
}

void or_hidr_free(ohidr *h) {
    if (!h) return;
    for (int i = 0; i < h->nnodes; i++) { free(h->xs[i]); free(h->ys[i]); }
    free(h->xs); free(h->ys); free(h->nx); free(h->ny); free(h);
}

/* ------------------------------------------------------------------------ */
/* getBasis: column-pivoted QR interpolative decomposition (eqs. (3)-(5)).   */
/* ------------------------------------------------------------------------ */

/* A: m x c column-major (overwritten).  Returns k.  piv[0..c): the column
 * order after pivoting.  T (k x (c-k), column-major, ld k) = R11^{-1} R12,
 * so that A[:, piv[k:]] ~= A[:, piv[:k]] T.  tie: first (smallest) index. */
int or_id(double *A, int m, int c, double eps, int *piv, double *T) {
    double *nrm = malloc(sizeof(double) * (c > 0 ? c : 1));
    double *nrm0 = malloc(sizeof(double) * (c > 0 ? c : 1));
    double *v = malloc(sizeof(double) * (m > 0 ? m : 1));
    const double tol3z = sqrt(ldexp(1.0, -53));
    for (int l = 0; l < c; l++) {
        double s = 0.0;
        for (int r = 0; r < m; r++) s = s + A[(i64)l * m + r] * A[(i64)l * m + r];
        nrm[l] = sqrt(s); nrm0[l] = nrm[l]; piv[l] = l;
    }
    int kmax = m < c ? m : c, k = 0;
    double r11 = 0.0;
    for (int j = 0; j < kmax; j++) {
        int p = j;
        for (int l = j + 1; l < c; l++) if (nrm[l] > nrm[p]) p = l;
        if (j == 0) r11 = nrm[p];
        if (!(nrm[p] > eps * r11) || nrm[p] == 0.0) break;
        if (p != j) {
            for (int r = 0; r < m; r++) {
                double tmp = A[(i64)j * m + r]; A[(i64)j * m + r] = A[(i64)p * m + r]; A[(i64)p * m + r] = tmp;
            }
            double tn = nrm[j]; nrm[j] = nrm[p]; nrm[p] = tn;
            tn = nrm0[j]; nrm0[j] = nrm0[p]; nrm0[p] = tn;
            int ti = piv[j]; piv[j] = piv[p]; piv[p] = ti;
        }
        /* Householder reflector H = I - tau v v^T with v[j] = 1 mapping
         * A[j:m, j] to (beta, 0, ..., 0) */
        double *aj = A + (i64)j * m;
        double alpha = aj[j], sigma = 0.0;
        for (int r = j + 1; r < m; r++) sigma = sigma + aj[r] * aj[r];
        if (alpha == 0.0 && sigma == 0.0) break; /* exactly zero pivot column */
        double tau = 0.0, beta = alpha;
        if (sigma != 0.0) {
            double xn = sqrt(alpha * alpha + sigma);
            beta = alpha >= 0.0 ? -xn : xn;
            tau = (beta - alpha) / beta;
            double sc = 1.0 / (alpha - beta);
            v[j] = 1.0;
            for (int r = j + 1; r < m; r++) v[r] = aj[r] * sc;
        }
        aj[j] = beta;
        for (int r = j + 1; r < m; r++) aj[r] = 0.0;
        for (int l = j + 1; l < c; l++) {
            double *al = A + (i64)l * m;
            if (tau != 0.0) {
                double w = al[j];
                for (int r = j + 1; r < m; r++) w = w + v[r] * al[r];
                w = w * tau;
                al[j] = al[j] - w;
                for (int r = j + 1; r < m; r++) al[r] = al[r] - w * v[r];
            }
            /* norm downdate; recompute once it has lost half its digits */
            if (nrm[l] != 0.0) {
                double tt = fabs(al[j]) / nrm[l];
                tt = 1.0 - tt * tt;
                if (tt < 0.0) tt = 0.0;
                double t2 = nrm[l] / nrm0[l];
                t2 = tt * t2 * t2;
                if (t2 <= tol3z) {
                    double s = 0.0;
                    for (int r = j + 1; r < m; r++) s = s + al[r] * al[r];
                    nrm[l] = sqrt(s); nrm0[l] = nrm[l];
                } else {
                    nrm[l] = nrm[l] * sqrt(tt);
                }
            }
        }
        k = j + 1;
    }
    /* T = R11^{-1} R12 by back substitution, one column of R12 at a time */
    for (int l = k; l < c; l++) {
        double *tc = T + (i64)(l - k) * k;
        for (int i = k - 1; i >= 0; i--) {
            double s = A[(i64)l * m + i];
            for (int p = i + 1; p < k; p++) s = s - A[(i64)p * m + i] * tc[p];
            tc[i] = s / A[(i64)i * m + i];
        }
    }
    free(nrm); free(nrm0); free(v);
    return k;
}

/* Bounded interpolation coefficients (eq. (3): ||G||_max bounded by a
 * prescribed constant f).  After or_id, while some |T[p, l]| > f (the largest
 * one, ties to the first in column-major order), skeleton column piv[p] and
 * non-skeleton column piv[k + l] trade places: with g = T[p, l],
 *   A[:, piv[k + l]] = sum_q A[:, piv[q]] T[q, l]
 * solved for A[:, piv[p]] and substituted into every other column gives
 *   T'[p, m] = T[p, m] / g,  T'[q, m] = T[q, m] - T[q, l] T'[p, m]  (m != l),
 *   T'[q, l] = -(T[q, l] / g),  T'[p, l] = 1 / g               (q != p),
 * a Gauss-Jordan pivot on T.  Each exchange multiplies the volume of the
 * skeleton columns by |g| > f, so the loop ends; it stops after maxex
 * exchanges in any case.  Returns the number of exchanges. */
int or_id_bound(int k, int nr, int *piv, double *T, double f, int maxex) {
    int nex = 0;
    while (nex < maxex) {
        int bp = -1, bl = -1;
        double bv = f;
        for (int l = 0; l < nr; l++)
            for (int p = 0; p < k; p++) {
                double v = fabs(T[(i64)l * k + p]);
                if (v > bv) { bv = v; bp = p; bl = l; }
            }
        if (bp < 0) break;
        double g = T[(i64)bl * k + bp];
        for (int m = 0; m < nr; m++)
            if (m != bl) T[(i64)m * k + bp] = T[(i64)m * k + bp] / g;
        for (int m = 0; m < nr; m++) {
            if (m == bl) continue;
            double tp = T[(i64)m * k + bp];
            for (int q = 0; q < k; q++)
                if (q != bp) T[(i64)m * k + q] = T[(i64)m * k + q] - T[(i64)bl * k + q] * tp;
        }
        for (int q = 0; q < k; q++)
            if (q != bp) T[(i64)bl * k + q] = -(T[(i64)bl * k + q] / g);
        T[(i64)bl * k + bp] = 1.0 / g;
        int ti = piv[bp]; piv[bp] = piv[k + bl]; piv[k + bl] = ti;
        nex++;
    }
    return nex;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: nested bases, bottom level to top level.                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    const otree *t;
    int kid;
    double kp[4];
    double eps;
    double gbound;   /* f of or_id_bound, 0 = no exchanges                   */
    i64 nex;         /* exchanges made                                       */
    int nnodes;
    int *k;          /* rank k_i (-1 = not computed)                        */
    int *c;          /* |Xbar_i|                                             */
    i64 **skel;      /* Xhat_i, sorted Morton positions                      */
    double **U;      /* U_i (leaf) or the stacked transfer matrix (parent): c_i x k_i, column-major */
} oh2;

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return x < y ? -1 : (x > y);
}

/* A = K(Y, Xbar): rows over Y, columns over Xbar (both Morton positions) */
static void kernel_block(const otree *t, int kid, const double *kp, const i64 *Y, int m,
                         const i64 *Xb, int c, double *A) {
    int d = t->d;
    for (int l = 0; l < c; l++)
        for (int r = 0; r < m; r++)
            A[(i64)l * m + r] = kxy(kid, kp, t->x + Y[r] * d, t->x + Xb[l] * d, d);
}

/* need: per-node flag (NULL = all); the basis is also built for every
 * descendant of a flagged node.  Y_i* must be available for those nodes. */
oh2 *or_construct(const otree *t, const ohidr *h, int kid, const double *kp, double eps,
                  const unsigned char *need, double gbound) {
    int nn = t->nnodes;
    oh2 *H = calloc(1, sizeof(oh2));
    H->t = t; H->kid = kid; H->eps = eps; H->nnodes = nn; H->gbound = gbound;
    for (int a = 0; a < 4; a++) H->kp[a] = kp ? kp[a] : 0.0;
    H->k = malloc(sizeof(int) * nn); H->c = malloc(sizeof(int) * nn);
    H->skel = calloc(nn, sizeof(i64 *)); H->U = calloc(nn, sizeof(double *));
    unsigned char *want = malloc(nn);
    for (int i = 0; i < nn; i++) { H->k[i] = -1; H->c[i] = 0; want[i] = need ? need[i] : 1; }
    for (int i = 1; i < nn; i++)
        if (want[t->parent[i]]) want[i] = 1;
    want[0] = 0; /* the root needs no basis */
    for (int l = t->nlevels - 1; l >= 1; l--) {
        int lb = t->lptr[l], le = t->lptr[l + 1];
#pragma omp parallel for schedule(dynamic, 1)
        for (int i = lb; i < le; i++) {
            if (!want[i]) continue;
            int c = 0;
            i64 *Xb;
            if (t->nchild[i] == 0) {
                c = (int)(t->end[i] - t->begin[i]);
                Xb = malloc(sizeof(i64) * c);
                for (int a = 0; a < c; a++) Xb[a] = t->begin[i] + a;
            } else {
                for (int ch = t->fchild[i]; ch < t->fchild[i] + t->nchild[i]; ch++) c += H->k[ch];
                Xb = malloc(sizeof(i64) * (c > 0 ? c : 1));
                int w = 0;
                for (int ch = t->fchild[i]; ch < t->fchild[i] + t->nchild[i]; ch++) {
                    memcpy(Xb + w, H->skel[ch], sizeof(i64) * H->k[ch]);
                    w += H->k[ch];
                }
            }
            H->c[i] = c;
            int m = (int)h->ny[i];
            if (m <= 0 || c == 0) {
                H->k[i] = 0; H->skel[i] = malloc(sizeof(i64)); H->U[i] = malloc(sizeof(double));
                free(Xb);
                continue;
            }
            double *A = malloc(sizeof(double) * (i64)m * c);
            kernel_block(t, kid, H->kp, h->ys[i], m, Xb, c, A);
            int *piv = malloc(sizeof(int) * c);
            int kmax = m < c ? m : c;
            double *T = malloc(sizeof(double) * ((i64)kmax * c + 1));
            int k = or_id(A, m, c, eps, piv, T);
            if (gbound > 0.0 && k > 0) {
                int nx = or_id_bound(k, c - k, piv, T, gbound, 8 * k);
#pragma omp atomic
                H->nex += nx;
            }
            /* sorted skeleton; sigma[p] = column of U for the p-th pivot */
            int *sk = malloc(sizeof(int) * (k > 0 ? k : 1));
            int *sigma = malloc(sizeof(int) * (k > 0 ? k : 1));
            memcpy(sk, piv, sizeof(int) * k);
            qsort(sk, k, sizeof(int), cmp_int);
            for (int p = 0; p < k; p++) {
                int lo = 0, hi = k - 1;
                while (lo < hi) { int mid = (lo + hi) / 2; if (sk[mid] < piv[p]) lo = mid + 1; else hi = mid; }
                sigma[p] = lo;
            }
            H->k[i] = k;
            H->skel[i] = malloc(sizeof(i64) * (k > 0 ? k : 1));
            for (int p = 0; p < k; p++) H->skel[i][p] = Xb[sk[p]];
            double *U = calloc((size_t)c * (k > 0 ? k : 1), sizeof(double));
            for (int p = 0; p < k; p++) U[(i64)sigma[p] * c + piv[p]] = 1.0;
            for (int l2 = k; l2 < c; l2++)
                for (int p = 0; p < k; p++) U[(i64)sigma[p] * c + piv[l2]] = T[(i64)(l2 - k) * k + p];
            H->U[i] = U;
            free(A); free(piv); free(T); free(sk); free(sigma); free(Xb);
        }
    }
    free(want);
    return H;
}

/* rank/skeleton/basis getters. which: 0 -> k, 1 -> c; skeleton copy; U copy */
int or_h2_rank(const oh2 *H, int node, int which) { return which ? H->c[node] : H->k[node]; }
i64 or_h2_exchanges(const oh2 *H) { return H->nex; }
void or_h2_skel(const oh2 *H, int node, i64 *out) { if (H->k[node] > 0) memcpy(out, H->skel[node], sizeof(i64) * H->k[node]); }
void or_h2_U(const oh2 *H, int node, double *out) {
    if (H->k[node] > 0) memcpy(out, H->U[node], sizeof(double) * (i64)H->c[node] * H->k[node]);
}

void or_h2_free(oh2 *H) {
    if (!H) return;
    for (int i = 0; i < H->nnodes; i++) { free(H->skel[i]); free(H->U[i]); }
    free(H->skel); free(H->U); free(H->k); free(H->c); free(H);
}

/* ------------------------------------------------------------------------ */
/* H^2 matvec: upward (U^T), coupling B_ij = K(Xhat_i, Xhat_j), downward (U), */
/* nearfield K(X_i, X_j).  x, y in the original point order.                 */
/* ------------------------------------------------------------------------ */
void or_matvec(const oh2 *H, const double *x, double *y) {
    const otree *t = H->t;
    int nn = t->nnodes, d = t->d;
    i64 n = t->n;
    double *xm = malloc(sizeof(double) * n), *ym = calloc(n, sizeof(double));
    for (i64 p = 0; p < n; p++) xm[p] = x[t->perm[p]];
    double **xh = calloc(nn, sizeof(double *)), **zh = calloc(nn, sizeof(double *));
    for (int i = 0; i < nn; i++) {
        int k = H->k[i] > 0 ? H->k[i] : 0;
        xh[i] = calloc(k + 1, sizeof(double));
        zh[i] = calloc(k + 1, sizeof(double));
    }
    /* upward: xh_i = U_i^T (x restricted to X_i, or the children's xh stacked) */
    for (int l = t->nlevels - 1; l >= 1; l--)
        for (int i = t->lptr[l]; i < t->lptr[l + 1]; i++) {
            int k = H->k[i], c = H->c[i];
            if (k <= 0) continue;
            double *in = malloc(sizeof(double) * c);
            if (t->nchild[i] == 0) {
                for (int a = 0; a < c; a++) in[a] = xm[t->begin[i] + a];
            } else {
                int w = 0;
                for (int ch = t->fchild[i]; ch < t->fchild[i] + t->nchild[i]; ch++)
                    for (int a = 0; a < H->k[ch]; a++) in[w++] = xh[ch][a];
            }
            for (int p = 0; p < k; p++) {
                double s = 0.0;
                for (int a = 0; a < c; a++) s = s + H->U[i][(i64)p * c + a] * in[a];
                xh[i][p] = s;
            }
            free(in);
        }
    /* coupling: zh_i = sum over far j of K(Xhat_i, Xhat_j) xh_j */
    for (int i = 0; i < nn; i++)
        for (i64 e = t->far_ptr[i]; e < t->far_ptr[i + 1]; e++) {
            int j = t->far_idx[e];
            for (int a = 0; a < H->k[i]; a++) {
                double s = 0.0;
                for (int b = 0; b < H->k[j]; b++)
                    s = s + kxy(H->kid, H->kp, t->x + H->skel[i][a] * d, t->x + H->skel[j][b] * d, d) * xh[j][b];
                zh[i][a] = zh[i][a] + s;
            }
        }
    /* downward: children's zh += U_i zh_i; leaves: y_i += U_i zh_i */
    for (int l = 1; l < t->nlevels; l++)
        for (int i = t->lptr[l]; i < t->lptr[l + 1]; i++) {
            int k = H->k[i], c = H->c[i];
            if (k <= 0) continue;
            double *o = malloc(sizeof(double) * c);
            for (int a = 0; a < c; a++) {
                double s = 0.0;
                for (int p = 0; p < k; p++) s = s + H->U[i][(i64)p * c + a] * zh[i][p];
                o[a] = s;
            }
            if (t->nchild[i] == 0) {
                for (int a = 0; a < c; a++) ym[t->begin[i] + a] += o[a];
            } else {
                int w = 0;
                for (int ch = t->fchild[i]; ch < t->fchild[i] + t->nchild[i]; ch++)
                    for (int a = 0; a < H->k[ch]; a++) zh[ch][a] += o[w++];
            }
            free(o);
        }
    /* nearfield: y_i += K(X_i, X_j) x_j over near leaf pairs */
    for (int i = 0; i < nn; i++)
        for (i64 e = t->near_ptr[i]; e < t->near_ptr[i + 1]; e++) {
            int j = t->near_idx[e];
            for (i64 a = t->begin[i]; a < t->end[i]; a++) {
                double s = 0.0;
                for (i64 b = t->begin[j]; b < t->end[j]; b++)
                    s = s + kxy(H->kid, H->kp, t->x + a * d, t->x + b * d, d) * xm[b];
                ym[a] += s;
            }
        }
    for (i64 p = 0; p < n; p++) y[t->perm[p]] = ym[p];
    for (int i = 0; i < nn; i++) { free(xh[i]); free(zh[i]); }
    free(xh); free(zh); free(xm); free(ym);
}

/* ------------------------------------------------------------------------ */
/* Dense reference and exact sampled rows (section 6 error metric).          */
/* ------------------------------------------------------------------------ */

/* pairwise sum of v[0..n) */
static double pairwise(const double *v, i64 n) {
    if (n <= 32) { double s = 0.0; for (i64 a = 0; a < n; a++) s = s + v[a]; return s; }
    i64 h = n / 2;
    return pairwise(v, h) + pairwise(v + h, n - h);
}

/* out[r] = sum_j kappa(x_rows[r], x_j) z_j, points in original order */
void or_exact_rows(const double *pts, i64 n, int d, int kid, const double *kp, const double *z,
                   const i64 *rows, i64 nrows, double *out) {
    double kpl[4] = {0, 0, 0, 0};
    if (kp) for (int a = 0; a < 4; a++) kpl[a] = kp[a];
#pragma omp parallel
    {
        double *term = malloc(sizeof(double) * n);
#pragma omp for schedule(dynamic, 1)
        for (i64 r = 0; r < nrows; r++) {
            const double *xr = pts + rows[r] * d;
            for (i64 j = 0; j < n; j++) term[j] = kxy(kid, kpl, xr, pts + j * d, d) * z[j];
            out[r] = pairwise(term, n);
        }
        free(term);
    }
}

/* y = K z, the O(n^2) product */
void or_dense_matvec(const double *pts, i64 n, int d, int kid, const double *kp, const double *z, double *y) {
    i64 *rows = malloc(sizeof(i64) * n);
    for (i64 r = 0; r < n; r++) rows[r] = r;
    or_exact_rows(pts, n, d, kid, kp, z, rows, n, y);
    free(rows);
}

/* ------------------------------------------------------------------------ */
/* r1 = r2 from epsilon (section 4.2).                                       */
/* ------------------------------------------------------------------------ */

/* relative Frobenius error of K(Z1,Z2) ~= U K(Zhat1, Z2) for grid size g */
double or_calib_error(int d, int kid, const double *kp, double id_tol, const double *Z1, int n1,
                      const double *Z2, int n2, int g, int *k_out, int *m_out) {
    double kpl[4] = {0, 0, 0, 0};
    if (kp) for (int a = 0; a < 4; a++) kpl[a] = kp[a];
    i64 *S = malloc(sizeof(i64) * n2), *R = malloc(sizeof(i64) * n2);
    for (int a = 0; a < n2; a++) S[a] = a;
    int m = (int)or_datareduct(Z2, d, S, n2, g, R);
    double *A = malloc(sizeof(double) * (i64)m * n1);
    for (int l = 0; l < n1; l++)
        for (int r = 0; r < m; r++) A[(i64)l * m + r] = kxy(kid, kpl, Z2 + R[r] * d, Z1 + (i64)l * d, d);
    int *piv = malloc(sizeof(int) * n1);
    int kmax = m < n1 ? m : n1;
    double *T = malloc(sizeof(double) * ((i64)kmax * n1 + 1));
    int k = or_id(A, m, n1, id_tol, piv, T);
    /* K(Z1, Z2) ~= U K(Zhat1, Z2): skeleton rows are exact; row piv[l], l >= k,
     * is approximated by sum_p T[p, l-k] K(Z1[piv[p]], Z2) (kappa symmetric) */
    double *Ks = malloc(sizeof(double) * ((i64)k * n2 + 1));
    for (int p = 0; p < k; p++)
        for (int b = 0; b < n2; b++) Ks[(i64)p * n2 + b] = kxy(kid, kpl, Z1 + (i64)piv[p] * d, Z2 + (i64)b * d, d);
    double num = 0.0, den = 0.0;
    for (int l = 0; l < n1; l++) {
        int a = piv[l];
        for (int b = 0; b < n2; b++) {
            double kab = kxy(kid, kpl, Z1 + (i64)a * d, Z2 + (i64)b * d, d);
            den = den + kab * kab;
            if (l < k) continue;
            double s = 0.0;
            for (int p = 0; p < k; p++) s = s + T[(i64)(l - k) * k + p] * Ks[(i64)p * n2 + b];
            double e = kab - s;
            num = num + e * e;
        }
    }
    free(Ks);
    if (k_out) *k_out = k;
    if (m_out) *m_out = m;
    free(S); free(R); free(A); free(piv); free(T);
    return den > 0.0 ? sqrt(num / den) : 0.0;
}

/* smallest g in [1, gmax] whose error is < 1e-2 eps, with the ID truncated at
 * 1e-2 eps as well; returns gmax + 1 if none is. */
int or_calibrate(int d, int kid, const double *kp, double eps, const double *Z1, int n1,
                 const double *Z2, int n2, int gmax) {
    for (int g = 1; g <= gmax; g++) {
        double e = or_calib_error(d, kid, kp, 1e-2 * eps, Z1, n1, Z2, n2, g, NULL, NULL);
        if (e < 1e-2 * eps) return g;
    }
    return gmax + 1;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
