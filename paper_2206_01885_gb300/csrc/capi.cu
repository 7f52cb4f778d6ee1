// capi.cu -- the extern "C" boundary declared in include/h2.h.  Validates
// arguments, owns handle lifetimes and turns internal exceptions into
// h2_status values plus a thread-local message.  Every compute step runs in
// the library's CUDA kernels.
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include <mutex>

#include "h2_internal.cuh"

namespace {
thread_local std::string g_last_error;

void set_error(const std::string &m) { g_last_error = m; }

template <class F>
h2_status guard(F &&f) {
    try {
        g_last_error.clear();
        f();
        return H2_OK;
    } catch (const h2::Error &e) {
        set_error(e.msg);
        return e.st;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return H2_ERR_OOM;
    } catch (...) {
        set_error("unknown error");
        return H2_ERR_CUDA;
    }
}

bool valid_kernel(int kid) { return kid >= H2_K_COULOMB && kid <= H2_K_COSDOT; }

void kparams_check(int kid, const double *kp, double out[4]) {
    for (int a = 0; a < 4; a++) out[a] = kp ? kp[a] : 0.0;
    if (kid == H2_K_GAUSSIAN || kid == H2_K_EXPONENTIAL) {
        H2_REQUIRE(kp != nullptr, "this kernel needs kparams[0]");
        H2_REQUIRE(std::isfinite(out[0]) && out[0] > 0.0, "kparams[0] must be a positive length");
    }
    if (kid == H2_K_BUMP || kid == H2_K_POWER) {
        H2_REQUIRE(kp != nullptr, "this kernel needs kparams[0]");
        H2_REQUIRE(std::isfinite(out[0]) && out[0] > 0.0, "kparams[0] must be positive and finite");
    }
}

void pool_keep_memory() {
    static std::once_flag done;
    std::call_once(done, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
        }
    });
}

// A pointer the kernels will dereference must be device (or managed) memory of
// the current device.  cudaPointerGetAttributes allocates nothing; an
// unregistered or pinned host pointer is refused here instead of faulting a
// kernel later.
void require_device_ptr(const void *p, const char *name) {
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h2::fail(H2_ERR_INVALID_ARG, std::string(name) + " is not a device pointer");
    }
    int dev = 0;
    H2_CUDA(cudaGetDevice(&dev));
    const bool on_gpu = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    if (!on_gpu || a.device != dev)
        h2::fail(H2_ERR_INVALID_ARG, std::string(name) + " must be device memory of the current device");
}

template <class T>
void copy_out(const std::vector<T> &v, void *buf, int64_t cap, int64_t *len) {
    if (len) *len = (int64_t)v.size();
    if (!buf) return;
    H2_REQUIRE(cap >= (int64_t)v.size(), "output buffer too small");
    if (!v.empty()) memcpy(buf, v.data(), v.size() * sizeof(T));
}

template <class Tsrc, class Tdst>
std::vector<Tdst> widen(const std::vector<Tsrc> &v) {
    return std::vector<Tdst>(v.begin(), v.end());
}
}  // namespace

namespace h2 {
h2_tree_s *as_tree(void *h) {
    auto *t = static_cast<h2_tree_s *>(h);
    if (!t || t->tag != TAG_TREE) fail(H2_ERR_INVALID_ARG, "not a tree handle");
    return t;
}
h2_hidr_s *as_hidr(void *h) {
    auto *t = static_cast<h2_hidr_s *>(h);
    if (!t || t->tag != TAG_HIDR) fail(H2_ERR_INVALID_ARG, "not a hidr handle");
    return t;
}
h2_matrix_s *as_matrix(void *h) {
    auto *t = static_cast<h2_matrix_s *>(h);
    if (!t || t->tag != TAG_MATRIX) fail(H2_ERR_INVALID_ARG, "not a matrix handle");
    return t;
}
}  // namespace h2

using namespace h2;

namespace {
// release every buffer of a tree / hidr on s from now on (s ordered after the
// work that built it), and make s the handle's stream
void tree_rebind(h2_tree_s *t, cudaStream_t s) {
    t->stream = s;
    for (int k = 0; k < 3; k++) {
        t->xs[k].rebind(s); t->cen[k].rebind(s); t->xr[k].rebind(s); t->cenf[k].rebind(s);
        t->cellA[k].rebind(s);
    }
    t->key.rebind(s); t->perm.rebind(s); t->iperm.rebind(s);
    t->level.rebind(s); t->parent.rebind(s); t->fchild.rebind(s); t->nchild.rebind(s);
    t->begin.rebind(s); t->end.rebind(s); t->prefix.rebind(s);
    t->near_ptr.rebind(s); t->far_ptr.rebind(s); t->near_idx.rebind(s); t->far_idx.rebind(s);
    t->xq.rebind(s); t->near_tiles.rebind(s); t->near_first.rebind(s); t->far_first.rebind(s);
    t->leaf_start.rebind(s); t->leaf_count.rebind(s); t->xcell.rebind(s);
    t->near_tiles_tc.rebind(s); t->tc_status.rebind(s);
}
void hidr_rebind(h2_hidr_s *h, cudaStream_t s) {
    h->stream = s;
    h->xcnt.rebind(s); h->ycnt.rebind(s); h->xptr.rebind(s); h->yptr.rebind(s);
    h->xbox.rebind(s); h->ybox.rebind(s);
    for (auto &b : h->xbufs) b.rebind(s);
    for (auto &b : h->ybufs) b.rebind(s);
}

// Runs work(p, stream) for p = 0..nprob-1 on up to eight internal streams
// driven by host threads, after the work queued on s; on return s is ordered
// after all of it.  Per-problem errors are collected (st, msg), not thrown.
template <class F>
void run_concurrently(int nprob, cudaStream_t s, std::vector<h2_status> &st, std::vector<std::string> &msg,
                      F &&work) {
    st.assign(nprob, H2_OK);
    msg.assign(nprob, std::string());
    int dev = 0;
    H2_CUDA(cudaGetDevice(&dev));
    const int nw = std::min(nprob, 8);
    std::vector<cudaStream_t> ws(nw, nullptr);
    std::vector<cudaEvent_t> done(nw, nullptr);
    cudaEvent_t ready = nullptr;
    auto cleanup = [&] {
        for (int w = 0; w < nw; w++) {
            if (done[w]) cudaEventDestroy(done[w]);
            if (ws[w]) cudaStreamDestroy(ws[w]);
        }
        if (ready) cudaEventDestroy(ready);
    };
    try {
        H2_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        H2_CUDA(cudaEventRecord(ready, s));
        for (int w = 0; w < nw; w++) {
            H2_CUDA(cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking));
            H2_CUDA(cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming));
            H2_CUDA(cudaStreamWaitEvent(ws[w], ready, 0));
        }
        std::atomic<int> next{0};
        auto worker = [&](int w) {
            if (cudaSetDevice(dev) != cudaSuccess) return;
            for (int p = next++; p < nprob; p = next++) {
                try {
                    work(p, ws[w]);
                } catch (const Error &e) {
                    st[p] = e.st;
                    msg[p] = e.msg;
                } catch (const std::bad_alloc &) {
                    st[p] = H2_ERR_OOM;
                    msg[p] = "host allocation failed";
                } catch (...) {
                    st[p] = H2_ERR_CUDA;
                    msg[p] = "unknown error";
                }
            }
        };
        std::vector<std::thread> th;
        try {
            for (int w = 0; w < nw; w++) th.emplace_back(worker, w);
        } catch (...) {
            next = nprob;
            for (auto &x : th) x.join();
            throw;
        }
        for (auto &x : th) x.join();
        for (int w = 0; w < nw; w++) {
            H2_CUDA(cudaEventRecord(done[w], ws[w]));
            H2_CUDA(cudaStreamWaitEvent(s, done[w], 0));
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}
}  // namespace

namespace {
// one tree: arguments checked, built on stream s; throws on failure (nothing leaks)
h2_tree_s *tree_build_one(const double *pts, int64_t n, int dim, int pts_on_device, const h2_tree_params *params,
                          cudaStream_t s) {
    H2_REQUIRE(pts != nullptr, "pts is NULL");
    H2_REQUIRE(params != nullptr, "params is NULL");
    H2_REQUIRE(n >= 1 && n < (int64_t)INT32_MAX, "n must be in [1, 2^31 - 1)");
    H2_REQUIRE(dim == 2 || dim == 3, "dim must be 2 or 3");
    H2_REQUIRE(params->leaf_size >= 1, "leaf_size must be >= 1");
    H2_REQUIRE(params->tau_num >= 0 && params->tau_den >= 1, "tau must be tau_num/tau_den with tau_den >= 1");
    pool_keep_memory();
    auto *t = new h2_tree_s();
    try {
        t->stream = s;
        t->n = n;
        t->d = dim;
        t->B = dim == 3 ? 21 : 31;
        t->q = params->leaf_size;
        t->tau_num = params->tau_num;
        t->tau_den = params->tau_den;
        DevBuf<double> tmp;
        const double *pd = pts;
        if (!pts_on_device) {
            tmp.alloc((size_t)n * dim, s);
            H2_CUDA(cudaMemcpyAsync(tmp.p, pts, (size_t)n * dim * sizeof(double), cudaMemcpyHostToDevice, s));
            pd = tmp.p;
        }
        cudaEvent_t e0, e1, e2;
        H2_CUDA(cudaEventCreate(&e0));
        H2_CUDA(cudaEventCreate(&e1));
        H2_CUDA(cudaEventCreate(&e2));
        H2_CUDA(cudaEventRecord(e0, s));
        tree_build_impl(t, pd);
        H2_CUDA(cudaEventRecord(e1, s));
        lists_build_impl(t);
        H2_CUDA(cudaEventRecord(e2, s));
        H2_CUDA(cudaEventSynchronize(e2));
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, e0, e1);
        cudaEventElapsedTime(&b, e1, e2);
        t->ms_tree = a;
        t->ms_lists = b;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
    } catch (...) {
        t->tag = TAG_DEAD;
        delete t;
        throw;
    }
    return t;
}
}  // namespace

namespace {
h2_hidr_s *hidr_one(h2_tree_s *t, int g1, int g2, int method, cudaStream_t s) {
    const bool il = (method & H2_HIDR_IL_REDUCE) != 0, copy = (method & H2_HIDR_COPY_SETS) != 0;
    method &= ~(H2_HIDR_IL_REDUCE | H2_HIDR_COPY_SETS);
    H2_REQUIRE(method == H2_DR_VOLUME || method == H2_DR_SURFACE || method == H2_DR_FPS,
               "unknown DataReduct method or flag");
    H2_REQUIRE(g1 >= 1 && g2 >= 1, "g1 and g2 must be >= 1");
    if (il) {
        int64_t G = 1;
        for (int k = 0; k < t->d; k++) G = std::min<int64_t>(G * g2, 1 << 20);
        H2_REQUIRE(G <= 4096, "the interaction-list reduction needs g2^dim <= 4096");
    }
    auto *h = new h2_hidr_s();
    h->tree = t;
    h->stream = s;
    h->g1 = g1;
    h->g2 = g2;
    h->method = method;
    h->il_reduce = il;
    h->copy_sets = copy;
    try {
        hidr_impl(h);
    } catch (...) {
        h->tag = TAG_DEAD;
        delete h;
        throw;
    }
    return h;
}
}  // namespace

extern "C" {

const char *h2_last_error(void) { return g_last_error.c_str(); }



h2_status h2_tree_build(const double *pts, int64_t n, int dim, int pts_on_device, const h2_tree_params *params,
                        void *stream, h2_tree *out) {
    return guard([&] {
        H2_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        *out = tree_build_one(pts, n, dim, pts_on_device, params, static_cast<cudaStream_t>(stream));
    });
}

h2_status h2_tree_get(h2_tree th, int what, void *buf, int64_t cap, int64_t *len) {
    return guard([&] {
        h2_tree_s *t = as_tree(th);
        cudaStream_t s = t->stream;
        const int nn = t->nnodes;
        switch (what) {
        case H2_TREE_PERM: copy_out(widen<int32_t, int64_t>(read_vec(t->perm.p, t->n, s)), buf, cap, len); break;
        case H2_TREE_KEYS: copy_out(read_vec(t->key.p, t->n, s), buf, cap, len); break;
        case H2_TREE_LEVEL: copy_out(read_vec(t->level.p, nn, s), buf, cap, len); break;
        case H2_TREE_PARENT: copy_out(read_vec(t->parent.p, nn, s), buf, cap, len); break;
        case H2_TREE_FCHILD: copy_out(read_vec(t->fchild.p, nn, s), buf, cap, len); break;
        case H2_TREE_NCHILD: copy_out(read_vec(t->nchild.p, nn, s), buf, cap, len); break;
        case H2_TREE_BEGIN: copy_out(widen<int32_t, int64_t>(read_vec(t->begin.p, nn, s)), buf, cap, len); break;
        case H2_TREE_END: copy_out(widen<int32_t, int64_t>(read_vec(t->end.p, nn, s)), buf, cap, len); break;
        case H2_TREE_PREFIX: copy_out(read_vec(t->prefix.p, nn, s), buf, cap, len); break;
        case H2_TREE_LPTR: copy_out(std::vector<int32_t>(t->lptr.begin(), t->lptr.end()), buf, cap, len); break;
        case H2_TREE_NEAR_PTR: copy_out(read_vec(t->near_ptr.p, nn + 1, s), buf, cap, len); break;
        case H2_TREE_FAR_PTR: copy_out(read_vec(t->far_ptr.p, nn + 1, s), buf, cap, len); break;
        case H2_TREE_NEAR_IDX: copy_out(read_vec(t->near_idx.p, t->nnear, s), buf, cap, len); break;
        case H2_TREE_FAR_IDX: copy_out(read_vec(t->far_idx.p, t->nfar, s), buf, cap, len); break;
        case H2_TREE_INFO: {
            std::vector<int64_t> v = {t->n, t->d, t->B, t->nnodes, t->nlevels, t->nnear, t->nfar, t->q};
            copy_out(v, buf, cap, len);
            break;
        }
        case H2_TREE_GEOM: {
            std::vector<double> v = {t->geom.lo[0], t->geom.lo[1], t->geom.lo[2], t->geom.side};
            copy_out(v, buf, cap, len);
            break;
        }
        default: fail(H2_ERR_INVALID_ARG, "unknown tree field");
        }
    });
}

h2_status h2_hidr_reduce(h2_tree th, int g1, int g2, void *stream, h2_hidr *out) {
    return h2_hidr_reduce_ex(th, g1, g2, H2_DR_VOLUME, stream, out);
}


h2_status h2_hidr_reduce_ex(h2_tree th, int g1, int g2, int method, void *stream, h2_hidr *out) {
    return guard([&] {
        H2_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        const int m = method & ~(H2_HIDR_IL_REDUCE | H2_HIDR_COPY_SETS);  // (checked before the handle)
        H2_REQUIRE(m == H2_DR_VOLUME || m == H2_DR_SURFACE || m == H2_DR_FPS, "unknown DataReduct method or flag");
        h2_tree_s *t = as_tree(th);
        h2_hidr_s *h = hidr_one(t, g1, g2, method, static_cast<cudaStream_t>(stream));
        t->refs++;
        *out = h;
    });
}

h2_status h2_tree_build_batched(int nprob, const double *const *pts, const int64_t *ns, int dim, int pts_on_device,
                                const h2_tree_params *params, void *stream, h2_tree *out) {
    return guard([&] {
        H2_REQUIRE(nprob >= 0, "nprob must be >= 0");
        if (nprob == 0) return;
        H2_REQUIRE(pts && ns && params && out, "NULL argument");
        for (int p = 0; p < nprob; p++) out[p] = nullptr;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        std::vector<h2_tree_s *> trees(nprob, nullptr);
        std::vector<h2_status> st;
        std::vector<std::string> msg;
        auto drop = [&] {
            for (auto *t : trees)
                if (t) { tree_rebind(t, s); t->tag = TAG_DEAD; delete t; }
        };
        try {
            run_concurrently(nprob, s, st, msg, [&](int p, cudaStream_t ws) {
                trees[p] = tree_build_one(pts[p], ns[p], dim, pts_on_device, params + p, ws);
            });
            for (auto *t : trees)
                if (t) tree_rebind(t, s);
        } catch (...) {
            drop();
            throw;
        }
        for (int p = 0; p < nprob; p++)
            if (st[p] != H2_OK) {
                drop();
                fail(st[p], "problem " + std::to_string(p) + ": " + msg[p]);
            }
        for (int p = 0; p < nprob; p++) out[p] = trees[p];
    });
}

h2_status h2_hidr_reduce_batched(int nprob, const h2_tree *trees, const int *g1, const int *g2, const int *methods,
                                 void *stream, h2_hidr *out) {
    return guard([&] {
        H2_REQUIRE(nprob >= 0, "nprob must be >= 0");
        if (nprob == 0) return;
        H2_REQUIRE(trees && g1 && g2 && out, "NULL argument");
        for (int p = 0; p < nprob; p++) out[p] = nullptr;
        std::vector<h2_tree_s *> ts(nprob);
        for (int p = 0; p < nprob; p++) {
            try {
                ts[p] = as_tree(trees[p]);
            } catch (const Error &e) {
                fail(e.st, "problem " + std::to_string(p) + ": " + e.msg);
            }
        }
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        std::vector<h2_hidr_s *> hs(nprob, nullptr);
        std::vector<h2_status> st;
        std::vector<std::string> msg;
        auto drop = [&] {
            for (auto *h : hs)
                if (h) { hidr_rebind(h, s); h->tag = TAG_DEAD; delete h; }
        };
        try {
            run_concurrently(nprob, s, st, msg, [&](int p, cudaStream_t ws) {
                hs[p] = hidr_one(ts[p], g1[p], g2[p], methods ? methods[p] : H2_DR_VOLUME, ws);
            });
            for (auto *h : hs)
                if (h) hidr_rebind(h, s);
        } catch (...) {
            drop();
            throw;
        }
        for (int p = 0; p < nprob; p++)
            if (st[p] != H2_OK) {
                drop();
                fail(st[p], "problem " + std::to_string(p) + ": " + msg[p]);
            }
        for (int p = 0; p < nprob; p++) {
            ts[p]->refs++;
            out[p] = hs[p];
        }
    });
}

h2_status h2_hidr_get(h2_hidr hh, int which, int32_t *counts, int32_t *data, int64_t cap, int64_t *total) {
    return guard([&] {
        h2_hidr_s *h = as_hidr(hh);
        H2_REQUIRE(which == 0 || which == 1, "which must be 0 (X*) or 1 (Y*)");
        cudaStream_t s = h->stream;
        const int nn = h->tree->nnodes;
        std::vector<int32_t> cnt = read_vec(which ? h->ycnt.p : h->xcnt.p, nn, s);
        std::vector<int32_t *> ptr = read_vec(which ? h->yptr.p : h->xptr.p, nn, s);
        int64_t tot = 0;
        for (int32_t c : cnt) tot += c;
        if (total) *total = tot;
        if (counts) memcpy(counts, cnt.data(), nn * sizeof(int32_t));
        if (data) {
            H2_REQUIRE(cap >= tot, "output buffer too small");
            int64_t w = 0;
            for (int i = 0; i < nn; i++) {
                if (cnt[i] > 0)
                    H2_CUDA(cudaMemcpyAsync(data + w, ptr[i], cnt[i] * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                w += cnt[i];
            }
            H2_CUDA(cudaStreamSynchronize(s));
        }
    });
}

h2_status h2_construct(h2_tree th, h2_hidr hh, int kernel, const double *kparams, double id_tol, int precision,
                       void *stream, h2_matrix *out) {
    return h2_construct_ex(th, hh, kernel, kparams, id_tol, precision, nullptr, stream, out);
}

h2_status h2_construct_ex(h2_tree th, h2_hidr hh, int kernel, const double *kparams, double id_tol,
                          int precision, const h2_construct_opts *opts, void *stream, h2_matrix *out) {
    return guard([&] {
        H2_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        h2_tree_s *t = as_tree(th);
        h2_hidr_s *h = as_hidr(hh);
        H2_REQUIRE(h->tree == t, "hidr was built on another tree");
        H2_REQUIRE(valid_kernel(kernel), "unknown kernel id");
        H2_REQUIRE(std::isfinite(id_tol) && id_tol >= 0.0, "id_tol must be finite and >= 0");
        H2_REQUIRE(precision == H2_PREC_FP64 || precision == H2_PREC_MIXED, "unknown precision");
        const double gb = opts ? opts->g_bound : 0.0;
        H2_REQUIRE(gb == 0.0 || (std::isfinite(gb) && gb > 1.0), "g_bound must be 0 or a finite number > 1");
        const int mm = opts ? opts->mem_mode : H2_MEM_ON_THE_FLY;
        H2_REQUIRE(mm == H2_MEM_ON_THE_FLY || mm == H2_MEM_STORE || mm == H2_MEM_AUTO, "unknown mem_mode");
        const double mf = opts ? opts->mem_fraction : 0.0;
        H2_REQUIRE(std::isfinite(mf) && mf >= 0.0 && mf <= 1.0, "mem_fraction must be in [0, 1]");
        auto *A = new h2_matrix_s();
        A->tree = t;
        A->stream = static_cast<cudaStream_t>(stream);
        A->kid = kernel;
        A->id_tol = id_tol;
        A->prec = precision;
        A->g_bound = gb;
        A->mem_mode = mm;
        A->mem_fraction = mf > 0.0 ? mf : 0.5;
        A->fp64_products = opts && opts->fp64_products != 0;
        A->tensor_core_products = opts && opts->tensor_core_products != 0;
        A->fp64_qr = opts && opts->fp64_qr != 0;
        try {
            kparams_check(kernel, kparams, A->kp);
            construct_impl(A, h);
            if (mm == H2_MEM_STORE || (mm == H2_MEM_AUTO && precision == H2_PREC_FP64))
                store_blocks_impl(A, mm, A->mem_fraction);
        } catch (...) {
            A->tag = TAG_DEAD;
            delete A;
            throw;
        }
        t->refs++;
        *out = A;
    });
}

h2_status h2_construct_batched(int nprob, const h2_tree *trees, const h2_hidr *hidrs, const int *kernels,
                               const double *kparams, const double *id_tols, const int *precisions, void *stream,
                               h2_matrix *out) {
    return guard([&] {
        H2_REQUIRE(nprob >= 0, "nprob must be >= 0");
        if (nprob == 0) return;
        H2_REQUIRE(trees && hidrs && kernels && id_tols && precisions && out, "NULL argument");
        for (int p = 0; p < nprob; p++) out[p] = nullptr;
        struct Job {
            h2_tree_s *t;
            h2_hidr_s *h;
            double kp[4];
        };
        std::vector<Job> jobs(nprob);
        for (int p = 0; p < nprob; p++) {
            try {
                jobs[p].t = as_tree(trees[p]);
                jobs[p].h = as_hidr(hidrs[p]);
                H2_REQUIRE(jobs[p].h->tree == jobs[p].t, "hidr was built on another tree");
                H2_REQUIRE(valid_kernel(kernels[p]), "unknown kernel id");
                H2_REQUIRE(std::isfinite(id_tols[p]) && id_tols[p] >= 0.0, "id_tol must be finite and >= 0");
                H2_REQUIRE(precisions[p] == H2_PREC_FP64 || precisions[p] == H2_PREC_MIXED, "unknown precision");
                kparams_check(kernels[p], kparams ? kparams + 4 * p : nullptr, jobs[p].kp);
            } catch (const Error &e) {
                fail(e.st, "problem " + std::to_string(p) + ": " + e.msg);
            }
        }
        pool_keep_memory();
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        int dev = 0;
        H2_CUDA(cudaGetDevice(&dev));
        const int nw = std::min(nprob, 8);
        std::vector<cudaStream_t> ws(nw, nullptr);
        std::vector<cudaEvent_t> done(nw, nullptr);
        cudaEvent_t ready = nullptr;
        auto cleanup = [&] {
            for (int w = 0; w < nw; w++) {
                if (done[w]) cudaEventDestroy(done[w]);
                if (ws[w]) cudaStreamDestroy(ws[w]);
            }
            if (ready) cudaEventDestroy(ready);
        };
        std::vector<h2_matrix_s *> mats(nprob, nullptr);
        std::vector<h2_status> st(nprob, H2_OK);
        std::vector<std::string> msg(nprob);
        try {
            H2_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
            H2_CUDA(cudaEventRecord(ready, s));  // after the work already queued on stream
            for (int w = 0; w < nw; w++) {
                H2_CUDA(cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking));
                H2_CUDA(cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming));
                H2_CUDA(cudaStreamWaitEvent(ws[w], ready, 0));
            }
            std::atomic<int> next{0};
            auto worker = [&](int w) {
                if (cudaSetDevice(dev) != cudaSuccess) return;
                for (int p = next++; p < nprob; p = next++) {
                    auto *A = new h2_matrix_s();
                    A->tree = jobs[p].t;
                    A->stream = ws[w];
                    A->kid = kernels[p];
                    A->id_tol = id_tols[p];
                    A->prec = precisions[p];
                    for (int a = 0; a < 4; a++) A->kp[a] = jobs[p].kp[a];
                    try {
                        construct_impl(A, jobs[p].h);
                        mats[p] = A;
                    } catch (const Error &e) {
                        st[p] = e.st;
                        msg[p] = e.msg;
                    } catch (const std::bad_alloc &) {
                        st[p] = H2_ERR_OOM;
                        msg[p] = "host allocation failed";
                    } catch (...) {
                        st[p] = H2_ERR_CUDA;
                        msg[p] = "unknown error";
                    }
                    if (!mats[p]) {
                        A->tag = TAG_DEAD;
                        delete A;
                    }
                }
            };
            std::vector<std::thread> th;
            try {
                for (int w = 0; w < nw; w++) th.emplace_back(worker, w);
            } catch (...) {  // no more threads: stop handing out problems, join the started ones
                next = nprob;
                for (auto &x : th) x.join();
                throw;
            }
            for (auto &x : th) x.join();
            // the caller's stream waits for every worker stream; the matrices
            // then live on it
            for (int w = 0; w < nw; w++) {
                H2_CUDA(cudaEventRecord(done[w], ws[w]));
                H2_CUDA(cudaStreamWaitEvent(s, done[w], 0));
            }
            for (int p = 0; p < nprob; p++)
                if (mats[p]) matrix_rebind(mats[p], s);
        } catch (...) {
            for (auto *A : mats)
                if (A) { matrix_rebind(A, s); A->tag = TAG_DEAD; delete A; }
            cleanup();
            throw;
        }
        cleanup();
        for (int p = 0; p < nprob; p++)
            if (st[p] != H2_OK) {
                for (auto *A : mats)
                    if (A) { A->tag = TAG_DEAD; delete A; }
                fail(st[p], "problem " + std::to_string(p) + ": " + msg[p]);
            }
        for (int p = 0; p < nprob; p++) {
            jobs[p].t->refs++;
            out[p] = mats[p];
        }
    });
}

h2_status h2_matrix_get(h2_matrix ah, int what, void *buf, int64_t cap, int64_t *len) {
    return guard([&] {
        h2_matrix_s *A = as_matrix(ah);
        cudaStream_t s = A->stream;
        const int nn = A->tree->nnodes;
        switch (what) {
        case H2_MAT_RANK: copy_out(read_vec(A->k.p, nn, s), buf, cap, len); break;
        case H2_MAT_NCAND: copy_out(read_vec(A->c.p, nn, s), buf, cap, len); break;
        case H2_MAT_SKEL: copy_out(read_vec(A->skel.p, A->ktotal, s), buf, cap, len); break;
        case H2_MAT_U: {
            std::vector<int32_t> k = read_vec(A->k.p, nn, s), c = read_vec(A->c.p, nn, s);
            std::vector<void *> up = read_vec(A->uptr.p, nn, s);
            int64_t tot = 0;
            for (int i = 0; i < nn; i++) tot += (int64_t)k[i] * c[i];
            if (len) *len = tot;
            if (!buf) break;
            H2_REQUIRE(cap >= tot, "output buffer too small");
            double *dst = static_cast<double *>(buf);
            const bool f64 = A->prec == H2_PREC_FP64;
            std::vector<float> tmp;
            for (int i = 0; i < nn; i++) {
                int64_t e = (int64_t)k[i] * c[i];
                if (e > 0) {
                    if (f64) {
                        H2_CUDA(cudaMemcpyAsync(dst, up[i], e * sizeof(double), cudaMemcpyDeviceToHost, s));
                    } else {  // float32 storage, widened on the host
                        tmp.resize(e);
                        H2_CUDA(cudaMemcpyAsync(tmp.data(), up[i], e * sizeof(float), cudaMemcpyDeviceToHost, s));
                        H2_CUDA(cudaStreamSynchronize(s));
                        for (int64_t q = 0; q < e; q++) dst[q] = tmp[q];
                    }
                }
                dst += e;
            }
            H2_CUDA(cudaStreamSynchronize(s));
            break;
        }
        case H2_MAT_INFO: {
            std::vector<int64_t> v = {A->ktotal, A->utotal, A->kmax, A->tree->nlevels};
            copy_out(v, buf, cap, len);
            break;
        }
        default: fail(H2_ERR_INVALID_ARG, "unknown matrix field");
        }
    });
}

namespace {
// h2_matvec's argument checks
void matvec_args_check(h2_matrix_s *A, const void *x, const void *y, int nrhs, int dtype, int64_t ld) {
    H2_REQUIRE(x != nullptr && y != nullptr, "x or y is NULL");
    H2_REQUIRE(nrhs >= 1, "nrhs must be >= 1");
    H2_REQUIRE(dtype == H2_DTYPE_F64 || dtype == H2_DTYPE_F32, "dtype must be H2_DTYPE_F64 or H2_DTYPE_F32");
    const int64_t n = A->tree->n;
    H2_REQUIRE(ld >= n, "ld must be >= n");
    const size_t es = dtype == H2_DTYPE_F64 ? sizeof(double) : sizeof(float);
    const size_t span = ((size_t)(nrhs - 1) * (size_t)ld + (size_t)n) * es;
    const char *xb = static_cast<const char *>(x), *yb = static_cast<const char *>(y);
    H2_REQUIRE(xb + span <= yb || yb + span <= xb, "x and y overlap");
}

// the product on device buffers
void matvec_device(h2_matrix_s *A, const void *x, void *y, int nrhs, int dtype, int64_t ld, cudaStream_t s) {
    if (nrhs == 1 && dtype == H2_DTYPE_F64)
        matvec_impl(A, static_cast<const double *>(x), static_cast<double *>(y), s);
    else
        matvec_multi_impl(A, x, y, nrhs, dtype, ld, s);
}

h2_graph_s *as_graph(void *h) {
    auto *g = static_cast<h2_graph_s *>(h);
    if (!g || g->tag != TAG_GRAPH) fail(H2_ERR_INVALID_ARG, "not a graph handle");
    return g;
}
}  // namespace

h2_status h2_matvec(h2_matrix ah, const void *x, void *y, int nrhs, int dtype, int64_t ld, int on_device,
                    void *stream) {
    return guard([&] {
        h2_matrix_s *A = as_matrix(ah);
        matvec_args_check(A, x, y, nrhs, dtype, ld);
        const int64_t n = A->tree->n;
        const size_t es = dtype == H2_DTYPE_F64 ? sizeof(double) : sizeof(float);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const bool single = nrhs == 1 && dtype == H2_DTYPE_F64;
        if (on_device) {
            matvec_device(A, x, y, nrhs, dtype, ld, s);
            return;
        }
        DevBuf<char> xd, yd;
        xd.alloc((size_t)n * nrhs * es, s);
        yd.alloc((size_t)n * nrhs * es, s);
        H2_CUDA(cudaMemcpy2DAsync(xd.p, n * es, x, ld * es, n * es, nrhs, cudaMemcpyHostToDevice, s));
        if (single)
            matvec_impl(A, reinterpret_cast<const double *>(xd.p), reinterpret_cast<double *>(yd.p), s);
        else
            matvec_multi_impl(A, xd.p, yd.p, nrhs, dtype, n, s);
        H2_CUDA(cudaMemcpy2DAsync(y, ld * es, yd.p, n * es, n * es, nrhs, cudaMemcpyDeviceToHost, s));
        H2_CUDA(cudaStreamSynchronize(s));
        if (A->tree->tc_status.p) {  // a tensor-core wait that gave up (the call synchronised)
            int st = 0;
            H2_CUDA(cudaMemcpy(&st, A->tree->tc_status.p, sizeof st, cudaMemcpyDeviceToHost));
            if (st) fail(H2_ERR_TIMEOUT, "a tensor-core wait of the nearfield gave up; the product is incomplete");
        }
    });
}

h2_status h2_matvec_graph_create(h2_matrix ah, void *x, void *y, int nrhs, int dtype, int64_t ld, void *stream,
                                 h2_graph *out) {
    return guard([&] {
        H2_REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        h2_matrix_s *A = as_matrix(ah);
        matvec_args_check(A, x, y, nrhs, dtype, ld);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        // one ordinary product: tiles, list starts and kernel attributes are set
        // up on first use, with host synchronisations a capture cannot hold
        matvec_device(A, x, y, nrhs, dtype, ld, s);
        H2_CUDA(cudaStreamSynchronize(s));
        cudaStream_t cs = nullptr;
        H2_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        const bool prof = profiling_enabled();
        if (prof) profile_set(false, false);  // no timing events inside the graph
        auto *G = new h2_graph_s();
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        std::string msg;
        if (e == cudaSuccess) {
            try {
                matvec_device(A, x, y, nrhs, dtype, ld, cs);
            } catch (const h2::Error &ex) {
                msg = ex.msg;
            } catch (...) {
                msg = "error during capture";
            }
            cudaGraph_t gr = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
            G->graph = gr;
            if (msg.empty() && e2 != cudaSuccess) msg = cudaGetErrorString(e2);
            if (msg.empty()) {
                const cudaError_t e3 = cudaGraphInstantiate(&G->exec, G->graph, 0);
                if (e3 != cudaSuccess) msg = cudaGetErrorString(e3);
            }
        } else {
            msg = cudaGetErrorString(e);
        }
        cudaStreamDestroy(cs);
        if (prof) profile_set(true, false);
        if (!msg.empty()) {
            cudaGetLastError();
            G->tag = TAG_DEAD;
            delete G;
            fail(H2_ERR_CUDA, "matvec graph: " + msg);
        }
        G->A = A;
        A->refs++;
        *out = G;
    });
}

h2_status h2_matvec_graph_launch(h2_graph gh, void *stream) {
    return guard([&] {
        h2_graph_s *G = as_graph(gh);
        H2_CUDA(cudaGraphLaunch(G->exec, static_cast<cudaStream_t>(stream)));
    });
}

h2_status h2_exact_rows(h2_tree th, int kernel, const double *kparams, const double *z, const int64_t *rows,
                        int64_t nrows, double *out, int on_device, void *stream) {
    return guard([&] {
        h2_tree_s *t = as_tree(th);
        H2_REQUIRE(valid_kernel(kernel), "unknown kernel id");
        H2_REQUIRE(z != nullptr && (nrows == 0 || (rows != nullptr && out != nullptr)), "NULL argument");
        H2_REQUIRE(nrows >= 0 && nrows < (int64_t)INT32_MAX, "bad nrows");
        double kp[4];
        kparams_check(kernel, kparams, kp);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (!on_device) {
            std::vector<int64_t> rv(rows, rows + nrows);
            for (int64_t r : rv) H2_REQUIRE(r >= 0 && r < t->n, "row index out of range");
            DevBuf<double> zd, od;
            DevBuf<int64_t> rd;
            zd.alloc(t->n, s);
            od.alloc(std::max<int64_t>(nrows, 1), s);
            rd.alloc(std::max<int64_t>(nrows, 1), s);
            H2_CUDA(cudaMemcpyAsync(zd.p, z, t->n * sizeof(double), cudaMemcpyHostToDevice, s));
            if (nrows) H2_CUDA(cudaMemcpyAsync(rd.p, rows, nrows * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            exact_rows_impl(t, kernel, kp, zd.p, rd.p, nrows, od.p, s);
            if (nrows) H2_CUDA(cudaMemcpyAsync(out, od.p, nrows * sizeof(double), cudaMemcpyDeviceToHost, s));
            H2_CUDA(cudaStreamSynchronize(s));
            return;
        }
        exact_rows_impl(t, kernel, kp, z, rows, nrows, out, s);
    });
}

h2_status h2_exact_rows_noalloc(h2_tree th, int kernel, const double *kparams, const double *z, const int64_t *rows,
                                int64_t nrows, double *out, void *stream) {
    return guard([&] {
        h2_tree_s *t = as_tree(th);
        H2_REQUIRE(valid_kernel(kernel), "unknown kernel id");
        H2_REQUIRE(z != nullptr && (nrows == 0 || (rows != nullptr && out != nullptr)), "NULL argument");
        H2_REQUIRE(nrows >= 0 && nrows < (int64_t)INT32_MAX, "bad nrows");
        double kp[4];
        kparams_check(kernel, kparams, kp);
        require_device_ptr(z, "z");
        if (nrows > 0) {
            require_device_ptr(rows, "rows");
            require_device_ptr(out, "out");
        }
        exact_rows_noalloc_impl(t, kernel, kp, z, rows, nrows, out, static_cast<cudaStream_t>(stream));
    });
}

h2_status h2_debug_fail_alloc(int64_t k, int64_t *allocs_since_last) {
    return guard([&] {
        H2_REQUIRE(k >= 0, "k must be >= 0");
        const int64_t made = debug_fail_alloc(k);
        if (allocs_since_last) *allocs_since_last = made;
    });
}

h2_status h2_autotune_leaf(const double *pts, int64_t n, int dim, int pts_on_device, const int *cands,
                           int ncand, int g, int kernel, const double *kparams, double id_tol, int precision,
                           int reps, void *stream, int *best, double *times) {
    return guard([&] {
        H2_REQUIRE(cands != nullptr && ncand >= 1, "no candidate leaf sizes");
        H2_REQUIRE(best != nullptr, "best is NULL");
        H2_REQUIRE(reps >= 1, "reps must be >= 1");
        H2_REQUIRE(n >= 1, "n must be >= 1");
        for (int c = 0; c < ncand; c++) H2_REQUIRE(cands[c] >= 1, "leaf sizes must be >= 1");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        DevBuf<double> x, y;
        x.alloc(n, s);
        y.alloc(n, s);
        H2_CUDA(cudaMemsetAsync(x.p, 0, n * sizeof(double), s));
        struct Events {  // destroyed on every way out
            cudaEvent_t a = nullptr, b = nullptr;
            ~Events() {
                if (a) cudaEventDestroy(a);
                if (b) cudaEventDestroy(b);
            }
        } ev;
        H2_CUDA(cudaEventCreate(&ev.a));
        H2_CUDA(cudaEventCreate(&ev.b));
        cudaEvent_t e0 = ev.a, e1 = ev.b;
        double best_ms = 0.0;
        // a failing call's status and message pass through; the handles of
        // the round in progress are released on the way out
        auto run = [&](int q) -> double {
            h2_tree_params prm{q, 7, 10};
            h2_tree t = nullptr;
            h2_hidr h = nullptr;
            h2_matrix A = nullptr;
            h2_status st = H2_OK;
            H2_CUDA(cudaEventRecord(e0, s));
            st = h2_tree_build(pts, n, dim, pts_on_device, &prm, stream, &t);
            if (st == H2_OK) st = h2_hidr_reduce(t, g, g, stream, &h);
            if (st == H2_OK) st = h2_construct(t, h, kernel, kparams, id_tol, precision, stream, &A);
            if (st == H2_OK) st = h2_matvec(A, x.p, y.p, 1, H2_DTYPE_F64, n, 1, stream);
            std::string msg = st == H2_OK ? std::string() : std::string(h2_last_error());
            float ms = 0.f;
            if (st == H2_OK) {
                H2_CUDA(cudaEventRecord(e1, s));
                H2_CUDA(cudaEventSynchronize(e1));
                H2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            }
            h2_free(A);
            h2_free(h);
            h2_free(t);
            if (st != H2_OK) fail(st, msg);
            return ms;
        };
        for (int c = 0; c < ncand; c++) {
            double tmin = 0.0;
            for (int r = 0; r < reps; r++) {
                const double ms = run(cands[c]);
                tmin = r == 0 ? ms : std::min(tmin, ms);
            }
            if (times) times[c] = tmin;
            if (c == 0 || tmin < best_ms) {
                best_ms = tmin;
                *best = cands[c];
            }
        }
    });
}

h2_status h2_free(void *handle) {
    return guard([&] {
        if (!handle) return;
        uint32_t tag = *static_cast<uint32_t *>(handle);
        if (tag == TAG_TREE) {
            auto *t = static_cast<h2_tree_s *>(handle);
            if (t->refs > 0) fail(H2_ERR_STATE, "tree still has live hidr/matrix handles");
            t->tag = TAG_DEAD;
            delete t;
        } else if (tag == TAG_HIDR) {
            auto *h = static_cast<h2_hidr_s *>(handle);
            h->tree->refs--;
            h->tag = TAG_DEAD;
            delete h;
        } else if (tag == TAG_MATRIX) {
            auto *A = static_cast<h2_matrix_s *>(handle);
            if (A->refs > 0) fail(H2_ERR_STATE, "matrix still has live graph handles");
            A->tree->refs--;
            A->tag = TAG_DEAD;
            delete A;
        } else if (tag == TAG_GRAPH) {
            auto *G = static_cast<h2_graph_s *>(handle);
            G->A->refs--;
            G->tag = TAG_DEAD;
            delete G;
        } else {
            fail(H2_ERR_INVALID_ARG, "not a live h2 handle");
        }
    });
}

h2_status h2_profile(int enable, int reset) {
    return guard([&] { profile_set(enable != 0, reset != 0); });
}

h2_status h2_fma_peak(double *fp64_tflops, double *fp32_tflops, void *stream) {
    return guard([&] {
        H2_REQUIRE(fp64_tflops || fp32_tflops, "NULL argument");
        fma_peaks(fp64_tflops, fp32_tflops, static_cast<cudaStream_t>(stream));
    });
}

h2_status h2_get_stats(const void *handle, char *json, int64_t cap) {
    return guard([&] {
        H2_REQUIRE(json && cap > 0, "NULL argument");
        if (!handle) {
            std::string js = profile_json();
            H2_REQUIRE((int64_t)js.size() < cap, "json buffer too small");
            memcpy(json, js.c_str(), js.size() + 1);
            return;
        }
        uint32_t tag = *static_cast<const uint32_t *>(handle);
        char buf[1024];
        if (tag == TAG_TREE) {
            auto *t = static_cast<const h2_tree_s *>(handle);
            snprintf(buf, sizeof buf,
                     "{\"n\": %lld, \"nodes\": %d, \"levels\": %d, \"near_pairs\": %lld, \"far_pairs\": %lld, "
                     "\"max_leaf\": %d, \"ms_tree\": %.4f, \"ms_lists\": %.4f}",
                     (long long)t->n, t->nnodes, t->nlevels, (long long)t->nnear, (long long)t->nfar, t->max_leaf,
                     t->ms_tree, t->ms_lists);
        } else if (tag == TAG_HIDR) {
            auto *h = static_cast<const h2_hidr_s *>(handle);
            snprintf(buf, sizeof buf,
                     "{\"g1\": %d, \"g2\": %d, \"x_total\": %lld, \"y_total\": %lld, \"t_max_level\": %lld, "
                     "\"t_total\": %lld, \"t_il_total\": %lld, \"ms_up\": %.4f, \"ms_down\": %.4f, "
                     "\"method\": \"%s\", \"il_reduce\": %s}",
                     h->g1, h->g2, (long long)h->xtotal, (long long)h->ytotal, (long long)h->tmax,
                     (long long)h->ttotal, (long long)h->iltotal, h->ms_up, h->ms_down,
                     h->method == H2_DR_SURFACE ? "surface" : (h->method == H2_DR_FPS ? "fps" : "volume"),
                     h->il_reduce ? "true" : "false");
        } else if (tag == TAG_MATRIX) {
            auto *A = static_cast<const h2_matrix_s *>(handle);
            snprintf(buf, sizeof buf,
                     "{\"k_total\": %lld, \"u_entries\": %lld, \"k_max\": %d, \"ms_construct\": %.4f, "
                     "\"qr_flops\": %.6e, \"block_evals\": %.6e, \"g_max\": %.6e, \"g_bound\": %.6e, "
                     "\"exchanges\": %lld, \"precision\": \"%s\", \"mem_mode\": \"%s\", "
                     "\"stored_bytes\": %lld, \"stored_far_bytes\": %lld, \"stored_near_bytes\": %lld, "
                     "\"planned_bytes\": %lld, \"ms_blocks\": %.4f, \"fp64_products\": %s, \"fp64_qr\": %s}",
                     (long long)A->ktotal, (long long)A->utotal, A->kmax, A->ms_construct, A->flops_qr,
                     A->evals_block, A->g_max, A->g_bound, (long long)A->exchanges,
                     A->prec == H2_PREC_FP64 ? "fp64" : "mixed", A->stored ? "stored" : "on_the_fly",
                     (long long)(A->stored_far_bytes + A->stored_near_bytes), (long long)A->stored_far_bytes,
                     (long long)A->stored_near_bytes, (long long)A->stored_bytes_plan, A->ms_blocks,
                     A->fp64_products ? "true" : "false", A->fp64_qr ? "true" : "false");
        } else {
            fail(H2_ERR_INVALID_ARG, "not a live h2 handle");
        }
        H2_REQUIRE((int64_t)strlen(buf) < cap, "json buffer too small");
        memcpy(json, buf, strlen(buf) + 1);
    });
}

h2_status h2_calibrate(int dim, int kernel, const double *kparams, double eps, const double *z1, int n1,
                       const double *z2, int n2, int gmax, void *stream, int *g_out, double *err_out) {
    return guard([&] {
        H2_REQUIRE(dim == 2 || dim == 3, "dim must be 2 or 3");
        H2_REQUIRE(valid_kernel(kernel), "unknown kernel id");
        H2_REQUIRE(z1 && z2 && g_out && n1 > 0 && n2 > 0 && gmax >= 1, "bad calibration arguments");
        H2_REQUIRE(std::isfinite(eps) && eps > 0.0, "eps must be > 0");
        double kp[4];
        kparams_check(kernel, kparams, kp);
        pool_keep_memory();
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        DevBuf<double> a[3], b[3];
        DevBuf<float4> bq;
        std::vector<double> col(std::max(n1, n2));
        std::vector<float4> packed(2 * (size_t)n2, make_float4(0.f, 0.f, 0.f, 0.f));
        long long zbox[6] = {LLONG_MAX, LLONG_MAX, LLONG_MAX, LLONG_MIN, LLONG_MIN, LLONG_MIN};
        DRPoints zb;
        zb.R = 0.0;
        bq.alloc(2 * (size_t)n2, s);
        zb.xq = bq.p;
        for (int k = 0; k < 3; k++) {
            a[k].alloc(k < dim ? n1 : 1, s);
            b[k].alloc(k < dim ? n2 : 1, s);
            zb.x[k] = b[k].p;
            zb.ref[k] = 0.0;
            if (k >= dim) continue;
            for (int i = 0; i < n1; i++) col[i] = z1[(int64_t)i * dim + k];
            H2_CUDA(cudaMemcpyAsync(a[k].p, col.data(), n1 * sizeof(double), cudaMemcpyHostToDevice, s));
            for (int i = 0; i < n2; i++) {
                col[i] = z2[(int64_t)i * dim + k];
                const float hi = (float)col[i];  // relative to ref = 0, split into float32 hi + lo
                const float lo = (float)(col[i] - (double)hi);
                float4 &qa = packed[2 * (size_t)i], &qb = packed[2 * (size_t)i + 1];
                if (k == 0) { qa.x = hi; qa.w = lo; }
                else if (k == 1) { qa.y = hi; qb.x = lo; }
                else { qa.z = hi; qb.y = lo; }
                zb.R = std::max(zb.R, std::fabs(col[i]));
                zbox[k] = std::min(zbox[k], dkey_host(col[i]));
                zbox[3 + k] = std::max(zbox[3 + k], dkey_host(col[i]));
            }
            H2_CUDA(cudaMemcpyAsync(b[k].p, col.data(), n2 * sizeof(double), cudaMemcpyHostToDevice, s));
            H2_CUDA(cudaStreamSynchronize(s));
        }
        H2_CUDA(cudaMemcpyAsync(bq.p, packed.data(), packed.size() * sizeof(float4), cudaMemcpyHostToDevice, s));
        H2_CUDA(cudaStreamSynchronize(s));
        const double *za[3] = {a[0].p, a[1].p, a[2].p};
        *g_out = gmax + 1;
        double err = INFINITY;
        for (int g = 1; g <= gmax; g++) {
            double gp = 1.0;
            for (int k = 0; k < dim; k++) gp *= g;
            if (gp > 16384) break;
            err = calib_error_gpu(dim, kernel, kp[0], 1e-2 * eps, za, n1, zb, zbox, n2, g, nullptr, nullptr, s);
            if (err < 1e-2 * eps) {
                *g_out = g;
                break;
            }
        }
        if (err_out) *err_out = err;
    });
}

h2_status h2_sampled_error(const double *exact, const double *approx, const int64_t *rows, int64_t nrows,
                           int64_t n, double *err_out, int on_device, void *stream) {
    return guard([&] {
        H2_REQUIRE(exact && approx && rows && err_out && nrows >= 1 && n >= 1, "bad arguments");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (on_device) {
            sampled_error_impl(exact, approx, rows, nrows, n, err_out, s);
            return;
        }
        DevBuf<double> e, a, o;
        DevBuf<int64_t> r;
        e.alloc(nrows, s); a.alloc(n, s); o.alloc(1, s); r.alloc(nrows, s);
        H2_CUDA(cudaMemcpyAsync(e.p, exact, nrows * sizeof(double), cudaMemcpyHostToDevice, s));
        H2_CUDA(cudaMemcpyAsync(a.p, approx, n * sizeof(double), cudaMemcpyHostToDevice, s));
        H2_CUDA(cudaMemcpyAsync(r.p, rows, nrows * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        sampled_error_impl(e.p, a.p, r.p, nrows, n, o.p, s);
        H2_CUDA(cudaMemcpyAsync(err_out, o.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        H2_CUDA(cudaStreamSynchronize(s));
    });
}

}  // extern "C"
