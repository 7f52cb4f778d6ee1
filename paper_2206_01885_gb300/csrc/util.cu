// util.cu -- errors, stream-ordered allocation, exclusive scan and a stable
// LSD radix sort of 64-bit keys (used for the Morton sort and for ordering the
// near/far pair lists).
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "h2_internal.cuh"

namespace h2 {

void fail(h2_status st, const std::string &msg) { throw Error{st, msg}; }

namespace {
std::atomic<long long> g_launches{0};
}
void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    fail(e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, buf);
}

// Allocation-failure injection (h2_debug_fail_alloc): device allocations are
// counted from the last arming; the one numbered g_fail_at fails as if the
// stream-ordered allocator had run out of memory.  0 = never.
static std::atomic<int64_t> g_alloc_count{0};
static std::atomic<int64_t> g_fail_at{0};

int64_t debug_fail_alloc(int64_t k) {
    const int64_t made = g_alloc_count.exchange(0);
    g_fail_at.store(k);
    return made;
}

void *dmalloc_bytes(size_t bytes, cudaStream_t s) {
    const int64_t k = ++g_alloc_count;
    const int64_t f = g_fail_at.load();
    if (f > 0 && k == f) {
        char buf[160];
        snprintf(buf, sizeof buf, "device allocation of %zu bytes failed: injected failure of allocation %lld",
                 bytes, (long long)k);
        fail(H2_ERR_OOM, buf);
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        fail(H2_ERR_OOM, buf);
    }
    return p;
}

void dfree_bytes(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// -------------------------------------------------------------- profiling
const char *const kernel_kind_names[KT_COUNT] = {"datareduct", "keval", "cpqr", "id_solve", "upward", "coupling",
                                                 "downward", "near", "exact_rows", "radix_sort", "lists",
                                                 "fill_blocks", "coupling_stored", "near_stored"};
namespace {
struct Pending {
    int kind;
    cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
double g_prof_ms[KT_COUNT] = {};
long long g_prof_n[KT_COUNT] = {};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void resolve_pending() {  // caller holds the lock
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
            g_prof_ms[p.kind] += ms;
            g_prof_n[p.kind] += 1;
        }
        g_event_pool.push_back(p.e0);
        g_event_pool.push_back(p.e1);
    }
    g_pending.clear();
}
}  // namespace

bool profiling_enabled() { return g_prof_on; }

void profile_set(bool on, bool reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    resolve_pending();
    if (reset)
        for (int k = 0; k < KT_COUNT; k++) { g_prof_ms[k] = 0; g_prof_n[k] = 0; }
    g_prof_on = on;
}

std::string profile_json() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    resolve_pending();
    std::string out = "{";
    char buf[160];
    for (int k = 0; k < KT_COUNT; k++) {
        snprintf(buf, sizeof buf, "%s\"%s\": {\"ms\": %.6f, \"launches\": %lld}", k ? ", " : "", kernel_kind_names[k],
                 g_prof_ms[k], g_prof_n[k]);
        out += buf;
    }
    snprintf(buf, sizeof buf, ", \"launches_total\": %lld", launches_total());
    return out + buf + "}";
}

ProfScope::ProfScope(int k, cudaStream_t st) : kind(k), s(st) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    e0 = take_event();
    cudaEventRecord(e0, s);
}

ProfScope::~ProfScope() {
    if (!e0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e1 = take_event();
    cudaEventRecord(e1, s);
    g_pending.push_back({kind, e0, e1});
}

// ------------------------------------------------------------------- scan
namespace {
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class Tin>
__global__ void k_scan_tile(const Tin *in, int64_t *out, int64_t *bsum, int64_t n) {
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t acc = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        v[i] = (base + i < n) ? (int64_t)in[base + i] : 0;
        acc += v[i];
    }
    // block exclusive scan of per-thread sums
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = acc;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
        int64_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < SCAN_THREADS / 32) wsum[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1 && bsum) bsum[blockIdx.x] = wi;
    }
    __syncthreads();
    int64_t run = wsum[warp] + inc - acc;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

__global__ void k_scan_add(int64_t *out, const int64_t *boff, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += boff[i / SCAN_TILE];
}

template <class Tin>
void scan_impl(const Tin *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        H2_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return;
    }
    if (n <= SCAN_TILE) {  // one tile: its block total is out[n]
        k_scan_tile<Tin><<<1, SCAN_THREADS, 0, s>>>(in, out, out + n, n);
        H2_LAUNCH("k_scan_tile");
        return;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    DevBuf<int64_t> bsum, boff;
    bsum.alloc(nb, s);
    boff.alloc(nb + 1, s);
    k_scan_tile<Tin><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, bsum.p, n);
    H2_LAUNCH("k_scan_tile");
    scan_impl<int64_t>(bsum.p, boff.p, nb, s);  // boff[nb] = total
    k_scan_add<<<blocks_for(n, 256), 256, 0, s>>>(out, boff.p, n);
    H2_LAUNCH("k_scan_add");
    H2_CUDA(cudaMemcpyAsync(out + n, boff.p + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
}
}  // namespace

void scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) { scan_impl<int64_t>(in, out, n, s); }
void scan_exclusive_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    scan_impl<int32_t>(in, out, n, s);
}

// ------------------------------------------------------------- radix sort
namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // keys per block
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void k_radix_hist(const uint64_t *keys, int64_t n, int shift, int32_t *hist, int nblk) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: inside a tile, keys are ranked in (round, warp, lane) order,
// which is their index order; tiles are ordered by the digit-major scan.
__global__ void k_radix_scatter(const uint64_t *kin, const int32_t *vin, uint64_t *kout, int32_t *vout, int64_t n,
                                int shift, const int64_t *offs, int nblk) {
    __shared__ int64_t running[256];
    __shared__ int32_t wcnt[RS_WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    running[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + r * RS_THREADS + tid;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        int digit = valid ? (int)((key >> shift) & 255u) : 256;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) wcnt[w][tid] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        int acc = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            int c = wcnt[w][tid];
            wcnt[w][tid] = acc;
            acc += c;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = running[digit] + wcnt[warp][digit] + rank;
            kout[pos] = key;
            if (vin) vout[pos] = vin[i];
        }
        __syncthreads();
        running[tid] += acc;
        __syncthreads();
    }
}
}  // namespace

void radix_sort(uint64_t *keys, int32_t *vals, int64_t n, int nbits, cudaStream_t s) {
    if (n <= 1 || nbits <= 0) return;
    int passes = (nbits + 7) / 8;
    int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
    DevBuf<uint64_t> k2;
    DevBuf<int32_t> v2;
    DevBuf<int32_t> hist;
    DevBuf<int64_t> offs;
    k2.alloc(n, s);
    if (vals) v2.alloc(n, s);
    hist.alloc((size_t)256 * nblk, s);
    offs.alloc((size_t)256 * nblk + 1, s);
    uint64_t *ka = keys, *kb = k2.p;
    int32_t *va = vals, *vb = v2.p;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        k_radix_hist<<<nblk, RS_THREADS, 0, s>>>(ka, n, shift, hist.p, nblk);
        H2_LAUNCH("k_radix_hist");
        scan_exclusive_i32(hist.p, offs.p, (int64_t)256 * nblk, s);
        k_radix_scatter<<<nblk, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, offs.p, nblk);
        H2_LAUNCH("k_radix_scatter");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        H2_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) H2_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
}

}  // namespace h2

// ------------------------------------------------------- ALU peak probe
namespace h2 {
namespace {
// Each thread runs FP_CHAINS independent multiply-add chains (enough
// instruction-level parallelism to cover the pipe latency); the results are
// stored so that nothing is optimised away.
constexpr int FP_CHAINS = 8;
template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b, T *sink) {
    T x[FP_CHAINS];
#pragma unroll
    for (int c = 0; c < FP_CHAINS; c++) x[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < FP_CHAINS; c++) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < FP_CHAINS; c++) s += x[c];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
double probe_tflops(int sms, int iters, cudaStream_t s) {
    const int ctas = sms * 8, threads = 256;
    DevBuf<T> sink;
    sink.alloc((size_t)ctas * threads, s);
    cudaEvent_t e0, e1;
    H2_CUDA(cudaEventCreate(&e0));
    H2_CUDA(cudaEventCreate(&e1));
    // a: slightly below one, b: small, so the chains stay finite
    k_fma_probe<T><<<ctas, threads, 0, s>>>(iters / 10, (T)0.999999, (T)1e-7, sink.p);  // warm-up
    H2_LAUNCH("k_fma_probe");
    H2_CUDA(cudaEventRecord(e0, s));
    k_fma_probe<T><<<ctas, threads, 0, s>>>(iters, (T)0.999999, (T)1e-7, sink.p);
    H2_LAUNCH("k_fma_probe");
    H2_CUDA(cudaEventRecord(e1, s));
    H2_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * FP_CHAINS * (double)iters * ctas * threads;
    return flops / (ms * 1e-3) / 1e12;
}
}  // namespace

void fma_peaks(double *fp64_tflops, double *fp32_tflops, cudaStream_t s) {
    int dev = 0, sms = 0;
    H2_CUDA(cudaGetDevice(&dev));
    H2_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (fp64_tflops) *fp64_tflops = probe_tflops<double>(sms, 4096, s);
    if (fp32_tflops) *fp32_tflops = probe_tflops<float>(sms, 65536, s);
}
}  // namespace h2
