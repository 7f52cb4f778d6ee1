// nbody_tc.cu -- the mixed form's nearfield product for 16 right-hand sides
// on the tensor cores (section 2.1's near term sum_j K(X_i, X_j) W_j, for
// every near leaf pair, with W an n x 16 block of right-hand sides).
//
// For each tile of 128 targets of a leaf i a CTA of 128 threads (one target
// a thread) walks i's near list in chunks of 32 source points: every thread
// evaluates kappa(x_t, x_s) for the chunk's 32 sources in float32 (the
// on-the-fly kernel's arithmetic, sources read as L1 broadcasts) and writes
// them, split as tf32 hi + lo, into the A operand (128 x 32, K-major); the
// chunk's 32 x 16 weights,
// split the same way, form the B operand; one thread issues
//   D_c = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// as 12 tcgen05.mma of kind tf32 (M = 128, N = 16, K = 8) into a float32
// accumulator in tensor memory.  The product's error per term is ~2^-21
// relative (the dropped A_lo B_lo term and the tf32 roundings of the lo
// parts), about float32's.  Two operand buffers and two accumulators
// alternate (an mbarrier each, armed by tcgen05.commit): the threads evaluate
// chunk c while the tensor cores multiply chunk c - 1, and chunk c - 2's
// accumulator is read back (tcgen05.ld) and folded into a compensated float32
// sum per target and column before its buffer is refilled, so no tensor-core
// accumulation runs over more than 32 sources.
#include <mutex>

#include "h2_internal.cuh"
#include "kappa_fast.cuh"
#include "tc_sm103.cuh"

namespace h2 {
namespace {

constexpr int TC_M = 128;  // targets per tile (tensor-memory lanes)
constexpr int TC_K = 32;   // sources per chunk
constexpr int TC_N = 16;   // right-hand sides
// operand layouts (K-major, no swizzle, 8-row x 16-byte core matrices):
//   A (128 x 32 floats): byte (k / 4) * 2048 + r * 16 + (k % 4) * 4
//   B (16 x 32 floats):  byte (k / 4) * 256 + n * 16 + (k % 4) * 4
// so the core matrices adjacent along K are 2048 (A) / 256 (B) bytes apart
// and those adjacent along M / N 128 bytes apart
constexpr uint32_t A_BYTES = TC_M * TC_K * 4, B_BYTES = TC_N * TC_K * 4;
constexpr uint32_t A_LBO = 2048, B_LBO = 256, MN_SBO = 128;
// one buffer: A hi, A lo, B hi, B lo
constexpr uint32_t BUF_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr uint32_t TC_SMEM = 2 * BUF_BYTES + 128;  // two buffers and alignment slack: three CTAs a SM
constexpr uint32_t WAIT_LIMIT = 1u << 17;           // mbarrier polls (of up to ~10 us) before a wait gives up

__device__ __forceinline__ void two_sum_acc(float &a, float &e, float b) {
    const float s = a + b, bp = s - a;
    e += (a - (s - bp)) + (b - bp);
    a = s;
}

constexpr int GEN_WARPS = TC_M / 32;               // generator warps: one target row a lane
constexpr int TC_THREADS = (GEN_WARPS + 1) * 32;    // and one warp that issues the products

template <int KID>
__global__ void __launch_bounds__(TC_THREADS, 3) k_nbody_tc(const int2 *tiles, const int64_t *start,
                                                            const int32_t *count, const float *X0, const float *X1,
                                                            const float *X2, const float2 *F0, const float2 *F1,
                                                            const float2 *F2, const float *w, int ws, double *out,
                                                            int os, const int64_t *lptr, const int32_t *lidx, int d,
                                                            double kpar, int *status) {
    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned operand buffers
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    // full[b]: the four generator warps have written buffer b's operands;
    // empty[b]: the products of the last chunk that used buffer b (and
    // accumulator b) are complete
    __shared__ uint64_t full[2], empty[2];
    __shared__ float4 stg[GEN_WARPS][TC_K];  // each generator warp's copy of the chunk's sources
    __shared__ uint32_t tmem_slot;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int2 tl = tiles[blockIdx.x];
    const int i = tl.x;
    const int64_t ts = start[i];
    const int tn = count[i];
    if (t == 0) {
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&full[b], GEN_WARPS);
            tc::mbar_init(&empty[b], 1);
        }
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 32);  // two accumulators of 16 columns
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int64_t e0 = lptr[i], e1 = lptr[i + 1];
    bool failed = false;
    if (warp == GEN_WARPS) {
        // the issuing warp: one lane issues 12 tf32 products per chunk into
        // accumulator gc % 2 once the chunk's operands are written
        if (lane == 0) {
            constexpr uint32_t IDESC = tc::idesc_tf32(TC_M, TC_N);
            const uint32_t abase = tc::smem_u32(base);
            uint32_t ph = 0;
            int gc = 0;
            for (int64_t e = e0; e < e1 && !failed; e++) {
                const int sn = count[lidx[e]];
                for (int q0 = 0; q0 < sn; q0 += TC_K) {
                    const int buf = gc & 1;
                    if (!tc::mbar_wait(&full[buf], (ph >> buf) & 1u, WAIT_LIMIT)) { failed = true; break; }
                    ph ^= 1u << buf;
                    tc::fence_after_sync();
                    const uint32_t ah = abase + buf * BUF_BYTES, al = ah + A_BYTES, bh = ah + 2 * A_BYTES,
                                   bl = bh + B_BYTES;
                    const uint32_t dt = tmem + (uint32_t)(buf * TC_N);
#pragma unroll
                    for (int st = 0; st < TC_K / 8; st++) {  // K = 8 per instruction: two core matrices along K
                        const uint32_t ao = st * 2 * A_LBO, bo = st * 2 * B_LBO;
                        tc::mma_tf32(dt, tc::smem_desc(ah + ao, A_LBO, MN_SBO),
                                     tc::smem_desc(bh + bo, B_LBO, MN_SBO), IDESC, st != 0);
                        tc::mma_tf32(dt, tc::smem_desc(ah + ao, A_LBO, MN_SBO),
                                     tc::smem_desc(bl + bo, B_LBO, MN_SBO), IDESC, true);
                        tc::mma_tf32(dt, tc::smem_desc(al + ao, A_LBO, MN_SBO),
                                     tc::smem_desc(bh + bo, B_LBO, MN_SBO), IDESC, true);
                    }
                    tc::commit(&empty[buf]);
                    gc++;
                }
            }
            if (failed) atomicExch(status, 1);
        }
        __syncwarp();
    } else {
        // a generator warp: rows 32 warp .. 32 warp + 31 of the tile
        const int a = tl.y + t;
        const bool act = a < tn;
        const float p = (float)kpar;
        const float tx0 = act ? X0[ts + a] : 0.f, tx1 = act && d > 1 ? X1[ts + a] : 0.f,
                    tx2 = act && d > 2 ? X2[ts + a] : 0.f;
        const uint32_t tmem_lane = tmem + ((uint32_t)(warp * 32) << 16);
        float acc[TC_N], cmp[TC_N];
#pragma unroll
        for (int n = 0; n < TC_N; n++) { acc[n] = 0.f; cmp[n] = 0.f; }
        uint32_t ph = 0;
        int gc = 0;
        // wait for chunk gc - 2's products (buffer and accumulator b) and fold
        // this warp's rows of its sums
        auto retire = [&](int b) -> bool {
            const bool ok = tc::mbar_wait(&empty[b], (ph >> b) & 1u, WAIT_LIMIT);
            ph ^= 1u << b;
            if (__any_sync(0xffffffffu, !ok)) return false;  // (the collective load runs in all lanes or none)
            tc::fence_after_sync();
            float v[TC_N];
            tc::tmem_ld16(tmem_lane + (uint32_t)(b * TC_N), v);
#pragma unroll
            for (int n = 0; n < TC_N; n++) two_sum_acc(acc[n], cmp[n], v[n]);
            return true;
        };
        for (int64_t e = e0; e < e1 && !failed; e++) {
            const int jn = lidx[e];
            const int64_t ss = start[jn];
            const int sn = count[jn];
            float o0 = 0.f, o1 = 0.f, o2 = 0.f;  // target coordinates in node jn's frame
            {
                const float2 a0 = F0[i], b0 = F0[jn];
                o0 = (a0.x - b0.x) + (a0.y - b0.y);
                if (d > 1) {
                    const float2 a1 = F1[i], b1 = F1[jn];
                    o1 = (a1.x - b1.x) + (a1.y - b1.y);
                }
                if (d > 2) {
                    const float2 a2 = F2[i], b2 = F2[jn];
                    o2 = (a2.x - b2.x) + (a2.y - b2.y);
                }
            }
            const float s0 = tx0 + o0, s1 = tx1 + o1, s2 = tx2 + o2;
            for (int q0 = 0; q0 < sn; q0 += TC_K) {
                const int buf = gc & 1;
                if (gc >= 2 && !retire(buf)) { failed = true; break; }
                unsigned char *bb = base + buf * BUF_BYTES;
                float *Ah = reinterpret_cast<float *>(bb), *Al = reinterpret_cast<float *>(bb + A_BYTES);
                const int cnt = min(TC_K, sn - q0);
                const int64_t sb = ss + q0;
                // this warp's copy of the chunk's sources
                stg[warp][lane] = lane < cnt ? make_float4(X0[sb + lane], d > 1 ? X1[sb + lane] : 0.f,
                                                           d > 2 ? X2[sb + lane] : 0.f, 0.f)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                if (warp == 0) {
                    // the chunk's weights, split (padding sources: 0).  Source group
                    // g (sources 4g .. 4g + 3) fills 256 contiguous bytes, column n
                    // at 16 n; lane l writes column l / 2, sources 4g + 2 (l % 2) + {0, 1}
                    // (8 bytes a lane, no bank conflicts)
                    float *Bh = reinterpret_cast<float *>(bb + 2 * A_BYTES), *Bl = Bh + B_BYTES / 4;
                    const int n = lane >> 1, qq = (lane & 1) * 2;
#pragma unroll
                    for (int g = 0; g < TC_K / 4; g++) {
                        const int q = 4 * g + qq;
                        const float v0 = q < cnt ? w[(sb + q) * (int64_t)ws + n] : 0.f;
                        const float v1 = q + 1 < cnt ? w[(sb + q + 1) * (int64_t)ws + n] : 0.f;
                        const float h0 = tc::tf32_hi(v0), h1 = tc::tf32_hi(v1);
                        const uint32_t off = (uint32_t)(g * 256 + n * 16 + qq * 4) >> 2;
                        *reinterpret_cast<float2 *>(Bh + off) = make_float2(h0, h1);
                        *reinterpret_cast<float2 *>(Bl + off) = make_float2(tc::tf32_hi(v0 - h0), tc::tf32_hi(v1 - h1));
                    }
                }
                __syncwarp();
                // kappa for this lane's target and the chunk's sources, four at a time
                // (padding sources and padding targets: 0)
#pragma unroll 2
                for (int q = 0; q < TC_K; q += 4) {
                    float hp[4], lp[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const float4 sv = stg[warp][q + u];
                        const float kv = act && q + u < cnt ? kap_pt<KID, false>(s0, s1, s2, sv.x, sv.y, sv.z, p)
                                                            : 0.f;
                        const float hi = tc::tf32_hi(kv);
                        hp[u] = hi;
                        lp[u] = tc::tf32_hi(kv - hi);
                    }
                    const uint32_t off = (uint32_t)((q >> 2) * 2048 + t * 16) >> 2;
                    *reinterpret_cast<float4 *>(Ah + off) = make_float4(hp[0], hp[1], hp[2], hp[3]);
                    *reinterpret_cast<float4 *>(Al + off) = make_float4(lp[0], lp[1], lp[2], lp[3]);
                }
                tc::fence_async_smem();
                tc::fence_before_sync();  // (this warp's reads of the accumulator precede the arrival)
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&full[buf]);
                gc++;
            }
        }
        // the last two chunks
        for (int c = max(0, gc - 2); c < gc && !failed; c++)
            if (!retire(c & 1)) failed = true;
        if (failed) {
            if (lane == 0) atomicExch(status, 1);
        } else if (act) {
            double *o = out + (ts + a) * (int64_t)os;
#pragma unroll
            for (int n = 0; n < TC_N; n++) o[n] += (double)acc[n] + (double)cmp[n];
        }
    }
    // teardown: products still in flight after a failure get a bounded wait
    // (the commit arms empty[0] once every issued product has completed)
    __syncthreads();
    if (t == GEN_WARPS * 32) {
        int st = 0;
        if (status) st = *(volatile int *)status;
        if (st) {
            tc::commit(&empty[0]);
            // (the phase parity is unknown after a failure: poll both)
            for (uint32_t it = 0; it < WAIT_LIMIT; it++)
                if (tc::mbar_wait(&empty[0], 0, 1) || tc::mbar_wait(&empty[0], 1, 1)) break;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_free(tmem, 32);
}

}  // namespace

// out[:, 0:16] (row stride os) += near products of the 16 float32 weight
// columns w[:, 0:16] (row stride ws); tiles of 128 targets; *status (device)
// becomes 1 if a tensor-core wait gave up
void nbody_tc16(int kid, const DevBuf<int2> &tiles, const int64_t *start, const int32_t *count, const float *X0,
                const float *X1, const float *X2, const float2 *F0, const float2 *F1, const float2 *F2,
                const float *w, int ws, double *out, int os, const int64_t *lptr, const int32_t *lidx, int d,
                double kp0, int *status, cudaStream_t s) {
    if (tiles.n == 0) return;
    static std::once_flag attr;
    std::call_once(attr, [] {
        for (const void *f : {(const void *)k_nbody_tc<H2_K_COULOMB>, (const void *)k_nbody_tc<H2_K_GAUSSIAN>,
                              (const void *)k_nbody_tc<H2_K_EXPONENTIAL>, (const void *)k_nbody_tc<H2_K_BUMP>,
                              (const void *)k_nbody_tc<H2_K_POWER>, (const void *)k_nbody_tc<H2_K_COSDOT>,
                              (const void *)k_nbody_tc<H2_K_MULTIQUADRIC>})
            H2_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    });
    const unsigned nb = (unsigned)tiles.n;
    const double p = kap_param(kid, kp0);
#define H2_TC(K)                                                                                              \
    k_nbody_tc<K><<<nb, TC_THREADS, TC_SMEM, s>>>(tiles.p, start, count, X0, X1, X2, F0, F1, F2, w, ws, out, os, lptr, \
                                            lidx, d, p, status)
    switch (kid) {
    case H2_K_COULOMB: H2_TC(H2_K_COULOMB); break;
    case H2_K_GAUSSIAN: H2_TC(H2_K_GAUSSIAN); break;
    case H2_K_EXPONENTIAL: H2_TC(H2_K_EXPONENTIAL); break;
    case H2_K_BUMP: H2_TC(H2_K_BUMP); break;
    case H2_K_POWER: H2_TC(H2_K_POWER); break;
    case H2_K_COSDOT: H2_TC(H2_K_COSDOT); break;
    default: H2_TC(H2_K_MULTIQUADRIC);
    }
#undef H2_TC
    H2_LAUNCH("k_nbody_tc");
}

}  // namespace h2
