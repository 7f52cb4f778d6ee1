// kappa_fast.cuh -- the kernel functions as the matvec evaluates them: fast
// forms (rsqrt, exp) in float64 or float32, shared by the on-the-fly N-body
// kernels and the fill of stored coupling and nearfield blocks, so that a
// stored block holds exactly the values the on-the-fly product would use.
#pragma once

#include <cfloat>

#include "h2_internal.cuh"

namespace h2 {
namespace {

// kappa for the matvec kernels: fast forms (rsqrt, exp) in float64 or float32
// (p: 1/h^2 Gaussian, 1/l exponential, a bump, p/2 power; see kap_param)
template <int KID>
__device__ __forceinline__ double kap(double r2, double p) {
    if constexpr (KID == H2_K_COULOMB) return h2_rsqrt64(r2);
    else if constexpr (KID == H2_K_GAUSSIAN) return exp(-r2 * p);
    else if constexpr (KID == H2_K_EXPONENTIAL) return exp(-sqrt(r2) * p);
    else if constexpr (KID == H2_K_BUMP) {
        const double t = r2 * p;
        return t < 1.0 ? exp(-1.0 / (1.0 - t)) : 0.0;
    } else if constexpr (KID == H2_K_POWER) {  // (kept finite: the symmetric kernel's padding has weight 0)
        return r2 > 0.0 ? fmin(pow(r2, p), DBL_MAX) : 0.0;
    } else return sqrt(1.0 + r2);
}
template <int KID>
__device__ __forceinline__ float kap(float r2, float p) {
    if constexpr (KID == H2_K_COULOMB) {
        float y;
        asm("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(r2));  // relative error below 2^-22
        return r2 > 0.0f ? y : 0.0f;
    }
    else if constexpr (KID == H2_K_GAUSSIAN) return __expf(-r2 * p);
    else if constexpr (KID == H2_K_EXPONENTIAL) return __expf(-sqrtf(r2) * p);
    else if constexpr (KID == H2_K_BUMP) {
        const float t = r2 * p;
        return t < 1.0f ? __expf(__fdividef(-1.0f, 1.0f - t)) : 0.0f;
    } else if constexpr (KID == H2_K_POWER) {  // (kept finite, as above)
        return r2 > 0.0f ? fminf(__powf(r2, p), FLT_MAX) : 0.0f;
    } else return sqrtf(1.0f + r2);
}
// the kernel parameter in the form kap takes
inline double kap_param(int kid, double kp0) { return h2_kappa_param(kid, kp0); }
// kappa for point pairs known to be distinct (r2 > 0): Coulomb skips the
// r2 = 0 test
template <int KID, class Real>
__device__ __forceinline__ Real kap_distinct(Real r2, Real p) {
    if constexpr (KID == H2_K_COULOMB && sizeof(Real) == 4) {
        float y;
        asm("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(r2));
        return y;
    } else {
        return kap<KID>(r2, p);
    }
}

// kappa of a target t and a source s: cos(t . s) for Table 1's kappa_3 (both
// in absolute coordinates), every other kernel from |t - s|^2 (DISTINCT: the
// points are known to differ)
template <int KID, bool DISTINCT, class Real>
__device__ __forceinline__ Real kap_pt(Real t0, Real t1, Real t2, Real s0, Real s1, Real s2, Real p) {
    if constexpr (KID == H2_K_COSDOT) {
        const Real x = t0 * s0 + t1 * s1 + t2 * s2;
        if constexpr (sizeof(Real) == 4) return __cosf(x);
        else return cos(x);
    } else {
        const Real dx = t0 - s0, dy = t1 - s1, dz = t2 - s2;
        if constexpr (DISTINCT) return kap_distinct<KID>(dx * dx + dy * dy + dz * dz, p);
        else return kap<KID>(dx * dx + dy * dy + dz * dz, p);
    }
}


}  // namespace
}  // namespace h2
