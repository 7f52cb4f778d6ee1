// df.cuh -- float-float ("double-float") arithmetic on the float32 units: a
// value is the unevaluated sum hi + lo of two float32 numbers (about 48
// significant bits).  Sums by Knuth's TwoSum, products with their exact
// rounding error from a fused multiply-add; every operation explicitly
// rounded (never contracted).  Used where the float64 form's arithmetic would
// otherwise run on this GPU's float64 pipe (1/74 of the float32 rate).
#pragma once

namespace h2 {
namespace df {

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float2 from_double(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ double to_double(float2 x) { return (double)x.x + (double)x.y; }

// the pair (s, e) renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ float2 norm(float s, float e) {
    float h, l;
    two_sum(s, e, h, l);
    return make_float2(h, l);
}

// b * c: hi exact product rounded, lo its error plus the cross terms
__device__ __forceinline__ void mul(float2 b, float2 c, float &ph, float &pl) {
    ph = __fmul_rn(b.x, c.x);
    pl = fmaf(b.x, c.y, fmaf(b.y, c.x, fmaf(b.x, c.x, -ph)));
}

__device__ __forceinline__ float2 mul(float2 b, float2 c) {
    float ph, pl;
    mul(b, c, ph, pl);
    return norm(ph, pl);
}

// a - b * c, renormalised
__device__ __forceinline__ float2 fms(float2 a, float2 b, float2 c) {
    float ph, pl;
    mul(b, c, ph, pl);
    float s, e;
    two_sum(a.x, -ph, s, e);
    return norm(s, __fadd_rn(e, __fsub_rn(a.y, pl)));
}

__device__ __forceinline__ float2 sub(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, -b.x, s, e);
    return norm(s, __fadd_rn(e, __fsub_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

// accumulator (sh, sl) += b * c, left unnormalised (call norm at the end)
__device__ __forceinline__ void mac(float &sh, float &sl, float2 b, float2 c) {
    float ph, pl;
    mul(b, c, ph, pl);
    float s, e;
    two_sum(sh, ph, s, e);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, pl));
}

// sum of a pair over the 32 lanes of a warp (every lane gets it), renormalised
__device__ __forceinline__ float2 warp_sum(float sh, float sl) {
    float2 x = norm(sh, sl);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, x.x, o), ol = __shfl_xor_sync(0xffffffffu, x.y, o);
        x = add(x, make_float2(oh, ol));
    }
    return x;
}

}  // namespace df
}  // namespace h2
