// ff.cuh -- float-float ("double-float") arithmetic: a value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48 significant
// bits.  GB300 issues FP32 at about 74 times its FP64 rate, so the FP64-mode
// moves evaluate the bilinear sizing field and the per-thread sums this way and
// keep FP64 instructions for the few operations that need all 53 bits
// (differences of nearby positions, the spring lengths).
//
// The error-free transformations are the classical ones: Knuth's TwoSum,
// Dekker's FastTwoSum (|a| >= |b|) and the FMA-based TwoProduct.  Every
// addition and product is written with an explicit round-to-nearest
// intrinsic so the compiler cannot contract a product into a later sum
// (which would break the transformations).
#pragma once
#include "common.cuh"

namespace trime {

struct ff {
    float h, l;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.h, b.h), t = two_sum(a.l, b.l);
    ff u = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(u.h, __fadd_rn(u.l, t.l));
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.h, b);
    return fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    float p = __fmul_rn(a.h, b);
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return fast_two_sum(p, e);
}

// a / b: a float quotient and one correction from the float-float remainder
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    float rb = __frcp_rn(b.h);
    float q1 = __fmul_rn(a.h, rb);
    ff r = ff_sub(a, ff_mul_f(b, q1));
    float q2 = __fmul_rn(r.h, rb);
    ff q = fast_two_sum(q1, q2);
    r = ff_sub(a, ff_mul(b, q));
    return ff_add_f(q, __fmul_rn(r.h, rb));
}

__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

__device__ __forceinline__ ff ff_scale2(ff a, float p2) { return {__fmul_rn(a.h, p2), __fmul_rn(a.l, p2)}; }

__device__ __forceinline__ ff ff_from_d(double d) {
    float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.h + (double)a.l; }

// a - b for values held exactly as three floats (h + l + t); the result
// rounded once to float-float
__device__ __forceinline__ ff ff_diff3(float ah, float al, float at, float bh, float bl, float bt) {
    ff s = two_sum(ah, -bh), t = two_sum(al, -bl);
    return ff_add_f(ff_add(s, t), __fsub_rn(at, bt));
}

// 1 / sqrt(a), a > 0: float estimate and two Newton corrections in float-float
__device__ __forceinline__ ff ff_rsqrt(ff a) {
    float r0 = rsqrtf(a.h);
    ff r{r0, 0.f};
#pragma unroll
    for (int k = 0; k < 2; k++) {
        ff e = ff_add_f(ff_neg(ff_mul(a, ff_mul(r, r))), 1.0f);  // 1 - a r^2, small
        r = ff_add_f(r, __fmul_rn(__fmul_rn(0.5f, r.h), e.h));
    }
    return r;
}

__device__ __forceinline__ bool ff_lt0(ff a) { return a.h < 0.f || (a.h == 0.f && a.l < 0.f); }
__device__ __forceinline__ bool ff_ge1(ff a) { return a.h > 1.f || (a.h == 1.f && a.l >= 0.f); }

__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
    return {__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}
__device__ __forceinline__ ff warp_sum_ff(ff a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = ff_add(a, ff_shfl_xor(a, o));
    return a;
}

// Grid coordinate t (in cells) -> cell index in [0, imax] and the fraction in
// [0, 1]: the cell that holds t exactly (t.h an integer with t.l < 0 belongs
// to the cell below), clamped like the FP64 lookup.
__device__ __forceinline__ ff cell_frac(ff t, int imax, int& i) {
    float fi = floorf(t.h);
    int k = fi < 0.f ? 0 : (fi > (float)imax ? imax : (int)fi);
    ff f = ff_add_f(t, -(float)k);
    if (ff_lt0(f) && k > 0) {
        k--;
        f = ff_add_f(f, 1.f);
    } else if (ff_ge1(f) && k < imax) {
        k++;
        f = ff_add_f(f, -1.f);
    }
    if (ff_lt0(f)) f = {0.f, 0.f};
    if (ff_ge1(f)) f = {1.f, 0.f};
    i = k;
    return f;
}

// Bilinear interpolation of a grid at (x, y) in float-float: the same
// formula as the FP64 lookup, a = v00 + fx (v10 - v00), b = v01 + fx (v11 - v01),
// value a + fy (b - a), with the node differences exact; relative error a few
// units of 2^-46 of the values involved.
__device__ __forceinline__ ff bilin_ff(const DevGrid& g, ff x, ff y) {
    ff tx = ff_mul(ff_sub(x, ff{g.fx0h, g.fx0l}), ff{g.fidxh, g.fidxl});
    ff ty = ff_mul(ff_sub(y, ff{g.fy0h, g.fy0l}), ff{g.fidyh, g.fidyl});
    int i, j;
    ff fx = cell_frac(tx, g.nx - 2, i), fy = cell_frac(ty, g.ny - 2, j);
    const float* r0 = g.v + (size_t)j * g.nx + i;
    const float* r1 = r0 + g.nx;
    float v00 = __ldg(r0), v10 = __ldg(r0 + 1), v01 = __ldg(r1), v11 = __ldg(r1 + 1);
    ff a = ff_add_f(ff_mul(fx, two_sum(v10, -v00)), v00);
    ff b = ff_add_f(ff_mul(fx, two_sum(v11, -v01)), v01);
    return ff_add(a, ff_mul(fy, ff_sub(b, a)));
}

}  // namespace trime
