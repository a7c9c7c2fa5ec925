// h3d_ff.cuh -- float-float ("double-single") arithmetic on the FP32 pipes, and
// kernel entries K(p_i, p_j) evaluated with it.
//
// A float-float value is an unevaluated sum h + l of two FP32 numbers.  The
// building blocks are the classic error-free transformations: Knuth's TwoSum
// (a + b = s + e exactly, any a, b), and the product a * b = p + e exactly,
// with e obtained by one fused multiply-add, fma(a, b, -p).  Every operation
// below uses explicitly rounded FP32 intrinsics, so the compiler can neither
// contract nor reorder them.
//
// Why: GB300 runs FP64 at about 1/64 of its FP32 rate.  The skeleton form of
// the admissible blocks (Sec. 4.1, Eq. prank) recomputes K(sigma,Y) and
// K(X,tau) in every product; FP32 entries (relative error ~1e-7) are too coarse
// for it, but entries good to ~1e-12 change the product by far less than the
// ACA tolerance, and float-float reaches that at a few dozen FP32 operations
// per entry.  Coordinates enter as float-float offsets from the centre of the
// domain cube (the FP64 coordinate to within 2^-48 of its magnitude), so the
// difference of two points is exact up to that representation error even when
// the points are close (vertex-sharing blocks).
#pragma once

#include <cuda_runtime.h>

namespace h3d {

struct FF {
    float h, l;
};

// s + e = a + b exactly (Knuth's TwoSum, six operations, no ordering condition)
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return FF{s, e};
}

// p + e = a * b exactly
__device__ __forceinline__ FF ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return FF{p, __fmaf_rn(a, b, -p)};
}

// Squared distance of two points given as float-float coordinates (hi.xyz,
// lo.xyz): per axis the difference of the high parts exactly (TwoSum) plus the
// low parts' difference, squared as s^2 + (2 s t + t^2); the three squares are
// summed with TwoSum.  Result unnormalised (|l| far below |h|).
__device__ __forceinline__ FF ff_dist2(float4 hi, float4 lo, float4 hj, float4 lj) {
    FF sq[3];
    const float ah[3] = {hi.x, hi.y, hi.z}, al[3] = {lo.x, lo.y, lo.z};
    const float bh[3] = {hj.x, hj.y, hj.z}, bl[3] = {lj.x, lj.y, lj.z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const FF s = ff_two_sum(ah[d], -bh[d]);
        const float t = __fadd_rn(s.l, __fsub_rn(al[d], bl[d]));
        const FF p = ff_two_prod(s.h, s.h);
        sq[d] = FF{p.h, __fadd_rn(p.l, __fmaf_rn(__fmul_rn(2.0f, s.h), t, __fmul_rn(t, t)))};
    }
    const FF a = ff_two_sum(sq[0].h, sq[1].h);
    const FF b = ff_two_sum(a.h, sq[2].h);
    return FF{b.h, __fadd_rn(__fadd_rn(a.l, b.l), __fadd_rn(__fadd_rn(sq[0].l, sq[1].l), sq[2].l))};
}

// 1 / sqrt(d2): an FP32 seed y0, then one Newton step whose residual
// 1 - d2 y0^2 is formed in float-float; the result y0 (1 + h/2) has a relative
// error of about (3/2) (seed error)^2 plus float-float rounding, ~1e-13.
__device__ __forceinline__ FF ff_rsqrt(FF d2) {
    const float y0 = rsqrtf(d2.h);
    const FF y2 = ff_two_prod(y0, y0);
    FF t = ff_two_prod(d2.h, y2.h);
    t.l = __fmaf_rn(d2.h, y2.l, __fmaf_rn(d2.l, y2.h, t.l));
    const float h = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);
    return FF{y0, __fmul_rn(__fmul_rn(0.5f, y0), h)};
}

// a * b for float-float a, b (the l * l term dropped: below 2^-46 |a b|)
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    FF p = ff_two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return p;
}

// 1 / (4 pi) as a float-float constant (h + l within 4e-17 of the value)
__device__ __forceinline__ FF ff_inv4pi() { return FF{0x1.45f306p-4f, 0x1.b93910p-29f}; }

// Kernel entries that float-float evaluates: Laplace 1/(4 pi r) and 1/r^4.
__host__ __device__ inline bool ff_kernel_supported(int kind) { return kind == 0 || kind == 2; }

// K(p_i, p_j), 0 for coincident points (points that agree to the 2^-48 of the
// representation count as coincident); kind is H3D_LAPLACE or H3D_INV_R4
__device__ __forceinline__ FF ff_kernel(int kind, float4 hi, float4 lo, float4 hj, float4 lj) {
    const FF d2 = ff_dist2(hi, lo, hj, lj);
    if (d2.h == 0.0f) return FF{0.0f, 0.0f};
    const FF y = ff_rsqrt(d2);
    if (kind == 2) {
        const FF y2 = ff_mul(y, y);
        return ff_mul(y2, y2);
    }
    return ff_mul(ff_inv4pi(), y);
}

// K(p_i, p_j), f'(rho) / rho and the difference p_i - p_j, all float-float, for
// the gradient dK/dp_i = (f'(rho) / rho) (p_i - p_j); 0 for coincident points
__device__ __forceinline__ void ff_kernel_grad(int kind, float4 hi, float4 lo, float4 hj, float4 lj, FF &f, FF &fr,
                                               FF (&d)[3]) {
    const float ah[3] = {hi.x, hi.y, hi.z}, al[3] = {lo.x, lo.y, lo.z};
    const float bh[3] = {hj.x, hj.y, hj.z}, bl[3] = {lj.x, lj.y, lj.z};
    FF sq[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const FF s = ff_two_sum(ah[a], -bh[a]);
        const float t = __fadd_rn(s.l, __fsub_rn(al[a], bl[a]));
        d[a] = FF{s.h, t};
        const FF p = ff_two_prod(s.h, s.h);
        sq[a] = FF{p.h, __fadd_rn(p.l, __fmaf_rn(__fmul_rn(2.0f, s.h), t, __fmul_rn(t, t)))};
    }
    const FF u = ff_two_sum(sq[0].h, sq[1].h);
    const FF v = ff_two_sum(u.h, sq[2].h);
    const FF d2{v.h, __fadd_rn(__fadd_rn(u.l, v.l), __fadd_rn(__fadd_rn(sq[0].l, sq[1].l), sq[2].l))};
    if (d2.h == 0.0f) {
        f = fr = FF{0.f, 0.f};
        return;
    }
    const FF y = ff_rsqrt(d2), y2 = ff_mul(y, y);
    if (kind == 2) {   // 1/r^4: f' / r = -4 / r^6
        f = ff_mul(y2, y2);
        const FF g = ff_mul(f, y2);
        fr = FF{__fmul_rn(-4.0f, g.h), __fmul_rn(-4.0f, g.l)};
    } else {           // 1/(4 pi r): f' / r = -f / r^2
        f = ff_mul(ff_inv4pi(), y);
        const FF g = ff_mul(f, y2);
        fr = FF{-g.h, -g.l};
    }
}

// acc + k * x for an FP32 x (exact product, then TwoSum of the high parts)
__device__ __forceinline__ FF ff_fma_acc(FF acc, FF k, float x) {
    FF p = ff_two_prod(k.h, x);
    p.l = __fmaf_rn(k.l, x, p.l);
    const FF s = ff_two_sum(acc.h, p.h);
    return FF{s.h, __fadd_rn(acc.l, __fadd_rn(s.l, p.l))};
}

// acc + k * c for a float-float coefficient c
__device__ __forceinline__ FF ff_fma_acc(FF acc, FF k, FF c) {
    const FF p = ff_mul(k, c);
    const FF s = ff_two_sum(acc.h, p.h);
    return FF{s.h, __fadd_rn(acc.l, __fadd_rn(s.l, p.l))};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.h + (double)a.l; }

// sum over the 32 lanes of a warp in float-float (TwoSum of the high parts at
// each butterfly step): FP64 additions run at 1/64 of the FP32 rate on GB300,
// so a warp sum of doubles costs more than the float-float entries it sums.
// Every lane receives a sum (the lanes' roundings may differ in the last bits).
__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, v.h, o), ol = __shfl_xor_sync(0xffffffffu, v.l, o);
        const FF s = ff_two_sum(v.h, oh);
        v = FF{s.h, __fadd_rn(__fadd_rn(v.l, ol), s.l)};
    }
    return v;
}

__device__ __forceinline__ FF ff_from_double(double v) {
    const float h = (float)v;
    return FF{h, (float)(v - (double)h)};
}

}  // namespace h3d
