// The spatial operator of the modelling scheme, shared by every kernel that
// evaluates it: the order-2R Laplacian (section "Testing approach": 4th/8th
// order in space) of the four points of one float4 column group.
//
// Per axis the operator is (1/h^2) [c_0 u + sum_m c_m (u_{+m} + u_{-m})].  For
// a wavefield of wavenumber k it cancels to a value of order (k h)^2 |u|, so a
// rounding of any term of size |u| costs about (sum_m |c_m|) / (k h)^2 units in
// the last place of the result; summed as written in FP32 that cancellation
// alone gives ~5e-5 relative trace error after 1414 steps at 6 Hz on a 20 m
// grid, and ~2e-4 after 3768 steps at 12 Hz on a 10 m grid.  Here the m = 1
// and m = 2 terms, which carry almost all of the weight, are taken as
// differences from the centre, c_m ((u_{+m} - u) + (u_{-m} - u)), and only the
// small remainder (c_0 + 2 c_1 + 2 c_2) u of the centre weight is added (zero
// for orders 2 and 4): the same operator in exact arithmetic, with the FP32
// rounding of the traces 30-70 times smaller.  Along x the m = 1 differences
// come from the forward differences e_j = u_{j+1} - u_j of the row
// (u_{i+1} - 2 u_i + u_{i-1} = e_i - e_{i-1}).
#pragma once

#include "internal.cuh"

namespace empso {

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 neg2(const float2 &v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// float4 groups of x-neighbours each side that an order-2R stencil reads
template <int R> struct XGroups {
    static constexpr int G = (R + 3) / 4;
};

// Laplacian of one group.  w[0 .. 2R]: the group in rows k - R .. k + R (w[R]
// is the group itself); xs[0 .. 4 (2G + 1) - 1]: the row's values from lane
// -4G to lane 3 + 4G (xs[4G + i] = u_i of this group's lanes i = 0..3).
// cx[m], cz[m] (m = 1..R): c_m / hx^2, c_m / hz^2; cres: the remaining centre
// weight (c_0 + 2 c_1 + 2 c_2)(1/hx^2 + 1/hz^2).  Returns lanes (0,1), (2,3).
template <int R>
__device__ __forceinline__ void lap_group(const float4 *w, const float *xs, const float *cx,
                                          const float *cz, float cres, float2 &l01, float2 &l23)
{
    constexpr int O = 4 * XGroups<R>::G;
    const float2 c01 = lo2(w[R]), c23 = hi2(w[R]);
    const float2 m1 = splat2(-1.f);
    // v - c as one fused operation (-c + v, rounded once): no separate negation
    auto dif = [&](const float2 &v, const float2 &c) { return __ffma2_rn(c, m1, v); };
    // z: m = 1 (and 2) as differences from the centre, then plain pair sums
    float2 z01 = __fmul2_rn(splat2(cz[1]), __fadd2_rn(dif(lo2(w[R - 1]), c01), dif(lo2(w[R + 1]), c01)));
    float2 z23 = __fmul2_rn(splat2(cz[1]), __fadd2_rn(dif(hi2(w[R - 1]), c23), dif(hi2(w[R + 1]), c23)));
    if (R >= 2) {
        z01 = __ffma2_rn(splat2(cz[2]), __fadd2_rn(dif(lo2(w[R - 2]), c01), dif(lo2(w[R + 2]), c01)), z01);
        z23 = __ffma2_rn(splat2(cz[2]), __fadd2_rn(dif(hi2(w[R - 2]), c23), dif(hi2(w[R + 2]), c23)), z23);
    }
#pragma unroll
    for (int m = 3; m <= R; ++m) {
        z01 = __ffma2_rn(splat2(cz[m]), __fadd2_rn(lo2(w[R - m]), lo2(w[R + m])), z01);
        z23 = __ffma2_rn(splat2(cz[m]), __fadd2_rn(hi2(w[R - m]), hi2(w[R + m])), z23);
    }
    // x: m = 1 from forward differences e_j = u_{j+1} - u_j, j = -1 .. 3
    float e[5];
#pragma unroll
    for (int j = -1; j <= 3; ++j) e[j + 1] = xs[O + j + 1] - xs[O + j];
    float2 x01 = __fmul2_rn(splat2(cx[1]), f2(e[1] - e[0], e[2] - e[1]));
    float2 x23 = __fmul2_rn(splat2(cx[1]), f2(e[3] - e[2], e[4] - e[3]));
    if (R >= 2) {   // m = 2: the pairs line up with the register pairs
        x01 = __ffma2_rn(splat2(cx[2]), __fadd2_rn(dif(f2(xs[O + 2], xs[O + 3]), c01),
                                                   dif(f2(xs[O - 2], xs[O - 1]), c01)), x01);
        x23 = __ffma2_rn(splat2(cx[2]), __fadd2_rn(dif(f2(xs[O + 4], xs[O + 5]), c23),
                                                   dif(f2(xs[O + 0], xs[O + 1]), c23)), x23);
    }
#pragma unroll
    for (int m = 3; m <= R; ++m) {
        const float2 s01 = (m & 1) ? f2(xs[O - m] + xs[O + m], xs[O + 1 - m] + xs[O + 1 + m])
                                   : __fadd2_rn(f2(xs[O - m], xs[O + 1 - m]), f2(xs[O + m], xs[O + 1 + m]));
        const float2 s23 = (m & 1) ? f2(xs[O + 2 - m] + xs[O + 2 + m], xs[O + 3 - m] + xs[O + 3 + m])
                                   : __fadd2_rn(f2(xs[O + 2 - m], xs[O + 3 - m]),
                                                f2(xs[O + 2 + m], xs[O + 3 + m]));
        x01 = __ffma2_rn(splat2(cx[m]), s01, x01);
        x23 = __ffma2_rn(splat2(cx[m]), s23, x23);
    }
    if (R >= 3) {   // the centre weight left over (zero for R <= 2)
        x01 = __ffma2_rn(splat2(cres), c01, x01);
        x23 = __ffma2_rn(splat2(cres), c23, x23);
    }
    l01 = __fadd2_rn(x01, z01);
    l23 = __fadd2_rn(x23, z23);
}

// lap_group for a thread that sweeps a run of rows: the z-differences from
// the centre are carried from row to row instead of formed twice.  With
// d_k = u_{k+1} - u_k and e_k = u_{k+2} - u_k (one rounding each, as dif
// forms them), the m = 1 and m = 2 pair sums are d_k - d_{k-1} and
// e_k - e_{k-2}: the same rounded operands as lap_group's
// (u_{k-1} - u_k) + (u_{k+1} - u_k) and (u_{k-2} - u_k) + (u_{k+2} - u_k),
// added in the other order, so the result is bit for bit lap_group's, with two
// packed operations fewer per pair.  dm = d_{k-1}, em = e_{k-2} in; dk = d_k,
// ek = e_k out (ek only for R >= 2).
template <int R>
__device__ __forceinline__ void lap_group_run(const float4 *w, const float *xs, const float *cx, const float *cz,
                                              float cres, float2 dm01, float2 dm23, float2 em01, float2 em23,
                                              float2 &dk01, float2 &dk23, float2 &ek01, float2 &ek23,
                                              float2 &l01, float2 &l23)
{
    constexpr int O = 4 * XGroups<R>::G;
    const float2 c01 = lo2(w[R]), c23 = hi2(w[R]);
    const float2 m1 = splat2(-1.f);
    dk01 = __ffma2_rn(c01, m1, lo2(w[R + 1]));
    dk23 = __ffma2_rn(c23, m1, hi2(w[R + 1]));
    float2 z01 = __fmul2_rn(splat2(cz[1]), __ffma2_rn(dm01, m1, dk01));
    float2 z23 = __fmul2_rn(splat2(cz[1]), __ffma2_rn(dm23, m1, dk23));
    if (R >= 2) {
        ek01 = __ffma2_rn(c01, m1, lo2(w[R + 2]));
        ek23 = __ffma2_rn(c23, m1, hi2(w[R + 2]));
        z01 = __ffma2_rn(splat2(cz[2]), __ffma2_rn(em01, m1, ek01), z01);
        z23 = __ffma2_rn(splat2(cz[2]), __ffma2_rn(em23, m1, ek23), z23);
    }
#pragma unroll
    for (int m = 3; m <= R; ++m) {
        z01 = __ffma2_rn(splat2(cz[m]), __fadd2_rn(lo2(w[R - m]), lo2(w[R + m])), z01);
        z23 = __ffma2_rn(splat2(cz[m]), __fadd2_rn(hi2(w[R - m]), hi2(w[R + m])), z23);
    }
    float e[5];
#pragma unroll
    for (int j = -1; j <= 3; ++j) e[j + 1] = xs[O + j + 1] - xs[O + j];
    float2 x01 = __fmul2_rn(splat2(cx[1]), f2(e[1] - e[0], e[2] - e[1]));
    float2 x23 = __fmul2_rn(splat2(cx[1]), f2(e[3] - e[2], e[4] - e[3]));
    auto dif = [&](const float2 &v, const float2 &c) { return __ffma2_rn(c, m1, v); };
    if (R >= 2) {
        x01 = __ffma2_rn(splat2(cx[2]), __fadd2_rn(dif(f2(xs[O + 2], xs[O + 3]), c01),
                                                   dif(f2(xs[O - 2], xs[O - 1]), c01)), x01);
        x23 = __ffma2_rn(splat2(cx[2]), __fadd2_rn(dif(f2(xs[O + 4], xs[O + 5]), c23),
                                                   dif(f2(xs[O + 0], xs[O + 1]), c23)), x23);
    }
#pragma unroll
    for (int m = 3; m <= R; ++m) {
        const float2 s01 = (m & 1) ? f2(xs[O - m] + xs[O + m], xs[O + 1 - m] + xs[O + 1 + m])
                                   : __fadd2_rn(f2(xs[O - m], xs[O + 1 - m]), f2(xs[O + m], xs[O + 1 + m]));
        const float2 s23 = (m & 1) ? f2(xs[O + 2 - m] + xs[O + 2 + m], xs[O + 3 - m] + xs[O + 3 + m])
                                   : __fadd2_rn(f2(xs[O + 2 - m], xs[O + 3 - m]),
                                                f2(xs[O + 2 + m], xs[O + 3 + m]));
        x01 = __ffma2_rn(splat2(cx[m]), s01, x01);
        x23 = __ffma2_rn(splat2(cx[m]), s23, x23);
    }
    if (R >= 3) {
        x01 = __ffma2_rn(splat2(cres), c01, x01);
        x23 = __ffma2_rn(splat2(cres), c23, x23);
    }
    l01 = __fadd2_rn(x01, z01);
    l23 = __fadd2_rn(x23, z23);
}

// The x-line of a group for R <= 8 from its float4 neighbours l2, l, r, r2.
__device__ __forceinline__ void xline2(const float4 &l2, const float4 &l, const float4 &c, const float4 &r,
                                       const float4 &r2, float *xs)
{
    xs[0] = l2.x; xs[1] = l2.y; xs[2] = l2.z; xs[3] = l2.w;
    xs[4] = l.x; xs[5] = l.y; xs[6] = l.z; xs[7] = l.w;
    xs[8] = c.x; xs[9] = c.y; xs[10] = c.z; xs[11] = c.w;
    xs[12] = r.x; xs[13] = r.y; xs[14] = r.z; xs[15] = r.w;
    xs[16] = r2.x; xs[17] = r2.y; xs[18] = r2.z; xs[19] = r2.w;
}

// The x-line of a group for R <= 4 from its float4 neighbours l and r.
__device__ __forceinline__ void xline1(const float4 &l, const float4 &c, const float4 &r, float *xs)
{
    xs[0] = l.x; xs[1] = l.y; xs[2] = l.z; xs[3] = l.w;
    xs[4] = c.x; xs[5] = c.y; xs[6] = c.z; xs[7] = c.w;
    xs[8] = r.x; xs[9] = r.y; xs[10] = r.z; xs[11] = r.w;
}

}  // namespace empso
