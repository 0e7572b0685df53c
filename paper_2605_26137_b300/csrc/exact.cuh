// Exact-difference and compensated-product helpers (FP32 only): edge vectors
// of FP32 vertices as hi + lo pairs (TwoSum, exact) and 2x2 determinants with
// the product rounding error recovered by an FMA (Kahan).  Used wherever a
// small difference of large coordinates would otherwise lose its direction
// (sliver triangles of marching-grid meshes).
#pragma once

#include "ag_internal.cuh"

namespace ag {

__device__ __forceinline__ void two_diff(float a, float b, float &hi, float &lo) {
    // hi + lo == a - b exactly
    float s = __fsub_rn(a, b);
    float bp = __fsub_rn(s, a);          // ~ -b
    float ap = __fsub_rn(s, bp);         // ~ a
    float db = __fsub_rn(__fmul_rn(-1.f, b), bp);
    float da = __fsub_rn(a, ap);
    hi = s;
    lo = __fadd_rn(da, db);
}

// a*b - c*d with the rounding error of c*d recovered by an FMA
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
    float w = __fmul_rn(c, d);
    float e = __fmaf_rn(-c, d, w);       // w - c*d exactly
    float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

__device__ __forceinline__ float3 exact_edge_hi(float3 a, float3 b, float3 &lo) {
    float3 hi;
    two_diff(a.x, b.x, hi.x, lo.x);
    two_diff(a.y, b.y, hi.y, lo.y);
    two_diff(a.z, b.z, hi.z, lo.z);
    return hi;
}

// (p1 - p0) x (p2 - p0) accurate to a few ulps of each component
__device__ __forceinline__ float3 face_cross(float3 p0, float3 p1, float3 p2) {
    float3 l1, l2;
    float3 h1 = exact_edge_hi(p1, p0, l1);
    float3 h2 = exact_edge_hi(p2, p0, l2);
    float3 r;
    r.x = det2(h1.y, h2.z, h1.z, h2.y) + ((h1.y * l2.z + l1.y * h2.z) - (h1.z * l2.y + l1.z * h2.y));
    r.y = det2(h1.z, h2.x, h1.x, h2.z) + ((h1.z * l2.x + l1.z * h2.x) - (h1.x * l2.z + l1.x * h2.z));
    r.z = det2(h1.x, h2.y, h1.y, h2.x) + ((h1.x * l2.y + l1.x * h2.y) - (h1.y * l2.x + l1.y * h2.x));
    return r;
}

// s1 * e1 - s2 * e2 for exact small integers s1, s2 and exact edges e = hi + lo
__device__ __forceinline__ float3 lincomb_edges(float s1, float3 h1, float3 l1, float s2, float3 h2, float3 l2) {
    float3 r;
    r.x = det2(s1, h1.x, s2, h2.x) + (s1 * l1.x - s2 * l2.x);
    r.y = det2(s1, h1.y, s2, h2.y) + (s1 * l1.y - s2 * l2.y);
    r.z = det2(s1, h1.z, s2, h2.z) + (s1 * l1.z - s2 * l2.z);
    return r;
}

}  // namespace ag
