// The closest-hit ray machinery shared by the texel traversal (trace.cu)
// and the hidden-face visibility pass (hidden.cu): the ray in the
// watertight-test form (Woop, Benthin, Wald 2013) with its origin as base +
// offset, the FP32 triangle test with explicit round-to-nearest edge
// functions (a shared edge gets exactly opposite values from both triangles;
// zero counts as inside) and the closest-|t| bookkeeping (equal |t| prefers
// t >= 0, equal t the lower original id), and the child-box tests of both
// node layouts with their conservative widening.
#pragma once

#include "traverse.cuh"

namespace ag {
namespace {

struct Ray {
    // exact-origin triangle test: permuted axes (two bits each: x, y, z ray
    // axes in bits 0-1, 2-3, 4-5), shear, origin as base + offset
    uint32_t kp;
    float Sx, Sy, Sz;
    float bx, by, bz;
    float ox, oy, oz;
    // box test: rounded origin, 1/d with zero components made tiny (its signs
    // are the direction's)
    float px, py, pz;
    float ix, iy, iz;
    __device__ __forceinline__ int kx() const { return (int)(kp & 3u); }
    __device__ __forceinline__ int ky() const { return (int)((kp >> 2) & 3u); }
    __device__ __forceinline__ int kz() const { return (int)((kp >> 4) & 3u); }
    __device__ __forceinline__ bool nx() const { return ix < 0.f; }
    __device__ __forceinline__ bool ny() const { return iy < 0.f; }
    __device__ __forceinline__ bool nz() const { return iz < 0.f; }
};

__device__ __forceinline__ float pick(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ Ray make_ray(float3 base, float3 off, float3 d) {
    Ray r;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    const int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    float dz = pick(d, kz);
    if (dz < 0.f) { int t = kx; kx = ky; ky = t; }
    r.kp = (uint32_t)kx | ((uint32_t)ky << 2) | ((uint32_t)kz << 4);
    r.Sx = pick(d, kx) / dz;
    r.Sy = pick(d, ky) / dz;
    r.Sz = 1.0f / dz;
    r.bx = pick(base, kx); r.by = pick(base, ky); r.bz = pick(base, kz);
    r.ox = pick(off, kx); r.oy = pick(off, ky); r.oz = pick(off, kz);
    float3 p = base + off;
    r.px = p.x; r.py = p.y; r.pz = p.z;
    float3 dd = d;
    // (2^15 s / d of the 8-bit decode stays finite for node scales up to ~1e10)
    if (fabsf(dd.x) < 1e-24f) dd.x = copysignf(1e-24f, dd.x);
    if (fabsf(dd.y) < 1e-24f) dd.y = copysignf(1e-24f, dd.y);
    if (fabsf(dd.z) < 1e-24f) dd.z = copysignf(1e-24f, dd.z);
    r.ix = 1.0f / dd.x; r.iy = 1.0f / dd.y; r.iz = 1.0f / dd.z;
    return r;
}

// vertex in ray space: (v - base) - offset, permuted and sheared
__device__ __forceinline__ void xform(const Ray &r, float4 v, float &X, float &Y, float &Z) {
    float3 a = make_float3(v.x, v.y, v.z);
    float ax = __fsub_rn(__fsub_rn(pick(a, r.kx()), r.bx), r.ox);
    float ay = __fsub_rn(__fsub_rn(pick(a, r.ky()), r.by), r.oy);
    float az = __fsub_rn(__fsub_rn(pick(a, r.kz()), r.bz), r.oz);
    X = __fmaf_rn(-r.Sx, az, ax);
    Y = __fmaf_rn(-r.Sy, az, ay);
    Z = __fmul_rn(r.Sz, az);
}

struct Best {
    float t, babs;
    uint32_t rec;
    float U, V, W, det;
    bool found;
};

// the three edge functions of triangle (A, B, C) in ray space, and the
// vertices' sheared depths
__device__ __forceinline__ void tri_edges(const Ray &r, float4 A, float4 B, float4 C, float &U, float &V, float &W,
                                          float &Az, float &Bz, float &Cz) {
    float Ax, Ay, Bx, By, Cx, Cy;
    xform(r, A, Ax, Ay, Az);
    xform(r, B, Bx, By, Bz);
    xform(r, C, Cx, Cy, Cz);
    U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
}

__device__ __forceinline__ void test_tri(const Ray &r, const float4 *__restrict__ tris,
                                         const int32_t *__restrict__ tri_ids, uint32_t rec, Best &b) {
    float4 A = __ldg(&tris[3 * (size_t)rec]), B = __ldg(&tris[3 * (size_t)rec + 1]), C = __ldg(&tris[3 * (size_t)rec + 2]);
    float U, V, W, Az, Bz, Cz;
    tri_edges(r, A, B, C, U, V, W, Az, Bz, Cz);
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return;
    float det = U + V + W;
    if (det == 0.f) return;
    float T = U * Az + V * Bz + W * Cz;
    // |T / det| <= babs, tested without the division (with slack; exact below)
    if (fabsf(T) > b.babs * fabsf(det) * 1.0000010f) return;
    float t = T / det;
    float at = fabsf(t);
    if (!(at <= b.babs)) return;
    if (b.found && at == b.babs) {
        if ((t >= 0.f) != (b.t >= 0.f)) {
            if (t < 0.f) return;
        } else if (t != b.t || tri_ids[rec] >= tri_ids[b.rec]) {
            return;
        }
    }
    b.t = t; b.babs = at; b.rec = rec; b.U = U; b.V = V; b.W = W; b.det = det; b.found = true;
}

// The same test for a lane that shares its ray with other lanes: `lim` is the
// closest |t| any lane of the ray has found (max_dist at the start), the
// lane's own best decides ties only among its own candidates, and an accepted
// hit lowers `lim`.  Candidates at an equal |t| held by different lanes are
// ordered when the lanes' bests are merged (t >= 0 first, then the lower id).
__device__ __forceinline__ void test_tri_shared(const Ray &r, const float4 *__restrict__ tris,
                                                const int32_t *__restrict__ tri_ids, uint32_t rec, Best &b,
                                                float &lim) {
    float4 A = __ldg(&tris[3 * (size_t)rec]), B = __ldg(&tris[3 * (size_t)rec + 1]), C = __ldg(&tris[3 * (size_t)rec + 2]);
    float U, V, W, Az, Bz, Cz;
    tri_edges(r, A, B, C, U, V, W, Az, Bz, Cz);
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return;
    float det = U + V + W;
    if (det == 0.f) return;
    float T = U * Az + V * Bz + W * Cz;
    if (fabsf(T) > lim * fabsf(det) * 1.0000010f) return;
    float t = T / det;
    float at = fabsf(t);
    if (!(at <= lim)) return;
    if (b.found && at == b.babs) {
        if ((t >= 0.f) != (b.t >= 0.f)) {
            if (t < 0.f) return;
        } else if (t != b.t || tri_ids[rec] >= tri_ids[b.rec]) {
            return;
        }
    }
    b.t = t; b.babs = at; b.rec = rec; b.U = U; b.V = V; b.W = W; b.det = det; b.found = true;
    lim = at;
}

template <int LAYOUT>
struct NodeOps;

// 80-byte quantised node.  Per node and axis the child planes become one
// PRMT and one FMA each: t(q) = Q * a + b with Q = 1 + q 2^-15 (exact),
// a = 2^(e+15) / d and b = (origin - p) / d - a.  The intervals are widened by
// eps = (2^-20 (|origin| + |p|) + 2^-7 2^e) / |d|.  The roundings on the way
// (the decoded plane, 1/d, the rounded ray origin, origin - p, the product and
// the subtraction of a in b, the widening's own subtraction, the FMA) sum to
// at most 2^-24 (7 (|origin| + |p|) + 66301 2^e) / |d| + 2^-23 eps, so the
// widening covers them by a factor of about 2 and a box the exact line meets
// is never rejected.
// With LEAVES, hit leaf children are recorded in *ls (to be tested by the
// caller right away) instead of being offered.
template <>
struct NodeOps<AG_BVH_Q8> {
    template <bool LEAVES = false>
    static __device__ __forceinline__ void visit(const void *nodes, uint32_t idx, const Ray &r, float lim, Next &nx,
                                                 uint2 *stack, int &sp, unsigned *status, int cap = STACK,
                                                 LeafSet *ls = nullptr) {
        const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const QNode *>(nodes) + idx);
        uint4 w0 = __ldg(p), w1 = __ldg(p + 1), w2 = __ldg(p + 2), w3 = __ldg(p + 3), w4 = __ldg(p + 4);
        float ox = __uint_as_float(w0.x), oy = __uint_as_float(w0.y), oz = __uint_as_float(w0.z);
        float sx = __uint_as_float((w0.w & 0xffu) << 23);
        float sy = __uint_as_float(((w0.w >> 8) & 0xffu) << 23);
        float sz = __uint_as_float(((w0.w >> 16) & 0xffu) << 23);
        // plane t = (origin + q s - p) / d = Q a + b with Q = 1 + q 2^-15,
        // a = 2^15 s / d (exact: s is a power of two), b = (origin - p) / d - a
        float ax = Q_SCALE * sx * r.ix, ay = Q_SCALE * sy * r.iy, az = Q_SCALE * sz * r.iz;
        float bx = (ox - r.px) * r.ix - ax, by = (oy - r.py) * r.iy - ay, bz = (oz - r.pz) * r.iz - az;
        float ex = (EPS_POS * (fabsf(ox) + fabsf(r.px)) + EPS_Q * sx) * fabsf(r.ix);
        float ey = (EPS_POS * (fabsf(oy) + fabsf(r.py)) + EPS_Q * sy) * fabsf(r.iy);
        float ez = (EPS_POS * (fabsf(oz) + fabsf(r.pz)) + EPS_Q * sz) * fabsf(r.iz);
        float bnx = bx - ex, bfx = bx + ex, bny = by - ey, bfy = by + ey, bnz = bz - ez, bfz = bz + ez;
        // near-plane bytes: lo for d > 0, hi for d < 0
        uint32_t nx0 = r.nx() ? w3.z : w2.x, nx1 = r.nx() ? w3.w : w2.y, fx0 = r.nx() ? w2.x : w3.z, fx1 = r.nx() ? w2.y : w3.w;
        uint32_t ny0 = r.ny() ? w4.x : w2.z, ny1 = r.ny() ? w4.y : w2.w, fy0 = r.ny() ? w2.z : w4.x, fy1 = r.ny() ? w2.w : w4.y;
        uint32_t nz0 = r.nz() ? w4.z : w3.x, nz1 = r.nz() ? w4.w : w3.y, fz0 = r.nz() ? w3.x : w4.z, fz1 = r.nz() ? w3.y : w4.w;
        uint32_t child_base = w1.x, tri_base = w1.y;
        if (LEAVES) *ls = LeafSet{0u, w1.z, w1.w, tri_base};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int k = c & 3;
            const bool hi = c >= 4;
            uint32_t m = ((hi ? w1.w : w1.z) >> (8 * k)) & 0xffu;
            // near and far plane of an axis in one packed FMA
            float tnx, tfx, tny, tfy, tnz, tfz;
            fma2(byte_q(hi ? nx1 : nx0, k), byte_q(hi ? fx1 : fx0, k), ax, ax, bnx, bfx, tnx, tfx);
            fma2(byte_q(hi ? ny1 : ny0, k), byte_q(hi ? fy1 : fy0, k), ay, ay, bny, bfy, tny, tfy);
            fma2(byte_q(hi ? nz1 : nz0, k), byte_q(hi ? fz1 : fz0, k), az, az, bnz, bfz, tnz, tfz);
            float te = max3f(tnx, tny, tnz);
            float tx = min3f(tfx, tfy, tfz);
            if (LEAVES) {
                // an empty slot (m = 0) recorded as a leaf holds no triangle
                if (te <= tx && te <= lim && tx >= -lim) {
                    if (m & 0x80u)
                        offer(child_base + (m & 0x7fu), max3f(te, -tx, 0.f), nx, stack, sp, status, cap);
                    else
                        ls->mask |= 1u << c;
                }
            } else if (m != 0 && te <= tx && te <= lim && tx >= -lim) {
                offer(child_ref(m, child_base, tri_base), max3f(te, -tx, 0.f), nx, stack, sp, status, cap);
            }
        }
    }
};

// 208-byte node with exact FP32 child boxes: t = plane / d - p / d, widened by
// eps = 2^-21 (scene bound + |p|) / |d| per axis.
template <>
struct NodeOps<AG_BVH_F32> {
    template <bool LEAVES = false>
    static __device__ __forceinline__ void visit(const void *nodes, uint32_t idx, const Ray &r, float lim, Next &nx,
                                                 uint2 *stack, int &sp, unsigned *status, float scene_abs,
                                                 int cap = STACK, LeafSet *ls = nullptr) {
        const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const FNode *>(nodes) + idx);
        uint4 h = __ldg(p);
        uint32_t child_base = h.x, tri_base = h.y;
        if (LEAVES) *ls = LeafSet{0u, h.z, h.w, tri_base};
        float ex = EPS_REL * (scene_abs + fabsf(r.px)) * fabsf(r.ix);
        float ey = EPS_REL * (scene_abs + fabsf(r.py)) * fabsf(r.iy);
        float ez = EPS_REL * (scene_abs + fabsf(r.pz)) * fabsf(r.iz);
        float cx = -r.px * r.ix, cy = -r.py * r.iy, cz = -r.pz * r.iz;
        float cnx = cx - ex, cfx = cx + ex, cny = cy - ey, cfy = cy + ey, cnz = cz - ez, cfz = cz + ez;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint4 lx = __ldg(p + 1 + half), ly = __ldg(p + 3 + half), lz = __ldg(p + 5 + half);
            uint4 hx = __ldg(p + 7 + half), hy = __ldg(p + 9 + half), hz = __ldg(p + 11 + half);
            const uint32_t LX[4] = {lx.x, lx.y, lx.z, lx.w}, LY[4] = {ly.x, ly.y, ly.z, ly.w}, LZ[4] = {lz.x, lz.y, lz.z, lz.w};
            const uint32_t HX[4] = {hx.x, hx.y, hx.z, hx.w}, HY[4] = {hy.x, hy.y, hy.z, hy.w}, HZ[4] = {hz.x, hz.y, hz.z, hz.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t m = ((half ? h.w : h.z) >> (8 * k)) & 0xffu;
                float plx = __uint_as_float(r.nx() ? HX[k] : LX[k]), pfx = __uint_as_float(r.nx() ? LX[k] : HX[k]);
                float ply = __uint_as_float(r.ny() ? HY[k] : LY[k]), pfy = __uint_as_float(r.ny() ? LY[k] : HY[k]);
                float plz = __uint_as_float(r.nz() ? HZ[k] : LZ[k]), pfz = __uint_as_float(r.nz() ? LZ[k] : HZ[k]);
                float tnx, tfx, tny, tfy, tnz, tfz;
                fma2(plx, pfx, r.ix, r.ix, cnx, cfx, tnx, tfx);
                fma2(ply, pfy, r.iy, r.iy, cny, cfy, tny, tfy);
                fma2(plz, pfz, r.iz, r.iz, cnz, cfz, tnz, tfz);
                float te = max3f(tnx, tny, tnz);
                float tx = min3f(tfx, tfy, tfz);
                if (m != 0 && te <= tx && te <= lim && tx >= -lim) {
                    if (LEAVES && !(m & 0x80u))
                        ls->mask |= 1u << (4 * half + k);
                    else
                        offer(child_ref(m, child_base, tri_base), max3f(te, -tx, 0.f), nx, stack, sp, status, cap);
                }
            }
        }
    }
};

}  // namespace
}  // namespace ag
