// Closest-point correspondence (the literal reading of Sec. 6.4): per texel,
// the high-poly surface point nearest to the texel's 3D position, found by a
// BVH search, with the smooth normal interpolated there by the point's
// barycentrics, followed by the same distance filter, UV-reliability filter
// and tangent-space shading as the ray query.
//
// One persistent launch per ray list; a warp takes 32 consecutive texels of
// the tile-ordered list (the "batch" schedule: a per-lane refill and a
// while-while node/leaf split were both measured slower here).  Per texel:
//   - query point p = v0 + b1 (v1 - v0) + b2 (v2 - v0), kept as (v0, offset)
//     so triangle vertices are taken relative to p with two roundings;
//   - branch and bound over the 8-wide BVH: a child is entered only when the
//     distance from p to its box (decoded exactly as built, shrunk by the
//     rounding slack of the decode and of p, so never overestimated) is within
//     the current best distance, the nearest child first; the bound starts at
//     the distance filter max_dist (inclusive);
//   - per triangle, the closest point by Voronoi-region classification
//     (Ericson, Real-Time Collision Detection, 2005, Sec. 5.1.5): vertex,
//     edge or face region from six dot products, evaluated branch-free (all
//     lanes of a warp run the same instructions); the barycentrics are formed
//     once, for the winning triangle, when shading;
//   - ties in squared distance prefer the lower original triangle id;
//   - displacement = distance signed by (x - p) . d (d the texel normal,
//     zero counts as +).
#include "traverse.cuh"

#include <cstring>

namespace ag {
namespace {

constexpr float LIM_REL = 1.0000010f;  // 1 + 2^-20: slack on squared-distance bounds

struct PBest {
    float d2;          // squared distance of the best point (or max_dist^2 before the first)
    uint32_t rec;      // its triangle record (point and barycentrics are recomputed when shading)
    bool found;
};

struct PointState {
    int job;
    int texel, face;
    float b1, b2;
    int4 fi;
    float3 d;          // unit texel normal
    float3 base, off;  // p = base + off
    float3 p;          // p rounded to FP32 (box tests)
    PBest best;
    uint32_t cur;
    int sp, steps;
};

// vertex relative to p: (v - base) - off
__device__ __forceinline__ float3 rel(const PointState &S, float4 v) {
    return make_float3(__fsub_rn(__fsub_rn(v.x, S.base.x), S.off.x), __fsub_rn(__fsub_rn(v.y, S.base.y), S.off.y),
                       __fsub_rn(__fsub_rn(v.z, S.base.z), S.off.z));
}

// Closest point of triangle (a, b, c) to the origin by Voronoi region, in a
// branch-free form: every region's point is x = P + E * (num / den),
//   vertex A / B / C:  P = that vertex, num = 0;
//   edge AB / AC / BC: P = its first vertex, E = the edge, num / den = the
//                      clamped projection parameter;
//   face:              P = 0, E = n = (b - a) x (c - a), num / den = (a . n) / (n . n),
//                      the foot of the perpendicular (accurate to a few FP32
//                      ulps of the vertex offsets where the region's
//                      barycentric numerators cancel).
// The region tests are those of the classification, taken in its order of
// precedence (later assignments below win).
enum { REG_A = 0, REG_B, REG_C, REG_AB, REG_AC, REG_BC, REG_FACE };

struct TriQ {
    float3 P, E;
    float num, den;
    float va, vb, vc;   // face-region barycentric numerators (a, b, c)
    int reg;
};

__device__ __forceinline__ void tri_query(float3 a, float3 b, float3 c, TriQ &q) {
    const float3 ab = b - a, ac = c - a;
    const float d1 = -dot3(ab, a), d2 = -dot3(ac, a);
    const float d3 = -dot3(ab, b), d4 = -dot3(ac, b);
    const float d5 = -dot3(ab, c), d6 = -dot3(ac, c);
    q.vc = d1 * d4 - d3 * d2;
    q.vb = d5 * d2 - d1 * d6;
    q.va = d3 * d6 - d5 * d4;
    const float e43 = d4 - d3, e56 = d5 - d6;
    const float3 n = cross3(ab, ac);
    const float3 zero = make_float3(0.f, 0.f, 0.f);
    int reg = REG_FACE;
    float3 P = zero, E = n;
    float num = dot3(a, n), den = dot3(n, n);
    const bool bc = q.va <= 0.f && e43 >= 0.f && e56 >= 0.f;
    reg = bc ? REG_BC : reg; P = bc ? b : P; E = bc ? c - b : E; num = bc ? e43 : num; den = bc ? e43 + e56 : den;
    const bool acr = q.vb <= 0.f && d2 >= 0.f && d6 <= 0.f;
    reg = acr ? REG_AC : reg; P = acr ? a : P; E = acr ? ac : E; num = acr ? d2 : num; den = acr ? d2 - d6 : den;
    const bool cv = d6 >= 0.f && d5 <= d6;
    reg = cv ? REG_C : reg; P = cv ? c : P; num = cv ? 0.f : num; den = cv ? 1.f : den;
    const bool abr = q.vc <= 0.f && d1 >= 0.f && d3 <= 0.f;
    reg = abr ? REG_AB : reg; P = abr ? a : P; E = abr ? ab : E; num = abr ? d1 : num; den = abr ? d1 - d3 : den;
    const bool bv = d3 >= 0.f && d4 <= d3;
    reg = bv ? REG_B : reg; P = bv ? b : P; num = bv ? 0.f : num; den = bv ? 1.f : den;
    const bool av = d1 <= 0.f && d2 <= 0.f;
    reg = av ? REG_A : reg; P = av ? a : P; num = av ? 0.f : num; den = av ? 1.f : den;
    q.P = P; q.E = E; q.num = num; q.den = den; q.reg = reg;
}

// the point of a query; false for a zero-area triangle in the face region
// (its edges belong to neighbouring triangles as well)
__device__ __forceinline__ bool tri_point(const TriQ &q, float3 &x) {
    if (!(q.den > 0.f)) {
        x = q.P;
        return q.reg != REG_FACE;
    }
    x = q.P + q.E * (q.num / q.den);
    return true;
}

// barycentrics (of a, b, c) of the query's point
__device__ __forceinline__ float3 tri_bary(const TriQ &q) {
    const float t = q.den > 0.f ? q.num / q.den : 0.f;
    switch (q.reg) {
        case REG_A: return make_float3(1.f, 0.f, 0.f);
        case REG_B: return make_float3(0.f, 1.f, 0.f);
        case REG_C: return make_float3(0.f, 0.f, 1.f);
        case REG_AB: return make_float3(1.f - t, t, 0.f);
        case REG_AC: return make_float3(1.f - t, 0.f, t);
        case REG_BC: return make_float3(0.f, 1.f - t, t);
        default: {
            const float s = q.va + q.vb + q.vc;
            if (!(s > 0.f)) return make_float3(1.f / 3.f, 1.f / 3.f, 1.f / 3.f);
            const float v = q.vb / s, w = q.vc / s;
            return make_float3(1.f - v - w, v, w);
        }
    }
}

__device__ __forceinline__ void test_tri(PointState &S, const float4 *__restrict__ tris,
                                         const int32_t *__restrict__ tri_ids, uint32_t rec) {
    float4 A = __ldg(&tris[3 * (size_t)rec]), B = __ldg(&tris[3 * (size_t)rec + 1]), C = __ldg(&tris[3 * (size_t)rec + 2]);
    TriQ q;
    tri_query(rel(S, A), rel(S, B), rel(S, C), q);
    float3 x;
    if (!tri_point(q, x)) return;
    float d2 = dot3(x, x);
    if (!(d2 <= S.best.d2)) return;
    if (S.best.found && d2 == S.best.d2 && tri_ids[rec] >= tri_ids[S.best.rec]) return;
    S.best.d2 = d2; S.best.rec = rec; S.best.found = true;
}

template <int LAYOUT>
struct PointNode;

// 80-byte quantised node.  Child planes decode as fmaf(q, 2^e, origin), the
// arithmetic the build verified to enclose the exact child box; here as
// Q * 2^(e+15) + (origin - p - 2^(e+15)) with the exact float Q = 1 + q 2^-15
// (one PRMT and one FMA per plane), and every distance component is shrunk by
// 2^-20 (|origin| + |p|) + 2^-7 2^e.  The roundings on the way (p,
// origin - p, the subtraction of 2^(e+15), the slack subtraction, the FMA,
// and the half ulp by which the build's rounded decode may exceed the exact
// plane) sum to at most 2^-24 (5 |origin| + 5 |p| + 66046 2^e) + 2^-23 of
// the slack, about half of it.
// With LEAVES, leaf children within the bound are recorded in *ls (to be
// tested by the caller right away) instead of being offered.
template <>
struct PointNode<AG_BVH_Q8> {
    template <bool LEAVES = false>
    static __device__ __forceinline__ void visit(const void *nodes, uint32_t idx, float3 p, float lim, Next &nx,
                                                 uint2 *stack, int &sp, unsigned *status, float,
                                                 LeafSet *ls = nullptr) {
        const uint4 *q = reinterpret_cast<const uint4 *>(static_cast<const QNode *>(nodes) + idx);
        uint4 w0 = __ldg(q), w1 = __ldg(q + 1), w2 = __ldg(q + 2), w3 = __ldg(q + 3), w4 = __ldg(q + 4);
        float ox = __uint_as_float(w0.x), oy = __uint_as_float(w0.y), oz = __uint_as_float(w0.z);
        float sx = __uint_as_float((w0.w & 0xffu) << 23);
        float sy = __uint_as_float(((w0.w >> 8) & 0xffu) << 23);
        float sz = __uint_as_float(((w0.w >> 16) & 0xffu) << 23);
        const float Ax = Q_SCALE * sx, Ay = Q_SCALE * sy, Az = Q_SCALE * sz;
        float rx = ox - p.x - Ax, ry = oy - p.y - Ay, rz = oz - p.z - Az;
        float ex = EPS_POS * (fabsf(ox) + fabsf(p.x)) + EPS_Q * sx;
        float ey = EPS_POS * (fabsf(oy) + fabsf(p.y)) + EPS_Q * sy;
        float ez = EPS_POS * (fabsf(oz) + fabsf(p.z)) + EPS_Q * sz;
        // lo - p - e  and  p - hi - e  as one FMA each
        float blx = rx - ex, bly = ry - ey, blz = rz - ez;
        float bhx = -rx - ex, bhy = -ry - ey, bhz = -rz - ez;
        uint32_t child_base = w1.x, tri_base = w1.y;
        if (LEAVES) *ls = LeafSet{0u, w1.z, w1.w, tri_base};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int k = c & 3;
            const bool hi = c >= 4;
            uint32_t m = ((hi ? w1.w : w1.z) >> (8 * k)) & 0xffu;
            float gx = fmaxf(fmaxf(__fmaf_rn(byte_q(hi ? w2.y : w2.x, k), Ax, blx),
                                   __fmaf_rn(byte_q(hi ? w3.w : w3.z, k), -Ax, bhx)), 0.f);
            float gy = fmaxf(fmaxf(__fmaf_rn(byte_q(hi ? w2.w : w2.z, k), Ay, bly),
                                   __fmaf_rn(byte_q(hi ? w4.y : w4.x, k), -Ay, bhy)), 0.f);
            float gz = fmaxf(fmaxf(__fmaf_rn(byte_q(hi ? w3.y : w3.x, k), Az, blz),
                                   __fmaf_rn(byte_q(hi ? w4.w : w4.z, k), -Az, bhz)), 0.f);
            float g2 = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, gz * gz));
            if (m != 0 && g2 <= lim) {
                if (LEAVES && !(m & 0x80u))
                    ls->mask |= 1u << c;
                else
                    offer(child_ref(m, child_base, tri_base), g2, nx, stack, sp, status);
            }
        }
    }
};

// 208-byte node with exact FP32 child boxes; the slack per axis is
// 2^-21 (scene bound + |p|).
template <>
struct PointNode<AG_BVH_F32> {
    template <bool LEAVES = false>
    static __device__ __forceinline__ void visit(const void *nodes, uint32_t idx, float3 p, float lim, Next &nx,
                                                 uint2 *stack, int &sp, unsigned *status, float scene_abs,
                                                 LeafSet *ls = nullptr) {
        const uint4 *q = reinterpret_cast<const uint4 *>(static_cast<const FNode *>(nodes) + idx);
        uint4 h = __ldg(q);
        uint32_t child_base = h.x, tri_base = h.y;
        if (LEAVES) *ls = LeafSet{0u, h.z, h.w, tri_base};
        float ex = EPS_REL * (scene_abs + fabsf(p.x));
        float ey = EPS_REL * (scene_abs + fabsf(p.y));
        float ez = EPS_REL * (scene_abs + fabsf(p.z));
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint4 lx = __ldg(q + 1 + half), ly = __ldg(q + 3 + half), lz = __ldg(q + 5 + half);
            uint4 hx = __ldg(q + 7 + half), hy = __ldg(q + 9 + half), hz = __ldg(q + 11 + half);
            const uint32_t LX[4] = {lx.x, lx.y, lx.z, lx.w}, LY[4] = {ly.x, ly.y, ly.z, ly.w}, LZ[4] = {lz.x, lz.y, lz.z, lz.w};
            const uint32_t HX[4] = {hx.x, hx.y, hx.z, hx.w}, HY[4] = {hy.x, hy.y, hy.z, hy.w}, HZ[4] = {hz.x, hz.y, hz.z, hz.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t m = ((half ? h.w : h.z) >> (8 * k)) & 0xffu;
                float gx = fmaxf(fmaxf(__uint_as_float(LX[k]) - p.x, p.x - __uint_as_float(HX[k])) - ex, 0.f);
                float gy = fmaxf(fmaxf(__uint_as_float(LY[k]) - p.y, p.y - __uint_as_float(HY[k])) - ey, 0.f);
                float gz = fmaxf(fmaxf(__uint_as_float(LZ[k]) - p.z, p.z - __uint_as_float(HZ[k])) - ez, 0.f);
                float g2 = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, gz * gz));
                if (m != 0 && g2 <= lim) {
                    if (LEAVES && !(m & 0x80u))
                        ls->mask |= 1u << (4 * half + k);
                    else
                        offer(child_ref(m, child_base, tri_base), g2, nx, stack, sp, status);
                }
            }
        }
    }
};

// jw: the query's asset when JOBS is JOBS_MANY (found by the caller)
template <int JOBS>
__device__ __forceinline__ void setup_point(const TraceArgs &A, long long r, PointState &S, int jw) {
    int j = 0;
    long long local = r;
    if (JOBS == JOBS_MANY) {
        j = jw;
        local = r - A.job_begin[j];
    }
    const TraceJob &J = job_t<JOBS>(A, j);
    int4 rr = J.rays[local];
    S.job = j;
    S.texel = rr.x;
    S.face = rr.y;
    S.b1 = __int_as_float(rr.z);
    S.b2 = __int_as_float(rr.w);
    S.fi = J.lface[S.face];
    float3 P0 = f3(J.lpos[S.fi.x]), P1 = f3(J.lpos[S.fi.y]), P2 = f3(J.lpos[S.fi.z]);
    float3 N0 = f3(J.lnrm[S.fi.x]), N1 = f3(J.lnrm[S.fi.y]), N2 = f3(J.lnrm[S.fi.z]);
    S.base = P0;
    S.off = (P1 - P0) * S.b1 + (P2 - P0) * S.b2;
    S.p = P0 + S.off;
    float3 sv = N0 + (N1 - N0) * S.b1 + (N2 - N0) * S.b2;
    S.d = sv * (1.0f / sqrtf(dot3(sv, sv)));
    S.best.d2 = J.max_dist * J.max_dist;
    S.best.rec = 0;
    S.best.found = false;
    S.cur = 0;
    S.sp = 0;
    S.steps = 0;
}

// A node visit that tests the node's leaf children within the bound right
// away (slot order); only inner children are offered and stacked.  Every step
// of a lane is a node visit (3.32 -> 2.72 ms on the 2.1M-triangle bake over
// 8-bit nodes, for 62 % more triangle tests: sibling leaves are no longer
// taken nearest first, so fewer are culled by a shrinking bound).
template <int LAYOUT, bool COUNT>
__device__ __forceinline__ bool step_point_leaves(const TraceArgs &A, const TraceJob &J, PointState &S, uint2 *stack,
                                                  unsigned long long &c_nodes, unsigned long long &c_tris) {
    Next nx;
    nx.has = false;
    nx.ref = 0;
    nx.dist = 0.f;
    LeafSet ls;
    PointNode<LAYOUT>::template visit<true>(J.nodes, S.cur, S.p, S.best.d2 * LIM_REL, nx, stack, S.sp, A.status,
                                            J.scene_abs, &ls);
    if (COUNT) ++c_nodes;
    while (ls.mask) {
        const int c = __ffs(ls.mask) - 1;
        ls.mask &= ls.mask - 1;
        uint32_t first;
        int cnt;
        leaf_range(ls, c, first, cnt);
        for (int t = 0; t < cnt; ++t) test_tri(S, J.tris, J.tri_ids, first + t);
        if (COUNT) c_tris += cnt;
    }
    if (nx.has) {
        S.cur = nx.ref;
    } else {
        bool done = true;
        const float lim = S.best.d2 * LIM_REL;
        while (S.sp > 0) {
            uint2 e = stack[--S.sp];
            if (__uint_as_float(e.y) <= lim) { S.cur = e.x; done = false; break; }
        }
        if (done) return false;
    }
    if (++S.steps > A.max_steps) {
        atomicOr(A.status, AGS_STEP_CAP);
        return false;
    }
    return true;
}

template <int JOBS>
__device__ __forceinline__ void finish_point(const TraceArgs &A, const PointState &S) {
    const TraceJob &J = job_t<JOBS>(A, S.job);
    const bool hit = S.best.found;
    float3 nh = make_float3(0.f, 0.f, 1.f);
    float disp = 0.f;
    int hit_id = -1;
    if (hit) {
        const size_t r3 = 3 * (size_t)S.best.rec;
        const float4 A = __ldg(&J.tris[r3]), B = __ldg(&J.tris[r3 + 1]), C = __ldg(&J.tris[r3 + 2]);
        TriQ q;
        tri_query(rel(S, A), rel(S, B), rel(S, C), q);
        float3 x;
        tri_point(q, x);
        const float3 bw = tri_bary(q);
        const float3 nA = f3(__ldg(&J.hnormals[__float_as_int(A.w)]));
        const float3 nB = f3(__ldg(&J.hnormals[__float_as_int(B.w)]));
        const float3 nC = f3(__ldg(&J.hnormals[__float_as_int(C.w)]));
        nh = normalize3(nA * bw.x + nB * bw.y + nC * bw.z);
        const float dist = sqrtf(S.best.d2);
        disp = dot3(x, S.d) >= 0.f ? dist : -dist;
        hit_id = J.tri_ids[S.best.rec];
    }
    store_forward(J, S.texel, S.face, S.fi, S.b1, S.b2, S.d, hit, nh, disp, hit_id);
}

// JOBS: one asset (JOBS_ONE, its job in the kernel's parameters) or a batch
// (JOBS_MANY: the warp finds the asset of its first query, each lane steps on
// from there, and the asset's traversal fields stay in registers per query).
template <int LAYOUT, bool COUNT, int JOBS>
__global__ void __launch_bounds__(256) k_closest(TraceArgs A) {
    const int lane = threadIdx.x & 31;
    const long long n_total = *A.n_rays_dev;
    unsigned long long c_nodes = 0, c_tris = 0, c_rays = 0, c_hits = 0;
    uint2 stack[STACK];
    PointState S;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(A.ray_counter, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= n_total) break;
        long long r = (long long)base + lane;
        int jw = 0;
        if (JOBS == JOBS_MANY) {
            if (lane == 0) jw = find_job(A, (long long)base);
            jw = __shfl_sync(0xffffffffu, jw, 0);
        }
        if (r >= n_total) continue;
        if (JOBS == JOBS_MANY)
            while (jw + 1 < A.n_jobs && A.job_begin[jw + 1] <= r) ++jw;
        setup_point<JOBS>(A, r, S, jw);
        if (COUNT) ++c_rays;
        if (JOBS == JOBS_MANY) {
            const TraceJob J = A.jobs[S.job];
            while (step_point_leaves<LAYOUT, COUNT>(A, J, S, stack, c_nodes, c_tris)) {
            }
        } else {
            const TraceJob &J = A.job0;
            while (step_point_leaves<LAYOUT, COUNT>(A, J, S, stack, c_nodes, c_tris)) {
            }
        }
        if (COUNT && S.best.found) ++c_hits;
        finish_point<JOBS>(A, S);
    }
    flush_counters<COUNT>(A, c_rays, c_nodes, c_tris, c_hits);
}

template <int LAYOUT, bool COUNT>
cudaError_t launch_one(const TraceLaunch &L, const TraceArgs &A, cudaStream_t s) {
    int dev;
    cudaGetDevice(&dev);
    int block = L.block_size > 0 ? (L.block_size > 256 ? 256 : L.block_size) : 128;
    int bps = L.blocks_per_sm;
    if (bps <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, A.n_jobs > 1 ? k_closest<LAYOUT, COUNT, JOBS_MANY> : k_closest<LAYOUT, COUNT, JOBS_ONE>, block, 0);
        bps = occ > 0 ? occ : 1;
    }
    unsigned grid = (unsigned)(device_sm_count(dev) * bps);
    if (A.n_jobs > 1)
        k_closest<LAYOUT, COUNT, JOBS_MANY><<<grid, block, 0, s>>>(A);
    else
        k_closest<LAYOUT, COUNT, JOBS_ONE><<<grid, block, 0, s>>>(A);
    return cudaGetLastError();
}

// Point-to-mesh distance (measurement tool): the same branch-and-bound query
// from arbitrary points, the radius starting at max_dist.
template <int LAYOUT>
__global__ void __launch_bounds__(256) k_point_dist(TraceArgs A, const float *__restrict__ pts, long long n,
                                                    float max_dist, float *__restrict__ dist,
                                                    int32_t *__restrict__ tri) {
    uint2 stack[STACK];
    PointState S;
    unsigned long long c0 = 0, c1 = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        S.job = 0;
        S.base = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        S.off = make_float3(0.f, 0.f, 0.f);
        S.p = S.base;
        S.d = make_float3(0.f, 0.f, 1.f);
        S.best.d2 = max_dist * max_dist;
        S.best.rec = 0;
        S.best.found = false;
        S.cur = 0;
        S.sp = 0;
        S.steps = 0;
        while (step_point_leaves<LAYOUT, false>(A, A.job0, S, stack, c0, c1)) {
        }
        dist[i] = S.best.found ? sqrtf(S.best.d2) : -1.f;
        if (tri) tri[i] = S.best.found ? A.job0.tri_ids[S.best.rec] : -1;
    }
}

// The "baked mean" measure of Sec. 6.1, one thread per sample point of the low
// mesh: the normal the RGBA8 map gives at the point (the texel holding its UV
// point, codes decoded as (q - 128) / 127 and renormalised, taken to world
// space through the bake's tangent frame at the point; on a face with
// degenerate UVs the interpolated low normal) against the raw mesh's
// smooth normal at its surface point nearest to the sample (the same
// branch-and-bound query as the closest-point bake, radius max_dist), as the
// angle atan2(|a x b|, a . b) in degrees; -1 where no raw point lies within
// max_dist or the sample's face was dropped.
template <int LAYOUT>
__global__ void __launch_bounds__(128) k_map_error(TraceArgs A, const uchar4 *__restrict__ rgba,
                                                   const float *__restrict__ luv, int64_t n_lfaces,
                                                   const int32_t *__restrict__ sface, const float *__restrict__ sbary,
                                                   long long n, float *__restrict__ angle) {
    uint2 stack[STACK];
    PointState S;
    const TraceJob &J = A.job0;
    unsigned long long c0 = 0, c1 = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int f = sface[i];
        if (f < 0 || f >= n_lfaces) {
            atomicOr(A.status, AGS_BAD_FACE);
            angle[i] = -1.f;
            continue;
        }
        const int4 fi = J.lface[f];
        if (fi.w & FACE_INVALID) {
            angle[i] = -1.f;
            continue;
        }
        const float b1 = sbary[2 * i], b2 = sbary[2 * i + 1];
        const float3 P0 = f3(J.lpos[fi.x]), P1 = f3(J.lpos[fi.y]), P2 = f3(J.lpos[fi.z]);
        const float3 N0 = f3(J.lnrm[fi.x]), N1 = f3(J.lnrm[fi.y]), N2 = f3(J.lnrm[fi.z]);
        S.job = 0;
        S.base = P0;
        S.off = (P1 - P0) * b1 + (P2 - P0) * b2;
        S.p = P0 + S.off;
        const float3 sv = N0 + (N1 - N0) * b1 + (N2 - N0) * b2;
        const float3 d = sv * (1.0f / sqrtf(dot3(sv, sv)));
        S.d = d;
        S.best.d2 = J.max_dist * J.max_dist;
        S.best.rec = 0;
        S.best.found = false;
        S.cur = 0;
        S.sp = 0;
        S.steps = 0;
        while (step_point_leaves<LAYOUT, false>(A, J, S, stack, c0, c1)) {
        }
        if (!S.best.found) {
            angle[i] = -1.f;
            continue;
        }
        const size_t r3 = 3 * (size_t)S.best.rec;
        const float4 TA = __ldg(&J.tris[r3]), TB = __ldg(&J.tris[r3 + 1]), TC = __ldg(&J.tris[r3 + 2]);
        TriQ q;
        tri_query(rel(S, TA), rel(S, TB), rel(S, TC), q);
        const float3 bw = tri_bary(q);
        const float3 nr = normalize3(f3(__ldg(&J.hnormals[__float_as_int(TA.w)])) * bw.x +
                                     f3(__ldg(&J.hnormals[__float_as_int(TB.w)])) * bw.y +
                                     f3(__ldg(&J.hnormals[__float_as_int(TC.w)])) * bw.z);
        // the bake's frame at the point
        const float4 T0 = J.ltan[3 * f], T1 = J.ltan[3 * f + 1], T2 = J.ltan[3 * f + 2];
        float3 tt = f3(T0) + (f3(T1) - f3(T0)) * b1 + (f3(T2) - f3(T0)) * b2;
        tt = normalize3(tt - d * dot3(tt, d));
        const float3 bb = cross3(d, tt) * T0.w;
        // the texel holding the point's UV
        const float *uv = luv + 6 * (size_t)f;
        const float u = uv[0] + (uv[2] - uv[0]) * b1 + (uv[4] - uv[0]) * b2;
        const float v = uv[1] + (uv[3] - uv[1]) * b1 + (uv[5] - uv[1]) * b2;
        const int x = min(max((int)floorf(u * (float)J.W), 0), J.W - 1);
        const int y = min(max((int)floorf(v * (float)J.H), 0), J.H - 1);
        const uchar4 c8 = rgba[(size_t)y * J.W + x];
        const float3 c = normalize3(make_float3(((float)c8.x - 128.f) * (1.f / 127.f), ((float)c8.y - 128.f) * (1.f / 127.f),
                                                ((float)c8.z - 128.f) * (1.f / 127.f)));
        // a face the UV-reliability filter marks has no usable frame: its normal is d
        const float3 nm = (fi.w & FACE_DEGEN) ? d : normalize3(tt * c.x + bb * c.y + d * c.z);
        const float3 cr = cross3(nm, nr);
        angle[i] = atan2f(sqrtf(dot3(cr, cr)), dot3(nm, nr)) * 57.29577951308232f;
    }
}

}  // namespace

cudaError_t launch_map_error(const TraceLaunch &L, const uint8_t *rgba, const float *luv, int64_t n_lfaces,
                             const int32_t *sface, const float *sbary, long long n, float *angle, cudaStream_t s) {
    TraceArgs A;
    memset(&A, 0, sizeof(A));
    A.job0 = L.job0;
    A.n_jobs = 1;
    A.status = L.status;
    A.max_steps = L.max_steps;
    int dev;
    cudaGetDevice(&dev);
    const unsigned grid = (unsigned)(device_sm_count(dev) * 8);
    const uchar4 *q = reinterpret_cast<const uchar4 *>(rgba);
    if (L.layout == AG_BVH_Q8)
        k_map_error<AG_BVH_Q8><<<grid, 128, 0, s>>>(A, q, luv, n_lfaces, sface, sbary, n, angle);
    else
        k_map_error<AG_BVH_F32><<<grid, 128, 0, s>>>(A, q, luv, n_lfaces, sface, sbary, n, angle);
    return cudaGetLastError();
}

cudaError_t launch_point_distance(const TraceLaunch &L, const float *pts, long long n, float max_dist, float *dist,
                                  int32_t *tri, cudaStream_t s) {
    TraceArgs A;
    memset(&A, 0, sizeof(A));
    A.job0 = L.job0;
    A.n_jobs = 1;
    A.status = L.status;
    A.max_steps = L.max_steps;
    int dev;
    cudaGetDevice(&dev);
    const unsigned grid = (unsigned)(device_sm_count(dev) * 8);
    if (L.layout == AG_BVH_Q8)
        k_point_dist<AG_BVH_Q8><<<grid, 128, 0, s>>>(A, pts, n, max_dist, dist, tri);
    else
        k_point_dist<AG_BVH_F32><<<grid, 128, 0, s>>>(A, pts, n, max_dist, dist, tri);
    return cudaGetLastError();
}

cudaError_t launch_closest(const TraceLaunch &L, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(L.ray_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    TraceArgs A;
    A.job0 = L.job0;
    A.jobs = L.jobs;
    A.job_begin = L.job_begin;
    A.n_jobs = L.n_jobs;
    A.n_rays_dev = L.n_rays_dev;
    A.ray_counter = L.ray_counter;
    A.status = L.status;
    A.max_steps = L.max_steps;
    A.counters = L.counters;
    const bool cnt = L.counters != nullptr;
    if (L.layout == AG_BVH_Q8) return cnt ? launch_one<AG_BVH_Q8, true>(L, A, s) : launch_one<AG_BVH_Q8, false>(L, A, s);
    return cnt ? launch_one<AG_BVH_F32, true>(L, A, s) : launch_one<AG_BVH_F32, false>(L, A, s);
}

}  // namespace ag
