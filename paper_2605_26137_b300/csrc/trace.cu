// Closest-hit traversal and shading (Sec. 6.4, stages two to four: the
// correspondence on the high-poly surface for each texel's world-space
// position with the smooth normal interpolated there, the distance filter,
// the UV-reliability filter and the projection into the texel's tangent
// frame).
//
// One persistent launch serves a whole ray list (one asset or a batch): each
// warp pops 32 consecutive rays from a global counter; rays are texels in
// 8x8-tile order, so a warp's rays are neighbours on the surface.  Per ray:
//   - origin p = v0 + b1 (v1 - v0) + b2 (v2 - v0), kept as (v0, offset) so the
//     triangle test sees it without the rounding of |p|;
//   - direction d = normalize(n0 + b1 (n1 - n0) + b2 (n2 - n0));
//   - closest |t| over the line (both directions), |t| <= max_dist inclusive;
//     8-wide nodes, children ordered near-to-far by the nearest |t| of their
//     box interval (sorting network), a per-thread stack of (ref, dist);
//   - box tests against outward-rounded boxes with an origin padded by a few
//     ulps, widened relative intervals: never reject a box the exact line
//     meets;
//   - watertight ray/triangle test (Woop, Benthin, Wald 2013) in FP32 with
//     the three edge functions in explicit round-to-nearest products, so a
//     shared edge gets exactly opposite values from both triangles and zero
//     counts as inside;
//   - ties: equal |t| prefers t >= 0, equal t the lower original id.
// The backward variant replaces the shading with the adjoint of the loss.
#include "traverse.cuh"

namespace ag {
namespace {

struct Ray {
    // exact-origin triangle test: permuted axes, shear, origin as base + offset
    int kx, ky, kz;
    float Sx, Sy, Sz;
    float bx, by, bz;
    float ox, oy, oz;
    // box test: rounded origin, 1/d with zero components made tiny, direction signs
    float px, py, pz;
    float ix, iy, iz;
    bool nx, ny, nz;
};

__device__ __forceinline__ float pick(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ Ray make_ray(float3 base, float3 off, float3 d) {
    Ray r;
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    r.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    r.kx = r.kz == 2 ? 0 : r.kz + 1;
    r.ky = r.kx == 2 ? 0 : r.kx + 1;
    float dz = pick(d, r.kz);
    if (dz < 0.f) { int t = r.kx; r.kx = r.ky; r.ky = t; }
    r.Sx = pick(d, r.kx) / dz;
    r.Sy = pick(d, r.ky) / dz;
    r.Sz = 1.0f / dz;
    r.bx = pick(base, r.kx); r.by = pick(base, r.ky); r.bz = pick(base, r.kz);
    r.ox = pick(off, r.kx); r.oy = pick(off, r.ky); r.oz = pick(off, r.kz);
    float3 p = base + off;
    r.px = p.x; r.py = p.y; r.pz = p.z;
    float3 dd = d;
    if (fabsf(dd.x) < 1e-30f) dd.x = copysignf(1e-30f, dd.x);
    if (fabsf(dd.y) < 1e-30f) dd.y = copysignf(1e-30f, dd.y);
    if (fabsf(dd.z) < 1e-30f) dd.z = copysignf(1e-30f, dd.z);
    r.ix = 1.0f / dd.x; r.iy = 1.0f / dd.y; r.iz = 1.0f / dd.z;
    r.nx = r.ix < 0.f; r.ny = r.iy < 0.f; r.nz = r.iz < 0.f;
    return r;
}

// vertex in ray space: (v - base) - offset, permuted and sheared
__device__ __forceinline__ void xform(const Ray &r, float4 v, float &X, float &Y, float &Z) {
    float3 a = make_float3(v.x, v.y, v.z);
    float ax = __fsub_rn(__fsub_rn(pick(a, r.kx), r.bx), r.ox);
    float ay = __fsub_rn(__fsub_rn(pick(a, r.ky), r.by), r.oy);
    float az = __fsub_rn(__fsub_rn(pick(a, r.kz), r.bz), r.oz);
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

__device__ __forceinline__ void test_tri(const Ray &r, const float4 *__restrict__ tris,
                                         const int32_t *__restrict__ tri_ids, uint32_t rec, Best &b) {
    float4 A = __ldg(&tris[3 * (size_t)rec]), B = __ldg(&tris[3 * (size_t)rec + 1]), C = __ldg(&tris[3 * (size_t)rec + 2]);
    float Ax, Ay, Az, Bx, By, Bz, Cx, Cy, Cz;
    xform(r, A, Ax, Ay, Az);
    xform(r, B, Bx, By, Bz);
    xform(r, C, Cx, Cy, Cz);
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
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

template <int LAYOUT>
struct NodeOps;

// 80-byte quantised node.  Per node and axis the child planes become one FMA
// each: t(q) = q * a + b with a = 2^e / d and b = (origin - p) / d.  The
// intervals are widened by eps = 2^-21 (|origin| + |p| + 255 * 2^e) / |d|,
// which bounds every rounding on the way (decoded plane, a, b, the FMA, the
// rounded ray origin) by a factor of at least 4, so a box the exact line
// meets is never rejected.
template <>
struct NodeOps<AG_BVH_Q8> {
    static __device__ __forceinline__ void visit(const void *nodes, uint32_t idx, const Ray &r, float lim, Next &nx,
                                                 uint2 *stack, int &sp, unsigned *status) {
        const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const QNode *>(nodes) + idx);
        uint4 w0 = __ldg(p), w1 = __ldg(p + 1), w2 = __ldg(p + 2), w3 = __ldg(p + 3), w4 = __ldg(p + 4);
        float ox = __uint_as_float(w0.x), oy = __uint_as_float(w0.y), oz = __uint_as_float(w0.z);
        float sx = __uint_as_float((w0.w & 0xffu) << 23);
        float sy = __uint_as_float(((w0.w >> 8) & 0xffu) << 23);
        float sz = __uint_as_float(((w0.w >> 16) & 0xffu) << 23);
        float ax = sx * r.ix, ay = sy * r.iy, az = sz * r.iz;
        float bx = (ox - r.px) * r.ix, by = (oy - r.py) * r.iy, bz = (oz - r.pz) * r.iz;
        float ex = EPS_REL * (fabsf(ox) + fabsf(r.px) + 255.f * sx) * fabsf(r.ix);
        float ey = EPS_REL * (fabsf(oy) + fabsf(r.py) + 255.f * sy) * fabsf(r.iy);
        float ez = EPS_REL * (fabsf(oz) + fabsf(r.pz) + 255.f * sz) * fabsf(r.iz);
        float bnx = bx - ex, bfx = bx + ex, bny = by - ey, bfy = by + ey, bnz = bz - ez, bfz = bz + ez;
        // near-plane bytes: lo for d > 0, hi for d < 0
        uint32_t nx0 = r.nx ? w3.z : w2.x, nx1 = r.nx ? w3.w : w2.y, fx0 = r.nx ? w2.x : w3.z, fx1 = r.nx ? w2.y : w3.w;
        uint32_t ny0 = r.ny ? w4.x : w2.z, ny1 = r.ny ? w4.y : w2.w, fy0 = r.ny ? w2.z : w4.x, fy1 = r.ny ? w2.w : w4.y;
        uint32_t nz0 = r.nz ? w4.z : w3.x, nz1 = r.nz ? w4.w : w3.y, fz0 = r.nz ? w3.x : w4.z, fz1 = r.nz ? w3.y : w4.w;
        uint32_t child_base = w1.x, tri_base = w1.y;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int k = c & 3;
            const bool hi = c >= 4;
            uint32_t m = ((hi ? w1.w : w1.z) >> (8 * k)) & 0xffu;
            float tnx = __fmaf_rn(byte_f(hi ? nx1 : nx0, k), ax, bnx);
            float tfx = __fmaf_rn(byte_f(hi ? fx1 : fx0, k), ax, bfx);
            float tny = __fmaf_rn(byte_f(hi ? ny1 : ny0, k), ay, bny);
            float tfy = __fmaf_rn(byte_f(hi ? fy1 : fy0, k), ay, bfy);
            float tnz = __fmaf_rn(byte_f(hi ? nz1 : nz0, k), az, bnz);
            float tfz = __fmaf_rn(byte_f(hi ? fz1 : fz0, k), az, bfz);
            float te = fmaxf(fmaxf(tnx, tny), tnz);
            float tx = fminf(fminf(tfx, tfy), tfz);
            if (m != 0 && te <= tx && te <= lim && tx >= -lim)
                offer(child_ref(m, child_base, tri_base), fmaxf(fmaxf(te, -tx), 0.f), nx, stack, sp, status);
        }
    }
};

// 208-byte node with exact FP32 child boxes: t = plane / d - p / d, widened by
// eps = 2^-21 (scene bound + |p|) / |d| per axis.
template <>
struct NodeOps<AG_BVH_F32> {
    static __device__ __forceinline__ void visit(const void *nodes, uint32_t idx, const Ray &r, float lim, Next &nx,
                                                 uint2 *stack, int &sp, unsigned *status, float scene_abs) {
        const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const FNode *>(nodes) + idx);
        uint4 h = __ldg(p);
        uint32_t child_base = h.x, tri_base = h.y;
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
                float plx = __uint_as_float(r.nx ? HX[k] : LX[k]), pfx = __uint_as_float(r.nx ? LX[k] : HX[k]);
                float ply = __uint_as_float(r.ny ? HY[k] : LY[k]), pfy = __uint_as_float(r.ny ? LY[k] : HY[k]);
                float plz = __uint_as_float(r.nz ? HZ[k] : LZ[k]), pfz = __uint_as_float(r.nz ? LZ[k] : HZ[k]);
                float te = fmaxf(fmaxf(__fmaf_rn(plx, r.ix, cnx), __fmaf_rn(ply, r.iy, cny)), __fmaf_rn(plz, r.iz, cnz));
                float tx = fminf(fminf(__fmaf_rn(pfx, r.ix, cfx), __fmaf_rn(pfy, r.iy, cfy)), __fmaf_rn(pfz, r.iz, cfz));
                if (m != 0 && te <= tx && te <= lim && tx >= -lim)
                    offer(child_ref(m, child_base, tri_base), fmaxf(fmaxf(te, -tx), 0.f), nx, stack, sp, status);
            }
        }
    }
};

// Per-lane traversal state of one ray.
struct RayState {
    int job;
    int texel, face;
    float b1, b2, sl;
    int4 fi;
    float3 d;
    Ray ray;
    Best best;
    uint32_t cur;
    int sp, steps;
};

__device__ __forceinline__ void setup_ray(const TraceArgs &A, long long r, RayState &S) {
    int j = 0;
    long long local = r;
    if (A.n_jobs > 1) {
        int lo = 0, hi = A.n_jobs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (A.job_begin[mid] <= r) lo = mid; else hi = mid - 1;
        }
        j = lo;
        local = r - A.job_begin[j];
    }
    const TraceJob &J = job_of(A, j);
    int4 rr = J.rays[local];
    S.job = j;
    S.texel = rr.x;
    S.face = rr.y;
    S.b1 = __int_as_float(rr.z);
    S.b2 = __int_as_float(rr.w);
    S.fi = J.lface[S.face];
    float3 P0 = f3(J.lpos[S.fi.x]), P1 = f3(J.lpos[S.fi.y]), P2 = f3(J.lpos[S.fi.z]);
    float3 N0 = f3(J.lnrm[S.fi.x]), N1 = f3(J.lnrm[S.fi.y]), N2 = f3(J.lnrm[S.fi.z]);
    float3 off = (P1 - P0) * S.b1 + (P2 - P0) * S.b2;
    float3 sv = N0 + (N1 - N0) * S.b1 + (N2 - N0) * S.b2;
    S.sl = sqrtf(dot3(sv, sv));
    S.d = sv * (1.0f / S.sl);
    S.ray = make_ray(P0, off, S.d);
    S.best.t = 0.f; S.best.babs = J.max_dist; S.best.rec = 0; S.best.found = false;
    S.best.U = S.best.V = S.best.W = 0.f; S.best.det = 1.f;
    S.cur = 0;   // root
    S.sp = 0;
    S.steps = 0;
}

// One traversal step (a node visit or a leaf's triangles); false when done.
template <int LAYOUT, bool COUNT>
__device__ __forceinline__ bool step(const TraceArgs &A, const TraceJob &J, RayState &S, uint2 *stack,
                                     unsigned long long &c_nodes, unsigned long long &c_tris) {
    Next nx;
    nx.has = false;
    nx.ref = 0;
    nx.dist = 0.f;
    if (ref_is_leaf(S.cur)) {
        uint32_t first = ref_first(S.cur);
        int cnt = ref_count(S.cur);
        for (int k = 0; k < cnt; ++k) test_tri(S.ray, J.tris, J.tri_ids, first + k, S.best);
        if (COUNT) c_tris += cnt;
    } else {
        if (LAYOUT == AG_BVH_Q8)
            NodeOps<AG_BVH_Q8>::visit(J.nodes, S.cur, S.ray, S.best.babs, nx, stack, S.sp, A.status);
        else
            NodeOps<AG_BVH_F32>::visit(J.nodes, S.cur, S.ray, S.best.babs, nx, stack, S.sp, A.status, J.scene_abs);
        if (COUNT) ++c_nodes;
    }
    if (nx.has) {
        S.cur = nx.ref;
    } else {
        bool done = true;
        while (S.sp > 0) {
            uint2 e = stack[--S.sp];
            if (__uint_as_float(e.y) <= S.best.babs) { S.cur = e.x; done = false; break; }
        }
        if (done) return false;
    }
    if (++S.steps > A.max_steps) {
        atomicOr(A.status, AGS_STEP_CAP);
        return false;
    }
    return true;
}

struct LossAcc {
    float t, n, c;
    int job;
};

__device__ __forceinline__ void flush_loss(const TraceArgs &A, LossAcc &L) {
    if (L.job >= 0 && L.c > 0.f) {
        float *la = A.n_jobs > 1 ? A.jobs[L.job].loss_acc : A.job0.loss_acc;
        atomicAdd(&la[0], L.t);
        atomicAdd(&la[1], L.n);
        atomicAdd(&la[2], L.c);
    }
    L.t = L.n = L.c = 0.f;
}

// Shading (forward) or the adjoint of the loss (backward) of a finished ray.
template <bool BWD>
__device__ __forceinline__ void finish(const TraceArgs &A, RayState &S, LossAcc &L) {
    const TraceJob &J = job_of(A, S.job);
    const bool hit = S.best.found;
    const float3 d = S.d;
    float3 nh = make_float3(0.f, 0.f, 1.f);
    float bA = 0.f, bB = 0.f, bC = 0.f;
    float4 TA = make_float4(0, 0, 0, 0), TB = TA, TC = TA;
    float3 nA = make_float3(0, 0, 0), nB = nA, nC = nA;
    if (hit) {
        float inv = 1.0f / S.best.det;
        bA = S.best.U * inv; bB = S.best.V * inv; bC = S.best.W * inv;
        TA = __ldg(&J.tris[3 * (size_t)S.best.rec]);
        TB = __ldg(&J.tris[3 * (size_t)S.best.rec + 1]);
        TC = __ldg(&J.tris[3 * (size_t)S.best.rec + 2]);
        nA = f3(__ldg(&J.hnormals[__float_as_int(TA.w)]));
        nB = f3(__ldg(&J.hnormals[__float_as_int(TB.w)]));
        nC = f3(__ldg(&J.hnormals[__float_as_int(TC.w)]));
        nh = normalize3(nA * bA + nB * bB + nC * bC);
    }
    if (!BWD) {
        store_forward(J, S.texel, S.face, S.fi, S.b1, S.b2, d, hit, nh, S.best.t, hit ? J.tri_ids[S.best.rec] : -1);
    } else if (hit) {
        // adjoint of t^2 + lambda (1 - nh . d), hit triangle held fixed
        const float lam = J.lambda;
        const float t = S.best.t;
        float3 A3 = f3(TA), B3 = f3(TB), C3 = f3(TC);
        float3 Nh = cross3(B3 - A3, C3 - A3);
        float nn = dot3(Nh, Nh), dn = dot3(d, Nh);
        float3 m = nA * bA + nB * bB + nC * bC;
        float ml = sqrtf(dot3(m, m));
        float3 g_nh = d * (-lam);
        float3 g_m = (g_nh - nh * dot3(nh, g_nh)) * (1.0f / ml);
        float gbA = dot3(nA, g_m), gbB = dot3(nB, g_m), gbC = dot3(nC, g_m);
        float inn = 1.0f / nn;
        float3 g_x = (cross3(Nh, C3 - B3) * gbA + cross3(Nh, A3 - C3) * gbB + cross3(Nh, B3 - A3) * gbC) * inn;
        float g_tt = 2.f * t + dot3(g_x, d);
        float3 g_p = g_x - Nh * (g_tt / dn);
        float3 g_d = nh * (-lam) + g_p * t;
        float3 g_s = (g_d - d * dot3(d, g_d)) * (1.0f / S.sl);
        float bw[3] = {1.f - S.b1 - S.b2, S.b1, S.b2};
        int vid[3] = {S.fi.x, S.fi.y, S.fi.z};
#pragma unroll
        for (int k = 0; k < 3 && J.g_pos; ++k) {
            atomicAdd(&J.g_pos[3 * vid[k]], g_p.x * bw[k]);
            atomicAdd(&J.g_pos[3 * vid[k] + 1], g_p.y * bw[k]);
            atomicAdd(&J.g_pos[3 * vid[k] + 2], g_p.z * bw[k]);
            atomicAdd(&J.g_nrm[3 * vid[k]], g_s.x * bw[k]);
            atomicAdd(&J.g_nrm[3 * vid[k] + 1], g_s.y * bw[k]);
            atomicAdd(&J.g_nrm[3 * vid[k] + 2], g_s.z * bw[k]);
        }
        if (L.job != S.job) {
            flush_loss(A, L);
            L.job = S.job;
        }
        L.t += t * t;
        L.n += 1.f - dot3(nh, d);
        L.c += 1.f;
    }
}

// Schedule "batch": a warp takes 32 consecutive rays and runs all of them to
// completion before taking the next 32.
template <int LAYOUT, bool BWD, bool COUNT>
__global__ void __launch_bounds__(256) k_trace(TraceArgs A) {
    const int lane = threadIdx.x & 31;
    const long long n_total = *A.n_rays_dev;
    unsigned long long c_nodes = 0, c_tris = 0, c_rays = 0, c_hits = 0;
    LossAcc L = {0.f, 0.f, 0.f, -1};
    uint2 stack[STACK];
    RayState S;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(A.ray_counter, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= n_total) break;
        long long r = (long long)base + lane;
        if (r >= n_total) continue;
        setup_ray(A, r, S);
        if (COUNT) ++c_rays;
        const TraceJob &J = job_of(A, S.job);
        while (step<LAYOUT, COUNT>(A, J, S, stack, c_nodes, c_tris)) {
        }
        if (COUNT && S.best.found) ++c_hits;
        finish<BWD>(A, S, L);
    }
    if (BWD) flush_loss(A, L);
    flush_counters<COUNT>(A, c_rays, c_nodes, c_tris, c_hits);
}

// Schedule "refill": lanes take new rays as they finish.  When at least
// REFILL_MIN lanes of the warp are idle (or all are), the idle lanes shade
// their finished rays and take new ones from the global counter with one
// warp-aggregated atomic, so shading and setup run for many lanes at once and
// no lane waits for the slowest ray of a 32-ray batch.
template <int LAYOUT, bool BWD, bool COUNT>
__global__ void __launch_bounds__(256) k_trace_refill(TraceArgs A, int refill_min) {
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long n_total = *A.n_rays_dev;
    unsigned long long c_nodes = 0, c_tris = 0, c_rays = 0, c_hits = 0;
    LossAcc L = {0.f, 0.f, 0.f, -1};
    uint2 stack[STACK];
    RayState S;
    bool active = false, pending = false, drained = false;
    for (;;) {
        unsigned act = __ballot_sync(0xffffffffu, active);
        int idle = 32 - __popc(act);
        if (idle >= refill_min || act == 0) {
            if (pending) {
                if (COUNT && S.best.found) ++c_hits;
                finish<BWD>(A, S, L);
                pending = false;
            }
            if (!drained) {
                unsigned want = ~act;
                unsigned long long base = 0;
                int leader = __ffs(want) - 1;
                if (lane == leader) base = atomicAdd(A.ray_counter, (unsigned long long)__popc(want));
                base = __shfl_sync(0xffffffffu, base, leader);
                if ((long long)base + __popc(want) >= n_total) drained = true;
                if (!active) {
                    long long r = (long long)base + __popc(want & lt_mask);
                    if (r < n_total) {
                        setup_ray(A, r, S);
                        if (COUNT) ++c_rays;
                        active = true;
                    }
                }
            }
            if (__ballot_sync(0xffffffffu, active) == 0) break;
        }
        if (active) {
            const TraceJob &J = job_of(A, S.job);
            if (!step<LAYOUT, COUNT>(A, J, S, stack, c_nodes, c_tris)) {
                active = false;
                pending = true;
            }
        }
    }
    if (BWD) flush_loss(A, L);
    flush_counters<COUNT>(A, c_rays, c_nodes, c_tris, c_hits);
}

template <int LAYOUT, bool BWD, bool COUNT>
cudaError_t launch_one(const TraceLaunch &L, const TraceArgs &A, cudaStream_t s) {
    int dev;
    cudaGetDevice(&dev);
    int block = L.block_size > 0 ? (L.block_size > 256 ? 256 : L.block_size) : 128;
    int bps = L.blocks_per_sm > 0 ? L.blocks_per_sm : 0;
    const bool refill = L.schedule == AG_SCHED_REFILL;
    if (bps == 0) {
        int occ = 0;
        if (refill)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_refill<LAYOUT, BWD, COUNT>, block, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace<LAYOUT, BWD, COUNT>, block, 0);
        bps = occ > 0 ? occ : 1;
    }
    unsigned grid = (unsigned)(device_sm_count(dev) * bps);
    if (refill)
        k_trace_refill<LAYOUT, BWD, COUNT><<<grid, block, 0, s>>>(A, 8);
    else
        k_trace<LAYOUT, BWD, COUNT><<<grid, block, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_trace(const TraceLaunch &L, cudaStream_t s) {
    if (L.query == AG_QUERY_CLOSEST) return launch_closest(L, s);
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
    if (L.layout == AG_BVH_Q8) {
        if (L.backward) return launch_one<AG_BVH_Q8, true, false>(L, A, s);
        return cnt ? launch_one<AG_BVH_Q8, false, true>(L, A, s) : launch_one<AG_BVH_Q8, false, false>(L, A, s);
    }
    if (L.backward) return launch_one<AG_BVH_F32, true, false>(L, A, s);
    return cnt ? launch_one<AG_BVH_F32, false, true>(L, A, s) : launch_one<AG_BVH_F32, false, false>(L, A, s);
}

}  // namespace ag
