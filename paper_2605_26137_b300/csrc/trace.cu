// Closest-hit traversal and shading (Sec. 6.4, stages two to four: "locates,
// for each texel's world-space position, the ... high-poly surface and
// retrieves its interpolated smooth normal", the distance filter, the
// UV-reliability filter and the projection into the texel's tangent frame).
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
#include "ag_internal.cuh"

namespace ag {
namespace {

constexpr int STACK = 64;
constexpr float BOX_REL = 9.5367431640625e-07f;  // 2^-20 relative interval widening

struct Ray {
    int kx, ky, kz;
    float Sx, Sy, Sz;
    float bx, by, bz;     // base (vertex 0 of the low face), permuted
    float ox, oy, oz;     // offset from base, permuted
    float3 plo, phi;      // padded origins for box planes (lo plane, hi plane)
    float3 inv;           // 1/d, zero components replaced by tiny values
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
    float m = fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z)));
    float dl = m * 9.5367431640625e-07f + 1e-30f;   // ~8 ulp of the largest coordinate
    r.plo = make_float3(p.x + dl, p.y + dl, p.z + dl);
    r.phi = make_float3(p.x - dl, p.y - dl, p.z - dl);
    float3 dd = d;
    if (fabsf(dd.x) < 1e-30f) dd.x = copysignf(1e-30f, dd.x);
    if (fabsf(dd.y) < 1e-30f) dd.y = copysignf(1e-30f, dd.y);
    if (fabsf(dd.z) < 1e-30f) dd.z = copysignf(1e-30f, dd.z);
    r.inv = make_float3(1.0f / dd.x, 1.0f / dd.y, 1.0f / dd.z);
    return r;
}

// line interval of a box; returns the nearest |t| in [-lim, lim] or +inf
__device__ __forceinline__ float box_dist(const Ray &r, float lx, float ly, float lz, float hx, float hy, float hz,
                                          float lim) {
    float ax = (lx - r.plo.x) * r.inv.x, bx = (hx - r.phi.x) * r.inv.x;
    float ay = (ly - r.plo.y) * r.inv.y, by = (hy - r.phi.y) * r.inv.y;
    float az = (lz - r.plo.z) * r.inv.z, bz = (hz - r.phi.z) * r.inv.z;
    float t0 = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fminf(az, bz));
    float t1 = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fmaxf(az, bz));
    t0 = t0 - fabsf(t0) * BOX_REL;
    t1 = t1 + fabsf(t1) * BOX_REL;
    if (!(t0 <= t1) || t0 > lim || t1 < -lim) return __int_as_float(0x7f800000);
    return t0 > 0.f ? t0 : (t1 < 0.f ? -t1 : 0.f);
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

template <>
struct NodeOps<AG_BVH_Q8> {
    // returns child refs / dists (dist = +inf for none)
    static __device__ __forceinline__ void visit(const void *nodes, uint32_t idx, const Ray &r, float lim,
                                                 float dist[8], uint32_t ref[8]) {
        const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const QNode *>(nodes) + idx);
        uint4 w0 = __ldg(p), w1 = __ldg(p + 1), w2 = __ldg(p + 2), w3 = __ldg(p + 3), w4 = __ldg(p + 4);
        float ox = __uint_as_float(w0.x), oy = __uint_as_float(w0.y), oz = __uint_as_float(w0.z);
        float sx = __uint_as_float((w0.w & 0xffu) << 23);
        float sy = __uint_as_float(((w0.w >> 8) & 0xffu) << 23);
        float sz = __uint_as_float(((w0.w >> 16) & 0xffu) << 23);
        uint32_t child_base = w1.x, tri_base = w1.y;
        uint32_t meta_lo = w1.z, meta_hi = w1.w;
        uint32_t qlx[2] = {w2.x, w2.y}, qly[2] = {w2.z, w2.w};
        uint32_t qlz[2] = {w3.x, w3.y}, qhx[2] = {w3.z, w3.w};
        uint32_t qhy[2] = {w4.x, w4.y}, qhz[2] = {w4.z, w4.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            int wd = c >> 2, sh = (c & 3) * 8;
            uint32_t m = ((c < 4 ? meta_lo : meta_hi) >> sh) & 0xffu;
            float lx = __fmaf_rn((float)((qlx[wd] >> sh) & 0xffu), sx, ox);
            float ly = __fmaf_rn((float)((qly[wd] >> sh) & 0xffu), sy, oy);
            float lz = __fmaf_rn((float)((qlz[wd] >> sh) & 0xffu), sz, oz);
            float hx = __fmaf_rn((float)((qhx[wd] >> sh) & 0xffu), sx, ox);
            float hy = __fmaf_rn((float)((qhy[wd] >> sh) & 0xffu), sy, oy);
            float hz = __fmaf_rn((float)((qhz[wd] >> sh) & 0xffu), sz, oz);
            float dd = box_dist(r, lx, ly, lz, hx, hy, hz, lim);
            if (m == 0) dd = __int_as_float(0x7f800000);
            dist[c] = dd;
            ref[c] = (m & 0x80u) ? child_base + (m & 0x7fu)
                                 : ref_leaf(tri_base + (m & 31u), (int)((m >> 5) & 3u) == 0 ? 1 : (int)((m >> 5) & 3u));
        }
    }
};

template <>
struct NodeOps<AG_BVH_F32> {
    static __device__ __forceinline__ void visit(const void *nodes, uint32_t idx, const Ray &r, float lim,
                                                 float dist[8], uint32_t ref[8]) {
        const FNode *nd = static_cast<const FNode *>(nodes) + idx;
        const uint4 *p = reinterpret_cast<const uint4 *>(nd);
        uint4 h = __ldg(p);
        uint32_t child_base = h.x, tri_base = h.y, meta_lo = h.z, meta_hi = h.w;
        float lo[3][8], hi[3][8];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            uint4 w = __ldg(p + 1 + q);
            float *dst = (q < 6) ? &lo[q / 2][(q & 1) * 4] : &hi[(q - 6) / 2][(q & 1) * 4];
            dst[0] = __uint_as_float(w.x); dst[1] = __uint_as_float(w.y);
            dst[2] = __uint_as_float(w.z); dst[3] = __uint_as_float(w.w);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t m = ((c < 4 ? meta_lo : meta_hi) >> ((c & 3) * 8)) & 0xffu;
            float dd = box_dist(r, lo[0][c], lo[1][c], lo[2][c], hi[0][c], hi[1][c], hi[2][c], lim);
            if (m == 0) dd = __int_as_float(0x7f800000);
            dist[c] = dd;
            ref[c] = (m & 0x80u) ? child_base + (m & 0x7fu)
                                 : ref_leaf(tri_base + (m & 31u), (int)((m >> 5) & 3u) == 0 ? 1 : (int)((m >> 5) & 3u));
        }
    }
};

__device__ __forceinline__ void cswap(float &da, uint32_t &ra, float &db, uint32_t &rb) {
    bool sw = db < da;
    float td = sw ? db : da;
    uint32_t tr = sw ? rb : ra;
    db = sw ? da : db;
    rb = sw ? ra : rb;
    da = td;
    ra = tr;
}

__device__ __forceinline__ void sort8(float d[8], uint32_t r[8]) {
    cswap(d[0], r[0], d[1], r[1]); cswap(d[2], r[2], d[3], r[3]);
    cswap(d[4], r[4], d[5], r[5]); cswap(d[6], r[6], d[7], r[7]);
    cswap(d[0], r[0], d[2], r[2]); cswap(d[1], r[1], d[3], r[3]);
    cswap(d[4], r[4], d[6], r[6]); cswap(d[5], r[5], d[7], r[7]);
    cswap(d[1], r[1], d[2], r[2]); cswap(d[5], r[5], d[6], r[6]);
    cswap(d[0], r[0], d[4], r[4]); cswap(d[3], r[3], d[7], r[7]);
    cswap(d[1], r[1], d[5], r[5]); cswap(d[2], r[2], d[6], r[6]);
    cswap(d[1], r[1], d[4], r[4]); cswap(d[3], r[3], d[6], r[6]);
    cswap(d[2], r[2], d[4], r[4]); cswap(d[3], r[3], d[5], r[5]);
    cswap(d[3], r[3], d[4], r[4]);
}

struct TraceArgs {
    TraceJob job0;
    const TraceJob *jobs;
    const long long *job_begin;
    int n_jobs;
    const long long *n_rays_dev;
    unsigned long long *ray_counter;
    unsigned *status;
    int max_steps;
    unsigned long long *counters;
};

template <int LAYOUT, bool BWD, bool COUNT>
__global__ void __launch_bounds__(256) k_trace(TraceArgs A) {
    const int lane = threadIdx.x & 31;
    const long long n_total = *A.n_rays_dev;
    unsigned long long c_nodes = 0, c_tris = 0, c_rays = 0, c_hits = 0;
    float acc_t = 0.f, acc_n = 0.f, acc_c = 0.f;
    int acc_job = -1;
    uint2 stack[STACK];
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(A.ray_counter, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= n_total) break;
        long long r = (long long)base + lane;
        if (r >= n_total) continue;
        int j = 0;
        if (A.n_jobs > 1) {
            int lo = 0, hi = A.n_jobs - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (A.job_begin[mid] <= r) lo = mid; else hi = mid - 1;
            }
            j = lo;
        }
        const TraceJob &J = A.n_jobs > 1 ? A.jobs[j] : A.job0;
        long long local = r - (A.n_jobs > 1 ? A.job_begin[j] : 0);
        int4 rr = J.rays[local];
        const int texel = rr.x, face = rr.y;
        const float b1 = __int_as_float(rr.z), b2 = __int_as_float(rr.w);
        int4 fi = J.lface[face];
        float3 P0 = f3(J.lpos[fi.x]), P1 = f3(J.lpos[fi.y]), P2 = f3(J.lpos[fi.z]);
        float3 N0 = f3(J.lnrm[fi.x]), N1 = f3(J.lnrm[fi.y]), N2 = f3(J.lnrm[fi.z]);
        float3 off = (P1 - P0) * b1 + (P2 - P0) * b2;
        float3 s = N0 + (N1 - N0) * b1 + (N2 - N0) * b2;
        float sl = sqrtf(dot3(s, s));
        float3 d = s * (1.0f / sl);
        Ray ray = make_ray(P0, off, d);
        Best best;
        best.t = 0.f; best.babs = J.max_dist; best.rec = 0; best.found = false;
        best.U = best.V = best.W = 0.f; best.det = 1.f;
        int sp = 0;
        uint32_t cur = 0;   // root
        int steps = 0;
        if (COUNT) ++c_rays;
        for (;;) {
            if (ref_is_leaf(cur)) {
                uint32_t first = ref_first(cur);
                int cnt = ref_count(cur);
                for (int k = 0; k < cnt; ++k) test_tri(ray, J.tris, J.tri_ids, first + k, best);
                if (COUNT) c_tris += cnt;
            } else {
                float dist[8];
                uint32_t ref[8];
                NodeOps<LAYOUT>::visit(J.nodes, cur, ray, best.babs, dist, ref);
                if (COUNT) ++c_nodes;
                sort8(dist, ref);
#pragma unroll
                for (int c = 7; c >= 0; --c) {
                    if (dist[c] <= best.babs) {
                        if (sp < STACK) {
                            stack[sp++] = make_uint2(ref[c], __float_as_uint(dist[c]));
                        } else {
                            atomicOr(A.status, AGS_STACK);
                        }
                    }
                }
            }
            bool done = false;
            for (;;) {
                if (sp == 0) { done = true; break; }
                uint2 e = stack[--sp];
                if (__uint_as_float(e.y) <= best.babs) { cur = e.x; break; }
            }
            if (done) break;
            if (++steps > A.max_steps) { atomicOr(A.status, AGS_STEP_CAP); break; }
        }
        const bool hit = best.found;
        if (COUNT && hit) ++c_hits;
        float3 nh = make_float3(0.f, 0.f, 1.f);
        float bA = 0.f, bB = 0.f, bC = 0.f;
        float4 TA = make_float4(0, 0, 0, 0), TB = TA, TC = TA;
        if (hit) {
            float inv = 1.0f / best.det;
            bA = best.U * inv; bB = best.V * inv; bC = best.W * inv;
            TA = __ldg(&J.tris[3 * (size_t)best.rec]);
            TB = __ldg(&J.tris[3 * (size_t)best.rec + 1]);
            TC = __ldg(&J.tris[3 * (size_t)best.rec + 2]);
            float3 nA = f3(__ldg(&J.hnormals[__float_as_int(TA.w)]));
            float3 nB = f3(__ldg(&J.hnormals[__float_as_int(TB.w)]));
            float3 nC = f3(__ldg(&J.hnormals[__float_as_int(TC.w)]));
            nh = normalize3(nA * bA + nB * bB + nC * bC);
        }
        if (!BWD) {
            float3 nts = make_float3(0.f, 0.f, 1.f);
            if (hit && !(fi.w & FACE_DEGEN)) {
                float4 T0 = J.ltan[3 * face], T1 = J.ltan[3 * face + 1], T2 = J.ltan[3 * face + 2];
                float3 tt = f3(T0) + (f3(T1) - f3(T0)) * b1 + (f3(T2) - f3(T0)) * b2;
                tt = normalize3(tt - d * dot3(tt, d));
                float3 bb = cross3(d, tt) * T0.w;
                nts = make_float3(dot3(nh, tt), dot3(nh, bb), dot3(nh, d));
            }
            J.ntsd[texel] = make_float4(nts.x, nts.y, nts.z, hit ? best.t : 0.f);
            J.mask[texel] = hit ? 1 : 0;
            if (J.hit_tri) J.hit_tri[texel] = hit ? J.tri_ids[best.rec] : -1;
            if (J.hit_t) J.hit_t[texel] = hit ? best.t : 0.f;
        } else if (hit) {
            // adjoint of t^2 + lambda (1 - nh . d), hit triangle held fixed
            const float lam = J.lambda;
            const float t = best.t;
            float3 A3 = f3(TA), B3 = f3(TB), C3 = f3(TC);
            float3 Nh = cross3(B3 - A3, C3 - A3);
            float nn = dot3(Nh, Nh), dn = dot3(d, Nh);
            float3 m = f3(__ldg(&J.hnormals[__float_as_int(TA.w)])) * bA +
                       f3(__ldg(&J.hnormals[__float_as_int(TB.w)])) * bB +
                       f3(__ldg(&J.hnormals[__float_as_int(TC.w)])) * bC;
            float ml = sqrtf(dot3(m, m));
            float3 g_nh = d * (-lam);
            float3 g_m = (g_nh - nh * dot3(nh, g_nh)) * (1.0f / ml);
            float gbA = dot3(f3(__ldg(&J.hnormals[__float_as_int(TA.w)])), g_m);
            float gbB = dot3(f3(__ldg(&J.hnormals[__float_as_int(TB.w)])), g_m);
            float gbC = dot3(f3(__ldg(&J.hnormals[__float_as_int(TC.w)])), g_m);
            float inn = 1.0f / nn;
            float3 g_x = (cross3(Nh, C3 - B3) * gbA + cross3(Nh, A3 - C3) * gbB + cross3(Nh, B3 - A3) * gbC) * inn;
            float g_tt = 2.f * t + dot3(g_x, d);
            float3 g_p = g_x - Nh * (g_tt / dn);
            float3 g_d = nh * (-lam) + g_p * t;
            float3 g_s = (g_d - d * dot3(d, g_d)) * (1.0f / sl);
            float bw[3] = {1.f - b1 - b2, b1, b2};
            int vid[3] = {fi.x, fi.y, fi.z};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                atomicAdd(&J.g_pos[3 * vid[k]], g_p.x * bw[k]);
                atomicAdd(&J.g_pos[3 * vid[k] + 1], g_p.y * bw[k]);
                atomicAdd(&J.g_pos[3 * vid[k] + 2], g_p.z * bw[k]);
                atomicAdd(&J.g_nrm[3 * vid[k]], g_s.x * bw[k]);
                atomicAdd(&J.g_nrm[3 * vid[k] + 1], g_s.y * bw[k]);
                atomicAdd(&J.g_nrm[3 * vid[k] + 2], g_s.z * bw[k]);
            }
            if (acc_job != j && acc_job >= 0) {
                float *la = A.n_jobs > 1 ? A.jobs[acc_job].loss_acc : A.job0.loss_acc;
                atomicAdd(&la[0], acc_t);
                atomicAdd(&la[1], acc_n);
                atomicAdd(&la[2], acc_c);
                acc_t = acc_n = acc_c = 0.f;
            }
            acc_job = j;
            acc_t += t * t;
            acc_n += 1.f - dot3(nh, d);
            acc_c += 1.f;
        }
    }
    if (BWD && acc_job >= 0) {
        float *la = A.n_jobs > 1 ? A.jobs[acc_job].loss_acc : A.job0.loss_acc;
        atomicAdd(&la[0], acc_t);
        atomicAdd(&la[1], acc_n);
        atomicAdd(&la[2], acc_c);
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) {
            c_nodes += __shfl_xor_sync(0xffffffffu, c_nodes, o);
            c_tris += __shfl_xor_sync(0xffffffffu, c_tris, o);
            c_rays += __shfl_xor_sync(0xffffffffu, c_rays, o);
            c_hits += __shfl_xor_sync(0xffffffffu, c_hits, o);
        }
        if (lane == 0) {
            atomicAdd(&A.counters[0], c_rays);
            atomicAdd(&A.counters[1], c_nodes);
            atomicAdd(&A.counters[2], c_tris);
            atomicAdd(&A.counters[3], c_hits);
        }
    }
}

template <int LAYOUT, bool BWD, bool COUNT>
cudaError_t launch_one(const TraceLaunch &L, const TraceArgs &A, cudaStream_t s) {
    int dev;
    cudaGetDevice(&dev);
    int block = L.block_size > 0 ? (L.block_size > 256 ? 256 : L.block_size) : 128;
    int bps = L.blocks_per_sm > 0 ? L.blocks_per_sm : 0;
    if (bps == 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace<LAYOUT, BWD, COUNT>, block, 0);
        bps = occ > 0 ? occ : 1;
    }
    unsigned grid = (unsigned)(device_sm_count(dev) * bps);
    k_trace<LAYOUT, BWD, COUNT><<<grid, block, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_trace(const TraceLaunch &L, cudaStream_t s) {
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
