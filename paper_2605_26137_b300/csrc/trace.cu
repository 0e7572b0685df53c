// Closest-hit traversal and shading (Sec. 6.4, stages two to four: a texel's
// 3D point is matched to a high-poly surface point whose smooth normal is
// interpolated; then the distance filter, the UV-reliability filter, and the
// normal expressed in the texel's tangent basis).
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
#include "rays.cuh"

namespace ag {
namespace {

// A texel ray as the traversal sees it and as shading sees it: both take it
// from this one function of the ray record, so the direction d used for
// shading is bit for bit the one that was traced.
struct TexelRay {
    int texel, face;
    float b1, b2, sl;
    int4 fi;
    float3 d, P0, off;
};

// Per-lane traversal state of one ray.  With KEEP the texel's record and
// frame (tex) and the hit's edge functions (in best) stay with the ray from
// set-up to shading; without it shading takes them again (texel_ray, the
// accepted triangle's edge functions), so they do not occupy registers while
// the ray is traced.  Measured on the 2.1M-triangle bake: keeping them is
// faster for the forward pass over 8-bit nodes (0.713-0.721 against
// 0.721-0.727 ms), taking them again for the FP32-node pass (0.84 against
// 0.89 ms) and the backward pass (1.75 against 1.82 ms).
struct RayState {
    int job, local;   // the ray's asset and its index in that asset's ray list
    Ray ray;
    Best best;
    uint32_t cur;
    int sp, steps;
    TexelRay tex;     // (KEEP only)
};

template <int LAYOUT, bool BWD>
struct Keep {
    static constexpr bool value = LAYOUT == AG_BVH_Q8 && !BWD;
};

__device__ __forceinline__ TexelRay texel_ray(const TraceJob &J, long long local) {
    TexelRay t;
    int4 rr = J.rays[local];
    t.texel = rr.x;
    t.face = rr.y;
    t.b1 = __int_as_float(rr.z);
    t.b2 = __int_as_float(rr.w);
    t.fi = J.lface[t.face];
    t.P0 = f3(J.lpos[t.fi.x]);
    float3 P1 = f3(J.lpos[t.fi.y]), P2 = f3(J.lpos[t.fi.z]);
    float3 N0 = f3(J.lnrm[t.fi.x]), N1 = f3(J.lnrm[t.fi.y]), N2 = f3(J.lnrm[t.fi.z]);
    t.off = (P1 - t.P0) * t.b1 + (P2 - t.P0) * t.b2;
    float3 sv = N0 + (N1 - N0) * t.b1 + (N2 - N0) * t.b2;
    t.sl = sqrtf(dot3(sv, sv));
    t.d = sv * (1.0f / t.sl);
    return t;
}

// jw: the ray's asset when JOBS is JOBS_MANY (found by the caller)
template <bool KEEP, int JOBS = JOBS_ANY>
__device__ __forceinline__ void setup_ray(const TraceArgs &A, long long r, RayState &S, int jw = 0) {
    int j = 0;
    long long local = r;
    if (JOBS == JOBS_MANY) {
        j = jw;
        local = r - A.job_begin[j];
    } else if (JOBS == JOBS_ANY && A.n_jobs > 1) {
        j = find_job(A, r);
        local = r - A.job_begin[j];
    }
    const TraceJob &J = job_t<JOBS>(A, j);
    const TexelRay t = texel_ray(J, local);
    S.job = j;
    S.local = (int)local;
    S.ray = make_ray(t.P0, t.off, t.d);
    if (KEEP) S.tex = t;
    S.best.t = 0.f; S.best.babs = J.max_dist; S.best.rec = 0; S.best.found = false;
    S.cur = 0;   // root
    S.sp = 0;
    S.steps = 0;
}

// One step of the traversal in which a node's hit leaf children are tested
// right away, in slot order, after its eight children are classified; only
// inner children go through the nearest-next bookkeeping and the stack.
// Every step of a lane is then a node visit, so the lanes of a warp no longer
// split between node visits and leaf tests, and no leaf is pushed and popped
// (0.92 -> 0.81 ms on the 2.1M-triangle bake over 8-bit nodes, for 8 % more
// triangle tests: sibling leaves are no longer culled nearest first).
template <int LAYOUT, bool COUNT>
__device__ __forceinline__ bool step_leaves(const TraceArgs &A, const TraceJob &J, RayState &S, uint2 *stack,
                                            unsigned long long &c_nodes, unsigned long long &c_tris) {
    Next nx;
    nx.has = false;
    nx.ref = 0;
    nx.dist = 0.f;
    LeafSet ls;
    const int cap = COUNT ? A.stack_cap : STACK;
    if (LAYOUT == AG_BVH_Q8)
        NodeOps<AG_BVH_Q8>::visit<true>(J.nodes, S.cur, S.ray, S.best.babs, nx, stack, S.sp, A.status, cap, &ls);
    else
        NodeOps<AG_BVH_F32>::visit<true>(J.nodes, S.cur, S.ray, S.best.babs, nx, stack, S.sp, A.status, J.scene_abs,
                                         cap, &ls);
    if (COUNT) ++c_nodes;
    while (ls.mask) {
        const int c = __ffs(ls.mask) - 1;
        ls.mask &= ls.mask - 1;
        uint32_t first;
        int cnt;
        leaf_range(ls, c, first, cnt);
        for (int t = 0; t < cnt; ++t) test_tri(S.ray, J.tris, J.tri_ids, first + t, S.best);
        if (COUNT) c_tris += cnt;
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
template <bool BWD, bool KEEP, int JOBS = JOBS_ANY>
__device__ __forceinline__ void finish(const TraceArgs &A, RayState &S, LossAcc &L) {
    const TraceJob &J = job_t<JOBS>(A, S.job);
    const TexelRay tr = KEEP ? S.tex : texel_ray(J, S.local);
    const bool hit = S.best.found;
    const float3 d = tr.d;
    float3 nh = make_float3(0.f, 0.f, 1.f);
    float bA = 0.f, bB = 0.f, bC = 0.f;
    float4 TA = make_float4(0, 0, 0, 0), TB = TA, TC = TA;
    float3 nA = make_float3(0, 0, 0), nB = nA, nC = nA;
    if (hit) {
        TA = __ldg(&J.tris[3 * (size_t)S.best.rec]);
        TB = __ldg(&J.tris[3 * (size_t)S.best.rec + 1]);
        TC = __ldg(&J.tris[3 * (size_t)S.best.rec + 2]);
        // the hit's barycentrics from the edge functions of the accepted test
        float U = S.best.U, V = S.best.V, W = S.best.W, Az, Bz, Cz;
        if (!KEEP) tri_edges(S.ray, TA, TB, TC, U, V, W, Az, Bz, Cz);
        float inv = 1.0f / (U + V + W);
        bA = U * inv; bB = V * inv; bC = W * inv;
        nA = f3(__ldg(&J.hnormals[__float_as_int(TA.w)]));
        nB = f3(__ldg(&J.hnormals[__float_as_int(TB.w)]));
        nC = f3(__ldg(&J.hnormals[__float_as_int(TC.w)]));
        nh = normalize3(nA * bA + nB * bB + nC * bC);
    }
    if (!BWD) {
        store_forward(J, tr.texel, tr.face, tr.fi, tr.b1, tr.b2, d, hit, nh, S.best.t, hit ? J.tri_ids[S.best.rec] : -1);
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
        float3 g_s = (g_d - d * dot3(d, g_d)) * (1.0f / tr.sl);
        float bw[3] = {1.f - tr.b1 - tr.b2, tr.b1, tr.b2};
        int vid[3] = {tr.fi.x, tr.fi.y, tr.fi.z};
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
template <int LAYOUT, bool BWD, bool COUNT, int JOBS = JOBS_ANY>
__device__ __forceinline__ void trace_batch(const TraceArgs &A) {
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
        int jw = 0;
        if (JOBS == JOBS_MANY) {
            // one search per warp, for its first ray; a lane past the end of
            // that asset steps on (a warp's 32 consecutive rays rarely span two)
            if (lane == 0) jw = find_job(A, (long long)base);
            jw = __shfl_sync(0xffffffffu, jw, 0);
        }
        if (r >= n_total) continue;
        if (JOBS == JOBS_MANY)
            while (jw + 1 < A.n_jobs && A.job_begin[jw + 1] <= r) ++jw;
        setup_ray<Keep<LAYOUT, BWD>::value, JOBS>(A, r, S, jw);
        if (COUNT) ++c_rays;
        if (JOBS == JOBS_MANY) {
            // the asset's traversal fields in registers for the whole ray
            const TraceJob J = A.jobs[S.job];
            while (step_leaves<LAYOUT, COUNT>(A, J, S, stack, c_nodes, c_tris)) {
            }
        } else {
            const TraceJob &J = job_t<JOBS>(A, S.job);
            while (step_leaves<LAYOUT, COUNT>(A, J, S, stack, c_nodes, c_tris)) {
            }
        }
        if (COUNT && S.best.found) ++c_hits;
        finish<BWD, Keep<LAYOUT, BWD>::value, JOBS>(A, S, L);
    }
    if (BWD) flush_loss(A, L);
    flush_counters<COUNT>(A, c_rays, c_nodes, c_tris, c_hits);
}

template <int LAYOUT, bool BWD, bool COUNT, int JOBS>
__global__ void __launch_bounds__(256) k_trace(TraceArgs A) {
    trace_batch<LAYOUT, BWD, COUNT, JOBS>(A);
}

// The forward pass over FP32 nodes, held to 64 registers like the 8-bit one
// (0.82 -> 0.78 ms on the 2.1M-triangle bake); the backward pass keeps the
// compiler's 80 (1.70 against 1.72 ms at 64).
template <int JOBS>
__global__ void __launch_bounds__(256, 4) k_trace_fwd_f32(TraceArgs A) {
    trace_batch<AG_BVH_F32, false, false, JOBS>(A);
}

// The forward bake over 8-bit nodes, held to 64 registers (4 blocks of 256
// threads per SM): the extra resident warps hide more of the gather latency
// than the few spilled values cost (1.08 -> 1.01 ms on the 2.1M-triangle bake;
// 56 or 72 registers were slower).
#ifndef AG_FWD_MIN_BLOCKS
#define AG_FWD_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(256, AG_FWD_MIN_BLOCKS) k_trace_fwd_q8(TraceArgs A) {
    trace_batch<AG_BVH_Q8, false, false, JOBS_ONE>(A);
}

// The same for a batch of assets (A.n_jobs > 1).
__global__ void __launch_bounds__(256, AG_FWD_MIN_BLOCKS) k_trace_fwd_q8_many(TraceArgs A) {
    trace_batch<AG_BVH_Q8, false, false, JOBS_MANY>(A);
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
                finish<BWD, Keep<LAYOUT, BWD>::value>(A, S, L);
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
                        setup_ray<Keep<LAYOUT, BWD>::value>(A, r, S);
                        if (COUNT) ++c_rays;
                        active = true;
                    }
                }
            }
            if (__ballot_sync(0xffffffffu, active) == 0) break;
        }
        if (active) {
            const TraceJob &J = job_of(A, S.job);
            if (!step_leaves<LAYOUT, COUNT>(A, J, S, stack, c_nodes, c_tris)) {
                active = false;
                pending = true;
            }
        }
    }
    if (BWD) flush_loss(A, L);
    flush_counters<COUNT>(A, c_rays, c_nodes, c_tris, c_hits);
}

// ---------------------------------------------------------------------------
// Schedule "coop": G lanes share one ray, so a warp carries 32/G rays.  At a
// node visit every lane loads the node (the group's loads of one address are
// served together) and tests 8/G of its children: lane g takes children
// g, g + G, ...  A hit child that is a leaf has its triangles tested on the
// spot by the lane that owns it, so the group tests up to 8 leaves at once;
// the group then agrees on the closest |t| so far (a min over its lanes) and
// on the nearest surviving inner child, which it visits next; the other
// surviving inner children go onto the group's stack in shared memory.  A
// pop reads the top G entries at once and takes the topmost one still within
// the closest |t|.  At the end the lanes' own closest hits are merged under
// the query's tie rules (|t|, then t >= 0, then the lower original id) and
// the winning lane shades the texel.  8-bit nodes, forward bake only.
// ---------------------------------------------------------------------------
constexpr int COOP_BLOCK = 128;
constexpr int COOP_STACK = 32;   // inner nodes only: leaves never go onto the stack
#ifndef AG_COOP_MIN_BLOCKS
#define AG_COOP_MIN_BLOCKS 8     // resident 128-thread blocks per SM the register budget is cut for (64 registers)
#endif

template <int G>
__device__ __forceinline__ float group_minf(float v, unsigned gmask) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v = fminf(v, __shfl_xor_sync(gmask, v, o, G));
    return v;
}

template <int G>
__device__ __forceinline__ unsigned long long group_min64(unsigned long long v, unsigned gmask) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        unsigned long long w = __shfl_xor_sync(gmask, v, o, G);
        v = w < v ? w : v;
    }
    return v;
}

// One node visit of the group's ray; false when the ray is done.
template <int G, bool COUNT>
__device__ __forceinline__ bool coop_step(const TraceArgs &A, const TraceJob &J, RayState &S, float &lim,
                                          uint2 *stk, int g, unsigned gmask, unsigned long long &c_nodes,
                                          unsigned long long &c_tris) {
    constexpr int CPL = 8 / G;
    const Ray &r = S.ray;
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const QNode *>(J.nodes) + S.cur);
    uint4 w0 = __ldg(p), w1 = __ldg(p + 1), w2 = __ldg(p + 2), w3 = __ldg(p + 3), w4 = __ldg(p + 4);
    if (COUNT && g == 0) ++c_nodes;
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
    uint32_t nx0 = r.nx() ? w3.z : w2.x, nx1 = r.nx() ? w3.w : w2.y, fx0 = r.nx() ? w2.x : w3.z, fx1 = r.nx() ? w2.y : w3.w;
    uint32_t ny0 = r.ny() ? w4.x : w2.z, ny1 = r.ny() ? w4.y : w2.w, fy0 = r.ny() ? w2.z : w4.x, fy1 = r.ny() ? w2.w : w4.y;
    uint32_t nz0 = r.nz() ? w4.z : w3.x, nz1 = r.nz() ? w4.w : w3.y, fz0 = r.nz() ? w3.x : w4.z, fz1 = r.nz() ? w3.y : w4.w;
    const uint32_t child_base = w1.x, tri_base = w1.y;
    bool ihit[CPL];
    uint32_t iref[CPL];
    float idist[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
        const int c = g + G * i;
        const int k = c & 3;
        const bool hi = c >= 4;
        uint32_t m = ((hi ? w1.w : w1.z) >> (8 * k)) & 0xffu;
        float tnx = __fmaf_rn(byte_q(hi ? nx1 : nx0, k), ax, bnx);
        float tfx = __fmaf_rn(byte_q(hi ? fx1 : fx0, k), ax, bfx);
        float tny = __fmaf_rn(byte_q(hi ? ny1 : ny0, k), ay, bny);
        float tfy = __fmaf_rn(byte_q(hi ? fy1 : fy0, k), ay, bfy);
        float tnz = __fmaf_rn(byte_q(hi ? nz1 : nz0, k), az, bnz);
        float tfz = __fmaf_rn(byte_q(hi ? fz1 : fz0, k), az, bfz);
        float te = fmaxf(fmaxf(tnx, tny), tnz);
        float tx = fminf(fminf(tfx, tfy), tfz);
        ihit[i] = false;
        iref[i] = 0;
        idist[i] = 0.f;
        if (m != 0 && te <= tx && te <= lim && tx >= -lim) {
            if (m & 0x80u) {
                ihit[i] = true;
                iref[i] = child_base + (m & 0x7fu);
                idist[i] = fmaxf(fmaxf(te, -tx), 0.f);
            } else {
                const uint32_t first = tri_base + (m & 31u);
                const int cnt = (int)((m >> 5) & 3u);   // the meta byte holds the count itself
                for (int t = 0; t < cnt; ++t) test_tri_shared(r, J.tris, J.tri_ids, first + t, S.best, lim);
                if (COUNT) c_tris += cnt;
            }
        }
    }
    lim = group_minf<G>(lim, gmask);
    // the nearest inner child within the closest |t| is visited next, the others are pushed
    unsigned long long key[CPL];
    unsigned long long mine = ~0ull;
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
        key[i] = (ihit[i] && idist[i] <= lim) ? ((unsigned long long)__float_as_uint(idist[i]) << 32) | iref[i] : ~0ull;
        mine = key[i] < mine ? key[i] : mine;
    }
    const unsigned long long near = group_min64<G>(mine, gmask);
    int npush = 0;
#pragma unroll
    for (int i = 0; i < CPL; ++i) npush += (key[i] != ~0ull && key[i] != near) ? 1 : 0;
    int incl = npush;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        int v = __shfl_up_sync(gmask, incl, o, G);
        if (g >= o) incl += v;
    }
    const int total = __shfl_sync(gmask, incl, G - 1, G);
    if (total) {
        const int cap = COUNT ? min(A.stack_cap, COOP_STACK) : COOP_STACK;
        int pos = S.sp + incl - npush;
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            if (key[i] != ~0ull && key[i] != near) {
                if (pos < cap) stk[pos] = make_uint2((uint32_t)key[i], (uint32_t)(key[i] >> 32));
                else atomicOr(A.status, AGS_STACK);
                ++pos;
            }
        }
        S.sp = min(S.sp + total, cap);
        __syncwarp(gmask);
    }
    if (++S.steps > A.max_steps) {
        atomicOr(A.status, AGS_STEP_CAP);
        return false;
    }
    if (near != ~0ull) {
        S.cur = (uint32_t)near;
        return true;
    }
    const unsigned base = (unsigned)(threadIdx.x & 31) & ~(unsigned)(G - 1);
    while (S.sp > 0) {
        const int idx = S.sp - 1 - g;
        uint2 e = make_uint2(0u, 0u);
        bool ok = false;
        if (idx >= 0) {
            e = stk[idx];
            ok = __uint_as_float(e.y) <= lim;
        }
        const unsigned b = (__ballot_sync(gmask, ok) >> base) & ((1u << G) - 1u);
        if (b) {
            const int w = __ffs(b) - 1;
            S.cur = __shfl_sync(gmask, e.x, w, G);
            S.sp -= 1 + w;
            return true;
        }
        S.sp = max(S.sp - G, 0);
    }
    return false;
}

template <int G, bool COUNT>
__device__ __forceinline__ void trace_coop(const TraceArgs &A) {
    __shared__ uint2 s_stack[(COOP_BLOCK / G) * COOP_STACK];
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int g = lane & (G - 1);
    const unsigned gmask = ((1u << G) - 1u) << (lane & ~(G - 1));
    uint2 *stk = s_stack + (threadIdx.x / G) * COOP_STACK;
    const long long n_total = *A.n_rays_dev;
    unsigned long long c_nodes = 0, c_tris = 0, c_rays = 0, c_hits = 0;
    LossAcc L = {0.f, 0.f, 0.f, -1};
    RayState S;
    float lim = 0.f;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(A.ray_counter, (unsigned long long)RPW);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= n_total) break;
        const long long r = (long long)base + lane / G;
        const bool mine = r < n_total;
        bool active = mine;
        if (mine) {
            setup_ray<true>(A, r, S);
            lim = job_of(A, S.job).max_dist;
            if (COUNT && g == 0) ++c_rays;
        }
        while (__any_sync(0xffffffffu, active)) {
            if (active) active = coop_step<G, COUNT>(A, job_of(A, S.job), S, lim, stk, g, gmask, c_nodes, c_tris);
        }
        if (mine) {
            // merge the lanes' closest hits: |t|, then t >= 0, then the lower original id
            const TraceJob &J = job_of(A, S.job);
            unsigned long long key = ~0ull;
            if (S.best.found)
                key = ((unsigned long long)__float_as_uint(S.best.babs) << 32) | (S.best.t < 0.f ? 0x80000000ull : 0ull) |
                      (unsigned long long)(uint32_t)J.tri_ids[S.best.rec];
            const unsigned long long kmin = group_min64<G>(key, gmask);
            const bool winner = S.best.found && key == kmin;
            if (winner || (kmin == ~0ull && g == 0)) {
                if (COUNT && winner) ++c_hits;
                finish<false, true>(A, S, L);
            }
        }
    }
    flush_counters<COUNT>(A, c_rays, c_nodes, c_tris, c_hits);
}

template <int G, bool COUNT>
__global__ void __launch_bounds__(COOP_BLOCK, AG_COOP_MIN_BLOCKS) k_trace_coop(TraceArgs A) {
    trace_coop<G, COUNT>(A);
}

template <int G, bool COUNT>
cudaError_t launch_coop(const TraceLaunch &L, const TraceArgs &A, cudaStream_t s) {
    int dev;
    cudaGetDevice(&dev);
    int bps = L.blocks_per_sm;
    if (bps <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_coop<G, COUNT>, COOP_BLOCK, 0);
        bps = occ > 0 ? occ : 1;
    }
    k_trace_coop<G, COUNT><<<(unsigned)(device_sm_count(dev) * bps), COOP_BLOCK, 0, s>>>(A);
    return cudaGetLastError();
}

template <int LAYOUT, bool BWD, bool COUNT>
cudaError_t launch_one(const TraceLaunch &L, const TraceArgs &A, cudaStream_t s) {
    int dev;
    cudaGetDevice(&dev);
    int block = L.block_size > 0 ? (L.block_size > 256 ? 256 : L.block_size) : 128;
    int bps = L.blocks_per_sm > 0 ? L.blocks_per_sm : 0;
    const bool refill = L.schedule == AG_SCHED_REFILL;
    constexpr bool fwd_q8 = LAYOUT == AG_BVH_Q8 && !BWD && !COUNT;
    constexpr bool fwd_f32 = LAYOUT == AG_BVH_F32 && !BWD && !COUNT;
    if (bps == 0) {
        int occ = 0;
        if (refill)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_refill<LAYOUT, BWD, COUNT>, block, 0);
        else if (fwd_q8)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, A.n_jobs > 1 ? k_trace_fwd_q8_many : k_trace_fwd_q8,
                                                          block, 0);
        else if (fwd_f32)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ, A.n_jobs > 1 ? k_trace_fwd_f32<JOBS_MANY> : k_trace_fwd_f32<JOBS_ONE>, block, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ, A.n_jobs > 1 ? k_trace<LAYOUT, BWD, COUNT, JOBS_MANY> : k_trace<LAYOUT, BWD, COUNT, JOBS_ONE>,
                block, 0);
        bps = occ > 0 ? occ : 1;
    }
    unsigned grid = (unsigned)(device_sm_count(dev) * bps);
    if (refill)
        k_trace_refill<LAYOUT, BWD, COUNT><<<grid, block, 0, s>>>(A, 8);
    else if (fwd_q8 && A.n_jobs > 1)
        k_trace_fwd_q8_many<<<grid, block, 0, s>>>(A);
    else if (fwd_q8)
        k_trace_fwd_q8<<<grid, block, 0, s>>>(A);
    else if (fwd_f32 && A.n_jobs > 1)
        k_trace_fwd_f32<JOBS_MANY><<<grid, block, 0, s>>>(A);
    else if (fwd_f32)
        k_trace_fwd_f32<JOBS_ONE><<<grid, block, 0, s>>>(A);
    else if (A.n_jobs > 1)
        k_trace<LAYOUT, BWD, COUNT, JOBS_MANY><<<grid, block, 0, s>>>(A);
    else
        k_trace<LAYOUT, BWD, COUNT, JOBS_ONE><<<grid, block, 0, s>>>(A);
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
    A.stack_cap = L.stack_cap > 0 && L.stack_cap < STACK ? L.stack_cap : STACK;
    const bool cnt = L.counters != nullptr;
    if (L.layout == AG_BVH_Q8 && !L.backward && L.schedule >= AG_SCHED_COOP4 && L.schedule <= AG_SCHED_COOP2) {
        switch (L.schedule) {
            case AG_SCHED_COOP2: return cnt ? launch_coop<2, true>(L, A, s) : launch_coop<2, false>(L, A, s);
            case AG_SCHED_COOP4: return cnt ? launch_coop<4, true>(L, A, s) : launch_coop<4, false>(L, A, s);
            default: return cnt ? launch_coop<8, true>(L, A, s) : launch_coop<8, false>(L, A, s);
        }
    }
    if (L.layout == AG_BVH_Q8) {
        if (L.backward) return launch_one<AG_BVH_Q8, true, false>(L, A, s);
        return cnt ? launch_one<AG_BVH_Q8, false, true>(L, A, s) : launch_one<AG_BVH_Q8, false, false>(L, A, s);
    }
    if (L.backward) return launch_one<AG_BVH_F32, true, false>(L, A, s);
    return cnt ? launch_one<AG_BVH_F32, false, true>(L, A, s) : launch_one<AG_BVH_F32, false, false>(L, A, s);
}

}  // namespace ag
