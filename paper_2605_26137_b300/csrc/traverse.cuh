// Traversal pieces shared by the ray query (trace.cu) and the closest-point
// query (closest.cu) over the same 8-wide BVH: launch arguments, the
// nearest-child-next bookkeeping, the 8-bit plane decode, the counting build's
// reduction and the forward shading store (Sec. 6.4: the hit normal written in
// the texel's tangent basis; the UV-reliability filter).
#pragma once

#include "ag_internal.cuh"

namespace ag {
namespace {

// Per-thread traversal stack entries.  A visit pushes at most 7 children, so
// a query whose radius still covers every box (a point-to-mesh distance with a
// large limit) needs up to 7 x the tree depth; 128 covers depths up to 18.
constexpr int STACK = 128;
constexpr float EPS_REL = 4.76837158203125e-07f;  // 2^-21: widening per unit of coordinate magnitude
// 8-bit node planes are decoded as fma(Q, 2^15 s, origin - 2^15 s) with the
// exact float Q = 1 + q 2^-15 (byte_q): one PRMT and one FMA per plane.  The
// extra rounding of origin - 2^15 s is covered by widening per unit of
// coordinate magnitude by EPS_POS and per unit of the node's scale s by EPS_Q
// (see the node visits).
constexpr float EPS_POS = 9.5367431640625e-07f;   // 2^-20
constexpr float EPS_Q = 0.0078125f;                // 2^-7
constexpr float Q_SCALE = 32768.0f;                // 2^15

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
    int stack_cap;   // counting build only: usable stack entries (test hook)
};

__device__ __forceinline__ const TraceJob &job_of(const TraceArgs &A, int j) {
    return A.n_jobs > 1 ? A.jobs[j] : A.job0;
}

// How a kernel finds a ray's asset: from A.n_jobs at run time (JOBS_ANY), or
// fixed when it is compiled: one asset (JOBS_ONE, the job in the kernel's
// parameters) or a batch (JOBS_MANY, the device table).
enum { JOBS_ANY = 0, JOBS_ONE = 1, JOBS_MANY = 2 };
template <int JOBS>
__device__ __forceinline__ const TraceJob &job_t(const TraceArgs &A, int j) {
    if (JOBS == JOBS_ONE) return A.job0;
    if (JOBS == JOBS_MANY) return A.jobs[j];
    return job_of(A, j);
}

// the asset of global ray r: the last j with job_begin[j] <= r
__device__ __forceinline__ int find_job(const TraceArgs &A, long long r) {
    int lo = 0, hi = A.n_jobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (A.job_begin[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Blackwell's three-input FP32 minimum / maximum (one instruction each; the
// same value and NaN rule as two fminf / fmaxf) and its packed FP32 FMA, which
// rounds each of its two lanes exactly as a scalar fmaf does.
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// (d0, d1) = (fma(a0, b0, c0), fma(a1, b1, c1)) in one packed instruction
__device__ __forceinline__ void fma2(float a0, float a1, float b0, float b1, float c0, float c1, float &d0,
                                     float &d1) {
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}

// byte k of w in mantissa bits 8..15 of 1.0: the exact float 1 + byte * 2^-15
__device__ __forceinline__ float byte_q(uint32_t w, int k) {
    return __uint_as_float(__byte_perm(w, 0x3F800000u, 0x7604u | ((unsigned)k << 4)));
}

// Traversal bookkeeping of one node visit: the nearest relevant child becomes
// the next node (no stack round trip); every other relevant child is pushed.
struct Next {
    uint32_t ref;
    float dist;
    bool has;
};

// cap: the stack's usable entries (STACK; less only in the counting build
// under the ag_opts.stack_limit test hook)
__device__ __forceinline__ void offer(uint32_t ref, float d, Next &nx, uint2 *stack, int &sp, unsigned *status,
                                      int cap = STACK) {
    uint32_t pr = ref;
    float pd = d;
    if (!nx.has || d < nx.dist) {
        pr = nx.ref;
        pd = nx.dist;
        nx.ref = ref;
        nx.dist = d;
        if (!nx.has) { nx.has = true; return; }
    }
    if (sp < cap) stack[sp++] = make_uint2(pr, __float_as_uint(pd));
    else atomicOr(status, AGS_STACK);
}

__device__ __forceinline__ uint32_t child_ref(uint32_t m, uint32_t child_base, uint32_t tri_base) {
    return (m & 0x80u) ? child_base + (m & 0x7fu) : ref_leaf(tri_base + (m & 31u), (int)((m >> 5) & 3u));
}

// The leaf children of one node visit that are to be tested right away
// instead of going through the nearest-next bookkeeping: a mask of child
// slots, and the node's meta words (one byte per slot: bit 7 inner child,
// bits 5-6 triangle count, bits 0-4 first triangle after tri_base).
struct LeafSet {
    uint32_t mask, meta_lo, meta_hi, tri_base;
};

__device__ __forceinline__ void leaf_range(const LeafSet &ls, int c, uint32_t &first, int &count) {
    const uint32_t m = ((c >= 4 ? ls.meta_hi : ls.meta_lo) >> (8 * (c & 3))) & 0xffu;
    first = ls.tri_base + (m & 31u);
    count = (int)((m >> 5) & 3u);
}

template <bool COUNT>
__device__ __forceinline__ void flush_counters(const TraceArgs &A, unsigned long long c_rays, unsigned long long c_nodes,
                                               unsigned long long c_tris, unsigned long long c_hits) {
    if (!COUNT) return;
    const int lane = threadIdx.x & 31;
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

// Forward outputs of one texel: tangent-space normal of the hit normal nh in
// the texel frame (N = d, T = the interpolated corner tangent made orthogonal
// to N, B = w (N x T)), (0,0,1) on a miss or a degenerate-UV face, the signed
// displacement, the mask and the optional hit id / displacement copies.
__device__ __forceinline__ void store_forward(const TraceJob &J, int texel, int face, int4 fi, float b1, float b2,
                                              float3 d, bool hit, float3 nh, float disp, int hit_id) {
    float3 nts = make_float3(0.f, 0.f, 1.f);
    if (hit && !(fi.w & FACE_DEGEN)) {
        float4 T0 = J.ltan[3 * face], T1 = J.ltan[3 * face + 1], T2 = J.ltan[3 * face + 2];
        float3 tt = f3(T0) + (f3(T1) - f3(T0)) * b1 + (f3(T2) - f3(T0)) * b2;
        tt = normalize3(tt - d * dot3(tt, d));
        float3 bb = cross3(d, tt) * T0.w;
        nts = make_float3(dot3(nh, tt), dot3(nh, bb), dot3(nh, d));
    }
    J.ntsd[texel] = make_float4(nts.x, nts.y, nts.z, hit ? disp : 0.f);
    J.mask[texel] = hit ? 1 : 0;
    if (J.hit_tri) J.hit_tri[texel] = hit ? hit_id : -1;
    if (J.hit_t) J.hit_t[texel] = hit ? disp : 0.f;
}

}  // namespace
}  // namespace ag
