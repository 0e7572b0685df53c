// LBVH over the high-poly mesh (the tree Sec. 6.4 searches), built entirely
// on the device:
//   triangle bounds + centroid bounds -> 30-bit Morton codes -> LSD radix
//   sort (8-bit digits, stable warp-ranked scatter) -> Karras (2012) binary
//   hierarchy -> bottom-up FP32 boxes (with the SAH collapse costs) ->
//   top-down collapse to 8-wide nodes (SAH-optimal children, or greedy
//   expansion; leaves of LEAF_MAX triangles) with child boxes quantised to 8 bits
//   and rounded outward (or kept in FP32) -> triangles reordered into 48-byte
//   leaf-order records -> area-weighted vertex normals.
#include "ag_internal.cuh"

#include <cstdlib>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace ag {
namespace {

constexpr int RS_BLOCK = 256;
// collapse levels launched one kernel each (a 30-bit Morton tree collapses to
// about 12 levels of 8-wide nodes); deeper levels run on one CTA
constexpr int COLLAPSE_LEVELS = 16;
// levels in all: the binary tree of 30-bit codes over at most 2^29 sorted
// triangles is at most 59 deep, and every wide level descends at least one
// binary level
constexpr int COLLAPSE_MAX = 64;

// what the host reads back from a build (one copy, once the build is done)
struct BuildSummary {
    unsigned counters[2];           // wide nodes, triangle records written by the collapse
    int levels[COLLAPSE_MAX + 1];   // queue length of every collapse level
    unsigned bounds[16];            // centroid and scene box keys of k_tri_prep (scene box at 6..11)
};
#ifndef AG_RS_ROUNDS
#define AG_RS_ROUNDS 4   // 1,024 keys per block: 4x the blocks of 16 rounds, build 1.45 -> 1.41 ms on 2.1M triangles
#endif
constexpr int RS_ROUNDS = AG_RS_ROUNDS;
constexpr int RS_TILE = RS_BLOCK * RS_ROUNDS;

__device__ __forceinline__ unsigned f2key(float f) {
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// bounds[0..5]: centroid lo xyz (min keys), centroid hi xyz (max keys);
// bounds[6..11]: vertex lo / hi.
__global__ void k_tri_prep(const float *__restrict__ V, const int32_t *__restrict__ F, int64_t nv,
                           int64_t nf, float4 *__restrict__ tlo, float4 *__restrict__ thi,
                           float4 *__restrict__ cent, unsigned *__restrict__ bounds,
                           unsigned *__restrict__ status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float c[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    bool valid = i < nf;
    if (valid) {
        int32_t id[3] = {F[3 * i], F[3 * i + 1], F[3 * i + 2]};
        for (int k = 0; k < 3; ++k)
            if (id[k] < 0 || id[k] >= nv) {
                atomicOr(status, AGS_BAD_FACE);
                id[0] = id[1] = id[2] = 0;
                break;
            }
        float p[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) p[k][a] = V[3 * (int64_t)id[k] + a];
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(p[0][a], fminf(p[1][a], p[2][a]));
            hi[a] = fmaxf(p[0][a], fmaxf(p[1][a], p[2][a]));
            c[a] = (p[0][a] + p[1][a] + p[2][a]) * (1.0f / 3.0f);
        }
        tlo[i] = make_float4(lo[0], lo[1], lo[2], 0.f);
        thi[i] = make_float4(hi[0], hi[1], hi[2], 0.f);
        cent[i] = make_float4(c[0], c[1], c[2], 0.f);
    }
    // block reduction of the 12 bound keys
    __shared__ unsigned s[12][32];
    unsigned mine[12];
    for (int a = 0; a < 3; ++a) {
        mine[a] = valid ? f2key(c[a]) : 0xffffffffu;
        mine[3 + a] = valid ? f2key(c[a]) : 0u;
        mine[6 + a] = valid ? f2key(lo[a]) : 0xffffffffu;
        mine[9 + a] = valid ? f2key(hi[a]) : 0u;
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int q = 0; q < 12; ++q) {
            unsigned other = __shfl_xor_sync(0xffffffffu, mine[q], o);
            bool is_min = (q < 3) || (q >= 6 && q < 9);
            mine[q] = is_min ? min(mine[q], other) : max(mine[q], other);
        }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int q = 0; q < 12; ++q) s[q][warp] = mine[q];
    __syncthreads();
    if (threadIdx.x < 12) {
        int q = threadIdx.x;
        bool is_min = (q < 3) || (q >= 6 && q < 9);
        unsigned r = s[q][0];
        for (int w = 1; w < nw; ++w) r = is_min ? min(r, s[q][w]) : max(r, s[q][w]);
        if (is_min) atomicMin(&bounds[q], r);
        else atomicMax(&bounds[q], r);
    }
}

__device__ __forceinline__ unsigned spread10(unsigned x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_morton(const float4 *__restrict__ cent, int64_t nf, const unsigned *__restrict__ bounds,
                         unsigned *__restrict__ keys, unsigned *__restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    float4 c = cent[i];
    float cc[3] = {c.x, c.y, c.z};
    unsigned q[3];
    for (int a = 0; a < 3; ++a) {
        float lo = key2f(bounds[a]), hi = key2f(bounds[3 + a]);
        float ext = hi - lo;
        float u = ext > 0.f ? (cc[a] - lo) / ext : 0.5f;
        int v = (int)(u * 1024.0f);
        q[a] = (unsigned)min(1023, max(0, v));
    }
    keys[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    vals[i] = (unsigned)i;
}

// ---- LSD radix sort, 8-bit digits ------------------------------------------------
__global__ void k_rs_hist(const unsigned *__restrict__ keys, int64_t n, int shift, unsigned *__restrict__ hist,
                          int nblocks) {
    __shared__ unsigned cnt[256];
    for (int d = threadIdx.x; d < 256; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + (int64_t)r * RS_BLOCK + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
}

__global__ void __launch_bounds__(RS_BLOCK) k_rs_scatter(const unsigned *__restrict__ kin,
                                                         const unsigned *__restrict__ vin,
                                                         unsigned *__restrict__ kout, unsigned *__restrict__ vout,
                                                         int64_t n, int shift, const unsigned *__restrict__ offs,
                                                         int nblocks) {
    __shared__ unsigned s_base[256];
    __shared__ unsigned s_w[RS_BLOCK / 32][256];
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int d = tid; d < 256; d += RS_BLOCK) s_base[d] = offs[(int64_t)d * nblocks + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + (int64_t)r * RS_BLOCK + tid;
        bool valid = i < n;
        unsigned key = valid ? kin[i] : 0u, val = valid ? vin[i] : 0u;
        unsigned digit = (key >> shift) & 255u;
        for (int d = lane; d < 256; d += 32) s_w[warp][d] = 0;
        __syncwarp();
        unsigned peers = __match_any_sync(0xffffffffu, valid ? digit : 0x100u);
        int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) s_w[warp][digit] = __popc(peers);
        __syncthreads();
        if (tid < 256) {
            unsigned run = s_base[tid];
            for (int w = 0; w < RS_BLOCK / 32; ++w) { unsigned c = s_w[w][tid]; s_w[w][tid] = run; run += c; }
            s_base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            unsigned pos = s_w[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

// ---- Karras 2012 hierarchy ----------------------------------------------------------
// Internal nodes 0..n-2, leaves n-1+k.  child[i] = (left, right), range[i] =
// (first, last) sorted positions covered.

// (32-bit positions: the build takes fewer than 2^29 triangles; the key at i
// is read once)
__device__ __forceinline__ int delta_at(const unsigned *__restrict__ k, int n, int i, unsigned ki, int j) {
    if (j < 0 || j >= n) return -1;
    const unsigned b = __ldg(&k[j]);
    if (ki == b) return 32 + __clz((unsigned)(i ^ j));
    return __clz(ki ^ b);
}

__global__ void k_karras(const unsigned *__restrict__ k, int64_t n64, int2 *__restrict__ child,
                         int2 *__restrict__ range, int *__restrict__ parent) {
    const int n = (int)n64;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const unsigned ki = __ldg(&k[i]);
    const int d = (delta_at(k, n, i, ki, i + 1) - delta_at(k, n, i, ki, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta_at(k, n, i, ki, i - d);
    int lmax = 2;
    while (delta_at(k, n, i, ki, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta_at(k, n, i, ki, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta_at(k, n, i, ki, j);
    int s = 0;
    int div = 2;
    while (true) {
        const int t = (l + div - 1) / div;
        if (delta_at(k, n, i, ki, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
        div <<= 1;
    }
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const int left = (lo == gamma) ? n - 1 + gamma : gamma;
    const int right = (hi == gamma + 1) ? n - 1 + gamma + 1 : gamma + 1;
    child[i] = make_int2(left, right);
    range[i] = make_int2(lo, hi);
    parent[left] = i;
    parent[right] = i;
}

// ---- SAH-optimal collapse (AG_COLLAPSE_SAH) ---------------------------------------------
// cost[8 * node + i - 1] = C(node, i) for the internal nodes: the least
// surface-area cost of the node's subtree when it may take up to i child
// slots of its wide parent.
//   leaf (a subtree of <= LEAF_MAX triangles): A(n) * SAH_TRI * count;
//   C(n, 1) = leaf cost, or A(n) * SAH_NODE + D(n, 8) for a wide node;
//   D(n, j) = min over k of C(left, k) + C(right, j - k);
//   C(n, i) = min(C(n, i - 1), D(n, i)) for i >= 2 (a leaf-sized subtree may
//   still spread over several slots as smaller leaves).
// A one-triangle binary leaf costs A * SAH_TRI for every i; it is not stored,
// the parent takes it from the leaf's box.
// dec[node] records the decisions the top-down collapse follows, 3 bits each
// for j = 2..8: bits 3(j-2).. hold k(j) - 1, the first k reaching D(n, j);
// bits 21 + 3(j-2).. hold f(j) - 1, the fewest slots f <= j with C(n, f) =
// C(n, j) (the node takes f slots when offered j).
// Computed in the bottom-up box pass (the second child to arrive computes the
// parent's box, then its costs).
constexpr float SAH_NODE = 1.0f;
#ifndef AG_SAH_TRI
#define AG_SAH_TRI 0.3f
#endif
constexpr float SAH_TRI = AG_SAH_TRI;

__device__ __forceinline__ float box_half_area(float4 lo, float4 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ void sah_child_cost(int c, int64_t n, float area, const float *cost, float *out) {
    if (c >= n - 1) {
#pragma unroll
        for (int i = 0; i < 8; ++i) out[i] = area * SAH_TRI;
    } else {
        const float4 *q = reinterpret_cast<const float4 *>(cost + 8 * (int64_t)c);
        const float4 u = __ldcg(q), v = __ldcg(q + 1);
        out[0] = u.x; out[1] = u.y; out[2] = u.z; out[3] = u.w;
        out[4] = v.x; out[5] = v.y; out[6] = v.z; out[7] = v.w;
    }
}

// costs and decisions of internal node `node` with children `ch`, the child
// boxes' half areas al, ar and its own half area a
__device__ __forceinline__ void sah_node_cost(int2 ch, int cnt, float a, float al, float ar, int64_t n,
                                              int64_t node, float *cost, uint64_t *dec) {
    float cl[8], cr[8];
    sah_child_cost(ch.x, n, al, cost, cl);
    sah_child_cost(ch.y, n, ar, cost, cr);
    float d[8];
    uint64_t code = 0;
#pragma unroll
    for (int j = 2; j <= 8; ++j) {
        float best = 3.0e38f;
        int kb = 1;
#pragma unroll
        for (int k = 1; k < j; ++k) {
            const float v = cl[k - 1] + cr[j - k - 1];
            if (v < best) { best = v; kb = k; }
        }
        d[j - 1] = best;
        code |= (uint64_t)(kb - 1) << (3 * (j - 2));
    }
    float c[8];
    c[0] = cnt <= LEAF_MAX ? a * SAH_TRI * (float)cnt : a * SAH_NODE + d[7];
    int f = 1;
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        c[i] = fminf(c[i - 1], d[i]);
        if (!(c[i - 1] <= c[i])) f = i + 1;   // C(n, i + 1) < C(n, i): the fewest is i + 1
        code |= (uint64_t)(f - 1) << (21 + 3 * (i - 1));
    }
    float4 *q = reinterpret_cast<float4 *>(cost + 8 * node);
    __stcg(q, make_float4(c[0], c[1], c[2], c[3]));
    __stcg(q + 1, make_float4(c[4], c[5], c[6], c[7]));
    __stcg(&dec[node], code);
}

// bottom-up boxes: box_lo/hi [2n-1]; flags [n-1] zeroed; with `cost` and
// `dec`, the SAH collapse costs and decisions of every internal node in the
// same pass
__global__ void k_bounds(const unsigned *__restrict__ vals, int64_t n, const float4 *__restrict__ tlo,
                         const float4 *__restrict__ thi, const int2 *__restrict__ child,
                         const int2 *__restrict__ range, const int *__restrict__ parent, float4 *box_lo,
                         float4 *box_hi, int *flags, float *cost, uint64_t *dec) {
    int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= n) return;
    int64_t node = n - 1 + kk;
    unsigned t = vals[kk];
    const float4 lo0 = tlo[t], hi0 = thi[t];
    box_lo[node] = lo0;
    box_hi[node] = hi0;
    if (n == 1) return;
    while (true) {
        __threadfence();
        int p = parent[node];
        if (atomicAdd(&flags[p], 1) == 0) return;
        int2 c = child[p];
        float4 a0 = __ldcg(&box_lo[c.x]), a1 = __ldcg(&box_hi[c.x]);
        float4 b0 = __ldcg(&box_lo[c.y]), b1 = __ldcg(&box_hi[c.y]);
        const float4 lo = make_float4(fminf(a0.x, b0.x), fminf(a0.y, b0.y), fminf(a0.z, b0.z), 0.f);
        const float4 hi = make_float4(fmaxf(a1.x, b1.x), fmaxf(a1.y, b1.y), fmaxf(a1.z, b1.z), 0.f);
        __stcg(&box_lo[p], lo);
        __stcg(&box_hi[p], hi);
        if (cost) {
            const int2 rg = range[p];
            sah_node_cost(c, rg.y - rg.x + 1, box_half_area(lo, hi), box_half_area(a0, a1),
                          box_half_area(b0, b1), n, p, cost, dec);
        }
        node = p;
        if (p == 0) return;
    }
}

// ---- collapse to 8-wide -----------------------------------------------------------------
struct CollapseArgs {
    int64_t n;
    const int2 *child, *range;
    const float4 *box_lo, *box_hi;
    const unsigned *vals;         // sorted position -> original triangle
    const float *V;
    const int32_t *F;
    int64_t nv;
    int layout;
    int rule;
    void *nodes;
    float4 *tris;
    int32_t *tri_ids;
    unsigned *node_count, *tri_count;
    int *q_count_out;
    uint32_t *rec_pos;            // leaf-order record -> sorted position (records written by k_tri_records)
    const uint64_t *sah_dec;      // decisions of the SAH collapse (internal nodes), or null (greedy rules)
};

__device__ __forceinline__ int subtree_count(const CollapseArgs &A, int b) {
    if (b >= A.n - 1) return 1;
    int2 r = A.range[b];
    return r.y - r.x + 1;
}
__device__ __forceinline__ float half_area(const CollapseArgs &A, int b) {
    float4 lo = A.box_lo[b], hi = A.box_hi[b];
    float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

// smallest power-of-two exponent (biased, as float exponent bits) such that
// every child box quantises into 0..255 with outward rounding verified in the
// exact decode arithmetic of the traversal: fmaf(q, 2^e, origin). Slots from
// nc on get the empty box (lo 255, hi 0).
__device__ __forceinline__ int choose_exp(float o, float hi_node, const float (&clo)[8], const float (&chi)[8],
                                          int nc, int (&qlo)[8], int (&qhi)[8]) {
    float ext = hi_node - o;
    int e;
    if (!(ext > 0.f)) e = 1;
    else {
        int ex;
        frexpf(ext / 255.0f, &ex);   // ext/255 = m*2^ex, m in [0.5,1)
        e = max(1, min(254, ex + 127 - 1));
    }
    for (;; ++e) {
        float s = __uint_as_float((unsigned)e << 23);
        const float inv = 1.0f / s;   // a power of two: x * inv is exactly x / s
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            qlo[c] = 255;
            qhi[c] = 0;
            if (c >= nc) continue;
            int ql = (int)floorf((clo[c] - o) * inv);
            ql = max(0, min(255, ql));
            while (ql > 0 && fmaf((float)ql, s, o) > clo[c]) --ql;
            int qh = (int)ceilf((chi[c] - o) * inv);
            qh = max(0, qh);
            while (qh <= 255 && fmaf((float)qh, s, o) < chi[c]) ++qh;
            while (qh > 0 && qh - 1 >= ql && fmaf((float)(qh - 1), s, o) >= chi[c]) --qh;
            if (qh > 255 || fmaf((float)ql, s, o) > clo[c]) ok = false;
            qlo[c] = ql;
            qhi[c] = min(qh, 255);
        }
        if (ok || e >= 254) return e;
    }
}

// all 32 lanes of the warp call this together: each lane gets `v` entries of
// the counter, with one atomic per warp
__device__ __forceinline__ unsigned warp_alloc(unsigned *ctr, unsigned v) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += t;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned base = 0;
    if (lane == 31u && total) base = atomicAdd(ctr, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + incl - v;
}

// the children of the wide node made from binary node item.x, written to wide
// slot item.y; `live` is false for the lanes past the end of the queue, which
// only take part in the warp's counter allocations
__device__ void collapse_node(const CollapseArgs &A, int2 item, bool live, int2 *__restrict__ q_out) {
    int b = item.x;
    unsigned wslot = (unsigned)item.y;
    int ch[8];
    int nc = 0;
    if (!live) {
    } else if (b >= A.n - 1 || subtree_count(A, b) <= LEAF_MAX) {
        ch[nc++] = b;   // only the root of a tiny mesh gets here
    } else if (A.sah_dec) {
        // the SAH decisions, breadth first: every round splits each entry
        // (node, slots) that still takes several slots, in place, so that the
        // children keep the binary tree's left-to-right order; the loads of
        // one round are independent of each other
        int sn[8], sk[8];
        bool fin[8];
        {
            const int2 c = A.child[b];
            const int kl = (int)((A.sah_dec[b] >> 18) & 7u) + 1;   // k(8) of the root
            sn[0] = c.x; sk[0] = kl; fin[0] = false;
            sn[1] = c.y; sk[1] = 8 - kl; fin[1] = false;
            nc = 2;
        }
        for (int round = 0; round < 8; ++round) {
            uint64_t dd[8];
            int2 cc[8];
            bool any = false;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (i < nc && !fin[i]) {
                    if (sn[i] >= A.n - 1 || sk[i] == 1) fin[i] = true;
                    else { dd[i] = A.sah_dec[sn[i]]; cc[i] = A.child[sn[i]]; any = true; }
                }
            }
            if (!any) break;
            int tn[8], tk[8];
            bool tf[8];
            int m = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (i >= nc) continue;
                if (fin[i]) { tn[m] = sn[i]; tk[m] = sk[i]; tf[m++] = true; continue; }
                // f(slots) <= slots and 1 <= k(f) < f by construction; the
                // clamps keep the list within 8 entries whatever the word holds
                const int j = min(sk[i], (int)((dd[i] >> (21 + 3 * (sk[i] - 2))) & 7u) + 1);
                if (j == 1) { tn[m] = sn[i]; tk[m] = 1; tf[m++] = true; continue; }
                const int kl = min(j - 1, (int)((dd[i] >> (3 * (j - 2))) & 7u) + 1);
                tn[m] = cc[i].x; tk[m] = kl; tf[m++] = false;
                tn[m] = cc[i].y; tk[m] = j - kl; tf[m++] = false;
            }
            nc = m;
            for (int i = 0; i < m; ++i) { sn[i] = tn[i]; sk[i] = tk[i]; fin[i] = tf[i]; }
        }
        for (int i = 0; i < nc; ++i) ch[i] = sn[i];
    } else {
        // greedy expansion; each child's priority (-1: a leaf-sized subtree) is
        // computed once when the child enters the list
        auto prio = [&](int node) {
            const int cnt = subtree_count(A, node);
            if (cnt <= LEAF_MAX) return -1.f;
            return A.rule == AG_COLLAPSE_COUNT ? (float)cnt
                 : A.rule == AG_COLLAPSE_AREA ? half_area(A, node)
                                              : half_area(A, node) * (float)cnt;
        };
        float pr[8];
        int2 c = A.child[b];
        ch[nc] = c.x; pr[nc++] = prio(c.x);
        ch[nc] = c.y; pr[nc++] = prio(c.y);
        while (nc < 8) {
            int best = -1;
            float ba = -1.f;
            for (int k = 0; k < nc; ++k)
                if (pr[k] >= 0.f && pr[k] > ba) { ba = pr[k]; best = k; }
            if (best < 0) break;
            int2 cc = A.child[ch[best]];
            ch[best] = cc.x; pr[best] = prio(cc.x);
            ch[nc] = cc.y; pr[nc++] = prio(cc.y);
        }
    }
    // per child: triangle count, first sorted position and box, the loads of
    // all children issued together
    const float4 nlo = A.box_lo[live ? b : 0], nhi = A.box_hi[live ? b : 0];
    int cnt[8], first[8];
    float clo[3][8], chi[3][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        cnt[k] = 0;
        first[k] = 0;
        clo[0][k] = clo[1][k] = clo[2][k] = 1.f;
        chi[0][k] = chi[1][k] = chi[2][k] = -1.f;
        if (k < nc) {
            const int c = ch[k];
            const int2 r = c >= A.n - 1 ? make_int2(c - (int)(A.n - 1), c - (int)(A.n - 1)) : A.range[c];
            cnt[k] = r.y - r.x + 1;
            first[k] = r.x;
            const float4 lo = A.box_lo[c], hi = A.box_hi[c];
            clo[0][k] = lo.x; clo[1][k] = lo.y; clo[2][k] = lo.z;
            chi[0][k] = hi.x; chi[1][k] = hi.y; chi[2][k] = hi.z;
        }
    }
    int n_int = 0, n_tri = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (cnt[k] > LEAF_MAX) ++n_int;
        else n_tri += cnt[k];
    }
    const unsigned child_base = warp_alloc(A.node_count, (unsigned)n_int);
    const unsigned tri_base = warp_alloc(A.tri_count, (unsigned)n_tri);
    const unsigned q_base = warp_alloc(reinterpret_cast<unsigned *>(A.q_count_out), (unsigned)n_int);
    if (!live) return;
    uint32_t meta[2] = {0u, 0u};
    int rank = 0, toff = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (k >= nc) continue;
        uint32_t m;
        if (cnt[k] > LEAF_MAX) {
            m = 0x80u | (uint32_t)rank;
            q_out[q_base + rank] = make_int2(ch[k], (int)(child_base + rank));
            ++rank;
        } else {
            m = (uint32_t)((cnt[k] << 5) | toff);
            for (int j = 0; j < cnt[k]; ++j) A.rec_pos[tri_base + toff + j] = (uint32_t)(first[k] + j);
            toff += cnt[k];
        }
        meta[k >> 2] |= m << (8 * (k & 3));
    }
    if (A.layout == AG_BVH_Q8) {
        // the 80-byte node as 20 words (the QNode field order), five 16-byte stores
        const float o[3] = {nlo.x, nlo.y, nlo.z}, h[3] = {nhi.x, nhi.y, nhi.z};
        uint32_t qw[12];
        int e[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int ql[8], qh[8];
            e[a] = choose_exp(o[a], h[a], clo[a], chi[a], nc, ql, qh);
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                qw[2 * a + w] = (uint32_t)ql[4 * w] | ((uint32_t)ql[4 * w + 1] << 8) |
                                ((uint32_t)ql[4 * w + 2] << 16) | ((uint32_t)ql[4 * w + 3] << 24);
                qw[6 + 2 * a + w] = (uint32_t)qh[4 * w] | ((uint32_t)qh[4 * w + 1] << 8) |
                                    ((uint32_t)qh[4 * w + 2] << 16) | ((uint32_t)qh[4 * w + 3] << 24);
            }
        }
        const uint32_t hdr = (uint32_t)e[0] | ((uint32_t)e[1] << 8) | ((uint32_t)e[2] << 16) | ((uint32_t)nc << 24);
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<QNode *>(A.nodes) + wslot);
        dst[0] = make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]), hdr);
        dst[1] = make_uint4(child_base, tri_base, meta[0], meta[1]);
        dst[2] = make_uint4(qw[0], qw[1], qw[2], qw[3]);
        dst[3] = make_uint4(qw[4], qw[5], qw[6], qw[7]);
        dst[4] = make_uint4(qw[8], qw[9], qw[10], qw[11]);
    } else {
        FNode nd;
        nd.child_base = child_base;
        nd.tri_base = tri_base;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            nd.meta[k] = (uint8_t)(meta[k >> 2] >> (8 * (k & 3)));
            nd.lox[k] = clo[0][k]; nd.loy[k] = clo[1][k]; nd.loz[k] = clo[2][k];
            nd.hix[k] = chi[0][k]; nd.hiy[k] = chi[1][k]; nd.hiz[k] = chi[2][k];
        }
        static_cast<FNode *>(A.nodes)[wslot] = nd;
    }
}

// one level of the top-down collapse: the level's queue length is read on the
// device, so the levels run back to back without a host round trip
#ifndef AG_COLLAPSE_MIN_BLOCKS
#define AG_COLLAPSE_MIN_BLOCKS 4   // 128 registers: 1.51 -> 1.46 ms per build against no cap (146 registers), 1.61 ms at 6 blocks
#endif
__global__ void __launch_bounds__(128, AG_COLLAPSE_MIN_BLOCKS) k_collapse(CollapseArgs A, const int2 *__restrict__ q_in,
                                                                         const int *__restrict__ nq_in,
                                                                         int2 *__restrict__ q_out) {
    const int nq = *nq_in;
    // the loop bound is uniform over the block, so that whole warps call the
    // counter allocations together
    for (int q0 = blockIdx.x * blockDim.x; q0 < nq; q0 += gridDim.x * blockDim.x) {
        const int qi = q0 + threadIdx.x;
        const bool live = qi < nq;
        collapse_node(A, live ? q_in[qi] : make_int2(0, 0), live, q_out);
    }
}

// the collapse levels from `first` (COLLAPSE_LEVELS) on, all on one CTA (only
// a tree deeper than that gets work here); qa holds the first of them. A queue left
// after COLLAPSE_MAX levels cannot happen for a tree of 30-bit Morton codes
// and at most 2^29 triangles; it would leave levels[COLLAPSE_MAX] set, which
// the summary check reports.
__global__ void __launch_bounds__(256) k_collapse_tail(CollapseArgs A, int2 *qa, int2 *qb, int *levels, int first) {
    int2 *qin = qa, *qout = qb;
    for (int l = first; l < COLLAPSE_MAX; ++l) {
        const int nq = __ldcg(&levels[l]);
        if (nq == 0) return;
        A.q_count_out = levels + l + 1;
        for (int q0 = 0; q0 < nq; q0 += blockDim.x) {
            const int qi = q0 + threadIdx.x;
            const bool live = qi < nq;
            collapse_node(A, live ? qin[qi] : make_int2(0, 0), live, qout);
        }
        __syncthreads();   // the level's nodes, queue and count are complete
        int2 *t = qin;
        qin = qout;
        qout = t;
    }
}

// One level of the top-down collapse with the SAH decisions, eight lanes per
// wide node (a warp takes four nodes of the level's queue): lane i holds the
// node's i-th entry while the decisions are followed (each round every lane
// splits its entry, the group's new list placed by a prefix sum), then its
// child's range and box, its share of the counters, its meta byte and its
// quantised planes (the group searches the exponent together: a candidate
// holds when it holds for every child).  The result is the node
// collapse_node writes for the same item, with one node's loads and
// arithmetic spread over eight lanes rather than chained in one.
__global__ void __launch_bounds__(128) k_collapse_coop(CollapseArgs A, const int2 *__restrict__ q_in,
                                                       const int *__restrict__ nq_in, int2 *__restrict__ q_out) {
    __shared__ int s_sn[4][4][8], s_sk[4][4][8], s_fin[4][4][8];
    const unsigned FULL = 0xffffffffu;
    const int nq = *nq_in;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 3, gl = lane & 7;
    const unsigned gmask = 0xffu << (8 * g);
    const unsigned below = gmask & ((1u << lane) - 1u);
    const int n1 = (int)(A.n - 1);
    // the loop bound is uniform over the warp, so that whole warps call the
    // counter allocations together
    for (int q0 = (blockIdx.x * 4 + warp) * 4; q0 < nq; q0 += gridDim.x * 16) {
        const int qi = q0 + g;
        const bool live = qi < nq;
        const int2 item = live ? q_in[qi] : make_int2(0, 0);
        const int b = item.x;
        const unsigned wslot = (unsigned)item.y;
        // ---- children: the SAH decisions followed breadth first
        int sn = -1, sk = 0;
        bool fin = true;
        int nc = 0;
        if (live) {
            if (b >= n1 || subtree_count(A, b) <= LEAF_MAX) {
                nc = 1;   // only the root of a tiny mesh gets here
                if (gl == 0) sn = b;
            } else {
                nc = 2;
                const int2 c = A.child[b];
                const int kl = (int)((A.sah_dec[b] >> 18) & 7u) + 1;   // k(8) of the root
                if (gl == 0) { sn = c.x; sk = kl; fin = false; }
                if (gl == 1) { sn = c.y; sk = 8 - kl; fin = false; }
            }
        }
        for (int round = 0; round < 8; ++round) {
            if (gl < nc && !fin && (sn >= n1 || sk == 1)) fin = true;
            const bool act = gl < nc && !fin;
            if (!__any_sync(FULL, act)) break;
            int j = 1, kl = 1;
            int2 cc = make_int2(0, 0);
            if (act) {
                const uint64_t dd = A.sah_dec[sn];
                cc = A.child[sn];
                // f(slots) <= slots and 1 <= k(f) < f by construction; the
                // clamps keep the list within 8 entries whatever the word holds
                j = min(sk, (int)((dd >> (21 + 3 * (sk - 2))) & 7u) + 1);
                if (j > 1) kl = min(j - 1, (int)((dd >> (3 * (j - 2))) & 7u) + 1);
            }
            const bool split = act && j > 1;
            const int pc = gl < nc ? (split ? 2 : 1) : 0;
            int pre = pc;   // inclusive prefix over the group's lanes
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const int t = __shfl_up_sync(FULL, pre, o, 8);
                if (gl >= o) pre += t;
            }
            const int m = min(8, __shfl_sync(FULL, pre, 7, 8));
            pre -= pc;
            if (gl < nc && pre + pc <= 8) {   // (a list of at most 8 entries by construction)
                if (!split) {
                    s_sn[warp][g][pre] = sn;
                    s_sk[warp][g][pre] = act ? 1 : sk;
                    s_fin[warp][g][pre] = 1;
                } else {
                    s_sn[warp][g][pre] = cc.x; s_sk[warp][g][pre] = kl; s_fin[warp][g][pre] = 0;
                    s_sn[warp][g][pre + 1] = cc.y; s_sk[warp][g][pre + 1] = j - kl; s_fin[warp][g][pre + 1] = 0;
                }
            }
            __syncwarp();
            if (gl < m) {
                sn = s_sn[warp][g][gl];
                sk = s_sk[warp][g][gl];
                fin = s_fin[warp][g][gl] != 0;
            }
            nc = m;
            __syncwarp();
        }
        // ---- this lane's child: triangle count, first sorted position, box
        const bool has = live && gl < nc;
        int cnt = 0, first = 0;
        float clo[3] = {1.f, 1.f, 1.f}, chi[3] = {-1.f, -1.f, -1.f};
        if (has) {
            const int2 r = sn >= n1 ? make_int2(sn - n1, sn - n1) : A.range[sn];
            cnt = r.y - r.x + 1;
            first = r.x;
            const float4 lo = A.box_lo[sn], hi = A.box_hi[sn];
            clo[0] = lo.x; clo[1] = lo.y; clo[2] = lo.z;
            chi[0] = hi.x; chi[1] = hi.y; chi[2] = hi.z;
        }
        const float4 nlo = A.box_lo[live ? b : 0], nhi = A.box_hi[live ? b : 0];
        const bool inner = has && cnt > LEAF_MAX;
        const unsigned bal_inner = __ballot_sync(FULL, inner);
        const int n_int = __popc(bal_inner & gmask);
        const int rank = __popc(bal_inner & below);
        const int lcnt = has && !inner ? cnt : 0;
        int toff = lcnt;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int t = __shfl_up_sync(FULL, toff, o, 8);
            if (gl >= o) toff += t;
        }
        const int n_tri = __shfl_sync(FULL, toff, 7, 8);
        toff -= lcnt;
        // ---- allocations: one request per node, made by its first lane
        const unsigned cb = warp_alloc(A.node_count, gl == 0 ? (unsigned)n_int : 0u);
        const unsigned tb = warp_alloc(A.tri_count, gl == 0 ? (unsigned)n_tri : 0u);
        const unsigned qb = warp_alloc(reinterpret_cast<unsigned *>(A.q_count_out), gl == 0 ? (unsigned)n_int : 0u);
        const unsigned child_base = __shfl_sync(FULL, cb, 0, 8);
        const unsigned tri_base = __shfl_sync(FULL, tb, 0, 8);
        const unsigned q_base = __shfl_sync(FULL, qb, 0, 8);
        uint32_t m8 = 0;
        if (inner) {
            m8 = 0x80u | (uint32_t)rank;
            q_out[q_base + rank] = make_int2(sn, (int)(child_base + rank));
        } else if (has) {
            m8 = (uint32_t)((cnt << 5) | toff);
            for (int t = 0; t < cnt; ++t) A.rec_pos[tri_base + toff + t] = (uint32_t)(first + t);
        }
        // bytes of the lanes 4w..4w+3 into one word (every lane of the four gets it)
        auto gather4 = [&](uint32_t byte) {
            uint32_t w = byte << (8 * (gl & 3));
            w |= __shfl_xor_sync(FULL, w, 1);
            w |= __shfl_xor_sync(FULL, w, 2);
            return w;
        };
        const uint32_t meta_w = gather4(m8);
        if (A.layout == AG_BVH_Q8) {
            const float o[3] = {nlo.x, nlo.y, nlo.z}, hn[3] = {nhi.x, nhi.y, nhi.z};
            uint32_t qlw[3], qhw[3];
            int e[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // the smallest exponent from the node extent's estimate up
                // that quantises every child into 0..255 with outward
                // rounding verified in the traversal's decode fmaf(q, 2^e, o)
                const float ext = hn[a] - o[a];
                int ea;
                if (!(ext > 0.f)) ea = 1;
                else {
                    int ex;
                    frexpf(ext / 255.0f, &ex);
                    ea = max(1, min(254, ex + 127 - 1));
                }
                int ql = 255, qh = 0;
                for (;; ++ea) {
                    const float sc = __uint_as_float((unsigned)ea << 23);
                    const float inv = 1.0f / sc;   // a power of two: x * inv is exactly x / sc
                    bool ok = true;
                    ql = 255;
                    qh = 0;
                    if (has) {
                        ql = (int)floorf((clo[a] - o[a]) * inv);
                        ql = max(0, min(255, ql));
                        while (ql > 0 && fmaf((float)ql, sc, o[a]) > clo[a]) --ql;
                        int h = (int)ceilf((chi[a] - o[a]) * inv);
                        h = max(0, h);
                        while (h <= 255 && fmaf((float)h, sc, o[a]) < chi[a]) ++h;
                        while (h > 0 && h - 1 >= ql && fmaf((float)(h - 1), sc, o[a]) >= chi[a]) --h;
                        if (h > 255 || fmaf((float)ql, sc, o[a]) > clo[a]) ok = false;
                        qh = min(h, 255);
                    }
                    if (__all_sync(gmask, ok) || ea >= 254) break;   // the group searches together
                }
                e[a] = ea;
                qlw[a] = gather4((uint32_t)ql);
                qhw[a] = gather4((uint32_t)qh);
            }
            // the second word of each byte row sits in lane 4 of the group
            const int src = (lane & ~7) | 4;
            const uint32_t meta_hi = __shfl_sync(FULL, meta_w, src);
            uint32_t qlh[3], qhh[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                qlh[a] = __shfl_sync(FULL, qlw[a], src);
                qhh[a] = __shfl_sync(FULL, qhw[a], src);
            }
            if (live && gl == 0) {
                const uint32_t hdr = (uint32_t)e[0] | ((uint32_t)e[1] << 8) | ((uint32_t)e[2] << 16) | ((uint32_t)nc << 24);
                uint4 *dst = reinterpret_cast<uint4 *>(static_cast<QNode *>(A.nodes) + wslot);
                dst[0] = make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]), hdr);
                dst[1] = make_uint4(child_base, tri_base, meta_w, meta_hi);
                dst[2] = make_uint4(qlw[0], qlh[0], qlw[1], qlh[1]);
                dst[3] = make_uint4(qlw[2], qlh[2], qhw[0], qhh[0]);
                dst[4] = make_uint4(qhw[1], qhh[1], qhw[2], qhh[2]);
            }
        } else {
            const uint32_t meta_hi = __shfl_sync(FULL, meta_w, (lane & ~7) | 4);
            if (live) {
                FNode *nd = static_cast<FNode *>(A.nodes) + wslot;
                nd->lox[gl] = clo[0]; nd->loy[gl] = clo[1]; nd->loz[gl] = clo[2];
                nd->hix[gl] = chi[0]; nd->hiy[gl] = chi[1]; nd->hiz[gl] = chi[2];
                if (gl == 0) {
                    nd->child_base = child_base;
                    nd->tri_base = tri_base;
                    reinterpret_cast<uint32_t *>(nd->meta)[0] = meta_w;
                    reinterpret_cast<uint32_t *>(nd->meta)[1] = meta_hi;
                }
            }
        }
    }
}

// the 48-byte leaf-order triangle records, one thread per record
__global__ void k_tri_records(const uint32_t *__restrict__ rec_pos, const unsigned *__restrict__ vals,
                              const float *__restrict__ V, const int32_t *__restrict__ F, int64_t nv, int64_t n,
                              float4 *__restrict__ tris, int32_t *__restrict__ tri_ids) {
    const int64_t rec = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (rec >= n) return;
    const unsigned orig = vals[rec_pos[rec]];
    int32_t id[3] = {F[3 * (int64_t)orig], F[3 * (int64_t)orig + 1], F[3 * (int64_t)orig + 2]};
    if (id[0] < 0 || id[0] >= nv || id[1] < 0 || id[1] >= nv || id[2] < 0 || id[2] >= nv)
        id[0] = id[1] = id[2] = 0;   // reported through the status word by k_tri_prep
    for (int v = 0; v < 3; ++v) {
        const float *p = V + 3 * (int64_t)id[v];
        tris[3 * rec + v] = make_float4(p[0], p[1], p[2], __int_as_float(id[v]));
    }
    tri_ids[rec] = (int32_t)orig;
}

// level 0 of the collapse queue: the binary root (internal node 0, or leaf 0
// for a one-triangle mesh), node counter 1, triangle counter 0
__global__ void k_collapse_init(int2 *q0, int *counts, unsigned *counters) {
    q0[0] = make_int2(0, 0);
    counts[0] = 1;
    counters[0] = 1u;
    counters[1] = 0u;
}

// bound keys: min keys start at all ones, max keys at zero
__global__ void k_bounds_init(unsigned *bounds) {
    const int q = threadIdx.x;
    if (q < 16) bounds[q] = (q < 3 || (q >= 6 && q < 9)) ? 0xffffffffu : 0u;
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

ag_status build_bvh(const float *d_verts, int64_t nv, const int32_t *d_faces, int64_t nf, int layout, int rule,
                    bool sync, cudaStream_t s, ag_bvh *h) {
    int dev = h->device;
    unsigned *status = device_status_word(dev);
    Scratch sc(s, dev);
    const int64_t n = nf;
    float4 *tlo, *thi, *cent, *box_lo, *box_hi;
    unsigned *k0, *v0, *k1, *v1, *hist;
    int2 *child, *range, *q0, *q1;
    int *parent, *flags;
    void *nscr;
    const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    const int64_t nbin = 2 * n - 1;
    AG_CUDA(sc.alloc((void **)&tlo, sizeof(float4) * n));
    AG_CUDA(sc.alloc((void **)&thi, sizeof(float4) * n));
    AG_CUDA(sc.alloc((void **)&cent, sizeof(float4) * n));
    AG_CUDA(sc.alloc((void **)&k0, sizeof(unsigned) * n));
    AG_CUDA(sc.alloc((void **)&v0, sizeof(unsigned) * n));
    AG_CUDA(sc.alloc((void **)&k1, sizeof(unsigned) * n));
    AG_CUDA(sc.alloc((void **)&v1, sizeof(unsigned) * n));
    AG_CUDA(sc.alloc((void **)&hist, sizeof(unsigned) * 256 * (size_t)nblocks));
    void *scan_tmp = nullptr;
    AG_CUDA(sc.alloc(&scan_tmp, scan_scratch_bytes((int64_t)256 * nblocks)));
    AG_CUDA(sc.alloc((void **)&child, sizeof(int2) * std::max<int64_t>(1, n - 1)));
    AG_CUDA(sc.alloc((void **)&range, sizeof(int2) * std::max<int64_t>(1, n - 1)));
    AG_CUDA(sc.alloc((void **)&parent, sizeof(int) * nbin));
    AG_CUDA(sc.alloc((void **)&flags, sizeof(int) * std::max<int64_t>(1, n - 1)));
    AG_CUDA(sc.alloc((void **)&box_lo, sizeof(float4) * nbin));
    AG_CUDA(sc.alloc((void **)&box_hi, sizeof(float4) * nbin));
    AG_CUDA(sc.alloc((void **)&q0, sizeof(int2) * std::max<int64_t>(1, n)));
    AG_CUDA(sc.alloc((void **)&q1, sizeof(int2) * std::max<int64_t>(1, n)));
    AG_CUDA(sc.alloc(&nscr, vertex_normal_scratch_bytes(nv, n)));
    uint32_t *rec_pos;
    AG_CUDA(sc.alloc((void **)&rec_pos, sizeof(uint32_t) * n));

    // arrays owned by the handle, from the device's memory pool so that
    // rebuilds reuse them: nodes for the worst-case count (one per internal
    // node of the binary tree; a synchronous build trims them to the count),
    // triangle records, ids, vertex normals and the build summary
    const int64_t max_nodes = std::max<int64_t>(1, n - 1);
    const size_t node_size = layout == AG_BVH_Q8 ? sizeof(QNode) : sizeof(FNode);
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return set_error(AG_ERR_OOM, "memory pool unavailable");
    AG_CUDA(cudaMallocFromPoolAsync(&h->nodes, node_size * max_nodes, pool, s));
    AG_CUDA(cudaMallocFromPoolAsync((void **)&h->tris, sizeof(float4) * 3 * n, pool, s));
    AG_CUDA(cudaMallocFromPoolAsync((void **)&h->tri_ids, sizeof(int32_t) * n, pool, s));
    AG_CUDA(cudaMallocFromPoolAsync((void **)&h->vnormals, sizeof(float4) * nv, pool, s));
    AG_CUDA(cudaMallocFromPoolAsync(&h->d_info, sizeof(BuildSummary), pool, s));
    BuildSummary *info = static_cast<BuildSummary *>(h->d_info);
    unsigned *bounds = info->bounds, *counters = info->counters;
    int *lcounts = info->levels;
    AG_CUDA(cudaEventCreate(&h->ev_start));
    AG_CUDA(cudaEventCreate(&h->ev_done));
    AG_CUDA(cudaEventRecord(h->ev_start, s));

    AG_CUDA(cudaMemsetAsync(info, 0, sizeof(BuildSummary), s));
    k_bounds_init<<<1, 32, 0, s>>>(bounds);
    AG_CUDA_LAUNCH("k_bounds_init");
    // the high mesh's vertex normals need nothing of the tree: they run on a
    // library side stream beside the build's chain of latency-bound kernels
    // and join it at the end
    cudaStream_t *side = nullptr;
    AG_CUDA(side_streams(dev, &side));
    cudaStream_t *nside = side + 1;
    EventSet es;
    AG_CUDA(fork_to(s, nside, 1, es));
    AG_CUDA(launch_vertex_normals(d_verts, d_faces, nv, n, nullptr, nullptr, h->vnormals, nullptr, nscr, nside[0]));
    k_tri_prep<<<grid_for(n, 256), 256, 0, s>>>(d_verts, d_faces, nv, n, tlo, thi, cent, bounds, status);
    AG_CUDA_LAUNCH("k_tri_prep");
    k_morton<<<grid_for(n, 256), 256, 0, s>>>(cent, n, bounds, k0, v0);
    AG_CUDA_LAUNCH("k_morton");
    unsigned *ka = k0, *va = v0, *kb = k1, *vb = v1;
    for (int pass = 0; pass < 4; ++pass) {
        int shift = pass * 8;
        k_rs_hist<<<nblocks, RS_BLOCK, 0, s>>>(ka, n, shift, hist, nblocks);
        AG_CUDA_LAUNCH("k_rs_hist");
        AG_CUDA(launch_scan_exclusive(hist, (int64_t)256 * nblocks, nullptr, scan_tmp, s));
        k_rs_scatter<<<nblocks, RS_BLOCK, 0, s>>>(ka, va, kb, vb, n, shift, hist, nblocks);
        AG_CUDA_LAUNCH("k_rs_scatter");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (n > 1) {
        k_karras<<<grid_for(n - 1, 256), 256, 0, s>>>(ka, n, child, range, parent);
        AG_CUDA_LAUNCH("k_karras");
        AG_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * (n - 1), s));
    }
    float *sah = nullptr;
    uint64_t *sah_dec = nullptr;
    if (rule == AG_COLLAPSE_SAH) {
        const size_t n_int = (size_t)std::max<int64_t>(1, n - 1);
        AG_CUDA(sc.alloc((void **)&sah, sizeof(float) * 8 * n_int));
        AG_CUDA(sc.alloc((void **)&sah_dec, sizeof(uint64_t) * n_int));
    }
    k_bounds<<<grid_for(n, 256), 256, 0, s>>>(va, n, tlo, thi, child, range, parent, box_lo, box_hi, flags, sah,
                                              sah_dec);
    AG_CUDA_LAUNCH("k_bounds");

    // top-down collapse: one launch per level for the first COLLAPSE_LEVELS
    // levels (queue lengths stay on the device), then one CTA for any deeper
    // levels; the host never waits
    CollapseArgs A;
    A.n = n; A.child = child; A.range = range; A.box_lo = box_lo; A.box_hi = box_hi; A.vals = va;
    A.V = d_verts; A.F = d_faces; A.nv = nv; A.layout = layout; A.rule = rule; A.nodes = h->nodes; A.tris = h->tris;
    A.tri_ids = h->tri_ids; A.node_count = counters; A.tri_count = counters + 1; A.rec_pos = rec_pos;
    A.sah_dec = sah_dec;
    k_collapse_init<<<1, 1, 0, s>>>(q0, lcounts, counters);
    AG_CUDA_LAUNCH("k_collapse_init");
    const unsigned cgrid = (unsigned)std::min<int64_t>(grid_for(n, 128), (int64_t)device_sm_count(dev) * 16);
    // AG_TEST_GRID_LEVELS (tests only) hands the tree to the one-CTA path
    // after fewer levels, so that path runs on ordinary meshes
    int grid_levels = COLLAPSE_LEVELS;
    if (const char *e = getenv("AG_TEST_GRID_LEVELS")) grid_levels = std::max(0, std::min(COLLAPSE_LEVELS, atoi(e)));
    int2 *qin = q0, *qout = q1;
    // the SAH collapse takes eight lanes per wide node
    const unsigned cgrid_coop = (unsigned)std::min<int64_t>(grid_for(n, 16), (int64_t)device_sm_count(dev) * 32);
    for (int l = 0; l < grid_levels; ++l) {
        A.q_count_out = lcounts + l + 1;
        if (rule == AG_COLLAPSE_SAH) k_collapse_coop<<<cgrid_coop, 128, 0, s>>>(A, qin, lcounts + l, qout);
        else k_collapse<<<cgrid, 128, 0, s>>>(A, qin, lcounts + l, qout);
        AG_CUDA_LAUNCH("k_collapse");
        std::swap(qin, qout);
    }
    k_collapse_tail<<<1, 256, 0, s>>>(A, qin, qout, lcounts, grid_levels);
    AG_CUDA_LAUNCH("k_collapse_tail");
    k_tri_records<<<grid_for(n, 256), 256, 0, s>>>(rec_pos, va, d_verts, d_faces, nv, n, h->tris, h->tri_ids);
    AG_CUDA_LAUNCH("k_tri_records");
    AG_CUDA(join_from(s, nside, 1, es));
    AG_CUDA(cudaEventRecord(h->ev_done, s));
    h->n_nodes = max_nodes;   // until the summary is read
    if (!sync) return AG_OK;

    ag_status st = bvh_ready(h);
    if (st != AG_OK) return st;
    if (h->n_nodes < max_nodes) {
        void *trimmed = nullptr;
        AG_CUDA(cudaMallocFromPoolAsync(&trimmed, node_size * h->n_nodes, pool, s));
        AG_CUDA(cudaMemcpyAsync(trimmed, h->nodes, node_size * h->n_nodes, cudaMemcpyDeviceToDevice, s));
        AG_CUDA(cudaFreeAsync(h->nodes, s));
        h->nodes = trimmed;
    }
    return AG_OK;
}

// read the build summary once the build has finished (waits for it)
ag_status bvh_ready(ag_bvh *h) {
    if (h->ready) return AG_OK;
    AG_CUDA(cudaEventSynchronize(h->ev_done));
    BuildSummary bs;
    AG_CUDA(cudaMemcpy(&bs, h->d_info, sizeof(bs), cudaMemcpyDeviceToHost));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev_start, h->ev_done);
    cudaEventDestroy(h->ev_start);
    cudaEventDestroy(h->ev_done);
    h->ev_start = h->ev_done = nullptr;
    h->build_ms = ms;
    h->ready = true;
    int depth = 0;
    while (depth <= COLLAPSE_MAX && bs.levels[depth] > 0) ++depth;
    h->max_depth = depth;
    auto k2f = [](unsigned k) {
        unsigned b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
        float f;
        memcpy(&f, &b, 4);
        return f;
    };
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        h->lo[a] = k2f(bs.bounds[6 + a]);
        h->hi[a] = k2f(bs.bounds[9 + a]);
        double e = (double)h->hi[a] - (double)h->lo[a];
        d2 += e * e;
    }
    h->diam = (float)sqrt(d2);
    if ((int64_t)bs.counters[1] != h->n_tris || bs.levels[COLLAPSE_MAX] > 0)
        return set_error(AG_ERR_CUDA, "BVH collapse wrote %u of %lld triangle records", bs.counters[1],
                         (long long)h->n_tris);
    h->n_nodes = bs.counters[0];
    return AG_OK;
}

cudaError_t wait_build(const ag_bvh *h, cudaStream_t s) {
    if (h->ready || !h->ev_done) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;   // a capture orders it itself
    return cudaStreamWaitEvent(s, h->ev_done, 0);
}

ag_status scene_abs_for(ag_bvh *h, float *out) {
    *out = 0.f;
    if (h->layout == AG_BVH_Q8) return AG_OK;
    ag_status st = bvh_ready(h);
    if (st) return st;
    for (int k = 0; k < 3; ++k) *out = fmaxf(*out, fmaxf(fabsf(h->lo[k]), fabsf(h->hi[k])));
    return AG_OK;
}

}  // namespace ag
