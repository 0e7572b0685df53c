// LBVH over the high-poly mesh (Sec. 6.4: "A GPU BVH built on the high-poly
// mesh"), built entirely on the device:
//   triangle bounds + centroid bounds -> 30-bit Morton codes -> LSD radix
//   sort (8-bit digits, stable warp-ranked scatter) -> Karras (2012) binary
//   hierarchy -> bottom-up FP32 boxes -> top-down collapse to 8-wide nodes
//   (greedy largest-area expansion, leaves of <= 2 triangles) with child boxes
//   quantised to 8 bits and rounded outward (or kept in FP32) -> triangles
//   reordered into 48-byte leaf-order records -> area-weighted vertex normals.
#include "ag_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace ag {
namespace {

constexpr int RS_BLOCK = 256;
// collapse levels launched before the host checks the queue (a 30-bit Morton
// tree collapses to about 12 levels of 8-wide nodes)
constexpr int COLLAPSE_LEVELS = 24;
constexpr int RS_ROUNDS = 16;
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
__device__ __forceinline__ int delta(const unsigned *__restrict__ k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    unsigned a = k[i], b = k[j];
    if (a == b) return 32 + __clz((unsigned)(i ^ j));
    return __clz(a ^ b);
}

__global__ void k_karras(const unsigned *__restrict__ k, int64_t n, int2 *__restrict__ child,
                         int2 *__restrict__ range, int *__restrict__ parent) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(k, n, i, i - d);
    int64_t lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = delta(k, n, i, j);
    int64_t s = 0;
    int64_t div = 2;
    while (true) {
        int64_t t = (l + div - 1) / div;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
        div <<= 1;
    }
    int64_t gamma = i + s * d + min(d, 0);
    int64_t lo = min(i, j), hi = max(i, j);
    int left = (lo == gamma) ? (int)(n - 1 + gamma) : (int)gamma;
    int right = (hi == gamma + 1) ? (int)(n - 1 + gamma + 1) : (int)(gamma + 1);
    child[i] = make_int2(left, right);
    range[i] = make_int2((int)lo, (int)hi);
    parent[left] = (int)i;
    parent[right] = (int)i;
}

// ---- SAH-optimal collapse (AG_COLLAPSE_SAH) ---------------------------------------------
// cost[8 * node + i - 1] = C(node, i): the least surface-area cost of the
// node's subtree when it may take up to i child slots of its wide parent.
//   leaf (a subtree of <= LEAF_MAX triangles): A(n) * SAH_TRI * count;
//   C(n, 1) = leaf cost, or A(n) * SAH_NODE + D(n, 8) for a wide node;
//   D(n, j) = min over k of C(left, k) + C(right, j - k);
//   C(n, i) = min(C(n, i - 1), D(n, i)) for i >= 2 (a leaf-sized subtree may
//   still spread over several slots as smaller leaves).
// Computed in the bottom-up box pass (the second child to arrive computes the
// parent's box, then its costs).
constexpr float SAH_NODE = 1.0f;
constexpr float SAH_TRI = 0.3f;

__device__ __forceinline__ float box_half_area(float4 lo, float4 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ void sah_node_cost(const int2 *__restrict__ range, const int2 *__restrict__ child,
                                              int64_t n, int64_t node, float a, float *cost) {
    float c[8];
    if (node >= n - 1) {   // one triangle
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = a * SAH_TRI;
    } else {
        const int2 ch = child[node];
        const int2 rg = range[node];
        const int cnt = rg.y - rg.x + 1;
        float cl[8], cr[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            cl[i] = __ldcg(&cost[8 * (int64_t)ch.x + i]);
            cr[i] = __ldcg(&cost[8 * (int64_t)ch.y + i]);
        }
        float d[8];
#pragma unroll
        for (int j = 2; j <= 8; ++j) {
            float best = 3.0e38f;
#pragma unroll
            for (int k = 1; k < j; ++k) best = fminf(best, cl[k - 1] + cr[j - k - 1]);
            d[j - 1] = best;
        }
        c[0] = cnt <= LEAF_MAX ? a * SAH_TRI * (float)cnt : a * SAH_NODE + d[7];
#pragma unroll
        for (int i = 1; i < 8; ++i) c[i] = fminf(c[i - 1], d[i]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) __stcg(&cost[8 * node + i], c[i]);
}

// bottom-up boxes: box_lo/hi [2n-1]; flags [n-1] zeroed; with `cost`, the
// SAH collapse costs of every node in the same pass
__global__ void k_bounds(const unsigned *__restrict__ vals, int64_t n, const float4 *__restrict__ tlo,
                         const float4 *__restrict__ thi, const int2 *__restrict__ child,
                         const int2 *__restrict__ range, const int *__restrict__ parent, float4 *box_lo,
                         float4 *box_hi, int *flags, float *cost) {
    int64_t kk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= n) return;
    int64_t node = n - 1 + kk;
    unsigned t = vals[kk];
    const float4 lo0 = tlo[t], hi0 = thi[t];
    box_lo[node] = lo0;
    box_hi[node] = hi0;
    if (cost) sah_node_cost(range, child, n, node, box_half_area(lo0, hi0), cost);
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
        if (cost) sah_node_cost(range, child, n, p, box_half_area(lo, hi), cost);
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
    const float *sah;             // C(node, 1..8) of the SAH collapse, or null (greedy rules)
};

__device__ __forceinline__ int subtree_count(const CollapseArgs &A, int b) {
    if (b >= A.n - 1) return 1;
    int2 r = A.range[b];
    return r.y - r.x + 1;
}
__device__ __forceinline__ int subtree_first(const CollapseArgs &A, int b) {
    if (b >= A.n - 1) return (int)(b - (A.n - 1));
    return A.range[b].x;
}
__device__ __forceinline__ float half_area(const CollapseArgs &A, int b) {
    float4 lo = A.box_lo[b], hi = A.box_hi[b];
    float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

// smallest power-of-two exponent (biased, as float exponent bits) such that
// every child box quantises into 0..255 with outward rounding verified in the
// exact decode arithmetic of the traversal: fmaf(q, 2^e, origin).
__device__ int choose_exp(float o, float hi_node, const float *clo, const float *chi, int nc,
                          unsigned char *qlo, unsigned char *qhi) {
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
        for (int c = 0; c < nc && ok; ++c) {
            int ql = (int)floorf((clo[c] - o) * inv);
            ql = max(0, min(255, ql));
            while (ql > 0 && fmaf((float)ql, s, o) > clo[c]) --ql;
            int qh = (int)ceilf((chi[c] - o) * inv);
            qh = max(0, qh);
            while (qh <= 255 && fmaf((float)qh, s, o) < chi[c]) ++qh;
            while (qh > 0 && qh - 1 >= ql && fmaf((float)(qh - 1), s, o) >= chi[c]) --qh;
            if (qh > 255 || fmaf((float)ql, s, o) > clo[c]) { ok = false; break; }
            qlo[c] = (unsigned char)ql;
            qhi[c] = (unsigned char)qh;
        }
        if (ok || e >= 254) return e;
    }
}

__device__ void collapse_node(const CollapseArgs &A, int2 item, int2 *__restrict__ q_out) {
    int b = item.x;
    unsigned wslot = (unsigned)item.y;
    int ch[8];
    int nc = 0;
    if (b >= A.n - 1 || subtree_count(A, b) <= LEAF_MAX) {
        ch[nc++] = b;   // only the root of a tiny mesh gets here
    } else if (A.sah) {
        // the slots of the SAH decision: (node, slots) pairs, split while a
        // node takes more than one slot and splitting is what its cost used
        int sn[8], sk[8], top = 0;
        auto split = [&](int node, int j, int &kl) {
            const int2 c = A.child[node];
            float best = 3.0e38f;
            kl = 1;
            for (int k = 1; k < j; ++k) {
                const float v = A.sah[8 * (int64_t)c.x + k - 1] + A.sah[8 * (int64_t)c.y + j - k - 1];
                if (v < best) { best = v; kl = k; }
            }
            return c;
        };
        int kl;
        int2 c = split(b, 8, kl);
        sn[top] = c.y; sk[top++] = 8 - kl;
        sn[top] = c.x; sk[top++] = kl;
        while (top > 0) {
            const int node = sn[--top];
            int j = sk[top];
            // fewer slots do as well: use the fewest that reach the cost
            while (j > 1 && A.sah[8 * (int64_t)node + j - 2] <= A.sah[8 * (int64_t)node + j - 1]) --j;
            if (j == 1 || node >= A.n - 1) {
                ch[nc++] = node;
                continue;
            }
            int k2;
            const int2 cc = split(node, j, k2);
            sn[top] = cc.y; sk[top++] = j - k2;
            sn[top] = cc.x; sk[top++] = k2;
        }
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
    int n_int = 0, n_tri = 0;
    for (int k = 0; k < nc; ++k) {
        int cnt = subtree_count(A, ch[k]);
        if (cnt <= LEAF_MAX) n_tri += cnt; else ++n_int;
    }
    unsigned child_base = n_int ? atomicAdd(A.node_count, (unsigned)n_int) : 0u;
    unsigned tri_base = n_tri ? atomicAdd(A.tri_count, (unsigned)n_tri) : 0u;
    unsigned char meta[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int rank = 0, toff = 0;
    for (int k = 0; k < nc; ++k) {
        int cnt = subtree_count(A, ch[k]);
        if (cnt > LEAF_MAX) {
            meta[k] = (unsigned char)(0x80 | rank);
            int slot = atomicAdd(A.q_count_out, 1);
            q_out[slot] = make_int2(ch[k], (int)(child_base + rank));
            ++rank;
        } else {
            meta[k] = (unsigned char)((cnt << 5) | toff);
            const int first = subtree_first(A, ch[k]);
            for (int j = 0; j < cnt; ++j) A.rec_pos[tri_base + toff + j] = (uint32_t)(first + j);
            toff += cnt;
        }
    }
    // node box = box of binary node b; child boxes
    float clo[3][8], chi[3][8];
    for (int k = 0; k < nc; ++k) {
        float4 lo = A.box_lo[ch[k]], hi = A.box_hi[ch[k]];
        clo[0][k] = lo.x; clo[1][k] = lo.y; clo[2][k] = lo.z;
        chi[0][k] = hi.x; chi[1][k] = hi.y; chi[2][k] = hi.z;
    }
    if (A.layout == AG_BVH_Q8) {
        QNode nd;
        float4 blo = A.box_lo[b], bhi = A.box_hi[b];
        float o[3] = {blo.x, blo.y, blo.z}, h[3] = {bhi.x, bhi.y, bhi.z};
        unsigned char qlo[3][8], qhi[3][8];
        int e[3];
        for (int a = 0; a < 3; ++a) {
            e[a] = choose_exp(o[a], h[a], clo[a], chi[a], nc, qlo[a], qhi[a]);
            for (int k = nc; k < 8; ++k) { qlo[a][k] = 255; qhi[a][k] = 0; }
        }
        nd.ox = o[0]; nd.oy = o[1]; nd.oz = o[2];
        nd.ex = (uint8_t)e[0]; nd.ey = (uint8_t)e[1]; nd.ez = (uint8_t)e[2];
        nd.nchild = (uint8_t)nc;
        nd.child_base = child_base;
        nd.tri_base = tri_base;
        for (int k = 0; k < 8; ++k) {
            nd.meta[k] = meta[k];
            nd.qlox[k] = qlo[0][k]; nd.qloy[k] = qlo[1][k]; nd.qloz[k] = qlo[2][k];
            nd.qhix[k] = qhi[0][k]; nd.qhiy[k] = qhi[1][k]; nd.qhiz[k] = qhi[2][k];
        }
        ((QNode *)A.nodes)[wslot] = nd;
    } else {
        FNode nd;
        nd.child_base = child_base;
        nd.tri_base = tri_base;
        for (int k = 0; k < 8; ++k) {
            nd.meta[k] = meta[k];
            bool v = k < nc;
            nd.lox[k] = v ? clo[0][k] : 1.f; nd.loy[k] = v ? clo[1][k] : 1.f; nd.loz[k] = v ? clo[2][k] : 1.f;
            nd.hix[k] = v ? chi[0][k] : -1.f; nd.hiy[k] = v ? chi[1][k] : -1.f; nd.hiz[k] = v ? chi[2][k] : -1.f;
        }
        ((FNode *)A.nodes)[wslot] = nd;
    }
}

// one level of the top-down collapse: the level's queue length is read on the
// device, so the levels run back to back without a host round trip
__global__ void k_collapse(CollapseArgs A, const int2 *__restrict__ q_in, const int *__restrict__ nq_in,
                           int2 *__restrict__ q_out) {
    const int nq = *nq_in;
    for (int qi = blockIdx.x * blockDim.x + threadIdx.x; qi < nq; qi += gridDim.x * blockDim.x)
        collapse_node(A, q_in[qi], q_out);
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
                    cudaStream_t s, ag_bvh *h) {
    int dev = h->device;
    unsigned *status = device_status_word(dev);
    Scratch sc(s, dev);
    const int64_t n = nf;
    float4 *tlo, *thi, *cent, *box_lo, *box_hi;
    unsigned *bounds, *k0, *v0, *k1, *v1, *hist;
    int2 *child, *range, *q0, *q1;
    int *parent, *flags, *qcount;
    unsigned *counters;
    void *nscr;
    const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    const int64_t nbin = 2 * n - 1;
    AG_CUDA(sc.alloc((void **)&tlo, sizeof(float4) * n));
    AG_CUDA(sc.alloc((void **)&thi, sizeof(float4) * n));
    AG_CUDA(sc.alloc((void **)&cent, sizeof(float4) * n));
    AG_CUDA(sc.alloc((void **)&bounds, sizeof(unsigned) * 16));
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
    AG_CUDA(sc.alloc((void **)&qcount, sizeof(int) * 2));
    AG_CUDA(sc.alloc((void **)&counters, sizeof(unsigned) * 2));
    AG_CUDA(sc.alloc(&nscr, vertex_normal_scratch_bytes(nv, n)));

    // persistent arrays owned by the handle (worst-case node count, compacted
    // later), from the device's memory pool so that rebuilds reuse them
    const int64_t max_nodes = std::max<int64_t>(1, n - 1);
    const size_t node_size = layout == AG_BVH_Q8 ? sizeof(QNode) : sizeof(FNode);
    void *nodes_tmp = nullptr;
    uint32_t *rec_pos;
    int *lcounts;
    AG_CUDA(sc.alloc(&nodes_tmp, node_size * max_nodes));
    AG_CUDA(sc.alloc((void **)&rec_pos, sizeof(uint32_t) * n));
    AG_CUDA(sc.alloc((void **)&lcounts, sizeof(int) * (COLLAPSE_LEVELS + 1)));
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return set_error(AG_ERR_OOM, "memory pool unavailable");
    AG_CUDA(cudaMallocFromPoolAsync((void **)&h->tris, sizeof(float4) * 3 * n, pool, s));
    AG_CUDA(cudaMallocFromPoolAsync((void **)&h->tri_ids, sizeof(int32_t) * n, pool, s));
    AG_CUDA(cudaMallocFromPoolAsync((void **)&h->vnormals, sizeof(float4) * nv, pool, s));

    cudaEvent_t e0, e1;
    AG_CUDA(cudaEventCreate(&e0));
    AG_CUDA(cudaEventCreate(&e1));
    AG_CUDA(cudaEventRecord(e0, s));

    k_bounds_init<<<1, 32, 0, s>>>(bounds);
    AG_CUDA_LAUNCH("k_bounds_init");
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
    if (rule == AG_COLLAPSE_SAH) AG_CUDA(sc.alloc((void **)&sah, sizeof(float) * 8 * (size_t)nbin));
    k_bounds<<<grid_for(n, 256), 256, 0, s>>>(va, n, tlo, thi, child, range, parent, box_lo, box_hi, flags, sah);
    AG_CUDA_LAUNCH("k_bounds");

    // top-down collapse, one launch per level; the queue lengths stay on the
    // device, and the host looks at them once after COLLAPSE_LEVELS levels
    CollapseArgs A;
    A.n = n; A.child = child; A.range = range; A.box_lo = box_lo; A.box_hi = box_hi; A.vals = va;
    A.V = d_verts; A.F = d_faces; A.nv = nv; A.layout = layout; A.rule = rule; A.nodes = nodes_tmp; A.tris = h->tris;
    A.tri_ids = h->tri_ids; A.node_count = counters; A.tri_count = counters + 1; A.rec_pos = rec_pos; A.sah = sah;
    AG_CUDA(cudaMemsetAsync(lcounts, 0, sizeof(int) * (COLLAPSE_LEVELS + 1), s));
    k_collapse_init<<<1, 1, 0, s>>>(q0, lcounts, counters);
    AG_CUDA_LAUNCH("k_collapse_init");
    const unsigned cgrid = (unsigned)std::min<int64_t>(grid_for(n, 128), (int64_t)device_sm_count(dev) * 16);
    int2 *qin = q0, *qout = q1;
    for (int l = 0; l < COLLAPSE_LEVELS; ++l) {
        A.q_count_out = lcounts + l + 1;
        k_collapse<<<cgrid, 128, 0, s>>>(A, qin, lcounts + l, qout);
        AG_CUDA_LAUNCH("k_collapse");
        std::swap(qin, qout);
    }
    int hl[COLLAPSE_LEVELS + 1];
    AG_CUDA(cudaMemcpyAsync(hl, lcounts, sizeof(hl), cudaMemcpyDeviceToHost, s));
    AG_CUDA(cudaStreamSynchronize(s));
    int depth = 0;
    while (depth <= COLLAPSE_LEVELS && hl[depth] > 0) ++depth;
    // a deeper tree than that (many equal Morton codes) continues level by level
    int nq = hl[COLLAPSE_LEVELS];
    while (nq > 0) {
        AG_CUDA(cudaMemsetAsync(lcounts + 1, 0, sizeof(int), s));
        AG_CUDA(cudaMemcpyAsync(lcounts, &nq, sizeof(int), cudaMemcpyHostToDevice, s));
        A.q_count_out = lcounts + 1;
        k_collapse<<<cgrid, 128, 0, s>>>(A, qin, lcounts, qout);
        AG_CUDA_LAUNCH("k_collapse");
        AG_CUDA(cudaMemcpyAsync(&nq, lcounts + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        AG_CUDA(cudaStreamSynchronize(s));
        std::swap(qin, qout);
        ++depth;
    }
    k_tri_records<<<grid_for(n, 256), 256, 0, s>>>(rec_pos, va, d_verts, d_faces, nv, n, h->tris, h->tri_ids);
    AG_CUDA_LAUNCH("k_tri_records");
    unsigned hc[2];
    AG_CUDA(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
    AG_CUDA(cudaStreamSynchronize(s));
    if ((int64_t)hc[1] != n)
        return set_error(AG_ERR_CUDA, "BVH collapse wrote %u of %lld triangle records", hc[1], (long long)n);
    h->n_nodes = hc[0];
    h->max_depth = depth;
    AG_CUDA(cudaMallocFromPoolAsync(&h->nodes, node_size * h->n_nodes, pool, s));
    AG_CUDA(cudaMemcpyAsync(h->nodes, nodes_tmp, node_size * h->n_nodes, cudaMemcpyDeviceToDevice, s));

    AG_CUDA(launch_vertex_normals(d_verts, d_faces, nv, n, nullptr, nullptr, h->vnormals, nullptr, nscr, s));
    AG_CUDA(cudaEventRecord(e1, s));

    unsigned hb[16];
    AG_CUDA(cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, s));
    AG_CUDA(cudaStreamSynchronize(s));
    auto k2f = [](unsigned k) {
        unsigned b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
        float f;
        memcpy(&f, &b, 4);
        return f;
    };
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        h->lo[a] = k2f(hb[6 + a]);
        h->hi[a] = k2f(hb[9 + a]);
        double e = (double)h->hi[a] - (double)h->lo[a];
        d2 += e * e;
    }
    h->diam = (float)sqrt(d2);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->build_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return AG_OK;
}

}  // namespace ag
