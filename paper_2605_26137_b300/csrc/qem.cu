// QEM mesh simplification (Sec. 6.1): parallel edge collapse ranked by
// quadric error, with the paper's contraction point: the unconstrained
// minimiser of the merged quadric projected onto the edge segment and
// clamped (the midpoint when the quadric is singular); boundary edges go to
// their lower-error endpoint, interior edges with one boundary endpoint to
// that endpoint.
//
// All quadric arithmetic is FP64 with every operation rounded to nearest in
// a fixed order (no fused multiply-adds), so cost ranking, validity and
// positions are decided exactly as the same expressions evaluate on any
// IEEE machine.
//
// A round (all kernels, stream-ordered; the host enqueues eight rounds at a
// time and reads the round control back after them: a one-thread kernel at
// the top of each round decides on the device whether it runs, and every
// kernel of a round that does not run returns at once):
//   1. vertex -> alive face adjacency (degrees counted while the last round
//      rewrote the faces, scan, fill);
//   2. the unique edges a < b, ranked in (a, b) order: every vertex lists its
//      distinct neighbours, sorted, with the faces of each edge (their
//      multiplicity in the list); boundary vertices (on an edge with one
//      face); an exclusive scan of the higher neighbours places the edges;
//   3. per edge: placement, cost E(v), validity (at most two faces, at most
//      64 neighbours per endpoint, link condition, no tetrahedron, no
//      surviving face turning over), key = float32 cost bits << 32 | rank;
//   4. m1(v) = min key at v, m2(v) = min of m1 over v and its neighbours; an
//      edge collapses when its key equals m2 at both ends (such edges never
//      touch adjacent vertices, so their collapses are independent);
//   5. if collapsing all of them would pass the target, only the smallest
//      keys that reach it (a one-block binary search over the selected keys);
//   6. collapse: keep a at v with Q_a + Q_b, rename b to a, drop the faces
//      that held both.
#include "ag_internal.cuh"

#include <algorithm>
#include <cstring>

namespace ag {
namespace {

constexpr int QEM_MAX_NBR = 64;
constexpr int ROUNDS_AHEAD = 8;   // rounds enqueued per host read of the round control
constexpr int64_t COMPACT_MIN = 4096;   // no renumbering below this many working faces
constexpr int TURN_CHUNK = 4;           // faces per step of the turn-over test
constexpr unsigned long long KEY_NONE = ~0ull;

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3v(double x, double y, double z) { D3 r; r.x = x; r.y = y; r.z = z; return r; }
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return d3v(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)); }
__device__ __forceinline__ D3 dadd(D3 a, D3 b) { return d3v(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y), __dadd_rn(a.z, b.z)); }
__device__ __forceinline__ D3 dscl(D3 a, double s) { return d3v(__dmul_rn(a.x, s), __dmul_rn(a.y, s), __dmul_rn(a.z, s)); }
__device__ __forceinline__ double ddot(D3 a, D3 b) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
}
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
    return d3v(__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)), __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
               __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ D3 ldv(const double *V, int64_t i) { return d3v(V[3 * i], V[3 * i + 1], V[3 * i + 2]); }

// plane quadric of a face (10 unique entries, q00 q01 q02 q03 q11 q12 q13 q22 q23 q33); false without a plane
__device__ __forceinline__ bool face_quadric(D3 P0, D3 P1, D3 P2, double K[10]) {
    const D3 n = dcross(dsub(P1, P0), dsub(P2, P0));
    const double len = __dsqrt_rn(ddot(n, n));
    if (!(len > 0.0)) return false;
    const D3 m = d3v(__ddiv_rn(n.x, len), __ddiv_rn(n.y, len), __ddiv_rn(n.z, len));
    const double p[4] = {m.x, m.y, m.z, -ddot(m, P0)};
    int k = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j) K[k++] = __dmul_rn(p[i], p[j]);
    return true;
}

__device__ __forceinline__ double quad_eval(const double q[10], D3 v) {
    double e = __dmul_rn(__dmul_rn(q[0], v.x), v.x);
    e = __dadd_rn(e, __dmul_rn(__dmul_rn(__dmul_rn(2.0, q[1]), v.x), v.y));
    e = __dadd_rn(e, __dmul_rn(__dmul_rn(__dmul_rn(2.0, q[2]), v.x), v.z));
    e = __dadd_rn(e, __dmul_rn(__dmul_rn(2.0, q[3]), v.x));
    e = __dadd_rn(e, __dmul_rn(__dmul_rn(q[4], v.y), v.y));
    e = __dadd_rn(e, __dmul_rn(__dmul_rn(__dmul_rn(2.0, q[5]), v.y), v.z));
    e = __dadd_rn(e, __dmul_rn(__dmul_rn(2.0, q[6]), v.y));
    e = __dadd_rn(e, __dmul_rn(__dmul_rn(q[7], v.z), v.z));
    e = __dadd_rn(e, __dmul_rn(__dmul_rn(2.0, q[8]), v.z));
    e = __dadd_rn(e, q[9]);
    return e;
}

// the paper's placement on the interior edge v0 -> v1: returns t
__device__ __forceinline__ double qem_place(const double q[10], D3 v0, D3 v1) {
    const double a00 = q[0], a01 = q[1], a02 = q[2], a11 = q[4], a12 = q[5], a22 = q[7];
    const double b0 = q[3], b1 = q[6], b2 = q[8];
    const double c00 = __dsub_rn(__dmul_rn(a11, a22), __dmul_rn(a12, a12));
    const double c01 = __dsub_rn(__dmul_rn(a02, a12), __dmul_rn(a01, a22));
    const double c02 = __dsub_rn(__dmul_rn(a01, a12), __dmul_rn(a02, a11));
    const double c11 = __dsub_rn(__dmul_rn(a00, a22), __dmul_rn(a02, a02));
    const double c12 = __dsub_rn(__dmul_rn(a01, a02), __dmul_rn(a00, a12));
    const double c22 = __dsub_rn(__dmul_rn(a00, a11), __dmul_rn(a01, a01));
    const double det = __dadd_rn(__dadd_rn(__dmul_rn(a00, c00), __dmul_rn(a01, c01)), __dmul_rn(a02, c02));
    const double s = fmax(fabs(a00), fmax(fabs(a11), fabs(a22)));
    if (!(fabs(det) > __dmul_rn(__dmul_rn(__dmul_rn(1e-12, s), s), s))) return 0.5;
    const D3 x = d3v(__ddiv_rn(-__dadd_rn(__dadd_rn(__dmul_rn(c00, b0), __dmul_rn(c01, b1)), __dmul_rn(c02, b2)), det),
                     __ddiv_rn(-__dadd_rn(__dadd_rn(__dmul_rn(c01, b0), __dmul_rn(c11, b1)), __dmul_rn(c12, b2)), det),
                     __ddiv_rn(-__dadd_rn(__dadd_rn(__dmul_rn(c02, b0), __dmul_rn(c12, b1)), __dmul_rn(c22, b2)), det));
    const D3 e = dsub(v1, v0);
    const double ee = ddot(e, e);
    if (!(ee > 0.0)) return 0.0;
    double t = __ddiv_rn(ddot(dsub(x, v0), e), ee);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

__device__ __forceinline__ unsigned long long qem_key(double cost, uint32_t rank) {
    const float c = __double2float_rn(cost > 0.0 ? cost : 0.0);
    return ((unsigned long long)__float_as_uint(c) << 32) | rank;
}

__device__ __forceinline__ bool has(const int32_t *F, int64_t f, int32_t v) {
    return F[3 * f] == v || F[3 * f + 1] == v || F[3 * f + 2] == v;
}

inline unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

struct Counters {
    unsigned long long alive;       // alive faces
    unsigned long long removable;   // faces the selected collapses would remove
    int nsel;              // selected collapses
    int pad;
};

// Round control, on the device: the host enqueues rounds ahead and reads
// this back every few rounds; once `done` is set every later kernel returns
// at once.
struct Control {
    long long rounds;   // rounds that ran (a last round that selected nothing is taken back)
    long long ne;       // edges of the current round
    int done;
    int pad;
};

// Decides whether the round runs: not when the last round selected nothing
// (it changed nothing, so it is not counted), nor once the alive faces are at
// or below the target, the round cap is reached or no edge is left.
__global__ void k_round_begin(Control *ctl, Counters *cnt, const unsigned *__restrict__ ne_total, long long target,
                              long long cap) {
    if (threadIdx.x != 0 || ctl->done) return;
    if (ctl->rounds > 0 && cnt->nsel == 0) {
        ctl->rounds -= 1;
        ctl->done = 1;
        return;
    }
    const long long ne = *ne_total;
    if ((long long)cnt->alive <= target || ctl->rounds >= cap || ne == 0) {
        ctl->done = 1;
        return;
    }
    ctl->rounds += 1;
    ctl->ne = ne;
    cnt->removable = 0;
    cnt->nsel = 0;
}

__global__ void k_init_faces(const int32_t *__restrict__ Fin, int64_t nf, int64_t nv, int32_t *__restrict__ F,
                             uint8_t *__restrict__ falive, uint8_t *__restrict__ valive, Counters *cnt,
                             unsigned *status) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int32_t i0 = Fin[3 * f], i1 = Fin[3 * f + 1], i2 = Fin[3 * f + 2];
    F[3 * f] = i0; F[3 * f + 1] = i1; F[3 * f + 2] = i2;
    if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) {
        falive[f] = 0;
        F[3 * f] = F[3 * f + 1] = F[3 * f + 2] = 0;
        atomicOr(status, AGS_BAD_FACE);
        return;
    }
    const bool ok = !(i0 == i1 || i1 == i2 || i0 == i2);
    falive[f] = ok;
    if (!ok) return;
    atomicAdd(&cnt->alive, 1ull);
    valive[i0] = 1; valive[i1] = 1; valive[i2] = 1;
}

__global__ void k_init_verts(const float *__restrict__ Vin, int64_t nv, double *__restrict__ V,
                             float *__restrict__ V32, int32_t *__restrict__ remap) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    V[3 * v] = Vin[3 * v]; V[3 * v + 1] = Vin[3 * v + 1]; V[3 * v + 2] = Vin[3 * v + 2];
    V32[3 * v] = Vin[3 * v]; V32[3 * v + 1] = Vin[3 * v + 1]; V32[3 * v + 2] = Vin[3 * v + 2];
    remap[v] = (int32_t)v;
}

// vertex -> alive faces
__global__ void k_deg(const int32_t *__restrict__ F, const uint8_t *__restrict__ falive, int64_t nf,
                      unsigned *__restrict__ deg) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || !falive[f]) return;
    for (int k = 0; k < 3; ++k) atomicAdd(&deg[F[3 * f + k]], 1u);
}

__global__ void k_fill(const Control *__restrict__ ctl, const int32_t *__restrict__ F,
                       const uint8_t *__restrict__ falive, int64_t nf, const unsigned *__restrict__ off,
                       unsigned *__restrict__ fill, int32_t *__restrict__ list) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || (ctl && ctl->done) || !falive[f]) return;
    for (int k = 0; k < 3; ++k) {
        const int32_t v = F[3 * f + k];
        list[off[v] + atomicAdd(&fill[v], 1u)] = (int32_t)f;
    }
}

// initial quadrics: each vertex sums its faces' plane quadrics in increasing face id
__global__ void k_quadric_init(const double *__restrict__ V, const int32_t *__restrict__ F, int64_t nv,
                               const unsigned *__restrict__ off, int32_t *__restrict__ list, double *__restrict__ Q) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const unsigned b = off[v], e = off[v + 1];
    for (unsigned i = b + 1; i < e; ++i) {
        const int32_t x = list[i];
        unsigned j = i;
        while (j > b && list[j - 1] > x) { list[j] = list[j - 1]; --j; }
        list[j] = x;
    }
    double q[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) q[k] = 0.0;
    for (unsigned i = b; i < e; ++i) {
        const int64_t f = list[i];
        double K[10];
        if (!face_quadric(ldv(V, F[3 * f]), ldv(V, F[3 * f + 1]), ldv(V, F[3 * f + 2]), K)) continue;
#pragma unroll
        for (int k = 0; k < 10; ++k) q[k] = __dadd_rn(q[k], K[k]);
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) Q[10 * v + k] = q[k];
}

// Every vertex's distinct neighbours, sorted ascending, once per round: the
// segment of vertex a starts at 2 off[a] and has room for 2 deg(a) entries
// (each incident face adds at most two), nbr_n[a] holds the count and up[a]
// the count of neighbours above a (the scan input of the ranked edge list).
// The edge list and the edge validity test read these lists instead of
// gathering neighbourhoods again.
// A vertex with more than NB_FAST candidates (two per incident face) is
// handed to k_nbrs_heavy, which sorts them with a whole warp: sorting
// hundreds of candidates by insertion in one thread made the few
// high-valence vertices of the late rounds the kernel's tail.
constexpr int NB_FAST = 32;
constexpr int NB_WARP = 1024;   // candidates a warp sorts in shared memory (more: one lane, in place)

// the sorted unique neighbours of a, by insertion, into nb (n of them), and
// in mult how many of a's faces hold each (the faces of that edge, capped
// at 255)
template <typename M>
__device__ __forceinline__ int insert_nbrs(const int32_t *__restrict__ F, const int32_t *__restrict__ list,
                                           unsigned b, unsigned e, int64_t a, int32_t *nb, M *mult) {
    int n = 0;
    for (unsigned i = b; i < e; ++i) {
        const int64_t f = list[i];
        const int32_t tri[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
        for (int k = 0; k < 3; ++k) {
            const int32_t u = tri[k];
            if (u == a) continue;
            int lo = 0, hi = n;   // insert u into the sorted unique list
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (nb[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (lo < n && nb[lo] == u) {
                if (mult[lo] < 255) mult[lo] = mult[lo] + 1;
                continue;
            }
            for (int m = n; m > lo; --m) {
                nb[m] = nb[m - 1];
                mult[m] = mult[m - 1];
            }
            nb[lo] = u;
            mult[lo] = 1;
            ++n;
        }
    }
    return n;
}

// ascending bitonic sort of the first N of c (all indices fixed at compile
// time, so c stays in registers)
template <int N>
__device__ __forceinline__ void sort_net(int32_t (&c)[NB_FAST]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t x = c[i], y = c[l], lo = min(x, y), hi = max(x, y);
                    if ((i & k) == 0) { c[i] = lo; c[l] = hi; } else { c[i] = hi; c[l] = lo; }
                }
            }
}

// Besides the list: nbr_m, the faces of each edge (a, u), and bnd[a], whether
// a lies on an edge with one face (a boundary vertex). A vertex with at most
// NB_FAST candidates (the two other corners of each incident face) gathers
// them into registers, sorts them with a fixed network and writes the first
// of each run of equal ids with the run's length.
__global__ void k_nbrs(const Control *__restrict__ ctl, const int32_t *__restrict__ F, int64_t nv,
                       const unsigned *__restrict__ off, const int32_t *__restrict__ list, int32_t *__restrict__ nbr,
                       uint8_t *__restrict__ nbr_m, unsigned *__restrict__ nbr_n, unsigned *__restrict__ up,
                       uint8_t *__restrict__ bnd, int32_t *__restrict__ heavy, unsigned *__restrict__ n_heavy) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nv || (ctl && ctl->done)) return;
    const unsigned b = off[a], e = off[a + 1];
    if (2 * (e - b) > NB_FAST) {
        heavy[atomicAdd(n_heavy, 1u)] = (int32_t)a;
        return;
    }
    const unsigned deg = e - b, nc = 2 * deg;
    int32_t c[NB_FAST];
#pragma unroll
    for (int i = 0; i < NB_FAST / 2; ++i) {
        int32_t x = 0x7fffffff, y = 0x7fffffff;
        if (i < (int)deg) {
            const int64_t f = list[b + i];
            const int32_t t0 = F[3 * f], t1 = F[3 * f + 1], t2 = F[3 * f + 2];
            x = t0 == a ? t1 : t0;
            y = t2 == a ? t1 : t2;
        }
        c[2 * i] = x;
        c[2 * i + 1] = y;
    }
    if (nc <= 8) sort_net<8>(c);
    else if (nc <= 16) sort_net<16>(c);
    else sort_net<32>(c);
    int32_t *seg = nbr + 2 * (size_t)b;
    uint8_t *segm = nbr_m + 2 * (size_t)b;
    unsigned n = 0, above = 0, run = 0;
    bool border = false;
#pragma unroll
    for (int m = 0; m < NB_FAST; ++m) {
        if (m < (int)nc) {
            if (m == 0 || c[m] != c[m - 1]) {
                if (m > 0) {
                    segm[n - 1] = (uint8_t)run;
                    border |= run == 1;
                }
                seg[n++] = c[m];
                above += c[m] > a;
                run = 1;
            } else {
                ++run;
            }
        }
    }
    if (n > 0) {
        segm[n - 1] = (uint8_t)run;
        border |= run == 1;
    }
    nbr_n[a] = n;
    up[a] = above;
    bnd[a] = border;
}

// one warp per heavy vertex: the candidates (the two other vertices of each
// incident face) into shared memory, a bitonic sort, then the first of each
// run of equal ids written out in order
__global__ void __launch_bounds__(128) k_nbrs_heavy(const Control *__restrict__ ctl, const int32_t *__restrict__ F,
                                                   const unsigned *__restrict__ off,
                                                   const int32_t *__restrict__ list,
                                                   const int32_t *__restrict__ heavy,
                                                   const unsigned *__restrict__ n_heavy, int32_t *__restrict__ nbr,
                                                   uint8_t *__restrict__ nbr_m, unsigned *__restrict__ nbr_n,
                                                   unsigned *__restrict__ up, uint8_t *__restrict__ bnd) {
    __shared__ int32_t buf[4][NB_WARP];
    if (ctl && ctl->done) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned nh = *n_heavy;
    int32_t *sb = buf[warp];
    for (unsigned h = blockIdx.x * 4u + (unsigned)warp; h < nh; h += gridDim.x * 4u) {
        const int64_t a = heavy[h];
        const unsigned b = off[a], e = off[a + 1], deg = e - b, nc = 2 * deg;
        int32_t *seg = nbr + 2 * (size_t)b;
        uint8_t *segm = nbr_m + 2 * (size_t)b;
        if (nc > (unsigned)NB_WARP) {
            if (lane == 0) {
                const int n = insert_nbrs(F, list, b, e, a, seg, segm);
                unsigned above = 0;
                bool border = false;
                for (int m = 0; m < n; ++m) {
                    above += seg[m] > a;
                    border |= segm[m] == 1;
                }
                nbr_n[a] = (unsigned)n;
                up[a] = above;
                bnd[a] = border;
            }
            __syncwarp();
            continue;
        }
        for (unsigned i = lane; i < deg; i += 32) {
            const int64_t f = list[b + i];
            const int32_t x = F[3 * f], y = F[3 * f + 1], z = F[3 * f + 2];
            sb[2 * i] = x == a ? y : x;
            sb[2 * i + 1] = z == a ? y : z;
        }
        unsigned P = 32;
        while (P < nc) P <<= 1;
        for (unsigned i = nc + lane; i < P; i += 32) sb[i] = 0x7fffffff;
        __syncwarp();
        for (unsigned k = 2; k <= P; k <<= 1)
            for (unsigned j = k >> 1; j > 0; j >>= 1) {
                for (unsigned i = lane; i < P; i += 32) {
                    const unsigned ixj = i ^ j;
                    if (ixj > i) {
                        const int32_t x = sb[i], y = sb[ixj];
                        if ((x > y) == ((i & k) == 0)) { sb[i] = y; sb[ixj] = x; }
                    }
                }
                __syncwarp();
            }
        unsigned n = 0, above = 0;
        bool border = false;
        for (unsigned base = 0; base < nc; base += 32) {
            const unsigned i = base + lane;
            const bool keep = i < nc && (i == 0 || sb[i] != sb[i - 1]);
            unsigned run = 0;   // the length of the run of equal ids that starts at i
            if (keep)
                while (i + run < nc && sb[i + run] == sb[i]) ++run;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                seg[n + __popc(bal & lt)] = sb[i];
                segm[n + __popc(bal & lt)] = (uint8_t)(run > 255 ? 255 : run);
            }
            above += __popc(__ballot_sync(0xffffffffu, keep && sb[i] > a));
            border |= __any_sync(0xffffffffu, keep && run == 1);
            n += __popc(bal);
        }
        if (lane == 0) {
            nbr_n[a] = n;
            up[a] = above;
            bnd[a] = border;
        }
        __syncwarp();
    }
}

// The ranked edge list: the edges (a, u > a) of vertex a at eoff[a], u
// ascending (the upper part of its sorted neighbour list), with the faces of
// each edge. The same pass clears the per-vertex state this round builds:
// the two-ring minima, the marks for the next round, and the next
// adjacency's degree and fill counters.
__global__ void k_edges(const Control *__restrict__ ctl, int64_t nv, const unsigned *__restrict__ off,
                        const int32_t *__restrict__ nbr, const uint8_t *__restrict__ nbr_m,
                        const unsigned *__restrict__ nbr_n, const unsigned *__restrict__ eoff,
                        int32_t *__restrict__ ea, int32_t *__restrict__ eb, uint8_t *__restrict__ nfaces,
                        unsigned long long *__restrict__ m1, unsigned long long *__restrict__ m2,
                        uint8_t *__restrict__ dirty_next, unsigned *__restrict__ deg_next,
                        unsigned *__restrict__ fill, unsigned *__restrict__ n_heavy) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nv || ctl->done) return;
    m1[a] = KEY_NONE;
    m2[a] = KEY_NONE;
    dirty_next[a] = 0;
    deg_next[a] = 0;
    fill[a] = 0;
    if (a == 0) *n_heavy = 0;
    const int32_t *seg = nbr + 2 * (size_t)off[a];
    const uint8_t *segm = nbr_m + 2 * (size_t)off[a];
    const unsigned n = nbr_n[a], o = eoff[a], n_up = eoff[a + 1] - o;
    for (unsigned m = 0; m < n_up; ++m) {
        ea[o + m] = (int32_t)a;
        eb[o + m] = seg[n - n_up + m];
        nfaces[o + m] = segm[n - n_up + m];
    }
}

// Sign of the turn-over product n_old . n_new of one face, decided in FP32
// when that is certain: +1 (> 0), -1 (< 0), 0 (undecided: the caller takes the
// FP64 test). The FP32 inputs are the FP64 positions rounded to FP32 (V32);
// the bound B covers, with a factor of two to spare, the rounding of the
// inputs (u |coordinate|), of the edge differences, the cross products and the
// dot product against exact arithmetic on the FP64 positions, which is also
// where the FP64 test lands to within far less than B/2. So whenever
// |s| > B the FP64 test takes the same decision, and the collapses stay
// identical. Near the bottom of the FP32 range the FP64 test decides.
// (P: the face's corners from V32, id: their vertex ids)
__device__ __forceinline__ int turn_sign32(const float3 *P, const int32_t *id, int32_t w, float3 v) {
    float3 R[3];
    float m = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fabsf(v.z));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R[k] = id[k] == w ? v : P[k];
        m = fmaxf(m, fmaxf(fmaxf(fabsf(P[k].x), fabsf(P[k].y)), fabsf(P[k].z)));
    }
    const float3 e1 = P[1] - P[0], e2 = P[2] - P[0], f1 = R[1] - R[0], f2 = R[2] - R[0];
    const float3 c0 = cross3(e1, e2), c1 = cross3(f1, f2);
    const float sgn = dot3(c0, c1);
    auto amax = [](float3 a, float3 b) {
        return fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(b.x))),
                     fmaxf(fabsf(b.y), fabsf(b.z)));
    };
    const float E0 = amax(e1, e2), E1 = amax(f1, f2);
    const float u = 5.9604645e-8f;   // 2^-24
    const float d = 4.f * u * (m + fmaxf(E0, E1));
    const float dc0 = 4.f * E0 * d + 2.f * d * d + 6.f * u * E0 * E0;
    const float dc1 = 4.f * E1 * d + 2.f * d * d + 6.f * u * E1 * E1;
    const float C0 = 2.f * E0 * E0 + dc0, C1 = 2.f * E1 * E1 + dc1;
    const float B = 2.f * (3.f * (C0 * dc1 + C1 * dc0 + dc0 * dc1) + 15.f * u * C0 * C1);
    if (!(B >= 1e-30f) || !(B < 1e30f)) return 0;
    if (sgn > B) return 1;
    if (sgn < -B) return -1;
    return 0;
}

struct EdgeCostArgs {
    const double *V;
    const float *V32;
    const int32_t *F;
    const double *Q;
    const unsigned *off;
    const int32_t *list;
    const int32_t *nbr;
    const unsigned *nbr_n;
    const int32_t *ea, *eb;
    const uint8_t *nfaces, *bnd;
    int placement;
    unsigned long long *key;
    double *tpos;
    const uint8_t *dirty;
    const unsigned *eoff_prev;
    const int32_t *eb_prev;
    const unsigned long long *key_prev;
    const double *tpos_prev;
};

// placement, cost and validity of edge i: its key (KEY_NONE when the
// collapse is not allowed) and its placement in tpos
__device__ unsigned long long edge_key(const EdgeCostArgs &A, int64_t i) {
    const double *__restrict__ V = A.V;
    const float *__restrict__ V32 = A.V32;
    const int32_t *__restrict__ F = A.F;
    const double *__restrict__ Q = A.Q;
    const unsigned *__restrict__ off = A.off;
    const int32_t *__restrict__ list = A.list;
    double *__restrict__ tpos = A.tpos;
    const int32_t a = A.ea[i], b = A.eb[i];
    if (A.key_prev && !A.dirty[a] && !A.dirty[b]) {
        // neither end nor any vertex of their faces changed in the last
        // round: the edge's cost, validity and placement are as they were
        unsigned lo = A.eoff_prev[a], hi = A.eoff_prev[a + 1];
        while (lo < hi) {
            const unsigned mid = (lo + hi) >> 1;
            if (A.eb_prev[mid] < b) lo = mid + 1; else hi = mid;
        }
        if (lo < A.eoff_prev[a + 1] && A.eb_prev[lo] == b) {
            const unsigned long long k = A.key_prev[lo];
            if (k == KEY_NONE) return KEY_NONE;
#pragma unroll
            for (int c = 0; c < 3; ++c) tpos[3 * i + c] = A.tpos_prev[3 * (int64_t)lo + c];
            return (k & 0xffffffff00000000ull) | (uint32_t)i;
        }
    }
    const int nfc = A.nfaces[i];
    if (nfc > 2) return KEY_NONE;
    double q[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) q[k] = __dadd_rn(Q[10 * (int64_t)a + k], Q[10 * (int64_t)b + k]);
    const D3 va = ldv(V, a), vb = ldv(V, b);
    D3 v;
    if (nfc == 1) {
        v = quad_eval(q, vb) < quad_eval(q, va) ? vb : va;
    } else if (A.bnd[a] && A.bnd[b]) {
        return KEY_NONE;
    } else if (A.bnd[a]) {
        v = va;
    } else if (A.bnd[b]) {
        v = vb;
    } else {
        const double t = A.placement == AG_QEM_MIDPOINT ? 0.5 : qem_place(q, va, vb);
        v = dadd(va, dscl(dsub(vb, va), t));
    }
    // at most QEM_MAX_NBR distinct neighbours per end; the link condition
    // counts the common ones by merging the two sorted lists
    const int na = (int)A.nbr_n[a], nb = (int)A.nbr_n[b];
    if (na > QEM_MAX_NBR || nb > QEM_MAX_NBR) return KEY_NONE;
    const int32_t *la = A.nbr + 2 * (size_t)off[a], *lb = A.nbr + 2 * (size_t)off[b];
    int common = 0;
    for (int m = 0, n = 0; m < na && n < nb;) {
        const int32_t x = la[m], y = lb[n];
        common += x == y;
        m += x <= y;
        n += y <= x;
    }
    if (common != nfc) return KEY_NONE;
    if (na + nb - common <= 4) return KEY_NONE;
    const float3 v32 = make_float3(__double2float_rn(v.x), __double2float_rn(v.y), __double2float_rn(v.z));
    // the faces around each end in chunks of TURN_CHUNK: the loads of a
    // chunk (face ids, corner ids, corners) are issued together, so a chunk
    // costs three dependent memory latencies rather than three per face
    for (int side = 0; side < 2; ++side) {
        const int32_t w = side ? b : a, o = side ? a : b;
        const unsigned je = off[w + 1];
        for (unsigned j0 = off[w]; j0 < je; j0 += TURN_CHUNK) {
            int32_t id[TURN_CHUNK][3];
            float3 P[TURN_CHUNK][3];
#pragma unroll
            for (int c = 0; c < TURN_CHUNK; ++c) {
                const int64_t g = j0 + c < je ? list[j0 + c] : 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) id[c][k] = j0 + c < je ? F[3 * g + k] : -1;
            }
#pragma unroll
            for (int c = 0; c < TURN_CHUNK; ++c)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int64_t x = id[c][k] < 0 ? 0 : id[c][k];
                    P[c][k] = make_float3(V32[3 * x], V32[3 * x + 1], V32[3 * x + 2]);
                }
#pragma unroll
            for (int c = 0; c < TURN_CHUNK; ++c) {
                if (id[c][0] < 0) continue;                                   // past the end
                if (id[c][0] == o || id[c][1] == o || id[c][2] == o) continue; // a face of the edge
                const int sg = turn_sign32(P[c], id[c], w, v32);
                if (sg > 0) continue;
                if (sg < 0) return KEY_NONE;
                D3 Pd[3], R[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Pd[k] = ldv(V, id[c][k]);
                    R[k] = id[c][k] == w ? v : Pd[k];
                }
                const D3 n0 = dcross(dsub(Pd[1], Pd[0]), dsub(Pd[2], Pd[0]));
                const D3 n1 = dcross(dsub(R[1], R[0]), dsub(R[2], R[0]));
                if (!(ddot(n0, n1) > 0.0)) return KEY_NONE;
            }
        }
    }
    tpos[3 * i] = v.x; tpos[3 * i + 1] = v.y; tpos[3 * i + 2] = v.z;
    return qem_key(quad_eval(q, v), (uint32_t)i);
}

// every edge of the round (grid-stride over the device-side count): its key,
// and m1(v) = the least key at each end
#ifndef AG_QEM_COST_MIN_BLOCKS
#define AG_QEM_COST_MIN_BLOCKS 1
#endif
__global__ void __launch_bounds__(128, AG_QEM_COST_MIN_BLOCKS) k_edge_cost(const Control *__restrict__ ctl, EdgeCostArgs A,
                                                    unsigned long long *__restrict__ m1) {
    if (ctl->done) return;
    const int64_t ne = ctl->ne;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = edge_key(A, i);
        A.key[i] = k;
        if (k != KEY_NONE) {
            atomicMin(&m1[A.ea[i]], k);
            atomicMin(&m1[A.eb[i]], k);
        }
    }
}

// m2(v) = the least m1 over v and its neighbours (every vertex with an edge
// meets its own m1 through that edge)
__global__ void k_m2(const Control *__restrict__ ctl, const int32_t *__restrict__ ea, const int32_t *__restrict__ eb,
                     const unsigned long long *__restrict__ m1, unsigned long long *__restrict__ m2) {
    if (ctl->done) return;
    const int64_t ne = ctl->ne;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = ea[i], b = eb[i];
        const unsigned long long x = m1[a], y = m1[b], m = x < y ? x : y;
        if (m == KEY_NONE) continue;
        atomicMin(&m2[a], m);
        atomicMin(&m2[b], m);
    }
}

__global__ void k_select(const Control *__restrict__ ctl, const int32_t *__restrict__ ea,
                         const int32_t *__restrict__ eb, const unsigned long long *__restrict__ key,
                         const uint8_t *__restrict__ nfaces, const unsigned long long *__restrict__ m2,
                         uint8_t *__restrict__ sel, unsigned long long *__restrict__ selk, uint8_t *__restrict__ selnf,
                         Counters *cnt) {
    if (ctl->done) return;
    const int64_t ne = ctl->ne;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = key[i];
        const bool s = k != KEY_NONE && k == m2[ea[i]] && k == m2[eb[i]];
        sel[i] = s;
        if (!s) continue;
        const int slot = atomicAdd(&cnt->nsel, 1);
        selk[slot] = k;
        selnf[slot] = nfaces[i];
        atomicAdd(&cnt->removable, (unsigned long long)nfaces[i]);
    }
}

// smallest selected key L with sum(nfaces of selected keys <= L) >= need
__global__ void __launch_bounds__(1024) k_limit(const Control *__restrict__ ctl,
                                                 const unsigned long long *__restrict__ selk,
                                                 const uint8_t *__restrict__ selnf, const Counters *cnt,
                                                 long long target, unsigned long long *limit) {
    __shared__ long long part[32];
    __shared__ unsigned long long s_lo, s_hi;
    if (ctl->done) return;
    if ((long long)cnt->alive - (long long)cnt->removable >= target) {   // no cut needed this round
        if (threadIdx.x == 0) *limit = ~0ull;
        return;
    }
    const int n = cnt->nsel;
    const long long need = (long long)cnt->alive - target;
    if (threadIdx.x == 0) { s_lo = 0ull; s_hi = KEY_NONE; }
    __syncthreads();
    for (int it = 0; it < 70; ++it) {
        const unsigned long long lo = s_lo, hi = s_hi;
        if (lo >= hi) break;
        const unsigned long long mid = lo + (hi - lo) / 2;
        long long sum = 0;
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            if (selk[j] <= mid) sum += selnf[j];
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
            if (t >= need) s_hi = mid; else s_lo = mid + 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *limit = s_lo;
}

// The collapses that pass the cut: keep a at the placement with Q_a + Q_b,
// rename b to a; and mark the vertices whose edges must be re-evaluated next
// round: both ends of every collapse and every vertex of their faces (read
// here, before k_faces rewrites the faces). Selected collapses share no
// vertex, so their writes do not meet.
__global__ void k_apply_mark(const Control *__restrict__ ctl, const int32_t *__restrict__ ea,
                             const int32_t *__restrict__ eb, const unsigned long long *__restrict__ key,
                             const uint8_t *__restrict__ sel, const double *__restrict__ tpos,
                             const unsigned long long *__restrict__ limit, double *__restrict__ V,
                             float *__restrict__ V32, double *__restrict__ Q, uint8_t *__restrict__ valive,
                             int32_t *__restrict__ remap, const int32_t *__restrict__ F,
                             const unsigned *__restrict__ off, const int32_t *__restrict__ list,
                             uint8_t *__restrict__ dirty) {
    if (ctl->done) return;
    const int64_t ne = ctl->ne;
    const unsigned long long L = *limit;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
        if (!sel[i] || key[i] > L) continue;
        const int64_t a = ea[i], b = eb[i];
        for (int side = 0; side < 2; ++side) {
            const int64_t w = side ? b : a;
            dirty[w] = 1;
            const unsigned je = off[w + 1];
            for (unsigned j0 = off[w]; j0 < je; j0 += TURN_CHUNK) {   // loads of a chunk issued together
                int32_t id[TURN_CHUNK][3];
#pragma unroll
                for (int c = 0; c < TURN_CHUNK; ++c) {
                    const int64_t f = j0 + c < je ? list[j0 + c] : -1;
#pragma unroll
                    for (int k = 0; k < 3; ++k) id[c][k] = f >= 0 ? F[3 * f + k] : -1;
                }
#pragma unroll
                for (int c = 0; c < TURN_CHUNK; ++c)
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (id[c][k] >= 0) dirty[id[c][k]] = 1;
            }
        }
        V[3 * a] = tpos[3 * i]; V[3 * a + 1] = tpos[3 * i + 1]; V[3 * a + 2] = tpos[3 * i + 2];
#pragma unroll
        for (int k = 0; k < 3; ++k) V32[3 * a + k] = __double2float_rn(tpos[3 * i + k]);
#pragma unroll
        for (int k = 0; k < 10; ++k) Q[10 * a + k] = __dadd_rn(Q[10 * a + k], Q[10 * b + k]);
        valive[b] = 0;
        remap[b] = (int32_t)a;
    }
}

// faces through the renaming: a face holding both ends of a collapse is
// dropped; the others count towards their vertices' degrees in the next
// adjacency
__global__ void k_faces(const Control *__restrict__ ctl, int32_t *__restrict__ F, uint8_t *__restrict__ falive,
                        int64_t nf, const int32_t *__restrict__ remap, Counters *cnt,
                        unsigned *__restrict__ deg_next) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || ctl->done || !falive[f]) return;
    const int32_t r0 = remap[F[3 * f]], r1 = remap[F[3 * f + 1]], r2 = remap[F[3 * f + 2]];
    if (r0 == r1 || r1 == r2 || r0 == r2) {
        falive[f] = 0;
        atomicAdd(&cnt->alive, ~0ull);   // -1
        return;
    }
    F[3 * f] = r0; F[3 * f + 1] = r1; F[3 * f + 2] = r2;
    atomicAdd(&deg_next[r0], 1u);
    atomicAdd(&deg_next[r1], 1u);
    atomicAdd(&deg_next[r2], 1u);
}

__global__ void k_flag_u32(const uint8_t *__restrict__ flag, int64_t n, unsigned *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = flag[i] ? 1u : 0u;
}

__global__ void k_compact_v(const double *__restrict__ V, const uint8_t *__restrict__ valive,
                            const unsigned *__restrict__ vid, const int32_t *__restrict__ vorig, int64_t nv,
                            double *__restrict__ Vout, int32_t *__restrict__ keep_v) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv || !valive[v]) return;
    const unsigned o = vid[v];
    Vout[3 * (int64_t)o] = V[3 * v]; Vout[3 * (int64_t)o + 1] = V[3 * v + 1]; Vout[3 * (int64_t)o + 2] = V[3 * v + 2];
    if (keep_v) keep_v[o] = vorig[v];
}

// Renumbering of the working mesh to its alive vertices and faces, both in
// increasing id (so every order the rounds depend on, the ranked edge list
// above all, is unchanged): the per-vertex state moves to the new ids, the
// faces are rewritten through them.
__global__ void k_gather_v(const uint8_t *__restrict__ valive, const unsigned *__restrict__ vid, int64_t nv,
                           const double *__restrict__ V, const float *__restrict__ V32, const double *__restrict__ Q,
                           const int32_t *__restrict__ vorig, double *__restrict__ V2, float *__restrict__ V32b,
                           double *__restrict__ Q2, int32_t *__restrict__ vorig2) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv || !valive[v]) return;
    const int64_t o = vid[v];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        V2[3 * o + k] = V[3 * v + k];
        V32b[3 * o + k] = V32[3 * v + k];
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) Q2[10 * o + k] = Q[10 * v + k];
    vorig2[o] = vorig[v];
}

__global__ void k_gather_f(const int32_t *__restrict__ F, const uint8_t *__restrict__ falive,
                           const unsigned *__restrict__ fid, const unsigned *__restrict__ vid, int64_t nf,
                           int32_t *__restrict__ F2) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || !falive[f]) return;
    const int64_t o = fid[f];
#pragma unroll
    for (int k = 0; k < 3; ++k) F2[3 * o + k] = (int32_t)vid[F[3 * f + k]];
}

__global__ void k_iota(int32_t *__restrict__ a, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}

__global__ void k_compact_f(const int32_t *__restrict__ F, const uint8_t *__restrict__ falive,
                            const unsigned *__restrict__ fid, const unsigned *__restrict__ vid, int64_t nf,
                            int32_t *__restrict__ Fout) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf || !falive[f]) return;
    const int64_t o = fid[f];
#pragma unroll
    for (int k = 0; k < 3; ++k) Fout[3 * o + k] = (int32_t)vid[F[3 * f + k]];
}

}  // namespace
}  // namespace ag

using namespace ag;

extern "C" AG_API ag_status ag_qem_simplify(const float *d_verts, int64_t n_verts, const int32_t *d_faces,
                                            int64_t n_faces, int64_t target, int32_t max_rounds, int32_t placement,
                                            ag_stream_t stream,
                                            double *d_verts_out, int32_t *d_faces_out, int32_t *d_keep_verts,
                                            int64_t *h_result) {
    if (!d_verts || !d_faces || !d_verts_out || !d_faces_out || !h_result)
        return set_error(AG_ERR_INVALID_ARG, "pointers must be non-NULL (d_keep_verts may be NULL)");
    if (n_verts < 3 || n_verts >= (1ll << 31)) return set_error(AG_ERR_INVALID_ARG, "n_verts out of range");
    if (n_faces < 1 || n_faces >= (1ll << 29)) return set_error(AG_ERR_INVALID_ARG, "n_faces out of range");
    if (target < 0) return set_error(AG_ERR_INVALID_ARG, "target must be >= 0");
    if (max_rounds < 0) return set_error(AG_ERR_INVALID_ARG, "max_rounds must be >= 0");
    if (placement != AG_QEM_OPTIMAL && placement != AG_QEM_MIDPOINT)
        return set_error(AG_ERR_INVALID_ARG, "placement must be AG_QEM_OPTIMAL or AG_QEM_MIDPOINT");
    const int rounds_cap = max_rounds > 0 ? max_rounds : 100000;
    int dev = 0;
    AG_CUDA(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(dev);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    const int64_t nv = n_verts, nf = n_faces, emax = 3 * nf;
    Scratch sc(s, dev);
    double *V, *Q, *tpos;
    int32_t *F, *remap, *list, *ea, *eb;
    uint8_t *falive, *valive, *bnd, *nfaces, *sel, *selnf;
    unsigned *off, *fill, *eoff, *scan_tmp, *vid, *fid;
    unsigned long long *key, *m1, *m2, *selk, *limit;
    Counters *cnt;
    AG_CUDA(sc.alloc((void **)&V, sizeof(double) * 3 * nv));
    float *V32;   // V rounded to FP32 (the turn-over filter's input)
    AG_CUDA(sc.alloc((void **)&V32, sizeof(float) * 3 * nv));
    AG_CUDA(sc.alloc((void **)&Q, sizeof(double) * 10 * nv));
    AG_CUDA(sc.alloc((void **)&tpos, sizeof(double) * 3 * emax));
    AG_CUDA(sc.alloc((void **)&F, sizeof(int32_t) * 3 * nf));
    AG_CUDA(sc.alloc((void **)&remap, sizeof(int32_t) * nv));
    AG_CUDA(sc.alloc((void **)&list, sizeof(int32_t) * 3 * nf));
    int32_t *nbr;        // per vertex: sorted distinct neighbours (2 deg entries of room)
    uint8_t *nbr_m;      // the faces of each of those edges
    unsigned *nbr_n;     // their count
    int32_t *heavy;      // vertices whose lists a whole warp sorts
    unsigned *n_heavy;
    AG_CUDA(sc.alloc((void **)&nbr, sizeof(int32_t) * 6 * nf));
    AG_CUDA(sc.alloc((void **)&nbr_m, 6 * nf));
    AG_CUDA(sc.alloc((void **)&nbr_n, sizeof(unsigned) * nv));
    AG_CUDA(sc.alloc((void **)&heavy, sizeof(int32_t) * nv));
    AG_CUDA(sc.alloc((void **)&n_heavy, sizeof(unsigned)));
    AG_CUDA(sc.alloc((void **)&ea, sizeof(int32_t) * emax));
    AG_CUDA(sc.alloc((void **)&eb, sizeof(int32_t) * emax));
    AG_CUDA(sc.alloc((void **)&falive, nf));
    AG_CUDA(sc.alloc((void **)&valive, nv));
    AG_CUDA(sc.alloc((void **)&bnd, nv));
    AG_CUDA(sc.alloc((void **)&nfaces, emax));
    AG_CUDA(sc.alloc((void **)&sel, emax));
    AG_CUDA(sc.alloc((void **)&selnf, emax));
    AG_CUDA(sc.alloc((void **)&off, sizeof(unsigned) * (nv + 1)));
    unsigned *off_next;   // the next round's adjacency offsets (degrees first)
    AG_CUDA(sc.alloc((void **)&off_next, sizeof(unsigned) * (nv + 1)));
    AG_CUDA(sc.alloc((void **)&fill, sizeof(unsigned) * nv));
    AG_CUDA(sc.alloc((void **)&eoff, sizeof(unsigned) * (nv + 1)));
    AG_CUDA(sc.alloc((void **)&scan_tmp, scan_scratch_bytes(nv > nf ? nv : nf)));
    AG_CUDA(sc.alloc((void **)&vid, sizeof(unsigned) * (nv + 1)));
    AG_CUDA(sc.alloc((void **)&fid, sizeof(unsigned) * (nf + 1)));
    AG_CUDA(sc.alloc((void **)&key, sizeof(unsigned long long) * emax));
    AG_CUDA(sc.alloc((void **)&m1, sizeof(unsigned long long) * nv));
    AG_CUDA(sc.alloc((void **)&m2, sizeof(unsigned long long) * nv));
    AG_CUDA(sc.alloc((void **)&selk, sizeof(unsigned long long) * emax));
    AG_CUDA(sc.alloc((void **)&limit, sizeof(unsigned long long)));
    AG_CUDA(sc.alloc((void **)&cnt, sizeof(Counters)));
    Control *ctl;
    AG_CUDA(sc.alloc((void **)&ctl, sizeof(Control)));
    // the previous round's edge list (ends b by segment of a), keys and
    // placements, reused for edges whose neighbourhood did not change
    int32_t *eb_prev;
    unsigned *eoff_prev;
    unsigned long long *key_prev;
    double *tpos_prev;
    uint8_t *dirty, *dirty_next;
    AG_CUDA(sc.alloc((void **)&eb_prev, sizeof(int32_t) * emax));
    AG_CUDA(sc.alloc((void **)&eoff_prev, sizeof(unsigned) * (nv + 1)));
    AG_CUDA(sc.alloc((void **)&key_prev, sizeof(unsigned long long) * emax));
    AG_CUDA(sc.alloc((void **)&tpos_prev, sizeof(double) * 3 * emax));
    AG_CUDA(sc.alloc((void **)&dirty, nv));
    AG_CUDA(sc.alloc((void **)&dirty_next, nv));
    struct HostRead {   // pinned: the round control and the alive-face count
        Control ctl;
        unsigned long long alive;
    } *h_read = nullptr;
    AG_CUDA(cudaMallocHost((void **)&h_read, sizeof(HostRead)));
    struct HostFree {
        HostRead *p;
        ~HostFree() { if (p) cudaFreeHost(p); }
    } hf{h_read};
    Control *h_ctl = &h_read->ctl;
    unsigned long long *h_alive = &h_read->alive;

    const int B = 256;
    AG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(Counters), s));
    AG_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Control), s));
    AG_CUDA(cudaMemsetAsync(dirty, 0, nv, s));
    AG_CUDA(cudaMemsetAsync(valive, 0, nv, s));
    k_init_faces<<<blocks(nf, B), B, 0, s>>>(d_faces, nf, nv, F, falive, valive, cnt, status);
    k_init_verts<<<blocks(nv, B), B, 0, s>>>(d_verts, nv, V, V32, remap);
    AG_CUDA_LAUNCH("qem init");

    // the working mesh: nvc vertices and nfc faces (every alive one among
    // them), renumbered to the alive ones when the alive faces fall to a
    // quarter of nfc; vorig holds each working vertex's original id
    int64_t nvc = nv, nfc = nf;
    double *V2, *Q2;
    float *V32b;
    int32_t *F2, *vorig, *vorig2;
    AG_CUDA(sc.alloc((void **)&V2, sizeof(double) * 3 * nv));
    AG_CUDA(sc.alloc((void **)&V32b, sizeof(float) * 3 * nv));
    AG_CUDA(sc.alloc((void **)&Q2, sizeof(double) * 10 * nv));
    AG_CUDA(sc.alloc((void **)&F2, sizeof(int32_t) * 3 * nf));
    AG_CUDA(sc.alloc((void **)&vorig, sizeof(int32_t) * nv));
    AG_CUDA(sc.alloc((void **)&vorig2, sizeof(int32_t) * nv));
    k_iota<<<blocks(nv, B), B, 0, s>>>(vorig, nv);

    // adjacency (vertex -> alive faces), neighbour lists and the ranked edge
    // offsets of the working mesh from scratch (at the start and after a
    // renumbering; between, each round builds the next one)
    const unsigned heavy_grid = (unsigned)device_sm_count(dev) * 4;
    auto build_adjacency = [&](bool quadrics) -> cudaError_t {
        cudaError_t e;
        if ((e = cudaMemsetAsync(off, 0, sizeof(unsigned) * (nvc + 1), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(fill, 0, sizeof(unsigned) * nvc, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(n_heavy, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
        k_deg<<<blocks(nfc, B), B, 0, s>>>(F, falive, nfc, off);
        if ((e = launch_scan_exclusive(off, nvc, off + nvc, scan_tmp, s)) != cudaSuccess) return e;
        k_fill<<<blocks(nfc, B), B, 0, s>>>(nullptr, F, falive, nfc, off, fill, list);
        if (quadrics) k_quadric_init<<<blocks(nvc, 128), 128, 0, s>>>(V, F, nvc, off, list, Q);
        k_nbrs<<<blocks(nvc, 128), 128, 0, s>>>(nullptr, F, nvc, off, list, nbr, nbr_m, nbr_n, eoff, bnd, heavy,
                                                 n_heavy);
        k_nbrs_heavy<<<heavy_grid, 128, 0, s>>>(nullptr, F, off, list, heavy, n_heavy, nbr, nbr_m, nbr_n, eoff, bnd);
        if ((e = launch_scan_exclusive(eoff, nvc, eoff + nvc, scan_tmp, s)) != cudaSuccess) return e;
        return cudaGetLastError();
    };
    AG_CUDA(build_adjacency(true));

    // Rounds are enqueued ROUNDS_AHEAD at a time with no host decision in
    // between: k_round_begin decides on the device whether each one runs,
    // and the kernels over edges take the edge count from the device.
    const unsigned sm = (unsigned)device_sm_count(dev);
    bool have_prev = false;   // the last round's edge list is there to reuse (same numbering)
    for (;;) {
        const unsigned eg128 = std::min(blocks(3 * nfc, 128), sm * 32);
        const unsigned eg256 = std::min(blocks(3 * nfc, B), sm * 16);
        for (int k = 0; k < ROUNDS_AHEAD; ++k) {
            k_round_begin<<<1, 32, 0, s>>>(ctl, cnt, eoff + nvc, (long long)target, (long long)rounds_cap);
            k_edges<<<blocks(nvc, 128), 128, 0, s>>>(ctl, nvc, off, nbr, nbr_m, nbr_n, eoff, ea, eb, nfaces, m1, m2,
                                                     dirty_next, off_next, fill, n_heavy);
            EdgeCostArgs A;
            A.V = V; A.V32 = V32; A.F = F; A.Q = Q; A.off = off; A.list = list; A.nbr = nbr; A.nbr_n = nbr_n;
            A.ea = ea; A.eb = eb; A.nfaces = nfaces; A.bnd = bnd; A.placement = placement; A.key = key;
            A.tpos = tpos; A.dirty = dirty; A.eoff_prev = eoff_prev; A.eb_prev = eb_prev;
            A.key_prev = have_prev ? key_prev : nullptr; A.tpos_prev = tpos_prev;
            k_edge_cost<<<eg128, 128, 0, s>>>(ctl, A, m1);
            k_m2<<<eg256, B, 0, s>>>(ctl, ea, eb, m1, m2);
            k_select<<<eg256, B, 0, s>>>(ctl, ea, eb, key, nfaces, m2, sel, selk, selnf, cnt);
            k_limit<<<1, 1024, 0, s>>>(ctl, selk, selnf, cnt, (long long)target, limit);
            k_apply_mark<<<eg256, B, 0, s>>>(ctl, ea, eb, key, sel, tpos, limit, V, V32, Q, valive, remap, F, off,
                                             list, dirty_next);
            k_faces<<<blocks(nfc, B), B, 0, s>>>(ctl, F, falive, nfc, remap, cnt, off_next);
            AG_CUDA_LAUNCH("qem round");
            // the next round's adjacency and ranked edge list
            std::swap(off, off_next);
            std::swap(eb, eb_prev);
            std::swap(eoff, eoff_prev);
            std::swap(key, key_prev);
            std::swap(tpos, tpos_prev);
            std::swap(dirty, dirty_next);
            have_prev = true;
            AG_CUDA(launch_scan_exclusive(off, nvc, off + nvc, scan_tmp, s));
            k_fill<<<blocks(nfc, B), B, 0, s>>>(ctl, F, falive, nfc, off, fill, list);
            k_nbrs<<<blocks(nvc, 128), 128, 0, s>>>(ctl, F, nvc, off, list, nbr, nbr_m, nbr_n, eoff, bnd, heavy,
                                                    n_heavy);
            k_nbrs_heavy<<<heavy_grid, 128, 0, s>>>(ctl, F, off, list, heavy, n_heavy, nbr, nbr_m, nbr_n, eoff, bnd);
            AG_CUDA(launch_scan_exclusive(eoff, nvc, eoff + nvc, scan_tmp, s));
            AG_CUDA_LAUNCH("qem adjacency");
        }
        AG_CUDA(cudaMemcpyAsync(h_ctl, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
        AG_CUDA(cudaMemcpyAsync(h_alive, &cnt->alive, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        AG_CUDA(cudaStreamSynchronize(s));
        if (h_ctl->done) break;
        if (nfc < COMPACT_MIN || (long long)*h_alive * 4 > nfc) continue;
        // renumber the working mesh to its alive vertices and faces
        k_flag_u32<<<blocks(nvc, B), B, 0, s>>>(valive, nvc, vid);
        AG_CUDA(launch_scan_exclusive(vid, nvc, vid + nvc, scan_tmp, s));
        k_flag_u32<<<blocks(nfc, B), B, 0, s>>>(falive, nfc, fid);
        AG_CUDA(launch_scan_exclusive(fid, nfc, fid + nfc, scan_tmp, s));
        k_gather_v<<<blocks(nvc, B), B, 0, s>>>(valive, vid, nvc, V, V32, Q, vorig, V2, V32b, Q2, vorig2);
        k_gather_f<<<blocks(nfc, B), B, 0, s>>>(F, falive, fid, vid, nfc, F2);
        AG_CUDA_LAUNCH("qem renumber");
        unsigned nv_new = 0, nf_new = 0;
        AG_CUDA(cudaMemcpyAsync(&nv_new, vid + nvc, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        AG_CUDA(cudaMemcpyAsync(&nf_new, fid + nfc, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        AG_CUDA(cudaStreamSynchronize(s));
        std::swap(V, V2);
        std::swap(V32, V32b);
        std::swap(Q, Q2);
        std::swap(vorig, vorig2);
        std::swap(F, F2);
        nvc = nv_new;
        nfc = nf_new;
        AG_CUDA(cudaMemsetAsync(valive, 1, nvc, s));
        AG_CUDA(cudaMemsetAsync(falive, 1, nfc, s));
        AG_CUDA(cudaMemsetAsync(dirty, 0, nvc, s));
        k_iota<<<blocks(nvc, B), B, 0, s>>>(remap, nvc);
        AG_CUDA(build_adjacency(false));
        have_prev = false;
    }
    const int64_t rounds = h_ctl->rounds;
    // compaction: surviving vertices and faces in increasing original id
    k_flag_u32<<<blocks(nvc, B), B, 0, s>>>(valive, nvc, vid);
    AG_CUDA(launch_scan_exclusive(vid, nvc, vid + nvc, scan_tmp, s));
    k_flag_u32<<<blocks(nfc, B), B, 0, s>>>(falive, nfc, fid);
    AG_CUDA(launch_scan_exclusive(fid, nfc, fid + nfc, scan_tmp, s));
    k_compact_v<<<blocks(nvc, B), B, 0, s>>>(V, valive, vid, vorig, nvc, d_verts_out, d_keep_verts);
    k_compact_f<<<blocks(nfc, B), B, 0, s>>>(F, falive, fid, vid, nfc, d_faces_out);
    AG_CUDA_LAUNCH("qem compact");
    unsigned nvo = 0, nfo = 0;
    AG_CUDA(cudaMemcpyAsync(&nvo, vid + nvc, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    AG_CUDA(cudaMemcpyAsync(&nfo, fid + nfc, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    AG_CUDA(cudaStreamSynchronize(s));
    h_result[0] = nvo;
    h_result[1] = nfo;
    h_result[2] = rounds;
    return AG_OK;
}
