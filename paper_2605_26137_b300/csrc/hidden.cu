// Hidden-face removal (Sec. 6.2): a visibility pass that casts orthographic
// rays from viewpoints spread over a sphere around the mesh through its BVH
// and marks every face that is some ray's first hit, then a flood fill that
// promotes faces linked to visible ones across edges whose two faces have
// normals pointing the same way.
//
// Visibility (k_visibility): one persistent launch over all views.  A warp
// takes 32 consecutive rays, an 8x4-pixel tile of one view, so its rays are
// neighbours and share their node fetches.  View k looks along -u_k, u_k on
// the Fibonacci (golden-angle) lattice; its res x res pixels tile the square
// [-R, R]^2 of the plane through the bounding-box centre c spanned by
// e1 = normalize(a x u) and e2 = u x e1 (a = +z, or +x when |u_z| >= 0.9);
// pixel (i, j) casts from c + 2R u + x e1 + y e2, x = (2 (i + 1/2) / res - 1) R,
// along -u.  The traversal and triangle test are those of the texel rays
// (rays.cuh); origins lie outside the bounding sphere, so the closest |t| is
// the first hit.  A hit stores 1 into the face's byte of the visibility mask.
//
// Exterior fill (k_flood): face normals n = (B - A) x (C - A) in FP64 with the
// operations in a fixed order, so the gate n_f . n_g > 0 is decided exactly as
// an FP64 evaluation of that expression; a vertex -> face adjacency gives each
// face's edge neighbours; a level-synchronous breadth-first search from all
// visible faces runs its first levels over the whole GPU, one launch per
// level, and one CTA finishes any deeper levels.  The exterior set
// (everything linked to a visible face) does not depend on the visiting order.
#include "rays.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace ag {
namespace {

struct __align__(16) ViewGeom {
    float4 base;   // c + 2R u
    float4 e1, e2;
    float4 dir;    // -u
};

struct VisArgs {
    const void *nodes;
    const float4 *tris;
    const int32_t *tri_ids;
    float scene_abs;
    float3 lo, hi;          // scene bounding box
    const ViewGeom *views;
    const Ray *templ;       // per view: the ray of make_ray for its direction, origin = view base
    int res, tiles_x, tiles_per_view, n_tiles;
    float R, scale, tmax;
    unsigned long long *counter;
    unsigned *status;
    int max_steps;
    uint8_t *visible;
    int32_t *hit_ids;
    unsigned long long *counters;
};

// a node visit whose hit leaf children are recorded in *ls (tested by the caller at the node)
template <int LAYOUT>
__device__ __forceinline__ void visit_node(const VisArgs &A, uint32_t idx, const Ray &r, float lim, Next &nx,
                                           uint2 *stack, int &sp, LeafSet *ls) {
    if (LAYOUT == AG_BVH_Q8)
        NodeOps<AG_BVH_Q8>::visit<true>(A.nodes, idx, r, lim, nx, stack, sp, A.status, STACK, ls);
    else
        NodeOps<AG_BVH_F32>::visit<true>(A.nodes, idx, r, lim, nx, stack, sp, A.status, A.scene_abs, STACK, ls);
}

// the direction-dependent part of every ray of a view, once per view
__global__ void k_view_rays(const ViewGeom *__restrict__ views, int n, Ray *__restrict__ templ) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const ViewGeom G = views[k];
    templ[k] = make_ray(f3(G.base), make_float3(0.f, 0.f, 0.f), f3(G.dir));
}

// false only when the ray misses the scene box even widened by the rounding
// slack of the node tests, so no node of the tree can accept it
__device__ __forceinline__ bool meets_scene(const VisArgs &A, const Ray &r) {
    const float ex = EPS_REL * (A.scene_abs + fabsf(r.px)) * fabsf(r.ix);
    const float ey = EPS_REL * (A.scene_abs + fabsf(r.py)) * fabsf(r.iy);
    const float ez = EPS_REL * (A.scene_abs + fabsf(r.pz)) * fabsf(r.iz);
    const float ax = (A.lo.x - r.px) * r.ix, bx = (A.hi.x - r.px) * r.ix;
    const float ay = (A.lo.y - r.py) * r.iy, by = (A.hi.y - r.py) * r.iy;
    const float az = (A.lo.z - r.pz) * r.iz, bz = (A.hi.z - r.pz) * r.iz;
    const float te = fmaxf(fmaxf(fminf(ax, bx) - ex, fminf(ay, by) - ey), fminf(az, bz) - ez);
    const float tx = fminf(fminf(fmaxf(ax, bx) + ex, fmaxf(ay, by) + ey), fmaxf(az, bz) + ez);
    return te <= tx && te <= A.tmax && tx >= -A.tmax;
}

// the ray of pixel (px, py) of a view: the view's template (direction part)
// with the pixel's offset in the view plane as origin offset
__device__ __forceinline__ Ray vis_ray(const VisArgs &A, int view, int px, int py) {
    const ViewGeom G = A.views[view];
    const float x = __fmaf_rn((float)px + 0.5f, A.scale, -A.R);
    const float y = __fmaf_rn((float)py + 0.5f, A.scale, -A.R);
    const float3 off = f3(G.e1) * x + f3(G.e2) * y;
    Ray ray = A.templ[view];
    ray.ox = pick(off, ray.kx()); ray.oy = pick(off, ray.ky()); ray.oz = pick(off, ray.kz());
    const float3 p = f3(G.base) + off;
    ray.px = p.x; ray.py = p.y; ray.pz = p.z;
    return ray;
}

// the closest hit of one visibility ray through the BVH (every step a node
// visit, its hit leaf children tested at the node; the root is always a node)
template <int LAYOUT, bool COUNT>
__device__ __forceinline__ Best trace_vis(const VisArgs &A, const Ray &ray, uint2 *stack, unsigned long long &c_nodes,
                                          unsigned long long &c_tris) {
    Best b;
    b.t = 0.f; b.babs = A.tmax; b.rec = 0; b.found = false;
    b.U = b.V = b.W = 0.f; b.det = 1.f;
    uint32_t cur = 0;
    int sp = 0, steps = 0;
    for (bool live = meets_scene(A, ray); live;) {
        Next nx;
        nx.has = false;
        nx.ref = 0;
        nx.dist = 0.f;
        LeafSet ls;
        visit_node<LAYOUT>(A, cur, ray, b.babs, nx, stack, sp, &ls);
        if (COUNT) ++c_nodes;
        while (ls.mask) {
            const int c = __ffs(ls.mask) - 1;
            ls.mask &= ls.mask - 1;
            uint32_t first;
            int cnt;
            leaf_range(ls, c, first, cnt);
            for (int k = 0; k < cnt; ++k) test_tri(ray, A.tris, A.tri_ids, first + k, b);
            if (COUNT) c_tris += cnt;
        }
        if (nx.has) {
            cur = nx.ref;
        } else {
            bool done = true;
            while (sp > 0) {
                uint2 e = stack[--sp];
                if (__uint_as_float(e.y) <= b.babs) { cur = e.x; done = false; break; }
            }
            if (done) break;
        }
        if (++steps > A.max_steps) {
            atomicOr(A.status, AGS_STEP_CAP);
            live = false;
        }
    }
    return b;
}

template <int LAYOUT, bool COUNT>
__global__ void __launch_bounds__(256) k_visibility(VisArgs A) {
    const int lane = threadIdx.x & 31;
    unsigned long long c_nodes = 0, c_tris = 0, c_rays = 0, c_hits = 0;
    uint2 stack[STACK];
    for (;;) {
        // a warp takes one 8x4 tile: view and tile position are warp-uniform
        int tile = 0;
        if (lane == 0) tile = (int)atomicAdd(A.counter, 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= A.n_tiles) break;
        const int view = tile / A.tiles_per_view;
        const int t = tile - view * A.tiles_per_view;
        const int ty = t / A.tiles_x;
        const int px = (t - ty * A.tiles_x) * 8 + (lane & 7);
        const int py = ty * 4 + (lane >> 3);
        if (px >= A.res || py >= A.res) continue;
        const Ray ray = vis_ray(A, view, px, py);
        if (COUNT) ++c_rays;
        const Best b = trace_vis<LAYOUT, COUNT>(A, ray, stack, c_nodes, c_tris);
        const int id = b.found ? A.tri_ids[b.rec] : -1;
        if (b.found) {
            A.visible[id] = 1;
            if (COUNT) ++c_hits;
        }
        if (A.hit_ids) A.hit_ids[(long long)view * A.res * A.res + (long long)py * A.res + px] = id;
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

// ---- z-buffer proposals for the orthographic views (AG_RENDER_RASTER).
// One lane per (view, triangle): the vertices in pixel units of the view
// plane, X = ((p - base) . e1 + R) / scale (pixel centre i + 1/2 <-> X = i + 1/2),
// ray parameter t = (p - base) . dir; edge functions from the lexicographically
// smaller endpoint (a shared edge gets exactly opposite values), t at a pixel
// centre from the barycentrics the edge values give; the warp walks its
// triangles' pixel boxes, a 64-bit atomicMin of (t bits, record) per covered
// centre.  Only a proposal the watertight test confirms is taken; the other
// pixels go to the traversal.  The first hits are the traversal's except
// where two triangles lie within rounding of each other along the ray (a
// shared edge, touching sheets).
constexpr unsigned long long VIS_NO_KEY = ~0ull;

struct VisRaster {
    const float4 *tris;
    int n_tris;
    const ViewGeom *views;
    int res, v0, nv;
    float R, scale;
    unsigned long long *keys;   // [nv * res * res]
    unsigned *next;             // work counter of this chunk (zero before the launch)
};

struct VisTri {
    float ax[3], ay[3], dx[3], dy[3];   // canonical edges, (dx, dy) negated where the inside is negative
    float t[3];                  // ray parameter of the vertex opposite each edge
    float inv_area;
    int x0, y0, bw;
    float rbw;
    unsigned rec, cnt;
};

__device__ __forceinline__ float vis_edge(float ax, float ay, float dx, float dy, float px, float py) {
    return __fsub_rn(__fmul_rn(dx, __fsub_rn(py, ay)), __fmul_rn(dy, __fsub_rn(px, ax)));
}

// persistent warps take (view, 32-triangle group) items from a counter, so
// the last wave is balanced at the grain of one group
__global__ void __launch_bounds__(256) k_vis_zbuffer(VisRaster A) {
    __shared__ VisTri ts[256];
    const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
    const int groups = (A.n_tris + 31) / 32;
    const unsigned total = (unsigned)A.nv * (unsigned)groups;
    const float rs = 1.0f / A.scale;
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(A.next, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        const int kv = (int)(item / (unsigned)groups);
        const int tri = (int)(item - (unsigned)kv * groups) * 32 + lane;
        const ViewGeom G = A.views[A.v0 + kv];
        VisTri T;
        T.cnt = 0;
        if (tri < A.n_tris) {
            float X[3], Y[3], Z[3];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const float4 p = __ldg(&A.tris[3 * (size_t)tri + m]);
                const float3 d = make_float3(p.x - G.base.x, p.y - G.base.y, p.z - G.base.z);
                X[m] = (d.x * G.e1.x + d.y * G.e1.y + d.z * G.e1.z + A.R) * rs;
                Y[m] = (d.x * G.e2.x + d.y * G.e2.y + d.z * G.e2.z + A.R) * rs;
                Z[m] = d.x * G.dir.x + d.y * G.dir.y + d.z * G.dir.z;
            }
            const float area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const int q = m == 2 ? 0 : m + 1;
                const bool sw = X[q] < X[m] || (X[q] == X[m] && Y[q] < Y[m]);
                const int a = sw ? q : m, b = sw ? m : q;
                // negating both factors' differences negates the rounded edge value exactly
                const float sg = (sw != (area < 0.f)) ? -1.f : 1.f;
                T.ax[m] = X[a];
                T.ay[m] = Y[a];
                T.dx[m] = sg * (X[b] - X[a]);
                T.dy[m] = sg * (Y[b] - Y[a]);
                T.t[m] = Z[m == 0 ? 2 : m - 1];     // edge m (vertex m -> m+1) weighs the vertex m+2
            }
            T.inv_area = 1.0f / fabsf(area);
            T.rec = (unsigned)tri;
            const float lo_x = fminf(X[0], fminf(X[1], X[2])), hi_x = fmaxf(X[0], fmaxf(X[1], X[2]));
            const float lo_y = fminf(Y[0], fminf(Y[1], Y[2])), hi_y = fmaxf(Y[0], fmaxf(Y[1], Y[2]));
            const int x0 = (int)fmaxf(ceilf(lo_x - 0.5f), 0.f), x1 = (int)fminf(floorf(hi_x - 0.5f), (float)(A.res - 1));
            const int y0 = (int)fmaxf(ceilf(lo_y - 0.5f), 0.f), y1 = (int)fminf(floorf(hi_y - 0.5f), (float)(A.res - 1));
            T.x0 = x0;
            T.y0 = y0;
            T.bw = x1 - x0 + 1;
            T.rbw = 1.0f / (float)T.bw;
            if (area != 0.f && x1 >= x0 && y1 >= y0) T.cnt = (unsigned)(x1 - x0 + 1) * (unsigned)(y1 - y0 + 1);
        }
        __syncwarp();
        ts[threadIdx.x] = T;
        __syncwarp();
        unsigned long long *keys = A.keys + (long long)kv * A.res * A.res;
        for (int q = 0; q < 32; ++q) {
            const VisTri &S = ts[wbase + q];
            const unsigned n = S.cnt;
            if (n == 0) continue;
            const int bw = S.bw;
            // the lane's pixels o = lane, lane + 32, ... of the box, o = y bw + x,
            // stepped by (32 mod bw, 32 div bw) with one wrap: exact integers
            // (and exact small floats for the centre coordinates)
            int yy = (int)((float)lane * S.rbw);
            int xx = lane - yy * bw;
            if (xx < 0) { --yy; xx += bw; } else if (xx >= bw) { ++yy; xx -= bw; }
            const int sx = bw > 32 ? 32 : 32 % bw, sy = bw > 32 ? 0 : 32 / bw;
            float px = (float)(S.x0 + xx) + 0.5f, py = (float)(S.y0 + yy) + 0.5f;
            int at = (S.y0 + yy) * A.res + S.x0 + xx;
            const int astep = sy * A.res + sx, awrap = A.res - bw;
            for (unsigned o = lane; o < n; o += 32) {
                float e[3];
                bool in = true;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    e[m] = vis_edge(S.ax[m], S.ay[m], S.dx[m], S.dy[m], px, py);
                    in = in && e[m] >= 0.f;
                }
                if (in) {
                    const float t = (e[0] * S.t[0] + e[1] * S.t[1] + e[2] * S.t[2]) * S.inv_area;
                    if (t > 0.f && t < 3.0e38f)
                        atomicMin(&keys[at], ((unsigned long long)__float_as_uint(t) << 32) | S.rec);
                }
                xx += sx;
                px += (float)sx;
                py += (float)sy;
                at += astep;
                if (xx >= bw) {
                    xx -= bw;
                    px -= (float)bw;
                    py += 1.f;
                    at += awrap;
                }
            }
        }
    }
}

// proposals confirmed by the watertight test mark their face; the others go
// to the deferred trace list (global pixel index, warp-aggregated append).
// The keys are reset behind the read for the next chunk.  A list that would
// overflow sets the chunk's flag instead, and the whole chunk is traced.
__global__ void __launch_bounds__(256) k_vis_resolve(VisArgs A, unsigned long long *__restrict__ keys, int v0,
                                                     unsigned long long *list, unsigned long long cap,
                                                     unsigned long long *count, int *overflow) {
    const unsigned npix = (unsigned)A.res * (unsigned)A.res;
    const int kv = blockIdx.y, view = v0 + kv;
    unsigned long long *vkeys = keys + (long long)kv * npix;
    const unsigned stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (unsigned pix = blockIdx.x * blockDim.x + threadIdx.x; pix < npix; pix += stride) {
        const unsigned long long key = vkeys[pix];
        bool queue = false;
        if (key == VIS_NO_KEY) {
            if (A.hit_ids) A.hit_ids[(long long)view * npix + pix] = -1;
        } else {
            vkeys[pix] = VIS_NO_KEY;
            const Ray ray = vis_ray(A, view, (int)(pix % (unsigned)A.res), (int)(pix / (unsigned)A.res));
            Best b;
            b.t = 0.f; b.babs = A.tmax; b.rec = 0; b.found = false;
            b.U = b.V = b.W = 0.f; b.det = 1.f;
            test_tri(ray, A.tris, A.tri_ids, (uint32_t)(key & 0xffffffffu), b);
            if (b.found) {
                const int id = A.tri_ids[b.rec];
                A.visible[id] = 1;
                if (A.hit_ids) A.hit_ids[(long long)view * npix + pix] = id;
            } else {
                queue = true;
            }
        }
        const unsigned act = __activemask();
        const unsigned want = __ballot_sync(act, queue);
        if (want) {
            const int leader = __ffs(want) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(want));
            base = __shfl_sync(act, base, leader);
            if (queue) {
                const unsigned long long at = base + __popc(want & ((1u << lane) - 1u));
                if (at < cap)
                    list[at] = (unsigned long long)view * npix + pix;
                else
                    *overflow = 1;
            }
        }
    }
}

// the full traversal for the deferred pixels (global pixel indices); with
// `overflow` set, every pixel of views [v0, v0 + nv) instead
template <int LAYOUT>
__global__ void __launch_bounds__(128) k_vis_trace(VisArgs A, const unsigned long long *__restrict__ list,
                                                   const unsigned long long *__restrict__ count,
                                                   unsigned long long cap, const int *overflow, int v0, int nv) {
    uint2 stack[STACK];
    unsigned long long cn = 0, ct = 0;
    const long long npix = (long long)A.res * A.res;
    long long n;
    if (overflow) {
        if (!*overflow) return;
        n = (long long)nv * npix;
    } else {
        n = (long long)min(*count, cap);
    }
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long g = overflow ? (long long)v0 * npix + e : (long long)list[e];
        const int view = (int)(g / npix);
        const int pix = (int)(g - (long long)view * npix);
        const Ray ray = vis_ray(A, view, pix % A.res, pix / A.res);
        const Best b = trace_vis<LAYOUT, false>(A, ray, stack, cn, ct);
        const int id = b.found ? A.tri_ids[b.rec] : -1;
        if (b.found) A.visible[id] = 1;
        if (A.hit_ids) A.hit_ids[(long long)view * npix + pix] = id;
    }
}

// FP64 face normals (fixed operation order) and the flood-fill state:
// -1 = face with an out-of-range index (never linked), 1 = visible, 0 = not yet
__global__ void k_face_normals64(const float *__restrict__ V, const int32_t *__restrict__ F, int64_t nf, int64_t nv,
                                 const uint8_t *__restrict__ vis, double *__restrict__ nrm, int32_t *__restrict__ state,
                                 unsigned *status) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int32_t i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
    if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) {
        state[f] = -1;
        nrm[3 * f] = nrm[3 * f + 1] = nrm[3 * f + 2] = 0.0;
        atomicOr(status, AGS_BAD_FACE);
        return;
    }
    const double ax = V[3 * i0], ay = V[3 * i0 + 1], az = V[3 * i0 + 2];
    const double e1x = __dsub_rn((double)V[3 * i1], ax), e1y = __dsub_rn((double)V[3 * i1 + 1], ay),
                 e1z = __dsub_rn((double)V[3 * i1 + 2], az);
    const double e2x = __dsub_rn((double)V[3 * i2], ax), e2y = __dsub_rn((double)V[3 * i2 + 1], ay),
                 e2z = __dsub_rn((double)V[3 * i2 + 2], az);
    nrm[3 * f] = __dsub_rn(__dmul_rn(e1y, e2z), __dmul_rn(e1z, e2y));
    nrm[3 * f + 1] = __dsub_rn(__dmul_rn(e1z, e2x), __dmul_rn(e1x, e2z));
    nrm[3 * f + 2] = __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x));
    state[f] = vis[f] ? 1 : 0;
}

__device__ __forceinline__ bool same_side(const double *__restrict__ nrm, int64_t f, int64_t g) {
    const double d = __dadd_rn(__dadd_rn(__dmul_rn(nrm[3 * f], nrm[3 * g]), __dmul_rn(nrm[3 * f + 1], nrm[3 * g + 1])),
                               __dmul_rn(nrm[3 * f + 2], nrm[3 * g + 2]));
    return d > 0.0;
}

constexpr int FLOOD_THREADS = 1024;
// breadth-first levels run over the whole GPU before one CTA finishes the
// (rare) deeper levels
constexpr int FLOOD_GRID_LEVELS = 16;

// claims every same-side edge neighbour of f that is not yet reached and
// appends it to q
__device__ __forceinline__ void flood_expand(const int32_t *__restrict__ F, const unsigned *__restrict__ off,
                                             const int32_t *__restrict__ list, const double *__restrict__ nrm,
                                             int32_t *state, int32_t f, int32_t *q, unsigned *cnt) {
    for (int m = 0; m < 3; ++m) {
        const int32_t a = F[3 * (int64_t)f + m], b = F[3 * (int64_t)f + (m == 2 ? 0 : m + 1)];
        if (a == b) continue;
        for (unsigned j = off[a]; j < off[a + 1]; ++j) {
            const int32_t g = list[j];
            if (g == f) continue;
            const int32_t *G = F + 3 * (int64_t)g;
            if (G[0] != b && G[1] != b && G[2] != b) continue;
            if (!same_side(nrm, f, g)) continue;
            if (atomicCAS(&state[g], 0, 1) == 0) q[atomicAdd(cnt, 1u)] = g;
        }
    }
}

// the first queue: every visible face
__global__ void k_flood_seed(const int32_t *__restrict__ state, int64_t nf, int32_t *q, unsigned *cnt) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < nf && state[f] == 1) q[atomicAdd(cnt, 1u)] = (int32_t)f;
}

// one breadth-first level over the whole GPU
__global__ void k_flood_level(const int32_t *__restrict__ F, const unsigned *__restrict__ off,
                              const int32_t *__restrict__ list, const double *__restrict__ nrm, int32_t *state,
                              const int32_t *__restrict__ qin, const unsigned *__restrict__ cin, int32_t *qout,
                              unsigned *cout) {
    const unsigned n = *cin;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flood_expand(F, off, list, nrm, state, qin[i], qout, cout);
}

// One CTA: the remaining levels from queue qa (count *cin), then the mask.
__global__ void __launch_bounds__(FLOOD_THREADS) k_flood(const int32_t *__restrict__ F, int64_t nf,
                                                          const unsigned *__restrict__ off,
                                                          const int32_t *__restrict__ list,
                                                          const double *__restrict__ nrm, int32_t *state, int32_t *qa,
                                                          const unsigned *__restrict__ cin, int32_t *qb,
                                                          uint8_t *__restrict__ ext) {
    __shared__ unsigned s_count;
    const int tid = threadIdx.x;
    unsigned cur = *cin;
    while (cur > 0) {
        if (tid == 0) s_count = 0;
        __syncthreads();
        for (unsigned i = tid; i < cur; i += FLOOD_THREADS) flood_expand(F, off, list, nrm, state, qa[i], qb, &s_count);
        __syncthreads();
        cur = s_count;
        int32_t *t = qa;
        qa = qb;
        qb = t;
        __syncthreads();
    }
    for (int64_t f = tid; f < nf; f += FLOOD_THREADS) ext[f] = state[f] == 1 ? 1 : 0;
}

ag_status check_bvh(ag_bvh_t h) {
    if (!h || h->magic != AG_BVH_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "invalid BVH handle");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->device) return set_error(AG_ERR_INVALID_ARG, "BVH handle belongs to device %d, current is %d",
                                           h->device, dev);
    return AG_OK;
}

// view k of n on the golden-angle lattice, in double precision, then FP32
ViewGeom view_geom(int k, int n, const double c[3], double R) {
    const double golden = 2.39996322972865332223;   // pi (3 - sqrt 5)
    const double z = 1.0 - (2.0 * k + 1.0) / n;
    const double rr = std::sqrt(std::fmax(0.0, 1.0 - z * z));
    const double phi = k * golden;
    const double u[3] = {rr * std::cos(phi), rr * std::sin(phi), z};
    const double a[3] = {std::fabs(u[2]) < 0.9 ? 0.0 : 1.0, 0.0, std::fabs(u[2]) < 0.9 ? 1.0 : 0.0};
    double e1[3] = {a[1] * u[2] - a[2] * u[1], a[2] * u[0] - a[0] * u[2], a[0] * u[1] - a[1] * u[0]};
    const double l = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (double &v : e1) v /= l;
    const double e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
    ViewGeom g;
    g.base = make_float4((float)(c[0] + 2.0 * R * u[0]), (float)(c[1] + 2.0 * R * u[1]), (float)(c[2] + 2.0 * R * u[2]), 0.f);
    g.e1 = make_float4((float)e1[0], (float)e1[1], (float)e1[2], 0.f);
    g.e2 = make_float4((float)e2[0], (float)e2[1], (float)e2[2], 0.f);
    g.dir = make_float4((float)-u[0], (float)-u[1], (float)-u[2], 0.f);
    return g;
}

// the keys of one chunk of views (8 bytes per pixel) stay within this
// budget, so that they live in L2 between the passes
constexpr long long VIS_CHUNK_BYTES = 96ll << 20;
// deferred trace list entries (8 bytes each)
constexpr long long VIS_LIST_CAP = 1ll << 22;

template <typename Kernel>
unsigned resident_blocks(Kernel kernel, int block, int dev) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (unsigned)(device_sm_count(dev) * per_sm);
}

template <int LAYOUT, bool COUNT>
cudaError_t launch_vis(const VisArgs &A, int block, int bps, cudaStream_t s) {
    int dev;
    cudaGetDevice(&dev);
    if (bps <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_visibility<LAYOUT, COUNT>, block, 0);
        bps = occ > 0 ? occ : 1;
    }
    k_visibility<LAYOUT, COUNT><<<(unsigned)(device_sm_count(dev) * bps), block, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace
}  // namespace ag

using namespace ag;

extern "C" {

AG_API ag_status ag_visibility(ag_bvh_t h, int32_t n_views, int32_t res, const ag_opts *opts, ag_stream_t stream,
                               uint8_t *d_visible, int32_t *d_hit_ids, uint64_t *d_counters) {
    ag_status st = check_bvh(h);
    if (st) return st;
    if (n_views < 1 || n_views > (1 << 20)) return set_error(AG_ERR_INVALID_ARG, "n_views must be in 1..2^20");
    if (res < 1 || res > 16384) return set_error(AG_ERR_INVALID_ARG, "res must be in 1..16384");
    if (!d_visible) return set_error(AG_ERR_INVALID_ARG, "d_visible must be non-NULL");
    ag_opts o;
    ag_opts_default(&o);
    if (opts) o = *opts;
    if (o.block_size != 0 && (o.block_size < 64 || o.block_size > 256 || o.block_size % 32))
        return set_error(AG_ERR_INVALID_ARG, "block_size must be 0 or a multiple of 32 in 64..256");
    if (o.blocks_per_sm < 0 || o.blocks_per_sm > 64) return set_error(AG_ERR_INVALID_ARG, "blocks_per_sm out of range");
    if (o.max_steps < 0) return set_error(AG_ERR_INVALID_ARG, "max_steps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(h->device);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    st = bvh_ready(h);   // the views are placed around the scene box
    if (st) return st;
    double c[3], R2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        c[k] = 0.5 * ((double)h->lo[k] + (double)h->hi[k]);
        const double e = (double)h->hi[k] - (double)h->lo[k];
        R2 += e * e;
    }
    const double R = 0.5 * std::sqrt(R2);
    std::vector<ViewGeom> views((size_t)n_views);
    for (int k = 0; k < n_views; ++k) views[(size_t)k] = view_geom(k, n_views, c, R);
    Scratch sc(s, h->device);
    ViewGeom *d_views;
    Ray *d_templ;
    unsigned long long *counter;
    AG_CUDA(sc.alloc((void **)&d_views, sizeof(ViewGeom) * views.size()));
    AG_CUDA(sc.alloc((void **)&d_templ, sizeof(Ray) * views.size()));
    AG_CUDA(sc.alloc((void **)&counter, sizeof(unsigned long long)));
    AG_CUDA(cudaMemcpyAsync(d_views, views.data(), sizeof(ViewGeom) * views.size(), cudaMemcpyHostToDevice, s));
    k_view_rays<<<(unsigned)((n_views + 127) / 128), 128, 0, s>>>(d_views, n_views, d_templ);
    AG_CUDA_LAUNCH("k_view_rays");
    AG_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    AG_CUDA(cudaMemsetAsync(d_visible, 0, (size_t)h->n_tris, s));
    VisArgs A;
    memset(&A, 0, sizeof(A));
    A.nodes = h->nodes;
    A.tris = h->tris;
    A.tri_ids = h->tri_ids;
    A.scene_abs = 0.f;
    for (int k = 0; k < 3; ++k) A.scene_abs = fmaxf(A.scene_abs, fmaxf(fabsf(h->lo[k]), fabsf(h->hi[k])));
    A.lo = make_float3(h->lo[0], h->lo[1], h->lo[2]);
    A.hi = make_float3(h->hi[0], h->hi[1], h->hi[2]);
    A.views = d_views;
    A.templ = d_templ;
    A.res = res;
    A.tiles_x = (res + 7) / 8;
    A.tiles_per_view = A.tiles_x * ((res + 3) / 4);
    if ((long long)A.tiles_per_view * n_views >= (1ll << 31))
        return set_error(AG_ERR_INVALID_ARG, "n_views * res^2 exceeds 2^36 rays");
    A.n_tiles = A.tiles_per_view * n_views;
    A.R = (float)R;
    A.scale = (float)(2.0 * R / res);
    A.tmax = (float)(4.0 * R);
    A.counter = counter;
    A.status = status;
    A.max_steps = o.max_steps > 0 ? o.max_steps : (1 << 20);
    A.visible = d_visible;
    A.hit_ids = d_hit_ids;
    A.counters = reinterpret_cast<unsigned long long *>(d_counters);
    if (o.render != AG_RENDER_RASTER && o.render != AG_RENDER_TRACE)
        return set_error(AG_ERR_INVALID_ARG, "render must be AG_RENDER_RASTER or AG_RENDER_TRACE");
    if (o.render == AG_RENDER_RASTER && !d_counters && h->n_tris > 0) {
        // z-buffer proposals per chunk of views (keys sized to stay in L2);
        // rejected pixels are traced once at the end
        const long long npix = (long long)res * res;
        // views per chunk: keys within the budget, the views on grid.y (< 2^16), and
        // the chunk's (view, 32-triangle group) items countable in 32 bits
        const long long groups = (h->n_tris + 31) / 32;
        const long long cmax = std::min(65535ll, 0xffffffffll / groups);
        const int chunk = (int)std::max(1ll, std::min<long long>(std::min<long long>(n_views, cmax),
                                                                 VIS_CHUNK_BYTES / (8ll * npix)));
        const unsigned long long cap = (unsigned long long)std::min<long long>((long long)n_views * npix, VIS_LIST_CAP);
        unsigned long long *keys, *list, *count;
        int *overflow;
        const int n_chunks = (n_views + chunk - 1) / chunk;
        AG_CUDA(sc.alloc((void **)&keys, sizeof(unsigned long long) * (size_t)chunk * npix));
        AG_CUDA(sc.alloc((void **)&list, sizeof(unsigned long long) * (size_t)cap));
        AG_CUDA(sc.alloc((void **)&count, sizeof(unsigned long long)));
        AG_CUDA(sc.alloc((void **)&overflow, sizeof(int) * (size_t)n_chunks));
        AG_CUDA(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * (size_t)chunk * npix, s));
        AG_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
        AG_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int) * (size_t)n_chunks, s));
        VisRaster Z;
        Z.tris = h->tris;
        Z.n_tris = (int)h->n_tris;
        Z.views = d_views;
        Z.res = res;
        Z.R = A.R;
        Z.scale = A.scale;
        Z.keys = keys;
        const unsigned zgrid = resident_blocks(k_vis_zbuffer, 256, h->device);
        // resolve: grid.y over the chunk's views, one wave of blocks in all
        const unsigned rgrid_x = std::max(1u, resident_blocks(k_vis_resolve, 256, h->device) / (unsigned)chunk);
        unsigned *next;
        AG_CUDA(sc.alloc((void **)&next, sizeof(unsigned) * (size_t)n_chunks));
        AG_CUDA(cudaMemsetAsync(next, 0, sizeof(unsigned) * (size_t)n_chunks, s));
        const unsigned tgrid = h->layout == AG_BVH_Q8 ? resident_blocks(k_vis_trace<AG_BVH_Q8>, 128, h->device)
                                                      : resident_blocks(k_vis_trace<AG_BVH_F32>, 128, h->device);
        auto trace = [&](const int *ovf, int v0, int nv) {
            if (h->layout == AG_BVH_Q8)
                k_vis_trace<AG_BVH_Q8><<<tgrid, 128, 0, s>>>(A, list, count, cap, ovf, v0, nv);
            else
                k_vis_trace<AG_BVH_F32><<<tgrid, 128, 0, s>>>(A, list, count, cap, ovf, v0, nv);
            return cudaGetLastError();
        };
        for (int c = 0; c < n_chunks; ++c) {
            const int v0 = c * chunk, nv = std::min(chunk, n_views - v0);
            Z.v0 = v0;
            Z.nv = nv;
            Z.next = next + c;
            k_vis_zbuffer<<<zgrid, 256, 0, s>>>(Z);
            AG_CUDA_LAUNCH("k_vis_zbuffer");
            k_vis_resolve<<<dim3(rgrid_x, (unsigned)nv), 256, 0, s>>>(A, keys, v0, list, cap, count, overflow + c);
            AG_CUDA_LAUNCH("k_vis_resolve");
            AG_CUDA(trace(overflow + c, v0, nv));   // exits at once unless the list overflowed
        }
        AG_CUDA(trace(nullptr, 0, 0));
        return AG_OK;
    }
    const int block = o.block_size > 0 ? o.block_size : 128;
    const bool cnt = d_counters != nullptr;
    cudaError_t e;
    if (h->layout == AG_BVH_Q8)
        e = cnt ? launch_vis<AG_BVH_Q8, true>(A, block, o.blocks_per_sm, s)
                : launch_vis<AG_BVH_Q8, false>(A, block, o.blocks_per_sm, s);
    else
        e = cnt ? launch_vis<AG_BVH_F32, true>(A, block, o.blocks_per_sm, s)
                : launch_vis<AG_BVH_F32, false>(A, block, o.blocks_per_sm, s);
    if (e != cudaSuccess) return cuda_error(e, "k_visibility");
    return AG_OK;
}

AG_API ag_status ag_exterior_fill(const float *d_verts, int64_t n_verts, const int32_t *d_faces, int64_t n_faces,
                                  const uint8_t *d_visible, ag_stream_t stream, uint8_t *d_exterior) {
    if (!d_verts || !d_faces || !d_visible || !d_exterior)
        return set_error(AG_ERR_INVALID_ARG, "pointers must be non-NULL");
    if (n_verts < 1 || n_verts >= (1ll << 31)) return set_error(AG_ERR_INVALID_ARG, "n_verts out of range");
    if (n_faces < 1 || n_faces >= (1ll << 29)) return set_error(AG_ERR_INVALID_ARG, "n_faces out of range");
    int dev = 0;
    AG_CUDA(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(dev);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    Scratch sc(s, dev);
    void *csr;
    double *nrm;
    int32_t *state, *qa, *qb;
    AG_CUDA(sc.alloc(&csr, vertex_normal_scratch_bytes(n_verts, n_faces)));
    AG_CUDA(sc.alloc((void **)&nrm, sizeof(double) * 3 * (size_t)n_faces));
    AG_CUDA(sc.alloc((void **)&state, sizeof(int32_t) * (size_t)n_faces));
    AG_CUDA(sc.alloc((void **)&qa, sizeof(int32_t) * (size_t)n_faces));
    AG_CUDA(sc.alloc((void **)&qb, sizeof(int32_t) * (size_t)n_faces));
    const unsigned *off;
    const int32_t *list;
    AG_CUDA(launch_vertex_face_csr(d_faces, n_faces, n_verts, csr, &off, &list, s));
    k_face_normals64<<<(unsigned)((n_faces + 255) / 256), 256, 0, s>>>(d_verts, d_faces, n_faces, n_verts, d_visible,
                                                                         nrm, state, status);
    AG_CUDA_LAUNCH("k_face_normals64");
    unsigned *counts;
    AG_CUDA(sc.alloc((void **)&counts, sizeof(unsigned) * (FLOOD_GRID_LEVELS + 1)));
    AG_CUDA(cudaMemsetAsync(counts, 0, sizeof(unsigned) * (FLOOD_GRID_LEVELS + 1), s));
    k_flood_seed<<<(unsigned)((n_faces + 255) / 256), 256, 0, s>>>(state, n_faces, qa, counts);
    AG_CUDA_LAUNCH("k_flood_seed");
    const unsigned lgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(device_sm_count(dev) * 4, (n_faces + 255) / 256));
    for (int l = 0; l < FLOOD_GRID_LEVELS; ++l) {
        k_flood_level<<<lgrid, 256, 0, s>>>(d_faces, off, list, nrm, state, qa, counts + l, qb, counts + l + 1);
        AG_CUDA_LAUNCH("k_flood_level");
        std::swap(qa, qb);
    }
    k_flood<<<1, FLOOD_THREADS, 0, s>>>(d_faces, n_faces, off, list, nrm, state, qa, counts + FLOOD_GRID_LEVELS, qb,
                                        d_exterior);
    AG_CUDA_LAUNCH("k_flood");
    return AG_OK;
}

}  // extern "C"
