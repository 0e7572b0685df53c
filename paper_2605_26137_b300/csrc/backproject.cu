// UV-space backprojection and incidence blending (Sec. 7.4): the colours of K
// generated views are carried back onto the texture atlas through the
// texels' surface points, weighted by how squarely and how visibly each view
// sees them.
//
// k_zbuffer: a z-buffer pass that proposes each pixel's first triangle: one
// lane per (view, triangle) sets up the projected triangle (edge functions
// evaluated with the lexicographically smaller endpoint first, so that two
// triangles sharing an edge get exactly opposite values and no pixel centre
// falls between them), the warp then walks the 32 triangles' pixel boxes
// together (a prefix sum over the box sizes spreads the pixels evenly over
// the lanes), and every covered pixel centre takes a 64-bit atomicMin of
// (camera depth bits, triangle record).  A view in which some triangle
// reaches the camera plane is traced whole instead.
// k_render_views: the depth buffer, world-point map of every view (pinhole
// camera, one thread per pixel, the ray through the pixel centre).  With a
// raster proposal the pixel's proposed triangle is tested with the
// watertight ray-triangle test of rays.cuh; when the test confirms it the
// hit is that of the full traversal, otherwise (a pixel centre within
// rounding of an edge) the ray is traced through the BVH with the
// closest-hit machinery of rays.cuh (camera depth of the first hit).
// k_edge_mask: pixels whose 4-neighbours miss or lie farther than edge_tol in
// world space (depth discontinuities and silhouettes).
// k_backproject: per ray texel (the bake's UV raster and ray list), for every
// view: camera coordinates of the surface point, its pixel, the depth test
// against the pixel's depth + depth_tol, the edge mask, the incidence
// I = max(0, n . direction to the camera), the bilinear colour at
// (u - 1/2, v - 1/2); the blend sum_k w_k I_k^alpha A_k / (sum_k w_k I_k^alpha
// + eps) is accumulated in one pass in log space (running maximum of
// log w_k + alpha log I_k, rescaled sums), so large alpha neither under- nor
// overflows.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "rays.cuh"

namespace ag {
namespace {

struct Cam {
    float R[9], t[3], fx, fy, cx, cy;
};

struct RenderArgs {
    const void *nodes;
    const float4 *tris;
    const int32_t *tri_ids;
    float scene_abs;
    const Cam *cams;
    int w, h, n_views;
    unsigned *status;
    int max_steps;
    float *depth;
    float *points;
    const unsigned long long *keys;   // raster proposals of views [v0, v0 + nv)
    const int *whole;                 // per view: 1 = a triangle reaches the camera plane, trace every pixel
    uint32_t *list;                   // pixels (within the launch's views) left to trace, or null: all
    unsigned *count;                  // entries of list
    int v0, nv;                       // the views of this launch
};

constexpr unsigned long long NO_KEY = ~0ull;

struct RasterArgs {
    const float4 *tris;
    int n_tris;
    const Cam *cams;
    int w, h, v0, nv;
    unsigned long long *keys;   // [nv*w*h], NO_KEY before the pass
    int *whole;                 // [n_views]
};

// one lane's triangle: three canonical edges (a, b - a) with the orientation
// that makes the inside non-negative, the camera-space plane n . X = d0, the
// pixel box
struct TriSetup {
    float ax[3], ay[3], dx[3], dy[3];   // canonical edges, (dx, dy) negated where the inside is negative
    float nx, ny, nz, d0;
    int x0, y0, bw;
    float rbw;        // 1 / bw, for the first pixel offset -> (x, y) split
    unsigned rec, cnt;
};

__device__ __forceinline__ float edge_fn(float ax, float ay, float dx, float dy, float px, float py) {
    return __fsub_rn(__fmul_rn(dx, __fsub_rn(py, ay)), __fmul_rn(dy, __fsub_rn(px, ax)));
}

__global__ void __launch_bounds__(256) k_zbuffer(RasterArgs A) {
    __shared__ TriSetup ts[256];
    const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
    const int kv = blockIdx.y;                       // view within the launch
    const int tri = blockIdx.x * 256 + threadIdx.x;
    const int k = A.v0 + kv;
    const Cam &c = A.cams[k];
    unsigned cnt = 0;
    TriSetup T;
    if (tri < A.n_tris) {
        float X[3], Y[3], Z[3], u[3], v[3];
        bool ok = true;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float4 p = __ldg(&A.tris[3 * (size_t)tri + m]);
            X[m] = c.R[0] * p.x + c.R[1] * p.y + c.R[2] * p.z + c.t[0];
            Y[m] = c.R[3] * p.x + c.R[4] * p.y + c.R[5] * p.z + c.t[1];
            Z[m] = c.R[6] * p.x + c.R[7] * p.y + c.R[8] * p.z + c.t[2];
            u[m] = c.fx * X[m] / Z[m] + c.cx;
            v[m] = c.fy * Y[m] / Z[m] + c.cy;
            ok = ok && Z[m] > 0.f && fabsf(u[m]) < 1.0e30f && fabsf(v[m]) < 1.0e30f;
        }
        if (!ok) {
            A.whole[k] = 1;
        } else {
            const float area = (u[1] - u[0]) * (v[2] - v[0]) - (v[1] - v[0]) * (u[2] - u[0]);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const int q = m == 2 ? 0 : m + 1;
                const bool sw = u[q] < u[m] || (u[q] == u[m] && v[q] < v[m]);
                const int a = sw ? q : m, b = sw ? m : q;
                // negating both differences negates the rounded edge value exactly
                const float sg = (sw != (area < 0.f)) ? -1.f : 1.f;
                T.ax[m] = u[a];
                T.ay[m] = v[a];
                T.dx[m] = sg * (u[b] - u[a]);
                T.dy[m] = sg * (v[b] - v[a]);
            }
            const float e1x = X[1] - X[0], e1y = Y[1] - Y[0], e1z = Z[1] - Z[0];
            const float e2x = X[2] - X[0], e2y = Y[2] - Y[0], e2z = Z[2] - Z[0];
            T.nx = e1y * e2z - e1z * e2y;
            T.ny = e1z * e2x - e1x * e2z;
            T.nz = e1x * e2y - e1y * e2x;
            T.d0 = T.nx * X[0] + T.ny * Y[0] + T.nz * Z[0];
            T.rec = (unsigned)tri;
            // pixel centres i + 1/2 inside [min u, max u] (and v), clamped to the image
            const float lo_u = fminf(u[0], fminf(u[1], u[2])), hi_u = fmaxf(u[0], fmaxf(u[1], u[2]));
            const float lo_v = fminf(v[0], fminf(v[1], v[2])), hi_v = fmaxf(v[0], fmaxf(v[1], v[2]));
            const int x0 = (int)fmaxf(ceilf(lo_u - 0.5f), 0.f), x1 = (int)fminf(floorf(hi_u - 0.5f), (float)(A.w - 1));
            const int y0 = (int)fmaxf(ceilf(lo_v - 0.5f), 0.f), y1 = (int)fminf(floorf(hi_v - 0.5f), (float)(A.h - 1));
            T.x0 = x0;
            T.y0 = y0;
            T.bw = x1 - x0 + 1;
            T.rbw = 1.0f / (float)T.bw;
            // at most 16384^2 = 2^28 pixels
            if (area != 0.f && x1 >= x0 && y1 >= y0) cnt = (unsigned)(x1 - x0 + 1) * (unsigned)(y1 - y0 + 1);
        }
    }
    T.cnt = cnt;
    ts[threadIdx.x] = T;
    __syncwarp();
    const long long npix = (long long)A.w * A.h;
    unsigned long long *keys = A.keys + (long long)kv * npix;
    const float icx = c.cx, icy = c.cy, rfx = 1.0f / c.fx, rfy = 1.0f / c.fy;
    // the warp walks its 32 triangles one after the other, the lanes over
    // the pixels of the current triangle's box (setup loads are broadcasts)
    for (int q = 0; q < 32; ++q) {
        const TriSetup &S = ts[wbase + q];
        const unsigned n = S.cnt;
        if (n == 0) continue;
        const int bw = S.bw;
        // the lane's pixels o = lane, lane + 32, ... of the box, o = y bw + x,
        // stepped by (32 mod bw, 32 div bw) with one wrap: exact integers and
        // exact small floats for the centre coordinates (the first split: a
        // float estimate of lane / bw is within one, one correction)
        int yy = (int)((float)lane * S.rbw);
        int xx = lane - yy * bw;
        if (xx < 0) { --yy; xx += bw; } else if (xx >= bw) { ++yy; xx -= bw; }
        const int sx = bw > 32 ? 32 : 32 % bw, sy = bw > 32 ? 0 : 32 / bw;
        float px = (float)(S.x0 + xx) + 0.5f, py = (float)(S.y0 + yy) + 0.5f;
        long long at = (long long)(S.y0 + yy) * A.w + S.x0 + xx;
        const long long astep = (long long)sy * A.w + sx, awrap = (long long)A.w - bw;
        for (unsigned o = lane; o < n; o += 32) {
            bool in = true;
#pragma unroll
            for (int m = 0; m < 3; ++m) in = in && edge_fn(S.ax[m], S.ay[m], S.dx[m], S.dy[m], px, py) >= 0.f;
            if (in) {
                const float xh = (px - icx) * rfx, yh = (py - icy) * rfy;
                const float z = __fdividef(S.d0, S.nx * xh + S.ny * yh + S.nz);
                if (z > 0.f && z < 3.0e38f)
                    atomicMin(&keys[at], ((unsigned long long)__float_as_uint(z) << 32) | S.rec);
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

// the watertight ray-triangle test of rays.cuh, keeping only hits in front
// of the camera: the smallest t > 0 (b.babs holds it), equal t: lower id
__device__ __forceinline__ void test_tri_front(const Ray &r, const float4 *__restrict__ tris,
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
    if (!(t > 0.f) || !(t <= b.babs)) return;
    if (b.found && t == b.babs && tri_ids[rec] >= tri_ids[b.rec]) return;
    b.t = t; b.babs = t; b.rec = rec; b.U = U; b.V = V; b.W = W; b.det = det; b.found = true;
}

// the ray through pixel (i, j): camera centre C = -R^T t and unit direction
// normalize(R^T ((i + 1/2 - cx) / fx, (j + 1/2 - cy) / fy, 1))
__device__ __forceinline__ void pixel_ray(const Cam &c, int i, int j, float3 &C, float3 &d) {
    const float dcx = ((float)i + 0.5f - c.cx) / c.fx, dcy = ((float)j + 0.5f - c.cy) / c.fy;
    d = normalize3(make_float3(c.R[0] * dcx + c.R[3] * dcy + c.R[6], c.R[1] * dcx + c.R[4] * dcy + c.R[7],
                               c.R[2] * dcx + c.R[5] * dcy + c.R[8]));
    C = make_float3(-(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]),
                    -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]),
                    -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]));
}

// depth = t (d . forward), point = C + t d; +inf / NaN on a miss
__device__ __forceinline__ void store_pixel(const RenderArgs &A, long long r, const Cam &c, float3 C, float3 d, bool hit,
                                            float t) {
    A.depth[r] = hit ? t * dot3(d, make_float3(c.R[6], c.R[7], c.R[8])) : __int_as_float(0x7f800000);
    if (A.points) {
        const float3 X = C + d * t;
        const float nanv = __int_as_float(0x7fc00000);
        A.points[3 * r] = hit ? X.x : nanv;
        A.points[3 * r + 1] = hit ? X.y : nanv;
        A.points[3 * r + 2] = hit ? X.z : nanv;
    }
}

// the light pass over the raster proposals: a miss where nothing covers the
// pixel centre, the proposed triangle's hit where the ray test confirms it;
// every other pixel (a rejected proposal, or a view traced whole) is
// appended to the trace list (warp-aggregated append)
__global__ void __launch_bounds__(256) k_resolve_views(RenderArgs A) {
    const long long npix = (long long)A.w * A.h;
    const long long n = (long long)A.nv * npix;
    const int lane = threadIdx.x & 31;
    for (long long rr = (long long)blockIdx.x * blockDim.x + threadIdx.x; rr < n; rr += (long long)gridDim.x * blockDim.x) {
        const int kv = (int)(rr / npix);
        const int k = A.v0 + kv;
        const int pix = (int)(rr - (long long)kv * npix);
        const long long r = (long long)k * npix + pix;
        bool queue = false;
        if (A.whole[k]) {
            queue = true;
        } else {
            const unsigned long long key = A.keys[rr];
            const Cam &c = A.cams[k];
            float3 C, d;
            if (key == NO_KEY) {
                A.depth[r] = __int_as_float(0x7f800000);
                if (A.points) {
                    const float nanv = __int_as_float(0x7fc00000);
                    A.points[3 * r] = nanv;
                    A.points[3 * r + 1] = nanv;
                    A.points[3 * r + 2] = nanv;
                }
            } else {
                pixel_ray(c, pix % A.w, pix / A.w, C, d);
                const Ray ray = make_ray(C, make_float3(0.f, 0.f, 0.f), d);
                Best b;
                b.t = 0.f; b.babs = 3.0e38f; b.rec = 0; b.found = false;
                b.U = b.V = b.W = 0.f; b.det = 1.f;
                test_tri_front(ray, A.tris, A.tri_ids, (uint32_t)(key & 0xffffffffu), b);
                if (b.found)
                    store_pixel(A, r, c, C, d, true, b.t);
                else
                    queue = true;
            }
        }
        const unsigned act = __activemask();
        const unsigned want = __ballot_sync(act, queue);
        if (want) {
            const int leader = __ffs(want) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(A.count, (unsigned)__popc(want));
            base = __shfl_sync(act, base, leader);
            if (queue) A.list[base + __popc(want & ((1u << lane) - 1u))] = (uint32_t)rr;
        }
    }
}

// the full closest-hit traversal for the pixels of the trace list (or for
// every pixel of the launch's views when there is no list)
template <int LAYOUT>
__global__ void __launch_bounds__(128) k_trace_views(RenderArgs A) {
    uint2 stack[STACK];
    const long long npix = (long long)A.w * A.h;
    const long long n = A.list ? (long long)*A.count : (long long)A.nv * npix;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long rr = A.list ? (long long)A.list[e] : e;
        const int kv = (int)(rr / npix);
        const int k = A.v0 + kv;
        const int pix = (int)(rr - (long long)kv * npix);
        const long long r = (long long)k * npix + pix;
        const Cam &c = A.cams[k];
        float3 C, d;
        pixel_ray(c, pix % A.w, pix / A.w, C, d);
        const Ray ray = make_ray(C, make_float3(0.f, 0.f, 0.f), d);
        Best b;
        b.t = 0.f; b.babs = 3.0e38f; b.rec = 0; b.found = false;
        b.U = b.V = b.W = 0.f; b.det = 1.f;
        uint32_t cur = 0;
        int sp = 0, steps = 0;
        for (;;) {
            Next nx;
            nx.has = false;
            nx.ref = 0;
            nx.dist = 0.f;
            // every step a node visit (the root is always a node), its hit leaf children tested here
            LeafSet ls;
            if (LAYOUT == AG_BVH_Q8)
                NodeOps<AG_BVH_Q8>::visit<true>(A.nodes, cur, ray, b.babs, nx, stack, sp, A.status, STACK, &ls);
            else
                NodeOps<AG_BVH_F32>::visit<true>(A.nodes, cur, ray, b.babs, nx, stack, sp, A.status, A.scene_abs,
                                                 STACK, &ls);
            while (ls.mask) {
                const int c = __ffs(ls.mask) - 1;
                ls.mask &= ls.mask - 1;
                uint32_t first;
                int cnt;
                leaf_range(ls, c, first, cnt);
                for (int q = 0; q < cnt; ++q) test_tri_front(ray, A.tris, A.tri_ids, first + q, b);
            }
            if (nx.has) {
                cur = nx.ref;
            } else {
                bool done = true;
                while (sp > 0) {
                    uint2 en = stack[--sp];
                    if (__uint_as_float(en.y) <= b.babs) { cur = en.x; done = false; break; }
                }
                if (done) break;
            }
            if (++steps > A.max_steps) {
                atomicOr(A.status, AGS_STEP_CAP);
                break;
            }
        }
        store_pixel(A, r, c, C, d, b.found, b.t);
    }
}

// edge pixels from the depth buffer alone: the world point of pixel (i, j)
// at camera depth z is C + z R^T ((i + 1/2 - cx) / fx, (j + 1/2 - cy) / fy, 1)
__global__ void k_edge_mask(const float *__restrict__ depth, const Cam *__restrict__ cams, int w, int h, int n_views,
                            float edge_tol, uint8_t *__restrict__ edge) {
    const long long n = (long long)n_views * w * h;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int k = (int)(r / ((long long)w * h));
    const int pix = (int)(r - (long long)k * w * h);
    const int i = pix % w, j = pix / w;
    uint8_t e = 0;
    const float z = depth[r];
    if (z < 3.0e38f) {
        const Cam &c = cams[k];
        const float rfx = 1.0f / c.fx, rfy = 1.0f / c.fy;
        const float3 C = make_float3(-(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]),
                                     -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]),
                                     -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]));
        const float3 ex = make_float3(c.R[0], c.R[1], c.R[2]), ey = make_float3(c.R[3], c.R[4], c.R[5]);
        const float3 ez = make_float3(c.R[6], c.R[7], c.R[8]);
        auto point = [&](int ii, int jj, float zz) {
            const float x = ((float)ii + 0.5f - c.cx) * rfx, y = ((float)jj + 0.5f - c.cy) * rfy;
            return C + (ex * x + ey * y + ez) * zz;
        };
        const float3 P = point(i, j, z);
        const float tol2 = edge_tol * edge_tol;
        const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int ii = i + di[m], jj = j + dj[m];
            if (ii < 0 || jj < 0 || ii >= w || jj >= h) continue;
            const float zq = depth[(long long)k * w * h + (long long)jj * w + ii];
            if (!(zq < 3.0e38f)) { e = 1; continue; }
            const float3 D = point(ii, jj, zq) - P;
            if (dot3(D, D) > tol2) e = 1;
        }
    }
    edge[r] = e;
}

// The views' Lanczos-2 pyramids: level 0 is the RGBA8 image itself, levels
// 1.. (sharpened, RGB in float4) are stored per view at off[l] within a
// block of `stride` pixels.
constexpr int MAX_LEV = 16;
struct Pyramid {
    int n;                       // levels, level 0 included
    int w[MAX_LEV], h[MAX_LEV];
    long long off[MAX_LEV];
    long long stride;
    const float4 *S;             // [n_views * stride]
};

struct BlendArgs {
    const float4 *lpos, *lnrm;
    const int4 *lface;
    const float *luv;            // per corner [F*3*2] (anisotropic footprint)
    const int4 *rays;
    const long long *n_rays;
    const Cam *cams;
    const float4 *centres;       // camera centres -R^T t
    const float *logw;           // log of the view prior weights
    const uint8_t *images;       // [K*h*w*4]
    const float *depth;          // [K*h*w]
    const uint8_t *edge;         // [K*h*w]
    int w, h, n_views, W, H;
    float alpha, eps, depth_tol;
    int filter;                  // AG_FILTER_*
    float lod_bias;
    int max_taps;
    Pyramid pyr;
    float4 *texture;             // [H*W]: rgb, filled
    float *incidence;            // optional [K*H*W]
};

// RGB of pixel (x, y) clamped to the image, one 32-bit load (the images are
// 4-byte aligned RGBA8)
__device__ __forceinline__ float3 texel_rgb(const uint8_t *img, int w, int h, int x, int y) {
    x = min(max(x, 0), w - 1);
    y = min(max(y, 0), h - 1);
    const uchar4 c = reinterpret_cast<const uchar4 *>(img)[(long long)y * w + x];
    return make_float3(c.x * (1.0f / 255.0f), c.y * (1.0f / 255.0f), c.z * (1.0f / 255.0f));
}

// bilinear RGB of the 8-bit image at image position (u, v): sample point
// (u - 1/2, v - 1/2) on the pixel-centre grid, clamped to the image
__device__ __forceinline__ float3 sample_image(const uint8_t *img, int w, int h, float u, float v) {
    const float x = u - 0.5f, y = v - 0.5f;
    const float fx0 = floorf(x), fy0 = floorf(y);
    const float ax = x - fx0, ay = y - fy0;
    const int x0 = (int)fx0, y0 = (int)fy0;
    const float3 p00 = texel_rgb(img, w, h, x0, y0), p10 = texel_rgb(img, w, h, x0 + 1, y0);
    const float3 p01 = texel_rgb(img, w, h, x0, y0 + 1), p11 = texel_rgb(img, w, h, x0 + 1, y0 + 1);
    const float w00 = (1.f - ax) * (1.f - ay), w10 = ax * (1.f - ay), w01 = (1.f - ax) * ay, w11 = ax * ay;
    return make_float3(w00 * p00.x + w10 * p10.x + w01 * p01.x + w11 * p11.x,
                       w00 * p00.y + w10 * p10.y + w01 * p01.y + w11 * p11.y,
                       w00 * p00.z + w10 * p10.z + w01 * p01.z + w11 * p11.z);
}

// bilinear RGB of pyramid level l >= 1 at level-0 image position (u, v)
__device__ __forceinline__ float3 sample_level(const float4 *lev, int w, int h, int l, float u, float v) {
    const float sc = __int_as_float((127 - l) << 23);     // 2^-l
    const float x = u * sc - 0.5f, y = v * sc - 0.5f;
    const float fx0 = floorf(x), fy0 = floorf(y);
    const float ax = x - fx0, ay = y - fy0;
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
    const int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
    const float4 p00 = lev[(long long)ya * w + xa], p10 = lev[(long long)ya * w + xb];
    const float4 p01 = lev[(long long)yb * w + xa], p11 = lev[(long long)yb * w + xb];
    const float w00 = (1.f - ax) * (1.f - ay), w10 = ax * (1.f - ay), w01 = (1.f - ax) * ay, w11 = ax * ay;
    return make_float3(w00 * p00.x + w10 * p10.x + w01 * p01.x + w11 * p11.x,
                       w00 * p00.y + w10 * p10.y + w01 * p01.y + w11 * p11.y,
                       w00 * p00.z + w10 * p10.z + w01 * p01.z + w11 * p11.z);
}

__device__ __forceinline__ float3 sample_lod(const BlendArgs &A, int k, int l, float u, float v) {
    if (l == 0) return sample_image(A.images + (long long)k * A.w * A.h * 4, A.w, A.h, u, v);
    const Pyramid &P = A.pyr;
    return sample_level(P.S + (long long)k * P.stride + P.off[l], P.w[l], P.h[l], l, u, v);
}

// anisotropic colour of view k at image position (u, v) for a texel of
// `face` at surface point p: central-difference footprint of the face's UV
// -> position map through the projection, its SVD, N taps along the major
// axis, each a trilinear sample at the level of the (compensated) minor axis
__device__ float3 aniso_color(const BlendArgs &A, int k, const Cam &c, int face, const int4 &fi, float3 p, float u,
                              float v) {
    const float *q = A.luv + 6 * (long long)face;
    const float x0 = q[0] * A.W, y0 = q[1] * A.H, x1 = q[2] * A.W, y1 = q[3] * A.H, x2 = q[4] * A.W, y2 = q[5] * A.H;
    const float det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
    bool ok = fabsf(det) * 0.5f >= 1e-4f;
    float J00 = 0.f, J01 = 0.f, J10 = 0.f, J11 = 0.f;
    if (ok) {
        const float b1x = (y2 - y0) / det, b1y = -(x2 - x0) / det;
        const float b2x = -(y1 - y0) / det, b2y = (x1 - x0) / det;
        const float3 P0 = f3(A.lpos[fi.x]);
        const float3 e1 = f3(A.lpos[fi.y]) - P0, e2 = f3(A.lpos[fi.z]) - P0;
        const float3 dpx = e1 * b1x + e2 * b2x, dpy = e1 * b1y + e2 * b2y;
        float Ju[2], Jv[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float3 d = (a ? dpy : dpx) * 0.5f;
            const float3 pa = p + d, pb = p - d;
            const float ax_ = c.R[0] * pa.x + c.R[1] * pa.y + c.R[2] * pa.z + c.t[0];
            const float ay_ = c.R[3] * pa.x + c.R[4] * pa.y + c.R[5] * pa.z + c.t[1];
            const float az_ = c.R[6] * pa.x + c.R[7] * pa.y + c.R[8] * pa.z + c.t[2];
            const float bx_ = c.R[0] * pb.x + c.R[1] * pb.y + c.R[2] * pb.z + c.t[0];
            const float by_ = c.R[3] * pb.x + c.R[4] * pb.y + c.R[5] * pb.z + c.t[1];
            const float bz_ = c.R[6] * pb.x + c.R[7] * pb.y + c.R[8] * pb.z + c.t[2];
            ok = ok && az_ > 0.f && bz_ > 0.f;
            Ju[a] = c.fx * ax_ / az_ - c.fx * bx_ / bz_;
            Jv[a] = c.fy * ay_ / az_ - c.fy * by_ / bz_;
        }
        J00 = Ju[0]; J01 = Ju[1]; J10 = Jv[0]; J11 = Jv[1];
    }
    if (!ok) return sample_image(A.images + (long long)k * A.w * A.h * 4, A.w, A.h, u, v);
    // J J^T = [[a, b], [b, d]]: singular values and the major image direction
    const float a = J00 * J00 + J01 * J01, b = J00 * J10 + J01 * J11, d = J10 * J10 + J11 * J11;
    const float half = 0.5f * (a + d), disc = sqrtf(0.25f * (a - d) * (a - d) + b * b);
    const float l1 = half + disc, l2 = fmaxf(half - disc, 0.f);
    const float s1 = sqrtf(l1), s2 = sqrtf(l2);
    float ex, ey;
    if (b != 0.f) { ex = l1 - d; ey = b; }
    else if (a >= d) { ex = 1.f; ey = 0.f; }
    else { ex = 0.f; ey = 1.f; }
    const float en = rsqrtf(ex * ex + ey * ey);
    ex *= en; ey *= en;
    int N = A.max_taps;
    if (s2 > 0.f) N = (int)fminf(fmaxf(ceilf(s1 / s2 - 0.05f), 1.f), (float)A.max_taps);
    const float mm = fmaxf(s2, s1 / (float)A.max_taps);
    float lam = mm > 0.f ? log2f(mm) + A.lod_bias : 0.f;
    lam = fminf(fmaxf(lam, 0.f), (float)(A.pyr.n - 1));
    const int l0 = (int)floorf(lam);
    const float fr = lam - (float)l0;
    const bool two = l0 < A.pyr.n - 1 && fr > 0.f;
    float3 acc = make_float3(0.f, 0.f, 0.f);
    for (int i = 0; i < N; ++i) {
        const float o = s1 * (((float)i + 0.5f) / (float)N - 0.5f);
        const float tu = u + ex * o, tv = v + ey * o;
        float3 sm = sample_lod(A, k, l0, tu, tv);
        if (two) sm = sm * (1.f - fr) + sample_lod(A, k, l0 + 1, tu, tv) * fr;
        acc = acc + sm;
    }
    return acc * (1.f / (float)N);
}

__global__ void __launch_bounds__(128) k_backproject(BlendArgs A) {
    const long long n = *A.n_rays;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const int4 rr = A.rays[r];
        const int texel = rr.x, face = rr.y;
        const float b1 = __int_as_float(rr.z), b2 = __int_as_float(rr.w);
        const int4 fi = A.lface[face];
        const float3 P0 = f3(A.lpos[fi.x]), P1 = f3(A.lpos[fi.y]), P2 = f3(A.lpos[fi.z]);
        const float3 N0 = f3(A.lnrm[fi.x]), N1 = f3(A.lnrm[fi.y]), N2 = f3(A.lnrm[fi.z]);
        const float3 p = P0 + (P1 - P0) * b1 + (P2 - P0) * b2;
        const float3 nrm = normalize3(N0 + (N1 - N0) * b1 + (N2 - N0) * b2);
        float m = -3.0e38f, den = 0.f, num0 = 0.f, num1 = 0.f, num2 = 0.f;
        bool any = false;
        const long long npix = (long long)A.w * A.h;
        for (int k = 0; k < A.n_views; ++k) {
            const Cam &c = A.cams[k];
            // incidence first (the cheapest test): a view that sees the back of the texel is skipped
            const float I = dot3(nrm, normalize3(f3(A.centres[k]) - p));
            if (!(I > 0.f)) continue;
            const float qx = c.R[0] * p.x + c.R[1] * p.y + c.R[2] * p.z + c.t[0];
            const float qy = c.R[3] * p.x + c.R[4] * p.y + c.R[5] * p.z + c.t[1];
            const float qz = c.R[6] * p.x + c.R[7] * p.y + c.R[8] * p.z + c.t[2];
            if (!(qz > 0.f)) continue;
            const float u = c.fx * qx / qz + c.cx, v = c.fy * qy / qz + c.cy;
            if (!(u >= 0.f && u < (float)A.w && v >= 0.f && v < (float)A.h)) continue;
            const int i = min((int)u, A.w - 1), j = min((int)v, A.h - 1);
            const long long px = (long long)k * npix + (long long)j * A.w + i;
            const float dz = A.depth[px];
            if (!(dz < 3.0e38f) || A.edge[px] || qz > dz + A.depth_tol) continue;
            if (A.incidence) A.incidence[(long long)k * A.W * A.H + texel] = I;
            // colour: anisotropic footprint taps, or one bilinear sample at (u - 1/2, v - 1/2)
            const float3 cc = A.filter == AG_FILTER_ANISO ? aniso_color(A, k, c, face, fi, p, u, v)
                                                           : sample_image(A.images + (long long)k * npix * 4, A.w,
                                                                          A.h, u, v);
            const float col[3] = {cc.x, cc.y, cc.z};
            // online log-sum-exp: keep den, num as sums of e^(L_k - m)
            const float L = A.logw[k] + A.alpha * logf(I);
            if (L > m) {
                const float s = any ? expf(m - L) : 0.f;
                den *= s; num0 *= s; num1 *= s; num2 *= s;
                m = L;
            }
            const float e = expf(L - m);
            den += e;
            num0 += e * col[0]; num1 += e * col[1]; num2 += e * col[2];
            any = true;
        }
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (any) {
            const float d = den + A.eps * expf(-m);
            out = make_float4(num0 / d, num1 / d, num2 / d, 1.f);
        }
        A.texture[texel] = out;
    }
}

// one 2x Lanczos-2 reduction for every view: level-l pixels 2x-3 .. 2x+4
// (clamped) with the normalised weights wt, rows first, clamped to [0, 1];
// the source is the RGBA8 image (level 0) or an unsharpened float level
struct MipArgs {
    const uint8_t *img0;
    const float4 *src;
    int sw, sh;
    float4 *dst;
    int dw, dh, n_views;
    float wt[8];
};

// a tile of 32 x 8 outputs per block: the 22 source rows it needs are first
// reduced horizontally into shared memory (8 taps each), then each output
// takes its 8 vertical taps from there
constexpr int MIP_TX = 32, MIP_TY = 8, MIP_ROWS = 2 * MIP_TY + 6;

__device__ __forceinline__ float3 mip_src(const MipArgs &M, long long q) {
    if (M.img0) {
        const uint8_t *c = M.img0 + 4 * q;
        return make_float3(c[0] * (1.0f / 255.0f), c[1] * (1.0f / 255.0f), c[2] * (1.0f / 255.0f));
    }
    const float4 c = M.src[q];
    return make_float3(c.x, c.y, c.z);
}

__global__ void __launch_bounds__(MIP_TX * MIP_TY) k_mip_down(MipArgs M) {
    __shared__ float3 hs[MIP_ROWS][MIP_TX];
    const int k = blockIdx.z;
    const int x = blockIdx.x * MIP_TX + threadIdx.x;
    const int y0 = blockIdx.y * MIP_TY;
    const long long sbase = (long long)k * M.sw * M.sh;
    // horizontal: source rows 2 y0 - 3 + r (clamped), output column x
    for (int r = threadIdx.y; r < MIP_ROWS; r += MIP_TY) {
        const int j = min(max(2 * y0 - 3 + r, 0), M.sh - 1);
        float3 acc = make_float3(0.f, 0.f, 0.f);
        if (x < M.dw) {
#pragma unroll
            for (int tx = 0; tx < 8; ++tx) {
                const int i = min(max(2 * x - 3 + tx, 0), M.sw - 1);
                const float3 v = mip_src(M, sbase + (long long)j * M.sw + i);
                acc.x += M.wt[tx] * v.x;
                acc.y += M.wt[tx] * v.y;
                acc.z += M.wt[tx] * v.z;
            }
        }
        hs[r][threadIdx.x] = acc;
    }
    __syncthreads();
    const int y = y0 + threadIdx.y;
    if (x >= M.dw || y >= M.dh) return;
    // vertical: output row y takes source rows 2y - 3 .. 2y + 4, local 2 (y - y0) + ty;
    // near the bottom edge the clamped rows repeat, which the local copy already holds
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int ty = 0; ty < 8; ++ty) {
        const float3 v = hs[2 * threadIdx.y + ty][threadIdx.x];
        a0 += M.wt[ty] * v.x;
        a1 += M.wt[ty] * v.y;
        a2 += M.wt[ty] * v.z;
    }
    M.dst[(long long)k * M.dw * M.dh + (long long)y * M.dw + x] =
        make_float4(fminf(fmaxf(a0, 0.f), 1.f), fminf(fmaxf(a1, 0.f), 1.f), fminf(fmaxf(a2, 0.f), 1.f), 0.f);
}

// the sampled copy of a level: clamp(P + amt (P - B P), 0, 1), B the
// separable [1, 2, 1] / 4 blur with clamped borders (rows first)
__global__ void k_mip_sharpen(const float4 *__restrict__ P, int w, int h, int n_views, float amt, float4 *S,
                              long long s_stride, long long s_off) {
    const long long per = (long long)w * h;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)n_views * per) return;
    const int k = (int)(r / per);
    const int pix = (int)(r - (long long)k * per);
    const int x = pix % w, y = pix / w;
    const int xl = max(x - 1, 0), xr = min(x + 1, w - 1);
    const float4 *Pk = P + (long long)k * per;
    float3 bl[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const int yy = min(max(y - 1 + m, 0), h - 1);
        const float4 l = Pk[(long long)yy * w + xl], c = Pk[(long long)yy * w + x], rr = Pk[(long long)yy * w + xr];
        bl[m] = make_float3(0.25f * l.x + 0.5f * c.x + 0.25f * rr.x, 0.25f * l.y + 0.5f * c.y + 0.25f * rr.y,
                            0.25f * l.z + 0.5f * c.z + 0.25f * rr.z);
    }
    const float3 b = bl[0] * 0.25f + bl[1] * 0.5f + bl[2] * 0.25f;
    const float4 c = Pk[pix];
    const float v0 = c.x + amt * (c.x - b.x), v1 = c.y + amt * (c.y - b.y), v2 = c.z + amt * (c.z - b.z);
    S[(long long)k * s_stride + s_off + pix] =
        make_float4(fminf(fmaxf(v0, 0.f), 1.f), fminf(fmaxf(v1, 0.f), 1.f), fminf(fmaxf(v2, 0.f), 1.f), 0.f);
}

// pyramid sizes for w x h views: level l + 1 has max(1, w_l / 2) x max(1, h_l / 2)
// pixels, down to 1 x 1 (at most MAX_LEV levels)
Pyramid pyramid_dims(int w, int h) {
    Pyramid P;
    memset(&P, 0, sizeof(P));
    P.n = 1;
    P.w[0] = w;
    P.h[0] = h;
    P.stride = 0;
    int pw = w, ph = h;
    while ((pw > 1 || ph > 1) && P.n < MAX_LEV) {
        pw = std::max(1, pw / 2);
        ph = std::max(1, ph / 2);
        P.w[P.n] = pw;
        P.h[P.n] = ph;
        P.off[P.n] = P.stride;
        P.stride += (long long)pw * ph;
        ++P.n;
    }
    return P;
}

// blocks of one wave: SMs x resident blocks per SM at this block size
template <typename Kernel>
unsigned resident_grid(Kernel kernel, int block, int dev) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return (unsigned)(device_sm_count(dev) * per_sm);
}

}  // namespace

cudaError_t launch_render_views(const TraceLaunch &L, int n_tris, const float *h_cams, int n_views, int w, int h,
                                float edge_tol, bool raster, float *depth, float *points, uint8_t *edge, void *scratch,
                                cudaStream_t s) {
    // scratch: cameras, per-view flags, list count | keys | list
    Cam *d_cams = static_cast<Cam *>(scratch);
    int *whole = reinterpret_cast<int *>(d_cams + n_views);
    unsigned *count = reinterpret_cast<unsigned *>(whole + n_views);
    const size_t head = render_head_bytes(n_views);
    const int chunk = render_chunk_views(n_views, w, h);
    const long long npix = (long long)w * h;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + head);
    uint32_t *list = reinterpret_cast<uint32_t *>(keys + (size_t)chunk * npix);
    cudaError_t e = cudaMemcpyAsync(d_cams, h_cams, sizeof(Cam) * n_views, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (raster && (e = cudaMemsetAsync(whole, 0, sizeof(int) * n_views, s)) != cudaSuccess) return e;
    RenderArgs A;
    A.nodes = L.job0.nodes;
    A.tris = L.job0.tris;
    A.tri_ids = L.job0.tri_ids;
    A.scene_abs = L.job0.scene_abs;
    A.cams = d_cams;
    A.w = w;
    A.h = h;
    A.n_views = n_views;
    A.status = L.status;
    A.max_steps = L.max_steps;
    A.depth = depth;
    A.points = points;
    A.whole = whole;
    A.count = count;
    int dev;
    cudaGetDevice(&dev);
    // one full wave of resident blocks (a partial second wave would double
    // the time of the grid-stride loops)
    const unsigned tgrid = L.layout == AG_BVH_Q8 ? resident_grid(k_trace_views<AG_BVH_Q8>, 128, dev)
                                                 : resident_grid(k_trace_views<AG_BVH_F32>, 128, dev);
    const unsigned rgrid = resident_grid(k_resolve_views, 256, dev);
    for (int v0 = 0; v0 < n_views; v0 += chunk) {
        const int nv = std::min(chunk, n_views - v0);
        A.v0 = v0;
        A.nv = nv;
        A.keys = nullptr;
        A.list = nullptr;
        if (raster && n_tris > 0) {
            if ((e = cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * (size_t)(nv * npix), s)) != cudaSuccess)
                return e;
            if ((e = cudaMemsetAsync(count, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
            RasterArgs R;
            R.tris = L.job0.tris;
            R.n_tris = n_tris;
            R.cams = d_cams;
            R.w = w;
            R.h = h;
            R.v0 = v0;
            R.nv = nv;
            R.keys = keys;
            R.whole = whole;
            k_zbuffer<<<dim3((unsigned)((n_tris + 255) / 256), (unsigned)nv), 256, 0, s>>>(R);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            A.keys = keys;
            A.list = list;
            k_resolve_views<<<rgrid, 256, 0, s>>>(A);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (L.layout == AG_BVH_Q8)
            k_trace_views<AG_BVH_Q8><<<tgrid, 128, 0, s>>>(A);
        else
            k_trace_views<AG_BVH_F32><<<tgrid, 128, 0, s>>>(A);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (edge) {
        const long long n = (long long)n_views * w * h;
        k_edge_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(depth, d_cams, w, h, n_views, edge_tol, edge);
        e = cudaGetLastError();
    }
    return e;
}

// cameras, per-view flags and the list count, rounded to 256 bytes
size_t render_head_bytes(int n_views) {
    return ((sizeof(Cam) + sizeof(int)) * (size_t)n_views + sizeof(unsigned) + 255) / 256 * 256;
}

// views per raster chunk: the chunk's proposal keys and trace list stay
// within 1.5 GiB
int render_chunk_views(int n_views, int w, int h) {
    const long long per_view = 12ll * w * h;
    return (int)std::max(1ll, std::min<long long>(n_views, (3ll << 29) / per_view));
}

size_t render_scratch_bytes(int n_views, int w, int h, bool raster) {
    return render_head_bytes(n_views) + (raster ? 12ull * (size_t)w * h * render_chunk_views(n_views, w, h) : 0);
}

static double lanczos2_host(double x) {
    if (x == 0.0) return 1.0;
    if (std::fabs(x) >= 2.0) return 0.0;
    const double px = 3.14159265358979323846 * x;
    return 2.0 * std::sin(px) * std::sin(0.5 * px) / (px * px);
}

// scratch: cameras | log-weights | (anisotropic) pyramid levels | two
// unsharpened level buffers
static size_t bp_head_bytes(int n_views) {
    return ((sizeof(Cam) + sizeof(float4) + sizeof(float)) * (size_t)n_views + 255) / 256 * 256;
}

size_t backproject_scratch_bytes(int n_views, int w, int h, int filter) {
    size_t b = bp_head_bytes(n_views);
    if (filter == AG_FILTER_ANISO) {
        const Pyramid P = pyramid_dims(w, h);
        b += sizeof(float4) * (size_t)n_views * (size_t)P.stride;
        if (P.n > 1) b += 2 * sizeof(float4) * (size_t)n_views * (size_t)P.w[1] * P.h[1];
    }
    return b;
}

cudaError_t launch_backproject(const float4 *lpos, const float4 *lnrm, const int4 *lface, const float *luv,
                               const int4 *rays, const long long *n_rays, int W, int H, const float *h_cams,
                               const float *h_centres, const float *h_logw, int n_views, const uint8_t *images, const float *depth,
                               const uint8_t *edge, int w, int h, float alpha, float eps, float depth_tol, int filter,
                               float lod_bias, int max_taps, float sharpen, float4 *texture, float *incidence,
                               void *scratch, cudaStream_t s) {
    Cam *d_cams = static_cast<Cam *>(scratch);
    float4 *d_centres = reinterpret_cast<float4 *>(d_cams + n_views);
    float *d_logw = reinterpret_cast<float *>(d_centres + n_views);
    cudaError_t e = cudaMemcpyAsync(d_cams, h_cams, sizeof(Cam) * n_views, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(d_logw, h_logw, sizeof(float) * n_views, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(d_centres, h_centres, sizeof(float4) * n_views, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(texture, 0, sizeof(float4) * (size_t)W * H, s)) != cudaSuccess) return e;
    if (incidence && (e = cudaMemsetAsync(incidence, 0, sizeof(float) * (size_t)n_views * W * H, s)) != cudaSuccess)
        return e;
    BlendArgs A;
    memset(&A, 0, sizeof(A));
    A.pyr = pyramid_dims(w, h);
    if (filter == AG_FILTER_ANISO && A.pyr.n > 1) {
        float4 *S = reinterpret_cast<float4 *>(static_cast<char *>(scratch) + bp_head_bytes(n_views));
        float4 *ping = S + (size_t)n_views * (size_t)A.pyr.stride;
        float4 *pong = ping + (size_t)n_views * (size_t)A.pyr.w[1] * A.pyr.h[1];
        MipArgs M;
        double wt[8], sw = 0.0;
        for (int t = 0; t < 8; ++t) { wt[t] = lanczos2_host((t - 3.5) / 2.0); sw += wt[t]; }
        for (int t = 0; t < 8; ++t) M.wt[t] = (float)(wt[t] / sw);
        M.n_views = n_views;
        for (int l = 1; l < A.pyr.n; ++l) {
            M.img0 = l == 1 ? images : nullptr;
            M.src = l == 1 ? nullptr : (l % 2 == 0 ? ping : pong);
            M.sw = A.pyr.w[l - 1];
            M.sh = A.pyr.h[l - 1];
            M.dst = l % 2 == 1 ? ping : pong;
            M.dw = A.pyr.w[l];
            M.dh = A.pyr.h[l];
            const long long n = (long long)n_views * M.dw * M.dh;
            const dim3 mgrid((unsigned)((M.dw + MIP_TX - 1) / MIP_TX), (unsigned)((M.dh + MIP_TY - 1) / MIP_TY),
                             (unsigned)n_views);
            k_mip_down<<<mgrid, dim3(MIP_TX, MIP_TY), 0, s>>>(M);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_mip_sharpen<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M.dst, M.dw, M.dh, n_views, sharpen, S,
                                                                     A.pyr.stride, A.pyr.off[l]);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        A.pyr.S = S;
    }
    A.lpos = lpos;
    A.lnrm = lnrm;
    A.lface = lface;
    A.luv = luv;
    A.rays = rays;
    A.n_rays = n_rays;
    A.cams = d_cams;
    A.centres = d_centres;
    A.logw = d_logw;
    A.images = images;
    A.depth = depth;
    A.edge = edge;
    A.w = w;
    A.h = h;
    A.n_views = n_views;
    A.W = W;
    A.H = H;
    A.alpha = alpha;
    A.eps = eps;
    A.depth_tol = depth_tol;
    A.filter = filter;
    A.lod_bias = lod_bias;
    A.max_taps = max_taps;
    A.texture = texture;
    A.incidence = incidence;
    int dev;
    cudaGetDevice(&dev);
    k_backproject<<<resident_grid(k_backproject, 128, dev), 128, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace ag
