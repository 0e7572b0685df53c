// UV-space backprojection and incidence blending (Sec. 7.4): the colours of K
// generated views are carried back onto the texture atlas through the
// texels' surface points, weighted by how squarely and how visibly each view
// sees them.
//
// k_render_views: the depth buffer, world-point map of every view (pinhole
// camera, one thread per pixel, the ray through the pixel centre traced with
// the closest-hit machinery of rays.cuh; camera depth of the first hit).
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
};

template <int LAYOUT>
__global__ void __launch_bounds__(128) k_render_views(RenderArgs A) {
    uint2 stack[STACK];
    const long long n = (long long)A.n_views * A.w * A.h;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(r / ((long long)A.w * A.h));
        const int pix = (int)(r - (long long)k * A.w * A.h);
        const int i = pix % A.w, j = pix / A.w;
        const Cam &c = A.cams[k];
        const float dcx = ((float)i + 0.5f - c.cx) / c.fx, dcy = ((float)j + 0.5f - c.cy) / c.fy;
        // world direction R^T (dcx, dcy, 1) and camera centre -R^T t
        float3 d = make_float3(c.R[0] * dcx + c.R[3] * dcy + c.R[6], c.R[1] * dcx + c.R[4] * dcy + c.R[7],
                               c.R[2] * dcx + c.R[5] * dcy + c.R[8]);
        d = normalize3(d);
        const float3 C = make_float3(-(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]),
                                     -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]),
                                     -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]));
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
            if (ref_is_leaf(cur)) {
                const uint32_t first = ref_first(cur);
                const int cnt = ref_count(cur);
                for (int q = 0; q < cnt; ++q) test_tri(ray, A.tris, A.tri_ids, first + q, b);
            } else if (LAYOUT == AG_BVH_Q8) {
                NodeOps<AG_BVH_Q8>::visit(A.nodes, cur, ray, b.babs, nx, stack, sp, A.status);
            } else {
                NodeOps<AG_BVH_F32>::visit(A.nodes, cur, ray, b.babs, nx, stack, sp, A.status, A.scene_abs);
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
                break;
            }
        }
        const bool hit = b.found && b.t > 0.f;
        const float3 fwd = make_float3(c.R[6], c.R[7], c.R[8]);
        A.depth[r] = hit ? b.t * dot3(d, fwd) : __int_as_float(0x7f800000);
        if (A.points) {
            const float3 X = C + d * b.t;
            const float nanv = __int_as_float(0x7fc00000);
            A.points[3 * r] = hit ? X.x : nanv;
            A.points[3 * r + 1] = hit ? X.y : nanv;
            A.points[3 * r + 2] = hit ? X.z : nanv;
        }
    }
}

__global__ void k_edge_mask(const float *__restrict__ depth, const float *__restrict__ points, int w, int h,
                            int n_views, float edge_tol, uint8_t *__restrict__ edge) {
    const long long n = (long long)n_views * w * h;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int k = (int)(r / ((long long)w * h));
    const int pix = (int)(r - (long long)k * w * h);
    const int i = pix % w, j = pix / w;
    uint8_t e = 0;
    if (depth[r] < 3.0e38f) {
        const float3 P = make_float3(points[3 * r], points[3 * r + 1], points[3 * r + 2]);
        const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
        for (int m = 0; m < 4 && !e; ++m) {
            const int ii = i + di[m], jj = j + dj[m];
            if (ii < 0 || jj < 0 || ii >= w || jj >= h) continue;
            const long long q = (long long)k * w * h + (long long)jj * w + ii;
            if (!(depth[q] < 3.0e38f)) { e = 1; break; }
            const float3 Q = make_float3(points[3 * q], points[3 * q + 1], points[3 * q + 2]);
            const float3 D = Q - P;
            if (dot3(D, D) > edge_tol * edge_tol) e = 1;
        }
    }
    edge[r] = e;
}

struct BlendArgs {
    const float4 *lpos, *lnrm;
    const int4 *lface;
    const int4 *rays;
    const long long *n_rays;
    const Cam *cams;
    const float *logw;           // log of the view prior weights
    const uint8_t *images;       // [K*h*w*4]
    const float *depth;          // [K*h*w]
    const uint8_t *edge;         // [K*h*w]
    int w, h, n_views, W, H;
    float alpha, eps, depth_tol;
    float4 *texture;             // [H*W]: rgb, filled
    float *incidence;            // optional [K*H*W]
};

__device__ __forceinline__ float texel_rgb(const uint8_t *img, int w, int h, int x, int y, int ch) {
    x = min(max(x, 0), w - 1);
    y = min(max(y, 0), h - 1);
    return (float)img[((long long)y * w + x) * 4 + ch] * (1.0f / 255.0f);
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
            const float3 C = make_float3(-(c.R[0] * c.t[0] + c.R[3] * c.t[1] + c.R[6] * c.t[2]),
                                         -(c.R[1] * c.t[0] + c.R[4] * c.t[1] + c.R[7] * c.t[2]),
                                         -(c.R[2] * c.t[0] + c.R[5] * c.t[1] + c.R[8] * c.t[2]));
            const float I = dot3(nrm, normalize3(C - p));
            if (!(I > 0.f)) continue;
            if (A.incidence) A.incidence[(long long)k * A.W * A.H + texel] = I;
            // bilinear colour at (u - 1/2, v - 1/2), clamped to the image
            const float x = u - 0.5f, y = v - 0.5f;
            const float fx0 = floorf(x), fy0 = floorf(y);
            const float ax = x - fx0, ay = y - fy0;
            const int x0 = (int)fx0, y0 = (int)fy0;
            const uint8_t *img = A.images + (long long)k * npix * 4;
            float col[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
                col[ch] = (1.f - ax) * (1.f - ay) * texel_rgb(img, A.w, A.h, x0, y0, ch) +
                          ax * (1.f - ay) * texel_rgb(img, A.w, A.h, x0 + 1, y0, ch) +
                          (1.f - ax) * ay * texel_rgb(img, A.w, A.h, x0, y0 + 1, ch) +
                          ax * ay * texel_rgb(img, A.w, A.h, x0 + 1, y0 + 1, ch);
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

}  // namespace

cudaError_t launch_render_views(const TraceLaunch &L, const float *h_cams, int n_views, int w, int h, float edge_tol,
                                float *depth, float *points, uint8_t *edge, void *scratch, cudaStream_t s) {
    Cam *d_cams = static_cast<Cam *>(scratch);
    cudaError_t e = cudaMemcpyAsync(d_cams, h_cams, sizeof(Cam) * n_views, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
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
    int dev;
    cudaGetDevice(&dev);
    const unsigned grid = (unsigned)(device_sm_count(dev) * 8);
    if (L.layout == AG_BVH_Q8)
        k_render_views<AG_BVH_Q8><<<grid, 128, 0, s>>>(A);
    else
        k_render_views<AG_BVH_F32><<<grid, 128, 0, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (edge) {
        const long long n = (long long)n_views * w * h;
        k_edge_mask<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(depth, points, w, h, n_views, edge_tol, edge);
        e = cudaGetLastError();
    }
    return e;
}

size_t render_scratch_bytes(int n_views) { return sizeof(Cam) * (size_t)n_views; }

cudaError_t launch_backproject(const float4 *lpos, const float4 *lnrm, const int4 *lface, const int4 *rays,
                               const long long *n_rays, int W, int H, const float *h_cams, const float *h_logw,
                               int n_views, const uint8_t *images, const float *depth, const uint8_t *edge, int w,
                               int h, float alpha, float eps, float depth_tol, float4 *texture, float *incidence,
                               void *scratch, cudaStream_t s) {
    Cam *d_cams = static_cast<Cam *>(scratch);
    float *d_logw = reinterpret_cast<float *>(d_cams + n_views);
    cudaError_t e = cudaMemcpyAsync(d_cams, h_cams, sizeof(Cam) * n_views, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(d_logw, h_logw, sizeof(float) * n_views, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(texture, 0, sizeof(float4) * (size_t)W * H, s)) != cudaSuccess) return e;
    if (incidence && (e = cudaMemsetAsync(incidence, 0, sizeof(float) * (size_t)n_views * W * H, s)) != cudaSuccess)
        return e;
    BlendArgs A;
    A.lpos = lpos;
    A.lnrm = lnrm;
    A.lface = lface;
    A.rays = rays;
    A.n_rays = n_rays;
    A.cams = d_cams;
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
    A.texture = texture;
    A.incidence = incidence;
    int dev;
    cudaGetDevice(&dev);
    k_backproject<<<(unsigned)(device_sm_count(dev) * 8), 128, 0, s>>>(A);
    return cudaGetLastError();
}

size_t backproject_scratch_bytes(int n_views) { return (sizeof(Cam) + sizeof(float)) * (size_t)n_views + 16; }

}  // namespace ag
