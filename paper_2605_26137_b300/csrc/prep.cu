// Low-poly side of the bake (Sec. 6.4, first stage: the G-buffer of the
// low-poly mesh rasterised into its own UV space):
//   area-weighted vertex normals -> per-face UV snapping, reliability flag and
//   corner tangent frames -> conservative UV raster (exact fixed-point keys,
//   atomicMin per texel) -> resolve to (face, barycentrics) and compact the
//   covered texels into a tile-ordered ray list.
#include "ag_internal.cuh"
#include "exact.cuh"

namespace ag {
namespace {

constexpr unsigned long long KEY_NONE = ~0ull;
constexpr unsigned long long KEY_CONS = 1ull << 63;

// round_half_away(u * W * 256), exact: the float's 24-bit significand times
// W*256 fits in 64 bits, and the shift rounds on the exact product.
__device__ __forceinline__ long long snap_exact(float u, int W) {
    unsigned bits = __float_as_uint(u);
    int e = (bits >> 23) & 255;
    if (e == 0) return 0;                       // zero / subnormal: |u*W*256| < 2^-100
    unsigned long long man = (bits & 0x7fffffu) | 0x800000u;
    unsigned long long P = man * (unsigned long long)W * 256ull;
    int sh = 150 - e;                           // value = P * 2^-sh ; sh >= 22 for |u| <= 2
    unsigned long long r = sh >= 63 ? 0ull : (P + (1ull << (sh - 1))) >> sh;
    return (bits >> 31) ? -(long long)r : (long long)r;
}

// A face is dropped (FACE_INVALID) when a UV is NaN or outside [-1, 2] or an
// index is out of range.
__device__ __forceinline__ bool face_ok(const float *__restrict__ uv, const int32_t *__restrict__ F, int64_t f,
                                        int64_t nv, int32_t id[3], float u[3], float v[3]) {
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        id[k] = F[3 * f + k];
        u[k] = uv[6 * f + 2 * k];
        v[k] = uv[6 * f + 2 * k + 1];
        if (!(u[k] >= -1.f && u[k] <= 2.f && v[k] >= -1.f && v[k] <= 2.f)) ok = false;
        if (id[k] < 0 || id[k] >= nv) ok = false;
    }
    return ok;
}

// UV side of the face set-up, all the raster needs: the snapped corners and
// twice the signed snapped area (a dropped face gets zeros, so it rasterises
// nothing).
__global__ void k_uv_setup(const float *__restrict__ uv, const int32_t *__restrict__ F, int64_t nf, int64_t nv,
                           int W, int H, int4 *__restrict__ uvfix, unsigned *__restrict__ status) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int32_t id[3];
    float u[3], v[3];
    if (!face_ok(uv, F, f, nv, id, u, v)) {
        atomicOr(status, AGS_BAD_UV);
        uvfix[2 * f] = make_int4(0, 0, 0, 0);
        uvfix[2 * f + 1] = make_int4(0, 0, 0, 0);
        return;
    }
    long long X[3], Y[3];
    for (int k = 0; k < 3; ++k) {
        X[k] = snap_exact(u[k], W);
        Y[k] = snap_exact(v[k], H);
    }
    long long a2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
    uvfix[2 * f] = make_int4((int)X[0], (int)Y[0], (int)X[1], (int)Y[1]);
    uvfix[2 * f + 1] = make_int4((int)X[2], (int)Y[2], (int)(unsigned)(a2 & 0xffffffffll), (int)(a2 >> 32));
}

// Frame side of the face set-up (needs the vertex normals): per face the
// reliability flag and the corner tangent frames from the snapped UVs.
__global__ void k_tangents(const float *__restrict__ uv, const int32_t *__restrict__ F, int64_t nf, int64_t nv,
                           const int4 *__restrict__ uvfix, const float4 *__restrict__ lpos,
                           const float4 *__restrict__ lnrm, int4 *__restrict__ lface, float4 *__restrict__ ltan) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int32_t id[3];
    float u[3], v[3];
    if (!face_ok(uv, F, f, nv, id, u, v)) {
        lface[f] = make_int4(0, 0, 0, FACE_INVALID);
        for (int k = 0; k < 3; ++k) ltan[3 * f + k] = make_float4(1.f, 0.f, 0.f, 1.f);
        return;
    }
    const int4 q0 = uvfix[2 * f], q1 = uvfix[2 * f + 1];
    const long long X[3] = {q0.x, q0.z, q1.x}, Y[3] = {q0.y, q0.w, q1.y};
    const long long a2 = (long long)(((unsigned long long)(unsigned)q1.w << 32) | (unsigned long long)(unsigned)q1.z);
    int flags = (a2 <= 13 && a2 >= -13) ? FACE_DEGEN : 0;
    float3 p0 = f3(lpos[id[0]]), p1 = f3(lpos[id[1]]), p2 = f3(lpos[id[2]]);
    float3 l1, l2;
    float3 h1 = exact_edge_hi(p1, p0, l1), h2 = exact_edge_hi(p2, p0, l2);
    float du1 = (float)(X[1] - X[0]), dv1 = (float)(Y[1] - Y[0]);
    float du2 = (float)(X[2] - X[0]), dv2 = (float)(Y[2] - Y[0]);
    float sg = a2 < 0 ? -1.f : 1.f;
    // dp/du and dp/dv of the affine UV map, up to the positive factor 1/|a2|
    // (snapped UV deltas are exact integers; edges are exact hi + lo pairs)
    float3 Tf = lincomb_edges(dv2, h1, l1, dv1, h2, l2) * sg;
    float3 Bf = lincomb_edges(du1, h2, l2, du2, h1, l1) * sg;
    float3 T[3];
    for (int k = 0; k < 3; ++k) {
        float3 n = f3(lnrm[id[k]]);
        float3 t = Tf - n * dot3(Tf, n);
        if (!flags && dot3(t, t) > 0.f) {
            T[k] = normalize3(t);
        } else {
            flags |= FACE_DEGEN;
            // Duff et al. 2017 orthonormal basis, FP64 (bookkeeping only:
            // unreliable texels output (0,0,1))
            double nx = n.x, ny = n.y, nz = n.z;
            double s = nz >= 0.0 ? 1.0 : -1.0;
            double a = -1.0 / (s + nz);
            double b = nx * ny * a;
            double tx = 1.0 + s * nx * nx * a, ty = s * b, tz = -s * nx;
            double l = sqrt(tx * tx + ty * ty + tz * tz);
            T[k] = make_float3((float)(tx / l), (float)(ty / l), (float)(tz / l));
        }
    }
    float hs = dot3(cross3(f3(lnrm[id[0]]), Tf), Bf);
    float w = hs < 0.f ? -1.f : 1.f;
    for (int k = 0; k < 3; ++k) ltan[3 * f + k] = make_float4(T[k].x, T[k].y, T[k].z, w);
    lface[f] = make_int4(id[0], id[1], id[2], flags);
}

// Snapped UV triangle: coordinates fit in 24 bits, so differences fit in 32
// and every product is one 32x32->64 multiply.
struct UvTri {
    int X[3], Y[3];
    long long a2;
};

__device__ __forceinline__ UvTri load_uvtri(const int4 *uvfix, int64_t f) {
    int4 a = uvfix[2 * f], b = uvfix[2 * f + 1];
    UvTri t;
    t.X[0] = a.x; t.Y[0] = a.y; t.X[1] = a.z; t.Y[1] = a.w; t.X[2] = b.x; t.Y[2] = b.y;
    t.a2 = (long long)(((unsigned long long)(unsigned)b.w << 32) | (unsigned long long)(unsigned)b.z);
    return t;
}

__device__ __forceinline__ long long mulw(int a, int b) { return (long long)a * (long long)b; }

__device__ __forceinline__ long long orient2(int ax, int ay, int bx, int by, int cx, int cy) {
    return mulw(bx - ax, cy - ay) - mulw(by - ay, cx - ax);
}

// e[i] = orient2(P[i+1], P[i+2], c): twice the signed area opposite vertex i
__device__ __forceinline__ bool uv_inside(const UvTri &t, int cx, int cy, long long e[3]) {
    e[0] = orient2(t.X[1], t.Y[1], t.X[2], t.Y[2], cx, cy);
    e[1] = orient2(t.X[2], t.Y[2], t.X[0], t.Y[0], cx, cy);
    e[2] = orient2(t.X[0], t.Y[0], t.X[1], t.Y[1], cx, cy);
    if (t.a2 > 0) return e[0] >= 0 && e[1] >= 0 && e[2] >= 0;
    return e[0] <= 0 && e[1] <= 0 && e[2] <= 0;
}

// Open interiors of the triangle and the texel square centred on c (side
// 256) intersect iff no separating axis exists among the square's axes and
// the triangle's edge normals.  Along the normal of edge (P[k], P[k+1]),
// measured from P[k]: the triangle spans [min(0,a2), max(0,a2)] and the
// square spans e_k(c) -/+ 128 (|dx| + |dy|), where e_k(c) = e[(k+2)%3] is the
// edge function already evaluated at the centre.
__device__ __forceinline__ bool uv_overlap(const UvTri &t, int cx, int cy, const long long e[3]) {
    int mnx = min(t.X[0], min(t.X[1], t.X[2])), mxx = max(t.X[0], max(t.X[1], t.X[2]));
    int mny = min(t.Y[0], min(t.Y[1], t.Y[2])), mxy = max(t.Y[0], max(t.Y[1], t.Y[2]));
    if (mxx <= cx - 128 || mnx >= cx + 128 || mxy <= cy - 128 || mny >= cy + 128) return false;
    long long lo = min(0ll, t.a2), hi = max(0ll, t.a2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int b = k == 2 ? 0 : k + 1;
        long long r = 128ll * (long long)(abs(t.X[b] - t.X[k]) + abs(t.Y[b] - t.Y[k]));
        long long ek = e[k == 0 ? 2 : k - 1];
        if (ek + r <= lo || ek - r >= hi) return false;
    }
    return true;
}

// floor(d^2 * 65536) for the distance from (cx,cy) to edge k (snapped units),
// ~0 when farther than one texel; *param = closest point's edge parameter.
__device__ unsigned long long edge_qdist(const UvTri &t, int k, int cx, int cy, float *param) {
    int a = k, b = k == 2 ? 0 : k + 1;
    int wx = cx - t.X[a], wy = cy - t.Y[a];
    int dx = t.X[b] - t.X[a], dy = t.Y[b] - t.Y[a];
    long long wd = mulw(wx, dx) + mulw(wy, dy), dd = mulw(dx, dx) + mulw(dy, dy);
    unsigned __int128 num, den;
    if (dd == 0 || wd <= 0) {
        num = (unsigned __int128)(unsigned long long)(mulw(wx, wx) + mulw(wy, wy));
        den = 1;
        *param = 0.f;
    } else if (wd >= dd) {
        int ux = cx - t.X[b], uy = cy - t.Y[b];
        num = (unsigned __int128)(unsigned long long)(mulw(ux, ux) + mulw(uy, uy));
        den = 1;
        *param = 1.f;
    } else {
        long long cr = mulw(wx, dy) - mulw(wy, dx);
        unsigned long long ac = (unsigned long long)(cr < 0 ? -cr : cr);
        num = (unsigned __int128)ac * ac;
        den = (unsigned __int128)(unsigned long long)dd;
        *param = (float)wd / (float)dd;
    }
    if (num > den * 65536u) return KEY_NONE;
    return (unsigned long long)((num * 65536u) / den);
}

__device__ unsigned long long tri_qdist(const UvTri &t, int cx, int cy, int *be, float *bp) {
    unsigned long long best = KEY_NONE;
    *be = -1;
    *bp = 0.f;
    for (int k = 0; k < 3; ++k) {
        float p;
        unsigned long long q = edge_qdist(t, k, cx, cy, &p);
        if (q < best) { best = q; *be = k; *bp = p; }
    }
    return best;
}

__device__ __forceinline__ int floordiv256(int a) { return a >> 8; }  // arithmetic shift = floor

// one warp per face: every texel within one texel of the face's UV bbox
// (a dropped face has zero snapped area and is skipped like a zero-area one)
__global__ void k_raster(const int4 *__restrict__ uvfix, int64_t nf, int W, int H,
                         unsigned long long *__restrict__ keys) {
    int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (f >= nf) return;
    UvTri t = load_uvtri(uvfix, f);
    if (t.a2 == 0) return;
    int mnx = min(t.X[0], min(t.X[1], t.X[2])), mxx = max(t.X[0], max(t.X[1], t.X[2]));
    int mny = min(t.Y[0], min(t.Y[1], t.Y[2])), mxy = max(t.Y[0], max(t.Y[1], t.Y[2]));
    int x0 = max(0, floordiv256(mnx) - 1), x1 = min(W - 1, floordiv256(mxx) + 1);
    int y0 = max(0, floordiv256(mny) - 1), y1 = min(H - 1, floordiv256(mxy) + 1);
    if (x0 > x1 || y0 > y1) return;
    const unsigned nx = (unsigned)(x1 - x0 + 1);
    const unsigned cnt = nx * (unsigned)(y1 - y0 + 1);   // bbox area <= 16384^2 < 2^32
    for (unsigned idx = lane; idx < cnt; idx += 32) {
        unsigned row = idx / nx;
        int x = x0 + (int)(idx - row * nx), y = y0 + (int)row;
        int cx = 256 * x + 128, cy = 256 * y + 128;
        long long e[3];
        unsigned long long key = KEY_NONE;
        if (uv_inside(t, cx, cy, e)) {
            key = (unsigned long long)f;
        } else if (uv_overlap(t, cx, cy, e)) {
            int be;
            float bp;
            unsigned long long q = tri_qdist(t, cx, cy, &be, &bp);
            if (q != KEY_NONE) key = KEY_CONS | (q << 31) | (unsigned long long)f;
        }
        if (key != KEY_NONE) atomicMin(&keys[(size_t)y * W + x], key);
    }
}

// Texels in tile order (row-major tiles of 2^lw x 2^lh texels, row-major
// inside a tile), so a warp's 32 consecutive rays come from one patch of the
// atlas; the tile shape is a launch option (ag_opts.ray_tile).
__global__ void __launch_bounds__(256) k_resolve(const unsigned long long *__restrict__ keys,
                                                 const int4 *__restrict__ uvfix, int W, int H, int lw, int lh,
                                                 int32_t *__restrict__ face_map, float *__restrict__ aux_bary,
                                                 int4 *__restrict__ rays, long long *__restrict__ n_rays) {
    __shared__ int s_warp[8];
    __shared__ long long s_base;
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // texel count <= 16384^2 = 2^28: 32-bit index math throughout
    const unsigned g = blockIdx.x * 256u + (unsigned)tid;
    const unsigned tile = g >> (lw + lh);
    const int within = (int)(g & ((1u << (lw + lh)) - 1u));
    const unsigned ntx = (unsigned)((W + (1 << lw) - 1) >> lw);
    const unsigned ty = tile / ntx, tx = tile - ty * ntx;
    const int x = (int)(tx << lw) + (within & ((1 << lw) - 1)), y = (int)(ty << lh) + (within >> lw);
    bool valid = x < W && y < H;
    const size_t tix = (size_t)y * W + x;
    unsigned long long key = valid ? keys[tix] : KEY_NONE;
    bool has = key != KEY_NONE;
    int4 rec = make_int4(0, 0, 0, 0);
    if (has) {
        int f = (int)(key & 0x7fffffffull);
        UvTri t = load_uvtri(uvfix, f);
        int cx = 256 * x + 128, cy = 256 * y + 128;
        float b[3];
        if (!(key & KEY_CONS)) {
            long long e[3];
            uv_inside(t, cx, cy, e);
            float inv = 1.0f / (float)t.a2;
            b[1] = (float)e[1] * inv;
            b[2] = (float)e[2] * inv;
        } else {
            int be;
            float bp;
            tri_qdist(t, cx, cy, &be, &bp);
            float bb[3] = {0.f, 0.f, 0.f};
            bb[be] = 1.f - bp;
            bb[(be + 1) % 3] = bp;
            b[1] = bb[1];
            b[2] = bb[2];
        }
        b[0] = 1.f - b[1] - b[2];
        rec = make_int4((int)tix, f, __float_as_int(b[1]), __float_as_int(b[2]));
        if (aux_bary) {
            aux_bary[3 * tix] = b[0];
            aux_bary[3 * tix + 1] = b[1];
            aux_bary[3 * tix + 2] = b[2];
        }
    }
    if (valid) {
        face_map[tix] = has ? (int)(key & 0x7fffffffull) : -1;
        if (aux_bary && !has) {
            aux_bary[3 * tix] = 0.f;
            aux_bary[3 * tix + 1] = 0.f;
            aux_bary[3 * tix + 2] = 0.f;
        }
    }
    unsigned bal = __ballot_sync(0xffffffffu, has);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int w = 0; w < 8; ++w) { int c = s_warp[w]; s_warp[w] = run; run += c; }
        s_base = run ? (long long)atomicAdd((unsigned long long *)n_rays, (unsigned long long)run) : 0;
    }
    __syncthreads();
    if (has) rays[s_base + s_warp[warp] + __popc(bal & ((1u << lane) - 1u))] = rec;
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

cudaError_t launch_uv_setup(const float *luv, const int32_t *lfaces, int64_t nf, int64_t nv, int W, int H,
                            int4 *uvfix, unsigned *status, cudaStream_t s) {
    k_uv_setup<<<grid_for(nf, 128), 128, 0, s>>>(luv, lfaces, nf, nv, W, H, uvfix, status);
    return cudaGetLastError();
}

cudaError_t launch_tangents(const float *luv, const int32_t *lfaces, int64_t nf, int64_t nv, const int4 *uvfix,
                            const float4 *lpos, const float4 *lnrm, int4 *lface, float4 *ltan, cudaStream_t s) {
    k_tangents<<<grid_for(nf, 128), 128, 0, s>>>(luv, lfaces, nf, nv, uvfix, lpos, lnrm, lface, ltan);
    return cudaGetLastError();
}

cudaError_t launch_face_setup(const float *luv, const int32_t *lfaces, int64_t nf, int64_t nv, int W, int H,
                              const float4 *lpos, const float4 *lnrm, int4 *lface, float4 *ltan, int4 *uvfix,
                              unsigned *status, cudaStream_t s) {
    cudaError_t e = launch_uv_setup(luv, lfaces, nf, nv, W, H, uvfix, status, s);
    if (e != cudaSuccess) return e;
    return launch_tangents(luv, lfaces, nf, nv, uvfix, lpos, lnrm, lface, ltan, s);
}

cudaError_t launch_raster(const int4 *uvfix, int64_t nf, int W, int H, unsigned long long *keys, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * (size_t)W * H, s);
    if (e != cudaSuccess) return e;
    k_raster<<<grid_for(nf * 32, 256), 256, 0, s>>>(uvfix, nf, W, H, keys);
    return cudaGetLastError();
}

void ray_tile_shape(int ray_tile, int *lw, int *lh) {
    switch (ray_tile) {
        case AG_TILE_16x16: *lw = 4; *lh = 4; break;
        case AG_TILE_32x8: *lw = 5; *lh = 3; break;
        case AG_TILE_4x4: *lw = 2; *lh = 2; break;
        default: *lw = 3; *lh = 3; break;  // AG_TILE_8x8
    }
}

cudaError_t launch_resolve(const unsigned long long *keys, const int4 *uvfix, int W, int H, int ray_tile,
                           int32_t *face_map, float *aux_bary, int4 *rays, long long *n_rays, cudaStream_t s) {
    int lw, lh;
    ray_tile_shape(ray_tile, &lw, &lh);
    long long ntiles = (long long)((W + (1 << lw) - 1) >> lw) * ((H + (1 << lh) - 1) >> lh);
    k_resolve<<<grid_for(ntiles << (lw + lh), 256), 256, 0, s>>>(keys, uvfix, W, H, lw, lh, face_map, aux_bary, rays,
                                                                n_rays);
    return cudaGetLastError();
}

}  // namespace ag
