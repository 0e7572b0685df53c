// Output stage (Sec. 6.4: the RGB8 encoding and the dilation across UV
// seams): `gutter` Jacobi dilation passes run in shared memory on a
// 32x8 output tile with a halo of `gutter` texels, then every texel of the
// tile is encoded (RGBA8, binary16/float32 displacement) in the same pass.
// Also the final reductions of the backward pass.
#include "ag_internal.cuh"

#include <algorithm>

namespace ag {
namespace {

// RGB8 code of c in [-1,1]: 128 + round_half_away(127 c) (codes 1..255,
// 128 = 0, so the frequent value c = 0 is in the middle of a code rather than
// on a code boundary); every step one FP32 rounding (no contraction).
__device__ __forceinline__ unsigned enc8(float c) {
    float v = fminf(fmaxf(c, -1.f), 1.f);
    float r = __fmul_rn(v, 127.f);
    float q = r >= 0.f ? floorf(__fadd_rn(r, 0.5f)) : -floorf(__fadd_rn(-r, 0.5f));
    return (unsigned)(128 + (int)q);
}

// One CTA = a TW x TH output tile; the tile plus a G-texel halo is staged in
// shared memory by asynchronous copies (no registers held for loads in
// flight), G Jacobi passes run there in place (the valid region shrinks by
// one texel per pass), then the TW x TH centre is encoded.  A texel filled in
// pass p is tagged p + 1 (a ray texel 0, an empty or outside one a large
// tag), and pass p reads only texels with a tag below p + 1, those filled
// before it: one buffer serves every pass with no copy between them, and a
// neighbour's weight is one compare.  The passes run
// over a list of the tile's empty texels, so the lanes of a warp all do the
// same neighbour sum rather than splitting between filled and empty texels.
// G, TW, TH are compile time so the cell loops need no integer division.
constexpr int RAY = 0, EMPTY = 0x7ffffffe, OUTSIDE = 0x7fffffff;   // texel tags (dilated in pass p: p + 1)

__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes16) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gmem) : "memory");
}

template <int G, int TW, int TH>
__global__ void __launch_bounds__(256) k_finalize(const float4 *__restrict__ ntsd, const int32_t *__restrict__ face_map,
                                                  int W, int H, int disp_fp16, uchar4 *__restrict__ rgba,
                                                  uint8_t *__restrict__ mask, void *__restrict__ disp,
                                                  float *__restrict__ aux_nts, float *__restrict__ aux_disp,
                                                  int32_t *__restrict__ aux_hit_tri, float *__restrict__ aux_hit_t) {
    constexpr int BW = TW + 2 * G, BH = TH + 2 * G, CELLS = BW * BH;
    static_assert(CELLS < 65536, "cell ids are 16-bit");
    __shared__ float4 sv[CELLS];
    __shared__ int32_t sf[CELLS];          // the face map, then the texel tag
    __shared__ uint16_t todo[CELLS];       // empty texels off the tile's rim
    __shared__ int n_todo;
    const int x0 = blockIdx.x * TW - G, y0 = blockIdx.y * TH - G;
    if (threadIdx.x == 0) n_todo = 0;
    // staging: every cell's face entry and value
    for (int i = threadIdx.x; i < CELLS; i += 256) {
        const int lx = i % BW, ly = i / BW;
        const int x = x0 + lx, y = y0 + ly;
        if (x >= 0 && y >= 0 && x < W && y < H) {
            const size_t t = (size_t)y * W + x;
            cp_async(&sf[i], &face_map[t], 0);
            cp_async(&sv[i], &ntsd[t], 1);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();   // n_todo cleared
    // tags (each thread the cells it copied); texels that hold no value get
    // a zero value, so the neighbour sums below can weight every neighbour
    const int lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < CELLS; i0 += 256) {
        const int i = i0 + (int)threadIdx.x;
        bool add = false;
        if (i < CELLS) {
            const int lx = i % BW, ly = i / BW;
            const int x = x0 + lx, y = y0 + ly;
            const bool in = x >= 0 && y >= 0 && x < W && y < H;
            const int f = !in ? OUTSIDE : (sf[i] >= 0 ? RAY : EMPTY);
            sf[i] = f;
            if (f != RAY) sv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            add = f == EMPTY && lx > 0 && ly > 0 && lx < BW - 1 && ly < BH - 1;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, add);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&n_todo, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (add) todo[base + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)i;
    }
    __syncthreads();
    const int nt = n_todo;
#pragma unroll 1
    for (int p = 0; p < G; ++p) {
        const int tag = p + 1;
        for (int j = threadIdx.x; j < nt; j += 256) {
            const int i = todo[j];
            if (sf[i] != EMPTY) continue;   // filled by an earlier pass
            float sx = 0.f, sy = 0.f, sz = 0.f, sd = 0.f, cnt = 0.f;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    // ray texels and texels filled by earlier passes (a
                    // texel tagged in this pass, or being tagged, has
                    // weight 0, and its value is not read)
                    const int n = i + dy * BW + dx;
                    const float w = sf[n] < tag ? 1.f : 0.f;
                    const float4 nv = w != 0.f ? sv[n] : make_float4(0.f, 0.f, 0.f, 0.f);
                    sx += w * nv.x; sy += w * nv.y; sz += w * nv.z; sd += w * nv.w;
                    cnt += w;
                }
            if (cnt > 0.f) {
                const float inv = 1.0f / cnt;
                const float3 m = make_float3(sx * inv, sy * inv, sz * inv);
                const float l2 = dot3(m, m);
                const float3 nn = l2 > 0.f ? m * (1.0f / sqrtf(l2)) : make_float3(0.f, 0.f, 1.f);
                sv[i] = make_float4(nn.x, nn.y, nn.z, sd * inv);
                sf[i] = tag;
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < TW * TH; i += blockDim.x) {
        int ox = i % TW, oy = i / TW;
        int x = blockIdx.x * TW + ox, y = blockIdx.y * TH + oy;
        if (x >= W || y >= H) continue;
        size_t t = (size_t)y * W + x;
        float4 v = sv[(oy + G) * BW + ox + G];
        const int f = sf[(oy + G) * BW + ox + G];
        const bool filled = f < EMPTY;
        if (!filled) v = make_float4(0.f, 0.f, 1.f, 0.f);
        rgba[t] = make_uchar4((unsigned char)enc8(v.x), (unsigned char)enc8(v.y), (unsigned char)enc8(v.z),
                              filled ? 255 : 0);
        if (disp_fp16) ((__half *)disp)[t] = __float2half_rn(v.w);
        else ((float *)disp)[t] = v.w;
        if (f != RAY) {
            mask[t] = 0;
            if (aux_hit_tri) aux_hit_tri[t] = -1;
            if (aux_hit_t) aux_hit_t[t] = 0.f;
        }
        if (aux_nts) {
            aux_nts[3 * t] = v.x;
            aux_nts[3 * t + 1] = v.y;
            aux_nts[3 * t + 2] = v.z;
        }
        if (aux_disp) aux_disp[t] = v.w;
    }
}

// dL/da_i = (I - n n^T) g_n / |a_i| (a_i: unnormalised area-weighted normal sum)
__global__ void k_bwd_vertex(const float *__restrict__ acc, const float *__restrict__ g_nrm, int64_t nv,
                             float *__restrict__ g_a) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    float3 a = make_float3(acc[3 * i], acc[3 * i + 1], acc[3 * i + 2]);
    float al = sqrtf(dot3(a, a));
    float3 r = make_float3(0.f, 0.f, 0.f);
    if (al > 0.f) {
        float3 n = a * (1.0f / al);
        float3 g = make_float3(g_nrm[3 * i], g_nrm[3 * i + 1], g_nrm[3 * i + 2]);
        r = (g - n * dot3(n, g)) * (1.0f / al);
    }
    g_a[3 * i] = r.x;
    g_a[3 * i + 1] = r.y;
    g_a[3 * i + 2] = r.z;
}

// a_i = sum over faces of (v1 - v0) x (v2 - v0): scatter the face cross-product adjoint
__global__ void k_bwd_face(const float4 *__restrict__ lpos, const int4 *__restrict__ lface, int64_t nf,
                           const float *__restrict__ g_a, float *__restrict__ g_pos) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int4 fi = lface[f];
    if (fi.w & FACE_INVALID) return;
    int id[3] = {fi.x, fi.y, fi.z};
    float3 g = make_float3(0.f, 0.f, 0.f);
    for (int k = 0; k < 3; ++k) g = g + make_float3(g_a[3 * id[k]], g_a[3 * id[k] + 1], g_a[3 * id[k] + 2]);
    float3 p0 = f3(lpos[id[0]]), p1 = f3(lpos[id[1]]), p2 = f3(lpos[id[2]]);
    float3 e1 = p1 - p0, e2 = p2 - p0;
    float3 g1 = cross3(e2, g), g2 = cross3(g, e1);
    atomicAdd(&g_pos[3 * id[1]], g1.x); atomicAdd(&g_pos[3 * id[1] + 1], g1.y); atomicAdd(&g_pos[3 * id[1] + 2], g1.z);
    atomicAdd(&g_pos[3 * id[2]], g2.x); atomicAdd(&g_pos[3 * id[2] + 1], g2.y); atomicAdd(&g_pos[3 * id[2] + 2], g2.z);
    atomicAdd(&g_pos[3 * id[0]], -(g1.x + g2.x));
    atomicAdd(&g_pos[3 * id[0] + 1], -(g1.y + g2.y));
    atomicAdd(&g_pos[3 * id[0] + 2], -(g1.z + g2.z));
}

__global__ void k_bwd_scale(const float *__restrict__ g_pos, int64_t n3, const float *__restrict__ loss_acc,
                            float lambda, float *__restrict__ d_loss, float *__restrict__ d_grad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float cnt = loss_acc[2];
    float inv = cnt > 0.f ? 1.0f / cnt : 0.f;
    if (d_grad && i < n3) d_grad[i] = g_pos[i] * inv;
    if (d_loss && i == 0) d_loss[0] = (loss_acc[0] + lambda * loss_acc[1]) * inv;
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

template <int G, int TW, int TH>
static cudaError_t finalize_g(const float4 *ntsd, const int32_t *face_map, int W, int H, int disp_fp16, uint8_t *rgba,
                              uint8_t *mask, void *disp, float *aux_nts, float *aux_disp, int32_t *aux_hit_tri,
                              float *aux_hit_t, cudaStream_t s) {
    dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH);
    k_finalize<G, TW, TH><<<grid, 256, 0, s>>>(ntsd, face_map, W, H, disp_fp16, (uchar4 *)rgba, mask, disp, aux_nts,
                                                aux_disp, aux_hit_tri, aux_hit_t);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const float4 *ntsd, const int32_t *face_map, int W, int H, int gutter, int disp_fp16,
                            uint8_t *rgba, uint8_t *mask, void *disp, float *aux_nts, float *aux_disp,
                            int32_t *aux_hit_tri, float *aux_hit_t, cudaStream_t s) {
#define AG_FIN(Gv, TWv, THv) \
    return finalize_g<Gv, TWv, THv>(ntsd, face_map, W, H, disp_fp16, rgba, mask, disp, aux_nts, aux_disp, aux_hit_tri, aux_hit_t, s)
    switch (gutter) {
        case 0: AG_FIN(0, 64, 16);
        case 1: AG_FIN(1, 64, 16);
        case 2: AG_FIN(2, 64, 16);
        case 3: AG_FIN(3, 64, 16);
        case 4: AG_FIN(4, 64, 8);
        case 5: AG_FIN(5, 32, 8);
        case 6: AG_FIN(6, 32, 8);
        case 7: AG_FIN(7, 32, 8);
        default: AG_FIN(8, 32, 8);
    }
#undef AG_FIN
}

cudaError_t launch_backward_finish(const float4 *lpos, const int4 *lface, int64_t nv, int64_t nf, const float *acc_nrm,
                                   float *g_pos, const float *g_nrm, float *g_a, const float *loss_acc, float lambda,
                                   float *d_loss, float *d_grad, cudaStream_t s) {
    if (d_grad) {
        k_bwd_vertex<<<grid_for(nv, 256), 256, 0, s>>>(acc_nrm, g_nrm, nv, g_a);
        k_bwd_face<<<grid_for(nf, 256), 256, 0, s>>>(lpos, lface, nf, g_a, g_pos);
    }
    k_bwd_scale<<<grid_for(std::max<int64_t>(1, 3 * nv), 256), 256, 0, s>>>(g_pos, 3 * nv, loss_acc, lambda, d_loss,
                                                                           d_grad);
    return cudaGetLastError();
}

}  // namespace ag
