// Internal declarations of the B300 normal baker (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "ag.h"

// ------------------------------------------------------------------ status
// Bits of the per-device status word written by kernels (atomicOr).
enum : unsigned {
    AGS_STEP_CAP = 1u,      // a ray exceeded ag_opts.max_steps
    AGS_STACK = 2u,         // a traversal stack overflowed
    AGS_BAD_FACE = 4u,      // a face index was out of range (build)
    AGS_BAD_UV = 8u,        // a UV was NaN or outside [-1, 2] (bake; face dropped)
};

namespace ag {

// ------------------------------------------------------------------ host error plumbing
ag_status set_error(ag_status s, const char *fmt, ...);
ag_status cuda_error(cudaError_t e, const char *what);
#define AG_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ag::cuda_error(e_, #call);   \
    } while (0)
#define AG_CUDA_LAUNCH(what)                                       \
    do {                                                           \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return ag::cuda_error(e_, what);    \
    } while (0)

// ------------------------------------------------------------------ side streams
// N_SIDE library-owned non-blocking streams per device, created on first use
// and kept for the process; fork_to makes the first n_used of them wait for
// what is enqueued on s so far, join_from makes s wait for what they hold.
constexpr int N_SIDE = 8;
cudaError_t side_streams(int dev, cudaStream_t **out);
struct EventSet {   // events of one call's edges, destroyed with it
    std::vector<cudaEvent_t> ev;
    ~EventSet();
    cudaError_t make(cudaEvent_t *e);
};
cudaError_t fork_to(cudaStream_t s, cudaStream_t *side, int n_used, EventSet &es);
cudaError_t join_from(cudaStream_t s, cudaStream_t *side, int n_used, EventSet &es);

unsigned *device_status_word(int device);      // 1 word per device, zero-initialised
cudaMemPool_t device_pool(int device);         // library-private stream-ordered pool
int device_sm_count(int device);

// stream-ordered scratch from the private pool
struct Scratch {
    cudaStream_t stream;
    int device;
    void *ptrs[48];
    int n = 0;
    explicit Scratch(cudaStream_t s, int dev) : stream(s), device(dev) {}
    cudaError_t alloc(void **p, size_t bytes);
    ~Scratch();
};

// ------------------------------------------------------------------ BVH layouts
// 80-byte node: origin, per-axis power-of-two scale, and 8 child boxes as
// 8-bit offsets on that grid, rounded outward at build time so the decoded
// box always contains the exact FP32 child box.
struct __align__(16) QNode {
    float ox, oy, oz;
    uint8_t ex, ey, ez, nchild;   // scale = 2^(e-127) (float exponent bits)
    uint32_t child_base;          // index of the first internal child
    uint32_t tri_base;            // first triangle record of the leaf children
    uint8_t meta[8];              // per child slot, see meta_* below
    uint8_t qlox[8], qloy[8], qloz[8], qhix[8], qhiy[8], qhiz[8];
};
static_assert(sizeof(QNode) == 80, "QNode must be 80 bytes");

// 208-byte node with exact FP32 child boxes (precision-study layout).
struct __align__(16) FNode {
    uint32_t child_base, tri_base;
    uint8_t meta[8];
    float lox[8], loy[8], loz[8], hix[8], hiy[8], hiz[8];
};
static_assert(sizeof(FNode) == 208, "FNode must be 208 bytes");

// meta byte: 0 = empty slot; internal child: 0x80 | rank among internal
// children (node = child_base + rank); leaf child: (count << 5) | offset,
// count in 1..3, offset in 0..23 (records tri_base + offset ...).
__host__ __device__ inline bool meta_internal(uint8_t m) { return (m & 0x80u) != 0; }
__host__ __device__ inline bool meta_leaf(uint8_t m) { return m != 0 && (m & 0x80u) == 0; }
__host__ __device__ inline int meta_rank(uint8_t m) { return m & 0x7f; }
__host__ __device__ inline int meta_count(uint8_t m) { return (m >> 5) & 3; }
__host__ __device__ inline int meta_offset(uint8_t m) { return m & 31; }

// Leaves hold one triangle. With leaves tested at their node, one triangle
// per leaf (a child box per triangle) measured fastest for both queries on
// the 2.1M-triangle, 2048^2 bake: ray trace 0.78-0.80 ms at 1, 0.82-0.83 at 2,
// 0.85 at 3; closest-point trace 2.51-2.54 ms at 1, 2.74-2.79 at 2, 2.86 at 3;
// for a tree of 456k instead of 308k nodes and a build 0.05 ms slower.
// (Before leaves were tested at their node, 2 had measured best.)
#ifndef AG_LEAF_MAX
#define AG_LEAF_MAX 1
#endif
constexpr int LEAF_MAX = AG_LEAF_MAX;

// Triangle record (48 B, leaf order): three float4 (vertex xyz, vertex index
// bits in .w).  The original triangle id is kept in a parallel array.

// traversal stack entry reference: bit31 leaf flag; leaf: bits 29..30 =
// count-1, bits 0..28 = first record; internal: node index.
__host__ __device__ inline uint32_t ref_leaf(uint32_t first, int count) {
    return 0x80000000u | ((uint32_t)(count - 1) << 29) | first;
}
__host__ __device__ inline bool ref_is_leaf(uint32_t r) { return (r & 0x80000000u) != 0; }
__host__ __device__ inline uint32_t ref_first(uint32_t r) { return r & 0x1fffffffu; }
__host__ __device__ inline int ref_count(uint32_t r) { return (int)((r >> 29) & 3u) + 1; }

}  // namespace ag

struct ag_bvh {
    uint64_t magic;
    int device;
    int layout;
    int64_t n_tris, n_verts, n_nodes;
    void *nodes;           // QNode[] or FNode[]
    float4 *tris;          // [n_tris*3]
    int32_t *tri_ids;      // [n_tris]
    float4 *vnormals;      // [n_verts] (xyz unit, w = 0)
    float lo[3], hi[3];
    float diam;
    int max_depth;
    float build_ms;
    // the build's summary (device) and its events; the scalars above except
    // n_tris and n_verts are valid once `ready` (ag::bvh_ready reads them)
    void *d_info;
    cudaEvent_t ev_start, ev_done;
    bool ready;
};
constexpr uint64_t AG_BVH_MAGIC = 0x4147425648414e44ull;

namespace ag {

// the build's summary (node count, depth, scene box, build time): waits for
// the build the first time, then reads the handle's copy
ag_status bvh_ready(ag_bvh *h);
// largest |coordinate| of the high mesh's box, the rounding slack of the
// FP32-node traversal; the 8-bit-node traversal does not use it, so for such
// a tree this returns 0 without waiting for the build
ag_status scene_abs_for(ag_bvh *h, float *out);
// work enqueued on s after this waits for the handle's build (an
// asynchronous build may run on another stream); nothing once the build's
// summary has been read, nor while s is being captured (the capture must
// order the build itself, as every stream-ordered call does)
cudaError_t wait_build(const ag_bvh *h, cudaStream_t s);

// ------------------------------------------------------------------ per-asset bake job
// Everything the trace needs for one asset (device-resident table).
struct TraceJob {
    const void *nodes;
    const float4 *tris;
    const int32_t *tri_ids;
    const float4 *hnormals;
    const float4 *lpos;     // [V] low positions (w unused)
    const float4 *lnrm;     // [V] low unit vertex normals
    const int4 *lface;      // [F] (i0, i1, i2, flags)
    const float4 *ltan;     // [F*3] per-corner unit tangent, w = handedness
    const int4 *rays;       // this asset's rays: (texel, face, b1 bits, b2 bits)
    float4 *ntsd;           // [H*W] out: tangent-space normal xyz, displacement w
    uint8_t *mask;          // [H*W] out
    int32_t *hit_tri;       // [H*W] optional
    float *hit_t;           // [H*W] optional
    float *g_pos;           // backward: [V*3] unscaled dL/dV via p
    float *g_nrm;           // backward: [V*3] unscaled dL/dn_i
    float *loss_acc;        // backward: [4] sum t^2, sum (1 - n.d), hit count, pad
    long long ray_begin;    // first ray of this asset in the global ray list
    int W, H;
    float max_dist;
    float lambda;
    float scene_abs;        // largest |coordinate| of the high mesh bbox
};

constexpr int FACE_DEGEN = 1;   // lface.w bit: unreliable UVs -> (0,0,1)
constexpr int FACE_INVALID = 2; // lface.w bit: dropped (bad UV)

// ------------------------------------------------------------------ launch helpers (defined per .cu)
// in-place exclusive prefix sum of n unsigned values; *total (device, may be
// NULL) receives the sum; scratch of scan_scratch_bytes(n)
size_t scan_scratch_bytes(int64_t n);
cudaError_t launch_scan_exclusive(unsigned *d, int64_t n, unsigned *total, void *scratch, cudaStream_t s);
// area-weighted vertex normals (deterministic, exact edge differences);
// `given` replaces the derived normals (normalised), acc_out [3nv] receives
// the unnormalised sums, pos [nv] (optional) the positions as float4
size_t vertex_normal_scratch_bytes(int64_t nv, int64_t nf);
cudaError_t launch_vertex_normals(const float *V, const int32_t *F, int64_t nv, int64_t nf,
                                  const float *given, float *acc_out, float4 *nrm, float4 *pos,
                                  void *scratch, cudaStream_t s);
// vertex -> incident faces (CSR, unsorted lists) in the same scratch layout
// as the vertex normals; faces with an out-of-range index are left out
cudaError_t launch_vertex_face_csr(const int32_t *F, int64_t nf, int64_t nv, void *scratch, const unsigned **off,
                                   const int32_t **list, cudaStream_t s);
// face set-up of the low mesh in two parts: the UV part (snapped corners and
// twice the signed snapped area, zeros for a dropped face; all the raster
// needs) and the frame part (needs the vertex normals: face flags and the
// corner tangent frames); launch_face_setup runs both in order
cudaError_t launch_uv_setup(const float *luv, const int32_t *lfaces, int64_t nf, int64_t nv, int W, int H,
                            int4 *uvfix, unsigned *status, cudaStream_t s);
cudaError_t launch_tangents(const float *luv, const int32_t *lfaces, int64_t nf, int64_t nv, const int4 *uvfix,
                            const float4 *lpos, const float4 *lnrm, int4 *lface, float4 *ltan, cudaStream_t s);
cudaError_t launch_face_setup(const float *luv, const int32_t *lfaces, int64_t nf, int64_t nv, int W,
                              int H, const float4 *lpos, const float4 *lnrm, int4 *lface, float4 *ltan,
                              int4 *uvfix, unsigned *status, cudaStream_t s);
cudaError_t launch_raster(const int4 *uvfix, int64_t nf, int W, int H, unsigned long long *keys, cudaStream_t s);
cudaError_t launch_resolve(const unsigned long long *keys, const int4 *uvfix, int W, int H,
                           int ray_tile, int32_t *face_map, float *aux_bary, int4 *rays,
                           long long *n_rays, cudaStream_t s);

struct TraceLaunch {
    TraceJob job0;              // the job of a single-asset launch (n_jobs == 1)
    const TraceJob *jobs;       // device table (n_jobs > 1)
    const long long *job_begin; // device [n_jobs+1] exclusive ray offsets (n_jobs > 1)
    int n_jobs;
    const long long *n_rays_dev; // device total ray count
    unsigned long long *ray_counter;
    unsigned *status;
    int max_steps;
    unsigned long long *counters;  // non-NULL -> counting build
    int stack_cap;              // counting build: usable traversal stack entries (0 = all)
    int layout;
    int schedule;
    int query;                  // AG_QUERY_RAY / AG_QUERY_CLOSEST
    int block_size, blocks_per_sm;
    bool backward;
};
// ray query (trace.cu); dispatches to launch_closest for AG_QUERY_CLOSEST
cudaError_t launch_trace(const TraceLaunch &L, cudaStream_t s);
// closest-point query, forward only (closest.cu)
cudaError_t launch_closest(const TraceLaunch &L, cudaStream_t s);
// UV-space backprojection (backproject.cu): per-view depth / point / edge
// maps of the mesh of L.job0, and the blended texture of the ray texels
int render_chunk_views(int n_views, int w, int h);
size_t render_head_bytes(int n_views);
size_t render_scratch_bytes(int n_views, int w, int h, bool raster);
cudaError_t launch_render_views(const TraceLaunch &L, int n_tris, const float *h_cams, int n_views, int w, int h,
                                float edge_tol, bool raster, float *depth, float *points, uint8_t *edge, void *scratch,
                                cudaStream_t s);
size_t backproject_scratch_bytes(int n_views, int w, int h, int filter);
cudaError_t launch_backproject(const float4 *lpos, const float4 *lnrm, const int4 *lface, const float *luv,
                               const int4 *rays, const long long *n_rays, int W, int H, const float *h_cams,
                               const float *h_centres, const float *h_logw, int n_views, const uint8_t *images, const float *depth,
                               const uint8_t *edge, int w, int h, float alpha, float eps, float depth_tol, int filter,
                               float lod_bias, int max_taps, float sharpen, float4 *texture, float *incidence,
                               void *scratch, cudaStream_t s);
// distance from n points to the mesh of L.job0 (nodes, tris, tri_ids, scene_abs), -1 beyond max_dist
cudaError_t launch_point_distance(const TraceLaunch &L, const float *pts, long long n, float max_dist, float *dist,
                                  int32_t *tri, cudaStream_t s);
// "baked mean" angle per sample point of the low mesh of L.job0 (closest.cu)
cudaError_t launch_map_error(const TraceLaunch &L, const uint8_t *rgba, const float *luv, int64_t n_lfaces,
                             const int32_t *sface, const float *sbary, long long n, float *angle, cudaStream_t s);

cudaError_t launch_finalize(const float4 *ntsd, const int32_t *face_map, int W, int H, int gutter,
                            int disp_fp16, uint8_t *rgba, uint8_t *mask, void *disp,
                            float *aux_nts, float *aux_disp, int32_t *aux_hit_tri, float *aux_hit_t,
                            cudaStream_t s);

cudaError_t launch_backward_finish(const float4 *lpos, const int4 *lface, int64_t nv, int64_t nf,
                                   const float *acc_nrm /*[V*3] unnormalised normal sums*/,
                                   float *g_pos, const float *g_nrm, float *g_a,
                                   const float *loss_acc, float lambda, float *d_loss,
                                   float *d_grad, cudaStream_t s);

}  // namespace ag

// ------------------------------------------------------------------ device math
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) {
    float l2 = dot3(a, a);
    return l2 > 0.f ? a * (1.0f / sqrtf(l2)) : a;
}
