/*
 * ag.h - C ABI of the B300 tangent-space normal baker.
 *
 * The operation is the normal-baking stage of AssetGen's geometry
 * post-processing (Sec. 6.4, normal-map baking): the low-poly mesh is
 * rasterised into its own UV space; for every covered texel a ray is cast
 * from the texel's surface point along its interpolated smooth normal against
 * a BVH over the dense high-poly mesh; the closest hit within the distance
 * filter gives a barycentric smooth normal that is written in the texel's
 * tangent frame (RGB8), with a hit mask and a signed displacement, and the
 * map is dilated across UV seams.  Texels of faces with a degenerate UV
 * parameterisation get the neutral normal (0,0,1).
 *
 * Conventions shared by every call
 *  - All mesh and image pointers are DEVICE pointers (CUDA global memory on
 *    the current device) owned by the caller; the library never frees them.
 *  - Vertices are float32 xyz, tightly packed ([n*3]); faces are int32 vertex
 *    indices ([n*3]); UVs are per face corner ([n_faces*3*2], u then v, in
 *    [0,1] atlas units; texel (x,y) has centre ((x+0.5)/W, (y+0.5)/H)).
 *  - Images are row-major, H rows of W texels, texel index y*W + x.
 *  - Every call is ordered on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) and returns after enqueueing work; nothing synchronises
 *    the host except ag_bvh_build (it reads back level sizes while
 *    collapsing the tree) and ag_sync_status.
 *  - Argument errors are detected on the host before any work is enqueued
 *    and returned as AG_ERR_INVALID_ARG / AG_ERR_BAD_HANDLE; the message is
 *    available from ag_last_error() on the calling thread.
 *  - Device-side limits (traversal step cap, traversal stack overflow) set a
 *    per-process status word that ag_sync_status() returns and clears.
 *  - Scratch memory is taken from the device's stream-ordered memory pool
 *    (cudaMallocAsync) and returned on the same stream.
 */
#ifndef AG_H
#define AG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(_WIN32)
#define AG_API __declspec(dllexport)
#else
#define AG_API __attribute__((visibility("default")))
#endif

typedef struct ag_bvh *ag_bvh_t;               /* opaque; owns the BVH's device memory */
typedef struct ag_batch_plan *ag_batch_plan_t; /* opaque; owns scratch + a CUDA graph */
typedef void *ag_stream_t;                     /* a cudaStream_t */

typedef enum {
    AG_OK = 0,
    AG_ERR_INVALID_ARG = 1,     /* bad pointer, size or option; nothing was enqueued */
    AG_ERR_OOM = 2,             /* device or host allocation failed */
    AG_ERR_CUDA = 3,            /* a CUDA runtime call failed (message has the CUDA error) */
    AG_ERR_TRAVERSAL_LIMIT = 4, /* a ray hit the step cap or overflowed its stack (results invalid) */
    AG_ERR_BAD_HANDLE = 5       /* NULL, freed or foreign handle */
} ag_status;

enum { AG_BVH_Q8 = 0, AG_BVH_F32 = 1 };
/* Collapse rules: expand the child with the largest surface area, the largest
 * surface area x triangle count, or the most triangles. */
enum { AG_COLLAPSE_AREA = 0, AG_COLLAPSE_AREA_COUNT = 1, AG_COLLAPSE_COUNT = 2, AG_COLLAPSE_SAH = 3 };

/* Ray-list tile shapes (texels), see ag_opts.ray_tile. */
enum { AG_TILE_8x8 = 0, AG_TILE_16x16 = 1, AG_TILE_32x8 = 2, AG_TILE_4x4 = 3 };

/* Traversal schedules:
 *  AG_SCHED_BATCH  - one ray per thread: a warp takes 32 consecutive rays and
 *                    finishes all of them before taking more;
 *  AG_SCHED_REFILL - one ray per thread: lanes take new rays as they finish
 *                    (in groups of at least 8 idle lanes), shading deferred
 *                    to the refill;
 *  AG_SCHED_COOP2, AG_SCHED_COOP4, AG_SCHED_COOP8 - warp-cooperative: 2, 4
 *                    or 8 lanes share one ray (16, 8 or 4 rays per warp)
 *                    and split each node's eight children among them; hit
 *                    leaves are tested at once by the lanes that own them;
 *                    128-thread blocks (block_size is ignored).  These apply to the forward
 *                    ray bake over 8-bit nodes (AG_BVH_Q8); other launches
 *                    (FP32 nodes, the backward pass, the closest-point
 *                    query) run AG_SCHED_BATCH in their place.
 * Every schedule produces the same bytes; only the speed differs. */
enum { AG_SCHED_AUTO = -1, AG_SCHED_BATCH = 0, AG_SCHED_REFILL = 1, AG_SCHED_COOP4 = 2, AG_SCHED_COOP8 = 3,
       AG_SCHED_COOP2 = 4 };

/* Correspondence queries (ag_opts.query):
 *  AG_QUERY_RAY     - the line from the texel's surface point p along its
 *                     interpolated normal d, closest |t| <= max_dist (both
 *                     directions); displacement = t;
 *  AG_QUERY_CLOSEST - the point x of the high surface nearest to p (Sec. 6.4
 *                     as worded), |x - p| <= max_dist; displacement = |x - p|
 *                     signed by (x - p) . d.  Hit normal, filters and encoding
 *                     are those of the ray query.  One schedule (batch);
 *                     ag_bake_backward supports the ray query only. */
enum { AG_QUERY_RAY = 0, AG_QUERY_CLOSEST = 1 };

/* View rendering (ag_opts.render).  Both give every pixel the first hit of
 * the ray through its centre under the watertight ray-triangle test:
 *  AG_RENDER_RASTER - a z-buffer pass proposes each pixel's triangle, the ray
 *                     test confirms it, and only a pixel whose proposal the
 *                     test rejects (a centre within rounding of an edge) is
 *                     traced through the BVH; a view in which a triangle
 *                     reaches the camera plane is traced whole.  The buffers
 *                     equal AG_RENDER_TRACE's except where two triangles lie
 *                     within rounding of each other along a pixel's ray.
 *  AG_RENDER_TRACE  - every pixel traced through the BVH. */
enum { AG_RENDER_RASTER = 0, AG_RENDER_TRACE = 1 };

/* View sampling of ag_backproject (ag_opts.filter):
 *  AG_FILTER_ANISO    - per texel and view, the image footprint of one texel
 *                       (central differences of the owning face's UV -> position
 *                       map through the projection), its SVD, up to AG_MAX_TAPS
 *                       taps along the major axis (N = ceil(s1 / s2 - 0.05)), each
 *                       a trilinear sample of the view's Lanczos-2 pyramid at
 *                       log2(max(s2, s1 / AG_MAX_TAPS)) + AG_LOD_BIAS, levels >= 1
 *                       sharpened by P + AG_SHARPEN (P - blur P) (Sec. 7.4).
 *  AG_FILTER_BILINEAR - one bilinear sample at the projected position. */
enum { AG_FILTER_ANISO = 0, AG_FILTER_BILINEAR = 1 };
#define AG_MAX_TAPS 8
#define AG_LOD_BIAS (-0.5f)
#define AG_SHARPEN 0.25f

/* Options.  Zero-initialise then call ag_opts_default, or pass NULL for the
 * defaults. */
typedef struct {
    int32_t bvh_layout;  /* ag_bvh_build: AG_BVH_Q8 (80-byte nodes, 8-bit child boxes rounded
                            outward) or AG_BVH_F32 (208-byte nodes, exact FP32 child boxes) */
    int32_t gutter;      /* dilation passes, 0..8 (default 2) */
    int32_t disp_fp16;   /* 1: d_disp is IEEE binary16 [H*W] (default); 0: float32 [H*W] */
    int32_t schedule;    /* traversal schedule, AG_SCHED_* (default AG_SCHED_AUTO) */
    int32_t block_size;  /* trace threads per block, 64..1024, multiple of 32 (0 = schedule default) */
    int32_t blocks_per_sm; /* persistent trace CTAs per SM (0 = schedule default) */
    int32_t max_steps;   /* per-ray traversal step cap (0 = 1<<20); exceeding it sets
                            AG_ERR_TRAVERSAL_LIMIT */
    int32_t collapse;    /* ag_bvh_build: how the binary tree collapses into 8-wide nodes:
                            AG_COLLAPSE_SAH (ag_opts_default: the children that minimise the
                            tree's surface-area cost, a bottom-up dynamic program over the
                            binary tree), or greedy expansion of the largest child by area
                            (AG_COLLAPSE_AREA, 0), area x count or count */
    int32_t ray_tile;    /* ag_bake*: atlas tile shape that orders the ray list, AG_TILE_*
                            (a warp's 32 rays come from one tile; default AG_TILE_8x8) */
    int32_t query;       /* ag_bake*, ag_autotune: AG_QUERY_RAY (0, default) or AG_QUERY_CLOSEST */
    int32_t render;      /* ag_render_views: AG_RENDER_RASTER (0, default) or AG_RENDER_TRACE */
    int32_t filter;      /* ag_backproject: AG_FILTER_ANISO (0, default) or AG_FILTER_BILINEAR */
    int32_t build_async; /* ag_bvh_build: 0 (default) waits for the build; 1 returns once it is
                            enqueued (see ag_bvh_build) */
    int32_t stack_limit; /* test hook, ag_bake with aux counters only (the counting build): use at
                            most this many traversal stack entries per ray (0 = all of them), so
                            that an overflow, reported as AG_ERR_TRAVERSAL_LIMIT, can be provoked
                            on purpose; the other builds ignore it */
    int32_t reserved[2];
} ag_opts;

/* Optional extra outputs of ag_bake (any member may be NULL). */
typedef struct {
    float *normal_ts;   /* [H*W*3] tangent-space normal, float32, after dilation */
    float *disp_f32;    /* [H*W] displacement, float32, after dilation */
    int32_t *face;      /* [H*W] owning low face of the UV raster, -1 where empty */
    float *bary;        /* [H*W*3] raster barycentrics of the texel's surface point */
    int32_t *hit_tri;   /* [H*W] high-poly triangle id of the closest hit, -1 on miss/empty */
    float *hit_t;       /* [H*W] signed ray parameter of the hit (0 on miss/empty) */
    uint64_t *counters; /* [4] device, accumulated (not cleared): rays traced, node visits,
                           triangle tests, hits.  Non-NULL selects the counting build of the
                           traversal (slower; used to measure bytes per ray). */
    int32_t *n_rays;    /* [1] device: number of ray texels */
    void **events;      /* HOST array of 4 cudaEvent_t created by the caller, recorded on
                           `stream`: before the UV raster, before the traversal, after the
                           traversal, after dilation/encoding (per-stage timing) */
} ag_bake_aux;

/* One asset of a batched bake: the arguments of ag_bake. */
typedef struct {
    ag_bvh_t bvh;
    const float *lverts;     /* [n_lverts*3] */
    const float *lnormals;   /* [n_lverts*3] or NULL (area-weighted normals are derived) */
    const float *luv;        /* [n_lfaces*3*2] */
    const int32_t *lfaces;   /* [n_lfaces*3] */
    int64_t n_lverts, n_lfaces;
    int32_t W, H;
    float max_dist;
    uint8_t *normal_rgba8;   /* [H*W*4] */
    uint8_t *mask;           /* [H*W] */
    void *disp;              /* [H*W] half or float (ag_opts.disp_fp16) */
} ag_asset_desc;

/* Size and shape of a built BVH. */
typedef struct {
    int64_t n_tris, n_verts, n_nodes;
    int64_t node_bytes, tri_bytes, normal_bytes; /* device bytes of each array */
    int32_t layout, node_size, max_depth, reserved;
    float scene_lo[3], scene_hi[3];
    float diam;                                  /* bbox diagonal of the high mesh */
    float build_ms;                              /* device time of the last build */
} ag_bvh_info_t;

/* Fill `o` with the defaults listed above. */
AG_API void ag_opts_default(ag_opts *o);

/*
 * ag_bvh_build - acceleration structure over the high-poly mesh
 * (Sec. 6.4: the device-built tree over the high-poly triangles).
 * d_verts [n_verts*3] float32, d_faces [n_faces*3] int32 (0 <= index < n_verts;
 * checked on the device: out-of-range faces are reported as AG_ERR_INVALID_ARG).
 * Builds a linear BVH (30-bit Morton codes of triangle centroids, device radix
 * sort, Karras hierarchy), collapses it to 8-wide nodes with leaves of one
 * triangle, stores child boxes per opts->bvh_layout, reorders triangles into
 * leaf order and computes area-weighted smooth vertex normals.  The handle
 * keeps its own copies.  1 <= n_faces < 2^29, 3 <= n_verts < 2^31.
 * Default (opts->build_async = 0): synchronises `stream`; the inputs may be
 * freed after the call returns; out-of-range face indices are returned as
 * AG_ERR_INVALID_ARG; the node array is trimmed to the node count.
 * opts->build_async = 1: returns once the build is enqueued on `stream`, with
 * no host round trip.  The inputs must stay valid until `stream` has run the
 * build; later calls on `stream` (or ordered after it) may use the handle at
 * once.  Face index errors reach the status word (ag_sync_status).  The node
 * array keeps its worst-case size (n_faces - 1 nodes).  ag_bvh_info,
 * ag_bvh_copy_out, ag_visibility, ag_render_views, ag_point_distance and
 * calls on an AG_BVH_F32 tree wait for the build the first time they need
 * its summary (node count, depth, scene box); ag_bake, ag_bake_backward and
 * ag_bake_batch on an AG_BVH_Q8 tree do not wait on the host.  ag_bake,
 * ag_bake_backward, ag_point_distance and ag_normal_map_error called on
 * another stream order their tree traversal after the build themselves (an
 * event wait, skipped while that stream is being captured), so a bake's
 * raster and frames may run beside the build; ag_bake_batch relies on the
 * caller's ordering.
 * Test hook: the environment variable AG_TEST_GRID_LEVELS=k (0..16) runs the
 * collapse levels from k on in the single-CTA kernel that otherwise serves
 * only trees deeper than 16 levels; the tree is the same.
 */
AG_API ag_status ag_bvh_build(const float *d_verts, int64_t n_verts, const int32_t *d_faces,
                              int64_t n_faces, const ag_opts *opts, ag_stream_t stream,
                              ag_bvh_t *out);

/* Free a handle (synchronises the device first).  NULL is a no-op. */
AG_API ag_status ag_bvh_free(ag_bvh_t h);

/* Free a handle in stream order: its device arrays return to the library's
 * memory pool once the work already queued on `stream` has run, without
 * synchronising.  Work that uses the handle on other streams must be ordered
 * before `stream` by the caller.  The handle is invalid on return.  NULL is a
 * no-op. */
AG_API ag_status ag_bvh_free_async(ag_bvh_t h, ag_stream_t stream);

/* Query sizes of a built BVH. */
AG_API ag_status ag_bvh_info(ag_bvh_t h, ag_bvh_info_t *out);

/*
 * ag_bvh_copy_out - copy a built BVH to HOST buffers (diagnostics and tests;
 * synchronises the device).  Any pointer may be NULL.  Sizes follow
 * ag_bvh_info: nodes [node_bytes] in the layout's node format (80-byte
 * quantised nodes or 208-byte FP32 nodes, see the node description in
 * paper_2605_26137_b300/csrc/ag_internal.cuh), tris [n_tris*12] float (three
 * vertices per leaf-order record, each xyz + the vertex index's bits),
 * tri_ids [n_tris] original triangle of each record, vnormals [n_verts*4]
 * float (unit smooth normal xyz, 0).
 */
AG_API ag_status ag_bvh_copy_out(ag_bvh_t h, void *nodes, float *tris, int32_t *tri_ids, float *vnormals);

/*
 * ag_bake - one tangent-space normal bake (Sec. 6.4, all four stages).
 * Low mesh: d_lverts [n_lverts*3], d_lnormals [n_lverts*3] or NULL
 * (area-weighted vertex normals are derived), d_luv per corner
 * [n_lfaces*3*2], d_lfaces [n_lfaces*3].  W, H in 1..16384 texels; UV
 * coordinates must lie in [-1, 2].  max_dist > 0: hits with |t| > max_dist
 * are rejected (the distance filter).
 * Outputs (caller-owned device buffers, fully overwritten):
 *   d_normal_rgba8 [H*W*4]: RGB = 128 + round(127 * n_ts) (codes 1..255,
 *     half-way cases away from zero), A = 255 on covered and dilated texels,
 *     else 0; empty texels encode (0,0,1) = (128,128,255);
 *   d_mask [H*W]: 1 where a ray texel found a hit, else 0 (not dilated);
 *   d_disp [H*W]: signed hit distance t (0 on miss), dilated like the normal;
 *     binary16 or float32 per opts->disp_fp16.
 * `aux` (NULL allowed) adds the optional outputs of ag_bake_aux.
 */
AG_API ag_status ag_bake(ag_bvh_t h, const float *d_lverts, const float *d_lnormals,
                         const float *d_luv, const int32_t *d_lfaces, int64_t n_lverts,
                         int64_t n_lfaces, int32_t W, int32_t H, float max_dist,
                         const ag_opts *opts, ag_stream_t stream, uint8_t *d_normal_rgba8,
                         uint8_t *d_mask, void *d_disp, const ag_bake_aux *aux);

/*
 * ag_bake_batch - bake n_assets (1..4096) independent assets with one
 * persistent traversal launch over a global ray queue (batch-level analogue
 * of the pipelined serving of Sec. 8).  `descs` is a HOST array; each entry
 * carries the arguments and outputs of one ag_bake call.  Results are those
 * of n_assets separate ag_bake calls.
 */
AG_API ag_status ag_bake_batch(int32_t n_assets, const ag_asset_desc *descs, const ag_opts *opts,
                               ag_stream_t stream);

/*
 * Captured batch: ag_batch_plan_create validates `descs`, allocates all
 * scratch once and captures the batched bake into a CUDA graph (it
 * synchronises `stream` once).  ag_batch_plan_launch replays the graph on
 * `stream` (inputs are re-read on every launch, so they may change between
 * launches as long as pointers and sizes do not).  ag_batch_plan_free
 * synchronises the device and releases everything.
 */
AG_API ag_status ag_batch_plan_create(int32_t n_assets, const ag_asset_desc *descs,
                                      const ag_opts *opts, ag_stream_t stream,
                                      ag_batch_plan_t *out);
AG_API ag_status ag_batch_plan_launch(ag_batch_plan_t p, ag_stream_t stream);
AG_API ag_status ag_batch_plan_free(ag_batch_plan_t p);

/*
 * ag_bake_backward - loss and gradient for cage optimisation (not in the
 * paper; the adjoint of the bake above).  With M the ray texels that hit,
 *   L = (1/|M|) sum_M t^2 + lambda (1/|M|) sum_M (1 - n_hit . d)
 * where d is the texel's interpolated unit normal (the ray direction) and
 * n_hit the hit's smooth normal, both in world space.  Hits are recomputed
 * (same traversal as ag_bake); the hit triangle and M are held fixed, so the
 * result is the derivative of the piecewise-smooth loss.  Low vertex normals
 * are always the area-weighted ones (their dependence on d_lverts is
 * differentiated).  d_loss [1] float and/or d_grad [n_lverts*3] float (fully
 * overwritten) may be NULL; both NULL is an argument error.
 */
AG_API ag_status ag_bake_backward(ag_bvh_t h, const float *d_lverts, const float *d_luv,
                                  const int32_t *d_lfaces, int64_t n_lverts, int64_t n_lfaces,
                                  int32_t W, int32_t H, float max_dist, float lambda,
                                  const ag_opts *opts, ag_stream_t stream, float *d_loss,
                                  float *d_grad);

/*
 * ag_vertex_normals_noalloc - area-weighted unit vertex normals of a mesh
 * (the same normals ag_bvh_build computes for the high-poly mesh), without
 * allocating anything.  The paper has no counterpart: this call exists for
 * callers that cannot allocate device memory at the point where they need
 * normals - code running inside a host application that owns the whole
 * device-memory budget through its own allocator, a plugin that must not
 * touch the CUDA allocator, or a latency-critical loop where an allocation's
 * implicit synchronisation or pool growth is not acceptable.
 * d_verts [n_verts*3] float32, d_faces [n_faces*3] int32 (indices outside
 * [0, n_verts) are skipped), d_normals [n_verts*4] float32, 16-byte aligned,
 * receives xyz = unit normal, w = 0.  The caller owns all three buffers.
 * Limits: 3 <= n_verts <= 131,072 and 1 <= n_faces <= 262,144; larger meshes
 * are rejected with AG_ERR_INVALID_ARG (use ag_bvh_build instead).
 * Scratch: one static device array of about 4.2 MB inside this library,
 * present on every device that loads the library until the process exits.
 * No cudaMalloc, cudaFree or pool allocation is made.  Every call looks up
 * that array's device address on the current device (cudaGetSymbolAddress);
 * the first call on a device may initialise the library's device code there,
 * so make that first call before capturing a stream into a CUDA graph.  All calls share the one array and
 * each call clears the parts that must start at zero, so calls that overlap
 * on the GPU (other streams or other host threads) race and must be
 * serialised by the caller.  Ordered on `stream`; does not synchronise.
 */
AG_API ag_status ag_vertex_normals_noalloc(const float *d_verts, int64_t n_verts,
                                           const int32_t *d_faces, int64_t n_faces,
                                           float *d_normals, ag_stream_t stream);

/*
 * ag_autotune - choose the launch configuration of ag_bake for one asset:
 * every combination of schedule (AG_SCHED_BATCH, AG_SCHED_REFILL), trace
 * block size (64, 128, 256) and ray tile (AG_TILE_*) is timed with CUDA
 * events on `stream` over whole bakes of this asset (1 warm-up + 3 timed,
 * median), and the fastest is written into *inout (schedule, block_size,
 * blocks_per_sm = 0, ray_tile; other fields are kept).  *best_ms (optional)
 * receives its median bake time.  Arguments as ag_bake; outputs go to
 * scratch.  Synchronises `stream`.  Results do not depend on the choice.
 */
AG_API ag_status ag_autotune(ag_bvh_t h, const float *d_lverts, const float *d_lnormals,
                             const float *d_luv, const int32_t *d_lfaces, int64_t n_lverts,
                             int64_t n_lfaces, int32_t W, int32_t H, float max_dist,
                             ag_stream_t stream, ag_opts *inout, float *best_ms);

/* Synchronise `stream`, then return and clear the device status word
 * (AG_ERR_TRAVERSAL_LIMIT if any ray since the last call hit a limit, or
 * AG_ERR_INVALID_ARG for out-of-range face indices seen by ag_bvh_build), or
 * AG_ERR_CUDA if the stream reported an error. */
/*
 * Hidden-face removal (Sec. 6.2 of the paper): a visibility pass over a BVH
 * of the mesh, then a normal-gated flood fill.
 *
 * ag_visibility - per-face visibility of the mesh the handle was built on.
 *   View k of n_views looks along -u_k, u_k on the Fibonacci (golden-angle)
 *   lattice: z = 1 - (2k+1)/n_views, phi = k * pi (3 - sqrt 5),
 *   u = (sqrt(1-z^2) cos phi, sqrt(1-z^2) sin phi, z).  Its image axes are
 *   e1 = normalize(a x u), e2 = u x e1 (a = +z, or +x when |u_z| >= 0.9);
 *   the res x res pixels tile [-R, R]^2 in that plane through c, the centre
 *   of the vertex bounding box (R = half its diagonal), and pixel (i, j)
 *   casts an orthographic ray from c + 2R u + x e1 + y e2,
 *   x = (2 (i + 1/2) / res - 1) R, y likewise with j, along -u.  A face is
 *   visible when it is the first hit of at least one ray (the closest-hit
 *   rules of ag_bake's ray query: watertight test, no culling, ties to the
 *   lower id).
 *   d_visible  [n_faces] u8, device: overwritten with 1 (visible) / 0.
 *   d_hit_ids  optional [n_views * res * res] int32, device: the first-hit
 *              face of pixel (i, j) of view k at k*res*res + j*res + i, -1
 *              on a miss (for tests and debugging; 4 bytes per ray).
 *   d_counters optional [4] u64, device, accumulated: rays, node visits,
 *              triangle tests, hits (selects the counting build, which
 *              traces every ray).
 *   opts: render (AG_RENDER_RASTER: z-buffer proposals of the orthographic
 *   views confirmed by the ray test, the other pixels traced: the first hits
 *   of tracing every ray except where two triangles lie within rounding of
 *   each other along a ray; AG_RENDER_TRACE: every ray traced),
 *   block_size (64..256), blocks_per_sm (tracing), max_steps are used.
 *   Errors: AG_ERR_BAD_HANDLE, AG_ERR_INVALID_ARG (n_views outside 1..2^20,
 *   res outside 1..16384, n_views * ceil(res/8) * ceil(res/4) >= 2^31, NULL
 *   d_visible); the step cap sets the status word.
 */
AG_API ag_status ag_visibility(ag_bvh_t h, int32_t n_views, int32_t res, const ag_opts *opts,
                               ag_stream_t stream, uint8_t *d_visible, int32_t *d_hit_ids,
                               uint64_t *d_counters);

/*
 * ag_exterior_fill - the exterior faces from a visibility mask: faces f and
 *   g are linked when they share an edge (two vertex indices) and
 *   n_f . n_g > 0, n = (B - A) x (C - A) evaluated in FP64 in that order
 *   (x: e1.y e2.z - e1.z e2.y, and so on; the dot product summed x, y, z);
 *   the exterior is every face linked to a visible face through any chain.
 *   The result does not depend on the order of the search.
 *   d_verts [n_verts*3] f32, d_faces [n_faces*3] i32, d_visible [n_faces] u8
 *   (nonzero = visible), d_exterior [n_faces] u8 out (1 = exterior, kept;
 *   0 = hidden, to be removed), all device.  Faces with an out-of-range
 *   vertex index are never exterior and set AG_ERR_INVALID_ARG in the
 *   status word.  Scratch: about 60 bytes per face + 8 per vertex.
 */
AG_API ag_status ag_exterior_fill(const float *d_verts, int64_t n_verts, const int32_t *d_faces,
                                  int64_t n_faces, const uint8_t *d_visible, ag_stream_t stream,
                                  uint8_t *d_exterior);

/*
 * ag_qem_simplify - quadric-error edge-collapse simplification (Sec. 6.1 of
 *   the paper) with its contraction point: the minimiser of the merged
 *   quadric (A x = -b) projected onto the edge and clamped to it, the
 *   midpoint when |det A| <= 1e-12 max_i |A_ii|^3; boundary edges go to the
 *   lower-error endpoint, interior edges with one boundary endpoint to that
 *   endpoint, interior edges with two are kept.  Quadrics are unweighted
 *   sums of the incident faces' plane quadrics.
 *   Collapses run in rounds: an edge (a < b) collapses when its key (its
 *   cost rounded to float32, then its rank in (a, b) order) is the smallest
 *   within two edges of both endpoints and the collapse is valid (at most two
 *   faces on the edge, at most 64 neighbours per endpoint, the link
 *   condition, no tetrahedron, no surviving face turning over); the round
 *   that would pass the target keeps only its cheapest collapses.  All
 *   quadric arithmetic is FP64, rounded to nearest in a fixed order.
 *   d_verts [n_verts*3] f32 and d_faces [n_faces*3] i32 (device) are read
 *   only; faces with a repeated index are dropped.
 *   target: stop at or below this many faces (or when nothing collapses).
 *   max_rounds: 0 = no limit.
 *   placement: AG_QEM_OPTIMAL (0, the paper's projected optimum) or
 *   AG_QEM_MIDPOINT (1, every interior edge at its midpoint: the baseline
 *   the paper improves on; boundary rules unchanged).
 *   d_verts_out [n_verts*3] f64, d_faces_out [n_faces*3] i32 (device): the
 *   surviving vertices in increasing original id (FP64 positions) and the
 *   surviving faces, renumbered, in increasing original id; only the first
 *   h_result[0] vertices and h_result[1] faces are written.
 *   d_keep_verts (optional) [n_verts] i32: original id of each output vertex.
 *   h_result [3] (host): output vertices, output faces, rounds.
 *   Synchronises `stream` once every eight rounds (the decision to stop is
 *   taken on the device; up to seven rounds past the end are enqueued and
 *   return at once) and at the end.  Faces with an out-of-range index
 *   are dropped and set AG_ERR_INVALID_ARG in the status word.
 */
enum { AG_QEM_OPTIMAL = 0, AG_QEM_MIDPOINT = 1 };
AG_API ag_status ag_qem_simplify(const float *d_verts, int64_t n_verts, const int32_t *d_faces,
                                 int64_t n_faces, int64_t target, int32_t max_rounds, int32_t placement,
                                 ag_stream_t stream,
                                 double *d_verts_out, int32_t *d_faces_out, int32_t *d_keep_verts,
                                 int64_t *h_result);

/*
 * ag_normal_map_error - the "baked mean" quality measure of Sec. 6.1 (the
 *   simplification benchmark's baked-normal error, a footnote there: points
 *   spread uniformly over the simplified mesh, the angle between the baked
 *   normal and the raw mesh's true normal, averaged).  Per sample point of
 *   the low mesh, the angle in degrees between
 *   - the normal the RGBA8 map gives there: the texel holding the point's UV
 *     (x = floor(u W), y = floor(v H), clamped), RGB codes decoded as
 *     (q - 128) / 127 and renormalised, taken to world space through the
 *     bake's tangent frame at the point (N the interpolated area-weighted
 *     vertex normal, T the interpolated corner tangent made orthogonal to N,
 *     B = w (N x T)); on a face whose UVs are degenerate (the bake's
 *     UV-reliability filter) the map is not used and the normal is N, and
 *   - the smooth normal of the handle's mesh (the raw mesh) at its surface
 *     point nearest to the sample (the AG_QUERY_CLOSEST search, radius
 *     max_dist),
 *   as atan2(|a x b|, a . b).
 *   h: BVH of the raw mesh.  Low mesh, d_luv, W, H: as in ag_bake.
 *   d_normal_rgba8 [H*W*4] (device, 4-byte aligned): a map baked for this
 *   low mesh and atlas (any map: it is only read).
 *   d_sample_face [n] i32, d_sample_bary [n*2] f32 (device): each sample's
 *   low face and its barycentrics (b1, b2) of corners 1 and 2; the caller
 *   draws them (uniform by area for the paper's measure).
 *   d_angle_deg [n] f32 (device, out): the angle, or -1 where no raw point
 *   lies within max_dist, or the sample's face was dropped (bad UVs); a face
 *   id out of range gives -1 and sets AG_ERR_INVALID_ARG in the status word.
 *   Ordered on `stream`; does not synchronise.
 */
AG_API ag_status ag_normal_map_error(ag_bvh_t h, const float *d_lverts, const float *d_luv,
                                     const int32_t *d_lfaces, int64_t n_lverts, int64_t n_lfaces,
                                     int32_t W, int32_t H, const uint8_t *d_normal_rgba8,
                                     const int32_t *d_sample_face, const float *d_sample_bary,
                                     int64_t n_samples, float max_dist, const ag_opts *opts,
                                     ag_stream_t stream, float *d_angle_deg);

/*
 * ag_point_distance - distance from each of n points to the mesh of the
 *   handle (the closed triangles; a measurement tool, e.g. for Chamfer and
 *   Hausdorff distances between meshes).  d_points [n*3] f32 device;
 *   d_dist [n] f32 out: the distance, or -1 when no triangle lies within
 *   max_dist; d_tri (optional) [n] i32 out: the nearest triangle (lowest id
 *   among equal distances), -1 when none.  The query and its FP32
 *   arithmetic are those of AG_QUERY_CLOSEST.
 */
AG_API ag_status ag_point_distance(ag_bvh_t h, const float *d_points, int64_t n_points, float max_dist,
                                   const ag_opts *opts, ag_stream_t stream, float *d_dist, int32_t *d_tri);

/*
 * UV-space backprojection and incidence blending (Sec. 7.4 of the paper).
 *
 * Cameras (host float [16] per view): R (3x3, row-major, world -> camera,
 * rows = right, down, forward), t (3), fx, fy, cx, cy in pixels.  A point p
 * has camera coordinates c = R p + t, depth c.z and image position
 * (fx c.x / c.z + cx, fy c.y / c.z + cy); pixel (i, j) covers
 * [i, i+1) x [j, j+1).
 *
 * ag_render_views - per view and pixel: the camera depth of the first hit in
 *   front of the camera of the ray through the pixel centre (smallest t > 0
 *   under the watertight test, equal t: lower id; d_depth [K*h*w] f32, +inf
 *   on a miss), its world point (d_points, optional [K*h*w*3] f32, NaN on a
 *   miss) and the edge mask (d_edge, optional [K*h*w] u8: a hit whose
 *   4-neighbour misses or lies farther than edge_tol from it, world points
 *   rebuilt from depth).  opts: render (AG_RENDER_*), max_steps.  Errors:
 *   AG_ERR_BAD_HANDLE, AG_ERR_INVALID_ARG (n_views outside 1..4096, w or h
 *   outside 1..16384, NULL h_cams or d_depth, edge_tol not finite and > 0).
 *
 * ag_backproject - the texture of the low mesh's atlas (the bake's raster)
 *   from K views: for every ray texel and view, its surface point p and
 *   smooth normal n; the view counts when c.z > 0, the pixel is inside the
 *   image, a hit, not an edge pixel, and c.z <= its depth + depth_tol; its
 *   incidence is I = max(0, n . normalize(C - p)) (C the camera centre) and
 *   its colour A_k the anisotropic footprint sample (opts->filter ==
 *   AG_FILTER_ANISO, the default) or the bilinear sample of the RGBA8 image
 *   at (u - 1/2, v - 1/2) (AG_FILTER_BILINEAR; clamped, codes / 255).
 *   T = sum_k w_k I^alpha A_k / (sum_k w_k I^alpha + eps) over the counting
 *   views, evaluated in log space.  opts: filter, ray_tile.
 *   d_images [K*h*w*4] u8 (4-byte aligned), d_depth, d_edge from
 *   ag_render_views (device);
 *   h_weights [K] host, > 0 (the view prior);
 *   d_texture [H*W*4] f32 out: RGB and 1 where at least one view counts
 *   (else all 0); d_incidence optional [K*H*W] f32 out.
 */
AG_API ag_status ag_render_views(ag_bvh_t h, int32_t n_views, const float *h_cams, int32_t w, int32_t hgt,
                                 float edge_tol, const ag_opts *opts, ag_stream_t stream, float *d_depth,
                                 float *d_points, uint8_t *d_edge);
AG_API ag_status ag_backproject(const float *d_lverts, const float *d_lnormals, const float *d_luv,
                                const int32_t *d_lfaces, int64_t n_lverts, int64_t n_lfaces, int32_t W, int32_t H,
                                int32_t n_views, const float *h_cams, const float *h_weights,
                                const uint8_t *d_images, const float *d_depth, const uint8_t *d_edge, int32_t w,
                                int32_t hgt, float alpha, float eps, float depth_tol, const ag_opts *opts,
                                ag_stream_t stream, float *d_texture, float *d_incidence);

AG_API ag_status ag_sync_status(ag_stream_t stream);

/* Message for the last failing call on this thread ("" if none). */
AG_API const char *ag_last_error(void);
/* Static name of a status code. */
AG_API const char *ag_status_string(ag_status s);
/* ABI version: major*10000 + minor*100 + patch. */
AG_API int32_t ag_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AG_H */
