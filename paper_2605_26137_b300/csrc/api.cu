// C ABI of the baker (include/ag.h): argument checks, scratch, launch order.
#include "ag_internal.cuh"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

namespace ag {

ag_status build_bvh(const float *d_verts, int64_t nv, const int32_t *d_faces, int64_t nf, int layout, int rule,
                    bool sync, cudaStream_t s, ag_bvh *h);

namespace {
thread_local std::string g_err;
std::mutex g_mu;
constexpr int MAXDEV = 64;
unsigned *g_status[MAXDEV] = {nullptr};
cudaMemPool_t g_pool[MAXDEV] = {nullptr};
int g_sms[MAXDEV] = {0};
}  // namespace

ag_status set_error(ag_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

ag_status cuda_error(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(AG_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(AG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

unsigned *device_status_word(int dev) {
    if (dev < 0 || dev >= MAXDEV) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status[dev]) {
        unsigned *p = nullptr;
        if (cudaMalloc(&p, 64) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, 64);
        cudaDeviceSynchronize();
        g_status[dev] = p;
    }
    return g_status[dev];
}

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= MAXDEV) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t thr = ~0ull;  // keep freed blocks for reuse by later calls
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

int device_sm_count(int dev) {
    if (dev < 0 || dev >= MAXDEV) return 1;
    if (!g_sms[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = n > 0 ? n : 1;
    }
    return g_sms[dev];
}

cudaError_t Scratch::alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (n >= (int)(sizeof(ptrs) / sizeof(ptrs[0]))) return cudaErrorInvalidValue;
    cudaMemPool_t pool = device_pool(device);
    if (!pool) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, stream);
    if (e == cudaSuccess) ptrs[n++] = *p;
    return e;
}

Scratch::~Scratch() {
    for (int i = n - 1; i >= 0; --i) cudaFreeAsync(ptrs[i], stream);
}

}  // namespace ag

using namespace ag;

namespace {

ag_opts resolve_opts(const ag_opts *o) {
    ag_opts r;
    ag_opts_default(&r);
    if (o) r = *o;
    return r;
}

ag_status check_opts(const ag_opts &o) {
    if (o.bvh_layout != AG_BVH_Q8 && o.bvh_layout != AG_BVH_F32)
        return set_error(AG_ERR_INVALID_ARG, "bvh_layout must be AG_BVH_Q8 or AG_BVH_F32");
    if (o.gutter < 0 || o.gutter > 8) return set_error(AG_ERR_INVALID_ARG, "gutter must be in 0..8");
    if (o.block_size != 0 && (o.block_size < 64 || o.block_size > 1024 || o.block_size % 32))
        return set_error(AG_ERR_INVALID_ARG, "block_size must be 0 or a multiple of 32 in 64..1024");
    if (o.blocks_per_sm < 0 || o.blocks_per_sm > 64) return set_error(AG_ERR_INVALID_ARG, "blocks_per_sm out of range");
    if (o.max_steps < 0) return set_error(AG_ERR_INVALID_ARG, "max_steps must be >= 0");
    if (o.schedule < AG_SCHED_AUTO || o.schedule > AG_SCHED_COOP2)
        return set_error(AG_ERR_INVALID_ARG, "unknown schedule");
    if (o.stack_limit < 0) return set_error(AG_ERR_INVALID_ARG, "stack_limit must be >= 0");
    if (o.collapse < AG_COLLAPSE_AREA || o.collapse > AG_COLLAPSE_SAH)
        return set_error(AG_ERR_INVALID_ARG, "unknown collapse rule");
    if (o.ray_tile < AG_TILE_8x8 || o.ray_tile > AG_TILE_4x4) return set_error(AG_ERR_INVALID_ARG, "unknown ray tile");
    if (o.query != AG_QUERY_RAY && o.query != AG_QUERY_CLOSEST)
        return set_error(AG_ERR_INVALID_ARG, "query must be AG_QUERY_RAY or AG_QUERY_CLOSEST");
    if (o.render != AG_RENDER_RASTER && o.render != AG_RENDER_TRACE)
        return set_error(AG_ERR_INVALID_ARG, "render must be AG_RENDER_RASTER or AG_RENDER_TRACE");
    if (o.filter != AG_FILTER_ANISO && o.filter != AG_FILTER_BILINEAR)
        return set_error(AG_ERR_INVALID_ARG, "filter must be AG_FILTER_ANISO or AG_FILTER_BILINEAR");
    if (o.build_async != 0 && o.build_async != 1) return set_error(AG_ERR_INVALID_ARG, "build_async must be 0 or 1");
    return AG_OK;
}

// the handle's arrays come from the device's memory pool (stream-ordered)
void free_handle_arrays(ag_bvh *h, cudaStream_t s) {
    void *arrays[5] = {h->nodes, h->tris, h->tri_ids, h->vnormals, h->d_info};
    for (void *p : arrays)
        if (p) cudaFreeAsync(p, s);
    h->nodes = nullptr;
    h->tris = nullptr;
    h->tri_ids = nullptr;
    h->vnormals = nullptr;
    h->d_info = nullptr;
    // events still pending are released by the runtime once they complete
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->ev_done) cudaEventDestroy(h->ev_done);
    h->ev_start = h->ev_done = nullptr;
}


ag_status check_handle(ag_bvh_t h) {
    if (!h || h->magic != AG_BVH_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "invalid BVH handle");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->device)
        return set_error(AG_ERR_INVALID_ARG, "handle lives on device %d but device %d is current", h->device, dev);
    return AG_OK;
}

ag_status check_low(const float *lv, const float *luv, const int32_t *lf, int64_t nv, int64_t nf, int W, int H,
                    float max_dist) {
    if (!lv || !luv || !lf) return set_error(AG_ERR_INVALID_ARG, "low mesh pointers must be non-NULL");
    if (nv < 3 || nv >= (1ll << 31)) return set_error(AG_ERR_INVALID_ARG, "n_lverts out of range");
    if (nf < 1 || nf >= (1ll << 31)) return set_error(AG_ERR_INVALID_ARG, "n_lfaces out of range");
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return set_error(AG_ERR_INVALID_ARG, "W and H must be in 1..16384");
    if (!(max_dist > 0.f) || !(max_dist < 3.0e38f)) return set_error(AG_ERR_INVALID_ARG, "max_dist must be a positive finite float");
    return AG_OK;
}

// scratch + launches of the per-asset stages that precede the trace
struct AssetScratch {
    float *acc;
    float4 *lpos, *lnrm, *ltan;
    int4 *lface, *uvfix, *rays;
    unsigned long long *keys;
    int32_t *face;
    float4 *ntsd;
    long long *n_rays;
    void *nscr;
};

ag_status alloc_asset(Scratch &sc, int64_t nv, int64_t nf, int W, int H, bool own_face, AssetScratch &a) {
    size_t hw = (size_t)W * H;
    AG_CUDA(sc.alloc((void **)&a.acc, sizeof(float) * 3 * nv));
    AG_CUDA(sc.alloc((void **)&a.lpos, sizeof(float4) * nv));
    AG_CUDA(sc.alloc((void **)&a.lnrm, sizeof(float4) * nv));
    AG_CUDA(sc.alloc((void **)&a.ltan, sizeof(float4) * 3 * nf));
    AG_CUDA(sc.alloc((void **)&a.lface, sizeof(int4) * nf));
    AG_CUDA(sc.alloc((void **)&a.uvfix, sizeof(int4) * 2 * nf));
    AG_CUDA(sc.alloc((void **)&a.keys, sizeof(unsigned long long) * hw));
    if (own_face) AG_CUDA(sc.alloc((void **)&a.face, sizeof(int32_t) * hw));
    AG_CUDA(sc.alloc((void **)&a.rays, sizeof(int4) * hw));
    AG_CUDA(sc.alloc((void **)&a.ntsd, sizeof(float4) * hw));
    AG_CUDA(sc.alloc((void **)&a.n_rays, sizeof(long long) * 2));
    AG_CUDA(sc.alloc(&a.nscr, vertex_normal_scratch_bytes(nv, nf)));
    return AG_OK;
}

ag_status run_prep(const float *lv, const float *ln, const float *luv, const int32_t *lf, int64_t nv, int64_t nf,
                   int W, int H, int ray_tile, float *aux_bary, unsigned *status, AssetScratch &a, cudaStream_t s) {
    // the UV set-up, raster and resolve (texel -> face) stay on s; the low
    // mesh's vertex normals and corner frames, needed only by the traversal,
    // run beside them on a side stream and join s before it returns
    int dev = 0;
    AG_CUDA(cudaGetDevice(&dev));
    cudaStream_t *side = nullptr;
    AG_CUDA(side_streams(dev, &side));
    AG_CUDA(launch_uv_setup(luv, lf, nf, nv, W, H, a.uvfix, status, s));
    EventSet es;
    AG_CUDA(fork_to(s, side, 1, es));
    AG_CUDA(launch_vertex_normals(lv, lf, nv, nf, ln, a.acc, a.lnrm, a.lpos, a.nscr, side[0]));
    AG_CUDA(launch_tangents(luv, lf, nf, nv, a.uvfix, a.lpos, a.lnrm, a.lface, a.ltan, side[0]));
    AG_CUDA(cudaMemsetAsync(a.n_rays, 0, sizeof(long long) * 2, s));
    AG_CUDA(launch_raster(a.uvfix, nf, W, H, a.keys, s));
    AG_CUDA(launch_resolve(a.keys, a.uvfix, W, H, ray_tile, a.face, aux_bary, a.rays, a.n_rays, s));
    AG_CUDA(join_from(s, side, 1, es));
    return AG_OK;
}

TraceJob make_job(ag_bvh_t h, const AssetScratch &a, int W, int H, float max_dist, float scene_abs, uint8_t *mask,
                  int32_t *hit_tri, float *hit_t) {
    TraceJob j;
    memset(&j, 0, sizeof(j));
    j.nodes = h->nodes;
    j.tris = h->tris;
    j.tri_ids = h->tri_ids;
    j.hnormals = h->vnormals;
    j.lpos = a.lpos;
    j.lnrm = a.lnrm;
    j.lface = a.lface;
    j.ltan = a.ltan;
    j.rays = a.rays;
    j.ntsd = a.ntsd;
    j.mask = mask;
    j.hit_tri = hit_tri;
    j.hit_t = hit_t;
    j.W = W;
    j.H = H;
    j.max_dist = max_dist;
    j.scene_abs = scene_abs;
    return j;
}

int pick_schedule(const ag_opts &o) { return o.schedule == AG_SCHED_AUTO ? AG_SCHED_BATCH : o.schedule; }

}  // namespace

extern "C" {

AG_API void ag_opts_default(ag_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->bvh_layout = AG_BVH_Q8;
    o->gutter = 2;
    o->disp_fp16 = 1;
    o->schedule = AG_SCHED_AUTO;
    o->collapse = AG_COLLAPSE_SAH;
}

AG_API int32_t ag_version(void) { return 100; }

AG_API const char *ag_last_error(void) { return g_err.c_str(); }

AG_API const char *ag_status_string(ag_status s) {
    switch (s) {
        case AG_OK: return "AG_OK";
        case AG_ERR_INVALID_ARG: return "AG_ERR_INVALID_ARG";
        case AG_ERR_OOM: return "AG_ERR_OOM";
        case AG_ERR_CUDA: return "AG_ERR_CUDA";
        case AG_ERR_TRAVERSAL_LIMIT: return "AG_ERR_TRAVERSAL_LIMIT";
        case AG_ERR_BAD_HANDLE: return "AG_ERR_BAD_HANDLE";
    }
    return "AG_ERR_UNKNOWN";
}

AG_API ag_status ag_bvh_build(const float *d_verts, int64_t n_verts, const int32_t *d_faces, int64_t n_faces,
                              const ag_opts *opts, ag_stream_t stream, ag_bvh_t *out) {
    g_err.clear();
    if (!out) return set_error(AG_ERR_INVALID_ARG, "out must be non-NULL");
    *out = nullptr;
    if (!d_verts || !d_faces) return set_error(AG_ERR_INVALID_ARG, "vertex and face pointers must be non-NULL");
    if (n_verts < 3 || n_verts >= (1ll << 31)) return set_error(AG_ERR_INVALID_ARG, "n_verts out of range");
    if (n_faces < 1 || n_faces >= (1ll << 29)) return set_error(AG_ERR_INVALID_ARG, "n_faces out of range");
    ag_opts o = resolve_opts(opts);
    ag_status st = check_opts(o);
    if (st) return st;
    int dev = 0;
    AG_CUDA(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(dev);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    ag_bvh *h = new (std::nothrow) ag_bvh;
    if (!h) return set_error(AG_ERR_OOM, "host allocation failed");
    memset(h, 0, sizeof(*h));
    h->magic = AG_BVH_MAGIC;
    h->device = dev;
    h->layout = o.bvh_layout;
    h->n_tris = n_faces;
    h->n_verts = n_verts;
    const bool sync = !o.build_async;
    unsigned word = 0;
    st = build_bvh(d_verts, n_verts, d_faces, n_faces, o.bvh_layout, o.collapse, sync, s, h);
    if (st == AG_OK && sync) {
        cudaError_t e = cudaMemcpyAsync(&word, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "ag_bvh_build status");
        else if (word & AGS_BAD_FACE) {
            unsigned keep = word & ~AGS_BAD_FACE;
            cudaMemcpy(status, &keep, sizeof(unsigned), cudaMemcpyHostToDevice);
            st = set_error(AG_ERR_INVALID_ARG, "face index out of range [0, n_verts)");
        }
    }
    if (st != AG_OK) {
        cudaStreamSynchronize(s);
        free_handle_arrays(h, s);
        cudaStreamSynchronize(s);
        h->magic = 0;
        delete h;
        return st;
    }
    *out = h;
    return AG_OK;
}

AG_API ag_status ag_bvh_free_async(ag_bvh_t h, ag_stream_t stream) {
    if (!h) return AG_OK;
    if (h->magic != AG_BVH_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "invalid BVH handle");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    free_handle_arrays(h, (cudaStream_t)stream);
    cudaSetDevice(prev);
    h->magic = 0;
    delete h;
    return AG_OK;
}

AG_API ag_status ag_bvh_free(ag_bvh_t h) {
    if (!h) return AG_OK;
    if (h->magic != AG_BVH_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "invalid BVH handle");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    free_handle_arrays(h, nullptr);
    cudaStreamSynchronize(nullptr);
    cudaSetDevice(prev);
    h->magic = 0;
    delete h;
    return AG_OK;
}

AG_API ag_status ag_bvh_info(ag_bvh_t h, ag_bvh_info_t *out) {
    g_err.clear();
    if (!h || h->magic != AG_BVH_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "invalid BVH handle");
    if (!out) return set_error(AG_ERR_INVALID_ARG, "out must be non-NULL");
    memset(out, 0, sizeof(*out));
    ag_status st = bvh_ready(h);
    if (st) return st;
    out->n_tris = h->n_tris;
    out->n_verts = h->n_verts;
    out->n_nodes = h->n_nodes;
    out->node_size = h->layout == AG_BVH_Q8 ? (int)sizeof(QNode) : (int)sizeof(FNode);
    out->node_bytes = h->n_nodes * out->node_size;
    out->tri_bytes = h->n_tris * 48;
    out->normal_bytes = h->n_verts * 16;
    out->layout = h->layout;
    out->max_depth = h->max_depth;
    for (int a = 0; a < 3; ++a) {
        out->scene_lo[a] = h->lo[a];
        out->scene_hi[a] = h->hi[a];
    }
    out->diam = h->diam;
    out->build_ms = h->build_ms;
    return AG_OK;
}

AG_API ag_status ag_bvh_copy_out(ag_bvh_t h, void *nodes, float *tris, int32_t *tri_ids, float *vnormals) {
    g_err.clear();
    ag_status st = check_handle(h);
    if (st) return st;
    if ((st = bvh_ready(h))) return st;
    AG_CUDA(cudaDeviceSynchronize());
    size_t ns = h->layout == AG_BVH_Q8 ? sizeof(QNode) : sizeof(FNode);
    if (nodes) AG_CUDA(cudaMemcpy(nodes, h->nodes, ns * h->n_nodes, cudaMemcpyDeviceToHost));
    if (tris) AG_CUDA(cudaMemcpy(tris, h->tris, sizeof(float4) * 3 * h->n_tris, cudaMemcpyDeviceToHost));
    if (tri_ids) AG_CUDA(cudaMemcpy(tri_ids, h->tri_ids, sizeof(int32_t) * h->n_tris, cudaMemcpyDeviceToHost));
    if (vnormals) AG_CUDA(cudaMemcpy(vnormals, h->vnormals, sizeof(float4) * h->n_verts, cudaMemcpyDeviceToHost));
    return AG_OK;
}

AG_API ag_status ag_bake(ag_bvh_t h, const float *d_lverts, const float *d_lnormals, const float *d_luv,
                         const int32_t *d_lfaces, int64_t n_lverts, int64_t n_lfaces, int32_t W, int32_t H,
                         float max_dist, const ag_opts *opts, ag_stream_t stream, uint8_t *d_normal_rgba8,
                         uint8_t *d_mask, void *d_disp, const ag_bake_aux *aux) {
    g_err.clear();
    ag_status st = check_handle(h);
    if (st) return st;
    if ((st = check_low(d_lverts, d_luv, d_lfaces, n_lverts, n_lfaces, W, H, max_dist))) return st;
    if (!d_normal_rgba8 || !d_mask || !d_disp) return set_error(AG_ERR_INVALID_ARG, "output pointers must be non-NULL");
    ag_opts o = resolve_opts(opts);
    if ((st = check_opts(o))) return st;
    ag_bake_aux ax;
    memset(&ax, 0, sizeof(ax));
    if (aux) ax = *aux;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(h->device);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    Scratch sc(s, h->device);
    AssetScratch a;
    memset(&a, 0, sizeof(a));
    if ((st = alloc_asset(sc, n_lverts, n_lfaces, W, H, ax.face == nullptr, a))) return st;
    if (ax.face) a.face = ax.face;
    unsigned long long *ray_counter;
    AG_CUDA(sc.alloc((void **)&ray_counter, sizeof(unsigned long long)));
    cudaEvent_t *ev = reinterpret_cast<cudaEvent_t *>(ax.events);
    if (ev) AG_CUDA(cudaEventRecord(ev[0], s));
    if ((st = run_prep(d_lverts, d_lnormals, d_luv, d_lfaces, n_lverts, n_lfaces, W, H, o.ray_tile, ax.bary, status, a,
                       s)))
        return st;
    if (ev) AG_CUDA(cudaEventRecord(ev[1], s));
    float sabs;
    if ((st = scene_abs_for(h, &sabs))) return st;
    TraceLaunch L;
    memset(&L, 0, sizeof(L));
    L.job0 = make_job(h, a, W, H, max_dist, sabs, d_mask, ax.hit_tri, ax.hit_t);
    L.n_jobs = 1;
    L.n_rays_dev = a.n_rays;
    L.ray_counter = ray_counter;
    L.status = status;
    L.max_steps = o.max_steps > 0 ? o.max_steps : (1 << 20);
    L.counters = reinterpret_cast<unsigned long long *>(ax.counters);
    L.stack_cap = o.stack_limit;
    L.layout = h->layout;
    L.schedule = pick_schedule(o);
    L.query = o.query;
    L.block_size = o.block_size;
    L.blocks_per_sm = o.blocks_per_sm;
    L.backward = false;
    AG_CUDA(wait_build(h, s));   // (the raster and frames above need no tree)
    AG_CUDA(launch_trace(L, s));
    if (ev) AG_CUDA(cudaEventRecord(ev[2], s));
    AG_CUDA(launch_finalize(a.ntsd, a.face, W, H, o.gutter, o.disp_fp16, d_normal_rgba8, d_mask, d_disp, ax.normal_ts,
                            ax.disp_f32, ax.hit_tri, ax.hit_t, s));
    if (ev) AG_CUDA(cudaEventRecord(ev[3], s));
    if (ax.n_rays) AG_CUDA(cudaMemcpyAsync(ax.n_rays, a.n_rays, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return AG_OK;
}

AG_API ag_status ag_bake_backward(ag_bvh_t h, const float *d_lverts, const float *d_luv, const int32_t *d_lfaces,
                                  int64_t n_lverts, int64_t n_lfaces, int32_t W, int32_t H, float max_dist,
                                  float lambda, const ag_opts *opts, ag_stream_t stream, float *d_loss,
                                  float *d_grad) {
    g_err.clear();
    ag_status st = check_handle(h);
    if (st) return st;
    if ((st = check_low(d_lverts, d_luv, d_lfaces, n_lverts, n_lfaces, W, H, max_dist))) return st;
    if (!d_loss && !d_grad) return set_error(AG_ERR_INVALID_ARG, "d_loss and d_grad are both NULL");
    if (!(lambda >= 0.f) || !(lambda < 3.0e38f)) return set_error(AG_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    ag_opts o = resolve_opts(opts);
    if ((st = check_opts(o))) return st;
    if (o.query != AG_QUERY_RAY) return set_error(AG_ERR_INVALID_ARG, "ag_bake_backward supports AG_QUERY_RAY only");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(h->device);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    Scratch sc(s, h->device);
    AssetScratch a;
    memset(&a, 0, sizeof(a));
    if ((st = alloc_asset(sc, n_lverts, n_lfaces, W, H, true, a))) return st;
    float *g_pos, *g_nrm, *g_a, *loss_acc;
    unsigned long long *ray_counter;
    AG_CUDA(sc.alloc((void **)&g_pos, sizeof(float) * 3 * n_lverts));
    AG_CUDA(sc.alloc((void **)&g_nrm, sizeof(float) * 3 * n_lverts));
    AG_CUDA(sc.alloc((void **)&g_a, sizeof(float) * 3 * n_lverts));
    AG_CUDA(sc.alloc((void **)&loss_acc, sizeof(float) * 4));
    AG_CUDA(sc.alloc((void **)&ray_counter, sizeof(unsigned long long)));
    AG_CUDA(cudaMemsetAsync(g_pos, 0, sizeof(float) * 3 * n_lverts, s));
    AG_CUDA(cudaMemsetAsync(g_nrm, 0, sizeof(float) * 3 * n_lverts, s));
    AG_CUDA(cudaMemsetAsync(loss_acc, 0, sizeof(float) * 4, s));
    if ((st = run_prep(d_lverts, nullptr, d_luv, d_lfaces, n_lverts, n_lfaces, W, H, o.ray_tile, nullptr, status, a,
                       s)))
        return st;
    float sabs;
    if ((st = scene_abs_for(h, &sabs))) return st;
    TraceLaunch L;
    memset(&L, 0, sizeof(L));
    L.job0 = make_job(h, a, W, H, max_dist, sabs, nullptr, nullptr, nullptr);
    L.job0.g_pos = d_grad ? g_pos : nullptr;   // loss only: no adjoint scatter
    L.job0.g_nrm = g_nrm;
    L.job0.loss_acc = loss_acc;
    L.job0.lambda = lambda;
    L.n_jobs = 1;
    L.n_rays_dev = a.n_rays;
    L.ray_counter = ray_counter;
    L.status = status;
    L.max_steps = o.max_steps > 0 ? o.max_steps : (1 << 20);
    L.layout = h->layout;
    L.schedule = pick_schedule(o);
    L.query = AG_QUERY_RAY;
    L.block_size = o.block_size;
    L.blocks_per_sm = o.blocks_per_sm;
    L.backward = true;
    AG_CUDA(wait_build(h, s));   // (the raster and frames above need no tree)
    AG_CUDA(launch_trace(L, s));
    AG_CUDA(launch_backward_finish(a.lpos, a.lface, n_lverts, n_lfaces, a.acc, g_pos, g_nrm, g_a, loss_acc, lambda,
                                   d_loss, d_grad, s));
    return AG_OK;
}

AG_API ag_status ag_normal_map_error(ag_bvh_t h, const float *d_lverts, const float *d_luv, const int32_t *d_lfaces,
                                     int64_t n_lverts, int64_t n_lfaces, int32_t W, int32_t H,
                                     const uint8_t *d_normal_rgba8, const int32_t *d_sample_face,
                                     const float *d_sample_bary, int64_t n_samples, float max_dist,
                                     const ag_opts *opts, ag_stream_t stream, float *d_angle_deg) {
    g_err.clear();
    ag_status st = check_handle(h);
    if (st) return st;
    if ((st = check_low(d_lverts, d_luv, d_lfaces, n_lverts, n_lfaces, W, H, max_dist))) return st;
    if (n_samples < 0 || n_samples >= (1ll << 40)) return set_error(AG_ERR_INVALID_ARG, "n_samples out of range");
    if (n_samples == 0) return AG_OK;
    if (!d_normal_rgba8 || !d_sample_face || !d_sample_bary || !d_angle_deg)
        return set_error(AG_ERR_INVALID_ARG, "map, sample and output pointers must be non-NULL");
    if (reinterpret_cast<uintptr_t>(d_normal_rgba8) % 4)
        return set_error(AG_ERR_INVALID_ARG, "d_normal_rgba8 must be 4-byte aligned");
    ag_opts o = resolve_opts(opts);
    if ((st = check_opts(o))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(h->device);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    Scratch sc(s, h->device);
    AssetScratch a;
    memset(&a, 0, sizeof(a));
    AG_CUDA(sc.alloc((void **)&a.acc, sizeof(float) * 3 * n_lverts));
    AG_CUDA(sc.alloc((void **)&a.lpos, sizeof(float4) * n_lverts));
    AG_CUDA(sc.alloc((void **)&a.lnrm, sizeof(float4) * n_lverts));
    AG_CUDA(sc.alloc((void **)&a.ltan, sizeof(float4) * 3 * n_lfaces));
    AG_CUDA(sc.alloc((void **)&a.lface, sizeof(int4) * n_lfaces));
    AG_CUDA(sc.alloc((void **)&a.uvfix, sizeof(int4) * 2 * n_lfaces));
    AG_CUDA(sc.alloc(&a.nscr, vertex_normal_scratch_bytes(n_lverts, n_lfaces)));
    // the bake's low-mesh set-up: vertex normals, corner tangents, face flags
    AG_CUDA(launch_vertex_normals(d_lverts, d_lfaces, n_lverts, n_lfaces, nullptr, a.acc, a.lnrm, a.lpos, a.nscr, s));
    AG_CUDA(launch_face_setup(d_luv, d_lfaces, n_lfaces, n_lverts, W, H, a.lpos, a.lnrm, a.lface, a.ltan, a.uvfix,
                              status, s));
    float sabs;
    if ((st = scene_abs_for(h, &sabs))) return st;
    TraceLaunch L;
    memset(&L, 0, sizeof(L));
    L.job0 = make_job(h, a, W, H, max_dist, sabs, nullptr, nullptr, nullptr);
    L.n_jobs = 1;
    L.status = status;
    L.max_steps = o.max_steps > 0 ? o.max_steps : (1 << 20);
    L.layout = h->layout;
    AG_CUDA(wait_build(h, s));
    AG_CUDA(launch_map_error(L, d_normal_rgba8, d_luv, n_lfaces, d_sample_face, d_sample_bary, n_samples, d_angle_deg,
                             s));
    return AG_OK;
}

AG_API ag_status ag_point_distance(ag_bvh_t h, const float *d_points, int64_t n_points, float max_dist,
                                   const ag_opts *opts, ag_stream_t stream, float *d_dist, int32_t *d_tri) {
    g_err.clear();
    ag_status st = check_handle(h);
    if (st) return st;
    if (n_points < 0) return set_error(AG_ERR_INVALID_ARG, "n_points must be >= 0");
    if (n_points == 0) return AG_OK;
    if (!d_points || !d_dist) return set_error(AG_ERR_INVALID_ARG, "d_points and d_dist must be non-NULL");
    if (!(max_dist > 0.f) || !(max_dist < 3.0e38f)) return set_error(AG_ERR_INVALID_ARG, "max_dist must be finite and > 0");
    ag_opts o = resolve_opts(opts);
    if ((st = check_opts(o))) return st;
    unsigned *status = device_status_word(h->device);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    TraceLaunch L;
    memset(&L, 0, sizeof(L));
    L.job0.nodes = h->nodes;
    L.job0.tris = h->tris;
    L.job0.tri_ids = h->tri_ids;
    if ((st = scene_abs_for(h, &L.job0.scene_abs))) return st;
    L.status = status;
    L.max_steps = o.max_steps > 0 ? o.max_steps : (1 << 20);
    L.layout = h->layout;
    AG_CUDA(wait_build(h, (cudaStream_t)stream));
    AG_CUDA(launch_point_distance(L, d_points, n_points, max_dist, d_dist, d_tri, (cudaStream_t)stream));
    return AG_OK;
}

AG_API ag_status ag_render_views(ag_bvh_t h, int32_t n_views, const float *h_cams, int32_t w, int32_t hgt,
                                 float edge_tol, const ag_opts *opts, ag_stream_t stream, float *d_depth,
                                 float *d_points, uint8_t *d_edge) {
    g_err.clear();
    ag_status st = check_handle(h);
    if (st) return st;
    if (n_views < 1 || n_views > 4096) return set_error(AG_ERR_INVALID_ARG, "n_views must be in 1..4096");
    if (w < 1 || hgt < 1 || w > 16384 || hgt > 16384) return set_error(AG_ERR_INVALID_ARG, "w and h must be in 1..16384");
    if (!h_cams || !d_depth) return set_error(AG_ERR_INVALID_ARG, "h_cams and d_depth must be non-NULL");
    if (!(edge_tol > 0.f) || !(edge_tol < 3.0e38f)) return set_error(AG_ERR_INVALID_ARG, "edge_tol must be finite and > 0");
    ag_opts o = resolve_opts(opts);
    if ((st = check_opts(o))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(h->device);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    Scratch sc(s, h->device);
    void *cams;
    const bool raster = o.render == AG_RENDER_RASTER;
    AG_CUDA(sc.alloc(&cams, render_scratch_bytes(n_views, w, hgt, raster)));
    float *points = d_points;
    TraceLaunch L;
    memset(&L, 0, sizeof(L));
    L.job0.nodes = h->nodes;
    L.job0.tris = h->tris;
    L.job0.tri_ids = h->tri_ids;
    if ((st = scene_abs_for(h, &L.job0.scene_abs))) return st;
    L.status = status;
    L.max_steps = o.max_steps > 0 ? o.max_steps : (1 << 20);
    L.layout = h->layout;
    AG_CUDA(launch_render_views(L, (int)h->n_tris, h_cams, n_views, w, hgt, edge_tol, raster, d_depth, points, d_edge,
                                cams, s));
    return AG_OK;
}

AG_API ag_status ag_backproject(const float *d_lverts, const float *d_lnormals, const float *d_luv,
                                const int32_t *d_lfaces, int64_t n_lverts, int64_t n_lfaces, int32_t W, int32_t H,
                                int32_t n_views, const float *h_cams, const float *h_weights, const uint8_t *d_images,
                                const float *d_depth, const uint8_t *d_edge, int32_t w, int32_t hgt, float alpha,
                                float eps, float depth_tol, const ag_opts *opts, ag_stream_t stream, float *d_texture,
                                float *d_incidence) {
    g_err.clear();
    ag_status st;
    if ((st = check_low(d_lverts, d_luv, d_lfaces, n_lverts, n_lfaces, W, H, 1.0f))) return st;
    if (n_views < 1 || n_views > 4096) return set_error(AG_ERR_INVALID_ARG, "n_views must be in 1..4096");
    if (w < 1 || hgt < 1 || w > 16384 || hgt > 16384) return set_error(AG_ERR_INVALID_ARG, "w and h must be in 1..16384");
    if (!h_cams || !h_weights || !d_images || !d_depth || !d_edge || !d_texture)
        return set_error(AG_ERR_INVALID_ARG, "cameras, weights, images, depth, edge and texture must be non-NULL");
    if (reinterpret_cast<uintptr_t>(d_images) % 4)
        return set_error(AG_ERR_INVALID_ARG, "d_images must be 4-byte aligned (RGBA8 pixels)");
    if (!(alpha >= 0.f) || !(alpha < 3.0e38f) || !(eps >= 0.f) || !(eps < 3.0e38f) || !(depth_tol >= 0.f) ||
        !(depth_tol < 3.0e38f))
        return set_error(AG_ERR_INVALID_ARG, "alpha, eps and depth_tol must be finite and >= 0");
    std::vector<float> logw((size_t)n_views);
    for (int k = 0; k < n_views; ++k) {
        if (!(h_weights[k] > 0.f) || !(h_weights[k] < 3.0e38f))
            return set_error(AG_ERR_INVALID_ARG, "view weights must be finite and > 0");
        logw[(size_t)k] = logf(h_weights[k]);
    }
    // camera centres C = -R^T t (float, 4 per view)
    std::vector<float> centres((size_t)n_views * 4);
    for (int k = 0; k < n_views; ++k) {
        const float *c = h_cams + 16 * (size_t)k;
        for (int a = 0; a < 3; ++a)
            centres[4 * (size_t)k + a] = -(c[a] * c[9] + c[3 + a] * c[10] + c[6 + a] * c[11]);
        centres[4 * (size_t)k + 3] = 0.f;
    }
    ag_opts o = resolve_opts(opts);
    if ((st = check_opts(o))) return st;
    int dev = 0;
    AG_CUDA(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *status = device_status_word(dev);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    Scratch sc(s, dev);
    AssetScratch a;
    memset(&a, 0, sizeof(a));
    if ((st = alloc_asset(sc, n_lverts, n_lfaces, W, H, true, a))) return st;
    void *scr;
    AG_CUDA(sc.alloc(&scr, backproject_scratch_bytes(n_views, w, hgt, o.filter)));
    if ((st = run_prep(d_lverts, d_lnormals, d_luv, d_lfaces, n_lverts, n_lfaces, W, H, o.ray_tile, nullptr, status, a,
                       s)))
        return st;
    AG_CUDA(launch_backproject(a.lpos, a.lnrm, a.lface, d_luv, a.rays, a.n_rays, W, H, h_cams, centres.data(),
                               logw.data(), n_views,
                               d_images, d_depth, d_edge, w, hgt, alpha, eps, depth_tol, o.filter, AG_LOD_BIAS,
                               AG_MAX_TAPS, AG_SHARPEN, reinterpret_cast<float4 *>(d_texture), d_incidence, scr, s));
    return AG_OK;   // the pageable copies of the cameras and log-weights were staged before returning
}

AG_API ag_status ag_sync_status(ag_stream_t stream) {
    g_err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    AG_CUDA(cudaStreamSynchronize(s));
    int dev = 0;
    AG_CUDA(cudaGetDevice(&dev));
    unsigned *w = device_status_word(dev);
    if (!w) return set_error(AG_ERR_OOM, "status word allocation failed");
    unsigned word = 0;
    AG_CUDA(cudaMemcpy(&word, w, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (word) AG_CUDA(cudaMemset(w, 0, sizeof(unsigned)));
    if (word & (AGS_STEP_CAP | AGS_STACK))
        return set_error(AG_ERR_TRAVERSAL_LIMIT, "traversal limit reached (%s%s)",
                         (word & AGS_STEP_CAP) ? "step cap " : "", (word & AGS_STACK) ? "stack overflow" : "");
    if (word & (AGS_BAD_UV | AGS_BAD_FACE))
        return set_error(AG_ERR_INVALID_ARG, "invalid input seen on the device (%s%s)",
                         (word & AGS_BAD_UV) ? "UV outside [-1,2] or NaN / bad low face index " : "",
                         (word & AGS_BAD_FACE) ? "high face index out of range" : "");
    return AG_OK;
}

}  // extern "C"
