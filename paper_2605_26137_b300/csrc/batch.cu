// Batched bake: many independent assets, one persistent traversal launch over
// the concatenation of their ray lists (a global work queue), optionally
// captured once into a CUDA graph and replayed.
#include "ag_internal.cuh"

#include <cstring>
#include <mutex>
#include <new>
#include <vector>

namespace ag {
namespace {

constexpr uint64_t PLAN_MAGIC = 0x414742415443484full;

__global__ void k_job_begin(const long long *const *__restrict__ counts, int n, long long *__restrict__ begin) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long run = 0;
    for (int a = 0; a < n; ++a) {
        begin[a] = run;
        run += *counts[a];
    }
    begin[n] = run;
}

struct Arena {
    char *base = nullptr;
    size_t off = 0, cap = 0;
    template <class T>
    T *take(size_t count) {
        size_t bytes = (sizeof(T) * count + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

struct AssetBufs {
    float *acc;
    float4 *lpos, *lnrm, *ltan, *ntsd;
    int4 *lface, *uvfix, *rays;
    unsigned long long *keys;
    int32_t *face;
    long long *n_rays;
    char *nscr;
};

// lays out (or measures, when ar.base is NULL) every buffer of the batch
void layout_batch(Arena &ar, int n, const ag_asset_desc *d, std::vector<AssetBufs> &bufs, TraceJob **jobs,
                  long long **begin, const long long ***counts, unsigned long long **ray_counter) {
    bufs.resize(n);
    for (int a = 0; a < n; ++a) {
        size_t hw = (size_t)d[a].W * d[a].H;
        AssetBufs &b = bufs[a];
        b.acc = ar.take<float>(3 * d[a].n_lverts);
        b.lpos = ar.take<float4>(d[a].n_lverts);
        b.lnrm = ar.take<float4>(d[a].n_lverts);
        b.ltan = ar.take<float4>(3 * d[a].n_lfaces);
        b.lface = ar.take<int4>(d[a].n_lfaces);
        b.uvfix = ar.take<int4>(2 * d[a].n_lfaces);
        b.keys = ar.take<unsigned long long>(hw);
        b.face = ar.take<int32_t>(hw);
        b.rays = ar.take<int4>(hw);
        b.ntsd = ar.take<float4>(hw);
        b.n_rays = ar.take<long long>(2);
        b.nscr = ar.take<char>(vertex_normal_scratch_bytes(d[a].n_lverts, d[a].n_lfaces));
    }
    *jobs = ar.take<TraceJob>(n);
    *begin = ar.take<long long>(n + 1);
    *counts = ar.take<const long long *>(n);
    *ray_counter = ar.take<unsigned long long>(1);
}

ag_status check_descs(int n, const ag_asset_desc *d, int *layout) {
    if (n < 1 || n > 4096) return set_error(AG_ERR_INVALID_ARG, "n_assets must be in 1..4096");
    if (!d) return set_error(AG_ERR_INVALID_ARG, "descs must be non-NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    for (int a = 0; a < n; ++a) {
        const ag_asset_desc &x = d[a];
        if (!x.bvh || x.bvh->magic != AG_BVH_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "asset %d: invalid BVH handle", a);
        if (x.bvh->device != dev) return set_error(AG_ERR_INVALID_ARG, "asset %d: handle on another device", a);
        if (x.bvh->layout != AG_BVH_Q8) {   // FP32 nodes: the job needs the scene box
            ag_status st = bvh_ready(x.bvh);
            if (st) return st;
        }
        if (a == 0) *layout = x.bvh->layout;
        else if (x.bvh->layout != *layout)
            return set_error(AG_ERR_INVALID_ARG, "asset %d: all BVHs of a batch must share one layout", a);
        if (!x.lverts || !x.luv || !x.lfaces) return set_error(AG_ERR_INVALID_ARG, "asset %d: NULL low mesh pointer", a);
        if (x.n_lverts < 3 || x.n_lverts >= (1ll << 31) || x.n_lfaces < 1 || x.n_lfaces >= (1ll << 31))
            return set_error(AG_ERR_INVALID_ARG, "asset %d: mesh size out of range", a);
        if (x.W < 1 || x.H < 1 || x.W > 16384 || x.H > 16384)
            return set_error(AG_ERR_INVALID_ARG, "asset %d: W and H must be in 1..16384", a);
        if (!(x.max_dist > 0.f) || !(x.max_dist < 3.0e38f))
            return set_error(AG_ERR_INVALID_ARG, "asset %d: max_dist must be positive and finite", a);
        if (!x.normal_rgba8 || !x.mask || !x.disp) return set_error(AG_ERR_INVALID_ARG, "asset %d: NULL output", a);
    }
    return AG_OK;
}

ag_status check_opts_batch(const ag_opts &o) {
    if (o.gutter < 0 || o.gutter > 8) return set_error(AG_ERR_INVALID_ARG, "gutter must be in 0..8");
    if (o.block_size != 0 && (o.block_size < 64 || o.block_size > 1024 || o.block_size % 32))
        return set_error(AG_ERR_INVALID_ARG, "block_size must be 0 or a multiple of 32 in 64..1024");
    if (o.blocks_per_sm < 0 || o.blocks_per_sm > 64) return set_error(AG_ERR_INVALID_ARG, "blocks_per_sm out of range");
    if (o.max_steps < 0) return set_error(AG_ERR_INVALID_ARG, "max_steps must be >= 0");
    if (o.schedule < AG_SCHED_AUTO || o.schedule > AG_SCHED_COOP2) return set_error(AG_ERR_INVALID_ARG, "unknown schedule");
    if (o.ray_tile < AG_TILE_8x8 || o.ray_tile > AG_TILE_4x4) return set_error(AG_ERR_INVALID_ARG, "unknown ray tile");
    if (o.query != AG_QUERY_RAY && o.query != AG_QUERY_CLOSEST)
        return set_error(AG_ERR_INVALID_ARG, "query must be AG_QUERY_RAY or AG_QUERY_CLOSEST");
    return AG_OK;
}

// host-side job table + count pointer table for the device arena
void fill_tables(int n, const ag_asset_desc *d, const std::vector<AssetBufs> &b, std::vector<TraceJob> &jobs,
                 std::vector<const long long *> &counts) {
    jobs.resize(n);
    counts.resize(n);
    for (int a = 0; a < n; ++a) {
        TraceJob &j = jobs[a];
        memset(&j, 0, sizeof(j));
        ag_bvh_t h = d[a].bvh;
        j.nodes = h->nodes;
        j.tris = h->tris;
        j.tri_ids = h->tri_ids;
        j.hnormals = h->vnormals;
        j.lpos = b[a].lpos;
        j.lnrm = b[a].lnrm;
        j.lface = b[a].lface;
        j.ltan = b[a].ltan;
        j.rays = b[a].rays;
        j.ntsd = b[a].ntsd;
        j.mask = d[a].mask;
        j.W = d[a].W;
        j.H = d[a].H;
        j.max_dist = d[a].max_dist;
        scene_abs_for(h, &j.scene_abs);   // ready: check_descs waited for FP32-node builds
        counts[a] = b[a].n_rays;
    }
}

// enqueue the whole batch on s (capturable: kernels, memsets and event edges)
ag_status enqueue_batch(int n, const ag_asset_desc *d, const ag_opts &o, int layout, const std::vector<AssetBufs> &b,
                        const TraceJob *host_jobs, const TraceJob *jobs, long long *begin,
                        const long long *const *counts, unsigned long long *ray_counter, unsigned *status,
                        cudaStream_t s, int dev) {
    cudaStream_t *side = nullptr;
    AG_CUDA(side_streams(dev, &side));
    const int used = n < N_SIDE ? n : N_SIDE;
    EventSet es;
    AG_CUDA(fork_to(s, side, used, es));
    for (int a = 0; a < n; ++a) {
        const AssetBufs &x = b[a];
        cudaStream_t q = side[a % N_SIDE];
        AG_CUDA(cudaMemsetAsync(x.n_rays, 0, sizeof(long long) * 2, q));
        AG_CUDA(launch_vertex_normals(d[a].lverts, d[a].lfaces, d[a].n_lverts, d[a].n_lfaces, d[a].lnormals, x.acc,
                                      x.lnrm, x.lpos, x.nscr, q));
        AG_CUDA(launch_face_setup(d[a].luv, d[a].lfaces, d[a].n_lfaces, d[a].n_lverts, d[a].W, d[a].H, x.lpos, x.lnrm,
                                  x.lface, x.ltan, x.uvfix, status, q));
        AG_CUDA(launch_raster(x.uvfix, d[a].n_lfaces, d[a].W, d[a].H, x.keys, q));
        AG_CUDA(launch_resolve(x.keys, x.uvfix, d[a].W, d[a].H, o.ray_tile, x.face, nullptr, x.rays, x.n_rays, q));
    }
    AG_CUDA(join_from(s, side, used, es));
    TraceLaunch L;
    memset(&L, 0, sizeof(L));
    if (n == 1) {
        L.job0 = host_jobs[0];
        L.n_jobs = 1;
        L.n_rays_dev = b[0].n_rays;
    } else {
        k_job_begin<<<1, 32, 0, s>>>(counts, n, begin);
        AG_CUDA_LAUNCH("k_job_begin");
        L.jobs = jobs;
        L.job_begin = begin;
        L.n_jobs = n;
        L.n_rays_dev = begin + n;
    }
    L.ray_counter = ray_counter;
    L.status = status;
    L.max_steps = o.max_steps > 0 ? o.max_steps : (1 << 20);
    L.layout = layout;
    L.schedule = o.schedule == AG_SCHED_AUTO ? AG_SCHED_BATCH : o.schedule;
    L.query = o.query;
    L.block_size = o.block_size;
    L.blocks_per_sm = o.blocks_per_sm;
    L.backward = false;
    AG_CUDA(launch_trace(L, s));
    AG_CUDA(fork_to(s, side, used, es));
    for (int a = 0; a < n; ++a)
        AG_CUDA(launch_finalize(b[a].ntsd, b[a].face, d[a].W, d[a].H, o.gutter, o.disp_fp16, d[a].normal_rgba8,
                                d[a].mask, d[a].disp, nullptr, nullptr, nullptr, nullptr, side[a % N_SIDE]));
    AG_CUDA(join_from(s, side, used, es));
    return AG_OK;
}

ag_opts batch_opts(const ag_opts *p) {
    ag_opts o;
    ag_opts_default(&o);
    if (p) o = *p;
    return o;
}

}  // namespace
}  // namespace ag

struct ag_batch_plan {
    uint64_t magic;
    int device;
    int n;
    void *arena;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

using namespace ag;

extern "C" {

AG_API ag_status ag_bake_batch(int32_t n_assets, const ag_asset_desc *descs, const ag_opts *opts, ag_stream_t stream) {
    int layout = 0;
    ag_status st = check_descs(n_assets, descs, &layout);
    if (st) return st;
    ag_opts o = batch_opts(opts);
    if ((st = check_opts_batch(o))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = descs[0].bvh->device;
    unsigned *status = device_status_word(dev);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    std::vector<AssetBufs> bufs;
    TraceJob *jobs;
    long long *begin;
    const long long **counts;
    unsigned long long *ray_counter;
    Arena measure;
    layout_batch(measure, n_assets, descs, bufs, &jobs, &begin, &counts, &ray_counter);
    Scratch sc(s, dev);
    Arena ar;
    AG_CUDA(sc.alloc((void **)&ar.base, measure.off));
    ar.cap = measure.off;
    layout_batch(ar, n_assets, descs, bufs, &jobs, &begin, &counts, &ray_counter);
    std::vector<TraceJob> hj;
    std::vector<const long long *> hc;
    fill_tables(n_assets, descs, bufs, hj, hc);
    AG_CUDA(cudaMemcpyAsync(jobs, hj.data(), sizeof(TraceJob) * n_assets, cudaMemcpyHostToDevice, s));
    AG_CUDA(cudaMemcpyAsync((void *)counts, hc.data(), sizeof(void *) * n_assets, cudaMemcpyHostToDevice, s));
    return enqueue_batch(n_assets, descs, o, layout, bufs, hj.data(), jobs, begin, counts, ray_counter, status, s, dev);
}

AG_API ag_status ag_batch_plan_create(int32_t n_assets, const ag_asset_desc *descs, const ag_opts *opts,
                                      ag_stream_t stream, ag_batch_plan_t *out) {
    if (!out) return set_error(AG_ERR_INVALID_ARG, "out must be non-NULL");
    *out = nullptr;
    int layout = 0;
    ag_status st = check_descs(n_assets, descs, &layout);
    if (st) return st;
    ag_opts o = batch_opts(opts);
    if ((st = check_opts_batch(o))) return st;
    int dev = descs[0].bvh->device;
    unsigned *status = device_status_word(dev);
    if (!status) return set_error(AG_ERR_OOM, "status word allocation failed");
    std::vector<AssetBufs> bufs;
    TraceJob *jobs;
    long long *begin;
    const long long **counts;
    unsigned long long *ray_counter;
    Arena measure;
    layout_batch(measure, n_assets, descs, bufs, &jobs, &begin, &counts, &ray_counter);
    ag_batch_plan *p = new (std::nothrow) ag_batch_plan;
    if (!p) return set_error(AG_ERR_OOM, "host allocation failed");
    memset(p, 0, sizeof(*p));
    p->device = dev;
    p->n = n_assets;
    cudaError_t e = cudaMalloc(&p->arena, measure.off);
    if (e != cudaSuccess) { delete p; return cuda_error(e, "batch arena"); }
    Arena ar;
    ar.base = (char *)p->arena;
    ar.cap = measure.off;
    layout_batch(ar, n_assets, descs, bufs, &jobs, &begin, &counts, &ray_counter);
    std::vector<TraceJob> hj;
    std::vector<const long long *> hc;
    fill_tables(n_assets, descs, bufs, hj, hc);
    cudaStream_t cap = nullptr;
    e = cudaMemcpy(jobs, hj.data(), sizeof(TraceJob) * n_assets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy((void *)counts, hc.data(), sizeof(void *) * n_assets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        if (cap) cudaStreamDestroy(cap);
        cudaFree(p->arena);
        delete p;
        return cuda_error(e, "batch plan capture setup");
    }
    st = enqueue_batch(n_assets, descs, o, layout, bufs, hj.data(), jobs, begin, counts, ray_counter, status, cap, dev);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st == AG_OK && e != cudaSuccess) st = cuda_error(e, "cudaStreamEndCapture");
    if (st == AG_OK) {
        e = cudaGraphInstantiate(&p->exec, g, 0);
        if (e != cudaSuccess) st = cuda_error(e, "cudaGraphInstantiate");
    }
    if (st != AG_OK) {
        if (g) cudaGraphDestroy(g);
        cudaFree(p->arena);
        delete p;
        return st;
    }
    p->graph = g;
    p->magic = PLAN_MAGIC;
    (void)stream;
    *out = p;
    return AG_OK;
}

AG_API ag_status ag_batch_plan_launch(ag_batch_plan_t p, ag_stream_t stream) {
    if (!p || p->magic != PLAN_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "invalid batch plan");
    AG_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    return AG_OK;
}

AG_API ag_status ag_batch_plan_free(ag_batch_plan_t p) {
    if (!p) return AG_OK;
    if (p->magic != PLAN_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "invalid batch plan");
    cudaDeviceSynchronize();
    cudaGraphExecDestroy(p->exec);
    cudaGraphDestroy(p->graph);
    cudaFree(p->arena);
    p->magic = 0;
    delete p;
    return AG_OK;
}

}  // extern "C"
