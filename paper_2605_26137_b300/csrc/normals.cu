// Area-weighted smooth vertex normals (Sec. 6.4: the G-buffer's "smooth
// normal" of the low-poly mesh and the high-poly "interpolated smooth
// normal"), computed deterministically and accurately in FP32:
//   - each face term (v1 - v0) x (v2 - v0) uses exact edge differences
//     (TwoSum: hi + lo) and a compensated 2x2 determinant (FMA error term), so
//     sliver triangles of marching-grid meshes keep a correct direction;
//   - each vertex sums its incident face terms in face-id order through a
//     CSR adjacency (degree count, exclusive scan, fill, per-vertex sort), so
//     the result does not depend on scheduling (no float atomics).
#include "ag_internal.cuh"
#include "exact.cuh"


namespace ag {

namespace {

__device__ __forceinline__ float3 ldv(const float *V, int64_t i) {
    return make_float3(V[3 * i], V[3 * i + 1], V[3 * i + 2]);
}

__device__ __forceinline__ bool face_ok(const int32_t *F, int64_t f, int64_t nv, int32_t id[3]) {
    id[0] = F[3 * f]; id[1] = F[3 * f + 1]; id[2] = F[3 * f + 2];
    return id[0] >= 0 && id[0] < nv && id[1] >= 0 && id[1] < nv && id[2] >= 0 && id[2] < nv;
}

__global__ void k_degree(const int32_t *__restrict__ F, int64_t nf, int64_t nv, unsigned *__restrict__ deg) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int32_t id[3];
    if (!face_ok(F, f, nv, id)) return;
    for (int k = 0; k < 3; ++k) atomicAdd(&deg[id[k]], 1u);
}

__global__ void k_fill(const int32_t *__restrict__ F, int64_t nf, int64_t nv, const unsigned *__restrict__ off,
                       unsigned *__restrict__ fill, int32_t *__restrict__ list) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int32_t id[3];
    if (!face_ok(F, f, nv, id)) return;
    for (int k = 0; k < 3; ++k) {
        unsigned slot = atomicAdd(&fill[id[k]], 1u);
        list[off[id[k]] + slot] = (int32_t)f;
    }
}

__global__ void k_gather(const float *__restrict__ V, const int32_t *__restrict__ F, int64_t nv,
                         const unsigned *__restrict__ off, int32_t *__restrict__ list, const float *__restrict__ given,
                         float *__restrict__ acc_out, float4 *__restrict__ nrm, float4 *__restrict__ pos) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    float3 s = make_float3(0.f, 0.f, 0.f);
    if (!given) {
        const unsigned b = off[v], e = off[v + 1];
        constexpr unsigned CAP = 32;
        if (e - b <= CAP) {
            // this vertex's faces sorted by id in a local list (written back:
            // the list leaves this kernel sorted either way)
            int32_t fl[CAP];
            unsigned n = 0;
            for (unsigned i = b; i < e; ++i) {
                const int32_t x = list[i];
                unsigned j = n++;
                while (j > 0 && fl[j - 1] > x) { fl[j] = fl[j - 1]; --j; }
                fl[j] = x;
            }
            for (unsigned i = 0; i < n; ++i) {
                list[b + i] = fl[i];
                const int64_t f = fl[i];
                const float3 c = face_cross(ldv(V, F[3 * f]), ldv(V, F[3 * f + 1]), ldv(V, F[3 * f + 2]));
                s = make_float3(__fadd_rn(s.x, c.x), __fadd_rn(s.y, c.y), __fadd_rn(s.z, c.z));
            }
        } else {
            // insertion sort of the faces by id in place
            for (unsigned i = b + 1; i < e; ++i) {
                int32_t x = list[i];
                unsigned j = i;
                while (j > b && list[j - 1] > x) { list[j] = list[j - 1]; --j; }
                list[j] = x;
            }
            for (unsigned i = b; i < e; ++i) {
                int64_t f = list[i];
                float3 c = face_cross(ldv(V, F[3 * f]), ldv(V, F[3 * f + 1]), ldv(V, F[3 * f + 2]));
                s = make_float3(__fadd_rn(s.x, c.x), __fadd_rn(s.y, c.y), __fadd_rn(s.z, c.z));
            }
        }
    } else {
        s = ldv(given, v);
    }
    if (acc_out) {
        acc_out[3 * v] = s.x;
        acc_out[3 * v + 1] = s.y;
        acc_out[3 * v + 2] = s.z;
    }
    float3 n = normalize3(s);
    nrm[v] = make_float4(n.x, n.y, n.z, 0.f);
    if (pos) {
        float3 p = ldv(V, v);
        pos[v] = make_float4(p.x, p.y, p.z, 0.f);
    }
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

size_t vertex_normal_scratch_bytes(int64_t nv, int64_t nf) {
    return sizeof(unsigned) * (size_t)(2 * nv + 1) + sizeof(int32_t) * (size_t)(3 * nf) + scan_scratch_bytes(nv);
}

cudaError_t launch_vertex_normals(const float *V, const int32_t *F, int64_t nv, int64_t nf, const float *given,
                                  float *acc_out, float4 *nrm, float4 *pos, void *scratch, cudaStream_t s) {
    unsigned *off = static_cast<unsigned *>(scratch);   // [nv+1]
    unsigned *fill = off + nv + 1;                      // [nv]
    int32_t *list = reinterpret_cast<int32_t *>(fill + nv);  // [3nf]
    unsigned *scan_tmp = reinterpret_cast<unsigned *>(list + 3 * nf);
    cudaError_t e;
    if (!given) {
        if ((e = cudaMemsetAsync(off, 0, sizeof(unsigned) * (size_t)(2 * nv + 1), s)) != cudaSuccess) return e;
        k_degree<<<grid_for(nf, 256), 256, 0, s>>>(F, nf, nv, off);
        if ((e = launch_scan_exclusive(off, nv, off + nv, scan_tmp, s)) != cudaSuccess) return e;
        k_fill<<<grid_for(nf, 256), 256, 0, s>>>(F, nf, nv, off, fill, list);
    }
    k_gather<<<grid_for(nv, 128), 128, 0, s>>>(V, F, nv, off, list, given, acc_out, nrm, pos);
    return cudaGetLastError();
}

cudaError_t launch_vertex_face_csr(const int32_t *F, int64_t nf, int64_t nv, void *scratch, const unsigned **off_out,
                                   const int32_t **list_out, cudaStream_t s) {
    unsigned *off = static_cast<unsigned *>(scratch);   // [nv+1]
    unsigned *fill = off + nv + 1;                      // [nv]
    int32_t *list = reinterpret_cast<int32_t *>(fill + nv);  // [3nf]
    unsigned *scan_tmp = reinterpret_cast<unsigned *>(list + 3 * nf);
    cudaError_t e;
    if ((e = cudaMemsetAsync(off, 0, sizeof(unsigned) * (size_t)(2 * nv + 1), s)) != cudaSuccess) return e;
    k_degree<<<grid_for(nf, 256), 256, 0, s>>>(F, nf, nv, off);
    if ((e = launch_scan_exclusive(off, nv, off + nv, scan_tmp, s)) != cudaSuccess) return e;
    k_fill<<<grid_for(nf, 256), 256, 0, s>>>(F, nf, nv, off, fill, list);
    *off_out = off;
    *list_out = list;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Vertex normals without any allocation, for callers that cannot allocate
// device memory themselves or through this library (see
// ag_vertex_normals_noalloc in include/ag.h).  The adjacency scratch lives in
// one file-scope device array, sized for the limits below; every device that
// loads this library keeps it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t NOALLOC_MAX_VERTS = 1 << 17;  // 131,072 vertices
constexpr int64_t NOALLOC_MAX_FACES = 1 << 18;  // 262,144 triangles
// adjacency of vertex_normal_scratch_bytes(NOALLOC_MAX_VERTS, NOALLOC_MAX_FACES): offsets, fill
// counters, face lists, and the prefix-sum chunk totals (2048 counts per chunk)
constexpr size_t NOALLOC_SCRATCH_BYTES = sizeof(unsigned) * (size_t)(2 * NOALLOC_MAX_VERTS + 1) +
                                         sizeof(int32_t) * (size_t)(3 * NOALLOC_MAX_FACES) +
                                         sizeof(unsigned) * (size_t)((NOALLOC_MAX_VERTS + 2047) / 2048 + 1);

// shared by every call: calls that overlap on the GPU (two streams, or two
// host threads) race on it
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the array on the current device.  In host code the
// symbol g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up with the device current, on every call: nothing is cached, so a
// new context on the device (after cudaDeviceReset, say) gets its own
// address rather than a stale one.
ag_status noalloc_scratch_on_current_device(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_error(e, "ag_vertex_normals_noalloc: cudaGetSymbolAddress");
    *out = p;
    return AG_OK;
}

}  // namespace
}  // namespace ag

extern "C" AG_API ag_status ag_vertex_normals_noalloc(const float *d_verts, int64_t n_verts, const int32_t *d_faces,
                                                      int64_t n_faces, float *d_normals, ag_stream_t stream) {
    using namespace ag;
    if (!d_verts || !d_faces || !d_normals)
        return set_error(AG_ERR_INVALID_ARG, "ag_vertex_normals_noalloc: pointers must be non-NULL");
    if (n_verts < 3 || n_verts > NOALLOC_MAX_VERTS)
        return set_error(AG_ERR_INVALID_ARG, "ag_vertex_normals_noalloc: n_verts must be in 3..%lld (static scratch limit)",
                         (long long)NOALLOC_MAX_VERTS);
    if (n_faces < 1 || n_faces > NOALLOC_MAX_FACES)
        return set_error(AG_ERR_INVALID_ARG, "ag_vertex_normals_noalloc: n_faces must be in 1..%lld (static scratch limit)",
                         (long long)NOALLOC_MAX_FACES);
    if (reinterpret_cast<uintptr_t>(d_normals) % 16)
        return set_error(AG_ERR_INVALID_ARG, "ag_vertex_normals_noalloc: d_normals must be 16-byte aligned");
    void *scratch = nullptr;
    ag_status st = noalloc_scratch_on_current_device(&scratch);
    if (st != AG_OK) return st;
    if (vertex_normal_scratch_bytes(n_verts, n_faces) > NOALLOC_SCRATCH_BYTES)
        return set_error(AG_ERR_INVALID_ARG, "ag_vertex_normals_noalloc: mesh exceeds the static scratch");
    // the degree/offset/fill counters are cleared inside (they must start at zero)
    cudaError_t e = launch_vertex_normals(d_verts, d_faces, n_verts, n_faces, nullptr, nullptr,
                                          reinterpret_cast<float4 *>(d_normals), nullptr, scratch,
                                          (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(e, "ag_vertex_normals_noalloc");
    return AG_OK;
}
