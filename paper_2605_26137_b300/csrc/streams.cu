// Library-owned side streams and the fork/join event edges that let small
// independent kernels of one call overlap (captured into a graph, they become
// independent branches).
#include "ag_internal.cuh"

#include <mutex>

namespace ag {
namespace {
constexpr int MAX_DEV = 64;
std::mutex g_side_mu;
cudaStream_t g_side[MAX_DEV][N_SIDE] = {};
}  // namespace

cudaError_t side_streams(int dev, cudaStream_t **out) {
    if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_side_mu);
    if (!g_side[dev][0]) {
        for (int k = 0; k < N_SIDE; ++k) {
            cudaError_t e = cudaStreamCreateWithFlags(&g_side[dev][k], cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
        }
    }
    *out = g_side[dev];
    return cudaSuccess;
}

EventSet::~EventSet() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
}

cudaError_t EventSet::make(cudaEvent_t *e) {
    cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    if (r == cudaSuccess) ev.push_back(*e);
    return r;
}

cudaError_t fork_to(cudaStream_t s, cudaStream_t *side, int n_used, EventSet &es) {
    cudaEvent_t f;
    cudaError_t e = es.make(&f);
    if (e == cudaSuccess) e = cudaEventRecord(f, s);
    for (int k = 0; k < n_used && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(side[k], f, 0);
    return e;
}

cudaError_t join_from(cudaStream_t s, cudaStream_t *side, int n_used, EventSet &es) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n_used && e == cudaSuccess; ++k) {
        cudaEvent_t j;
        e = es.make(&j);
        if (e == cudaSuccess) e = cudaEventRecord(j, side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, j, 0);
    }
    return e;
}

}  // namespace ag
