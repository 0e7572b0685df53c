// Launch-configuration autotuner: times whole bakes of the caller's asset for
// every candidate (schedule x trace block size x ray tile) and keeps the
// fastest.  The traversal result does not depend on the configuration.
#include "ag_internal.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

using namespace ag;

extern "C" AG_API ag_status ag_autotune(ag_bvh_t h, const float *d_lverts, const float *d_lnormals, const float *d_luv,
                                        const int32_t *d_lfaces, int64_t n_lverts, int64_t n_lfaces, int32_t W,
                                        int32_t H, float max_dist, ag_stream_t stream, ag_opts *inout,
                                        float *best_ms) {
    if (!inout) return set_error(AG_ERR_INVALID_ARG, "inout must be non-NULL");
    if (!h || h->magic != AG_BVH_MAGIC) return set_error(AG_ERR_BAD_HANDLE, "invalid BVH handle");
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return set_error(AG_ERR_INVALID_ARG, "W and H must be in 1..16384");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s, h->device);
    uint8_t *rgba, *mask;
    void *disp;
    size_t hw = (size_t)W * H;
    AG_CUDA(sc.alloc((void **)&rgba, 4 * hw));
    AG_CUDA(sc.alloc((void **)&mask, hw));
    AG_CUDA(sc.alloc(&disp, 2 * hw));
    cudaEvent_t e0, e1;
    AG_CUDA(cudaEventCreate(&e0));
    AG_CUDA(cudaEventCreate(&e1));
    // candidates: the one-ray-per-thread schedules at three block sizes, and
    // the warp-cooperative ones (fixed 128-thread blocks; forward ray bake
    // over 8-bit nodes only), each with every ray tile
    struct Cand { int schedule, block; };
    Cand cands[8];
    int n_cand = 0;
    const int blocks[3] = {64, 128, 256};
    for (int bi = 0; bi < 3; ++bi) cands[n_cand++] = {AG_SCHED_BATCH, blocks[bi]};
    if (inout->query != AG_QUERY_CLOSEST) {   // the closest-point query has one schedule
        for (int bi = 0; bi < 3; ++bi) cands[n_cand++] = {AG_SCHED_REFILL, blocks[bi]};
        if (h->layout == AG_BVH_Q8) {
            cands[n_cand++] = {AG_SCHED_COOP2, 0};
            cands[n_cand++] = {AG_SCHED_COOP4, 0};
        }
    }
    const int tiles[4] = {AG_TILE_8x8, AG_TILE_16x16, AG_TILE_32x8, AG_TILE_4x4};
    ag_opts best = *inout;
    float best_t = 3.0e38f;
    ag_status st = AG_OK;
    for (int ci = 0; ci < n_cand && st == AG_OK; ++ci)
        for (int ti = 0; ti < 4 && st == AG_OK; ++ti) {
            ag_opts o = *inout;
            o.schedule = cands[ci].schedule;
            o.block_size = cands[ci].block;
            o.blocks_per_sm = 0;
            o.ray_tile = tiles[ti];
            o.disp_fp16 = 1;
            float ts[3];
            for (int rep = 0; rep < 4 && st == AG_OK; ++rep) {
                if (rep) cudaEventRecord(e0, s);
                st = ag_bake(h, d_lverts, d_lnormals, d_luv, d_lfaces, n_lverts, n_lfaces, W, H, max_dist, &o,
                             stream, rgba, mask, disp, nullptr);
                if (rep && st == AG_OK) {
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ts[rep - 1], e0, e1);
                }
            }
            if (st != AG_OK) break;
            std::sort(ts, ts + 3);
            if (ts[1] < best_t) {
                best_t = ts[1];
                best = o;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != AG_OK) return st;
    AG_CUDA(cudaStreamSynchronize(s));
    inout->schedule = best.schedule;
    inout->block_size = best.block_size;
    inout->blocks_per_sm = 0;
    inout->ray_tile = best.ray_tile;
    if (best_ms) *best_ms = best_t;
    return AG_OK;
}
