// lf_find_tracks_static: the persistent form for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: a host process whose device
// memory is entirely owned by its own pool or arena, code on a hard-latency
// path where cudaMalloc/cudaFree (cudaFree synchronises the whole device)
// are not acceptable, or an embedding framework that forbids allocation
// after start-up.  They cannot create an lf_ctx (lf_create allocates its
// status word and work-queue cursor).  This entry point takes no context:
// the scratch of the persistent kernel (the work-queue cursor and the
// per-event found counts of the compaction) lives in one file-scope device
// array of fixed size that every GPU loading the library holds until exit.
//
// Host code never names the array as a device address.  On the first call on
// a device (with that device current) the entry point looks its address up
// with cudaGetSymbolAddress, checks the result and keeps it per device; that
// first call should therefore be made before any stream capture.  Every call
// shares the array: the cursor is cleared at the start of each call and the
// per-event counts are fully rewritten, and calls that overlap on the GPU
// race on it.
#include <mutex>

#include "lf.h"
#include "lf_internal.h"

namespace {

constexpr int kScratchHead = 64;  // [0]: work-queue cursor; the rest pads to 256 bytes

// the only scratch of lf_find_tracks_static: cursor, then per-event counts
static __device__ __align__(256) int g_static_scratch[kScratchHead + LF_STATIC_MAX_EVENTS];

constexpr int kMaxDevices = 256;
int* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup;

// address of g_static_scratch on the current device, looked up once per device
lf_status scratch_address(int** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LF_ERR_INTERNAL;
    std::lock_guard<std::mutex> lock(g_setup);
    if (!g_scratch_addr[dev]) {
        int* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_static_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return LF_ERR_CUDA;
        }
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return LF_OK;
}

}  // namespace

extern "C" lf_status lf_find_tracks_static(const lf_geometry* geometry, const lf_params* params, const lf_batch* b,
                                           const lf_output* o, void* stream) {
    if (!geometry || !params || !b || !o) return LF_ERR_ARG;
    if (b->n_events > LF_STATIC_MAX_EVENTS) return LF_ERR_CAPACITY;
    if (b->n_events < 0 || b->n_tracks < 0 || b->n_hits < 0) return LF_ERR_ARG;
    char msg[256];
    if (lfk::param_error(geometry, params, msg, sizeof msg)) return LF_ERR_ARG;
    if (params->no_ut != 0) return LF_ERR_ARG;  // the tile kernel follows VELO-UT input only
    if (!b->hit_offsets || !b->trk_offsets || !o->out_offsets || !o->n_out) return LF_ERR_ARG;
    if (b->n_hits > 0 && (!b->x || !b->z || !b->dxdy || !b->w)) return LF_ERR_ARG;
    if (b->n_tracks > 0 && (!b->sx || !b->sy || !b->stx || !b->sty || !b->sqop || !o->found || !o->nhits ||
                            !o->hit_idx || !o->state || !o->quality || !o->out_trk))
        return LF_ERR_ARG;
    int* scratch = nullptr;
    lf_status st = scratch_address(&scratch);
    if (st != LF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const lfk::KParams k = lfk::make_kparams(geometry, params);
    int dev = 0, n_sm = 0, bps = 0;
    // block tiles with stage barriers (grain bit 4); tracks per warp follow
    // n_triplets (two, 16 lanes each, when n_triplets <= 16), as in
    // lf_find_tracks_batched with queue 1
    const int wpb = 8, grain = 16;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LF_ERR_CUDA;
    if (lfk::fused_max_blocks_per_sm(k, wpb, grain, &bps) != cudaSuccess || bps < 1) return LF_ERR_CUDA;
    int* cursor = scratch;
    int* ev_count = scratch + kScratchHead;
    if (cudaMemsetAsync(cursor, 0, sizeof(int), s) != cudaSuccess) return LF_ERR_CUDA;
    lfk::KBatch kb{b->n_events, b->n_hits, b->n_tracks, b->hit_offsets, b->x, b->z, b->dxdy, b->w,
                   b->trk_offsets, b->sx, b->sy, b->stx, b->sty, b->sqop, nullptr, b->x_coarse};
    lfk::KOut ko{o->found, o->nhits, o->hit_idx, o->state, o->quality};
    if (b->n_tracks > 0 && lfk::launch_fused(k, kb, ko, cursor, grain, wpb, bps * n_sm, s) != cudaSuccess)
        return LF_ERR_CUDA;
    if (lfk::launch_compact(b->trk_offsets, o->found, b->n_events, ev_count, o->out_offsets, o->out_trk, o->n_out,
                            s) != cudaSuccess)
        return LF_ERR_CUDA;
    return LF_OK;
}
