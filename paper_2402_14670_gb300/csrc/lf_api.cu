// Host side of the C ABI declared in include/lf.h: context, scratch memory,
// argument checks, launches, and the CUDA graphs of the persistent form.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>

#include "lf.h"
#include "lf_internal.h"

using namespace lfk;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct GraphKey {
    std::tuple<int, int, int, int, int, int, const void*, const void*, const void*, const void*, const void*,
               const void*, const void*> v;
    bool operator<(const GraphKey& o) const { return v < o.v; }
};

}  // namespace

struct lf_ctx {
    lf_geometry g;
    lf_params p;
    KParams kp;
    int device = 0;
    int n_sm = 0;
    char err[512] = {0};
    int* status = nullptr;   // device status word
    int* cursor = nullptr;   // device work-queue cursor
    DevBuf trk_event, wbeg, wcnt, keys, ntrip, cands, ev_count, tmp, big_list;
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        cudaStream_t stream = nullptr;
    };
    std::map<GraphKey, GraphEntry> graphs;
};

namespace {

lf_status fail(lf_ctx* c, lf_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return s;
}

#define LF_CUDA(ctx, call)                                                                          \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(ctx, LF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

lf_status ensure(lf_ctx* c, DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return LF_OK;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);  // synchronises: no call of this context is in flight
        if (e != cudaSuccess) return fail(c, LF_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
        b.p = nullptr;
        b.cap = 0;
    }
    size_t want = bytes + bytes / 8;  // grow with headroom
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LF_ERR_OOM, "scratch allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    }
    b.cap = want;
    return LF_OK;
}

bool finite(float v) { return v == v && v - v == 0.0f; }

lf_status check_params(lf_ctx* c, const lf_geometry* g, const lf_params* p) {
    if (p->n_hits_window < 1 || p->n_hits_window > LF_MAX_WINDOW)
        return fail(c, LF_ERR_ARG, "n_hits_window %d outside 1..%d", p->n_hits_window, LF_MAX_WINDOW);
    if (p->n_triplets < 0 || p->n_triplets > LF_MAX_TRIPLETS)
        return fail(c, LF_ERR_ARG, "n_triplets %d outside 0..%d", p->n_triplets, LF_MAX_TRIPLETS);
    if (p->min_hits < 9 || p->min_hits > 12) return fail(c, LF_ERR_ARG, "min_hits %d outside 9..12", p->min_hits);
    if (g->polarity != 1 && g->polarity != -1) return fail(c, LF_ERR_ARG, "polarity must be +1 or -1");
    for (int l = 0; l < LF_N_LAYERS; ++l)
        if (!finite(g->z[l]) || !finite(g->dxdy[l])) return fail(c, LF_ERR_ARG, "geometry of layer %d not finite", l);
    for (int l = 1; l < LF_N_LAYERS; ++l)
        if (!(g->z[l] > g->z[l - 1])) return fail(c, LF_ERR_ARG, "layer z must increase");
    for (int l = 0; l < LF_N_LAYERS; ++l) {
        bool x = (l % 4 == 0) || (l % 4 == 3);
        if (!x && g->dxdy[l] == 0.0f) return fail(c, LF_ERR_ARG, "stereo layer %d has dxdy 0", l);
    }
    if (!(g->z_magnet < g->z[0])) return fail(c, LF_ERR_ARG, "z_magnet must lie before the first layer");
    if (!(p->magtol_max >= p->magtol_min)) return fail(c, LF_ERR_ARG, "magtol_max < magtol_min");
    if (g->kappa == 0.0f) return fail(c, LF_ERR_ARG, "kappa must be non-zero");
    return LF_OK;
}

KParams make_kparams(const lf_geometry* g, const lf_params* p) {
    KParams k;
    std::memset(&k, 0, sizeof k);
    for (int l = 0; l < NL; ++l) {
        k.z[l] = g->z[l];
        k.dxdy[l] = g->dxdy[l];
    }
    k.z_state = g->z_state;
    k.z_magnet = g->z_magnet;
    k.z_ref = g->z_ref;
    k.kappa = g->kappa;
    k.gamma = g->gamma;
    k.dratio = g->dratio;
    k.polarity = g->polarity;
    k.xtol_c = p->xtol_c;
    k.xtol_p = p->xtol_p;
    k.x_asym = p->x_asym;
    k.uv_tol = p->uv_tol;
    k.cap = p->n_hits_window;
    k.n_trip = p->n_triplets;
    k.min_hits = p->min_hits;
    k.K_first = p->K_first;
    k.K_last = p->K_last;
    k.p_bend = p->p_bend;
    k.magtol_min = p->magtol_min;
    k.magtol_max = p->magtol_max;
    k.magtol_c = p->magtol_c;
    k.magtol_tx = p->magtol_tx;
    k.T_triplet = p->T_triplet;
    k.T_x = p->T_x;
    k.T_uv_scale = p->T_uv_scale;
    k.T_uv_min = p->T_uv_min;
    k.T_ty = p->T_ty;
    k.T_y = p->T_y;
    k.T_Q = p->T_Q;
    for (int i = 0; i < 4; ++i) k.C_n[i] = p->C_n[i];
    volatile float pol = (float)g->polarity;  // binary32 products, as the method forms them
    k.pol_f = pol;
    k.pk = pol * g->kappa;
    k.pg = pol * g->gamma;
    k.D = g->dratio * 1000.0f;
    return k;
}

KBatch to_kbatch(const lf_batch* b) {
    KBatch k;
    k.n_events = b->n_events;
    k.n_hits = b->n_hits;
    k.n_tracks = b->n_tracks;
    k.hit_offsets = b->hit_offsets;
    k.x = b->x;
    k.z = b->z;
    k.dxdy = b->dxdy;
    k.w = b->w;
    k.trk_offsets = b->trk_offsets;
    k.sx = b->sx;
    k.sy = b->sy;
    k.stx = b->stx;
    k.sty = b->sty;
    k.sqop = b->sqop;
    return k;
}

lf_status check_batch(lf_ctx* c, const lf_batch* b) {
    if (!b) return fail(c, LF_ERR_ARG, "batch is NULL");
    if (b->n_events < 0 || b->n_tracks < 0 || b->n_hits < 0) return fail(c, LF_ERR_ARG, "negative size");
    if (!b->hit_offsets || !b->trk_offsets) return fail(c, LF_ERR_ARG, "offsets are NULL");
    if (b->n_hits > 0 && (!b->x || !b->z || !b->dxdy || !b->w)) return fail(c, LF_ERR_ARG, "hit arrays are NULL");
    if (b->n_tracks > 0 && (!b->sx || !b->sy || !b->stx || !b->sty || !b->sqop))
        return fail(c, LF_ERR_ARG, "state arrays are NULL");
    return LF_OK;
}

lf_status check_out(lf_ctx* c, const lf_output* o, int n_tracks) {
    if (!o) return fail(c, LF_ERR_ARG, "output is NULL");
    if (!o->out_offsets || !o->n_out) return fail(c, LF_ERR_ARG, "out_offsets or n_out is NULL");
    if (n_tracks > 0 && (!o->found || !o->nhits || !o->hit_idx || !o->state || !o->quality || !o->out_trk))
        return fail(c, LF_ERR_ARG, "an output array is NULL");
    return LF_OK;
}

KOut to_kout(const lf_output* o) {
    KOut k;
    k.found = o->found;
    k.nhits = o->nhits;
    k.hit_idx = o->hit_idx;
    k.state = o->state;
    k.quality = o->quality;
    return k;
}

lf_status plain_stages(lf_ctx* c, const lf_batch* b, cudaStream_t s) {
    const size_t nt = (size_t)b->n_tracks, NT = (size_t)(c->p.n_triplets > 0 ? c->p.n_triplets : 1);
    lf_status st;
    if ((st = ensure(c, c->trk_event, nt * 4)) != LF_OK) return st;
    if ((st = ensure(c, c->wbeg, nt * NL * 4)) != LF_OK) return st;
    if ((st = ensure(c, c->wcnt, nt * NL)) != LF_OK) return st;
    if ((st = ensure(c, c->keys, nt * NT * 8)) != LF_OK) return st;
    if ((st = ensure(c, c->ntrip, nt)) != LF_OK) return st;
    KBatch kb = to_kbatch(b);
    auto* te = (int*)c->trk_event.p;
    auto* wb = (int*)c->wbeg.p;
    auto* wc = (uint8_t*)c->wcnt.p;
    LF_CUDA(c, launch_track_event(kb, te, s));
    LF_CUDA(c, launch_windows(c->kp, kb, te, wb, wc, s));
    LF_CUDA(c, launch_triplets(c->kp, kb, te, wb, wc, (uint64_t*)c->keys.p, (uint8_t*)c->ntrip.p, s));
    return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_create(const lf_geometry* geometry, const lf_params* params, lf_ctx** out) {
    if (!geometry || !params || !out) return LF_ERR_ARG;
    *out = nullptr;
    lf_ctx* c = new (std::nothrow) lf_ctx();
    if (!c) return LF_ERR_OOM;
    lf_status st = check_params(c, geometry, params);
    if (st != LF_OK) {
        delete c;
        return st;
    }
    c->g = *geometry;
    c->p = *params;
    c->kp = make_kparams(geometry, params);
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return LF_ERR_CUDA;
    }
    if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess || cudaMalloc(&c->cursor, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(c->status);
        cudaFree(c->cursor);
        delete c;
        return LF_ERR_OOM;
    }
    *out = c;
    return LF_OK;
}

void lf_destroy(lf_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    for (auto& kv : c->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    DevBuf* bufs[] = {&c->trk_event, &c->wbeg, &c->wcnt, &c->keys, &c->ntrip,
                      &c->cands, &c->ev_count, &c->tmp, &c->big_list};
    for (DevBuf* b : bufs)
        if (b->p) cudaFree(b->p);
    cudaFree(c->status);
    cudaFree(c->cursor);
    delete c;
}

const char* lf_last_error(const lf_ctx* c) { return c ? c->err : "no context"; }

int32_t lf_device_sm_count(void) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

lf_status lf_pack_hits(lf_ctx* c, const lf_raw_hits* raw, const lf_packed* pk, void* stream) {
    if (!c) return LF_ERR_ARG;
    if (!raw || !pk) return fail(c, LF_ERR_ARG, "raw or packed is NULL");
    if (raw->n_events < 0 || raw->n_hits < 0) return fail(c, LF_ERR_ARG, "negative size");
    if (!raw->raw_offsets || !pk->hit_offsets) return fail(c, LF_ERR_ARG, "offsets are NULL");
    if (raw->n_hits > 0 && (!raw->x || !raw->z || !raw->dxdy || !raw->w || !raw->plane || !pk->x || !pk->z ||
                            !pk->dxdy || !pk->w || !pk->layer || !pk->perm))
        return fail(c, LF_ERR_ARG, "a hit array is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    lf_status st;
    if ((st = ensure(c, c->tmp, (size_t)raw->n_hits * 4)) != LF_OK) return st;
    if ((st = ensure(c, c->big_list, ((size_t)raw->n_events * NB + 1) * 4)) != LF_OK) return st;
    LF_CUDA(c, launch_pack(raw->raw_offsets, raw->x, raw->z, raw->dxdy, raw->w, raw->plane, raw->n_events,
                           raw->n_hits, pk->hit_offsets, pk->x, pk->z, pk->dxdy, pk->w, pk->layer, pk->perm,
                           (int*)c->tmp.p, (int*)c->big_list.p, c->status, c->n_sm, s));
    return LF_OK;
}

lf_status lf_find_tracks(lf_ctx* c, const lf_batch* b, const lf_output* o, void* stream) {
    if (!c) return LF_ERR_ARG;
    lf_status st;
    if ((st = check_batch(c, b)) != LF_OK) return st;
    if ((st = check_out(c, o, b->n_tracks)) != LF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nt = (size_t)b->n_tracks, NT = (size_t)(c->p.n_triplets > 0 ? c->p.n_triplets : 1);
    if ((st = ensure(c, c->cands, nt * NT * sizeof(CandRec))) != LF_OK) return st;
    if ((st = ensure(c, c->ev_count, (size_t)b->n_events * 4)) != LF_OK) return st;
    if ((st = plain_stages(c, b, s)) != LF_OK) return st;
    KBatch kb = to_kbatch(b);
    KOut ko = to_kout(o);
    LF_CUDA(c, launch_extend(c->kp, kb, (int*)c->trk_event.p, (int*)c->wbeg.p, (uint8_t*)c->wcnt.p,
                             (uint64_t*)c->keys.p, (uint8_t*)c->ntrip.p, (CandRec*)c->cands.p, s));
    LF_CUDA(c, launch_select(c->kp, kb, (int*)c->wbeg.p, (uint8_t*)c->ntrip.p, (CandRec*)c->cands.p, ko, s));
    LF_CUDA(c, launch_compact(b->trk_offsets, o->found, b->n_events, (int*)c->ev_count.p, o->out_offsets,
                              o->out_trk, o->n_out, s));
    return LF_OK;
}

lf_status lf_find_tracks_batched(lf_ctx* c, const lf_batch* b, const lf_output* o, const lf_tuning* tuning,
                                 void* stream) {
    if (!c) return LF_ERR_ARG;
    lf_status st;
    if ((st = check_batch(c, b)) != LF_OK) return st;
    if ((st = check_out(c, o, b->n_tracks)) != LF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int wpb = tuning && tuning->warps_per_block > 0 ? tuning->warps_per_block : 8;
    int grain = tuning && tuning->grain > 0 ? tuning->grain : 4;
    if (wpb > 16) return fail(c, LF_ERR_ARG, "warps_per_block %d above 16", wpb);
    int max_bps = 0;
    LF_CUDA(c, fused_max_blocks_per_sm(c->kp, wpb, &max_bps));
    if (max_bps < 1) return fail(c, LF_ERR_ARG, "launch shape does not fit on an SM");
    int bps = tuning && tuning->blocks_per_sm > 0 ? tuning->blocks_per_sm : max_bps;
    if (bps > max_bps) bps = max_bps;
    if ((st = ensure(c, c->ev_count, (size_t)b->n_events * 4)) != LF_OK) return st;

    GraphKey key;
    key.v = std::make_tuple(wpb, bps, grain, b->n_events, b->n_tracks, b->n_hits, (const void*)b->hit_offsets,
                            (const void*)b->x, (const void*)b->trk_offsets, (const void*)b->sx, (const void*)o->found,
                            (const void*)o->out_trk, (const void*)c->ev_count.p);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        // capture: queue reset, persistent kernel, compaction
        cudaStream_t cap;
        LF_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->cursor, 0, sizeof(int), cap);
        KBatch kb = to_kbatch(b);
        KOut ko = to_kout(o);
        if (e == cudaSuccess && b->n_tracks > 0)
            e = launch_fused(c->kp, kb, ko, c->cursor, grain, wpb, bps * c->n_sm, cap);
        if (e == cudaSuccess)
            e = launch_compact(b->trk_offsets, o->found, b->n_events, (int*)c->ev_count.p, o->out_offsets, o->out_trk,
                               o->n_out, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return fail(c, LF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        // keep a bounded cache of shapes
        if (c->graphs.size() >= 64) {
            for (auto& kv : c->graphs)
                if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            c->graphs.clear();
        }
        lf_ctx::GraphEntry ge;
        ge.exec = exec;
        it = c->graphs.emplace(key, ge).first;
    }
    LF_CUDA(c, cudaGraphLaunch(it->second.exec, s));
    return LF_OK;
}

lf_status lf_debug_stages(lf_ctx* c, const lf_batch* b, int32_t* win_begin, int32_t* win_count, int32_t* n_trip,
                          int32_t* trip, float* trip_chi2, void* stream) {
    if (!c) return LF_ERR_ARG;
    lf_status st;
    if ((st = check_batch(c, b)) != LF_OK) return st;
    if (!win_begin || !win_count || !n_trip || !trip || !trip_chi2) return fail(c, LF_ERR_ARG, "dump array is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = plain_stages(c, b, s)) != LF_OK) return st;
    const size_t nt = (size_t)b->n_tracks;
    if (nt == 0) return LF_OK;
    LF_CUDA(c, cudaMemcpyAsync(win_begin, c->wbeg.p, nt * NL * 4, cudaMemcpyDeviceToDevice, s));
    LF_CUDA(c, launch_debug_triplets(c->kp, to_kbatch(b), (int*)c->wbeg.p, (uint8_t*)c->wcnt.p,
                                     (uint64_t*)c->keys.p, (uint8_t*)c->ntrip.p, win_count, n_trip, trip, trip_chi2,
                                     s));
    return LF_OK;
}

lf_status lf_sync_status(lf_ctx* c, void* stream, int32_t* flags) {
    if (!c) return LF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int v = 0;
    LF_CUDA(c, cudaStreamSynchronize(s));
    LF_CUDA(c, cudaMemcpy(&v, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    LF_CUDA(c, cudaMemset(c->status, 0, sizeof(int)));
    if (flags) *flags = v;
    if (v & LF_FLAG_TIMEOUT) return fail(c, LF_ERR_TIMEOUT, "a bounded device wait ran out");
    if (v & (LF_FLAG_BUCKET_OVERFLOW | LF_FLAG_PLANE_RANGE))
        return fail(c, LF_ERR_CAPACITY, "bucket over %d hits or plane code >= 24 (flags 0x%x)", LF_MAX_BUCKET, v);
    return LF_OK;
}

}  // extern "C"
