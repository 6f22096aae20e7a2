// Host side of the C ABI declared in include/lf.h: context, scratch memory,
// argument checks, launches, and the CUDA graphs of the persistent form.
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <cstdint>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lf.h"
#include "lf_internal.h"

using namespace lfk;

namespace {

// NVTX range over a scope: names the host-side enqueueing of each stage for a
// timeline profiler (no cost without one attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// A captured graph holds every pointer and size of its launch, so its key is
// the launch shape, the sizes, the scratch generation and every batch and
// output pointer: a call that changes any of them is a new shape.
struct GraphKey {
    std::array<uintptr_t, 48> v{};
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
    int* cursor = nullptr;   // device work-queue cursors (8 ints)
    unsigned long long generation = 0;  // bumped whenever scratch is reallocated
    int stage_bps[4] = {0, 0, 0, 0};
    DevBuf trk_event, wbeg, wcnt, keys, ntrip, cands, ev_count, coarse, valid;
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        unsigned long long used = 0;   // last use (graph_clock), for eviction
    };
    std::map<GraphKey, GraphEntry> graphs;
    unsigned long long graph_clock = 0;
    unsigned long long graph_captures = 0;   // graphs captured since creation
    // launch shapes seen once: a shape is captured into a graph only when it
    // comes back (a serving loop's batch sizes rarely repeat)
    std::map<GraphKey, unsigned long long> seen;
    unsigned long long seen_clock = 0;
    // end-to-end host pipeline: a compute sub-context (own scratch), three
    // streams (copies in, compute, copies out), events chaining them, and
    // three device staging arenas
    static constexpr int NSLOT = 3;
    lf_ctx* sub = nullptr;
    cudaStream_t pipe_stream[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_in[NSLOT] = {}, ev_comp[NSLOT] = {}, ev_out[NSLOT] = {};
    DevBuf arena[NSLOT];
    // page-locked host block of the chunks' rebased offsets, kept between
    // calls (pinning and unpinning memory on every call costs time and
    // cudaFreeHost can wait on the device)
    int32_t* host_pin = nullptr;
    size_t host_pin_cap = 0;
};

// ---- parameter checks and the kernels' parameter block, shared by every
// entry point (lf_create and the context-free lf_find_tracks_static)
namespace lfk {

static bool finite(float v) { return v == v && v - v == 0.0f; }

bool param_error(const lf_geometry* g, const lf_params* p, char* msg, size_t n) {
    auto bad = [&](const char* fmt, auto... a) {
        snprintf(msg, n, fmt, a...);
        return true;
    };
    if (p->n_hits_window < 1 || p->n_hits_window > LF_MAX_WINDOW)
        return bad("n_hits_window %d outside 1..%d", p->n_hits_window, LF_MAX_WINDOW);
    if (p->n_triplets < 0 || p->n_triplets > LF_MAX_TRIPLETS)
        return bad("n_triplets %d outside 0..%d", p->n_triplets, LF_MAX_TRIPLETS);
    if (p->min_hits < 9 || p->min_hits > 12) return bad("min_hits %d outside 9..12", p->min_hits);
    if (g->polarity != 1 && g->polarity != -1) return bad("polarity must be +1 or -1");
    for (int l = 0; l < LF_N_LAYERS; ++l)
        if (!finite(g->z[l]) || !finite(g->dxdy[l])) return bad("geometry of layer %d not finite", l);
    for (int l = 1; l < LF_N_LAYERS; ++l)
        if (!(g->z[l] > g->z[l - 1])) return bad("layer z must increase");
    for (int l = 0; l < LF_N_LAYERS; ++l) {
        bool x = (l % 4 == 0) || (l % 4 == 3);
        if (!x && g->dxdy[l] == 0.0f) return bad("stereo layer %d has dxdy 0", l);
    }
    if (!(g->z_magnet < g->z[0])) return bad("z_magnet must lie before the first layer");
    if (!(p->magtol_max >= p->magtol_min)) return bad("magtol_max < magtol_min");
    if (g->kappa == 0.0f) return bad("kappa must be non-zero");
    if (p->no_ut != 0 && p->no_ut != 1) return bad("no_ut must be 0 or 1");
    if (p->qop_poly != 0 && p->qop_poly != 1) return bad("qop_poly must be 0 or 1");
    if (p->qop_poly)
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 10; ++j)
                if (!finite(p->qop_c[i][j])) return bad("qop_c[%d][%d] not finite", i, j);
    if (p->no_ut) {
        if (!(p->p_min > 0.0f) || !(p->pt_min > 0.0f) || !finite(p->p_min) || !finite(p->pt_min))
            return bad("p_min and pt_min must be positive");
        if (!(p->x_overlap >= 0.0f) || !finite(p->x_overlap)) return bad("x_overlap must be >= 0");
        for (int i = 0; i < 8; ++i)
            if (!finite(p->tol_c[i])) return bad("tol_c[%d] not finite", i);
    }
    return false;
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
    k.inv_T_x = pow2_reciprocal(p->T_x);
    k.T_uv_scale = p->T_uv_scale;
    k.T_uv_min = p->T_uv_min;
    k.T_ty = p->T_ty;
    k.T_y = p->T_y;
    k.T_Q = p->T_Q;
    for (int i = 0; i < 4; ++i) k.C_n[i] = p->C_n[i];
    k.no_ut = p->no_ut;
    k.p_min = p->p_min;
    k.pt_min = p->pt_min;
    k.x_overlap = p->x_overlap;
    for (int i = 0; i < 8; ++i) k.tol_c[i] = p->tol_c[i];
    k.qop_poly = p->qop_poly;
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 10; ++j) k.qop_c[i][j] = p->qop_c[i][j];
    volatile float pol = (float)g->polarity;  // binary32 products, as the method forms them
    k.pol_f = pol;
    k.pk = pol * g->kappa;
    k.pg = pol * g->gamma;
    k.D = g->dratio * 1000.0f;
    k.pf_bound = std::nextafter((float)(std::sqrt((double)p->T_triplet) + (double)PF_MARGIN), INFINITY);
    return k;
}

}  // namespace lfk

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
    ++c->generation;
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

lf_status check_params(lf_ctx* c, const lf_geometry* g, const lf_params* p) {
    char msg[256];
    if (lfk::param_error(g, p, msg, sizeof msg)) return fail(c, LF_ERR_ARG, "%s", msg);
    return LF_OK;
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
    k.n_dev = nullptr;
    k.x_coarse = b->x_coarse;
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
    const size_t ns = c->p.no_ut ? 2 : 1;  // window sets per track
    if ((st = ensure(c, c->trk_event, nt * 4)) != LF_OK) return st;
    if ((st = ensure(c, c->wbeg, nt * ns * NL * 4)) != LF_OK) return st;
    if ((st = ensure(c, c->wcnt, nt * ns * NL)) != LF_OK) return st;
    if ((st = ensure(c, c->keys, nt * NT * 8)) != LF_OK) return st;
    if ((st = ensure(c, c->ntrip, nt)) != LF_OK) return st;
    if (!b->x_coarse && (st = ensure(c, c->coarse, coarse_count(b->n_hits) * 4)) != LF_OK) return st;
    KBatch kb = to_kbatch(b);
    auto* te = (int*)c->trk_event.p;
    auto* wb = (int*)c->wbeg.p;
    auto* wc = (uint8_t*)c->wcnt.p;
    LF_CUDA(c, launch_track_event(kb, te, s));
    if (!b->x_coarse) {
        kb.x_coarse = (const float*)c->coarse.p;
        LF_CUDA(c, launch_coarse(kb, (float*)c->coarse.p, c->n_sm, s));
    }
    {
        NvtxRange r("lf windows");
        LF_CUDA(c, launch_windows(c->kp, kb, te, wb, wc, s));
    }
    {
        NvtxRange r("lf triplets");
        LF_CUDA(c, launch_triplets(c->kp, kb, te, wb, wc, (uint64_t*)c->keys.p, (uint8_t*)c->ntrip.p, s));
    }
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
    if (cudaMalloc(&c->status, sizeof(int)) != cudaSuccess || cudaMalloc(&c->cursor, 8 * sizeof(int)) != cudaSuccess ||
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
    if (c->sub) lf_destroy(c->sub);
    for (int i = 0; i < 3; ++i)
        if (c->pipe_stream[i]) cudaStreamDestroy(c->pipe_stream[i]);
    for (int i = 0; i < lf_ctx::NSLOT; ++i) {
        if (c->ev_in[i]) cudaEventDestroy(c->ev_in[i]);
        if (c->ev_comp[i]) cudaEventDestroy(c->ev_comp[i]);
        if (c->ev_out[i]) cudaEventDestroy(c->ev_out[i]);
        if (c->arena[i].p) cudaFree(c->arena[i].p);
    }
    if (c->host_pin) cudaFreeHost(c->host_pin);
    for (auto& kv : c->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    DevBuf* bufs[] = {&c->trk_event, &c->wbeg, &c->wcnt, &c->keys, &c->ntrip, &c->coarse,
                      &c->cands, &c->ev_count, &c->valid};
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

int32_t lf_device_host_numa(void) {
    int dev = 0, id = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&id, cudaDevAttrHostNumaId, dev) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return id;
}

lf_status lf_pack_hits(lf_ctx* c, const lf_raw_hits* raw, const lf_packed* pk, void* stream) {
    NvtxRange r("lf pack");
    if (!c) return LF_ERR_ARG;
    if (!raw || !pk) return fail(c, LF_ERR_ARG, "raw or packed is NULL");
    if (raw->n_events < 0 || raw->n_hits < 0) return fail(c, LF_ERR_ARG, "negative size");
    if (!raw->raw_offsets || !pk->hit_offsets) return fail(c, LF_ERR_ARG, "offsets are NULL");
    if (raw->n_hits > 0 && (!raw->x || !raw->z || !raw->dxdy || !raw->w || !raw->plane || !pk->x || !pk->z ||
                            !pk->dxdy || !pk->w || !pk->layer || !pk->perm))
        return fail(c, LF_ERR_ARG, "a hit array is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    // the pack's two work-queue cursors are the context's last two (the find
    // stages use the first ones; calls of one context are stream-ordered)
    LF_CUDA(c, launch_pack(raw->raw_offsets, raw->x, raw->z, raw->dxdy, raw->w, raw->plane, raw->n_events,
                           raw->n_hits, pk->hit_offsets, pk->x, pk->z, pk->dxdy, pk->w, pk->layer, pk->perm, c->cursor + 6,
                           c->status, c->n_sm, s, nullptr, nullptr, pk->x_coarse));
    return LF_OK;
}

lf_status lf_find_tracks(lf_ctx* c, const lf_batch* b, const lf_output* o, void* stream) {
    NvtxRange r("lf find (plain)");
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
                             (uint64_t*)c->keys.p, (uint8_t*)c->ntrip.p, (CandRec*)c->cands.p, ko, s));
    LF_CUDA(c, launch_select(c->kp, kb, (int*)c->wbeg.p, (uint8_t*)c->ntrip.p, (CandRec*)c->cands.p, ko, s));
    LF_CUDA(c, launch_compact(b->trk_offsets, o->found, b->n_events, (int*)c->ev_count.p, o->out_offsets,
                              o->out_trk, o->n_out, s));
    return LF_OK;
}

namespace {

struct Shape {
    int wpb, bps, grain, queue;
    int stage_bps[3];   // per-stage blocks per SM of the stage pipeline (0: bps, else as many as fit)
    int prefilter;      // triplet pre-filter (stage pipeline)
    int extend_form;    // extension of the stage pipeline: 1 block form, 2 warp form
};

// queue modes of lf_tuning
constexpr int Q_STAGES = 0, Q_TILE_SYNC = 1;

lf_status resolve_shape(lf_ctx* c, const lf_tuning* tuning, Shape& sh) {
    sh.queue = tuning ? tuning->queue : Q_STAGES;
    if (sh.queue < 0 || sh.queue > 2) return fail(c, LF_ERR_ARG, "queue mode %d outside 0..2", sh.queue);
    sh.wpb = tuning && tuning->warps_per_block > 0 ? tuning->warps_per_block : 8;
    sh.grain = (tuning && tuning->grain > 0 ? (tuning->grain & 15) : 0) + (sh.queue == Q_TILE_SYNC ? 16 : 0);
    if (sh.wpb > 16) return fail(c, LF_ERR_ARG, "warps_per_block %d above 16", sh.wpb);
    if (c->p.no_ut && sh.queue != Q_STAGES)
        return fail(c, LF_ERR_ARG, "the no-UT variant runs on the staged pipeline (queue 0) only");
    sh.stage_bps[0] = tuning ? tuning->windows_bps : 0;
    sh.stage_bps[1] = tuning ? tuning->triplets_bps : 0;
    sh.stage_bps[2] = tuning ? tuning->extend_bps : 0;
    for (int i = 0; i < 3; ++i)
        if (sh.stage_bps[i] < 0) return fail(c, LF_ERR_ARG, "negative blocks per SM");
    sh.prefilter = tuning ? tuning->triplet_prefilter : 0;
    if (sh.prefilter < 0 || sh.prefilter > 1) return fail(c, LF_ERR_ARG, "triplet_prefilter %d outside 0..1", sh.prefilter);
    if (sh.prefilter && (sh.queue != Q_STAGES || c->p.no_ut))
        return fail(c, LF_ERR_ARG, "the triplet pre-filter runs on the stage pipeline (queue 0) with VELO-UT input");
    sh.extend_form = tuning ? tuning->extend_form : 0;
    if (sh.extend_form < 0 || sh.extend_form > 2)
        return fail(c, LF_ERR_ARG, "extend_form %d outside 0..2", sh.extend_form);
    if (sh.extend_form && sh.queue != Q_STAGES)
        return fail(c, LF_ERR_ARG, "extend_form applies to the stage pipeline (queue 0)");
    if (sh.extend_form == 1 && c->p.no_ut)
        return fail(c, LF_ERR_ARG, "the block form of the extension follows VELO-UT input only");
    if (sh.extend_form == 0) sh.extend_form = c->p.no_ut ? 2 : 1;
    if (sh.queue == Q_STAGES) {
        if (!c->stage_bps[0]) LF_CUDA(c, stage_blocks_per_sm(c->kp, c->stage_bps));
        sh.bps = tuning && tuning->blocks_per_sm > 0 ? tuning->blocks_per_sm : 0;
        return LF_OK;
    }
    int max_bps = 0;
    LF_CUDA(c, fused_max_blocks_per_sm(c->kp, sh.wpb, sh.grain, &max_bps));
    if (max_bps < 1) return fail(c, LF_ERR_ARG, "launch shape does not fit on an SM");
    sh.bps = tuning && tuning->blocks_per_sm > 0 ? tuning->blocks_per_sm : max_bps;
    if (sh.bps > max_bps) sh.bps = max_bps;
    return LF_OK;
}

// scratch of the persistent form, allocated before any capture
lf_status prepare_batched(lf_ctx* c, const lf_batch* b, const Shape& sh) {
    lf_status st;
    if ((st = ensure(c, c->ev_count, (size_t)b->n_events * 4)) != LF_OK) return st;
    if (!b->x_coarse && (st = ensure(c, c->coarse, coarse_count(b->n_hits) * 4)) != LF_OK) return st;
    if (sh.queue == Q_STAGES) {
        const size_t nt = (size_t)b->n_tracks, NT = (size_t)(c->p.n_triplets > 0 ? c->p.n_triplets : 1);
        const size_t ns = c->p.no_ut ? 2 : 1;
        if ((st = ensure(c, c->trk_event, nt * 4)) != LF_OK) return st;
        if ((st = ensure(c, c->wbeg, nt * ns * NL * 4)) != LF_OK) return st;
        if ((st = ensure(c, c->wcnt, nt * ns * NL)) != LF_OK) return st;
        if ((st = ensure(c, c->keys, nt * NT * 8)) != LF_OK) return st;
        if ((st = ensure(c, c->ntrip, nt)) != LF_OK) return st;
    }
    return LF_OK;
}

int stage_grid(lf_ctx* c, const Shape& sh, int i) {
    const int want = sh.stage_bps[i] > 0 ? sh.stage_bps[i] : sh.bps;
    int bps = want > 0 && want < c->stage_bps[i] ? want : c->stage_bps[i];
    return (bps > 0 ? bps : 1) * c->n_sm;
}

// persistent form, launches only (scratch prepared): queue reset, the stage
// pipeline or the tile kernel, compaction
lf_status launch_batched(lf_ctx* c, const lf_batch* b, const lf_output* o, const Shape& sh, cudaStream_t s,
                         const int* n_dev = nullptr) {
    KBatch kb = to_kbatch(b);
    kb.n_dev = n_dev;
    KOut ko = to_kout(o);
    LF_CUDA(c, cudaMemsetAsync(c->cursor, 0, 8 * sizeof(int), s));
    if (b->n_tracks > 0) {
        if (!b->x_coarse) {
            kb.x_coarse = (const float*)c->coarse.p;
            LF_CUDA(c, launch_coarse(kb, (float*)c->coarse.p, c->n_sm, s));
        }
        if (sh.queue == Q_STAGES) {
            auto* te = (int*)c->trk_event.p;
            auto* wb = (int*)c->wbeg.p;
            auto* wc = (uint8_t*)c->wcnt.p;
            auto* ky = (uint64_t*)c->keys.p;
            auto* nt = (uint8_t*)c->ntrip.p;
            auto* cd = (CandRec*)c->cands.p;
            LF_CUDA(c, launch_track_event(kb, te, s));
            NvtxRange r("lf find stages (windows, triplets, extension)");
            LF_CUDA(c, launch_windows(c->kp, kb, te, wb, wc, s, c->cursor + 0, stage_grid(c, sh, 0)));
            LF_CUDA(c, launch_triplets(c->kp, kb, te, wb, wc, ky, nt, s, c->cursor + 1, stage_grid(c, sh, 1),
                                       sh.prefilter));
            // the persistent extension selects and writes the output itself
            LF_CUDA(c, launch_extend(c->kp, kb, te, wb, wc, ky, nt, cd, ko, s, c->cursor + 2, stage_grid(c, sh, 2),
                                     sh.extend_form == 1 ? 1 : 0));
        } else {
            LF_CUDA(c, launch_fused(c->kp, kb, ko, c->cursor, sh.grain, sh.wpb, sh.bps * c->n_sm, s));
        }
    }
    LF_CUDA(c, launch_compact(b->trk_offsets, o->found, b->n_events, (int*)c->ev_count.p, o->out_offsets, o->out_trk,
                              o->n_out, s, n_dev));
    return LF_OK;
}

lf_status batched_direct(lf_ctx* c, const lf_batch* b, const lf_output* o, const Shape& sh, cudaStream_t s) {
    lf_status st = prepare_batched(c, b, sh);
    if (st != LF_OK) return st;
    return launch_batched(c, b, o, sh, s);
}

}  // namespace

extern "C++" {
namespace {

constexpr size_t MAX_GRAPHS = 64;

// The graph of `key`, captured from `launch(stream)` when missing (the least
// recently used graph is dropped when the cache is full), then replayed on s.
template <class Launch>
lf_status graph_replay(lf_ctx* c, const GraphKey& key, cudaStream_t s, Launch&& launch) {
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        cudaStream_t cap;
        LF_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        lf_status ls = LF_OK;
        if (e == cudaSuccess) ls = launch(cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess && ls == LF_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (ls != LF_OK) return ls;
        if (e != cudaSuccess) return fail(c, LF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        if (c->graphs.size() >= MAX_GRAPHS) {
            auto old = c->graphs.begin();
            for (auto jt = c->graphs.begin(); jt != c->graphs.end(); ++jt)
                if (jt->second.used < old->second.used) old = jt;
            if (old->second.exec) cudaGraphExecDestroy(old->second.exec);
            c->graphs.erase(old);
        }
        lf_ctx::GraphEntry ge;
        ge.exec = exec;
        it = c->graphs.emplace(key, ge).first;
        ++c->graph_captures;
    }
    it->second.used = ++c->graph_clock;
    NvtxRange r("lf graph replay");
    LF_CUDA(c, cudaGraphLaunch(it->second.exec, s));
    return LF_OK;
}

// key words: the launch shape, then the caller's sizes and pointers
void key_shape(GraphKey& key, size_t& i, const Shape& sh, unsigned long long generation, uintptr_t form) {
    key.v[i++] = form;
    key.v[i++] = (uintptr_t)sh.wpb;
    key.v[i++] = (uintptr_t)sh.bps;
    key.v[i++] = (uintptr_t)(sh.grain + 64 * sh.queue + ((uintptr_t)sh.stage_bps[0] << 8) +
                             ((uintptr_t)sh.stage_bps[1] << 16) + ((uintptr_t)sh.stage_bps[2] << 24) +
                             ((uintptr_t)sh.prefilter << 32) + ((uintptr_t)sh.extend_form << 33));
    key.v[i++] = (uintptr_t)generation;
}
void key_batch(GraphKey& key, size_t& i, const lf_batch* b, const lf_output* o) {
    const uintptr_t w[] = {(uintptr_t)b->n_events, (uintptr_t)b->n_tracks, (uintptr_t)b->n_hits,
                           (uintptr_t)b->hit_offsets, (uintptr_t)b->x, (uintptr_t)b->z, (uintptr_t)b->dxdy,
                           (uintptr_t)b->w, (uintptr_t)b->trk_offsets, (uintptr_t)b->sx, (uintptr_t)b->sy,
                           (uintptr_t)b->stx, (uintptr_t)b->sty, (uintptr_t)b->sqop, (uintptr_t)o->found,
                           (uintptr_t)o->nhits, (uintptr_t)o->hit_idx, (uintptr_t)o->state, (uintptr_t)o->quality,
                           (uintptr_t)o->out_offsets, (uintptr_t)o->out_trk, (uintptr_t)o->n_out,
                           (uintptr_t)b->x_coarse};
    for (uintptr_t x : w) key.v[i++] = x;
}

}  // namespace
}  // extern "C++"

lf_status lf_find_tracks_batched(lf_ctx* c, const lf_batch* b, const lf_output* o, const lf_tuning* tuning,
                                 void* stream) {
    if (!c) return LF_ERR_ARG;
    lf_status st;
    if ((st = check_batch(c, b)) != LF_OK) return st;
    if ((st = check_out(c, o, b->n_tracks)) != LF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Shape sh;
    if ((st = resolve_shape(c, tuning, sh)) != LF_OK) return st;
    if ((st = prepare_batched(c, b, sh)) != LF_OK) return st;

    GraphKey key;
    size_t i = 0;
    key_shape(key, i, sh, c->generation, 1);
    key_batch(key, i, b, o);
    if (c->graphs.find(key) == c->graphs.end()) {
        // first use of this shape: launch directly and remember it (bounded)
        if (c->seen.find(key) == c->seen.end()) {
            if (c->seen.size() >= 256) {
                auto oldest = c->seen.begin();
                for (auto jt = c->seen.begin(); jt != c->seen.end(); ++jt)
                    if (jt->second < oldest->second) oldest = jt;
                c->seen.erase(oldest);
            }
            c->seen[key] = ++c->seen_clock;
            return launch_batched(c, b, o, sh, s);
        }
    }
    return graph_replay(c, key, s, [&](cudaStream_t cs) { return launch_batched(c, b, o, sh, cs); });
}

lf_status lf_process_slot(lf_ctx* c, const lf_raw_hits* raw, const lf_packed* pk, const lf_batch* b,
                          const lf_gather* g, const int32_t* n_events_dev, const lf_output* o,
                          const lf_tuning* tuning, void* stream) {
    if (!c) return LF_ERR_ARG;
    NvtxRange r("lf slot");
    lf_status st;
    if (!raw || !pk || !n_events_dev) return fail(c, LF_ERR_ARG, "raw, packed or n_events_dev is NULL");
    if ((st = check_batch(c, b)) != LF_OK) return st;
    if ((st = check_out(c, o, b->n_tracks)) != LF_OK) return st;
    if (raw->n_events != b->n_events || raw->n_hits != b->n_hits)
        return fail(c, LF_ERR_ARG, "raw and batch capacities differ");
    if (!raw->raw_offsets || !raw->x || !raw->z || !raw->dxdy || !raw->w || !raw->plane || !pk->layer || !pk->perm)
        return fail(c, LF_ERR_ARG, "a raw or packed array is NULL");
    if (b->hit_offsets != pk->hit_offsets || b->x != pk->x || b->z != pk->z || b->dxdy != pk->dxdy || b->w != pk->w ||
        b->x_coarse != pk->x_coarse)
        return fail(c, LF_ERR_ARG, "the batch's hit arrays are not the packed arrays");
    if (g && (!g->hit_src || !g->trk_src || !g->sx || !g->sy || !g->stx || !g->sty || !g->sqop))
        return fail(c, LF_ERR_ARG, "a gather array is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    Shape sh;
    if ((st = resolve_shape(c, tuning, sh)) != LF_OK) return st;
    if ((st = prepare_batched(c, b, sh)) != LF_OK) return st;

    GraphKey key;
    size_t i = 0;
    key_shape(key, i, sh, c->generation, 2);
    key_batch(key, i, b, o);
    const uintptr_t w[] = {(uintptr_t)n_events_dev, (uintptr_t)raw->raw_offsets, (uintptr_t)raw->x,
                           (uintptr_t)raw->z, (uintptr_t)raw->dxdy, (uintptr_t)raw->w, (uintptr_t)raw->plane,
                           (uintptr_t)pk->layer, (uintptr_t)pk->perm, (uintptr_t)(g ? g->hit_src : nullptr),
                           (uintptr_t)(g ? g->trk_src : nullptr), (uintptr_t)(g ? g->sx : nullptr),
                           (uintptr_t)(g ? g->sy : nullptr), (uintptr_t)(g ? g->stx : nullptr),
                           (uintptr_t)(g ? g->sty : nullptr), (uintptr_t)(g ? g->sqop : nullptr)};
    for (uintptr_t x : w) key.v[i++] = x;
    return graph_replay(c, key, s, [&](cudaStream_t cs) -> lf_status {
        if (g) {
            KBatch kb = to_kbatch(b);
            kb.n_dev = n_events_dev;
            LF_CUDA(c, launch_gather_states(kb, g->trk_src, g->sx, g->sy, g->stx, g->sty, g->sqop, c->n_sm, cs));
        }
        LF_CUDA(c, launch_pack(raw->raw_offsets, raw->x, raw->z, raw->dxdy, raw->w, raw->plane, raw->n_events,
                               raw->n_hits, pk->hit_offsets, pk->x, pk->z, pk->dxdy, pk->w, pk->layer, pk->perm,
                               c->cursor + 6, c->status, c->n_sm, cs, n_events_dev, g ? g->hit_src : nullptr,
                               pk->x_coarse));
        return launch_batched(c, b, o, sh, cs, n_events_dev);
    });
}

int64_t lf_graph_count(const lf_ctx* c) { return c ? (int64_t)c->graph_captures : -1; }

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
    const size_t ns = c->p.no_ut ? 2 : 1;
    LF_CUDA(c, cudaMemcpyAsync(win_begin, c->wbeg.p, nt * ns * NL * 4, cudaMemcpyDeviceToDevice, s));
    LF_CUDA(c, launch_debug_triplets(c->kp, to_kbatch(b), (int*)c->wbeg.p, (uint8_t*)c->wcnt.p,
                                     (uint64_t*)c->keys.p, (uint8_t*)c->ntrip.p, win_count, n_trip, trip, trip_chi2,
                                     s));
    return LF_OK;
}

lf_status lf_debug_triplets(lf_ctx* c, const lf_batch* b, int32_t* win_count, int32_t* n_trip, int32_t* trip,
                            float* trip_chi2, void* stream) {
    if (!c) return LF_ERR_ARG;
    lf_status st;
    if ((st = check_batch(c, b)) != LF_OK) return st;
    if (!win_count || !n_trip || !trip || !trip_chi2) return fail(c, LF_ERR_ARG, "dump array is NULL");
    const size_t nt = (size_t)b->n_tracks;
    if (nt == 0) return LF_OK;
    const size_t ns = c->p.no_ut ? 2 : 1, NT = (size_t)(c->p.n_triplets > 0 ? c->p.n_triplets : 1);
    if (c->wbeg.cap < nt * ns * NL * 4 || c->wcnt.cap < nt * ns * NL || c->keys.cap < nt * NT * 8 || c->ntrip.cap < nt)
        return fail(c, LF_ERR_ARG, "no stage-pipeline results of this size in the context");
    LF_CUDA(c, launch_debug_triplets(c->kp, to_kbatch(b), (int*)c->wbeg.p, (uint8_t*)c->wcnt.p,
                                     (uint64_t*)c->keys.p, (uint8_t*)c->ntrip.p, win_count, n_trip, trip, trip_chi2,
                                     (cudaStream_t)stream));
    return LF_OK;
}

lf_status lf_validate_batch(lf_ctx* c, const lf_batch* b, void* stream) {
    if (!c) return LF_ERR_ARG;
    lf_status st;
    if ((st = check_batch(c, b)) != LF_OK) return st;
    if ((st = ensure(c, c->valid, 2 * sizeof(int))) != LF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int* bad = (int*)c->valid.p;
    const int none = INT_MAX;
    int h[2];
    const KBatch kb = to_kbatch(b);
    // offsets first: the bucket checks index with them
    LF_CUDA(c, cudaMemcpyAsync(bad, &none, sizeof(int), cudaMemcpyHostToDevice, s));
    LF_CUDA(c, cudaMemcpyAsync(bad + 1, &none, sizeof(int), cudaMemcpyHostToDevice, s));
    LF_CUDA(c, launch_validate_offsets(kb, bad, c->n_sm, s));
    LF_CUDA(c, cudaMemcpyAsync(h, bad, sizeof h, cudaMemcpyDeviceToHost, s));
    LF_CUDA(c, cudaStreamSynchronize(s));
    if (h[0] != none)
        return fail(c, LF_ERR_ARG, "hit_offsets[%d] is outside 0..n_hits (%d) or decreases to the next entry", h[0],
                    b->n_hits);
    if (h[1] != none)
        return fail(c, LF_ERR_ARG, "trk_offsets[%d] is outside 0..n_tracks (%d), decreases, or the last entry is not "
                    "n_tracks", h[1], b->n_tracks);
    LF_CUDA(c, cudaMemcpyAsync(bad, &none, sizeof(int), cudaMemcpyHostToDevice, s));
    LF_CUDA(c, cudaMemcpyAsync(bad + 1, &none, sizeof(int), cudaMemcpyHostToDevice, s));
    LF_CUDA(c, launch_validate_hits(kb, bad, c->n_sm, s));
    LF_CUDA(c, cudaMemcpyAsync(h, bad, sizeof h, cudaMemcpyDeviceToHost, s));
    LF_CUDA(c, cudaStreamSynchronize(s));
    if (h[0] != none)
        return fail(c, LF_ERR_ARG, "x is not ascending inside a bucket: packed hits %d and %d", h[0], h[0] + 1);
    if (h[1] != none) return fail(c, LF_ERR_ARG, "x_coarse[%d] differs from x[%d]", h[1], 32 * h[1]);
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

lf_status lf_reserve(lf_ctx* c, int32_t n_events, int32_t n_hits, int32_t n_tracks, const lf_tuning* tuning) {
    if (!c) return LF_ERR_ARG;
    if (n_events < 0 || n_hits < 0 || n_tracks < 0) return fail(c, LF_ERR_ARG, "negative size");
    Shape sh;
    lf_status st;
    if ((st = resolve_shape(c, tuning, sh)) != LF_OK) return st;
    lf_batch big{n_events, n_hits, n_tracks, nullptr, nullptr, nullptr, nullptr, nullptr,
                 nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    return prepare_batched(c, &big, sh);
}

lf_status lf_host_alloc(size_t bytes, void** out) {
    if (!out) return LF_ERR_ARG;
    *out = nullptr;
    if (bytes == 0) return LF_OK;
    if (cudaHostAlloc(out, bytes, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return LF_ERR_OOM;
    }
    return LF_OK;
}

void lf_host_free(void* p) {
    if (p) cudaFreeHost(p);
}

lf_status lf_process_host(lf_ctx* c, const lf_host_batch* hb, const lf_host_output* ho, const lf_tuning* tuning,
                          int64_t chunk_hits) {
    if (!c) return LF_ERR_ARG;
    if (!hb || !ho) return fail(c, LF_ERR_ARG, "batch or output is NULL");
    if (hb->n_events < 0 || hb->n_hits < 0 || hb->n_tracks < 0) return fail(c, LF_ERR_ARG, "negative size");
    if (!hb->raw_offsets || !hb->trk_offsets) return fail(c, LF_ERR_ARG, "offsets are NULL");
    if (hb->raw_offsets[hb->n_events] != hb->n_hits || hb->trk_offsets[hb->n_events] != hb->n_tracks)
        return fail(c, LF_ERR_ARG, "offsets do not end at n_hits / n_tracks");
    if (hb->raw_offsets[0] != 0 || hb->trk_offsets[0] != 0) return fail(c, LF_ERR_ARG, "offsets do not start at 0");
    for (int e = 0; e < hb->n_events; ++e)
        if (hb->raw_offsets[e + 1] < hb->raw_offsets[e] || hb->trk_offsets[e + 1] < hb->trk_offsets[e])
            return fail(c, LF_ERR_ARG, "offsets decrease at event %d", e);
    if (hb->n_hits > 0 && (!hb->x || !hb->z || !hb->dxdy || !hb->w || !hb->plane))
        return fail(c, LF_ERR_ARG, "hit arrays are NULL");
    if (hb->n_tracks > 0 && (!hb->sx || !hb->sy || !hb->stx || !hb->sty || !hb->sqop))
        return fail(c, LF_ERR_ARG, "state arrays are NULL");
    if (hb->n_events == 0) return LF_OK;
    if (chunk_hits <= 0) chunk_hits = (int64_t)1 << 26;
    constexpr int NS = lf_ctx::NSLOT;
    lf_status st;
    if (!c->sub && (st = lf_create(&c->g, &c->p, &c->sub)) != LF_OK) return fail(c, st, "sub-context creation failed");
    lf_ctx* sc = c->sub;
    for (int i = 0; i < 3; ++i)
        if (!c->pipe_stream[i]) LF_CUDA(c, cudaStreamCreateWithFlags(&c->pipe_stream[i], cudaStreamNonBlocking));
    for (int i = 0; i < NS; ++i) {
        if (!c->ev_in[i]) LF_CUDA(c, cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming));
        if (!c->ev_comp[i]) LF_CUDA(c, cudaEventCreateWithFlags(&c->ev_comp[i], cudaEventDisableTiming));
        if (!c->ev_out[i]) LF_CUDA(c, cudaEventCreateWithFlags(&c->ev_out[i], cudaEventDisableTiming));
    }
    cudaStream_t s_in = c->pipe_stream[0], s_comp = c->pipe_stream[1], s_out = c->pipe_stream[2];
    Shape sh;
    if ((st = resolve_shape(sc, tuning, sh)) != LF_OK) return fail(c, st, "%s", sc->err);
    // chunk boundaries at event boundaries
    std::vector<int> cut{0};
    const int32_t* ro = hb->raw_offsets;
    const int32_t* to = hb->trk_offsets;
    for (int e = 0; e < hb->n_events; ++e) {
        int s0 = cut.back();
        if (e > s0 && (int64_t)ro[e + 1] - ro[s0] > chunk_hits) cut.push_back(e);
    }
    cut.push_back(hb->n_events);
    size_t H = 0, E = 0, T = 0;
    for (size_t k = 0; k + 1 < cut.size(); ++k) {
        H = std::max(H, (size_t)(ro[cut[k + 1]] - ro[cut[k]]));
        E = std::max(E, (size_t)(cut[k + 1] - cut[k]));
        T = std::max(T, (size_t)(to[cut[k + 1]] - to[cut[k]]));
    }
    // the compute context's scratch at the largest chunk's size before any
    // copy is queued (growing it later would synchronise the device)
    {
        lf_batch big{(int32_t)E, (int32_t)H, (int32_t)T, nullptr, nullptr, nullptr, nullptr, nullptr,
                     nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        if ((st = prepare_batched(sc, &big, sh)) != LF_OK) return fail(c, st, "%s", sc->err);
    }
    // rebased offsets of every chunk, in one pinned block
    const size_t n_chunks = cut.size() - 1;
    const size_t pin_n = 2 * ((size_t)hb->n_events + n_chunks);
    if (c->host_pin_cap < pin_n) {
        if (c->host_pin) cudaFreeHost(c->host_pin);
        c->host_pin = nullptr;
        c->host_pin_cap = 0;
        const size_t want = pin_n + pin_n / 8;
        LF_CUDA(c, cudaMallocHost(&c->host_pin, want * sizeof(int32_t)));
        c->host_pin_cap = want;
    }
    int32_t* pin = c->host_pin;
    std::vector<size_t> pin_off(n_chunks);
    {
        size_t q = 0;
        for (size_t k = 0; k < n_chunks; ++k) {
            pin_off[k] = q;
            int e0 = cut[k], e1 = cut[k + 1];
            for (int e = e0; e <= e1; ++e) pin[q++] = ro[e] - ro[e0];
            for (int e = e0; e <= e1; ++e) pin[q++] = to[e] - to[e0];
        }
    }
    // device arena per slot
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    size_t sz = 0;
    size_t o_x = sz; sz += al(4 * H);
    size_t o_z = sz; sz += al(4 * H);
    size_t o_d = sz; sz += al(4 * H);
    size_t o_w = sz; sz += al(4 * H);
    size_t o_pl = sz; sz += al(H);
    size_t o_ro = sz; sz += al(4 * (E + 1));
    size_t o_to = sz; sz += al(4 * (E + 1));
    size_t o_st = sz; sz += al(4 * 5 * T);
    size_t o_ho = sz; sz += al(4 * (NB * E + 1));
    size_t o_px = sz; sz += al(4 * H);
    size_t o_pz = sz; sz += al(4 * H);
    size_t o_pd = sz; sz += al(4 * H);
    size_t o_pw = sz; sz += al(4 * H);
    size_t o_pl2 = sz; sz += al(H);
    size_t o_pm = sz; sz += al(4 * H);
    size_t o_pc = sz; sz += al(4 * coarse_count((int)H));
    size_t o_fd = sz; sz += al(T);
    size_t o_nh = sz; sz += al(T);
    size_t o_hi = sz; sz += al(4 * NL * T);
    size_t o_sv = sz; sz += al(4 * 6 * T);
    size_t o_q = sz; sz += al(4 * T);
    size_t o_oo = sz; sz += al(4 * (E + 1));
    size_t o_ot = sz; sz += al(4 * (T + 1));
    size_t o_no = sz; sz += al(4);
    for (int i = 0; i < NS; ++i) {
        if ((st = ensure(c, c->arena[i], sz)) != LF_OK) return st;
    }
    // three-stage pipeline over NS arena slots: chunk k's copies in (stream
    // s_in) wait until the slot's previous chunk has left (its copies out),
    // its compute (s_comp) waits for its copies in, its copies out (s_out)
    // wait for its compute; so copies in of chunk k+1, compute of chunk k and
    // copies out of chunk k-1 overlap
    lf_status rc = LF_OK;
    cudaError_t ce = cudaSuccess;
    for (size_t k = 0; k < n_chunks && rc == LF_OK && ce == cudaSuccess; ++k) {
        const int slot = (int)(k % NS);
        char* A = (char*)c->arena[slot].p;
        const int e0 = cut[k], e1 = cut[k + 1];
        const int ne = e1 - e0, h0 = ro[e0], nh = ro[e1] - ro[e0], t0 = to[e0], nt = to[e1] - to[e0];
        if (k >= (size_t)NS && (ce = cudaStreamWaitEvent(s_in, c->ev_out[slot], 0)) != cudaSuccess) break;
        auto cp = [&](size_t dst, const void* src, size_t bytes) {
            if (ce == cudaSuccess && bytes) ce = cudaMemcpyAsync(A + dst, src, bytes, cudaMemcpyHostToDevice, s_in);
        };
        cp(o_ro, pin + pin_off[k], 4 * (size_t)(ne + 1));
        cp(o_to, pin + pin_off[k] + ne + 1, 4 * (size_t)(ne + 1));
        cp(o_x, hb->x + h0, 4 * (size_t)nh);
        cp(o_z, hb->z + h0, 4 * (size_t)nh);
        cp(o_d, hb->dxdy + h0, 4 * (size_t)nh);
        cp(o_w, hb->w + h0, 4 * (size_t)nh);
        cp(o_pl, hb->plane + h0, (size_t)nh);
        cp(o_st + 0 * 4 * T, hb->sx + t0, 4 * (size_t)nt);
        cp(o_st + 1 * 4 * T, hb->sy + t0, 4 * (size_t)nt);
        cp(o_st + 2 * 4 * T, hb->stx + t0, 4 * (size_t)nt);
        cp(o_st + 3 * 4 * T, hb->sty + t0, 4 * (size_t)nt);
        cp(o_st + 4 * 4 * T, hb->sqop + t0, 4 * (size_t)nt);
        if (ce == cudaSuccess) ce = cudaEventRecord(c->ev_in[slot], s_in);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s_comp, c->ev_in[slot], 0);
        if (ce != cudaSuccess) break;
        lf_raw_hits raw{ne, nh, (const int32_t*)(A + o_ro), (const float*)(A + o_x), (const float*)(A + o_z),
                        (const float*)(A + o_d), (const float*)(A + o_w), (const uint8_t*)(A + o_pl)};
        lf_packed pk{(int32_t*)(A + o_ho), (float*)(A + o_px), (float*)(A + o_pz), (float*)(A + o_pd),
                     (float*)(A + o_pw), (uint8_t*)(A + o_pl2), (int32_t*)(A + o_pm), (float*)(A + o_pc)};
        NvtxRange rk("lf host chunk (pack, find, copies out)");
        if ((rc = lf_pack_hits(sc, &raw, &pk, s_comp)) != LF_OK) break;
        lf_batch bt{ne, nh, nt, pk.hit_offsets, pk.x, pk.z, pk.dxdy, pk.w, (const int32_t*)(A + o_to),
                    (const float*)(A + o_st), (const float*)(A + o_st + 4 * T), (const float*)(A + o_st + 8 * T),
                    (const float*)(A + o_st + 12 * T), (const float*)(A + o_st + 16 * T), pk.x_coarse};
        lf_output out{(uint8_t*)(A + o_fd), (uint8_t*)(A + o_nh), (int32_t*)(A + o_hi), (float*)(A + o_sv),
                      (float*)(A + o_q), (int32_t*)(A + o_oo), (int32_t*)(A + o_ot), (int32_t*)(A + o_no)};
        if ((rc = batched_direct(sc, &bt, &out, sh, s_comp)) != LF_OK) break;
        ce = launch_hits_to_raw(out.found, out.hit_idx, pk.perm, nt, h0, s_comp);
        if (ce == cudaSuccess) ce = cudaEventRecord(c->ev_comp[slot], s_comp);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s_out, c->ev_comp[slot], 0);
        auto back = [&](void* dst, size_t src, size_t bytes) {
            if (ce == cudaSuccess && bytes && dst) ce = cudaMemcpyAsync(dst, A + src, bytes, cudaMemcpyDeviceToHost, s_out);
        };
        back(ho->found + t0, o_fd, (size_t)nt);
        back(ho->nhits + t0, o_nh, (size_t)nt);
        back(ho->hit_idx + (size_t)t0 * NL, o_hi, 4 * NL * (size_t)nt);
        back(ho->state + (size_t)t0 * 6, o_sv, 4 * 6 * (size_t)nt);
        back(ho->quality + t0, o_q, 4 * (size_t)nt);
        if (ce == cudaSuccess) ce = cudaEventRecord(c->ev_out[slot], s_out);
    }
    for (int i = 0; i < 3; ++i) {
        cudaError_t e2 = cudaStreamSynchronize(c->pipe_stream[i]);
        if (ce == cudaSuccess) ce = e2;
    }
    if (rc != LF_OK) return fail(c, rc, "chunk failed: %s", lf_last_error(sc));
    if (ce != cudaSuccess) return fail(c, LF_ERR_CUDA, "host pipeline: %s", cudaGetErrorString(ce));
    int32_t flags = 0;
    lf_status s2 = lf_sync_status(sc, s_comp, &flags);
    if (s2 != LF_OK) return fail(c, s2, "device status flags 0x%x", flags);
    return LF_OK;
}

}  // extern "C"
