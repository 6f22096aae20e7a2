/*
 * lf.h — C ABI of the GB300 (sm_103a) forward-tracking library.
 *
 * The library follows upstream (VELO-UT) track states into the twelve
 * x-u-v-x layers of the downstream tracker, as in "Looking Forward"
 * (arXiv:2402.14670):
 *   Sec. "Defining the search windows"            magnet extrapolation with a pT
 *       kick, per-layer windows x_tol = xtol_c + xtol_p/p plus the magnet
 *       asymmetry term, u/v windows around the stereo-corrected centre,
 *       at most n_hits_window hits kept symmetrically around the centre;
 *   Sec. "Triplet Seeding"                        doublets from the first/last
 *       x layers of T1 and T3 with the bending and magnet-opening filters,
 *       x1_expected with K, chi2_triplet < T_triplet, the n_triplets smallest;
 *   Sec. "Extending triplets to other layers"     Eq. dratio_model_x_expected
 *       around z_ref, T_x and T_uv acceptance;
 *   Sec. "Quality Filter"                         y line fit, T_ty, Q_x, Q_y,
 *       Q = (Q_x/nDoF_x + Q_y/nDoF_y) C(n_hits) (Table C_nhits), Q < T_Q,
 *       best Q per input track;
 *   Sec. "Calculation of momentum and track states" q/p from the slope change,
 *       in the linear kick form or (lf_params.qop_poly) through the field
 *       integral's polynomial in dSlope (Eq. pt_kick).
 *
 * Conventions
 *   - Every pointer inside lf_raw_hits, lf_packed, lf_batch and lf_output is a
 *     DEVICE pointer owned by the caller, unless a function says otherwise.
 *     The library never frees caller memory.
 *   - The context owns its scratch memory and the device copy of geometry
 *     and parameters; scratch grows on demand and is freed by lf_destroy.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream).  The returned status covers
 *     argument checks and launch errors only.  Device-side conditions (a
 *     bucket or window over capacity, a bounded wait that ran out) are
 *     recorded in a status word that lf_sync_status reads.
 *   - One context per stream at a time; different contexts are independent.
 *   - Floating point: binary32, round to nearest, no contraction, in the
 *     expression order of the method's definition, so results are
 *     deterministic and independent of launch shape.
 *   - Hit indices are indices into the packed (sorted) hit arrays; perm maps
 *     them back to raw indices.
 */
#ifndef LF_H
#define LF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LF_N_LAYERS 12
#define LF_N_BUCKETS 24          /* (zone, layer) buckets per event: zone*12 + layer */
#define LF_MAX_WINDOW 64         /* largest n_hits_window */
#define LF_MAX_TRIPLETS 32       /* largest n_triplets */
#define LF_MAX_BUCKET 16384      /* largest number of hits in one (event, zone, layer) bucket */

typedef enum {
    LF_OK = 0,
    LF_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, bad parameter) */
    LF_ERR_CUDA = 2,       /* a CUDA call failed; lf_last_error has the message */
    LF_ERR_OOM = 3,        /* scratch allocation failed */
    LF_ERR_CAPACITY = 4,   /* device status: a bucket above LF_MAX_BUCKET hits */
    LF_ERR_TIMEOUT = 5,    /* device status: a bounded wait ran out (reserved: no kernel of this
                              library waits on a flag or barrier, so none sets it today) */
    LF_ERR_INTERNAL = 6
} lf_status;

/* device status word bits, read by lf_sync_status */
#define LF_FLAG_BUCKET_OVERFLOW 0x1
#define LF_FLAG_PLANE_RANGE     0x2
#define LF_FLAG_TIMEOUT         0x4   /* reserved; see LF_ERR_TIMEOUT */

typedef struct lf_ctx lf_ctx;

/* Detector and field constants (Sec. "Context", Sec. "Propagation of tracks
 * in LHCb's magnetic field").  Layers are ordered x,u,v,x per station. */
typedef struct {
    float z[LF_N_LAYERS];      /* layer z, mm */
    float dxdy[LF_N_LAYERS];   /* stereo slope: 0 for x layers, +-tan(5 deg) for u/v */
    float z_state;             /* z of the input states */
    float z_magnet;            /* pT-kick plane */
    float z_ref;               /* reference plane of the T-station model */
    float kappa;               /* slope kick per unit q/p */
    float gamma;               /* curvature per unit q/p */
    float dratio;              /* dRatio of Eq. trackfitmodel */
    int32_t polarity;          /* +1 MagUp, -1 MagDown */
} lf_geometry;

/* Tunable parameters (Table tolerances, Table C_nhits). */
typedef struct {
    float xtol_c, xtol_p;      /* x_tol = xtol_c + xtol_p / p */
    float x_asym;              /* magnet asymmetry term */
    float uv_tol;              /* u/v window half width */
    int32_t n_hits_window;     /* 1..64 */
    int32_t n_triplets;        /* 0..32 */
    int32_t min_hits;          /* 9..12 */
    float K_first, K_last;     /* correction factor of x1_expected */
    float p_bend;              /* the bending-sign filter applies below this p */
    float magtol_min, magtol_max, magtol_c, magtol_tx; /* clamp(min + c/p + tx*|t_x|, min, max) */
    float T_triplet, T_x, T_uv_scale, T_uv_min, T_ty, T_y, T_Q;
    float C_n[4];              /* C(9), C(10), C(11), C(12) */
    /* Sec. "No-UT tuning": input tracks without a momentum estimate.
     * no_ut = 0: VELO-UT input, sqop is used.  no_ut = 1: sqop is ignored; the
     * windows assume the momentum 1/ip with ip = min(1/p_min, sin(theta)/pt_min)
     * (the tighter threshold), x_tol = ip*(c0 + tx(c1 + c2 tx) + ty^2(c3 +
     * tx(c4 + c5 tx)) + ip(c6 tx + c7 ip)) (Eq. tol_noUT), and every input
     * track gets two window sets (Eq. noUT_size_window): side 0 =
     * [x - x_tol, x + x_overlap], side 1 = [x - x_overlap, x + x_tol] around
     * the straight-line extrapolation x (u/v: uv_tol around the
     * stereo-corrected line).  Triplets are seeded per side and the
     * n_triplets smallest of both sides are kept, ordered by (chi2, side,
     * configuration, h0, h2); a triplet is extended in its own side's
     * windows.  Supported by lf_find_tracks and lf_find_tracks_batched with
     * queue 0; the tile kernel (queue 1, 2) and lf_find_tracks_static
     * return LF_ERR_ARG. */
    int32_t no_ut;             /* 0 or 1 */
    float p_min, pt_min;       /* GeV, > 0 */
    float x_overlap;           /* mm, >= 0 */
    float tol_c[8];            /* c0..c7 (Table poly_tol) */
    /* Sec. "Calculation of momentum and track states": the q/p of a found
     * track.  qop_poly = 0: linear kick, (t_x,fit - t_x,in) / (polarity kappa).
     * qop_poly = 1: Eq. pt_kick, q/p = (t_x,f / sqrt(1 + t_x,f^2 + t_y,f^2) -
     * t_x,i / sqrt(1 + t_x,i^2 + t_y,i^2)) / (polarity F), f = the fit at
     * z_ref, i = the input state, with the field integral F = c_0 + d (c_1 +
     * d (c_2 + d (c_3 + d c_4))), d = t_x,f - t_x,i, and c_i = sum_j
     * qop_c[i][j] t_x,i^k t_y,i^m over the (k, m) of entry j: for even i
     * (0,0) (0,2) (0,4) (0,6) (2,0) (2,2) (2,4) (4,0) (4,2) (6,0), for odd i
     * (1,0) (1,2) (1,4) (3,0) (3,2) (5,0) (entries 6..9 unused), summed in
     * entry order.  The coefficients come from a fit on toy tracks
     * (paper_2402_14670_gb300.qop_fit). */
    int32_t qop_poly;          /* 0 or 1 */
    float qop_c[5][10];
} lf_params;

/* Raw hits of n_events events, unsorted inside each event (device). */
typedef struct {
    int32_t n_events;
    int32_t n_hits;            /* == raw_offsets[n_events] */
    const int32_t* raw_offsets;/* [n_events+1] */
    const float* x;            /* measured coordinate */
    const float* z;
    const float* dxdy;
    const float* w;            /* weight */
    const uint8_t* plane;      /* zone*12 + layer, zone 1 = upper half */
} lf_raw_hits;

/* Packed hits written by lf_pack_hits (caller-allocated device arrays). */
typedef struct {
    int32_t* hit_offsets;      /* [24*n_events+1] bucket starts */
    float* x; float* z; float* dxdy; float* w;   /* [n_hits] */
    uint8_t* layer;            /* [n_hits] */
    int32_t* perm;             /* [n_hits] packed index -> raw index */
    float* x_coarse;           /* optional [(n_hits+31)/32]: x_coarse[i] = x[32 i], the index the
                                  window searches use (NULL: not written) */
} lf_packed;

/* Input of the track finding: packed hits plus input states (device). */
typedef struct {
    int32_t n_events;
    int32_t n_hits;
    int32_t n_tracks;          /* == trk_offsets[n_events] */
    const int32_t* hit_offsets;/* [24*n_events+1], x ascending inside each bucket */
    const float* x; const float* z; const float* dxdy; const float* w;
    const int32_t* trk_offsets;/* [n_events+1] */
    const float* sx; const float* sy; const float* stx; const float* sty; const float* sqop;
    const float* x_coarse;     /* optional: the packed x_coarse (NULL: the find computes it in
                                  context scratch, reading x once more) */
} lf_batch;

/* Output per input track t (device, caller-allocated).
 *   found[t] 0/1; nhits[t];
 *   hit_idx[t*12 + layer]: packed hit index or -1; state[t*6 + k]:
 *   (x, y, tx, ty, c, q/p) at z_ref; quality[t] = Q.
 *   hit_idx, state and quality are written only where found[t] == 1.
 * Compaction: out_offsets[n_events+1] (found tracks before each event),
 *   out_trk[n_tracks] (indices of found tracks, event order), n_out[1]. */
typedef struct {
    uint8_t* found; uint8_t* nhits; int32_t* hit_idx; float* state; float* quality;
    int32_t* out_offsets; int32_t* out_trk; int32_t* n_out;
} lf_output;

/* Launch shape of the persistent form (filled by the autotuner or the user;
 * zeros select the defaults). */
typedef struct {
    int32_t warps_per_block;   /* tile kernel (queue 1, 2): 1..16 warps per block; ignored otherwise */
    int32_t blocks_per_sm;     /* resident blocks per SM of the persistent grid (0: as many as fit) */
    int32_t grain;             /* tile kernel: input tracks per warp per step, 1 or 2 (default when
                                  n_triplets <= 16: the extension runs two tracks per warp, 16 lanes each) */
    int32_t queue;             /* 0: pipeline of persistent stage kernels (windows, triplets, extension
                                  with selection), each draining its own device work queue (default);
                                  1: one tile kernel, blocks take tiles of tracks and their warps step
                                  through the stages together; 2: the tile kernel, warps take their
                                  own tracks */
    int32_t windows_bps;       /* stage pipeline: resident blocks per SM of the windows, triplet and */
    int32_t triplets_bps;      /* extension kernels (0: blocks_per_sm, or as many as fit; a value   */
    int32_t extend_bps;        /* above what fits is lowered to it)                                  */
    int32_t triplet_prefilter; /* stage pipeline, VELO-UT input: 0 (default) none; 1 the half-precision
                                  pre-filter of the triplet pairs (Sec. "Performance", the triplet
                                  seeding's chi2 in half2 arithmetic): every (h0, h2) pair is first
                                  tested against all hits of its h1 window in binary16, with a margin
                                  above binary16 rounding, and only the pairs that pass get the exact
                                  binary32 filters, closest-hit search and chi2.  Same results as 0;
                                  LF_ERR_ARG with queue != 0 or the no-UT variant. */
    int32_t extend_form;       /* stage pipeline's extension: 0 default (1 for VELO-UT input, 2 for
                                  the no-UT variant); 1 block form: a block of 256 threads takes
                                  min(256 / n_triplets, 32) tracks and runs one candidate per thread
                                  (VELO-UT input only, else LF_ERR_ARG); 2 warp form: a track per 16
                                  lanes (two per warp when n_triplets <= 16), else per warp.  Same
                                  results; LF_ERR_ARG with a nonzero value and queue != 0. */
} lf_tuning;

/* Create a context: validates and copies geometry and parameters (the
 * constants of Sec. "Defining the search windows", "Triplet Seeding",
 * "Extending triplets to other layers" and "Quality Filter"; Table
 * tolerances, Table C_nhits, Table poly_tol).  Returns LF_ERR_ARG on a
 * parameter outside its range. */
lf_status lf_create(const lf_geometry* geometry, const lf_params* params, lf_ctx** out);

/* Release the context and its scratch (synchronises the device).
 * Infrastructure: no step of the paper. */
void lf_destroy(lf_ctx* ctx);

/* Message of the last error on this context ("" if none).  Infrastructure. */
const char* lf_last_error(const lf_ctx* ctx);

/* Number of SMs of the current device (for launch sizing).  Infrastructure. */
int32_t lf_device_sm_count(void);

/* Host NUMA node nearest to the current device (cudaDevAttrHostNumaId), or
 * -1 when the platform does not report one.  Page-locked host buffers placed
 * on that node (allocated by a thread running there) give the host link its
 * full bandwidth to this device.  Infrastructure. */
int32_t lf_device_host_numa(void);

/* Bucket and sort raw hits (the per-layer x-sorted hit containers the
 * search windows of Sec. "Defining the search windows" are index ranges
 * of): per event, buckets ordered zone*12+layer, x ascending inside a
 * bucket, ties by raw index; -0.0 becomes +0.0.  Output
 * arrays hold raw->n_hits entries and hit_offsets 24*n_events+1.  A plane
 * code >= 24 sets status flag 0x2 (the hit is counted in bucket 23); a
 * bucket above LF_MAX_BUCKET hits sets flag 0x1 and is not sorted (its perm
 * entries are -1, its other outputs meaningless).  Scratch: none beyond the
 * context's work-queue cursor. */
lf_status lf_pack_hits(lf_ctx* ctx, const lf_raw_hits* raw, const lf_packed* packed, void* stream);

/* Plain form of the whole method (Sec. "Defining the search windows",
 * "Triplet Seeding", "Extending triplets to other layers", "Quality
 * Filter", "Calculation of momentum and track states"): one launch per
 * stage (windows, triplets, extension+fit, selection, compaction) over the
 * whole batch, intermediate results in context scratch. */
lf_status lf_find_tracks(lf_ctx* ctx, const lf_batch* batch, const lf_output* out, void* stream);

/* Persistent form of the same method (the sections listed for
 * lf_find_tracks): persistent kernels over device work queues (by default a
 * pipeline of one persistent kernel per stage; see lf_tuning.queue), then
 * compaction.  The first call with a given launch shape (tuning, sizes and
 * every batch and output pointer) launches the kernels directly; when the
 * same shape comes back it is captured into a CUDA graph, which later calls
 * replay (at most 64 graphs per context, the least recently used dropped
 * first, and 256 remembered shapes), reading the buffers' current contents.
 * A call that changes any pointer or size is a new shape (lf_process_slot
 * replays one graph across batch sizes).  tuning may be NULL (defaults).  Results are identical to
 * lf_find_tracks. */
lf_status lf_find_tracks_batched(lf_ctx* ctx, const lf_batch* batch, const lf_output* out,
                                 const lf_tuning* tuning, void* stream);

/* Gather source of a slot batch (device pointers, caller-owned): batch event
 * e of lf_process_slot reads its hits from the raw arrays starting at raw
 * index hit_src[e], and its input states from sx..sqop starting at
 * trk_src[e]; the batch's own offsets give each event's counts and its place
 * in the slot's buffers. */
typedef struct {
    const int32_t* hit_src;    /* [event capacity] */
    const int32_t* trk_src;    /* [event capacity] */
    const float* sx; const float* sy; const float* stx; const float* sty; const float* sqop;
} lf_gather;

/* Slot form, for a serving loop: pack (as lf_pack_hits) and the persistent
 * find (as lf_find_tracks_batched; the method of the sections listed for
 * lf_find_tracks) of one batch held in a slot, the buffers
 * of fixed capacity a server reuses from batch to batch, with the batch's
 * event count read from device memory when the kernels run.
 *   - raw, packed, batch and out are the slot's buffers.  raw->n_events ==
 *     batch->n_events is the event capacity, raw->n_hits == batch->n_hits the
 *     hit capacity, batch->n_tracks the track capacity; the batch's hit arrays
 *     must be the packed arrays.
 *   - *n_events_dev (device int32, written by the caller on `stream` before
 *     this call) is the batch's event count n; raw->raw_offsets[0..n] and
 *     batch->trk_offsets[0..n] (device data) give its hits and tracks.  They
 *     must start at 0, not decrease and end within the capacities (the
 *     kernels clamp n to the event capacity and the track count to the track
 *     capacity; hit offsets are not checked on the device, as in
 *     lf_pack_hits).
 *   - gather == NULL: the raw arrays and the batch's state arrays hold the
 *     batch itself.  Otherwise the raw arrays are a larger hit pool that the
 *     pack reads event by event through gather->hit_src (no copy of the hits),
 *     and the states are first copied from gather's arrays into the batch's
 *     state arrays; perm then gives hit indices in the batch's own numbering
 *     (hit k of batch event e is raw index raw_offsets[e] + k).
 *   - Every call with the same buffers, gather arrays, count pointer and
 *     tuning replays one CUDA graph, captured on the first such call, whatever
 *     the batch's size (a context keeps at most 64 graphs, dropping the least
 *     recently used).  Results are identical to lf_pack_hits followed by
 *     lf_find_tracks_batched on the same batch.
 *   - LF_ERR_ARG on a NULL array, capacities that differ between raw and
 *     batch, or batch hit arrays other than the packed ones; LF_ERR_CUDA on a
 *     launch or capture error.  Asynchronous on stream. */
lf_status lf_process_slot(lf_ctx* ctx, const lf_raw_hits* raw, const lf_packed* packed, const lf_batch* batch,
                          const lf_gather* gather, const int32_t* n_events_dev, const lf_output* out,
                          const lf_tuning* tuning, void* stream);

/* Number of CUDA graphs the context has captured since its creation (the
 * batched and slot forms), or -1 for a NULL context.  Infrastructure. */
int64_t lf_graph_count(const lf_ctx* ctx);

/* Host-resident batch for lf_process_host: pointers are HOST pointers
 * (pinned memory gives full copy bandwidth; pageable memory also works). */
typedef struct {
    int32_t n_events;
    int32_t n_hits;
    int32_t n_tracks;
    const int32_t* raw_offsets;   /* [n_events+1] */
    const float* x; const float* z; const float* dxdy; const float* w;
    const uint8_t* plane;
    const int32_t* trk_offsets;   /* [n_events+1] */
    const float* sx; const float* sy; const float* stx; const float* sty; const float* sqop;
} lf_host_batch;

/* Host-resident per-track results of lf_process_host (HOST pointers).
 * hit_idx holds RAW hit indices of the input batch (-1 none); hit_idx,
 * state and quality are written only where found[t] == 1. */
typedef struct {
    uint8_t* found; uint8_t* nhits; int32_t* hit_idx; float* state; float* quality;
} lf_host_output;

/* Size the context's scratch for persistent-form batches of up to n_events
 * events, n_hits hits and n_tracks input tracks (with this tuning; NULL for
 * the defaults),
 * so that later calls within those sizes allocate nothing.  Growing scratch
 * inside a call frees and reallocates device memory, and cudaFree
 * synchronises the whole device, so a serving loop reserves once at start.
 * LF_ERR_OOM when the allocation fails.  Infrastructure: no step of the
 * paper. */
lf_status lf_reserve(lf_ctx* ctx, int32_t n_events, int32_t n_hits, int32_t n_tracks, const lf_tuning* tuning);

/* Page-locked host memory of exactly `bytes` bytes (cudaHostAlloc, portable
 * across devices) for the host-side buffers of lf_process_host and of a
 * serving loop: copies from it run asynchronously and overlap device work.
 * (Memory pinned after the fact with cudaHostRegister can give copies that
 * block the calling thread until they finish, which serialises the copies
 * with the compute queued behind them.)  *out receives the pointer (NULL
 * when bytes is 0); LF_ERR_OOM when the allocation fails.  Release with
 * lf_host_free.  Infrastructure: no step of the paper. */
lf_status lf_host_alloc(size_t bytes, void** out);
void lf_host_free(void* p);

/* End-to-end call on host buffers (the method of the sections listed for
 * lf_find_tracks, with the pack of lf_pack_hits): the batch is cut at event boundaries into
 * chunks of at most chunk_hits hits; each chunk is copied to the device,
 * packed, followed (persistent form) and its results copied back.  Three
 * internal streams (copies in, compute, copies out) chained by events over
 * three device staging slots form a pipeline: the copies in of chunk k+1,
 * the compute of chunk k and the copies out of chunk k-1 overlap.  The
 * staging slots and the compute scratch belong to the context and are sized
 * before the first copy.  Synchronous: returns after the results are in host
 * memory.  chunk_hits <= 0 selects 1<<26.  LF_ERR_ARG, before anything is
 * copied, when the offsets do not start at 0, decrease or do not end at
 * n_hits / n_tracks, or when an input array the sizes need is NULL (a NULL
 * output array is skipped); LF_ERR_CUDA on a copy or launch error, after
 * the internal streams have drained. */
lf_status lf_process_host(lf_ctx* ctx, const lf_host_batch* batch, const lf_host_output* out,
                          const lf_tuning* tuning, int64_t chunk_hits);

/* Largest batch (events) lf_find_tracks_static accepts. */
#define LF_STATIC_MAX_EVENTS 262144

/* lf_find_tracks_static — for callers that cannot allocate device memory.
 * (The paper has no counterpart: this is a deployment variant.)
 * Some callers may not call cudaMalloc: a process whose device memory is all
 * owned by its own pool, code on a latency-critical path where cudaMalloc and
 * cudaFree (which synchronises the device) are not acceptable, or a framework
 * that forbids allocation after start-up.  Such callers cannot use lf_create.
 * This call runs the same method (the sections listed for lf_find_tracks) in
 * the persistent kernel and compaction of lf_find_tracks_batched (default
 * launch shape) without a context and without
 * allocating: its scratch (work-queue cursor, per-event counts) is a static
 * device array of 4*(64 + LF_STATIC_MAX_EVENTS) bytes (about 1 MiB) that every
 * GPU loading the library keeps until the process exits.  The caller passes
 * inputs and outputs as for lf_find_tracks_batched.
 *   - The first call on a device (with that device current) looks the array's
 *     address up once; make that first call before any stream capture.  A
 *     device reset (cudaDeviceReset) may move the array: the address looked
 *     up before it is not valid after it, so do not call this entry point
 *     on a device that was reset in the same process.
 *   - All calls share the array; each call clears the cursor it needs.  Calls
 *     that overlap on the GPU (other streams, other threads) race on it.
 *   - Returns LF_ERR_CAPACITY, without launching, when batch->n_events is
 *     above LF_STATIC_MAX_EVENTS; LF_ERR_ARG on invalid parameters or a NULL
 *     pointer; LF_ERR_CUDA on a launch error.  Asynchronous on stream. */
lf_status lf_find_tracks_static(const lf_geometry* geometry, const lf_params* params, const lf_batch* batch,
                                const lf_output* out, void* stream);

/* Stage dumps of the plain form for debugging and parity tests (the windows
 * of Sec. "Defining the search windows", the kept triplets of Sec. "Triplet
 * Seeding"):
 * win_begin/win_count [n_tracks*12] (int32), n_trip [n_tracks] (int32),
 * trip [n_tracks*n_triplets*4] (int32 cfg, h0, h1, h2; packed indices),
 * trip_chi2 [n_tracks*n_triplets] (float).  Device pointers. */
lf_status lf_debug_stages(lf_ctx* ctx, const lf_batch* batch, int32_t* win_begin, int32_t* win_count,
                          int32_t* n_trip, int32_t* trip, float* trip_chi2, void* stream);

/* The same triplet dumps (win_count, n_trip, trip, trip_chi2 as above; the
 * kept triplets of Sec. "Triplet Seeding")
 * decoded from what the last lf_find_tracks_batched call on the stage
 * pipeline (lf_tuning.queue 0) left in the context's scratch, for that call's
 * batch: no stage runs again.  For parity tests of the persistent triplet
 * kernel's launch options.  LF_ERR_ARG when the scratch holds fewer tracks. */
lf_status lf_debug_triplets(lf_ctx* ctx, const lf_batch* batch, int32_t* win_count, int32_t* n_trip,
                            int32_t* trip, float* trip_chi2, void* stream);

/* Debug check of a batch, outside the hot path (the find kernels assume
 * these conventions and do not check them): hit_offsets within 0..n_hits and
 * non-decreasing; trk_offsets within 0..n_tracks, non-decreasing and ending
 * at n_tracks; then x ascending inside every (event, zone, layer) bucket of
 * Sec. "Defining the search windows" (ties allowed, NaN refused) and, if
 * given, x_coarse[i] == x[32 i] bit for bit.  Synchronises the stream.
 * Returns LF_OK, or LF_ERR_ARG with the first violation in lf_last_error
 * (the buckets are checked only once the offsets pass). */
lf_status lf_validate_batch(lf_ctx* ctx, const lf_batch* batch, void* stream);

/* Synchronise the stream, read and clear the device status word (the
 * capacity flags of the pack and of the capped windows and triplet lists of
 * Sec. "Defining the search windows" and "Triplet Seeding").
 * Returns LF_OK, LF_ERR_CAPACITY or LF_ERR_TIMEOUT; *flags gets the bits. */
lf_status lf_sync_status(lf_ctx* ctx, void* stream, int32_t* flags);

#ifdef __cplusplus
}
#endif
#endif /* LF_H */
