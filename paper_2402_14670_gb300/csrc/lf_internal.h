// Internal declarations shared by the library's translation units.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "lf.h"

namespace lfk {

constexpr int NL = 12;
constexpr int NB = 24;
constexpr int MAX_CAP = 64;     // largest n_hits_window
constexpr int MAX_NT = 32;      // largest n_triplets
constexpr int BLOCK_SORT_MAX = 16384; // largest bucket the pack sorts (LF_MAX_BUCKET)

// Geometry, parameters and the few products both the method and the oracle
// form once per call (polarity*kappa, polarity*gamma, 1000*dRatio).
struct KParams {
    float z[NL], dxdy[NL];
    float z_state, z_magnet, z_ref, kappa, gamma, dratio;
    int polarity;
    float xtol_c, xtol_p, x_asym, uv_tol;
    int cap, n_trip, min_hits;
    float K_first, K_last, p_bend, magtol_min, magtol_max, magtol_c, magtol_tx;
    float T_triplet, T_x, T_uv_scale, T_uv_min, T_ty, T_y, T_Q;
    float C_n[4];
    int no_ut;    // Sec. "No-UT tuning": two window sets per track, q/p unused
    float p_min, pt_min, x_overlap;
    float tol_c[8];
    float pol_f;  // (float)polarity
    float pk;     // pol_f * kappa
    float pg;     // pol_f * gamma
    float D;      // dratio * 1000 (model in u = dz/1000)
    float inv_T_x;  // 1/T_x when T_x is a power of two (then r^2 / T_x == r^2 * inv_T_x exactly), else 0
    int qop_poly;   // q/p from Eq. pt_kick with the polynomial field integral
    float qop_c[5][10];
    float pf_bound; // half-precision triplet pre-filter: sqrt(T_triplet) + PF_MARGIN, rounded up
};

// Half-precision pre-filter of the triplet pairs (lf_tuning.triplet_prefilter).
// It applies to a configuration whose h1 window spans at most PF_SPAN mm
// (its x relative to the window's first hit then stay below 2048, where a
// binary16 ulp is at most 1 mm) and whose h0 and h2 windows each share one z.
// PF_MARGIN bounds the difference between the binary16 distance of a hit to
// the approximate x1_expected and its exact distance to the binary32
// x1_expected: 0.5 mm for each of the two roundings to binary16, about
// 1e-3 mm for the binary16 subtraction near the cut, and the slope taken as a
// product by 1/(z2 - z0) instead of a quotient (below 0.05 mm).
constexpr float PF_SPAN = 2000.0f;
constexpr float PF_MARGIN = 1.1f;

// 1/t when t is a power of two whose reciprocal is a normal float (dividing by
// t and multiplying by 1/t then give the same correctly rounded result for any
// operand), else 0
inline float pow2_reciprocal(float t) {
    if (!(t > 0.0f) || !(t < 1e30f)) return 0.0f;
    int e = 0;
    const float m = std::frexp(t, &e);   // t = m * 2^e, m in [0.5, 1)
    if (m != 0.5f || e - 1 > 126 || e - 1 < -126) return 0.0f;
    return std::ldexp(1.0f, 1 - e);
}

struct KBatch {
    int n_events, n_hits, n_tracks;
    const int* hit_offsets;
    const float *x, *z, *dxdy, *w;
    const int* trk_offsets;
    const float *sx, *sy, *stx, *sty, *sqop;
    // slot form: the batch's event count in device memory; n_events and
    // n_tracks above are then the slot's capacities (nullptr otherwise)
    const int* n_dev;
    // every 32nd packed x (x_coarse[i] = x[32 i]), written by k_coarse for
    // the window searches (nullptr: plain binary searches)
    const float* x_coarse;
};

// Sizes of a slot batch, read when the kernel runs: the event count from
// device memory, clamped to the slot's capacity, and the track count from
// the batch's offsets, clamped likewise.  No-op outside the slot form.
__device__ __forceinline__ void slot_sizes(KBatch& b) {
    if (b.n_dev) {
        int n = *b.n_dev;
        n = n < 0 ? 0 : (n > b.n_events ? b.n_events : n);
        const int t = b.trk_offsets[n];
        b.n_tracks = t < 0 ? 0 : (t > b.n_tracks ? b.n_tracks : t);
        b.n_events = n;
    }
}
// the event count of a slot batch (n_dev set) or n (otherwise), clamped to n
__device__ __forceinline__ int slot_events(const int* n_dev, int n) {
    if (!n_dev) return n;
    const int v = *n_dev;
    return v < 0 ? 0 : (v > n ? n : v);
}

struct KOut {
    uint8_t* found;
    uint8_t* nhits;
    int* hit_idx;
    float* state;
    float* quality;
};

// One candidate of the plain form's extension stage (48 bytes).
struct CandRec {
    float Q;
    int8_t status;   // 0 accepted
    int8_t n;
    int8_t hl[NL];   // window-local hit index per layer, -1 none
    int8_t side;     // window set of the triplet (no-UT variant; 0 otherwise)
    int8_t pad[5];
    float st[6];
};
static_assert(sizeof(CandRec) == 48, "CandRec layout");

constexpr int PAIR_CAP = 512;   // (h0, h2) pairs materialised at a time per warp
constexpr int CAND_CAP = 64;    // passing triplet keys buffered per warp before a selection

// Shared-memory block of one track: window descriptors, then the staged
// window hits (x and z), 12 x cap each.  dxdy and w of the hits a candidate
// uses are read from global memory (L2) by the extension.
struct SlotHead {
    int wbeg[NL];
    int wcnt[NL];
    int zuni[NL];
    int pad[4];
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ inline size_t slot_bytes(int cap) {
    return align16(sizeof(SlotHead)) + size_t(2) * NL * cap * sizeof(float);
}
// per-warp scratch of the triplet stage: key buffer and materialised pairs;
// with the half-precision pre-filter (hp) also the two configurations' h1
// windows as binary16 pairs and their constants
constexpr size_t PF_BYTES = 2 * (MAX_CAP / 2) * 4 + 2 * 4 * sizeof(float);
__host__ __device__ inline size_t scratch_bytes(bool hp = false) {
    return align16(CAND_CAP * sizeof(unsigned long long) + PAIR_CAP * sizeof(unsigned short)) +
           (hp ? align16(PF_BYTES) : 0);
}
// shared memory of a block of nw warps holding tpw tracks per warp
__host__ __device__ inline size_t block_smem_bytes(int cap, int nw, int tpw, bool hp = false) {
    return size_t(nw) * tpw * slot_bytes(cap) + size_t(nw) * scratch_bytes(hp);
}

// ---- parameters (lf_api.cu), shared by every entry point ----
// true (message in msg) when a geometry or parameter value is outside its range
bool param_error(const lf_geometry* g, const lf_params* p, char* msg, size_t n);
// the kernels' parameter block from a checked geometry and parameter set
KParams make_kparams(const lf_geometry* g, const lf_params* p);

// ---- launchers (defined in the .cu files) ----
// persistent per-event pack; cursor: two device ints (the work queues)
// n_dev: slot form (event count in device memory, n_events and n_hits the
// capacities; nullptr otherwise); hit_src: per event, the raw index of its
// first hit (the event is read from there and written at raw_offsets[e] of
// the output; nullptr: read at raw_offsets[e])
cudaError_t launch_pack(const int* raw_offsets, const float* x, const float* z, const float* dxdy,
                        const float* w, const uint8_t* plane, int n_events, int n_hits, int* hit_offsets,
                        float* ox, float* oz, float* odxdy, float* ow, uint8_t* olayer, int* perm, int* cursor,
                        int* status, int n_sm, cudaStream_t s, const int* n_dev = nullptr,
                        const int* hit_src = nullptr, float* ocoarse = nullptr);
// slot form with a gather source: the states of batch event e's tracks are
// copied from src (starting at trk_src[e]) to the batch's state arrays
cudaError_t launch_gather_states(const KBatch& b, const int* trk_src, const float* sx, const float* sy,
                                 const float* stx, const float* sty, const float* sqop, int n_sm, cudaStream_t s);

cudaError_t launch_track_event(const KBatch& b, int* trk_event, cudaStream_t s);
// x_coarse[i] = x[32 i] for 32 i < n_hits (slot form: up to the batch's hits)
cudaError_t launch_coarse(const KBatch& b, float* x_coarse, int n_sm, cudaStream_t s);
inline size_t coarse_count(int n_hits) { return ((size_t)n_hits + 31) / 32 + 1; }
// stage kernels: cursor == nullptr launches the plain one-pass grid,
// otherwise a persistent grid of `blocks` blocks draining the stage's queue
cudaError_t launch_windows(const KParams& k, const KBatch& b, const int* trk_event, int* wbeg, uint8_t* wcnt,
                           cudaStream_t s, int* cursor = nullptr, int blocks = 0);
// prefilter 1: the half-precision pre-filter of the pairs (persistent form,
// VELO-UT input only; same results)
cudaError_t launch_triplets(const KParams& k, const KBatch& b, const int* trk_event, const int* wbeg,
                            const uint8_t* wcnt, uint64_t* keys, uint8_t* ntrip, cudaStream_t s,
                            int* cursor = nullptr, int blocks = 0, int prefilter = 0);
// with a cursor (persistent) the extension also selects and writes `o`
// form 1 (persistent, VELO-UT input): the block form, one candidate per
// thread over a tile of tracks
cudaError_t launch_extend(const KParams& k, const KBatch& b, const int* trk_event, const int* wbeg,
                          const uint8_t* wcnt, const uint64_t* keys, const uint8_t* ntrip, CandRec* cands,
                          const KOut& o, cudaStream_t s, int* cursor = nullptr, int blocks = 0, int form = 0);
cudaError_t launch_select(const KParams& k, const KBatch& b, const int* wbeg, const uint8_t* ntrip,
                          const CandRec* cands, const KOut& o, cudaStream_t s, int* cursor = nullptr,
                          int blocks = 0);
cudaError_t stage_blocks_per_sm(const KParams& k, int* out4);
// persistent tile kernel: grain = tracks per warp per tile (1 or 2; 0 picks 2
// when n_triplets <= 16)
cudaError_t launch_fused(const KParams& k, const KBatch& b, const KOut& o, int* cursor, int grain,
                         int warps_per_block, int n_blocks, cudaStream_t s);
cudaError_t fused_max_blocks_per_sm(const KParams& k, int warps_per_block, int grain, int* out);
cudaError_t launch_hits_to_raw(const uint8_t* found, int* hit_idx, const int* perm, int n_tracks, int base,
                              cudaStream_t s);
cudaError_t launch_compact(const int* trk_offsets, const uint8_t* found, int n_events, int* ev_count,
                           int* out_offsets, int* out_trk, int* n_out, cudaStream_t s, const int* n_dev = nullptr);
// batch validation (lf_validate.cu): bad2[0] <- first bad hit_offsets entry,
// bad2[1] <- first bad trk_offsets entry; then, with valid offsets,
// bad2[0] <- first packed hit out of x order inside its bucket, bad2[1] <-
// first x_coarse entry that differs from x[32 i].  bad2 preset to INT_MAX.
cudaError_t launch_validate_offsets(const KBatch& b, int* bad2, int n_sm, cudaStream_t s);
cudaError_t launch_validate_hits(const KBatch& b, int* bad2, int n_sm, cudaStream_t s);
cudaError_t launch_debug_triplets(const KParams& k, const KBatch& b, const int* wbeg, const uint8_t* wcnt,
                                  const uint64_t* keys, const uint8_t* ntrip, int* win_count_out, int* n_trip_out,
                                  int* trip_out, float* chi2_out, cudaStream_t s);

}  // namespace lfk
