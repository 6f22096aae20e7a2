/*
 * CPU oracle of the Looking Forward track-following path — TEST INFRASTRUCTURE.
 *
 * A plain, single-threaded, obviously-correct restatement of the paper's
 * method (Sec. "Algorithm logic": search windows, triplet seeding, extension,
 * quality filter; Sec. "Calculation of momentum and track states" in its
 * linear pT-kick form).  It exists only to check the CUDA library: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header or table with the CUDA path.
 *
 * Arithmetic: binary32 with round-to-nearest and no contraction (built with
 * -ffp-contract=off), expressions evaluated in the order written; a binary64
 * refit of the selected hits runs alongside (lfo_fit64).
 */
#ifndef LF_ORACLE_H
#define LF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LFO_NL 12   /* SciFi layers: three x-u-v-x stations */
#define LFO_NB 24   /* (zone, layer) buckets per event: bucket = zone*12 + layer */

typedef struct {
    float z[LFO_NL];      /* layer z (mm) */
    float dxdy[LFO_NL];   /* stereo slope: 0 for x layers, +-tan(5 deg) for u/v */
    float z_state;        /* z of the upstream state */
    float z_magnet;       /* kick plane */
    float z_ref;          /* reference plane of the T-station model (8520 mm) */
    float kappa;          /* slope kick per unit q/p (GeV rad) */
    float gamma;          /* curvature per unit q/p (GeV/mm^2) */
    float dratio;         /* dRatio (1/mm) */
    int32_t polarity;     /* +1 MagUp, -1 MagDown */
} lfo_geometry;

typedef struct {
    float xtol_c, xtol_p;       /* x_tol = xtol_c + xtol_p / p */
    float x_asym;               /* magnet asymmetry term */
    float uv_tol;               /* u/v window half width */
    int32_t n_hits_window;      /* hits kept per window (<= 64) */
    int32_t n_triplets;         /* triplets kept per input track (<= 32) */
    int32_t min_hits;           /* >= 9 */
    float K_first, K_last;      /* sagitta-like correction of x1_expected */
    float p_bend;               /* bending-sign filter applies below this p */
    float magtol_min, magtol_max, magtol_c, magtol_tx; /* doublet tolerance at the magnet */
    float T_triplet, T_x, T_uv_scale, T_uv_min, T_ty, T_y, T_Q;
    float C_n[4];               /* C(9), C(10), C(11), C(12) */
    /* Sec. "No-UT tuning": VELO-only input, q/p unknown */
    int32_t no_ut;              /* 0: VELO-UT input (q/p used), 1: no-UT variant */
    float p_min, pt_min;        /* assumed momentum: the tighter of p_min and pt_min / sin(theta) */
    float x_overlap;            /* overlap of the two one-sided windows (mm) */
    float tol_c[8];             /* c0..c7 of Eq. tol_noUT (Table poly_tol) */
    /* Sec. "Calculation of momentum and track states": qop_poly = 0 takes q/p
     * from the slope change in the linear kick form, (t_x,FT - t_x,VELO) /
     * (polarity kappa); qop_poly = 1 from Eq. pt_kick with the field integral
     * F = sum_i c_i dSlope^i (i = 0..4, dSlope = t_x,FT - t_x,VELO) whose
     * c_i = sum c_i^km t_x^k t_y^m (k + m <= 6; m even; k even for even i,
     * odd for odd i): q/p = (t_x,f / sqrt(1 + t_x,f^2 + t_y,f^2) - t_x,i /
     * sqrt(1 + t_x,i^2 + t_y,i^2)) / (polarity F).  qop_c[i][j] is c_i^km of
     * the j-th (k, m) of LFO_QOP_KM_EVEN (even i) or LFO_QOP_KM_ODD (odd i). */
    int32_t qop_poly;
    float qop_c[5][10];
} lfo_params;

/* (k, m) exponents of t_x^k t_y^m in each c_i, in coefficient order */
#define LFO_QOP_KM_EVEN {{0, 0}, {0, 2}, {0, 4}, {0, 6}, {2, 0}, {2, 2}, {2, 4}, {4, 0}, {4, 2}, {6, 0}}
#define LFO_QOP_KM_ODD  {{1, 0}, {1, 2}, {1, 4}, {3, 0}, {3, 2}, {5, 0}}

/* Outputs of lfo_find_tracks.  Per input track t (global index):
 *   found[t], nhits[t], hit_idx[t*12 + layer] (packed hit index or -1),
 *   state[t*6 + k] = (x, y, tx, ty, c, q/p) at z_ref, quality[t].
 * Optional stage dumps (NULL to skip); S = 1 window set per track, 2 in the
 * no-UT variant (side 0 the window below the straight line, 1 above):
 *   win_begin/win_count [(t*S + side)*12 + l], win_xmin/xmax/centre alike,
 *   n_trip[t], trip[(t*32 + r)*4 + {cfg + 2*side, h0, h1, h2}], trip_chi2[t*32 + r],
 *   cand_status[t*32 + r] (0 accepted, else the first failed requirement),
 *   cand_q[t*32 + r], state64[t*6 + k] (binary64 refit of the selected hits). */
typedef struct {
    uint8_t* found; uint8_t* nhits; int32_t* hit_idx; float* state; float* quality;
    int32_t* win_begin; int32_t* win_count; float* win_xmin; float* win_xmax; float* win_centre;
    int32_t* n_trip; int32_t* trip; float* trip_chi2; int32_t* cand_status; float* cand_q;
    double* state64;
} lfo_output;

#define LFO_MAX_TRIP 32

/* Sort each event's raw hits into (zone, layer) buckets, ascending x inside a
 * bucket, ties by raw index.  Returns 0, or -1 on a plane code >= 24. */
int lfo_pack(int32_t n_events, const int32_t* raw_offsets,
             const float* x, const float* z, const float* dxdy, const float* w, const uint8_t* plane,
             int32_t* hit_offsets, float* ox, float* oz, float* odxdy, float* ow,
             uint8_t* olayer, int32_t* perm);

/* lfo_pack with the events split over n_threads POSIX threads. */
int lfo_pack_mt(int32_t n_events, const int32_t* raw_offsets,
                const float* x, const float* z, const float* dxdy, const float* w, const uint8_t* plane,
                int32_t* hit_offsets, float* ox, float* oz, float* odxdy, float* ow,
                uint8_t* olayer, int32_t* perm, int32_t n_threads);

/* Run windows -> triplets -> extension -> fit/quality -> selection for every
 * input track of events [0, n_events).  x64 (optional) gives binary64 hit
 * coordinates for the state64 refit; NULL promotes the binary32 ones. */
int lfo_find_tracks(const lfo_geometry* g, const lfo_params* p, int32_t n_events,
                    const int32_t* hit_offsets, const float* x, const float* z,
                    const float* dxdy, const float* w, const double* x64,
                    const int32_t* trk_offsets, const float* sx, const float* sy,
                    const float* stx, const float* sty, const float* sqop,
                    lfo_output* out);

/* Same, with the events split over n_threads POSIX threads (the per-event
 * code is unchanged).  Used to time the oracle on all host cores. */
int lfo_find_tracks_mt(const lfo_geometry* g, const lfo_params* p, int32_t n_events,
                       const int32_t* hit_offsets, const float* x, const float* z,
                       const float* dxdy, const float* w,
                       const int32_t* trk_offsets, const float* sx, const float* sy,
                       const float* stx, const float* sty, const float* sqop,
                       lfo_output* out, int32_t n_threads);

/* Stream compaction of found tracks: out_offsets[e] = number of found tracks
 * in events before e; out_trk lists found track indices in event order.
 * Returns the total. */
int32_t lfo_compact(int32_t n_events, const int32_t* trk_offsets, const uint8_t* found,
                    int32_t* out_offsets, int32_t* out_trk);

#ifdef __cplusplus
}
#endif
#endif
