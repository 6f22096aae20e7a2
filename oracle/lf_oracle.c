/*
 * CPU oracle of the Looking Forward track-following path — TEST INFRASTRUCTURE.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Each function restates one step of the paper in the order the paper gives:
 *   windows      Sec. "Defining the search windows" (x_tol, x_asym, u/v centre,
 *                hit cap n_hits^window, Table tolerances)
 *   triplets     Sec. "Triplet Seeding" (doublet filters, x1_expected with K,
 *                chi2_triplet < T_triplet, the n_triplets smallest chi2)
 *   extension    Sec. "Extending triplets to other layers" (Eq.
 *                dratio_model_x_expected, z_ref, T_x, stereo-corrected T_uv)
 *   quality      Sec. "Quality Filter" (y fit, T_ty, Q_x, Q_y, Q, C(n_hits)
 *                from Table C_nhits, T_Q)
 *   state        Sec. "Calculation of momentum and track states", linear kick.
 *   no-UT        Sec. "No-UT tuning": straight-line extrapolation of a VELO
 *                track, assumed minimum momentum, Eq. tol_noUT window
 *                tolerance, the two one-sided windows of Eq.
 *                noUT_size_window, seeding per charge assumption.
 * Where the paper leaves a choice open the reading used is stated inline.
 *
 * Searches are plain linear scans and the triplet stage enumerates every
 * (h0, h2) pair of the two windows: no interval search, no early exit.
 *
 * Binary32 arithmetic, round to nearest, no contraction: build with
 * -ffp-contract=off.  Every expression is written in evaluation order.
 */
#include "lf_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* layer roles of an x-u-v-x station (Sec. "Context") */
static const int IS_X[LFO_NL] = {1, 0, 0, 1, 1, 0, 0, 1, 1, 0, 0, 1};
/* the x layer next to each stereo layer: u follows the first x layer of its
 * station, v precedes the last one */
static int neighbour_x(int l) { return (l % 4 == 1) ? (l / 4) * 4 : (l / 4) * 4 + 3; }
/* triplet configurations: first or last layer of each T station */
static const int CFG_L[2][3] = {{0, 4, 8}, {3, 7, 11}};
static const int CFG_MISSING[2][3] = {{3, 7, 11}, {0, 4, 8}};

/* ------------------------------------------------------------------ pack */

typedef struct { int plane; float x; int32_t raw; } pk_item;

static int pk_cmp(const void* a, const void* b)
{
    const pk_item* p = (const pk_item*)a;
    const pk_item* q = (const pk_item*)b;
    if (p->plane != q->plane) return p->plane < q->plane ? -1 : 1;
    if (p->x < q->x) return -1;
    if (p->x > q->x) return 1;
    return (p->raw > q->raw) - (p->raw < q->raw);
}

int lfo_pack(int32_t n_events, const int32_t* raw_offsets,
             const float* x, const float* z, const float* dxdy, const float* w, const uint8_t* plane,
             int32_t* hit_offsets, float* ox, float* oz, float* odxdy, float* ow,
             uint8_t* olayer, int32_t* perm)
{
    int32_t maxn = 0;
    for (int32_t e = 0; e < n_events; ++e) {
        int32_t n = raw_offsets[e + 1] - raw_offsets[e];
        if (n > maxn) maxn = n;
    }
    pk_item* it = (pk_item*)malloc(sizeof(pk_item) * (size_t)(maxn > 0 ? maxn : 1));
    if (!it) return -2;
    for (int32_t e = 0; e < n_events; ++e) {
        int32_t b0 = raw_offsets[e], n = raw_offsets[e + 1] - b0;
        int32_t count[LFO_NB];
        memset(count, 0, sizeof count);
        for (int32_t i = 0; i < n; ++i) {
            int pl = plane[b0 + i];
            if (pl >= LFO_NB) { free(it); return -1; }
            it[i].plane = pl;
            it[i].x = x[b0 + i];
            it[i].raw = b0 + i;
            count[pl]++;
        }
        qsort(it, (size_t)n, sizeof(pk_item), pk_cmp);
        int32_t acc = b0;
        for (int b = 0; b < LFO_NB; ++b) {
            hit_offsets[e * LFO_NB + b] = acc;
            acc += count[b];
        }
        for (int32_t i = 0; i < n; ++i) {
            int32_t r = it[i].raw, o = b0 + i;
            ox[o] = x[r] + 0.0f;  /* -0 -> +0; all other values unchanged */
            oz[o] = z[r];
            odxdy[o] = dxdy[r];
            ow[o] = w[r];
            olayer[o] = (uint8_t)(it[i].plane % LFO_NL);
            perm[o] = r;
        }
    }
    hit_offsets[n_events * LFO_NB] = n_events > 0 ? raw_offsets[n_events] : 0;
    free(it);
    return 0;
}

/* --------------------------------------------------------------- windows */

typedef struct {
    int32_t begin[LFO_NL], count[LFO_NL];
    float xmin[LFO_NL], xmax[LFO_NL], centre[LFO_NL];
} win_t;

typedef struct {
    float xs, ys, txs, tys, qop;
} state_t;

/* x extrapolated to layer l (Sec. "Defining the search windows"): straight
 * line to the magnet centre, slope kick there, then the T-station model of
 * Eq. trackfitmodel with curvature gamma*q/p around z_ref. */
static float x_extrap(const lfo_geometry* g, const state_t* s, int l)
{
    float pol = (float)g->polarity;
    float x_mag = s->xs + s->txs * (g->z_magnet - g->z_state);
    float tx_f = s->txs + (pol * g->kappa) * s->qop;
    float c = (pol * g->gamma) * s->qop;
    float dz = g->z[l] - g->z_ref;
    float t1 = tx_f * (g->z[l] - g->z_magnet);
    float t2 = c * (dz * dz);
    float t3 = 1.0f + g->dratio * dz;
    return (x_mag + t1) + t2 * t3;
}

/* first index in [lo, hi) with x >= v (linear scan) */
static int32_t first_ge(const float* x, int32_t lo, int32_t hi, float v)
{
    int32_t i = lo;
    while (i < hi && x[i] < v) ++i;
    return i;
}
/* first index in [lo, hi) with x > v (linear scan) */
static int32_t first_gt(const float* x, int32_t lo, int32_t hi, float v)
{
    int32_t i = lo;
    while (i < hi && !(x[i] > v)) ++i;
    return i;
}

/* Hits of bucket [b, e) inside [xmin, xmax]; above n_hits^window of them,
 * the n_hits^window placed symmetrically around the centre are kept. */
static void fill_window(const float* hx, int32_t b, int32_t e, float xmin, float xmax, float centre,
                        int cap, win_t* W, int l)
{
    int32_t lo = first_ge(hx, b, e, xmin);
    int32_t hi = first_gt(hx, lo, e, xmax);
    int32_t cnt = hi - lo;
    int32_t start = lo;
    if (cnt > cap) {
        int32_t c = first_ge(hx, lo, hi, centre);
        start = c - cap / 2;
        if (start > hi - cap) start = hi - cap;
        if (start < lo) start = lo;
        cnt = cap;
    }
    W->begin[l] = start;
    W->count[l] = cnt;
    W->xmin[l] = xmin;
    W->xmax[l] = xmax;
    W->centre[l] = centre;
}

static void track_windows(const lfo_geometry* g, const lfo_params* p, const int32_t* ev_off,
                          const float* hx, const state_t* s, win_t* W)
{
    int zone = (s->tys >= 0.0f) ? 1 : 0;         /* upper half if ty >= 0 */
    float pmom = 1.0f / fabsf(s->qop);
    float x_tol = p->xtol_c + p->xtol_p / pmom;
    /* charge x polarity decides which side gets the asymmetry term */
    int qpos = s->qop >= 0.0f;
    int mu = g->polarity > 0;
    float a_left = ((qpos && mu) || (!qpos && !mu)) ? p->x_asym : 0.0f;
    float a_right = ((!qpos && mu) || (qpos && !mu)) ? p->x_asym : 0.0f;
    float pol = (float)g->polarity;
    float tx_f = s->txs + (pol * g->kappa) * s->qop;

    for (int l = 0; l < LFO_NL; ++l) {
        float centre, xmin, xmax;
        if (IS_X[l]) {
            centre = x_extrap(g, s, l);
            xmin = (centre - x_tol) - a_left;
            xmax = (centre + x_tol) + a_right;
        } else {
            int n = neighbour_x(l);
            float xn = x_extrap(g, s, n);
            float yl = s->ys + s->tys * (g->z[l] - g->z_state);
            centre = (xn + tx_f * (g->z[l] - g->z[n])) - yl * g->dxdy[l];
            xmin = centre - p->uv_tol;
            xmax = centre + p->uv_tol;
        }
        fill_window(hx, ev_off[zone * LFO_NL + l], ev_off[zone * LFO_NL + l + 1], xmin, xmax, centre,
                    p->n_hits_window, W, l);
    }
}

/* Sec. "No-UT tuning": the momentum is unknown, so the windows assume the
 * lowest one searched for.  Of the two thresholds (p_min, and pt_min turned
 * into a momentum with the track's polar angle, p = pt_min / sin(theta)) the
 * tighter, i.e. the higher momentum, is used; returned as 1/p. */
static float assumed_inv_p(const lfo_params* p, const state_t* s)
{
    float t2 = s->txs * s->txs + s->tys * s->tys;
    float sin_theta = sqrtf(t2) / sqrtf(1.0f + t2);
    float ip_pt = sin_theta / p->pt_min;
    float ip_p = 1.0f / p->p_min;
    return fminf(ip_p, ip_pt);
}

/* Eq. tol_noUT with the coefficients of Table poly_tol, ip = 1/p_Velo */
static float no_ut_xtol(const lfo_params* p, float ip, float tx, float ty)
{
    const float* c = p->tol_c;
    float a = c[0] + tx * (c[1] + c[2] * tx);
    float b = (ty * ty) * (c[3] + tx * (c[4] + c[5] * tx));
    float d = ip * (c[6] * tx + c[7] * ip);
    return ip * ((a + b) + d);
}

/* Windows of one charge assumption (Eq. noUT_size_window): side 0 reaches
 * x_tol below the straight-line extrapolation and x_overlap above it, side 1
 * the mirror image.  The u/v windows are built the same way around the
 * stereo-corrected straight line from the neighbouring x layer, with the u/v
 * tolerance.  The window centre, around which a full window is capped, is
 * the extrapolated position (as for VELO-UT input). */
static void track_windows_no_ut(const lfo_geometry* g, const lfo_params* p, const int32_t* ev_off,
                                const float* hx, const state_t* s, int side, win_t* W)
{
    int zone = (s->tys >= 0.0f) ? 1 : 0;
    float ip = assumed_inv_p(p, s);
    float x_tol = no_ut_xtol(p, ip, s->txs, s->tys);
    for (int l = 0; l < LFO_NL; ++l) {
        float centre, tol;
        if (IS_X[l]) {
            centre = s->xs + s->txs * (g->z[l] - g->z_state);
            tol = x_tol;
        } else {
            int n = neighbour_x(l);
            float xn = s->xs + s->txs * (g->z[n] - g->z_state);
            float yl = s->ys + s->tys * (g->z[l] - g->z_state);
            centre = (xn + s->txs * (g->z[l] - g->z[n])) - yl * g->dxdy[l];
            tol = p->uv_tol;
        }
        float xmin = side ? centre - p->x_overlap : centre - tol;
        float xmax = side ? centre + tol : centre + p->x_overlap;
        fill_window(hx, ev_off[zone * LFO_NL + l], ev_off[zone * LFO_NL + l + 1], xmin, xmax, centre,
                    p->n_hits_window, W, l);
    }
}

/* closest hit to e among [b, b+n): smallest |x - e|, ties to the lower index */
static int32_t closest(const float* hx, int32_t b, int32_t n, float e)
{
    int32_t best = -1;
    float bd = 0.0f;
    for (int32_t k = 0; k < n; ++k) {
        float d = fabsf(hx[b + k] - e);
        if (best < 0 || d < bd) { best = b + k; bd = d; }
    }
    return best;
}

/* -------------------------------------------------------------- triplets */

typedef struct { float chi2; int32_t side, cfg, h0, h1, h2; } trip_t;

static int trip_cmp(const void* a, const void* b)
{
    const trip_t* p = (const trip_t*)a;
    const trip_t* q = (const trip_t*)b;
    if (p->chi2 < q->chi2) return -1;
    if (p->chi2 > q->chi2) return 1;
    if (p->side != q->side) return p->side < q->side ? -1 : 1;
    if (p->cfg != q->cfg) return p->cfg < q->cfg ? -1 : 1;
    if (p->h0 != q->h0) return p->h0 < q->h0 ? -1 : 1;
    return (p->h2 > q->h2) - (p->h2 < q->h2);
}

/* All triplets passing the doublet filters and chi2_triplet < T_triplet, then
 * the n_triplets smallest by (chi2, side, configuration, h0, h2).  With
 * VELO-UT input there is one window set (side 0); the no-UT variant seeds
 * each charge assumption in its own window set and pools the triplets. */
static int track_triplets(const lfo_geometry* g, const lfo_params* p, const float* hx,
                          const float* hz, const state_t* s, const win_t* Ws, int n_sides,
                          trip_t* buf, trip_t* out)
{
    float x_mag_in = s->xs + s->txs * (g->z_magnet - g->z_state);
    float pol = (float)g->polarity;
    int nb = 0;
    for (int side = 0; side < n_sides; ++side) {
        const win_t* W = &Ws[side];
        float pmom, bend;  /* momentum, and the sign of the expected slope change */
        if (p->no_ut) {
            pmom = 1.0f / assumed_inv_p(p, s);
            bend = side ? 1.0f : -1.0f;  /* side 1 holds the tracks bending to larger x */
        } else {
            pmom = 1.0f / fabsf(s->qop);
            bend = (s->qop > 0.0f) ? pol : -pol;
        }
        float tol_base = p->magtol_min + p->magtol_c / pmom;
        for (int cfg = 0; cfg < 2; ++cfg) {
            int L0 = CFG_L[cfg][0], L1 = CFG_L[cfg][1], L2 = CFG_L[cfg][2];
            float K = cfg == 0 ? p->K_first : p->K_last;
            float z1 = g->z[L1];
            for (int32_t i0 = 0; i0 < W->count[L0]; ++i0) {
                int32_t h0 = W->begin[L0] + i0;
                float x0 = hx[h0], z0 = hz[h0];
                for (int32_t i2 = 0; i2 < W->count[L2]; ++i2) {
                    int32_t h2 = W->begin[L2] + i2;
                    float x2 = hx[h2], z2 = hz[h2];
                    float tx_d = (x2 - x0) / (z2 - z0);
                    /* filter 1: below p_bend the doublet must bend the way the charge says */
                    if (pmom < p->p_bend) {
                        float d = tx_d - s->txs;
                        int ok = (bend > 0.0f) ? (d > 0.0f) : (d < 0.0f);
                        if (!ok) continue;
                    }
                    /* filter 2: x opening at the magnet centre within a p- and slope-dependent tolerance */
                    float x_mag_d = x0 + tx_d * (g->z_magnet - z0);
                    float tol = tol_base + p->magtol_tx * fabsf(tx_d);
                    tol = fminf(fmaxf(tol, p->magtol_min), p->magtol_max);
                    if (!(fabsf(x_mag_d - x_mag_in) < tol)) continue;
                    /* upgrade to a triplet with the closest hit to x1_expected */
                    float x1_exp = z1 * tx_d + (x0 - tx_d * z0) * K;
                    int32_t h1 = closest(hx, W->begin[L1], W->count[L1], x1_exp);
                    if (h1 < 0) continue;
                    float dx = hx[h1] - x1_exp;
                    float chi2 = dx * dx;
                    if (!(chi2 < p->T_triplet)) continue;
                    buf[nb].chi2 = chi2;
                    buf[nb].side = side;
                    buf[nb].cfg = cfg;
                    buf[nb].h0 = h0;
                    buf[nb].h1 = h1;
                    buf[nb].h2 = h2;
                    ++nb;
                }
            }
        }
    }
    qsort(buf, (size_t)nb, sizeof(trip_t), trip_cmp);
    int keep = nb < p->n_triplets ? nb : p->n_triplets;
    memcpy(out, buf, sizeof(trip_t) * (size_t)keep);
    return keep;
}

/* ---------------------------------------------------- momentum (Eq. pt_kick) */

/* q/p of Sec. "Calculation of momentum and track states" with the field
 * integral as a polynomial in dSlope whose coefficients are 2-D polynomials in
 * the VELO slopes: c_i = sum_j qop_c[i][j] t_x^k_j t_y^m_j (terms summed in
 * coefficient order), F = c_0 + dSlope (c_1 + dSlope (c_2 + dSlope (c_3 +
 * dSlope c_4))), q/p = (sin-like slope after - before) / (polarity F). */
static float qop_polynomial(const lfo_geometry* g, const lfo_params* p, float tx_i, float ty_i, float tx_f,
                            float ty_f)
{
    static const int KM_EVEN[10][2] = LFO_QOP_KM_EVEN;
    static const int KM_ODD[6][2] = LFO_QOP_KM_ODD;
    float txp[7], typ[7];
    txp[0] = 1.0f;
    typ[0] = 1.0f;
    for (int e = 1; e < 7; ++e) {
        txp[e] = txp[e - 1] * tx_i;
        typ[e] = typ[e - 1] * ty_i;
    }
    float c[5];
    for (int i = 0; i < 5; ++i) {
        float acc = 0.0f;
        int nt = (i % 2 == 0) ? 10 : 6;
        for (int j = 0; j < nt; ++j) {
            int k = (i % 2 == 0) ? KM_EVEN[j][0] : KM_ODD[j][0];
            int m = (i % 2 == 0) ? KM_EVEN[j][1] : KM_ODD[j][1];
            acc = acc + p->qop_c[i][j] * (txp[k] * typ[m]);
        }
        c[i] = acc;
    }
    float ds = tx_f - tx_i;
    float F = c[0] + ds * (c[1] + ds * (c[2] + ds * (c[3] + ds * c[4])));
    float sf = tx_f / sqrtf((1.0f + tx_f * tx_f) + ty_f * ty_f);
    float si = tx_i / sqrtf((1.0f + tx_i * tx_i) + ty_i * ty_i);
    return (sf - si) / ((float)g->polarity * F);
}

/* ------------------------------------------------------- extension + fit */

typedef struct {
    int status;              /* 0 accepted; see CS_* */
    float Q;
    int32_t hit[LFO_NL];
    int n;
    float state[6];
} cand_t;

enum { CS_OK = 0, CS_DEGENERATE = 1, CS_NHITS = 2, CS_UV_STATION = 3, CS_TY = 4, CS_Q = 5 };

/* Eq. trackfitmodel in scaled units u = (z - z_ref)/1000 mm:
 *   x = A + T u + C u^2 (1 + D u),  T = 1e3 t_x,  C = 1e6 c_x,  D = 1e3 dRatio */
static float f2_of(float u, float D) { return (u * u) * (1.0f + D * u); }
static float u_of(const lfo_geometry* g, float z) { return (z - g->z_ref) * 1e-3f; }
static float model_x(float A, float T, float C, float u, float D) { return (A + T * u) + C * f2_of(u, D); }

static void extend_fit(const lfo_geometry* g, const lfo_params* p, const float* hx,
                       const float* hz, const float* hdxdy, const float* hw, const state_t* s,
                       const win_t* W, const trip_t* tr, cand_t* cd)
{
    float D = g->dratio * 1000.0f;
    for (int l = 0; l < LFO_NL; ++l) cd->hit[l] = -1;
    cd->Q = 0.0f;
    cd->n = 0;
    const int* Ls = CFG_L[tr->cfg];
    int32_t hh[3] = {tr->h0, tr->h1, tr->h2};
    for (int k = 0; k < 3; ++k) cd->hit[Ls[k]] = hh[k];

    /* three-point solution through the triplet (a_x, t_x, c_x with fixed dRatio) */
    float x0 = hx[tr->h0], x1 = hx[tr->h1], x2 = hx[tr->h2];
    float u0 = u_of(g, hz[tr->h0]), u1 = u_of(g, hz[tr->h1]), u2 = u_of(g, hz[tr->h2]);
    float g0 = f2_of(u0, D), g1 = f2_of(u1, D), g2 = f2_of(u2, D);
    float d1 = u1 - u0, d2 = u2 - u0;
    float e1 = g1 - g0, e2 = g2 - g0;
    float r1 = x1 - x0, r2 = x2 - x0;
    float det = d1 * e2 - d2 * e1;
    if (!(det != 0.0f)) { cd->status = CS_DEGENERATE; return; }
    float T = (r1 * e2 - r2 * e1) / det;
    float C = (d1 * r2 - d2 * r1) / det;
    float A = (x0 - T * u0) - C * g0;

    /* extension to the three missing x layers: closest hit, chi2 < T_x */
    for (int k = 0; k < 3; ++k) {
        int l = CFG_MISSING[tr->cfg][k];
        float xe = model_x(A, T, C, u_of(g, g->z[l]), D);
        int32_t h = closest(hx, W->begin[l], W->count[l], xe);
        if (h < 0) continue;
        float dx = hx[h] - xe;
        if (dx * dx < p->T_x) cd->hit[l] = h;
    }

    /* weighted least-squares refit of (A, T, C) on all x hits, as a
     * correction to the three-point solution; sums in layer order */
    float S00 = 0, S01 = 0, S02 = 0, S11 = 0, S12 = 0, S22 = 0, b0 = 0, b1 = 0, b2 = 0;
    for (int l = 0; l < LFO_NL; ++l) {
        if (!IS_X[l] || cd->hit[l] < 0) continue;
        int32_t h = cd->hit[l];
        float u = u_of(g, hz[h]);
        float f = f2_of(u, D);
        float r = hx[h] - model_x(A, T, C, u, D);
        float wt = hw[h];
        float wu = wt * u, wf = wt * f;
        S00 = S00 + wt; S01 = S01 + wu; S02 = S02 + wf;
        S11 = S11 + wu * u; S12 = S12 + wu * f; S22 = S22 + wf * f;
        b0 = b0 + wt * r; b1 = b1 + wu * r; b2 = b2 + wf * r;
    }
    float c00 = S11 * S22 - S12 * S12;
    float c01 = S02 * S12 - S01 * S22;
    float c02 = S01 * S12 - S02 * S11;
    float c11 = S00 * S22 - S02 * S02;
    float c12 = S01 * S02 - S00 * S12;
    float c22 = S00 * S11 - S01 * S01;
    float dt = (S00 * c00 + S01 * c01) + S02 * c02;
    if (!(dt != 0.0f)) { cd->status = CS_DEGENERATE; return; }
    A = A + ((c00 * b0 + c01 * b1) + c02 * b2) / dt;
    T = T + ((c01 * b0 + c11 * b1) + c12 * b2) / dt;
    C = C + ((c02 * b0 + c12 * b1) + c22 * b2) / dt;

    /* extension to the u/v layers: x model corrected by the stereo angle,
     * y from the input state; tolerance grows with the slopes */
    float T_uv = p->T_uv_scale * (fabsf(s->txs) + fabsf(s->tys));
    T_uv = fmaxf(p->T_uv_min, T_uv);
    for (int l = 0; l < LFO_NL; ++l) {
        if (IS_X[l]) continue;
        float yl = s->ys + s->tys * (g->z[l] - g->z_state);
        float xe = model_x(A, T, C, u_of(g, g->z[l]), D) - yl * g->dxdy[l];
        int32_t h = closest(hx, W->begin[l], W->count[l], xe);
        if (h < 0) continue;
        float dx = hx[h] - xe;
        if (dx * dx < T_uv) cd->hit[l] = h;
    }

    /* content requirements: >= min_hits, >= 1 stereo hit per station */
    int n_x = 0, n_uv = 0, st_uv[3] = {0, 0, 0};
    for (int l = 0; l < LFO_NL; ++l) {
        if (cd->hit[l] < 0) continue;
        if (IS_X[l]) ++n_x; else { ++n_uv; st_uv[l / 4]++; }
    }
    int n = n_x + n_uv;
    cd->n = n;
    if (n < p->min_hits) { cd->status = CS_NHITS; return; }
    if (!st_uv[0] || !st_uv[1] || !st_uv[2]) { cd->status = CS_UV_STATION; return; }

    /* quality filter: linear y fit from the stereo hits */
    float Y0s = 0, Y1s = 0, Y2s = 0, yb0 = 0, yb1 = 0;
    float yv[LFO_NL];
    for (int l = 0; l < LFO_NL; ++l) {
        if (IS_X[l] || cd->hit[l] < 0) continue;
        int32_t h = cd->hit[l];
        float u = u_of(g, hz[h]);
        float y = (model_x(A, T, C, u, D) - hx[h]) / hdxdy[h];
        yv[l] = y;
        float wt = hw[h];
        float wu = wt * u;
        Y0s = Y0s + wt; Y1s = Y1s + wu; Y2s = Y2s + wu * u;
        yb0 = yb0 + wt * y; yb1 = yb1 + wu * y;
    }
    float ydet = Y0s * Y2s - Y1s * Y1s;
    if (!(ydet != 0.0f)) { cd->status = CS_DEGENERATE; return; }
    float Y0 = (Y2s * yb0 - Y1s * yb1) / ydet;
    float TY = (Y0s * yb1 - Y1s * yb0) / ydet;
    float ty_fit = TY * 1e-3f;
    if (!(fabsf(ty_fit - s->tys) < p->T_ty)) { cd->status = CS_TY; return; }

    /* Q_x, Q_y against the final fits, then Q with C(n_hits) */
    float qx = 0.0f, qy = 0.0f;
    for (int l = 0; l < LFO_NL; ++l) {
        if (cd->hit[l] < 0) continue;
        int32_t h = cd->hit[l];
        float u = u_of(g, hz[h]);
        float xf = model_x(A, T, C, u, D);
        if (IS_X[l]) {
            float r = hx[h] - xf;
            qx = qx + (r * r) / p->T_x;
        } else {
            float yf = Y0 + TY * u;
            float r = hx[h] - (xf - yf * hdxdy[h]);
            qx = qx + (r * r) / T_uv;
            float ry = yv[l] - yf;
            qy = qy + (ry * ry) / p->T_y;
        }
    }
    float Q = (qx / (float)(n - 3) + qy / (float)(n_uv - 2)) * p->C_n[n - 9];
    cd->Q = Q;
    if (!(Q < p->T_Q)) { cd->status = CS_Q; return; }
    cd->status = CS_OK;

    /* state at z_ref and q/p from the slope change (linear kick) */
    float tx = T * 1e-3f;
    cd->state[0] = A;
    cd->state[1] = Y0;
    cd->state[2] = tx;
    cd->state[3] = ty_fit;
    cd->state[4] = C * 1e-6f;
    if (p->qop_poly)
        cd->state[5] = qop_polynomial(g, p, s->txs, s->tys, tx, ty_fit);
    else
        cd->state[5] = (tx - s->txs) / ((float)g->polarity * g->kappa);
}

/* ------------------------------------------------------- binary64 refit */

/* Direct weighted least squares of Eq. trackfitmodel (unscaled dz) on the x
 * hits and of the straight y line on the stereo hits, in binary64.  Inputs
 * are indexed by layer; has[l] == 0 marks a layer without a hit. */
static void fit64(const lfo_geometry* g, const lfo_params* p, const int* has, const double* hx, const float* hz,
                  const float* hdxdy, const float* hw, const state_t* s, double* st)
{
    double zr = g->z_ref, dR = g->dratio;
    double M[3][4] = {{0}};
    for (int l = 0; l < LFO_NL; ++l) {
        if (!IS_X[l] || !has[l]) continue;
        double dz = (double)hz[l] - zr;
        double f[3] = {1.0, dz, dz * dz * (1.0 + dR * dz)};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) M[i][j] += hw[l] * f[i] * f[j];
            M[i][3] += hw[l] * f[i] * hx[l];
        }
    }
    /* Gauss-Jordan elimination with partial pivoting */
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r) if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        for (int k = 0; k < 4; ++k) { double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
        for (int r = 0; r < 3; ++r) {
            if (r == c || M[c][c] == 0.0) continue;
            double fac = M[r][c] / M[c][c];
            for (int k = c; k < 4; ++k) M[r][k] -= fac * M[c][k];
        }
    }
    double a = M[0][3] / M[0][0], t = M[1][3] / M[1][1], c = M[2][3] / M[2][2];
    double s0 = 0, s1 = 0, s2 = 0, r0 = 0, r1 = 0;
    for (int l = 0; l < LFO_NL; ++l) {
        if (IS_X[l] || !has[l]) continue;
        double dz = (double)hz[l] - zr;
        double xf = a + t * dz + c * dz * dz * (1.0 + dR * dz);
        double y = (xf - hx[l]) / (double)hdxdy[l];
        double wt = hw[l];
        s0 += wt; s1 += wt * dz; s2 += wt * dz * dz; r0 += wt * y; r1 += wt * dz * y;
    }
    double det = s0 * s2 - s1 * s1;
    double y0 = (s2 * r0 - s1 * r1) / det;
    double ty = (s0 * r1 - s1 * r0) / det;
    st[0] = a; st[1] = y0; st[2] = t; st[3] = ty; st[4] = c;
    if (p->qop_poly) {
        /* Eq. pt_kick with the polynomial field integral, in binary64 */
        static const int KM_EVEN[10][2] = LFO_QOP_KM_EVEN;
        static const int KM_ODD[6][2] = LFO_QOP_KM_ODD;
        double txi = s->txs, tyi = s->tys, c[5];
        for (int i = 0; i < 5; ++i) {
            c[i] = 0.0;
            int nt = (i % 2 == 0) ? 10 : 6;
            for (int j = 0; j < nt; ++j) {
                int k = (i % 2 == 0) ? KM_EVEN[j][0] : KM_ODD[j][0];
                int m = (i % 2 == 0) ? KM_EVEN[j][1] : KM_ODD[j][1];
                c[i] += (double)p->qop_c[i][j] * pow(txi, k) * pow(tyi, m);
            }
        }
        double ds = t - txi;
        double F = c[0] + ds * (c[1] + ds * (c[2] + ds * (c[3] + ds * c[4])));
        double sf = t / sqrt(1.0 + t * t + ty * ty), si = txi / sqrt(1.0 + txi * txi + tyi * tyi);
        st[5] = (sf - si) / ((double)g->polarity * F);
    } else {
        st[5] = (t - (double)s->txs) / ((double)g->polarity * (double)g->kappa);
    }
}

/* ------------------------------------------------------------ per event */

static int find_event_range(const lfo_geometry* g, const lfo_params* p, int32_t e0, int32_t e1,
                            const int32_t* hit_offsets, const float* x, const float* z,
                            const float* dxdy, const float* w, const double* x64,
                            const int32_t* trk_offsets, const float* sx, const float* sy,
                            const float* stx, const float* sty, const float* sqop,
                            lfo_output* out)
{
    int cap = p->n_hits_window;
    const int n_sides = p->no_ut ? 2 : 1;
    trip_t* buf = (trip_t*)malloc(sizeof(trip_t) * 2 * (size_t)n_sides * (size_t)cap * (size_t)cap + sizeof(trip_t));
    if (!buf) return -2;
    trip_t trips[LFO_MAX_TRIP];
    cand_t cd;
    for (int32_t e = e0; e < e1; ++e) {
        const int32_t* ev_off = hit_offsets + (size_t)e * LFO_NB;
        for (int32_t t = trk_offsets[e]; t < trk_offsets[e + 1]; ++t) {
            state_t s = {sx[t], sy[t], stx[t], sty[t], sqop[t]};
            win_t Ws[2];
            if (p->no_ut) {
                track_windows_no_ut(g, p, ev_off, x, &s, 0, &Ws[0]);
                track_windows_no_ut(g, p, ev_off, x, &s, 1, &Ws[1]);
            } else {
                track_windows(g, p, ev_off, x, &s, &Ws[0]);
            }
            if (out->win_begin) for (int sd = 0; sd < n_sides; ++sd) for (int l = 0; l < LFO_NL; ++l) {
                size_t i = ((size_t)t * n_sides + sd) * LFO_NL + l;
                out->win_begin[i] = Ws[sd].begin[l];
                out->win_count[i] = Ws[sd].count[l];
                if (out->win_xmin) {
                    out->win_xmin[i] = Ws[sd].xmin[l];
                    out->win_xmax[i] = Ws[sd].xmax[l];
                    out->win_centre[i] = Ws[sd].centre[l];
                }
            }
            int nt = track_triplets(g, p, x, z, &s, Ws, n_sides, buf, trips);
            if (out->n_trip) {
                out->n_trip[t] = nt;
                for (int r = 0; r < nt; ++r) {
                    int32_t* q = out->trip + ((size_t)t * LFO_MAX_TRIP + r) * 4;
                    q[0] = trips[r].cfg + 2 * trips[r].side;
                    q[1] = trips[r].h0; q[2] = trips[r].h1; q[3] = trips[r].h2;
                    out->trip_chi2[(size_t)t * LFO_MAX_TRIP + r] = trips[r].chi2;
                }
            }
            /* best candidate: lowest Q among accepted ones, ties to the lower triplet rank */
            int best = -1;
            cand_t bc;
            memset(&bc, 0, sizeof bc);
            for (int r = 0; r < nt; ++r) {
                /* the triplet's own window set: its charge assumption */
                extend_fit(g, p, x, z, dxdy, w, &s, &Ws[trips[r].side], &trips[r], &cd);
                if (out->cand_status) {
                    out->cand_status[(size_t)t * LFO_MAX_TRIP + r] = cd.status;
                    out->cand_q[(size_t)t * LFO_MAX_TRIP + r] = cd.Q;
                }
                if (cd.status == CS_OK && (best < 0 || cd.Q < bc.Q)) { best = r; bc = cd; }
            }
            out->found[t] = best >= 0;
            out->nhits[t] = best >= 0 ? (uint8_t)bc.n : 0;
            out->quality[t] = best >= 0 ? bc.Q : 0.0f;
            for (int l = 0; l < LFO_NL; ++l) out->hit_idx[(size_t)t * LFO_NL + l] = best >= 0 ? bc.hit[l] : -1;
            for (int k = 0; k < 6; ++k) out->state[(size_t)t * 6 + k] = best >= 0 ? bc.state[k] : 0.0f;
            if (out->state64) {
                double* st = out->state64 + (size_t)t * 6;
                if (best >= 0) {
                    int has[LFO_NL];
                    double hx[LFO_NL];
                    float hz[LFO_NL], hd[LFO_NL], hw[LFO_NL];
                    for (int l = 0; l < LFO_NL; ++l) {
                        int32_t h = bc.hit[l];
                        has[l] = h >= 0;
                        hx[l] = h >= 0 ? (x64 ? x64[h] : (double)x[h]) : 0.0;
                        hz[l] = h >= 0 ? z[h] : 0.0f;
                        hd[l] = h >= 0 ? dxdy[h] : 0.0f;
                        hw[l] = h >= 0 ? w[h] : 0.0f;
                    }
                    fit64(g, p, has, hx, hz, hd, hw, &s, st);
                } else {
                    for (int k = 0; k < 6; ++k) st[k] = 0.0;
                }
            }
        }
    }
    free(buf);
    return 0;
}

static int check_params(const lfo_params* p)
{
    if (p->n_hits_window < 1 || p->n_hits_window > 64) return -3;
    if (p->n_triplets < 0 || p->n_triplets > LFO_MAX_TRIP) return -3;
    if (p->min_hits < 9 || p->min_hits > 12) return -3;
    if (p->no_ut != 0 && p->no_ut != 1) return -3;
    if (p->no_ut && !(p->p_min > 0.0f && p->pt_min > 0.0f && p->x_overlap >= 0.0f)) return -3;
    return 0;
}

int lfo_find_tracks(const lfo_geometry* g, const lfo_params* p, int32_t n_events,
                    const int32_t* hit_offsets, const float* x, const float* z,
                    const float* dxdy, const float* w, const double* x64,
                    const int32_t* trk_offsets, const float* sx, const float* sy,
                    const float* stx, const float* sty, const float* sqop,
                    lfo_output* out)
{
    int rc = check_params(p);
    if (rc) return rc;
    return find_event_range(g, p, 0, n_events, hit_offsets, x, z, dxdy, w, x64, trk_offsets,
                            sx, sy, stx, sty, sqop, out);
}

typedef struct {
    const lfo_geometry* g; const lfo_params* p; int32_t e0, e1;
    const int32_t* hit_offsets; const float *x, *z, *dxdy, *w;
    const int32_t* trk_offsets; const float *sx, *sy, *stx, *sty, *sqop;
    lfo_output* out; int rc;
} mt_job;

static void* mt_run(void* arg)
{
    mt_job* j = (mt_job*)arg;
    j->rc = find_event_range(j->g, j->p, j->e0, j->e1, j->hit_offsets, j->x, j->z, j->dxdy, j->w,
                             NULL, j->trk_offsets, j->sx, j->sy, j->stx, j->sty, j->sqop, j->out);
    return NULL;
}

int lfo_find_tracks_mt(const lfo_geometry* g, const lfo_params* p, int32_t n_events,
                       const int32_t* hit_offsets, const float* x, const float* z,
                       const float* dxdy, const float* w,
                       const int32_t* trk_offsets, const float* sx, const float* sy,
                       const float* stx, const float* sty, const float* sqop,
                       lfo_output* out, int32_t n_threads)
{
    int rc = check_params(p);
    if (rc) return rc;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 1024) n_threads = 1024;
    pthread_t th[1024];
    mt_job jobs[1024];
    /* interleave events over threads in contiguous chunks */
    int32_t per = (n_events + n_threads - 1) / n_threads;
    int started = 0;
    for (int i = 0; i < n_threads; ++i) {
        int32_t e0 = i * per, e1 = e0 + per;
        if (e1 > n_events) e1 = n_events;
        if (e0 >= e1) break;
        mt_job jb = {g, p, e0, e1, hit_offsets, x, z, dxdy, w, trk_offsets, sx, sy, stx, sty, sqop, out, 0};
        jobs[i] = jb;
        if (pthread_create(&th[i], NULL, mt_run, &jobs[i]) != 0) { jobs[i].rc = -4; break; }
        ++started;
    }
    rc = 0;
    for (int i = 0; i < started; ++i) {
        pthread_join(th[i], NULL);
        if (jobs[i].rc) rc = jobs[i].rc;
    }
    return rc;
}

/* pack with the events split over n_threads POSIX threads (the per-event
 * code is lfo_pack's; offsets are absolute, so ranges are independent) */
typedef struct {
    int32_t e0, e1; const int32_t* raw_offsets; const float *x, *z, *dxdy, *w; const uint8_t* plane;
    int32_t* hit_offsets; float *ox, *oz, *odxdy, *ow; uint8_t* olayer; int32_t* perm; int rc;
} pk_job;

static void* pk_run(void* arg)
{
    pk_job* j = (pk_job*)arg;
    int32_t n = j->e1 - j->e0;
    /* run lfo_pack on the sub-range: it writes hit_offsets[e*24 ..] for its
     * events relative to the sub-range base, so shift the pointer */
    j->rc = lfo_pack(n, j->raw_offsets + j->e0, j->x, j->z, j->dxdy, j->w, j->plane,
                     j->hit_offsets + (size_t)j->e0 * LFO_NB, j->ox, j->oz, j->odxdy, j->ow, j->olayer, j->perm);
    return NULL;
}

int lfo_pack_mt(int32_t n_events, const int32_t* raw_offsets,
                const float* x, const float* z, const float* dxdy, const float* w, const uint8_t* plane,
                int32_t* hit_offsets, float* ox, float* oz, float* odxdy, float* ow,
                uint8_t* olayer, int32_t* perm, int32_t n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 1024) n_threads = 1024;
    pthread_t th[1024];
    pk_job jobs[1024];
    int32_t per = (n_events + n_threads - 1) / n_threads;
    int started = 0, rc = 0;
    for (int i = 0; i < n_threads; ++i) {
        int32_t e0 = i * per, e1 = e0 + per;
        if (e1 > n_events) e1 = n_events;
        if (e0 >= e1) break;
        pk_job jb = {e0, e1, raw_offsets, x, z, dxdy, w, plane, hit_offsets, ox, oz, odxdy, ow, olayer, perm, 0};
        jobs[i] = jb;
        if (pthread_create(&th[i], NULL, pk_run, &jobs[i]) != 0) { rc = -4; break; }
        ++started;
    }
    for (int i = 0; i < started; ++i) {
        pthread_join(th[i], NULL);
        if (jobs[i].rc) rc = jobs[i].rc;
    }
    return rc;
}

/* ------------------------------------------------------------- compaction */

int32_t lfo_compact(int32_t n_events, const int32_t* trk_offsets, const uint8_t* found,
                    int32_t* out_offsets, int32_t* out_trk)
{
    int32_t n = 0;
    for (int32_t e = 0; e < n_events; ++e) {
        out_offsets[e] = n;
        for (int32_t t = trk_offsets[e]; t < trk_offsets[e + 1]; ++t)
            if (found[t]) out_trk[n++] = t;
    }
    out_offsets[n_events] = n;
    return n;
}
