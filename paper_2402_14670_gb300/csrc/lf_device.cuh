// Device helpers of the track-following kernels (lf_track.cu): the method's
// extrapolation and window arithmetic, the fit model, warp primitives and the
// warp-vote selection.  Every helper is inline (or static), so each
// translation unit that includes this header holds its own copy.
#pragma once
#include <cstdint>

#include "lf_internal.h"

namespace lfk {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t NOKEY = ~0ull;

struct TState {
    float xs, ys, txs, tys, qop;
};

__device__ __forceinline__ bool is_x(int l) { return (l & 3) == 0 || (l & 3) == 3; }
__device__ __forceinline__ int neighbour_x(int l) { return ((l & 3) == 1) ? (l >> 2) * 4 : (l >> 2) * 4 + 3; }

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    unsigned lo = __shfl_sync(FULL, (unsigned)v, src), hi = __shfl_sync(FULL, (unsigned)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}
// IEEE quotient, out of line (keeps rarely taken or repeated divisions out of
// the unrolled loops' code)
static __device__ __noinline__ float div_call(float a, float b) { return a / b; }

// ------------------------------------------------------------------ windows

// x of the input track extrapolated to layer l (straight line to the magnet
// centre, kick, T-station model of Eq. trackfitmodel).
__device__ __forceinline__ float x_extrap(const KParams& k, const TState& s, int l) {
    float x_mag = s.xs + s.txs * (k.z_magnet - k.z_state);
    float tx_f = s.txs + k.pk * s.qop;
    float c = k.pg * s.qop;
    float dz = k.z[l] - k.z_ref;
    float t1 = tx_f * (k.z[l] - k.z_magnet);
    float t2 = c * (dz * dz);
    float t3 = 1.0f + k.dratio * dz;
    return (x_mag + t1) + t2 * t3;
}

// Assumed inverse momentum of a track without a momentum estimate: the
// tighter of p_min and pt_min / sin(theta) (Sec. "No-UT tuning").
__device__ __forceinline__ float no_ut_inv_p(const KParams& k, const TState& s) {
    float t2 = s.txs * s.txs + s.tys * s.tys;
    float sin_theta = sqrtf(t2) / sqrtf(1.0f + t2);
    float ip_pt = sin_theta / k.pt_min;
    float ip_p = 1.0f / k.p_min;
    return fminf(ip_p, ip_pt);
}

// Eq. tol_noUT (coefficients of Table poly_tol), ip = 1/p
__device__ __forceinline__ float no_ut_xtol(const KParams& k, float ip, float tx, float ty) {
    float a = k.tol_c[0] + tx * (k.tol_c[1] + k.tol_c[2] * tx);
    float b = (ty * ty) * (k.tol_c[3] + tx * (k.tol_c[4] + k.tol_c[5] * tx));
    float d = ip * (k.tol_c[6] * tx + k.tol_c[7] * ip);
    return ip * ((a + b) + d);
}

// Limits and centre of the window of layer l.  NOUT: window set `side` of
// Eq. noUT_size_window (side 0 reaches x_tol below the straight line and
// x_overlap above it, side 1 the mirror image; u/v layers alike with uv_tol).
template <bool NOUT>
__device__ __forceinline__ void window_limits(const KParams& k, const TState& s, int l, int side, float& xmin,
                                              float& xmax, float& centre) {
    if (NOUT) {
        float tol;
        if (is_x(l)) {
            centre = s.xs + s.txs * (k.z[l] - k.z_state);
            tol = no_ut_xtol(k, no_ut_inv_p(k, s), s.txs, s.tys);
        } else {
            int n = neighbour_x(l);
            float xn = s.xs + s.txs * (k.z[n] - k.z_state);
            float yl = s.ys + s.tys * (k.z[l] - k.z_state);
            centre = (xn + s.txs * (k.z[l] - k.z[n])) - yl * k.dxdy[l];
            tol = k.uv_tol;
        }
        xmin = side ? centre - k.x_overlap : centre - tol;
        xmax = side ? centre + tol : centre + k.x_overlap;
        return;
    }
    const float pmom = 1.0f / fabsf(s.qop);
    if (is_x(l)) {
        float x_tol = k.xtol_c + k.xtol_p / pmom;
        bool qpos = s.qop >= 0.0f;
        bool mu = k.polarity > 0;
        float a_left = ((qpos && mu) || (!qpos && !mu)) ? k.x_asym : 0.0f;
        float a_right = ((!qpos && mu) || (qpos && !mu)) ? k.x_asym : 0.0f;
        centre = x_extrap(k, s, l);
        xmin = (centre - x_tol) - a_left;
        xmax = (centre + x_tol) + a_right;
    } else {
        int n = neighbour_x(l);
        float tx_f = s.txs + k.pk * s.qop;
        float xn = x_extrap(k, s, n);
        float yl = s.ys + s.tys * (k.z[l] - k.z_state);
        centre = (xn + tx_f * (k.z[l] - k.z[n])) - yl * k.dxdy[l];
        xmin = centre - k.uv_tol;
        xmax = centre + k.uv_tol;
    }
}
__device__ __forceinline__ TState load_state(const KBatch& b, int t) {
    TState s;
    s.xs = __ldg(b.sx + t);
    s.ys = __ldg(b.sy + t);
    s.txs = __ldg(b.stx + t);
    s.tys = __ldg(b.sty + t);
    s.qop = __ldg(b.sqop + t);
    return s;
}
__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
    unsigned lo = __shfl_xor_sync(FULL, (unsigned)v, m), hi = __shfl_xor_sync(FULL, (unsigned)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

// Bitonic sort of 64 keys held two per lane (element lane in a, lane+32 in
// b), ascending.
__device__ __forceinline__ void warp_sort64(uint64_t& a, uint64_t& b, int lane) {
#pragma unroll
    for (int kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
                a = lo;
                b = hi;
            } else {
                uint64_t pa = shfl_xor64(a, j), pb = shfl_xor64(b, j);
                bool lower = (lane & j) == 0;
                bool up_a = (lane & kk) == 0, up_b = ((lane + 32) & kk) == 0;
                a = (lower == up_a) ? (a < pa ? a : pa) : (a < pa ? pa : a);
                b = (lower == up_b) ? (b < pb ? b : pb) : (b < pb ? pb : b);
            }
        }
    }
}

// Bitonic sort of 32 keys, one per lane, ascending.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v, int lane) {
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            uint64_t o = shfl_xor64(v, j);
            bool lower = (lane & j) == 0;
            bool up = (lane & kk) == 0;
            v = (lower == up) ? (v < o ? v : o) : (v < o ? o : v);
        }
    }
    return v;
}
struct Cand {
    int status;   // 0 accepted, 1 degenerate, 2 too few hits, 3 no stereo hit in a station, 4 t_y, 5 Q
    float Q;
    int hl[NL];
    int n;
    float st[6];
};

__device__ __forceinline__ float f2_of(float u, float D) { return (u * u) * (1.0f + D * u); }
__device__ __forceinline__ float model_x(float A, float T, float C, float u, float D) {
    return (A + T * u) + C * f2_of(u, D);
}
// ------------------------------------------------------------ momentum

// q/p of Sec. "Calculation of momentum and track states" (Eq. pt_kick) with
// the field integral as a fourth-order polynomial in dSlope whose
// coefficients are 2-D polynomials in the input slopes (the layout of
// lf_params.qop_c); every sum in entry order, the polynomial in dSlope by
// Horner's rule.  Out of line: evaluated once per accepted candidate.
static __device__ __noinline__ float qop_polynomial(const KParams& k, float tx_i, float ty_i, float tx_f, float ty_f) {
    constexpr int KE[10] = {0, 0, 0, 0, 2, 2, 2, 4, 4, 6}, ME[10] = {0, 2, 4, 6, 0, 2, 4, 0, 2, 0};
    constexpr int KO[6] = {1, 1, 1, 3, 3, 5}, MO[6] = {0, 2, 4, 0, 2, 0};
    float txp[7], typ[7];
    txp[0] = 1.0f;
    typ[0] = 1.0f;
#pragma unroll
    for (int e = 1; e < 7; ++e) {
        txp[e] = txp[e - 1] * tx_i;
        typ[e] = typ[e - 1] * ty_i;
    }
    float c[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float acc = 0.0f;
        if (i % 2 == 0) {
#pragma unroll
            for (int j = 0; j < 10; ++j) acc = acc + k.qop_c[i][j] * (txp[KE[j]] * typ[ME[j]]);
        } else {
#pragma unroll
            for (int j = 0; j < 6; ++j) acc = acc + k.qop_c[i][j] * (txp[KO[j]] * typ[MO[j]]);
        }
        c[i] = acc;
    }
    const float ds = tx_f - tx_i;
    const float F = c[0] + ds * (c[1] + ds * (c[2] + ds * (c[3] + ds * c[4])));
    const float sf = tx_f / sqrtf((1.0f + tx_f * tx_f) + ty_f * ty_f);
    const float si = tx_i / sqrtf((1.0f + tx_i * tx_i) + ty_i * ty_i);
    return (sf - si) / (k.pol_f * F);
}

// ---------------------------------------------------------------- selection

// Lowest Q among the accepted candidates of a group of G consecutive lanes
// (G = 16 or 32; candidate rank = lane within the group; ties to the lower
// rank).  The winner writes the track's output; without a winner the
// group's first lane writes found = 0.
template <int G>
__device__ __forceinline__ void group_select_write(const KOut& o, int t, bool live, int rank, bool have, float Q,
                                                   int n, const int* hglob, const float* st) {
    uint64_t key = have ? (((uint64_t)__float_as_uint(Q) << 32) | (unsigned)rank) : NOKEY;
    uint64_t best = key;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        uint64_t u = shfl_xor64(best, off);
        best = u < best ? u : best;
    }
    if (!live) return;
    if (best == NOKEY) {
        if (rank == 0) {
            o.found[t] = 0;
            o.nhits[t] = 0;
        }
        return;
    }
    if (have && key == best) {
#pragma unroll
        for (int l = 0; l < NL; ++l) o.hit_idx[(size_t)t * NL + l] = hglob[l];
#pragma unroll
        for (int q = 0; q < 6; ++q) o.state[(size_t)t * 6 + q] = st[q];
        o.quality[t] = Q;
        o.nhits[t] = (uint8_t)n;
        o.found[t] = 1;
    }
}
__device__ __forceinline__ int queue_take(int* cursor, int n, int lane) {
    int v = 0;
    if (lane == 0) v = atomicAdd(cursor, n);
    return __shfl_sync(FULL, v, 0);
}

}  // namespace lfk
