// Forward-tracking kernels for sm_103a.
//
// One warp follows one input track.  The stages are device functions shared
// by the plain form (one kernel per stage, results in scratch) and the
// persistent form (all stages in one kernel, results in shared memory and
// registers, input-track grains taken from a device work queue).
//
//   windows    Sec. "Defining the search windows": lanes 0..11 each open one
//              layer's window with binary searches in the x-sorted bucket.
//   staging    the window hits (x, z, dxdy, w; <= n_hits_window per layer)
//              are copied into the warp's shared-memory block with coalesced
//              loads, once per track.
//   triplets   Sec. "Triplet Seeding": for each h0 the h2 candidates that can
//              pass the magnet-opening filter form an interval of the sorted
//              window (bounded with the largest tolerance plus slack); the
//              (h0, h2) pairs of all intervals are flattened across the 32
//              lanes, each pair gets the exact filters, the closest h1 and
//              chi2_triplet, and passing triplets are merged into a sorted
//              list of the n_triplets smallest (chi2, cfg, h0, h2) keys held
//              one per lane.  The exact filters on a superset give the same
//              triplet set as enumerating every pair.
//   extension  Sec. "Extending triplets to other layers" and "Quality Filter":
//              lane r extends triplet r (three-point solution, missing x
//              layers, weighted x refit, u/v layers, y line fit, Q).
//   selection  lowest Q among accepted candidates by a warp-wide minimum of
//              (Q bits, rank); the winner's hits and state go out coalesced.
//
// Arithmetic: binary32, no contraction (built with -fmad=false), IEEE
// division; every expression is written in the evaluation order of the
// method's definition so that results do not depend on the launch shape.
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
__device__ __forceinline__ uint64_t shfl64_up(uint64_t v, int d) {
    unsigned lo = __shfl_up_sync(FULL, (unsigned)v, d), hi = __shfl_up_sync(FULL, (unsigned)(v >> 32), d);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t u = ((uint64_t)__shfl_xor_sync(FULL, (unsigned)(v >> 32), o) << 32) |
                     __shfl_xor_sync(FULL, (unsigned)v, o);
        v = u < v ? u : v;
    }
    return v;
}
__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// first index in [lo, hi) with x >= v
__device__ __forceinline__ int lb_global(const float* __restrict__ x, int lo, int hi, float v) {
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (__ldg(x + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
// first index in [lo, hi) with x > v
__device__ __forceinline__ int ub_global(const float* __restrict__ x, int lo, int hi, float v) {
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (!(__ldg(x + mid) > v)) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int lb_smem(const float* x, int n, float v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (x[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int ub_smem(const float* x, int n, float v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (!(x[mid] > v)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Closest hit to e in a sorted window of n hits: smallest |x - e|, ties to
// the lower index.  |x - e| is non-increasing below the first x >= e and
// non-decreasing from it (rounding is monotone), so the answer is the first
// index of the run of equal distances just below that point, or that point.
__device__ __forceinline__ int closest_smem(const float* x, int n, float e) {
    int j = lb_smem(x, n, e);
    int best = -1;
    float bd = 0.0f;
    if (j > 0) {
        int k = j - 1;
        float d = fabsf(x[k] - e);
        while (k > 0 && fabsf(x[k - 1] - e) == d) --k;
        best = k;
        bd = d;
    }
    if (j < n) {
        float d = fabsf(x[j] - e);
        if (best < 0 || d < bd) best = j;
    }
    return best;
}

// ----------------------------------------------------------- stage: windows

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

// Window of layer l: [begin, begin+count) in packed hit indices.
__device__ __forceinline__ void layer_window(const KParams& k, const KBatch& b, const TState& s, int e, int l,
                                             int& begin, int& count) {
    const int zone = (s.tys >= 0.0f) ? 1 : 0;
    const float pmom = 1.0f / fabsf(s.qop);
    float centre, xmin, xmax;
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
    const int* off = b.hit_offsets + (size_t)e * NB + zone * NL + l;
    int bb = __ldg(off), be = __ldg(off + 1);
    int lo = lb_global(b.x, bb, be, xmin);
    int hi = ub_global(b.x, lo, be, xmax);
    int cnt = hi - lo, start = lo;
    if (cnt > k.cap) {
        int c = lb_global(b.x, lo, hi, centre);
        start = c - k.cap / 2;
        if (start > hi - k.cap) start = hi - k.cap;
        if (start < lo) start = lo;
        cnt = k.cap;
    }
    begin = start;
    count = cnt;
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

struct WarpSmem {
    WarpHead* h;
    float *wx, *wz, *wd, *ww;
};

__device__ __forceinline__ WarpSmem warp_smem(char* base, int warp, int cap) {
    char* p = base + (size_t)warp * warp_smem_bytes(cap);
    WarpSmem m;
    m.h = reinterpret_cast<WarpHead*>(p);
    float* f = reinterpret_cast<float*>(p + align16(sizeof(WarpHead)));
    m.wx = f;
    m.wz = f + NL * cap;
    m.wd = f + 2 * NL * cap;
    m.ww = f + 3 * NL * cap;
    return m;
}

// Copy the window hits into shared memory (coalesced, one layer at a time)
// and note which windows hold hits of a single z.
__device__ __forceinline__ void stage_windows(const KParams& k, const KBatch& b, const WarpSmem& m, int lane) {
    const int cap = k.cap;
#pragma unroll 1
    for (int l = 0; l < NL; ++l) {
        int beg = m.h->wbeg[l], cnt = m.h->wcnt[l];
        bool same = true;
        for (int j = lane; j < cnt; j += 32) {
            float zz = __ldg(b.z + beg + j);
            m.wx[l * cap + j] = __ldg(b.x + beg + j);
            m.wz[l * cap + j] = zz;
            m.wd[l * cap + j] = __ldg(b.dxdy + beg + j);
            m.ww[l * cap + j] = __ldg(b.w + beg + j);
            same = same && (zz == __ldg(b.z + beg));
        }
        unsigned all = __ballot_sync(FULL, same);
        if (lane == 0) m.h->zuni[l] = (all == FULL);
    }
    __syncwarp();
}

// ---------------------------------------------------------- stage: triplets

// Returns this lane's entry of the sorted list of kept triplet keys
// (lane r holds rank r; NOKEY past the end) and the list length.
// key = chi2 bits << 32 | cfg << 18 | j0 << 12 | j2 << 6 | j1 (window-local
// indices), which orders by (chi2, cfg, h0, h2).
__device__ __forceinline__ uint64_t triplet_scan(const KParams& k, const TState& s, const WarpSmem& m, int lane,
                                                 int& n_trip) {
    const int cap = k.cap;
    const int NT = k.n_trip;
    const float pmom = 1.0f / fabsf(s.qop);
    const float x_mag_in = s.xs + s.txs * (k.z_magnet - k.z_state);
    const float bend = (s.qop > 0.0f) ? k.pol_f : -k.pol_f;
    const float tol_base = k.magtol_min + k.magtol_c / pmom;
    const bool f1 = pmom < k.p_bend;
    const int c0 = m.h->wcnt[0], c1 = m.h->wcnt[3];
    const int n_items = c0 + c1;

    // h2 interval of each h0 item (items lane, lane+32, lane+64, lane+96)
    constexpr int NIT = (2 * MAX_CAP) / 32;
    int n_it[NIT], a_it[NIT];
#pragma unroll
    for (int part = 0; part < NIT; ++part) {
        int i = lane + 32 * part;
        int n = 0, a = 0;
        if (i < n_items) {
            int cfg = i < c0 ? 0 : 1;
            int j0 = cfg ? i - c0 : i;
            int L0 = cfg ? 3 : 0, L2 = cfg ? 11 : 8;
            float x0 = m.wx[L0 * cap + j0], z0 = m.wz[L0 * cap + j0];
            int n2 = m.h->wcnt[L2];
            n = n2;
            if (n2 > 0 && m.h->zuni[L2]) {
                float z2 = m.wz[L2 * cap];
                float r = (k.z_magnet - z0) / (z2 - z0);
                if (z2 > z0 && r < 0.0f) {
                    // |x0 + (x2 - x0) r - x_mag_in| < magtol_max, widened by a
                    // slack far above the rounding of the exact test
                    float slack = 0.5f + 1e-4f * (fabsf(x0) + fabsf(x_mag_in));
                    float lo = x0 + (x_mag_in - x0 + k.magtol_max) / r - slack;
                    float hi = x0 + (x_mag_in - x0 - k.magtol_max) / r + slack;
                    const float* x2w = m.wx + L2 * cap;
                    a = lb_smem(x2w, n2, lo);
                    int bnd = ub_smem(x2w, n2, hi);
                    n = bnd > a ? bnd - a : 0;
                }
            }
        }
        n_it[part] = n;
        a_it[part] = a;
    }
    int P = 0;
#pragma unroll
    for (int part = 0; part < NIT; ++part) {
        int inc = warp_incl_scan(n_it[part], lane);
        m.h->pre[lane + 32 * part] = P + inc - n_it[part];
        m.h->aa[lane + 32 * part] = a_it[part];
        P += __shfl_sync(FULL, inc, 31);
    }
    __syncwarp();

    uint64_t top = NOKEY;
#pragma unroll 1
    for (int base = 0; base < P; base += 32) {
        int p = base + lane;
        bool valid = false;
        uint64_t key = NOKEY;
        if (p < P) {
            int lo = 0, hi = 2 * MAX_CAP;
            while (lo < hi) {
                int mid = lo + ((hi - lo) >> 1);
                if (m.h->pre[mid] <= p) lo = mid + 1; else hi = mid;
            }
            int item = lo - 1;
            int cfg = item < c0 ? 0 : 1;
            int j0 = cfg ? item - c0 : item;
            int L0 = cfg ? 3 : 0, L1 = cfg ? 7 : 4, L2 = cfg ? 11 : 8;
            int j2 = m.h->aa[item] + (p - m.h->pre[item]);
            float x0 = m.wx[L0 * cap + j0], z0 = m.wz[L0 * cap + j0];
            float x2 = m.wx[L2 * cap + j2], z2 = m.wz[L2 * cap + j2];
            float tx_d = (x2 - x0) / (z2 - z0);
            bool ok = true;
            if (f1) {
                float d = tx_d - s.txs;
                ok = (bend > 0.0f) ? (d > 0.0f) : (d < 0.0f);
            }
            if (ok) {
                float x_mag_d = x0 + tx_d * (k.z_magnet - z0);
                float tol = tol_base + k.magtol_tx * fabsf(tx_d);
                tol = fminf(fmaxf(tol, k.magtol_min), k.magtol_max);
                ok = fabsf(x_mag_d - x_mag_in) < tol;
            }
            if (ok) {
                float K = cfg ? k.K_last : k.K_first;
                float x1_exp = k.z[L1] * tx_d + (x0 - tx_d * z0) * K;
                int j1 = closest_smem(m.wx + L1 * cap, m.h->wcnt[L1], x1_exp);
                if (j1 >= 0) {
                    float dx = m.wx[L1 * cap + j1] - x1_exp;
                    float chi2 = dx * dx;
                    if (chi2 < k.T_triplet) {
                        valid = true;
                        key = ((uint64_t)__float_as_uint(chi2) << 32) | ((uint64_t)cfg << 18) |
                              ((uint64_t)j0 << 12) | ((uint64_t)j2 << 6) | (uint64_t)j1;
                    }
                }
            }
        }
        if (NT > 0) {
            uint64_t thr = shfl64(top, NT - 1);
            valid = valid && key < thr;
            unsigned msk = __ballot_sync(FULL, valid);
            while (msk) {
                int src = __ffs(msk) - 1;
                msk &= msk - 1;
                uint64_t kk = shfl64(key, src);
                uint64_t last = shfl64(top, NT - 1);
                if (kk < last) {
                    unsigned lt = __ballot_sync(FULL, lane < NT && top < kk);
                    int pos = __popc(lt);
                    uint64_t up = shfl64_up(top, 1);
                    if (lane == pos) top = kk;
                    else if (lane > pos && lane < NT) top = up;
                }
            }
        }
    }
    n_trip = __popc(__ballot_sync(FULL, lane < NT && top != NOKEY));
    return top;
}

// --------------------------------------------------- stage: extension + fit

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

__device__ __noinline__ void extend_fit(const KParams& k, const TState& s, const WarpSmem& m, uint64_t key,
                                        Cand& cd) {
    const int cap = k.cap;
    const float D = k.D;
    const int cfg = (int)((key >> 18) & 1);
    const int j0 = (int)((key >> 12) & 63), j2 = (int)((key >> 6) & 63), j1 = (int)(key & 63);
    const int L0 = cfg ? 3 : 0, L1 = cfg ? 7 : 4, L2 = cfg ? 11 : 8;
    int hl[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) hl[l] = (l == L0) ? j0 : (l == L1) ? j1 : (l == L2) ? j2 : -1;
    cd.Q = 0.0f;
    cd.n = 0;

    // three-point solution through the triplet
    float x0 = m.wx[L0 * cap + j0], x1 = m.wx[L1 * cap + j1], x2 = m.wx[L2 * cap + j2];
    float u0 = (m.wz[L0 * cap + j0] - k.z_ref) * 1e-3f;
    float u1 = (m.wz[L1 * cap + j1] - k.z_ref) * 1e-3f;
    float u2 = (m.wz[L2 * cap + j2] - k.z_ref) * 1e-3f;
    float g0 = f2_of(u0, D), g1 = f2_of(u1, D), g2 = f2_of(u2, D);
    float d1 = u1 - u0, d2 = u2 - u0;
    float e1 = g1 - g0, e2 = g2 - g0;
    float r1 = x1 - x0, r2 = x2 - x0;
    float det = d1 * e2 - d2 * e1;
    if (!(det != 0.0f)) {
        cd.status = 1;
        return;
    }
    float T = (r1 * e2 - r2 * e1) / det;
    float C = (d1 * r2 - d2 * r1) / det;
    float A = (x0 - T * u0) - C * g0;

    // missing x layers
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (!is_x(l) || l == L0 || l == L1 || l == L2) continue;
        float xe = model_x(A, T, C, (k.z[l] - k.z_ref) * 1e-3f, D);
        int j = closest_smem(m.wx + l * cap, m.h->wcnt[l], xe);
        if (j < 0) continue;
        float dx = m.wx[l * cap + j] - xe;
        if (dx * dx < k.T_x) hl[l] = j;
    }

    // weighted refit on the x hits, as a correction to the three-point solution
    float S00 = 0.0f, S01 = 0.0f, S02 = 0.0f, S11 = 0.0f, S12 = 0.0f, S22 = 0.0f, b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (!is_x(l) || hl[l] < 0) continue;
        int q = l * cap + hl[l];
        float u = (m.wz[q] - k.z_ref) * 1e-3f;
        float f = f2_of(u, D);
        float r = m.wx[q] - model_x(A, T, C, u, D);
        float wt = m.ww[q];
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
    if (!(dt != 0.0f)) {
        cd.status = 1;
        return;
    }
    A = A + ((c00 * b0 + c01 * b1) + c02 * b2) / dt;
    T = T + ((c01 * b0 + c11 * b1) + c12 * b2) / dt;
    C = C + ((c02 * b0 + c12 * b1) + c22 * b2) / dt;

    // u/v layers
    float T_uv = k.T_uv_scale * (fabsf(s.txs) + fabsf(s.tys));
    T_uv = fmaxf(k.T_uv_min, T_uv);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (is_x(l)) continue;
        float yl = s.ys + s.tys * (k.z[l] - k.z_state);
        float xe = model_x(A, T, C, (k.z[l] - k.z_ref) * 1e-3f, D) - yl * k.dxdy[l];
        int j = closest_smem(m.wx + l * cap, m.h->wcnt[l], xe);
        if (j < 0) continue;
        float dx = m.wx[l * cap + j] - xe;
        if (dx * dx < T_uv) hl[l] = j;
    }

    int n_x = 0, n_uv = 0;
    bool st_ok = true;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (hl[l] < 0) continue;
        if (is_x(l)) ++n_x; else ++n_uv;
    }
#pragma unroll
    for (int st = 0; st < 3; ++st) st_ok = st_ok && (hl[4 * st + 1] >= 0 || hl[4 * st + 2] >= 0);
    int n = n_x + n_uv;
    cd.n = n;
#pragma unroll
    for (int l = 0; l < NL; ++l) cd.hl[l] = hl[l];
    if (n < k.min_hits) {
        cd.status = 2;
        return;
    }
    if (!st_ok) {
        cd.status = 3;
        return;
    }

    // y line fit from the stereo hits
    float Y0s = 0.0f, Y1s = 0.0f, Y2s = 0.0f, yb0 = 0.0f, yb1 = 0.0f;
    float yv[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        yv[l] = 0.0f;
        if (is_x(l) || hl[l] < 0) continue;
        int q = l * cap + hl[l];
        float u = (m.wz[q] - k.z_ref) * 1e-3f;
        float y = (model_x(A, T, C, u, D) - m.wx[q]) / m.wd[q];
        yv[l] = y;
        float wt = m.ww[q];
        float wu = wt * u;
        Y0s = Y0s + wt; Y1s = Y1s + wu; Y2s = Y2s + wu * u;
        yb0 = yb0 + wt * y; yb1 = yb1 + wu * y;
    }
    float ydet = Y0s * Y2s - Y1s * Y1s;
    if (!(ydet != 0.0f)) {
        cd.status = 1;
        return;
    }
    float Y0 = (Y2s * yb0 - Y1s * yb1) / ydet;
    float TY = (Y0s * yb1 - Y1s * yb0) / ydet;
    float ty_fit = TY * 1e-3f;
    if (!(fabsf(ty_fit - s.tys) < k.T_ty)) {
        cd.status = 4;
        return;
    }

    // quality factor
    float qx = 0.0f, qy = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (hl[l] < 0) continue;
        int q = l * cap + hl[l];
        float u = (m.wz[q] - k.z_ref) * 1e-3f;
        float xf = model_x(A, T, C, u, D);
        if (is_x(l)) {
            float r = m.wx[q] - xf;
            qx = qx + (r * r) / k.T_x;
        } else {
            float yf = Y0 + TY * u;
            float r = m.wx[q] - (xf - yf * m.wd[q]);
            qx = qx + (r * r) / T_uv;
            float ry = yv[l] - yf;
            qy = qy + (ry * ry) / k.T_y;
        }
    }
    float Cn = n == 9 ? k.C_n[0] : n == 10 ? k.C_n[1] : n == 11 ? k.C_n[2] : k.C_n[3];
    float Q = (qx / (float)(n - 3) + qy / (float)(n_uv - 2)) * Cn;
    cd.Q = Q;
    if (!(Q < k.T_Q)) {
        cd.status = 5;
        return;
    }
    cd.status = 0;
    float tx = T * 1e-3f;
    cd.st[0] = A;
    cd.st[1] = Y0;
    cd.st[2] = tx;
    cd.st[3] = ty_fit;
    cd.st[4] = C * 1e-6f;
    cd.st[5] = (tx - s.txs) / k.pk;
}

// ---------------------------------------------------------- stage: selection

// Warp-wide choice of the lowest Q among accepted candidates (ties to the
// lower rank) and coalesced output of the winner.
__device__ __forceinline__ void select_and_write(const KOut& o, int t, int lane, bool have, float Q, int n,
                                                 const int* hl_glob, const float* st) {
    uint64_t key = have ? (((uint64_t)__float_as_uint(Q) << 32) | (unsigned)lane) : NOKEY;
    uint64_t best = warp_min64(key);
    if (best == NOKEY) {
        if (lane == 0) {
            o.found[t] = 0;
            o.nhits[t] = 0;
        }
        return;
    }
    int w = (int)(best & 31u);
    int mine = -1;
    float stv = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        int v = __shfl_sync(FULL, hl_glob[l], w);
        if (lane == l) mine = v;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float v = __shfl_sync(FULL, st[q], w);
        if (lane == NL + q) stv = v;
    }
    float Qw = __shfl_sync(FULL, Q, w);
    int nw = __shfl_sync(FULL, n, w);
    if (lane < NL) o.hit_idx[(size_t)t * NL + lane] = mine;
    else if (lane < NL + 6) o.state[(size_t)t * 6 + (lane - NL)] = stv;
    else if (lane == NL + 6) o.quality[t] = Qw;
    else if (lane == NL + 7) {
        o.found[t] = 1;
        o.nhits[t] = (uint8_t)nw;
    }
}

// ------------------------------------------------------------ event lookup

// event e with trk_offsets[e] <= t < trk_offsets[e+1]
__device__ __forceinline__ int event_of(const int* __restrict__ trk_offsets, int n_events, int t) {
    int lo = 0, hi = n_events + 1;
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (__ldg(trk_offsets + mid) <= t) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

// ================================================================ kernels

__global__ void k_track_event(KBatch b, int* trk_event) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < b.n_events; e += gridDim.x * blockDim.x) {
        int t0 = b.trk_offsets[e], t1 = b.trk_offsets[e + 1];
        for (int t = t0; t < t1; ++t) trk_event[t] = e;
    }
}

// plain form, stage 1: windows (warp per track, lanes 0..11 one layer each)
__global__ void k_windows(KParams k, KBatch b, const int* __restrict__ trk_event, int* wbeg, uint8_t* wcnt) {
    int lane = threadIdx.x & 31;
    int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= b.n_tracks) return;
    if (lane < NL) {
        TState s = load_state(b, t);
        int beg, cnt;
        layer_window(k, b, s, __ldg(trk_event + t), lane, beg, cnt);
        wbeg[(size_t)t * NL + lane] = beg;
        wcnt[(size_t)t * NL + lane] = (uint8_t)cnt;
    }
}

__device__ __forceinline__ void load_windows(const int* wbeg, const uint8_t* wcnt, int t, const WarpSmem& m,
                                             int lane) {
    if (lane < NL) {
        m.h->wbeg[lane] = wbeg[(size_t)t * NL + lane];
        m.h->wcnt[lane] = wcnt[(size_t)t * NL + lane];
    }
    __syncwarp();
}

// plain form, stage 2: triplet seeding
__global__ void k_triplets(KParams k, KBatch b, const int* __restrict__ wbeg, const uint8_t* __restrict__ wcnt,
                           uint64_t* keys, uint8_t* ntrip) {
    extern __shared__ __align__(16) char smem[];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int t = blockIdx.x * (blockDim.x >> 5) + warp;
    if (t >= b.n_tracks) return;
    WarpSmem m = warp_smem(smem, warp, k.cap);
    load_windows(wbeg, wcnt, t, m, lane);
    stage_windows(k, b, m, lane);
    TState s = load_state(b, t);
    int nt;
    uint64_t top = triplet_scan(k, s, m, lane, nt);
    if (lane < nt) keys[(size_t)t * k.n_trip + lane] = top;
    if (lane == 0) ntrip[t] = (uint8_t)nt;
}

// plain form, stage 3: extension and fit of every kept triplet
__global__ void k_extend(KParams k, KBatch b, const int* __restrict__ wbeg, const uint8_t* __restrict__ wcnt,
                         const uint64_t* __restrict__ keys, const uint8_t* __restrict__ ntrip, CandRec* cands) {
    extern __shared__ __align__(16) char smem[];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int t = blockIdx.x * (blockDim.x >> 5) + warp;
    if (t >= b.n_tracks) return;
    int nt = ntrip[t];
    if (nt == 0) return;
    WarpSmem m = warp_smem(smem, warp, k.cap);
    load_windows(wbeg, wcnt, t, m, lane);
    stage_windows(k, b, m, lane);
    if (lane < nt) {
        TState s = load_state(b, t);
        Cand cd;
        extend_fit(k, s, m, keys[(size_t)t * k.n_trip + lane], cd);
        CandRec r;
        r.Q = cd.Q;
        r.status = (int8_t)cd.status;
        r.n = (int8_t)cd.n;
#pragma unroll
        for (int l = 0; l < NL; ++l) r.hl[l] = (int8_t)(cd.status == 0 ? cd.hl[l] : -1);
        for (int q = 0; q < 6; ++q) r.pad[q] = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) r.st[q] = cd.status == 0 ? cd.st[q] : 0.0f;
        cands[(size_t)t * k.n_trip + lane] = r;
    }
}

// plain form, stage 4: warp-vote selection and output
__global__ void k_select(KParams k, KBatch b, const int* __restrict__ wbeg, const uint8_t* __restrict__ ntrip,
                         const CandRec* __restrict__ cands, KOut o) {
    int lane = threadIdx.x & 31;
    int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= b.n_tracks) return;
    int nt = ntrip[t];
    bool have = false;
    float Q = 0.0f;
    int n = 0;
    int hg[NL];
    float st[6];
#pragma unroll
    for (int l = 0; l < NL; ++l) hg[l] = -1;
#pragma unroll
    for (int q = 0; q < 6; ++q) st[q] = 0.0f;
    if (lane < nt) {
        CandRec r = cands[(size_t)t * k.n_trip + lane];
        have = r.status == 0;
        Q = r.Q;
        n = r.n;
#pragma unroll
        for (int l = 0; l < NL; ++l) hg[l] = r.hl[l] >= 0 ? wbeg[(size_t)t * NL + l] + r.hl[l] : -1;
#pragma unroll
        for (int q = 0; q < 6; ++q) st[q] = r.st[q];
    }
    select_and_write(o, t, lane, have, Q, n, hg, st);
}

// One track through every stage, inside the persistent kernel.
__device__ __forceinline__ void follow_track(const KParams& k, const KBatch& b, const KOut& o, int t, int e,
                                             const WarpSmem& m, int lane) {
    TState s = load_state(b, t);
    if (lane < NL) {
        int beg, cnt;
        layer_window(k, b, s, e, lane, beg, cnt);
        m.h->wbeg[lane] = beg;
        m.h->wcnt[lane] = cnt;
    }
    __syncwarp();
    stage_windows(k, b, m, lane);
    int nt;
    uint64_t top = triplet_scan(k, s, m, lane, nt);
    Cand cd;
    cd.status = 9;
    cd.Q = 0.0f;
    cd.n = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) cd.st[q] = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) cd.hl[l] = -1;
    if (lane < nt) extend_fit(k, s, m, top, cd);
    int hg[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) hg[l] = (lane < nt && cd.status == 0 && cd.hl[l] >= 0) ? m.h->wbeg[l] + cd.hl[l] : -1;
    select_and_write(o, t, lane, lane < nt && cd.status == 0, cd.Q, cd.n, hg, cd.st);
    __syncwarp();
}

// persistent form: warps take grains of consecutive input tracks from a
// device work queue until it is empty
__global__ void k_fused(KParams k, KBatch b, KOut o, int* cursor, int grain) {
    extern __shared__ __align__(16) char smem[];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem m = warp_smem(smem, warp, k.cap);
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(cursor, grain);
        base = __shfl_sync(FULL, base, 0);
        if (base >= b.n_tracks) break;
        int end = min(base + grain, b.n_tracks);
        int e = event_of(b.trk_offsets, b.n_events, base);
        for (int t = base; t < end; ++t) {
            while (t >= __ldg(b.trk_offsets + e + 1)) ++e;
            follow_track(k, b, o, t, e, m, lane);
        }
    }
}

// debug dump of the plain form's triplet stage in packed hit indices
__global__ void k_debug_triplets(KParams k, KBatch b, const int* __restrict__ wbeg, const uint8_t* __restrict__ wcnt,
                                 const uint64_t* __restrict__ keys, const uint8_t* __restrict__ ntrip,
                                 int* win_count_out, int* n_trip_out, int* trip_out, float* chi2_out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.n_tracks) return;
    for (int l = 0; l < NL; ++l) win_count_out[(size_t)t * NL + l] = wcnt[(size_t)t * NL + l];
    int nt = ntrip[t];
    n_trip_out[t] = nt;
    for (int r = 0; r < nt; ++r) {
        uint64_t key = keys[(size_t)t * k.n_trip + r];
        int cfg = (int)((key >> 18) & 1);
        int j0 = (int)((key >> 12) & 63), j2 = (int)((key >> 6) & 63), j1 = (int)(key & 63);
        int L0 = cfg ? 3 : 0, L1 = cfg ? 7 : 4, L2 = cfg ? 11 : 8;
        int* q = trip_out + ((size_t)t * k.n_trip + r) * 4;
        q[0] = cfg;
        q[1] = wbeg[(size_t)t * NL + L0] + j0;
        q[2] = wbeg[(size_t)t * NL + L1] + j1;
        q[3] = wbeg[(size_t)t * NL + L2] + j2;
        chi2_out[(size_t)t * k.n_trip + r] = __uint_as_float((unsigned)(key >> 32));
    }
}

// packed hit indices -> raw hit indices (+ base), for results leaving the device
__global__ void k_hits_to_raw(const uint8_t* __restrict__ found, int* hit_idx, const int* __restrict__ perm,
                              int n_tracks, int base) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tracks * NL) return;
    if (!found[i / NL]) return;
    int h = hit_idx[i];
    hit_idx[i] = h >= 0 ? __ldg(perm + h) + base : -1;
}

// ------------------------------------------------------------- compaction

// per-event count of found tracks (warp per event)
__global__ void k_compact_count(const int* __restrict__ trk_offsets, const uint8_t* __restrict__ found, int n_events,
                                int* ev_count) {
    int lane = threadIdx.x & 31;
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= n_events) return;
    int t0 = trk_offsets[e], t1 = trk_offsets[e + 1];
    int c = 0;
    for (int t = t0 + lane; t < t1; t += 32) c += found[t] ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane == 0) ev_count[e] = c;
}

// exclusive scan of the per-event counts by one block
__global__ void k_compact_scan(const int* __restrict__ ev_count, int n_events, int* out_offsets, int* n_out) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n_events; base += blockDim.x) {
        int i = base + tid;
        int v = i < n_events ? ev_count[i] : 0;
        int inc = warp_incl_scan(v, lane);
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int wv = lane < nw ? warp_tot[lane] : 0;
            int wi = warp_incl_scan(wv, lane);
            if (lane < nw) warp_tot[lane] = wi - wv;
        }
        __syncthreads();
        int excl = carry + warp_tot[warp] + inc - v;
        if (i < n_events) out_offsets[i] = excl;
        __syncthreads();
        if (tid == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (tid == 0) {
        out_offsets[n_events] = carry;
        *n_out = carry;
    }
}

// scatter of found track indices (warp per event, ballot positions)
__global__ void k_compact_scatter(const int* __restrict__ trk_offsets, const uint8_t* __restrict__ found, int n_events,
                                  const int* __restrict__ out_offsets, int* out_trk) {
    int lane = threadIdx.x & 31;
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= n_events) return;
    int t0 = trk_offsets[e], t1 = trk_offsets[e + 1];
    int pos = out_offsets[e];
    for (int base = t0; base < t1; base += 32) {
        int t = base + lane;
        bool f = t < t1 && found[t];
        unsigned msk = __ballot_sync(FULL, f);
        if (f) out_trk[pos + __popc(msk & ((1u << lane) - 1u))] = t;
        pos += __popc(msk);
    }
}

// ================================================================ launchers

static inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }
constexpr int PLAIN_WARPS = 8;

cudaError_t launch_track_event(const KBatch& b, int* trk_event, cudaStream_t s) {
    if (b.n_events <= 0) return cudaSuccess;
    k_track_event<<<cdiv(b.n_events, 256), 256, 0, s>>>(b, trk_event);
    return cudaGetLastError();
}

cudaError_t launch_windows(const KParams& k, const KBatch& b, const int* trk_event, int* wbeg, uint8_t* wcnt,
                           cudaStream_t s) {
    if (b.n_tracks <= 0) return cudaSuccess;
    k_windows<<<cdiv((long)b.n_tracks * 32, 256), 256, 0, s>>>(k, b, trk_event, wbeg, wcnt);
    return cudaGetLastError();
}

static cudaError_t set_smem(const void* fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_triplets(const KParams& k, const KBatch& b, const int* trk_event, const int* wbeg,
                            const uint8_t* wcnt, uint64_t* keys, uint8_t* ntrip, cudaStream_t s) {
    (void)trk_event;
    if (b.n_tracks <= 0) return cudaSuccess;
    size_t sm = warp_smem_bytes(k.cap) * PLAIN_WARPS;
    cudaError_t err = set_smem((const void*)k_triplets, sm);
    if (err != cudaSuccess) return err;
    k_triplets<<<cdiv(b.n_tracks, PLAIN_WARPS), PLAIN_WARPS * 32, sm, s>>>(k, b, wbeg, wcnt, keys, ntrip);
    return cudaGetLastError();
}

cudaError_t launch_extend(const KParams& k, const KBatch& b, const int* trk_event, const int* wbeg,
                          const uint8_t* wcnt, const uint64_t* keys, const uint8_t* ntrip, CandRec* cands,
                          cudaStream_t s) {
    (void)trk_event;
    if (b.n_tracks <= 0) return cudaSuccess;
    size_t sm = warp_smem_bytes(k.cap) * PLAIN_WARPS;
    cudaError_t err = set_smem((const void*)k_extend, sm);
    if (err != cudaSuccess) return err;
    k_extend<<<cdiv(b.n_tracks, PLAIN_WARPS), PLAIN_WARPS * 32, sm, s>>>(k, b, wbeg, wcnt, keys, ntrip, cands);
    return cudaGetLastError();
}

cudaError_t launch_select(const KParams& k, const KBatch& b, const int* wbeg, const uint8_t* ntrip,
                          const CandRec* cands, const KOut& o, cudaStream_t s) {
    if (b.n_tracks <= 0) return cudaSuccess;
    k_select<<<cdiv((long)b.n_tracks * 32, 256), 256, 0, s>>>(k, b, wbeg, ntrip, cands, o);
    return cudaGetLastError();
}

cudaError_t fused_max_blocks_per_sm(const KParams& k, int warps_per_block, int* out) {
    size_t sm = warp_smem_bytes(k.cap) * warps_per_block;
    cudaError_t err = set_smem((const void*)k_fused, sm);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_fused, warps_per_block * 32, sm);
}

cudaError_t launch_fused(const KParams& k, const KBatch& b, const KOut& o, int* cursor, int grain,
                         int warps_per_block, int n_blocks, cudaStream_t s) {
    size_t sm = warp_smem_bytes(k.cap) * warps_per_block;
    cudaError_t err = set_smem((const void*)k_fused, sm);
    if (err != cudaSuccess) return err;
    k_fused<<<n_blocks, warps_per_block * 32, sm, s>>>(k, b, o, cursor, grain);
    return cudaGetLastError();
}

cudaError_t launch_hits_to_raw(const uint8_t* found, int* hit_idx, const int* perm, int n_tracks, int base,
                              cudaStream_t s) {
    if (n_tracks <= 0) return cudaSuccess;
    k_hits_to_raw<<<cdiv((long)n_tracks * NL, 256), 256, 0, s>>>(found, hit_idx, perm, n_tracks, base);
    return cudaGetLastError();
}

cudaError_t launch_compact(const int* trk_offsets, const uint8_t* found, int n_events, int* ev_count,
                           int* out_offsets, int* out_trk, int* n_out, cudaStream_t s) {
    if (n_events > 0) {
        k_compact_count<<<cdiv((long)n_events * 32, 256), 256, 0, s>>>(trk_offsets, found, n_events, ev_count);
    }
    k_compact_scan<<<1, 1024, 0, s>>>(ev_count, n_events, out_offsets, n_out);
    if (n_events > 0) {
        k_compact_scatter<<<cdiv((long)n_events * 32, 256), 256, 0, s>>>(trk_offsets, found, n_events, out_offsets,
                                                                         out_trk);
    }
    return cudaGetLastError();
}

cudaError_t launch_debug_triplets(const KParams& k, const KBatch& b, const int* wbeg, const uint8_t* wcnt,
                                  const uint64_t* keys, const uint8_t* ntrip, int* win_count_out, int* n_trip_out,
                                  int* trip_out, float* chi2_out, cudaStream_t s) {
    if (b.n_tracks <= 0) return cudaSuccess;
    k_debug_triplets<<<cdiv(b.n_tracks, 128), 128, 0, s>>>(k, b, wbeg, wcnt, keys, ntrip, win_count_out, n_trip_out,
                                                           trip_out, chi2_out);
    return cudaGetLastError();
}

}  // namespace lfk
