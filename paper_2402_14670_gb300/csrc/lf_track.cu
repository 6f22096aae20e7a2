// Forward-tracking kernels for sm_103a.
//
// A warp follows an input track.  The stages are device functions shared by
// the plain form (one kernel per stage, results in scratch) and the
// persistent form (k_tile: blocks take tiles of consecutive input tracks from
// a device work queue and run the stages on them with results in shared
// memory and registers; the warps of a block step through the stages
// together, and the extension runs two tracks per warp).
//
//   windows    Sec. "Defining the search windows": lanes 0..11 each open one
//              layer's window with binary searches in the x-sorted bucket
//              (lanes 12..23 the upper bounds, in the same loop); the
//              persistent kernel runs two tracks per warp with their
//              searches interleaved, so twice the loads are in flight.
//   staging    x and z of the window hits (<= n_hits_window per layer) are
//              copied into the track's shared-memory slot, once per track;
//              dxdy and w are read from L2 for the hits a candidate uses.
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
//              the x of all twelve windows is staged (z, dxdy and w of the hits
//              a candidate uses are read from global memory);
//              lane r of a 16- or 32-lane group extends triplet r
//              (three-point solution, missing x layers, weighted x refit,
//              u/v layers, y line fit, Q).
//   selection  lowest Q among accepted candidates by a warp-wide minimum of
//              (Q bits, rank); the winner's hits and state go out coalesced.
//
// No-UT variant (Sec. "No-UT tuning", NOUT = true): an input track has two
// window sets, one per charge assumption, built around its straight-line
// extrapolation with the Eq. tol_noUT tolerance; the triplet stage stages and
// scans the two sets in turn into one kept-triplet list (the side is a key
// bit), and the extension stages each set in turn for the triplets seeded in
// it.
//
// Arithmetic: binary32, no contraction (built with -fmad=false), IEEE
// division; every expression is written in the evaluation order of the
// method's definition so that results do not depend on the launch shape.
#include <climits>
#include <cstdint>

#include <cuda_fp16.h>

#include "lf_device.cuh"
#include "lf_internal.h"

namespace lfk {


// first index in [lo, hi) whose x is not left of v: left means x < v (lower
// bound, upper = false) or !(x > v) (upper bound, upper = true); one loop for
// both, so lanes searching lower and upper bounds do not diverge
__device__ __forceinline__ int bound_global(const float* __restrict__ x, int lo, int hi, float v, bool upper) {
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        const float xm = __ldg(x + mid);
        if (upper ? !(xm > v) : (xm < v)) lo = mid + 1; else hi = mid;
    }
    return lo;
}
// two independent bound searches in lockstep (more loads in flight per lane)
__device__ __forceinline__ void bound2_global(const float* __restrict__ x, int& lo0, int hi0, float v0, int& lo1,
                                              int hi1, float v1, bool upper) {
    while (lo0 < hi0 || lo1 < hi1) {
        const bool a0 = lo0 < hi0, a1 = lo1 < hi1;
        const int m0 = lo0 + ((hi0 - lo0) >> 1), m1 = lo1 + ((hi1 - lo1) >> 1);
        const float x0 = a0 ? __ldg(x + m0) : 0.0f;
        const float x1 = a1 ? __ldg(x + m1) : 0.0f;
        if (a0) {
            if (upper ? !(x0 > v0) : (x0 < v0)) lo0 = m0 + 1; else hi0 = m0;
        }
        if (a1) {
            if (upper ? !(x1 > v1) : (x1 < v1)) lo1 = m1 + 1; else hi1 = m1;
        }
    }
}
// The same two searches through the coarse index c (c[i] = x[32 i]): first
// over the coarse entries inside each range (a few neighbouring words, so
// after the first load mostly L1 hits), which leaves at most 32 candidates,
// then over those (one or two cache lines).  Same results as bound2_global:
// the first coarse entry not left of v brackets the answer from above and
// the entry before it from below.
__device__ __forceinline__ void bound2_coarse(const float* __restrict__ x, const float* __restrict__ c, int& lo0,
                                              int hi0, float v0, int& lo1, int hi1, float v1, bool upper) {
    // coarse entries with lo <= 32 i < hi
    int a0 = (lo0 + 31) >> 5, b0 = (hi0 + 31) >> 5, a1 = (lo1 + 31) >> 5, b1 = (hi1 + 31) >> 5;
    const int s0 = a0, s1 = a1;
    if (lo0 >= hi0) b0 = a0;
    if (lo1 >= hi1) b1 = a1;
    bound2_global(c, a0, b0, v0, a1, b1, v1, upper);
    // a = first coarse index (in range) not left of v: the answer is in
    // (32 (a - 1), 32 a] within [lo, hi)
    int h0 = hi0, h1 = hi1;
    if (a0 > s0) lo0 = 32 * (a0 - 1) + 1;
    if (32 * a0 < hi0 && a0 < ((hi0 + 31) >> 5)) h0 = 32 * a0;
    if (a1 > s1) lo1 = 32 * (a1 - 1) + 1;
    if (32 * a1 < hi1 && a1 < ((hi1 + 31) >> 5)) h1 = 32 * a1;
    bound2_global(x, lo0, h0, v0, lo1, h1, v1, upper);
}
// one search through the coarse index
__device__ __forceinline__ int bound_coarse(const float* __restrict__ x, const float* __restrict__ c, int lo, int hi,
                                            float v, bool upper) {
    int lo1 = 0;
    bound2_coarse(x, c, lo, hi, v, lo1, 0, 0.0f, upper);
    return lo;
}
// first index in [0, n) of a window in shared memory with x >= v
__device__ __forceinline__ int lb_smem(const float* x, int n, float v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (x[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
// first index in [0, n) with x > v
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


// the same search, out of line, on a window given by its shared-memory address
__device__ __noinline__ int closest_shared(unsigned xs, int n, float e) {
    auto at = [&](int i) -> float {
        float v;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(xs + 4u * (unsigned)i));
        return v;
    };
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (at(mid) < e) lo = mid + 1; else hi = mid;
    }
    const int j = lo;
    int best = -1;
    float bd = 0.0f;
    if (j > 0) {
        int q = j - 1;
        float d = fabsf(at(q) - e);
        while (q > 0 && fabsf(at(q - 1) - e) == d) --q;
        best = q;
        bd = d;
    }
    if (j < n) {
        float d = fabsf(at(j) - e);
        if (best < 0 || d < bd) best = j;
    }
    return best;
}


// Windows of all twelve layers, [begin, begin+count) in packed hit indices,
// returned on lanes 0..11: lanes 0..11 search the lower bounds and lanes
// 12..23 the upper bounds in parallel, then lanes 0..11 apply the cap.
template <bool NOUT>
__device__ __forceinline__ void warp_windows(const KParams& k, const KBatch& b, const TState& s, int e, int lane,
                                             int side, int& begin, int& count) {
    const int zone = (s.tys >= 0.0f) ? 1 : 0;
    const int l = lane < NL ? lane : (lane < 2 * NL ? lane - NL : 0);
    float xmin, xmax, centre;
    window_limits<NOUT>(k, s, l, side, xmin, xmax, centre);
    const int* off = b.hit_offsets + (size_t)e * NB + zone * NL + l;
    const int bb = __ldg(off), be = __ldg(off + 1);
    int v = 0;
    if (lane < 2 * NL)
        v = b.x_coarse ? bound_coarse(b.x, b.x_coarse, bb, be, lane < NL ? xmin : xmax, lane >= NL)
                       : bound_global(b.x, bb, be, lane < NL ? xmin : xmax, lane >= NL);
    int hi = __shfl_sync(FULL, v, (lane + NL) & 31);
    begin = 0;
    count = 0;
    if (lane < NL) {
        const int lo = v;
        if (hi < lo) hi = lo;
        int cnt = hi - lo, start = lo;
        if (cnt > k.cap) {
            int c = b.x_coarse ? bound_coarse(b.x, b.x_coarse, lo, hi, centre, false)
                               : bound_global(b.x, lo, hi, centre, false);
            start = c - k.cap / 2;
            if (start > hi - k.cap) start = hi - k.cap;
            if (start < lo) start = lo;
            cnt = k.cap;
        }
        begin = start;
        count = cnt;
    }
}


// ------------------------------------------------------- shared-memory slots

struct Slot {
    SlotHead* h;
    float* wx;
    float* wz;
};

struct Scratch {
    unsigned long long* cand;
    unsigned short* pairs;
    // half-precision pre-filter: per configuration the h1 window's x
    // relative to its first hit as binary16 pairs (MAX_CAP / 2 words each),
    // then per configuration {reference x, 1/(z2 - z0), z0, applies}
    __half2* hw;
    float* pf;
};

__device__ __forceinline__ Slot slot_at(char* base, int i, int cap) {
    char* p = base + (size_t)i * slot_bytes(cap);
    Slot s;
    s.h = reinterpret_cast<SlotHead*>(p);
    s.wx = reinterpret_cast<float*>(p + align16(sizeof(SlotHead)));
    s.wz = s.wx + NL * cap;
    return s;
}

__device__ __forceinline__ Scratch scratch_at(char* base, int i, bool hp = false) {
    char* p = base + (size_t)i * scratch_bytes(hp);
    Scratch s;
    s.cand = reinterpret_cast<unsigned long long*>(p);
    s.pairs = reinterpret_cast<unsigned short*>(p + CAND_CAP * sizeof(unsigned long long));
    s.hw = reinterpret_cast<__half2*>(p + scratch_bytes(false));
    s.pf = reinterpret_cast<float*>(s.hw + MAX_CAP);
    return s;
}

// Asynchronous 4-byte copy global -> shared (cp.async, cached in L1); the
// copying lane waits for its copies with cp_async_wait_all.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copy x and z of the window hits into the slot, one asynchronous copy per
// hit and array: layer by layer, lane j copying hit j (and j + 32), so the
// copies of all of a track's windows are in flight at once (stage_issue);
// stage_finish waits for them and flags a window whose hits do not all
// share one z.
template <bool XONLY = false, bool ZTOO = true>
__device__ __forceinline__ void stage_issue(const KParams& k, const KBatch& b, const Slot& m, int lane) {
    const int cap = k.cap;
#pragma unroll 1
    for (int l = 0; l < NL; ++l) {
        if (XONLY && !is_x(l)) continue;
        const int n = m.h->wcnt[l], src = m.h->wbeg[l];
        for (int j = lane; j < n; j += 32) {
            cp_async4(m.wx + l * cap + j, b.x + src + j);
            if (ZTOO) cp_async4(m.wz + l * cap + j, b.z + src + j);
        }
    }
}

// z-uniformity flag of window l of a staged slot (lane-private loop)
template <bool XONLY = false>
__device__ __forceinline__ void window_zuni(const KParams& k, const Slot& m, int l) {
    int u = 1;
    if (!(XONLY && !is_x(l))) {
        const float* wz = m.wz + l * k.cap;
        const int n = m.h->wcnt[l];
        for (int j = 1; j < n; ++j) u &= (wz[j] == wz[0]) ? 1 : 0;
    }
    m.h->zuni[l] = u;
}

// Wait for the staging copies of the warp's TPW slots (lanes 16q.. of slot q)
// and set their z-uniformity flags.
template <int TPW, bool XONLY = false, bool ZTOO = true>
__device__ __forceinline__ void stage_finish(const KParams& k, const Slot* sl, int lane) {
    cp_async_wait_all();
    __syncwarp();
    if (ZTOO) {
        const int q = lane >> 4, l = lane & 15;
        if (q < TPW && l < NL) window_zuni<XONLY>(k, (TPW == 2 && q == 1) ? sl[TPW - 1] : sl[0], l);
        __syncwarp();
    }
}

template <bool XONLY = false>
__device__ __forceinline__ void stage_windows(const KParams& k, const KBatch& b, const Slot& m, int lane) {
    stage_issue<XONLY>(k, b, m, lane);
    stage_finish<1, XONLY>(k, &m, lane);
}


// Sort the buffered keys; keep the NT smallest at the front of the buffer.
// Returns the new buffer size; thr becomes the NT-th smallest key once the
// buffer holds NT keys (no later key at or above it can be kept).
__device__ __forceinline__ int select_buffer(const Scratch& sc, int nb, int NT, uint64_t& thr, int lane,
                                             uint64_t& mine) {
    uint64_t a = lane < nb ? sc.cand[lane] : NOKEY;
    __syncwarp();
    if (nb <= 32) {
        a = warp_sort32(a, lane);
    } else {
        uint64_t b = lane + 32 < nb ? sc.cand[lane + 32] : NOKEY;
        __syncwarp();
        warp_sort64(a, b, lane);
    }
    int keep = nb < NT ? nb : NT;
    if (lane < keep) sc.cand[lane] = a;
    mine = lane < keep ? a : NOKEY;
    if (keep == NT) thr = shfl64(a, NT - 1);
    __syncwarp();
    return keep;
}

// ---------------------------------------------------------- stage: triplets

// One window set's triplets, merged into the warp's key buffer (nb keys,
// threshold thr, this lane's kept key `mine`; see select_buffer).
// key = chi2 bits << 32 | side << 19 | cfg << 18 | j0 << 12 | j2 << 6 | j1
// (window-local indices), which orders by (chi2, side, cfg, h0, h2).
// Half-precision pre-filter, set-up for one track: the h1 windows of both
// configurations as binary16 pairs relative to their first hit (padded with
// +inf) and each configuration's constants.  The pre-filter applies to a
// configuration only if its h1 window spans at most PF_SPAN and its h0 and
// h2 windows each share one z (the exact path then divides by the same
// z2 - z0 for every pair of the configuration).
__device__ __forceinline__ void prefilter_setup(const KParams& k, const Slot& m, const Scratch& sc, int lane) {
    const int cap = k.cap, hc = (cap + 1) >> 1;
    const __half inf = __ushort_as_half((unsigned short)0x7c00u);
    for (int wd = lane; wd < 2 * hc; wd += 32) {
        const int cfg = wd >= hc ? 1 : 0, i = wd - cfg * hc;
        const int L1 = cfg ? 7 : 4, n1 = m.h->wcnt[L1];
        const float* x1 = m.wx + L1 * cap;
        __half a = inf, b = inf;
        if (2 * i < n1) a = __float2half_rn(x1[2 * i] - x1[0]);
        if (2 * i + 1 < n1) b = __float2half_rn(x1[2 * i + 1] - x1[0]);
        sc.hw[cfg * (MAX_CAP / 2) + i] = __halves2half2(a, b);
    }
    if (lane < 2) {
        const int cfg = lane;
        const int L0 = cfg ? 3 : 0, L1 = cfg ? 7 : 4, L2 = cfg ? 11 : 8;
        const int n0 = m.h->wcnt[L0], n1 = m.h->wcnt[L1], n2 = m.h->wcnt[L2];
        float xr = 0.0f, rdz = 0.0f, z0 = 0.0f, ok = 0.0f;
        if (n0 > 0 && n1 > 0 && n2 > 0 && m.h->zuni[L0] && m.h->zuni[L2]) {
            const float* x1 = m.wx + L1 * cap;
            z0 = m.wz[L0 * cap];
            const float dz = m.wz[L2 * cap] - z0;
            xr = x1[0];
            // x1_expected of a pair the exact path accepts then lies within
            // PF_SPAN + pf_bound < 2048 of xr, where the binary16 ulp is <= 1
            if (dz > 0.0f && x1[n1 - 1] - xr <= PF_SPAN && k.pf_bound < 2048.0f - PF_SPAN) {
                rdz = 1.0f / dz;
                ok = 1.0f;
            }
        }
        sc.pf[4 * cfg + 0] = xr;
        sc.pf[4 * cfg + 1] = rdz;
        sc.pf[4 * cfg + 2] = z0;
        sc.pf[4 * cfg + 3] = ok;
    }
    __syncwarp();
}

// Half-precision pre-filter of np materialised pairs (Sec. "Performance",
// the triplet seeding's chi2 in half2): a pair is kept if some hit of its h1
// window lies within pf_bound of x1_expected computed with the slope as a
// product by 1/(z2 - z0), the distances taken in binary16 two hits at a time.
// A pair the exact path accepts has a hit within sqrt(T_triplet) of the
// exact x1_expected, so within pf_bound in binary16 (PF_MARGIN covers the
// roundings): the exact results are those without the pre-filter.  The kept
// pairs are compacted in place (a kept pair never moves to a later index);
// returns their number.
__device__ __forceinline__ int prefilter_pairs(const KParams& k, const Slot& m, const Scratch& sc, int np,
                                               int lane) {
    const int cap = k.cap, hc = (cap + 1) >> 1;
    const __half2 inf2 = __half2half2(__ushort_as_half((unsigned short)0x7c00u));
    int ns = 0;
#pragma unroll 1
    for (int base = 0; base < np; base += 32) {
        const int q = base + lane;
        bool keep = false;
        unsigned code = 0;
        if (q < np) {
            code = sc.pairs[q];
            const int cfg = (int)(code >> 12), j0 = (int)((code >> 6) & 63), j2 = (int)(code & 63);
            keep = true;
            if (sc.pf[4 * cfg + 3] != 0.0f) {
                const int L0 = cfg ? 3 : 0, L2 = cfg ? 11 : 8;
                const float x0 = m.wx[L0 * cap + j0], x2 = m.wx[L2 * cap + j2];
                const float t = (x2 - x0) * sc.pf[4 * cfg + 1];
                const float K = cfg ? k.K_last : k.K_first;
                const float z1 = cfg ? k.z[7] : k.z[4];
                const float e = z1 * t + (x0 - t * sc.pf[4 * cfg + 2]) * K;
                const __half2 e2 = __half2half2(__float2half_rn(e - sc.pf[4 * cfg + 0]));
                const __half2* w = sc.hw + cfg * (MAX_CAP / 2);
                __half2 mn = inf2;
                for (int i = 0; i < hc; ++i) mn = __hmin2(mn, __habs2(__hsub2(w[i], e2)));
                keep = fminf(__low2float(mn), __high2float(mn)) < k.pf_bound;
            }
        }
        const unsigned msk = __ballot_sync(FULL, keep);
        __syncwarp();
        if (keep) sc.pairs[ns + __popc(msk & ((1u << lane) - 1u))] = (unsigned short)code;
        ns += __popc(msk);
    }
    __syncwarp();
    return ns;
}

template <int NIT, bool NOUT, bool HP = false>
__device__ __forceinline__ void triplet_pass(const KParams& k, const TState& s, const Slot& m, const Scratch& sc,
                                             int lane, int side, int& nb, uint64_t& thr, uint64_t& mine) {
    const int cap = k.cap;
    const int NT = k.n_trip;
    float pmom, bend;  // momentum, and the sign of the expected slope change
    if (NOUT) {
        pmom = 1.0f / no_ut_inv_p(k, s);
        bend = side ? 1.0f : -1.0f;  // side 1 holds the tracks bending to larger x
    } else {
        pmom = 1.0f / fabsf(s.qop);
        bend = (s.qop > 0.0f) ? k.pol_f : -k.pol_f;
    }
    const float x_mag_in = s.xs + s.txs * (k.z_magnet - k.z_state);
    const float tol_base = k.magtol_min + k.magtol_c / pmom;
    const bool f1 = pmom < k.p_bend;
    const int c0 = m.h->wcnt[0], c1 = m.h->wcnt[3];
    const int n_items = c0 + c1;

    // h2 interval of each (cfg, h0) item: items lane + 32*part (NIT*32 >= 2*cap)
    int n_it[NIT], a_it[NIT], code_it[NIT];
#pragma unroll
    for (int part = 0; part < NIT; ++part) {
        int i = lane + 32 * part;
        int n = 0, a = 0, code = 0;
        if (i < n_items) {
            int cfg = i < c0 ? 0 : 1;
            int j0 = cfg ? i - c0 : i;
            int L0 = cfg ? 3 : 0, L2 = cfg ? 11 : 8;
            code = (cfg << 12) | (j0 << 6);
            float x0 = m.wx[L0 * cap + j0], z0 = m.wz[L0 * cap + j0];
            int n2 = m.h->wcnt[L2];
            n = n2;
            if (n2 > 0 && m.h->zuni[L2]) {
                float dzl = m.wz[L2 * cap] - z0;
                if (dzl > 0.0f && z0 > k.z_magnet) {
                    // x2 with |x0 + (x2 - x0) r - x_mag_in| < tol form an interval
                    // (r < 0); bound it first with the largest tolerance, then
                    // with the largest tolerance the slopes inside allow, and
                    // below p_bend with the bending sign; widen by a slack far
                    // above the rounding of the exact tests applied later
                    // (bounds only: approximate division, far inside the slack)
                    float ir = __fdividef(dzl, k.z_magnet - z0);     // 1/r
                    float slack = 0.5f + 1e-4f * (fabsf(x0) + fabsf(x_mag_in));
                    float lo = x0 + (x_mag_in - x0 + k.magtol_max) * ir - slack;
                    float hi = x0 + (x_mag_in - x0 - k.magtol_max) * ir + slack;
                    float txm = __fdividef(fmaxf(fabsf(lo - x0), fabsf(hi - x0)), dzl);
                    float t2 = fminf(fmaxf(tol_base + k.magtol_tx * txm, k.magtol_min), k.magtol_max);
                    lo = x0 + (x_mag_in - x0 + t2) * ir - slack;
                    hi = x0 + (x_mag_in - x0 - t2) * ir + slack;
                    if (f1) {
                        float xb = x0 + s.txs * dzl;
                        if (bend > 0.0f) lo = fmaxf(lo, xb - slack); else hi = fminf(hi, xb + slack);
                    }
                    const float* x2w = m.wx + L2 * cap;
                    a = lb_smem(x2w, n2, lo);
                    int bnd = ub_smem(x2w, n2, hi);
                    n = bnd > a ? bnd - a : 0;
                }
            }
        }
        n_it[part] = n;
        a_it[part] = a;
        code_it[part] = code;
    }
    int pre_it[NIT];
    int P = 0;
#pragma unroll
    for (int part = 0; part < NIT; ++part) {
        int inc = warp_incl_scan(n_it[part], lane);
        pre_it[part] = P + inc - n_it[part];
        P += __shfl_sync(FULL, inc, 31);
    }
    if (HP && P > 0) prefilter_setup(k, m, sc, lane);

#pragma unroll 1
    for (int seg = 0; seg < P; seg += PAIR_CAP) {
        // materialise the pairs of this segment
#pragma unroll
        for (int part = 0; part < NIT; ++part) {
            int q0 = max(pre_it[part], seg), q1 = min(pre_it[part] + n_it[part], seg + PAIR_CAP);
            for (int q = q0; q < q1; ++q)
                sc.pairs[q - seg] = (unsigned short)(code_it[part] | (a_it[part] + (q - pre_it[part])));
        }
        __syncwarp();
        int np = min(P - seg, PAIR_CAP);
        if (HP) np = prefilter_pairs(k, m, sc, np, lane);
#pragma unroll 1
        for (int base = 0; base < np; base += 32) {
            int q = base + lane;
            bool valid = false;
            uint64_t key = NOKEY;
            if (q < np) {
                unsigned code = sc.pairs[q];
                int cfg = (int)(code >> 12), j0 = (int)((code >> 6) & 63), j2 = (int)(code & 63);
                int L0 = cfg ? 3 : 0, L1 = cfg ? 7 : 4, L2 = cfg ? 11 : 8;
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
                            key = ((uint64_t)__float_as_uint(chi2) << 32) | ((uint64_t)side << 19) |
                                  ((uint64_t)cfg << 18) | ((uint64_t)j0 << 12) | ((uint64_t)j2 << 6) |
                                  (uint64_t)j1;
                            valid = key < thr;
                        }
                    }
                }
            }
            unsigned msk = __ballot_sync(FULL, valid);
            if (msk) {
                if (nb + __popc(msk) > CAND_CAP) {
                    nb = select_buffer(sc, nb, NT, thr, lane, mine);
                    valid = valid && key < thr;
                    msk = __ballot_sync(FULL, valid);
                }
                if (valid) sc.cand[nb + __popc(msk & ((1u << lane) - 1u))] = key;
                nb += __popc(msk);
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

// Triplet stage of one window set: returns this lane's entry of the sorted
// list of kept triplet keys (lane r holds rank r; NOKEY past the end) and
// the list length.
template <int NIT, bool HP = false>
__device__ __forceinline__ uint64_t triplet_scan(const KParams& k, const TState& s, const Slot& m, const Scratch& sc,
                                                 int lane, int& n_trip) {
    n_trip = 0;
    if (k.n_trip <= 0) return NOKEY;
    int nb = 0;            // keys in the buffer
    uint64_t thr = NOKEY;  // keys at or above thr cannot be kept
    uint64_t mine = NOKEY;
    triplet_pass<NIT, false, HP>(k, s, m, sc, lane, 0, nb, thr, mine);
    nb = select_buffer(sc, nb, k.n_trip, thr, lane, mine);
    n_trip = nb;
    return mine;
}

// --------------------------------------------------- stage: extension + fit


// A float of a shared-memory array read through an explicit 32-bit shared
// address.  The extension reads its staged window x this way: with the
// quality-factor loop rolled, the plain-form kernel's generic-pointer load
// of m.wx[l * cap + j] was measured to return the element of a neighbouring
// layer's window (same j), although the index and the hit's other data were
// right, while this form of the same rolled loop gave exact results.
__device__ __forceinline__ float lds_f(const float* base, int i) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"((unsigned)__cvta_generic_to_shared(base) + 4u * (unsigned)i));
    return v;
}

// Extension and fit of one triplet (Sec. "Extending triplets to other
// layers", "Quality Filter"); x and z of the window hits come from the
// slot, dxdy and w of the hits used from global memory.
template <bool ZG = false>
__device__ __forceinline__ void extend_fit(const KParams& k, const KBatch& b, const TState& s, const Slot& m,
                                           uint64_t key, Cand& cd) {
    // z of window hit j of layer l: staged, or read from global memory
    auto zat = [&](int l, int j) -> float {
        return ZG ? __ldg(b.z + m.h->wbeg[l] + j) : lds_f(m.wz, l * k.cap + j);
    };
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
    float x0 = lds_f(m.wx, L0 * cap + j0), x1 = lds_f(m.wx, L1 * cap + j1), x2 = lds_f(m.wx, L2 * cap + j2);
    float u0 = (zat(L0, j0) - k.z_ref) * 1e-3f;
    float u1 = (zat(L1, j1) - k.z_ref) * 1e-3f;
    float u2 = (zat(L2, j2) - k.z_ref) * 1e-3f;
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

    // missing x layers: 3, 7, 11 after configuration 0; 0, 4, 8 after configuration 1
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int l = 4 * i + (cfg ? 0 : 3);
        const float zl = cfg ? k.z[4 * i] : k.z[4 * i + 3];
        float xe = model_x(A, T, C, (zl - k.z_ref) * 1e-3f, D);
        int j = closest_shared((unsigned)__cvta_generic_to_shared(m.wx + l * cap), m.h->wcnt[l], xe);
        int jm = -1;
        if (j >= 0) {
            float dx = lds_f(m.wx, l * cap + j) - xe;
            if (dx * dx < k.T_x) jm = j;
        }
        if (cfg) hl[4 * i] = jm; else hl[4 * i + 3] = jm;
    }

    // weighted refit on the x hits, as a correction to the three-point solution
    float S00 = 0.0f, S01 = 0.0f, S02 = 0.0f, S11 = 0.0f, S12 = 0.0f, S22 = 0.0f, b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (!is_x(l) || hl[l] < 0) continue;
        int q = l * cap + hl[l];
        float u = (zat(l, hl[l]) - k.z_ref) * 1e-3f;
        float f = f2_of(u, D);
        float r = lds_f(m.wx, q) - model_x(A, T, C, u, D);
        float wt = __ldg(b.w + m.h->wbeg[l] + hl[l]);
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
        int j = closest_shared((unsigned)__cvta_generic_to_shared(m.wx + l * cap), m.h->wcnt[l], xe);
        if (j < 0) continue;
        float dx = lds_f(m.wx, l * cap + j) - xe;
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
    float yv[NL], dv[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        yv[l] = 0.0f;
        dv[l] = 0.0f;
        if (is_x(l) || hl[l] < 0) continue;
        int q = l * cap + hl[l];
        int g = m.h->wbeg[l] + hl[l];
        float u = (zat(l, hl[l]) - k.z_ref) * 1e-3f;
        float dd = __ldg(b.dxdy + g);
        dv[l] = dd;
        float y = (model_x(A, T, C, u, D) - lds_f(m.wx, q)) / dd;
        yv[l] = y;
        float wt = __ldg(b.w + g);
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
        float u = (zat(l, hl[l]) - k.z_ref) * 1e-3f;
        float xf = model_x(A, T, C, u, D);
        if (is_x(l)) {
            float r = lds_f(m.wx, q) - xf;
            // T_x a power of two: the product by its reciprocal is the quotient
            qx = qx + (k.inv_T_x != 0.0f ? (r * r) * k.inv_T_x : div_call(r * r, k.T_x));
        } else {
            float yf = Y0 + TY * u;
            float r = lds_f(m.wx, q) - (xf - yf * dv[l]);
            qx = qx + div_call(r * r, T_uv);
            float ry = yv[l] - yf;
            qy = qy + div_call(ry * ry, k.T_y);
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
    cd.st[5] = k.qop_poly ? qop_polynomial(k, s.txs, s.tys, tx, ty_fit) : (tx - s.txs) / k.pk;
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
    slot_sizes(b);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < b.n_events; e += gridDim.x * blockDim.x) {
        int t0 = b.trk_offsets[e], t1 = b.trk_offsets[e + 1];
        for (int t = t0; t < t1; ++t) trk_event[t] = e;
    }
}

// Stage kernels.  Each stage's per-track work is a device function; the
// plain kernel (P = false) calls it once for the tracks given by its global
// warp index, the persistent kernel (P = true) is sized to the GPU and its
// warps take tracks from the stage's device work queue (an atomic cursor)
// until it is empty.

// Window sets in scratch: set ws = t (VELO-UT) or 2t + side (no-UT), its
// twelve windows at [ws * 12, ws * 12 + 12).
template <bool NOUT>
__device__ __forceinline__ void windows_track(const KParams& k, const KBatch& b, const int* __restrict__ trk_event,
                                              int* wbeg, uint8_t* wcnt, int t, int lane) {
    TState s = load_state(b, t);
    const int e = __ldg(trk_event + t);
    constexpr int NS = NOUT ? 2 : 1;
#pragma unroll
    for (int side = 0; side < NS; ++side) {
        int beg, cnt;
        warp_windows<NOUT>(k, b, s, e, lane, side, beg, cnt);
        if (lane < NL) {
            wbeg[((size_t)t * NS + side) * NL + lane] = beg;
            wcnt[((size_t)t * NS + side) * NL + lane] = (uint8_t)cnt;
        }
    }
}

// windows of tracks t0 and t0 + 1 (if it exists) with interleaved searches
__device__ __forceinline__ void windows_track2(const KParams& k, const KBatch& b, const int* __restrict__ trk_event,
                                               int* wbeg, uint8_t* wcnt, int t0, int lane) {
    const bool has1 = t0 + 1 < b.n_tracks;
    const TState s0 = load_state(b, t0);
    const TState s1 = has1 ? load_state(b, t0 + 1) : s0;
    const int e0 = __ldg(trk_event + t0), e1 = has1 ? __ldg(trk_event + t0 + 1) : e0;
    const int l = lane < NL ? lane : (lane < 2 * NL ? lane - NL : 0);
    float xmin0, xmax0, c0, xmin1, xmax1, c1;
    window_limits<false>(k, s0, l, 0, xmin0, xmax0, c0);
    window_limits<false>(k, s1, l, 0, xmin1, xmax1, c1);
    const int* off0 = b.hit_offsets + (size_t)e0 * NB + ((s0.tys >= 0.0f) ? 1 : 0) * NL + l;
    const int* off1 = b.hit_offsets + (size_t)e1 * NB + ((s1.tys >= 0.0f) ? 1 : 0) * NL + l;
    int v0 = 0, v1 = 0;
    if (lane < 2 * NL) {
        v0 = __ldg(off0);
        v1 = has1 ? __ldg(off1) : 0;
        const int h0 = __ldg(off0 + 1), h1 = has1 ? __ldg(off1 + 1) : 0;
        const bool up = lane >= NL;
        if (b.x_coarse) bound2_coarse(b.x, b.x_coarse, v0, h0, up ? xmax0 : xmin0, v1, h1, up ? xmax1 : xmin1, up);
        else bound2_global(b.x, v0, h0, up ? xmax0 : xmin0, v1, h1, up ? xmax1 : xmin1, up);
    }
    int hi0 = __shfl_sync(FULL, v0, (lane + NL) & 31), hi1 = __shfl_sync(FULL, v1, (lane + NL) & 31);
    if (lane < NL) {
        const int lo0 = v0, lo1 = v1;
        if (hi0 < lo0) hi0 = lo0;
        if (hi1 < lo1) hi1 = lo1;
        // the capped windows' centre searches, together
        int cc0 = lo0, cc1 = lo1;
        const bool cap0 = hi0 - lo0 > k.cap, cap1 = has1 && hi1 - lo1 > k.cap;
        if (b.x_coarse) bound2_coarse(b.x, b.x_coarse, cc0, cap0 ? hi0 : lo0, c0, cc1, cap1 ? hi1 : lo1, c1, false);
        else bound2_global(b.x, cc0, cap0 ? hi0 : lo0, c0, cc1, cap1 ? hi1 : lo1, c1, false);
        int st0 = lo0, n0 = hi0 - lo0, st1 = lo1, n1 = hi1 - lo1;
        if (cap0) {
            st0 = cc0 - k.cap / 2;
            if (st0 > hi0 - k.cap) st0 = hi0 - k.cap;
            if (st0 < lo0) st0 = lo0;
            n0 = k.cap;
        }
        if (cap1) {
            st1 = cc1 - k.cap / 2;
            if (st1 > hi1 - k.cap) st1 = hi1 - k.cap;
            if (st1 < lo1) st1 = lo1;
            n1 = k.cap;
        }
        wbeg[(size_t)t0 * NL + lane] = st0;
        wcnt[(size_t)t0 * NL + lane] = (uint8_t)n0;
        if (has1) {
            wbeg[(size_t)(t0 + 1) * NL + lane] = st1;
            wcnt[(size_t)(t0 + 1) * NL + lane] = (uint8_t)n1;
        }
    }
}

// stage 1: windows (warp per track)
template <bool P, bool NOUT>
__global__ void k_windows(KParams k, KBatch b, const int* __restrict__ trk_event, int* wbeg, uint8_t* wcnt,
                          int* cursor) {
    const int lane = threadIdx.x & 31;
    slot_sizes(b);
    if (!P) {
        const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (t < b.n_tracks) windows_track<NOUT>(k, b, trk_event, wbeg, wcnt, t, lane);
        return;
    }
    if (!NOUT) {
        for (;;) {
            const int t0 = queue_take(cursor, 2, lane);
            if (t0 >= b.n_tracks) break;
            windows_track2(k, b, trk_event, wbeg, wcnt, t0, lane);
        }
        return;
    }
    for (;;) {
        const int t = queue_take(cursor, 1, lane);
        if (t >= b.n_tracks) break;
        windows_track<NOUT>(k, b, trk_event, wbeg, wcnt, t, lane);
    }
}

// window set ws into the slot's descriptors
__device__ __forceinline__ void load_windows(const int* wbeg, const uint8_t* wcnt, int ws, const Slot& m, int lane) {
    if (lane < NL) {
        m.h->wbeg[lane] = wbeg[(size_t)ws * NL + lane];
        m.h->wcnt[lane] = wcnt[(size_t)ws * NL + lane];
    }
    __syncwarp();
}

constexpr int PLAIN_WARPS = 8;

template <int NIT, bool NOUT, bool HP = false>
__device__ __forceinline__ void triplets_track(const KParams& k, const KBatch& b, const int* __restrict__ wbeg,
                                               const uint8_t* __restrict__ wcnt, uint64_t* keys, uint8_t* ntrip,
                                               const Slot& m, const Scratch& sc, int t, int lane) {
    TState s = load_state(b, t);
    int nt = 0;
    uint64_t top = NOKEY;
    if (!NOUT) {
        load_windows(wbeg, wcnt, t, m, lane);
        stage_windows<true>(k, b, m, lane);
        top = triplet_scan<NIT, HP>(k, s, m, sc, lane, nt);
    } else if (k.n_trip > 0) {
        // both charge assumptions into one list: stage and scan each set
        int nb = 0;
        uint64_t thr = NOKEY;
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
            load_windows(wbeg, wcnt, 2 * t + side, m, lane);
            stage_windows<true>(k, b, m, lane);
            triplet_pass<NIT, true>(k, s, m, sc, lane, side, nb, thr, top);
        }
        nt = select_buffer(sc, nb, k.n_trip, thr, lane, top);
    }
    if (lane < nt) keys[(size_t)t * k.n_trip + lane] = top;
    if (lane == 0) ntrip[t] = (uint8_t)nt;
    __syncwarp();
}

// stage 2: triplet seeding (warp per track); HP: the half-precision
// pre-filter of the pairs
template <int NIT, bool P, bool NOUT, bool HP = false>
__global__ void __launch_bounds__(PLAIN_WARPS * 32, 5) k_triplets(KParams k, KBatch b, const int* __restrict__ wbeg, const uint8_t* __restrict__ wcnt,
                           uint64_t* keys, uint8_t* ntrip, int* cursor) {
    static_assert(!HP || !NOUT, "the pre-filter follows VELO-UT input only");
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Slot m = slot_at(smem, warp, k.cap);
    const Scratch sc = scratch_at(smem + PLAIN_WARPS * slot_bytes(k.cap), warp, HP);
    slot_sizes(b);
    if (!P) {
        const int t = blockIdx.x * PLAIN_WARPS + warp;
        if (t < b.n_tracks) triplets_track<NIT, NOUT, HP>(k, b, wbeg, wcnt, keys, ntrip, m, sc, t, lane);
        return;
    }
    for (;;) {
        const int t = queue_take(cursor, 1, lane);
        if (t >= b.n_tracks) break;
        triplets_track<NIT, NOUT, HP>(k, b, wbeg, wcnt, keys, ntrip, m, sc, t, lane);
    }
}

__device__ __forceinline__ void write_cand(CandRec* cands, const KParams& k, int t, int r, const Cand& cd, int side) {
    CandRec rec;
    rec.Q = cd.Q;
    rec.status = (int8_t)cd.status;
    rec.n = (int8_t)cd.n;
#pragma unroll
    for (int l = 0; l < NL; ++l) rec.hl[l] = (int8_t)(cd.status == 0 ? cd.hl[l] : -1);
    rec.side = (int8_t)side;
#pragma unroll
    for (int p = 0; p < 5; ++p) rec.pad[p] = 0;
#pragma unroll
    for (int p = 0; p < 6; ++p) rec.st[p] = cd.status == 0 ? cd.st[p] : 0.0f;
    cands[(size_t)t * k.n_trip + r] = rec;
}

__device__ __forceinline__ void clear_cand(Cand& cd) {
    cd.status = 9;
    cd.Q = 0.0f;
    cd.n = 0;
#pragma unroll
    for (int p = 0; p < 6; ++p) cd.st[p] = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) cd.hl[l] = -1;
}

// No-UT extension of track t (one track per warp, lane r extends triplet
// r): each window set is staged in turn and extends the triplets seeded in
// it.
template <bool SEL>
__device__ __forceinline__ void extend_track_no_ut(const KParams& k, const KBatch& b, const int* __restrict__ wbeg,
                                                   const uint8_t* __restrict__ wcnt,
                                                   const uint64_t* __restrict__ keys,
                                                   const uint8_t* __restrict__ ntrip, CandRec* cands,
                                                   const KOut& o, const Slot& m, int t, int lane) {
    const bool live = t < b.n_tracks;
    const bool act = live && lane < ntrip[t];
    const uint64_t key = act ? keys[(size_t)t * k.n_trip + lane] : NOKEY;
    const int side_r = (int)((key >> 19) & 1);
    Cand cd;
    clear_cand(cd);
    int hg[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) hg[l] = -1;
    TState s = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (live) s = load_state(b, t);
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const bool mine = act && side_r == side;
        if (!__any_sync(FULL, mine)) continue;
        load_windows(wbeg, wcnt, 2 * t + side, m, lane);
        stage_windows(k, b, m, lane);
        if (mine) {
            extend_fit(k, b, s, m, key, cd);
#pragma unroll
            for (int l = 0; l < NL; ++l) hg[l] = (cd.status == 0 && cd.hl[l] >= 0) ? m.h->wbeg[l] + cd.hl[l] : -1;
        }
        __syncwarp();
    }
    if (SEL) group_select_write<32>(o, t, live, lane, act && cd.status == 0, cd.Q, cd.n, hg, cd.st);
    else if (act) write_cand(cands, k, t, lane, cd, side_r);
    __syncwarp();
}

// SEL = false: write every candidate for the selection kernel; SEL = true:
// select inside the 16/32-lane group and write the track's output directly.
template <int TPW, bool SEL>
__device__ __forceinline__ void extend_tracks(const KParams& k, const KBatch& b, const int* __restrict__ wbeg,
                                              const uint8_t* __restrict__ wcnt, const uint64_t* __restrict__ keys,
                                              const uint8_t* __restrict__ ntrip, CandRec* cands, const KOut& o,
                                              const Slot* sl, int t0, int lane) {
    // the window descriptors of the TPW tracks in one round trip (lanes 16q..
    // for track q; a track past the end gets empty windows), then every
    // staging copy of both tracks in flight at once
    {
        const int qw = lane >> 4, lw = lane & 15, tw = t0 + qw;
        int wb = 0, wc = 0;
        if (qw < TPW && lw < NL && tw < b.n_tracks) {
            wb = wbeg[(size_t)tw * NL + lw];
            wc = wcnt[(size_t)tw * NL + lw];
        }
        if (qw < TPW && lw < NL) {
            const Slot& mw = (TPW == 2 && qw == 1) ? sl[TPW - 1] : sl[0];
            mw.h->wbeg[lw] = wb;
            mw.h->wcnt[lw] = wc;
        }
        __syncwarp();
    }
#pragma unroll
    for (int qq = 0; qq < TPW; ++qq) stage_issue<false, false>(k, b, sl[qq], lane);
    // the z, dxdy and w lines of every window go to L2 while x is staged: the
    // candidates read them for the hits they use
    {
        const int qw = lane >> 4, lw = lane & 15;
        if (qw < TPW && lw < NL) {
            const Slot& mw = (TPW == 2 && qw == 1) ? sl[TPW - 1] : sl[0];
            const int wb = mw.h->wbeg[lw], wc = mw.h->wcnt[lw];
            if (wc > 0) {
                const uintptr_t lines[3] = {reinterpret_cast<uintptr_t>(b.z + wb), reinterpret_cast<uintptr_t>(b.dxdy + wb),
                                            reinterpret_cast<uintptr_t>(b.w + wb)};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const uintptr_t p0 = lines[a] & ~uintptr_t(127), p1 = lines[a] + (uintptr_t)wc * 4;
                    for (uintptr_t q = p0; q < p1; q += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
                }
            }
        }
    }
    constexpr int G = 32 / TPW;
    const int q = lane / G, r = lane % G;
    const int t = t0 + q;
    Slot mq = sl[0];
    if (TPW == 2 && q == 1) mq = sl[TPW - 1];
    const bool live = t < b.n_tracks;
    // this lane's candidate inputs load while the copies are in flight
    const bool act = live && r < ntrip[t];
    const uint64_t key = act ? keys[(size_t)t * k.n_trip + r] : NOKEY;
    TState s = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (act) s = load_state(b, t);
    stage_finish<TPW, false, false>(k, sl, lane);
    Cand cd;
    cd.status = 9;
    cd.Q = 0.0f;
    cd.n = 0;
#pragma unroll
    for (int p = 0; p < 6; ++p) cd.st[p] = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) cd.hl[l] = -1;
    if (act) extend_fit<true>(k, b, s, mq, key, cd);
    if (SEL) {
        int hg[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) hg[l] = (act && cd.status == 0 && cd.hl[l] >= 0) ? mq.h->wbeg[l] + cd.hl[l] : -1;
        group_select_write<G>(o, t, live, r, act && cd.status == 0, cd.Q, cd.n, hg, cd.st);
    } else if (act) {
        write_cand(cands, k, t, r, cd, 0);
    }
    __syncwarp();
}

// stage 3: extension and fit of every kept triplet; TPW tracks per warp
// (two when n_triplets <= 16: lanes 0..15 and 16..31).  The persistent
// variant also selects and writes the output (no candidate round trip).
// NOUT: one track per warp (TPW = 1), window sets staged in turn.
template <int TPW, bool P, bool NOUT>
__global__ void __launch_bounds__(PLAIN_WARPS * 32, 4) k_extend(
    KParams k, KBatch b, const int* __restrict__ wbeg, const uint8_t* __restrict__ wcnt,
    const uint64_t* __restrict__ keys, const uint8_t* __restrict__ ntrip, CandRec* cands, KOut o, int* cursor) {
    static_assert(!NOUT || TPW == 1, "the no-UT extension runs one track per warp");
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Slot sl[TPW];
#pragma unroll
    for (int q = 0; q < TPW; ++q) sl[q] = slot_at(smem, warp * TPW + q, k.cap);
    slot_sizes(b);
    if (!P) {
        const int t0 = (blockIdx.x * PLAIN_WARPS + warp) * TPW;
        if (t0 < b.n_tracks) {
            if (NOUT) extend_track_no_ut<false>(k, b, wbeg, wcnt, keys, ntrip, cands, o, sl[0], t0, lane);
            else extend_tracks<TPW, false>(k, b, wbeg, wcnt, keys, ntrip, cands, o, sl, t0, lane);
        }
        return;
    }
    for (;;) {
        const int t0 = queue_take(cursor, TPW, lane);
        if (t0 >= b.n_tracks) break;
        if (NOUT) extend_track_no_ut<true>(k, b, wbeg, wcnt, keys, ntrip, cands, o, sl[0], t0, lane);
        else extend_tracks<TPW, true>(k, b, wbeg, wcnt, keys, ntrip, cands, o, sl, t0, lane);
    }
}

// Block form of the persistent extension (VELO-UT input): a block takes a
// tile of TT = min(256 / n_triplets, 32) consecutive input tracks and runs one
// candidate per thread, thread c extending triplet c % n_triplets of track
// c / n_triplets, so that the candidates of about 21 tracks (n_triplets 12)
// fill all of the block's lanes instead of 24 of every warp's 32.  The
// tile's x windows are staged once per track (warp w stages tracks w, w + 8,
// ...); the lowest (Q bits, rank) key of a track is found with a
// shared-memory minimum, and its candidate's thread writes the output.
constexpr int XB_THREADS = 256;
constexpr int XB_MAX_TRACKS = 32;   // tracks of a tile, most (shared memory of their windows)

__host__ __device__ inline size_t xslot_bytes(int cap) { return align16(sizeof(SlotHead)) + size_t(NL) * cap * sizeof(float); }
__host__ __device__ inline int xtile_tracks(int n_trip) {
    const int tt = XB_THREADS / (n_trip > 0 ? n_trip : 1);
    return tt < XB_MAX_TRACKS ? tt : XB_MAX_TRACKS;
}
__host__ __device__ inline size_t xblock_smem_bytes(int cap, int n_trip) {
    return align16((size_t)xtile_tracks(n_trip) * sizeof(unsigned long long)) + (size_t)xtile_tracks(n_trip) * xslot_bytes(cap);
}

__device__ __forceinline__ Slot xslot_at(char* base, int i, int cap) {
    char* p = base + (size_t)i * xslot_bytes(cap);
    Slot s;
    s.h = reinterpret_cast<SlotHead*>(p);
    s.wx = reinterpret_cast<float*>(p + align16(sizeof(SlotHead)));
    s.wz = nullptr;
    return s;
}

// L2 prefetch of the z, dxdy and w lines of window lw of a staged slot
__device__ __forceinline__ void prefetch_window_lines(const KBatch& b, const Slot& m, int lw) {
    const int wb = m.h->wbeg[lw], wc = m.h->wcnt[lw];
    if (wc <= 0) return;
    const uintptr_t lines[3] = {reinterpret_cast<uintptr_t>(b.z + wb), reinterpret_cast<uintptr_t>(b.dxdy + wb),
                                reinterpret_cast<uintptr_t>(b.w + wb)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uintptr_t p0 = lines[a] & ~uintptr_t(127), p1 = lines[a] + (uintptr_t)wc * 4;
        for (uintptr_t q = p0; q < p1; q += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
    }
}

__global__ void __launch_bounds__(XB_THREADS, 5) k_extend_block(KParams k, KBatch b, const int* __restrict__ wbeg,
                                                              const uint8_t* __restrict__ wcnt,
                                                              const uint64_t* __restrict__ keys,
                                                              const uint8_t* __restrict__ ntrip, KOut o, int* cursor) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NT = k.n_trip > 0 ? k.n_trip : 1;
    const int TT = xtile_tracks(k.n_trip);
    unsigned long long* sel = reinterpret_cast<unsigned long long*>(smem);
    char* slots = smem + align16((size_t)TT * sizeof(unsigned long long));
    slot_sizes(b);
    const int q = tid / NT, r = tid - q * NT;   // this thread's track in the tile and triplet rank
    for (;;) {
        if (tid == 0) s_t0 = atomicAdd(cursor, TT);
        __syncthreads();
        const int t0 = s_t0;
        if (t0 >= b.n_tracks) break;
        // stage the tile's windows: warp w stages tracks w, w + 8, ...
        for (int qq = warp; qq < TT; qq += XB_THREADS / 32) {
            const Slot m = xslot_at(slots, qq, k.cap);
            const int t = t0 + qq;
            if (lane < NL) {
                int wb = 0, wc = 0;
                if (t < b.n_tracks) {
                    wb = wbeg[(size_t)t * NL + lane];
                    wc = wcnt[(size_t)t * NL + lane];
                }
                m.h->wbeg[lane] = wb;
                m.h->wcnt[lane] = wc;
            }
            __syncwarp();
            stage_issue<false, false>(k, b, m, lane);
            if (lane < NL) prefetch_window_lines(b, m, lane);
        }
        if (tid < TT) sel[tid] = NOKEY;
        // this thread's candidate inputs load while the copies are in flight
        const int t = t0 + q;
        const bool live = q < TT && t < b.n_tracks;
        const bool act = live && r < ntrip[t];
        const uint64_t key = act ? keys[(size_t)t * k.n_trip + r] : NOKEY;
        TState s = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (act) s = load_state(b, t);
        cp_async_wait_all();
        __syncthreads();
        Cand cd;
        cd.status = 9;
        cd.Q = 0.0f;
        cd.n = 0;
        Slot m;
        m.h = nullptr;
        m.wx = nullptr;
        m.wz = nullptr;
        if (act) {
            m = xslot_at(slots, q, k.cap);
            extend_fit<true>(k, b, s, m, key, cd);
        }
        const bool have = act && cd.status == 0;
        const unsigned long long mine = have ? (((unsigned long long)__float_as_uint(cd.Q) << 32) | (unsigned)r) : NOKEY;
        if (have) atomicMin(&sel[q], mine);
        __syncthreads();
        if (live) {
            const unsigned long long best = sel[q];
            if (best == NOKEY) {
                if (r == 0) {
                    o.found[t] = 0;
                    o.nhits[t] = 0;
                }
            } else if (have && mine == best) {
#pragma unroll
                for (int l = 0; l < NL; ++l)
                    o.hit_idx[(size_t)t * NL + l] = cd.hl[l] >= 0 ? m.h->wbeg[l] + cd.hl[l] : -1;
#pragma unroll
                for (int p = 0; p < 6; ++p) o.state[(size_t)t * 6 + p] = cd.st[p];
                o.quality[t] = cd.Q;
                o.nhits[t] = (uint8_t)cd.n;
                o.found[t] = 1;
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void select_track(const KParams& k, const int* __restrict__ wbeg,
                                             const uint8_t* __restrict__ ntrip, const CandRec* __restrict__ cands,
                                             const KOut& o, int t, int lane) {
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
        const size_t ws = (size_t)t * (k.no_ut ? 2 : 1) + r.side;
#pragma unroll
        for (int l = 0; l < NL; ++l) hg[l] = r.hl[l] >= 0 ? wbeg[ws * NL + l] + r.hl[l] : -1;
#pragma unroll
        for (int q = 0; q < 6; ++q) st[q] = r.st[q];
    }
    group_select_write<32>(o, t, true, lane, have, Q, n, hg, st);
}

// stage 4: warp-vote selection and output (warp per track)
template <bool P>
__global__ void k_select(KParams k, KBatch b, const int* __restrict__ wbeg, const uint8_t* __restrict__ ntrip,
                         const CandRec* __restrict__ cands, KOut o, int* cursor) {
    const int lane = threadIdx.x & 31;
    if (!P) {
        const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        if (t < b.n_tracks) select_track(k, wbeg, ntrip, cands, o, t, lane);
        return;
    }
    for (;;) {
        const int t = queue_take(cursor, 1, lane);
        if (t >= b.n_tracks) break;
        select_track(k, wbeg, ntrip, cands, o, t, lane);
    }
}

// persistent form.  SYNC: blocks take tiles of (warps x TPW) consecutive
// input tracks from the device work queue and their warps step through the
// stages together (block barriers between windows + staging, triplet
// seeding, extension + selection).  !SYNC: every warp takes its own TPW
// tracks from the queue and runs on without waiting for the others.
template <int NIT, int TPW, bool SYNC>
__global__ void __launch_bounds__(512, 1) k_tile(KParams k, KBatch b, KOut o, int* cursor) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_base, s_ev;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    Slot sl[TPW];
#pragma unroll
    for (int q = 0; q < TPW; ++q) sl[q] = slot_at(smem, warp * TPW + q, k.cap);
    const Scratch sc = scratch_at(smem + (size_t)nw * TPW * slot_bytes(k.cap), warp);
    slot_sizes(b);
    for (;;) {
        int first, e;
        if (SYNC) {
            if (threadIdx.x == 0) {
                int base = atomicAdd(cursor, nw * TPW);
                s_base = base;
                s_ev = base < b.n_tracks ? event_of(b.trk_offsets, b.n_events, base) : 0;
            }
            __syncthreads();
            const int base = s_base;
            e = s_ev;
            __syncthreads();
            if (base >= b.n_tracks) break;
            first = base + warp * TPW;
        } else {
            int v = 0;
            if (lane == 0) v = atomicAdd(cursor, TPW);
            first = __shfl_sync(FULL, v, 0);
            if (first >= b.n_tracks) break;
            e = event_of(b.trk_offsets, b.n_events, first);
        }

        TState st[TPW];
        bool live[TPW];
#pragma unroll
        for (int q = 0; q < TPW; ++q) {
            const int t = first + q;
            live[q] = t < b.n_tracks;
            if (live[q]) {
                while (t >= __ldg(b.trk_offsets + e + 1)) ++e;
                st[q] = load_state(b, t);
                int beg, cnt;
                warp_windows<false>(k, b, st[q], e, lane, 0, beg, cnt);
                if (lane < NL) {
                    sl[q].h->wbeg[lane] = beg;
                    sl[q].h->wcnt[lane] = cnt;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < TPW; ++q)
            if (live[q]) stage_windows(k, b, sl[q], lane);
        if (SYNC) __syncthreads();

        uint64_t top[TPW];
        int nt[TPW];
#pragma unroll
        for (int q = 0; q < TPW; ++q) {
            nt[q] = 0;
            top[q] = NOKEY;
            if (live[q]) top[q] = triplet_scan<NIT>(k, st[q], sl[q], sc, lane, nt[q]);
        }
        if (SYNC) __syncthreads();

        constexpr int G = 32 / TPW;
        const int qg = lane / G, r = lane % G;
        uint64_t key = NOKEY;
#pragma unroll
        for (int q = 0; q < TPW; ++q) {
            uint64_t kq = shfl64(top[q], r);
            if (q == qg) key = kq;
        }
        bool lv = false;
        int ntq = 0;
        TState sq = st[0];
#pragma unroll
        for (int q = 0; q < TPW; ++q)
            if (q == qg) {
                lv = live[q];
                ntq = nt[q];
                sq = st[q];
            }
        Cand cd;
        cd.status = 9;
        cd.Q = 0.0f;
        cd.n = 0;
#pragma unroll
        for (int p = 0; p < 6; ++p) cd.st[p] = 0.0f;
#pragma unroll
        for (int l = 0; l < NL; ++l) cd.hl[l] = -1;
        const bool act = lv && r < ntq;
        Slot mq = sl[0];
        if (TPW == 2 && qg == 1) mq = sl[TPW - 1];
        if (act) extend_fit(k, b, sq, mq, key, cd);
        int hg[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) hg[l] = (act && cd.status == 0 && cd.hl[l] >= 0) ? mq.h->wbeg[l] + cd.hl[l] : -1;
        group_select_write<G>(o, first + qg, lv, r, act && cd.status == 0, cd.Q, cd.n, hg, cd.st);
        if (SYNC) __syncthreads(); else __syncwarp();
    }
}

// debug dump of the plain form's windows and triplet stage in packed indices
__global__ void k_debug_triplets(KParams k, KBatch b, const int* __restrict__ wbeg, const uint8_t* __restrict__ wcnt,
                                 const uint64_t* __restrict__ keys, const uint8_t* __restrict__ ntrip,
                                 int* win_count_out, int* n_trip_out, int* trip_out, float* chi2_out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.n_tracks) return;
    const int ns = k.no_ut ? 2 : 1;
    for (int l = 0; l < ns * NL; ++l) win_count_out[(size_t)t * ns * NL + l] = wcnt[(size_t)t * ns * NL + l];
    int nt = ntrip[t];
    n_trip_out[t] = nt;
    for (int r = 0; r < nt; ++r) {
        uint64_t key = keys[(size_t)t * k.n_trip + r];
        int side = (int)((key >> 19) & 1), cfg = (int)((key >> 18) & 1);
        int j0 = (int)((key >> 12) & 63), j2 = (int)((key >> 6) & 63), j1 = (int)(key & 63);
        int L0 = cfg ? 3 : 0, L1 = cfg ? 7 : 4, L2 = cfg ? 11 : 8;
        const int* wb = wbeg + ((size_t)t * ns + side) * NL;
        int* q = trip_out + ((size_t)t * k.n_trip + r) * 4;
        q[0] = cfg + 2 * side;
        q[1] = wb[L0] + j0;
        q[2] = wb[L1] + j1;
        q[3] = wb[L2] + j2;
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
                                int* ev_count, const int* n_dev) {
    int lane = threadIdx.x & 31;
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    n_events = slot_events(n_dev, n_events);
    if (e >= n_events) return;
    int t0 = trk_offsets[e], t1 = trk_offsets[e + 1];
    int c = 0;
    for (int t = t0 + lane; t < t1; t += 32) c += found[t] ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane == 0) ev_count[e] = c;
}

// exclusive scan of the per-event counts by one block
__global__ void k_compact_scan(const int* __restrict__ ev_count, int n_events, int* out_offsets, int* n_out,
                               const int* n_dev) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    n_events = slot_events(n_dev, n_events);
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
                                  const int* __restrict__ out_offsets, int* out_trk, const int* n_dev) {
    int lane = threadIdx.x & 31;
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    n_events = slot_events(n_dev, n_events);
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

// Coarse index of the packed x: every 32nd value (slot form: up to the
// batch's last hit).
__global__ void k_coarse(KBatch b, float* __restrict__ c) {
    int n_hits = b.n_hits;
    if (b.n_dev) {
        slot_sizes(b);
        const int h = b.hit_offsets[(size_t)b.n_events * NB];
        n_hits = h < 0 ? 0 : (h < n_hits ? h : n_hits);
    }
    const int n = (n_hits + 31) >> 5;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) c[i] = __ldg(b.x + 32 * (size_t)i);
}

// Slot form with a gather source: the input states of batch event e's
// tracks are copied from the source arrays, starting at trk_src[e], to the
// batch's own state arrays (warp per event, lanes over its tracks).
__global__ void k_gather_states(KBatch b, const int* __restrict__ trk_src, const float* __restrict__ sx,
                                const float* __restrict__ sy, const float* __restrict__ stx,
                                const float* __restrict__ sty, const float* __restrict__ sqop, float* dx, float* dy,
                                float* dtx, float* dty, float* dqop) {
    slot_sizes(b);
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < b.n_events; e += nw) {
        const int t0 = b.trk_offsets[e], t1 = min(b.trk_offsets[e + 1], b.n_tracks);
        const long d = (long)trk_src[e] - t0;
        for (int t = t0 + lane; t < t1; t += 32) {
            dx[t] = sx[d + t];
            dy[t] = sy[d + t];
            dtx[t] = stx[d + t];
            dty[t] = sty[d + t];
            dqop[t] = sqop[d + t];
        }
    }
}

// ================================================================ launchers

static inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

static cudaError_t set_smem(const void* fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_track_event(const KBatch& b, int* trk_event, cudaStream_t s) {
    if (b.n_events <= 0) return cudaSuccess;
    k_track_event<<<cdiv(b.n_events, 256), 256, 0, s>>>(b, trk_event);
    return cudaGetLastError();
}

// Stage launches.  cursor == nullptr: plain grid (one pass); otherwise a
// persistent grid of `blocks` blocks that drains the stage's work queue.
cudaError_t launch_windows(const KParams& k, const KBatch& b, const int* trk_event, int* wbeg, uint8_t* wcnt,
                           cudaStream_t s, int* cursor, int blocks) {
    if (b.n_tracks <= 0) return cudaSuccess;
    const int plain_grid = cdiv((long)b.n_tracks * 32, 256);
    if (k.no_ut) {
        if (cursor) k_windows<true, true><<<blocks, 256, 0, s>>>(k, b, trk_event, wbeg, wcnt, cursor);
        else k_windows<false, true><<<plain_grid, 256, 0, s>>>(k, b, trk_event, wbeg, wcnt, nullptr);
    } else {
        if (cursor) k_windows<true, false><<<blocks, 256, 0, s>>>(k, b, trk_event, wbeg, wcnt, cursor);
        else k_windows<false, false><<<plain_grid, 256, 0, s>>>(k, b, trk_event, wbeg, wcnt, nullptr);
    }
    return cudaGetLastError();
}

template <int NIT, bool P, bool NOUT, bool HP = false>
static cudaError_t launch_triplets_t(const KParams& k, const KBatch& b, const int* wbeg, const uint8_t* wcnt,
                                     uint64_t* keys, uint8_t* ntrip, cudaStream_t s, int* cursor, int blocks) {
    size_t sm = block_smem_bytes(k.cap, PLAIN_WARPS, 1, HP);
    cudaError_t err = set_smem((const void*)k_triplets<NIT, P, NOUT, HP>, sm);
    if (err != cudaSuccess) return err;
    const int grid = P ? blocks : cdiv(b.n_tracks, PLAIN_WARPS);
    k_triplets<NIT, P, NOUT, HP><<<grid, PLAIN_WARPS * 32, sm, s>>>(k, b, wbeg, wcnt, keys, ntrip, cursor);
    return cudaGetLastError();
}

// items per lane NIT: 32 * NIT >= 2 * cap; the no-UT variant always takes 4
template <bool P>
static cudaError_t launch_triplets_p(const KParams& k, const KBatch& b, const int* wbeg, const uint8_t* wcnt,
                                     uint64_t* keys, uint8_t* ntrip, cudaStream_t s, int* cursor, int blocks) {
    if (k.no_ut) return launch_triplets_t<4, P, true>(k, b, wbeg, wcnt, keys, ntrip, s, cursor, blocks);
    if (k.cap <= 16) return launch_triplets_t<1, P, false>(k, b, wbeg, wcnt, keys, ntrip, s, cursor, blocks);
    if (k.cap <= 32) return launch_triplets_t<2, P, false>(k, b, wbeg, wcnt, keys, ntrip, s, cursor, blocks);
    return launch_triplets_t<4, P, false>(k, b, wbeg, wcnt, keys, ntrip, s, cursor, blocks);
}

cudaError_t launch_triplets(const KParams& k, const KBatch& b, const int* trk_event, const int* wbeg,
                            const uint8_t* wcnt, uint64_t* keys, uint8_t* ntrip, cudaStream_t s, int* cursor,
                            int blocks, int prefilter) {
    (void)trk_event;
    if (b.n_tracks <= 0) return cudaSuccess;
    if (prefilter) {
        // persistent form, VELO-UT input (the entry points refuse the rest)
        if (!cursor || k.no_ut) return cudaErrorInvalidValue;
        if (k.cap <= 16) return launch_triplets_t<1, true, false, true>(k, b, wbeg, wcnt, keys, ntrip, s, cursor, blocks);
        if (k.cap <= 32) return launch_triplets_t<2, true, false, true>(k, b, wbeg, wcnt, keys, ntrip, s, cursor, blocks);
        return launch_triplets_t<4, true, false, true>(k, b, wbeg, wcnt, keys, ntrip, s, cursor, blocks);
    }
    if (cursor) return launch_triplets_p<true>(k, b, wbeg, wcnt, keys, ntrip, s, cursor, blocks);
    return launch_triplets_p<false>(k, b, wbeg, wcnt, keys, ntrip, s, nullptr, 0);
}

template <int TPW, bool P, bool NOUT>
static cudaError_t launch_extend_t(const KParams& k, const KBatch& b, const int* wbeg, const uint8_t* wcnt,
                                   const uint64_t* keys, const uint8_t* ntrip, CandRec* cands, const KOut& o,
                                   cudaStream_t s, int* cursor, int blocks) {
    size_t sm = (size_t)PLAIN_WARPS * TPW * slot_bytes(k.cap);
    cudaError_t err = set_smem((const void*)k_extend<TPW, P, NOUT>, sm);
    if (err != cudaSuccess) return err;
    const int grid = P ? blocks : cdiv(b.n_tracks, PLAIN_WARPS * TPW);
    k_extend<TPW, P, NOUT><<<grid, PLAIN_WARPS * 32, sm, s>>>(k, b, wbeg, wcnt, keys, ntrip, cands, o, cursor);
    return cudaGetLastError();
}

cudaError_t launch_extend(const KParams& k, const KBatch& b, const int* trk_event, const int* wbeg,
                          const uint8_t* wcnt, const uint64_t* keys, const uint8_t* ntrip, CandRec* cands,
                          const KOut& o, cudaStream_t s, int* cursor, int blocks, int form) {
    (void)trk_event;
    if (b.n_tracks <= 0) return cudaSuccess;
    if (k.no_ut) {
        if (cursor) return launch_extend_t<1, true, true>(k, b, wbeg, wcnt, keys, ntrip, cands, o, s, cursor, blocks);
        return launch_extend_t<1, false, true>(k, b, wbeg, wcnt, keys, ntrip, cands, o, s, nullptr, 0);
    }
    if (cursor && form == 1) {
        const size_t sm = xblock_smem_bytes(k.cap, k.n_trip);
        cudaError_t err = set_smem((const void*)k_extend_block, sm);
        if (err != cudaSuccess) return err;
        k_extend_block<<<blocks, XB_THREADS, sm, s>>>(k, b, wbeg, wcnt, keys, ntrip, o, cursor);
        return cudaGetLastError();
    }
    if (k.n_trip <= 16) {
        if (cursor)
            return launch_extend_t<2, true, false>(k, b, wbeg, wcnt, keys, ntrip, cands, o, s, cursor, blocks);
        return launch_extend_t<2, false, false>(k, b, wbeg, wcnt, keys, ntrip, cands, o, s, nullptr, 0);
    }
    if (cursor) return launch_extend_t<1, true, false>(k, b, wbeg, wcnt, keys, ntrip, cands, o, s, cursor, blocks);
    return launch_extend_t<1, false, false>(k, b, wbeg, wcnt, keys, ntrip, cands, o, s, nullptr, 0);
}

cudaError_t launch_select(const KParams& k, const KBatch& b, const int* wbeg, const uint8_t* ntrip,
                          const CandRec* cands, const KOut& o, cudaStream_t s, int* cursor, int blocks) {
    if (b.n_tracks <= 0) return cudaSuccess;
    if (cursor) k_select<true><<<blocks, 256, 0, s>>>(k, b, wbeg, ntrip, cands, o, cursor);
    else k_select<false><<<cdiv((long)b.n_tracks * 32, 256), 256, 0, s>>>(k, b, wbeg, ntrip, cands, o, nullptr);
    return cudaGetLastError();
}

// resident blocks per SM of each persistent stage kernel (for grid sizing)
cudaError_t stage_blocks_per_sm(const KParams& k, int* out4) {
    cudaError_t err;
    size_t smt = block_smem_bytes(k.cap, PLAIN_WARPS, 1);
    const int tpw = (k.n_trip <= 16 && !k.no_ut) ? 2 : 1;
    size_t sme = (size_t)PLAIN_WARPS * tpw * slot_bytes(k.cap);
    const void* ft = k.no_ut ? (const void*)k_triplets<4, true, true>
                   : k.cap <= 16 ? (const void*)k_triplets<1, true, false>
                   : k.cap <= 32 ? (const void*)k_triplets<2, true, false>
                                 : (const void*)k_triplets<4, true, false>;
    // the extension's grid follows its default form: the block form for
    // VELO-UT input (the warp form, when chosen instead, then has a few more
    // blocks than fit at once; the extra ones find the queue drained)
    if (!k.no_ut) sme = xblock_smem_bytes(k.cap, k.n_trip);
    const void* fe = k.no_ut ? (const void*)k_extend<1, true, true> : (const void*)k_extend_block;
    const void* fw = k.no_ut ? (const void*)k_windows<true, true> : (const void*)k_windows<true, false>;
    if ((err = set_smem(ft, smt)) != cudaSuccess) return err;
    if ((err = set_smem(fe, sme)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out4[0], fw, 256, 0)) != cudaSuccess)
        return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out4[1], ft, PLAIN_WARPS * 32, smt)) != cudaSuccess)
        return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out4[2], fe, PLAIN_WARPS * 32, sme)) != cudaSuccess)
        return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out4[3], k_select<true>, 256, 0);
}

static int tile_tpw(const KParams& k, int grain) {
    if (grain == 1) return 1;
    return k.n_trip <= 16 ? 2 : 1;
}

// grain: tracks per warp (1, 2; 0 = 2 when n_triplets <= 16); queue: 0 warp
// fetch, 1 block tiles with stage barriers (both carried in `grain`:
// grain + 16 * queue)
template <int NIT>
static const void* tile_fn_nit(int tpw, bool sync) {
    if (tpw == 2) return sync ? (const void*)k_tile<NIT, 2, true> : (const void*)k_tile<NIT, 2, false>;
    return sync ? (const void*)k_tile<NIT, 1, true> : (const void*)k_tile<NIT, 1, false>;
}

static const void* tile_fn(const KParams& k, int tpw, bool sync) {
    if (k.cap <= 16) return tile_fn_nit<1>(tpw, sync);
    if (k.cap <= 32) return tile_fn_nit<2>(tpw, sync);
    return tile_fn_nit<4>(tpw, sync);
}

// the tile kernel follows VELO-UT input only (no_ut is refused by the API)
cudaError_t fused_max_blocks_per_sm(const KParams& k, int warps_per_block, int grain, int* out) {
    if (k.no_ut) return cudaErrorInvalidValue;
    const int tpw = tile_tpw(k, grain & 15);
    const bool sync = (grain >> 4) & 1;
    size_t sm = block_smem_bytes(k.cap, warps_per_block, tpw);
    const void* fn = tile_fn(k, tpw, sync);
    cudaError_t err = set_smem(fn, sm);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, warps_per_block * 32, sm);
}

cudaError_t launch_fused(const KParams& k, const KBatch& b, const KOut& o, int* cursor, int grain,
                         int warps_per_block, int n_blocks, cudaStream_t s) {
    if (k.no_ut) return cudaErrorInvalidValue;
    const int tpw = tile_tpw(k, grain & 15);
    const bool sync = (grain >> 4) & 1;
    size_t sm = block_smem_bytes(k.cap, warps_per_block, tpw);
    const void* fn = tile_fn(k, tpw, sync);
    cudaError_t err = set_smem(fn, sm);
    if (err != cudaSuccess) return err;
    void* args[] = {(void*)&k, (void*)&b, (void*)&o, (void*)&cursor};
    return cudaLaunchKernel(fn, dim3(n_blocks), dim3(warps_per_block * 32), args, sm, s);
}

cudaError_t launch_hits_to_raw(const uint8_t* found, int* hit_idx, const int* perm, int n_tracks, int base,
                              cudaStream_t s) {
    if (n_tracks <= 0) return cudaSuccess;
    k_hits_to_raw<<<cdiv((long)n_tracks * NL, 256), 256, 0, s>>>(found, hit_idx, perm, n_tracks, base);
    return cudaGetLastError();
}

cudaError_t launch_compact(const int* trk_offsets, const uint8_t* found, int n_events, int* ev_count,
                           int* out_offsets, int* out_trk, int* n_out, cudaStream_t s, const int* n_dev) {
    if (n_events > 0) {
        k_compact_count<<<cdiv((long)n_events * 32, 256), 256, 0, s>>>(trk_offsets, found, n_events, ev_count,
                                                                       n_dev);
    }
    k_compact_scan<<<1, 1024, 0, s>>>(ev_count, n_events, out_offsets, n_out, n_dev);
    if (n_events > 0) {
        k_compact_scatter<<<cdiv((long)n_events * 32, 256), 256, 0, s>>>(trk_offsets, found, n_events, out_offsets,
                                                                         out_trk, n_dev);
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse(const KBatch& b, float* x_coarse, int n_sm, cudaStream_t s) {
    if (b.n_hits <= 0) return cudaSuccess;
    const int want = cdiv(((long)b.n_hits + 31) / 32, 256);
    const int grid = want < 16 * n_sm ? want : 16 * n_sm;
    k_coarse<<<grid, 256, 0, s>>>(b, x_coarse);
    return cudaGetLastError();
}

cudaError_t launch_gather_states(const KBatch& b, const int* trk_src, const float* sx, const float* sy,
                                 const float* stx, const float* sty, const float* sqop, int n_sm, cudaStream_t s) {
    if (b.n_events <= 0 || b.n_tracks <= 0) return cudaSuccess;
    const int want = cdiv((long)b.n_events * 32, 256);
    const int grid = want < 8 * n_sm ? want : 8 * n_sm;
    k_gather_states<<<grid, 256, 0, s>>>(b, trk_src, sx, sy, stx, sty, sqop, const_cast<float*>(b.sx),
                                         const_cast<float*>(b.sy), const_cast<float*>(b.stx),
                                         const_cast<float*>(b.sty), const_cast<float*>(b.sqop));
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
