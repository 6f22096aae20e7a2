// Per-event persistent kernel for sm_103a: the persistent form's default.
//
// A block takes one event at a time from a device work queue and follows
// its input tracks zone by zone (Sec. "Defining the search windows": a track
// searches the half of the detector its t_y points to).  For a zone:
//   staging    the x of the zone's hits (twelve x-sorted buckets, contiguous
//              in the packed arrays) is copied once into shared memory by a
//              TMA bulk copy (cp.async.bulk, completion on an mbarrier); a
//              zone larger than the staging area is read from global memory
//              through the same generic pointer.  Meanwhile the block checks
//              whether every bucket's hits share one z; the uniform case uses
//              per-bucket constants (z, u = (z - z_ref)/1000, f2(u)) instead
//              of per-hit loads.
//   phase A    a warp per track: the windows of all twelve layers (binary
//              searches in the staged buckets), then triplet seeding
//              (Sec. "Triplet Seeding") over the (h0, h2) pairs that can pass
//              the magnet filter, flattened over the lanes, keeping the
//              n_triplets smallest keys; windows and keys go to scratch.
//   phase B    two tracks per warp (16 lanes each, lane = kept triplet) or
//              one: extension, fits and quality (Sec. "Extending triplets to
//              other layers", "Quality Filter"), then the warp-vote
//              selection writes the track's output.
// While a zone is processed, the next event's hits are prefetched into L2
// (cp.async.bulk.prefetch.L2).
//
// Arithmetic: binary32, no contraction (built with -fmad=false), IEEE
// division, every expression in the evaluation order of the method's
// definition, so results equal the per-track kernels' and do not depend on
// the launch shape.
#include <cstdint>

#include "lf.h"
#include "lf_device.cuh"
#include "lf_internal.h"

namespace lfk {

namespace {

constexpr int EV_WARPS = 8;              // warps per block
constexpr int EV_THREADS = EV_WARPS * 32;
constexpr int LIST_CAP = 1024;           // tracks of one zone handled per pass
constexpr int ITEM_CAP = 2 * MAX_CAP;    // (configuration, h0) items of one window set
constexpr int SEG_PAIRS = 2048;          // (h0, h2) pairs per mask segment
constexpr int MASK_WORDS = SEG_PAIRS / 32;
constexpr long long WAIT_LIMIT = 1ll << 24;  // polls of the staging barrier (about a second) before giving up

struct ZoneHead {
    unsigned long long bar;  // mbarrier of the staging copy
    int e, next_e, zone, zb, nz, n_list, next_a, next_b;
    int boff[NL + 1];        // bucket starts relative to zb
    float bz[NL];            // z shared by a bucket's hits (uniform zones)
    float bu[NL], bf[NL];    // u = (z - z_ref)/1000 and f2(u) of those z
    float gu[NL];            // u of the layers' geometry z (expected positions)
    int uni;                 // every bucket of the zone has a single z
    int failed;              // the staging wait ran out
};

// per-warp scratch of phase A (windows, items, pair mask, key buffer); phase
// B reuses the front for its window descriptors
struct WarpA {
    int wb[2][NL];           // window starts relative to zb, per window set
    int wc[2][NL];           // window counts
    int it_start[ITEM_CAP];  // first flattened pair of each non-empty item
    int it_a[ITEM_CAP];      // first h2 (window-local) of the item's interval
    int it_code[ITEM_CAP];   // cfg << 6 | j0
    float it_x0[ITEM_CAP];
    unsigned mask[MASK_WORDS];
    unsigned long long keys[CAND_CAP];
};

struct WarpB {
    int wb[2][2][NL];        // [track of the warp][window set][layer]
    int wc[2][2][NL];
};

__host__ __device__ constexpr size_t align16c(size_t v) { return (v + 15) & ~size_t(15); }
constexpr size_t WARP_BYTES = align16c(sizeof(WarpA) > sizeof(WarpB) ? sizeof(WarpA) : sizeof(WarpB));
constexpr size_t HEAD_BYTES = align16c(sizeof(ZoneHead)) + align16c(LIST_CAP * sizeof(int));

size_t ev_smem_bytes(int stage_cap) {
    return HEAD_BYTES + EV_WARPS * WARP_BYTES + align16c(((size_t)stage_cap + 8) * sizeof(float));
}

// --------------------------------------------------------- TMA + mbarrier

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase `parity` of the barrier: false when it ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}
// global -> shared bulk copy of `bytes` (16-byte aligned addresses, size a
// multiple of 16), completing on bar
__device__ __forceinline__ void tma_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes) {
    // the 16-byte aligned inner part of [p, p + bytes)
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
    const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
    if (e > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
}

// ------------------------------------------------------------- searches

// first index in [lo, hi) whose x is not left of v (see bound_global)
__device__ __forceinline__ int bound_gen(const float* x, int lo, int hi, float v, bool upper) {
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        const float xm = x[mid];
        if (upper ? !(xm > v) : (xm < v)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// closest hit to e among x[0..n) (sorted): smallest |x - e|, ties to the
// lower index (the distance is monotone on each side of the first x >= e)
__device__ __noinline__ int closest_gen(const float* x, int n, float e) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (x[mid] < e) lo = mid + 1; else hi = mid;
    }
    const int j = lo;
    int best = -1;
    float bd = 0.0f;
    if (j > 0) {
        int q = j - 1;
        const float d = fabsf(x[q] - e);
        while (q > 0 && fabsf(x[q - 1] - e) == d) --q;
        best = q;
        bd = d;
    }
    if (j < n) {
        const float d = fabsf(x[j] - e);
        if (best < 0 || d < bd) best = j;
    }
    return best;
}
// the same, inline (pair loop)
__device__ __forceinline__ int closest_inl(const float* x, int n, float e) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (x[mid] < e) lo = mid + 1; else hi = mid;
    }
    const int j = lo;
    int best = -1;
    float bd = 0.0f;
    if (j > 0) {
        int q = j - 1;
        const float d = fabsf(x[q] - e);
        while (q > 0 && fabsf(x[q - 1] - e) == d) --q;
        best = q;
        bd = d;
    }
    if (j < n) {
        const float d = fabsf(x[j] - e);
        if (best < 0 || d < bd) best = j;
    }
    return best;
}

// ------------------------------------------------------------ selection

// Sort the buffered keys; keep the NT smallest at the front of the buffer.
// Returns the new buffer size; thr becomes the NT-th smallest key once the
// buffer holds NT keys (no later key at or above it can be kept).
__device__ __forceinline__ int select_keys(unsigned long long* buf, int nb, int NT, uint64_t& thr, int lane,
                                           uint64_t& mine) {
    uint64_t a = lane < nb ? buf[lane] : NOKEY;
    __syncwarp();
    if (nb <= 32) {
        a = warp_sort32(a, lane);
    } else {
        uint64_t b2 = lane + 32 < nb ? buf[lane + 32] : NOKEY;
        __syncwarp();
        warp_sort64(a, b2, lane);
    }
    const int keep = nb < NT ? nb : NT;
    if (lane < keep) buf[lane] = a;
    mine = lane < keep ? a : NOKEY;
    if (keep == NT) thr = shfl64(a, NT - 1);
    __syncwarp();
    return keep;
}

// ------------------------------------------------------------- phase A

// Windows of window set `side` of a track: lanes 0..11 search the lower
// bounds and lanes 12..23 the upper bounds in the staged buckets, then
// lanes 0..11 apply the cap; the result goes to the warp's descriptors
// (zone-relative) and to scratch (packed indices).
template <bool NOUT>
__device__ __forceinline__ void ev_windows(const KParams& k, const ZoneHead& zh, const float* ex, const TState& s,
                                           int side, WarpA& wa, int* wbeg, uint8_t* wcnt, size_t ws, int lane) {
    const int l = lane < NL ? lane : (lane < 2 * NL ? lane - NL : 0);
    float xmin, xmax, centre;
    window_limits<NOUT>(k, s, l, side, xmin, xmax, centre);
    int v = 0;
    if (lane < 2 * NL) v = bound_gen(ex, zh.boff[l], zh.boff[l + 1], lane < NL ? xmin : xmax, lane >= NL);
    int hi = __shfl_sync(FULL, v, (lane + NL) & 31);
    if (lane < NL) {
        const int lo = v;
        if (hi < lo) hi = lo;
        int cnt = hi - lo, start = lo;
        if (cnt > k.cap) {
            const int c = bound_gen(ex, lo, hi, centre, false);
            start = c - k.cap / 2;
            if (start > hi - k.cap) start = hi - k.cap;
            if (start < lo) start = lo;
            cnt = k.cap;
        }
        wa.wb[side][lane] = start;
        wa.wc[side][lane] = cnt;
        wbeg[ws * NL + lane] = zh.zb + start;
        wcnt[ws * NL + lane] = (uint8_t)cnt;
    }
    __syncwarp();
}

// One window set's triplets merged into the warp's key buffer (nb keys,
// threshold thr, this lane's kept key `mine`).  key = chi2 bits << 32 |
// side << 19 | cfg << 18 | j0 << 12 | j2 << 6 | j1 (window-local indices),
// which orders by (chi2, side, cfg, h0, h2).
template <bool NOUT, bool UNI>
__device__ __forceinline__ void ev_triplets(const KParams& k, const KBatch& b, const ZoneHead& zh, const float* ex,
                                            const TState& s, int side, WarpA& wa, int lane, int& nb, uint64_t& thr,
                                            uint64_t& mine) {
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
    const int* wb = wa.wb[side];
    const int* wc = wa.wc[side];
    const int c0 = wc[0], c3 = wc[3];
    const int n_items = c0 + c3;
    // z of hit j of window layer l
    auto zhit = [&](int l, int j) -> float { return UNI ? zh.bz[l] : __ldg(b.z + zh.zb + wb[l] + j); };

    // items (cfg, j0): the h2 interval of each, compacted to the non-empty
    // ones with their first flattened pair
    int P = 0, n_ne = 0;
    for (int base = 0; base < n_items; base += 32) {
        const int i = base + lane;
        int n = 0, a = 0, code = 0;
        float x0 = 0.0f;
        if (i < n_items) {
            const int cfg = i < c0 ? 0 : 1;
            const int j0 = cfg ? i - c0 : i;
            const int L0 = cfg ? 3 : 0, L2 = cfg ? 11 : 8;
            code = (cfg << 6) | j0;
            x0 = ex[wb[L0] + j0];
            const float z0 = zhit(L0, j0);
            const int n2 = wc[L2];
            n = n2;
            // the interval bound needs one z for the whole h2 window: in a
            // uniform zone always; otherwise every pair is tested
            if (UNI && n2 > 0) {
                const float dzl = zh.bz[L2] - z0;
                if (dzl > 0.0f && z0 > k.z_magnet) {
                    // x2 with |x0 + (x2 - x0) r - x_mag_in| < tol form an interval
                    // (r < 0); bound it with the largest tolerance, then with the
                    // largest the slopes inside allow, below p_bend with the
                    // bending sign; widen by a slack far above the rounding of
                    // the exact tests applied later (bounds only)
                    const float ir = __fdividef(dzl, k.z_magnet - z0);
                    const float slack = 0.5f + 1e-4f * (fabsf(x0) + fabsf(x_mag_in));
                    float lo = x0 + (x_mag_in - x0 + k.magtol_max) * ir - slack;
                    float hi = x0 + (x_mag_in - x0 - k.magtol_max) * ir + slack;
                    const float txm = __fdividef(fmaxf(fabsf(lo - x0), fabsf(hi - x0)), dzl);
                    const float t2 = fminf(fmaxf(tol_base + k.magtol_tx * txm, k.magtol_min), k.magtol_max);
                    lo = x0 + (x_mag_in - x0 + t2) * ir - slack;
                    hi = x0 + (x_mag_in - x0 - t2) * ir + slack;
                    if (f1) {
                        const float xb = x0 + s.txs * dzl;
                        if (bend > 0.0f) lo = fmaxf(lo, xb - slack); else hi = fminf(hi, xb + slack);
                    }
                    const float* x2w = ex + wb[L2];
                    a = bound_gen(x2w, 0, n2, lo, false);
                    const int e2 = bound_gen(x2w, 0, n2, hi, true);
                    n = e2 > a ? e2 - a : 0;
                }
            }
        }
        const int inc = warp_incl_scan(n, lane);
        const unsigned ne = __ballot_sync(FULL, n > 0);
        if (n > 0) {
            const int ci = n_ne + __popc(ne & ((1u << lane) - 1u));
            wa.it_start[ci] = P + inc - n;
            wa.it_a[ci] = a;
            wa.it_code[ci] = code;
            wa.it_x0[ci] = x0;
        }
        P += __shfl_sync(FULL, inc, 31);
        n_ne += __popc(ne);
    }
    __syncwarp();

#pragma unroll 1
    for (int seg = 0; seg < P; seg += SEG_PAIRS) {
        // bit (start - seg) marks the first pair of each item starting here
        for (int w = lane; w < MASK_WORDS; w += 32) wa.mask[w] = 0u;
        __syncwarp();
        int before = 0;  // non-empty items starting before this segment
        for (int c = lane; c < n_ne; c += 32) {
            const int st = wa.it_start[c];
            if (st >= seg && st < seg + SEG_PAIRS) atomicOr(&wa.mask[(st - seg) >> 5], 1u << ((st - seg) & 31));
            before += st < seg ? 1 : 0;
        }
        before = __reduce_add_sync(FULL, before);
        __syncwarp();
        const int np = min(P - seg, SEG_PAIRS);
        int cum = before;
#pragma unroll 1
        for (int base = 0; base < np; base += 32) {
            const unsigned m = wa.mask[base >> 5];
            const int ci = cum + __popc(m & (0xffffffffu >> (31 - lane))) - 1;
            cum += __popc(m);
            const int q = seg + base + lane;
            bool valid = false;
            uint64_t key = NOKEY;
            if (base + lane < np) {
                const int code = wa.it_code[ci];
                const int cfg = code >> 6, j0 = code & 63;
                const int j2 = wa.it_a[ci] + (q - wa.it_start[ci]);
                const int L0 = cfg ? 3 : 0, L1 = cfg ? 7 : 4, L2 = cfg ? 11 : 8;
                const float x0 = wa.it_x0[ci];
                const float z0 = UNI ? (cfg ? zh.bz[3] : zh.bz[0]) : zhit(L0, j0);
                const float x2 = ex[wb[L2] + j2];
                const float z2 = UNI ? (cfg ? zh.bz[11] : zh.bz[8]) : zhit(L2, j2);
                const float tx_d = (x2 - x0) / (z2 - z0);
                bool ok = true;
                if (f1) {
                    const float d = tx_d - s.txs;
                    ok = (bend > 0.0f) ? (d > 0.0f) : (d < 0.0f);
                }
                if (ok) {
                    const float x_mag_d = x0 + tx_d * (k.z_magnet - z0);
                    float tol = tol_base + k.magtol_tx * fabsf(tx_d);
                    tol = fminf(fmaxf(tol, k.magtol_min), k.magtol_max);
                    ok = fabsf(x_mag_d - x_mag_in) < tol;
                }
                if (ok) {
                    const float K = cfg ? k.K_last : k.K_first;
                    const float x1_exp = k.z[L1] * tx_d + (x0 - tx_d * z0) * K;
                    const float* x1w = ex + wb[L1];
                    const int j1 = closest_inl(x1w, wc[L1], x1_exp);
                    if (j1 >= 0) {
                        const float dx = x1w[j1] - x1_exp;
                        const float chi2 = dx * dx;
                        if (chi2 < k.T_triplet) {
                            key = ((uint64_t)__float_as_uint(chi2) << 32) | ((uint64_t)side << 19) |
                                  ((uint64_t)cfg << 18) | ((uint64_t)j0 << 12) | ((uint64_t)j2 << 6) | (uint64_t)j1;
                            valid = key < thr;
                        }
                    }
                }
            }
            unsigned msk = __ballot_sync(FULL, valid);
            if (msk) {
                if (nb + __popc(msk) > CAND_CAP) {
                    nb = select_keys(wa.keys, nb, NT, thr, lane, mine);
                    valid = valid && key < thr;
                    msk = __ballot_sync(FULL, valid);
                }
                if (valid) wa.keys[nb + __popc(msk & ((1u << lane) - 1u))] = key;
                nb += __popc(msk);
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

template <bool NOUT, bool UNI>
__device__ __forceinline__ void ev_phase_a(const KParams& k, const KBatch& b, const ZoneHead& zh, const int* list,
                                           ZoneHead& zw, const float* ex, WarpA& wa, int* wbeg, uint8_t* wcnt,
                                           uint64_t* keys, uint8_t* ntrip, int lane) {
    constexpr int NS = NOUT ? 2 : 1;
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(&zw.next_a, 1);
        i = __shfl_sync(FULL, i, 0);
        if (i >= zh.n_list) break;
        const int t = list[i];
        const TState s = load_state(b, t);
#pragma unroll
        for (int side = 0; side < NS; ++side) ev_windows<NOUT>(k, zh, ex, s, side, wa, wbeg, wcnt, (size_t)t * NS + side, lane);
        int nb = 0, nt = 0;
        uint64_t thr = NOKEY, mine = NOKEY;
        if (k.n_trip > 0) {
#pragma unroll 1
            for (int side = 0; side < NS; ++side) ev_triplets<NOUT, UNI>(k, b, zh, ex, s, side, wa, lane, nb, thr, mine);
            nt = select_keys(wa.keys, nb, k.n_trip, thr, lane, mine);
        }
        if (lane < nt) keys[(size_t)t * k.n_trip + lane] = mine;
        if (lane == 0) ntrip[t] = (uint8_t)nt;
        __syncwarp();
    }
}

// ------------------------------------------------------------- phase B

// Extension and fit of one triplet (Sec. "Extending triplets to other
// layers", "Quality Filter") in the staged zone: x of window hit j of layer
// l is ex[wb[l] + j], its packed index zb + wb[l] + j.
template <bool UNI>
__device__ __forceinline__ void ev_extend_fit(const KParams& k, const KBatch& b, const ZoneHead& zh, const float* ex,
                                              const int* wb, const int* wc, const TState& s, uint64_t key, Cand& cd) {
    const float D = k.D;
    auto hx = [&](int l, int j) -> float { return ex[wb[l] + j]; };
    auto hg = [&](int l, int j) -> int { return zh.zb + wb[l] + j; };
    // u and f2(u) of hit j of layer l (its own z)
    auto hu = [&](int l, int j) -> float { return UNI ? zh.bu[l] : (__ldg(b.z + hg(l, j)) - k.z_ref) * 1e-3f; };
    auto hf = [&](int l, float u) -> float { return UNI ? zh.bf[l] : f2_of(u, D); };
    const int cfg = (int)((key >> 18) & 1);
    const int j0 = (int)((key >> 12) & 63), j2 = (int)((key >> 6) & 63), j1 = (int)(key & 63);
    const int L0 = cfg ? 3 : 0, L1 = cfg ? 7 : 4, L2 = cfg ? 11 : 8;
    int hl[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) hl[l] = (l == L0) ? j0 : (l == L1) ? j1 : (l == L2) ? j2 : -1;
    cd.Q = 0.0f;
    cd.n = 0;

    // three-point solution through the triplet
    const float x0 = hx(L0, j0), x1 = hx(L1, j1), x2 = hx(L2, j2);
    const float u0 = hu(L0, j0), u1 = hu(L1, j1), u2 = hu(L2, j2);
    const float g0 = hf(L0, u0), g1 = hf(L1, u1), g2 = hf(L2, u2);
    const float d1 = u1 - u0, d2 = u2 - u0;
    const float e1 = g1 - g0, e2 = g2 - g0;
    const float r1 = x1 - x0, r2 = x2 - x0;
    const float det = d1 * e2 - d2 * e1;
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
        const float xe = model_x(A, T, C, cfg ? zh.gu[4 * i] : zh.gu[4 * i + 3], D);
        const int j = closest_gen(ex + wb[l], wc[l], xe);
        int jm = -1;
        if (j >= 0) {
            const float dx = hx(l, j) - xe;
            if (dx * dx < k.T_x) jm = j;
        }
        if (cfg) hl[4 * i] = jm; else hl[4 * i + 3] = jm;
    }

    // weighted refit on the x hits, as a correction to the three-point solution
    float S00 = 0.0f, S01 = 0.0f, S02 = 0.0f, S11 = 0.0f, S12 = 0.0f, S22 = 0.0f, b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (!is_x(l) || hl[l] < 0) continue;
        const float u = hu(l, hl[l]);
        const float f = hf(l, u);
        const float r = hx(l, hl[l]) - model_x(A, T, C, u, D);
        const float wt = __ldg(b.w + hg(l, hl[l]));
        const float wu = wt * u, wf = wt * f;
        S00 = S00 + wt; S01 = S01 + wu; S02 = S02 + wf;
        S11 = S11 + wu * u; S12 = S12 + wu * f; S22 = S22 + wf * f;
        b0 = b0 + wt * r; b1 = b1 + wu * r; b2 = b2 + wf * r;
    }
    const float c00 = S11 * S22 - S12 * S12;
    const float c01 = S02 * S12 - S01 * S22;
    const float c02 = S01 * S12 - S02 * S11;
    const float c11 = S00 * S22 - S02 * S02;
    const float c12 = S01 * S02 - S00 * S12;
    const float c22 = S00 * S11 - S01 * S01;
    const float dt = (S00 * c00 + S01 * c01) + S02 * c02;
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
        const float yl = s.ys + s.tys * (k.z[l] - k.z_state);
        const float xe = model_x(A, T, C, zh.gu[l], D) - yl * k.dxdy[l];
        const int j = closest_gen(ex + wb[l], wc[l], xe);
        if (j < 0) continue;
        const float dx = hx(l, j) - xe;
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
    const int n = n_x + n_uv;
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
        const int g = hg(l, hl[l]);
        const float u = hu(l, hl[l]);
        const float dd = __ldg(b.dxdy + g);
        dv[l] = dd;
        const float y = (model_x(A, T, C, u, D) - hx(l, hl[l])) / dd;
        yv[l] = y;
        const float wt = __ldg(b.w + g);
        const float wu = wt * u;
        Y0s = Y0s + wt; Y1s = Y1s + wu; Y2s = Y2s + wu * u;
        yb0 = yb0 + wt * y; yb1 = yb1 + wu * y;
    }
    const float ydet = Y0s * Y2s - Y1s * Y1s;
    if (!(ydet != 0.0f)) {
        cd.status = 1;
        return;
    }
    const float Y0 = (Y2s * yb0 - Y1s * yb1) / ydet;
    const float TY = (Y0s * yb1 - Y1s * yb0) / ydet;
    const float ty_fit = TY * 1e-3f;
    if (!(fabsf(ty_fit - s.tys) < k.T_ty)) {
        cd.status = 4;
        return;
    }

    // quality factor
    float qx = 0.0f, qy = 0.0f;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        if (hl[l] < 0) continue;
        const float u = hu(l, hl[l]);
        const float xf = model_x(A, T, C, u, D);
        if (is_x(l)) {
            const float r = hx(l, hl[l]) - xf;
            // T_x a power of two: the product by its reciprocal is the quotient
            qx = qx + (k.inv_T_x != 0.0f ? (r * r) * k.inv_T_x : div_call(r * r, k.T_x));
        } else {
            const float yf = Y0 + TY * u;
            const float r = hx(l, hl[l]) - (xf - yf * dv[l]);
            qx = qx + div_call(r * r, T_uv);
            const float ry = yv[l] - yf;
            qy = qy + div_call(ry * ry, k.T_y);
        }
    }
    const float Cn = n == 9 ? k.C_n[0] : n == 10 ? k.C_n[1] : n == 11 ? k.C_n[2] : k.C_n[3];
    const float Q = (qx / (float)(n - 3) + qy / (float)(n_uv - 2)) * Cn;
    cd.Q = Q;
    if (!(Q < k.T_Q)) {
        cd.status = 5;
        return;
    }
    cd.status = 0;
    const float tx = T * 1e-3f;
    cd.st[0] = A;
    cd.st[1] = Y0;
    cd.st[2] = tx;
    cd.st[3] = ty_fit;
    cd.st[4] = C * 1e-6f;
    cd.st[5] = (tx - s.txs) / k.pk;
}

template <bool NOUT, int TPW, bool UNI>
__device__ __forceinline__ void ev_phase_b(const KParams& k, const KBatch& b, const KOut& o, const ZoneHead& zh,
                                           const int* list, ZoneHead& zw, const float* ex, WarpB& wbk,
                                           const int* wbeg, const uint8_t* wcnt, const uint64_t* keys,
                                           const uint8_t* ntrip, int lane) {
    // (windows, keys and counts were written by this kernel's phase A: plain
    // coherent loads, no read-only path)
    constexpr int NS = NOUT ? 2 : 1;
    constexpr int G = 32 / TPW;
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(&zw.next_b, TPW);
        i = __shfl_sync(FULL, i, 0);
        if (i >= zh.n_list) break;
        // window descriptors of the warp's tracks: lane (q, side, l) for
        // q < TPW, side < NS, l < 12 (at most 24 lanes)
        {
            const int q = lane / (NS * NL), rem = lane % (NS * NL), sd = rem / NL, l = rem % NL;
            if (q < TPW && i + q < zh.n_list) {
                const int t = list[i + q];
                const size_t w = ((size_t)t * NS + sd) * NL + l;
                wbk.wb[q][sd][l] = wbeg[w] - zh.zb;
                wbk.wc[q][sd][l] = wcnt[w];
            }
        }
        __syncwarp();
        const int q = lane / G, r = lane % G;
        const bool live = i + q < zh.n_list;
        const int t = live ? list[i + q] : 0;
        const bool act = live && r < ntrip[t];
        const uint64_t key = act ? keys[(size_t)t * k.n_trip + r] : NOKEY;
        const int side = NOUT ? (int)((key >> 19) & 1) : 0;
        Cand cd;
        cd.status = 9;
        cd.Q = 0.0f;
        cd.n = 0;
#pragma unroll
        for (int p = 0; p < 6; ++p) cd.st[p] = 0.0f;
#pragma unroll
        for (int l = 0; l < NL; ++l) cd.hl[l] = -1;
        TState s = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (act) {
            s = load_state(b, t);
            ev_extend_fit<UNI>(k, b, zh, ex, wbk.wb[q][side], wbk.wc[q][side], s, key, cd);
        }
        int hgl[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l)
            hgl[l] = (act && cd.status == 0 && cd.hl[l] >= 0) ? zh.zb + wbk.wb[q][side][l] + cd.hl[l] : -1;
        group_select_write<G>(o, t, live, r, act && cd.status == 0, cd.Q, cd.n, hgl, cd.st);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- kernel

template <bool NOUT, int TPW>
__global__ void __launch_bounds__(EV_THREADS, 3)
    k_event(KParams k, KBatch b, KOut o, int* wbeg, uint8_t* wcnt, uint64_t* keys, uint8_t* ntrip, int* cursor,
            int* status, int stage_cap) {
    extern __shared__ __align__(16) char smem[];
    ZoneHead& zh = *reinterpret_cast<ZoneHead*>(smem);
    int* list = reinterpret_cast<int*>(smem + align16c(sizeof(ZoneHead)));
    char* warp_area = smem + HEAD_BYTES;
    float* sbuf = reinterpret_cast<float*>(warp_area + EV_WARPS * WARP_BYTES);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    WarpA& wa = *reinterpret_cast<WarpA*>(warp_area + warp * WARP_BYTES);
    WarpB& wbk = *reinterpret_cast<WarpB*>(warp_area + warp * WARP_BYTES);

    if (tid == 0) {
        mbar_init(&zh.bar);
        zh.next_e = atomicAdd(cursor, 1);
        zh.failed = 0;
    }
    if (tid < NL) zh.gu[tid] = (k.z[tid] - k.z_ref) * 1e-3f;
    unsigned phase = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            zh.e = zh.next_e;
            zh.next_e = zh.e < b.n_events ? atomicAdd(cursor, 1) : b.n_events;
        }
        __syncthreads();
        const int e = zh.e;
        if (e >= b.n_events || zh.failed) break;
        const int t0 = __ldg(b.trk_offsets + e), t1 = __ldg(b.trk_offsets + e + 1);
        if (tid == 0 && zh.next_e < b.n_events) {
            // the next event's hits go to L2 while this one is followed
            const int h0 = __ldg(b.hit_offsets + (size_t)zh.next_e * NB), h1 = __ldg(b.hit_offsets + (size_t)zh.next_e * NB + NB);
            if (h1 > h0) {
                l2_prefetch(b.x + h0, (size_t)(h1 - h0) * 4);
                l2_prefetch(b.z + h0, (size_t)(h1 - h0) * 4);
            }
        }
        if (t1 <= t0) continue;
        for (int zone = 0; zone < 2; ++zone) {
            bool staged = false;
            const float* ex = nullptr;
            for (int c0 = t0; c0 < t1; c0 += LIST_CAP) {
                // the chunk's tracks of this zone (the barrier first: every
                // thread is done reading the head of the previous pass)
                __syncthreads();
                if (tid == 0) {
                    zh.n_list = 0;
                    zh.next_a = 0;
                    zh.next_b = 0;
                }
                __syncthreads();
                const int c1 = min(c0 + LIST_CAP, t1);
                for (int base = c0; base < c1; base += EV_THREADS) {
                    const int t = base + tid;
                    const bool in = t < c1 && ((__ldg(b.sty + t) >= 0.0f) ? 1 : 0) == zone;
                    const unsigned m = __ballot_sync(FULL, in);
                    int pos = 0;
                    if (lane == 0 && m) pos = atomicAdd(&zh.n_list, __popc(m));
                    pos = __shfl_sync(FULL, pos, 0);
                    if (in) list[pos + __popc(m & ((1u << lane) - 1u))] = t;
                }
                __syncthreads();
                if (zh.n_list == 0) continue;   // (read by all threads before the next reset's barrier)
                if (!staged) {
                    // ---- stage the zone
                    const size_t bo = (size_t)e * NB + zone * NL;
                    if (tid <= NL) zh.boff[tid] = __ldg(b.hit_offsets + bo + tid);
                    __syncthreads();
                    const int zb = zh.boff[0], nz = zh.boff[NL] - zb;
                    __syncthreads();
                    if (tid <= NL) zh.boff[tid] -= zb;
                    if (tid == 0) {
                        zh.zb = zb;
                        zh.nz = nz;
                        zh.uni = 1;
                    }
                    const bool in_smem = nz <= stage_cap;
                    // head: floats before the first 16-byte aligned address
                    const int head = min(nz, (int)(((16u - (unsigned)(reinterpret_cast<uintptr_t>(b.x + zb) & 15u)) & 15u) >> 2));
                    const int mid = (nz - head) & ~3;
                    float* exs = sbuf + (head ? 4 - head : 0);
                    if (in_smem) {
                        if (tid == 0 && mid > 0) {
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            mbar_expect(&zh.bar, (unsigned)mid * 4u);
                            tma_load(exs + head, b.x + zb + head, (unsigned)mid * 4u, &zh.bar);
                        }
                        if (tid < head) exs[tid] = __ldg(b.x + zb + tid);
                        const int tl = nz - head - mid;
                        if (tid < tl) exs[head + mid + tid] = __ldg(b.x + zb + head + mid + tid);
                    }
                    __syncthreads();   // boff relative, zb, head/tail copies
                    // z of each bucket, and whether all its hits share it
                    int uni = 1;
                    for (int l = 0; l < NL; ++l) {
                        const int s0 = zh.boff[l], s1 = zh.boff[l + 1];
                        if (s1 <= s0) continue;
                        const float z0 = __ldg(b.z + zb + s0);
                        for (int j = s0 + tid; j < s1; j += EV_THREADS) uni &= (__ldg(b.z + zb + j) == z0) ? 1 : 0;
                        if (tid == 0) zh.bz[l] = z0;
                    }
                    uni = __syncthreads_and(uni);
                    if (tid < NL) {
                        const float u = (zh.bz[tid] - k.z_ref) * 1e-3f;
                        zh.bu[tid] = u;
                        zh.bf[tid] = f2_of(u, k.D);
                    }
                    if (tid == 0) zh.uni = uni;
                    if (in_smem && mid > 0) {
                        if (!mbar_wait(&zh.bar, phase)) {
                            // the copy did not complete: record it, wait once
                            // more for it (bounded), and stop this block
                            atomicOr(status, LF_FLAG_TIMEOUT);
                            zh.failed = 1;
                            mbar_wait(&zh.bar, phase);
                        }
                        phase ^= 1u;
                    }
                    __syncthreads();
                    if (zh.failed) break;
                    staged = true;
                    ex = in_smem ? exs : b.x + zb;
                }
                // ---- phase A: windows and triplets, a warp per track
                if (zh.uni) ev_phase_a<NOUT, true>(k, b, zh, list, zh, ex, wa, wbeg, wcnt, keys, ntrip, lane);
                else ev_phase_a<NOUT, false>(k, b, zh, list, zh, ex, wa, wbeg, wcnt, keys, ntrip, lane);
                __syncthreads();
                // ---- phase B: extension, fit, selection
                if (zh.uni) ev_phase_b<NOUT, TPW, true>(k, b, o, zh, list, zh, ex, wbk, wbeg, wcnt, keys, ntrip, lane);
                else ev_phase_b<NOUT, TPW, false>(k, b, o, zh, list, zh, ex, wbk, wbeg, wcnt, keys, ntrip, lane);
                __syncthreads();
            }
            if (zh.failed) break;
        }
    }
}

template <bool NOUT, int TPW>
cudaError_t launch_event_t(const KParams& k, const KBatch& b, const KOut& o, int* wbeg, uint8_t* wcnt, uint64_t* keys,
                           uint8_t* ntrip, int* cursor, int* status, int stage_cap, int blocks, cudaStream_t s) {
    const size_t sm = ev_smem_bytes(stage_cap);
    cudaError_t err = cudaFuncSetAttribute(k_event<NOUT, TPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    k_event<NOUT, TPW><<<blocks, EV_THREADS, sm, s>>>(k, b, o, wbeg, wcnt, keys, ntrip, cursor, status, stage_cap);
    return cudaGetLastError();
}

const void* event_fn(const KParams& k) {
    if (k.no_ut) return (const void*)k_event<true, 1>;
    return k.n_trip <= 16 ? (const void*)k_event<false, 2> : (const void*)k_event<false, 1>;
}

}  // namespace

int event_stage_cap_default(int blocks_per_sm) {
    // shared memory of an SM (228 KB, 1 KB reserved per block) shared by the
    // resident blocks; the rest of a block's share after its head and warp
    // scratch holds staged x
    const int bps = blocks_per_sm > 0 ? blocks_per_sm : 3;
    const long per_block = (228l * 1024) / bps - 1024;
    const long rest = per_block - (long)(HEAD_BYTES + EV_WARPS * WARP_BYTES) - 64;
    return rest > 0 ? (int)(rest / 4) : 0;
}

cudaError_t event_max_blocks_per_sm(const KParams& k, int stage_cap, int* out) {
    const void* fn = event_fn(k);
    const size_t sm = ev_smem_bytes(stage_cap);
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, EV_THREADS, sm);
}

cudaError_t launch_event(const KParams& k, const KBatch& b, const KOut& o, int* wbeg, uint8_t* wcnt, uint64_t* keys,
                         uint8_t* ntrip, int* cursor, int* status, int stage_cap, int blocks, cudaStream_t s) {
    if (b.n_events <= 0 || b.n_tracks <= 0) return cudaSuccess;
    if (k.no_ut) return launch_event_t<true, 1>(k, b, o, wbeg, wcnt, keys, ntrip, cursor, status, stage_cap, blocks, s);
    if (k.n_trip <= 16)
        return launch_event_t<false, 2>(k, b, o, wbeg, wcnt, keys, ntrip, cursor, status, stage_cap, blocks, s);
    return launch_event_t<false, 1>(k, b, o, wbeg, wcnt, keys, ntrip, cursor, status, stage_cap, blocks, s);
}

}  // namespace lfk
