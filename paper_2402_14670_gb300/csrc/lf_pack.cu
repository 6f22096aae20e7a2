// Hit packing for sm_103a: per event, bucket the raw hits by (zone, layer),
// sort every bucket by x (ties by raw index) and write the SoA.
//
// One persistent kernel, k_pack_event: a block of 1024 threads takes one
// event at a time from a device work queue and sorts it as a distribution
// sort whose bins are ordered like the result:
//   range    the x range of a strided sample of at most 1024 of the event's
//            hits, widened by 1/128 of it on each side (a hit outside it
//            lands in an edge bin);
//   bins     every bucket gets nbb equal x bins over that range (nbb a power
//            of two between 16 and 512, about one hit per bin); the global
//            bin of a hit is bucket * nbb + bin, a monotone function of
//            (bucket, x), so bin order is already the bucket order and the x
//            order up to the inside of a bin;
//   count    one pass over (plane, x) counts the hits per bin (shared
//            atomics); an exclusive scan gives every bin's start, and the
//            bucket offsets are the starts of each bucket's first bin;
//   place    one pass over the raw hits puts each at its bin's next free
//            position;
//   order    each bin is ordered by (x, raw index) with an insertion sort, so
//            the result is the exact (bucket, x, raw index) order whatever
//            the data (a skewed x distribution costs time, never exactness);
//   write    x, layer and perm leave coalesced (and, when asked for, every
//            32nd x into the coarse index of the window searches).
// An event of at most CHUNK_N hits is placed straight into shared memory as
// (x, 16-bit raw index), 6 bytes per hit; its z, dxdy and w are then copied
// from the raw arrays (prefetched into L2 when the event was taken) into
// shared memory with cp.async, one array at a time, and written in sorted
// order, gathered by raw index.  A larger event is sorted in chunks of consecutive
// bins: per chunk a pass over the raw hits places the chunk's hits in shared
// memory, and after the ordering a second pass reads the payload coalesced and
// stores each of the chunk's hits' z, dxdy and w at its position inside its
// bin.  (Staging a larger event once through its output range instead costs
// five scattered 4-byte stores per hit, which measured slower than the
// repeated coalesced passes.)  An event above 65535 hits uses 32-bit bins and
// indices.  The layer of an output position is the bucket whose offsets
// contain it.
// While an event is processed, the block has already taken its next event
// from the queue and prefetched that event's plane codes and x into L2.
// A bucket above LF_MAX_BUCKET hits is not sorted: it is flagged (status bit
// 0x1), its perm entries are set to -1 and its other outputs to 0; a plane
// code >= 24 is flagged (0x2) and counted in the last bucket.
#include <cstdint>
#include <type_traits>

#include "lf.h"
#include "lf_internal.h"

namespace lfk {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PACK_THREADS = 1024;
constexpr int PACK_WARPS = PACK_THREADS / 32;
constexpr int NBB_MIN = 16;                 // x bins per bucket, fewest
constexpr int NBB_MAX = 512;                // x bins per bucket, most
constexpr int NBIN_MAX = NB * NBB_MAX;      // bins of an event, most
constexpr int UNROLL = 4;                   // hits per thread with loads in flight together
constexpr uint32_t ID_MASK = (1u << 27) - 1u;  // largest event (hits) the pack sorts
constexpr int RANGE_SAMPLE = 1024;          // hits sampled for the event's x range

// Shared memory: the bin counters / starts (nbin + 1 of them), then x and the
// raw index (inside the event) of a chunk's hits in bin order.  An event of at
// most 65535 hits keeps 16-bit bins and 16-bit raw indices (6 B per hit),
// which leaves room to sort CHUNK_N hits at once; a larger event keeps 32-bit
// bins and indices and chunks of CHUNK_W hits.  Either layout fits AREA_BYTES.
constexpr size_t BINS16_BYTES = 2 * (size_t)(NBIN_MAX + 8);
constexpr size_t BINS32_BYTES = 4 * (size_t)(NBIN_MAX + 4);
constexpr int CHUNK_N = 34432;
constexpr int CHUNK_W = 22752;
constexpr size_t AREA_BYTES = BINS16_BYTES + (size_t)CHUNK_N * 6;
static_assert(BINS32_BYTES + (size_t)CHUNK_W * 8 <= AREA_BYTES, "wide layout fits");
static_assert(CHUNK_W >= BLOCK_SORT_MAX, "a sortable bucket must fit one chunk");
static_assert(CHUNK_N <= 65535, "positions and raw indices of a narrow event fit 16 bits");
static_assert((CHUNK_N * 4) % 16 == 0, "the index area stays aligned");

struct EvShared {
    unsigned red_mn[PACK_WARPS], red_mx[PACK_WARPS];
    int warp_tot[PACK_WARPS];
    int boff[NB + 1];        // bucket offsets inside the event
    int event, next;
    unsigned flagged;        // buckets above LF_MAX_BUCKET
    int b1;                  // end bin of the current chunk
    int n_big;               // bins above SMALL_BIN hits in the current pass
    int big[64];             // their indices (BIG_BINS)
};

// x as an unsigned integer with the same order (-0 already turned into +0)
__device__ __forceinline__ unsigned ordered(float x) {
    unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// x bin inside a bucket: monotone non-decreasing in x
__device__ __forceinline__ int bin_of(float x, float lo, float scale, int nbb) {
    float f = (x - lo) * scale;
    if (!(f > 0.0f)) return 0;
    if (!(f < (float)nbb)) return nbb - 1;
    return (int)f;
}

__device__ __forceinline__ int wscan_incl(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// L2 prefetch of bytes [p, p + bytes): one instruction per 128-byte line,
// each line holding at least one byte of the range
__device__ __forceinline__ void prefetch_range(const void* p, size_t bytes, int tid) {
    if (bytes == 0) return;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(127);
    const uintptr_t b1 = reinterpret_cast<uintptr_t>(p) + bytes - 1;
    const int lines = (int)((b1 - b0) / 128) + 1;
    for (int q = tid; q < lines; q += PACK_THREADS)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(b0 + (uintptr_t)q * 128));
}

// plane code of a raw hit as a bucket (codes >= 24 go to the last bucket)
__device__ __forceinline__ int bucket_code(int p, bool& bad) {
    if (p >= NB) {
        bad = true;
        return NB - 1;
    }
    return p;
}

// bins above this population are sorted by the whole block (bitonic), the
// others by one thread each (insertion sort), so that a skewed x distribution
// (many hits at one x) costs O(n log^2 n), not O(n^2)
constexpr int SMALL_BIN = 32;
constexpr int BIG_BINS = 64;   // big bins of one sorting pass recorded (more: another pass)

// insertion sort of the bin [s, e) by (x, raw index) (the hits of one bin
// share their bucket)
template <typename K>
__device__ __forceinline__ void sort_bin(float* xs, K* ks, int s, int e) {
    for (int i = s + 1; i < e; ++i) {
        const float xv = xs[i];
        const K kv = ks[i];
        int j = i - 1;
        while (j >= s) {
            const float xj = xs[j];
            const K kj = ks[j];
            if (!(xv < xj || (xv == xj && kv < kj))) break;
            xs[j + 1] = xj;
            ks[j + 1] = kj;
            --j;
        }
        xs[j + 1] = xv;
        ks[j + 1] = kv;
    }
}

// Bin counters of one event: 16-bit halves of 32-bit words (WIDE = false) or
// 32-bit words; the halves never carry into each other because no count or
// start of a narrow event exceeds 65535.
template <bool WIDE>
struct Bins {
    char* base;
    __device__ __forceinline__ int get(int b) const {
        return WIDE ? reinterpret_cast<const int*>(base)[b] : (int)reinterpret_cast<const uint16_t*>(base)[b];
    }
    __device__ __forceinline__ void set(int b, int v) const {
        if (WIDE) reinterpret_cast<int*>(base)[b] = v;
        else reinterpret_cast<uint16_t*>(base)[b] = (uint16_t)v;
    }
    // old value, then +1
    __device__ __forceinline__ int add(int b) const {
        if (WIDE) return atomicAdd(reinterpret_cast<int*>(base) + b, 1);
        const unsigned old = atomicAdd(reinterpret_cast<unsigned*>(base) + (b >> 1), (b & 1) ? 0x10000u : 1u);
        return (b & 1) ? (int)(old >> 16) : (int)(old & 0xffffu);
    }
    __device__ __forceinline__ void clear(int nbin, int tid) const {
        if (WIDE) {
            for (int b = tid; b <= nbin; b += PACK_THREADS) set(b, 0);
        } else {
            for (int b = tid; b <= nbin / 2; b += PACK_THREADS) reinterpret_cast<unsigned*>(base)[b] = 0u;
        }
    }
};

// Block-wide sort of [s, e) by (x, raw index): the bitonic network on the
// next power of two, positions at or beyond e standing for +infinity, in
// its form that compares every pair towards the lower index (so padded
// positions never move).  All PACK_THREADS threads call it.
template <typename K>
__device__ __forceinline__ void sort_range_block(float* xs, K* ks, int s, int e, int tid) {
    const int n = e - s;
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int kk = 2; kk <= p2; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < p2; i += PACK_THREADS) {
                // the partner: mirrored inside the kk-block on its first step
                const int pi = (j == (kk >> 1)) ? (i ^ (kk - 1)) : (i ^ j);
                if (pi > i && pi < n) {
                    const float xa = xs[s + i], xb = xs[s + pi];
                    const K ka = ks[s + i], kb = ks[s + pi];
                    if (xb < xa || (xb == xa && kb < ka)) {
                        xs[s + i] = xb;
                        ks[s + i] = kb;
                        xs[s + pi] = xa;
                        ks[s + pi] = ka;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Order every bin of [b0, b1) (starts at pos(b - 1), ends at pos(b), both
// relative to `base`): small bins by their thread, big ones by the block.
template <bool WIDE, typename K>
__device__ __forceinline__ void sort_bins(const Bins<WIDE>& bins, float* xs, K* ks, int b0, int b1, int base,
                                          EvShared& sh, int tid) {
    // (sh.n_big was cleared before the barrier that precedes this call)
    for (int b = b0 + tid; b < b1; b += PACK_THREADS) {
        const int s0 = (b == b0 ? base : bins.get(b - 1)) - base, s1 = bins.get(b) - base;
        if (s1 - s0 <= SMALL_BIN) {
            sort_bin(xs, ks, s0, s1);
        } else {
            const int q = atomicAdd(&sh.n_big, 1);
            if (q < BIG_BINS) sh.big[q] = b;
        }
    }
    __syncthreads();
    const int nbig = sh.n_big;
    if (nbig == 0) return;
    if (nbig <= BIG_BINS) {
        for (int q = 0; q < nbig; ++q) {
            const int b = sh.big[q];
            const int s0 = (b == b0 ? base : bins.get(b - 1)) - base, s1 = bins.get(b) - base;
            sort_range_block(xs, ks, s0, s1, tid);
        }
    } else {
        // more big bins than the record holds: visit every bin in order
        for (int b = b0; b < b1; ++b) {
            const int s0 = (b == b0 ? base : bins.get(b - 1)) - base, s1 = bins.get(b) - base;
            if (s1 - s0 > SMALL_BIN) sort_range_block(xs, ks, s0, s1, tid);
        }
    }
    __syncthreads();
}

// bucket of event position j: the last q with boff[q] <= j (an empty bucket
// shares its offset with the next one)
__device__ __forceinline__ int bucket_at(const int* boff, int j) {
    int lo = 0, hi = NB - 1;
#pragma unroll
    for (int it = 0; it < 5; ++it) {   // 2^5 >= 24 buckets
        const int mid = (lo + hi + 1) >> 1;
        if (lo < hi) {
            if (boff[mid] <= j) lo = mid; else hi = mid - 1;
        }
    }
    return lo;
}

struct PackIO {
    const float* __restrict__ x;
    const float* __restrict__ z;
    const float* __restrict__ dxdy;
    const float* __restrict__ w;
    const uint8_t* __restrict__ plane;
    int* hit_offsets;
    float *ox, *oz, *od, *ow;
    uint8_t* ol;
    int* perm;
    int* status;
    float* oc;   // coarse index: oc[p / 32] = x of output position p, p a multiple of 32 (or nullptr)
};

// Sort one event of n >= 1 hits starting at raw index rb (event e).
template <bool WIDE>
__device__ __forceinline__ void sort_event(const PackIO& io, EvShared& sh, char* smem, int e, int rb, int n,
                                           int tid, int lane, int warp) {
    using K = typename std::conditional<WIDE, uint32_t, uint16_t>::type;
    const Bins<WIDE> bins{smem};
    constexpr int chunk = WIDE ? CHUNK_W : CHUNK_N;
    float* xs = reinterpret_cast<float*>(smem + (WIDE ? BINS32_BYTES : BINS16_BYTES));
    K* ks = reinterpret_cast<K*>(xs + chunk);
    const float* __restrict__ x = io.x;
    const uint8_t* __restrict__ plane = io.plane;

    // x range of the event from a strided sample, widened by 1/128 of it on
    // each side: it only shapes the bins (a hit outside it lands in an edge
    // bin, which the ordering inside bins absorbs)
    unsigned mn = 0xffffffffu, mx = 0u;
    {
        const int ns = n < RANGE_SAMPLE ? n : RANGE_SAMPLE;
        const int stride = n / ns;
        if (tid < ns) {
            const unsigned ov = ordered(x[rb + tid * stride] + 0.0f);
            mn = ov;
            mx = ov;
        }
    }
    mn = __reduce_min_sync(FULL, mn);
    mx = __reduce_max_sync(FULL, mx);
    if (lane == 0) {
        sh.red_mn[warp] = mn;
        sh.red_mx[warp] = mx;
    }
    // bins per bucket: a power of two near n / 24
    int nbb = NBB_MIN;
    while (nbb < NBB_MAX && nbb * NB < n) nbb <<= 1;
    const int nbin = nbb * NB;
    bins.clear(nbin, tid);
    __syncthreads();
    mn = sh.red_mn[lane];
    mx = sh.red_mx[lane];
    mn = __reduce_min_sync(FULL, mn);
    mx = __reduce_max_sync(FULL, mx);
    float lo, scale;
    {
        const float slo = unordered(mn), shi = unordered(mx);
        const float pad = (shi - slo) * (1.0f / 128.0f);
        lo = slo - pad;
        const float hi = shi + pad;
        scale = hi > lo ? (float)nbb / (hi - lo) : 0.0f;
    }

    // count per bin
    bool bad = false;
    for (int base = 0; base < n; base += PACK_THREADS * UNROLL) {
        int pu[UNROLL];
        float xu[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int i = base + u * PACK_THREADS + tid;
            pu[u] = -1;
            xu[u] = 0.0f;
            if (i < n) {
                pu[u] = plane[rb + i];
                xu[u] = x[rb + i];
            }
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            if (pu[u] < 0) continue;
            const int q = bucket_code(pu[u], bad);
            bins.add(q * nbb + bin_of(xu[u] + 0.0f, lo, scale, nbb));
        }
    }
    if (bad) atomicOr(io.status, LF_FLAG_PLANE_RANGE);
    __syncthreads();

    // exclusive scan of the nbin counters: thread tid owns a run of per (an
    // even number, so a 16-bit pair has a single owner)
    {
        const int per = 2 * ((nbin + 2 * PACK_THREADS - 1) / (2 * PACK_THREADS));
        const int s0 = min(tid * per, nbin), s1 = min(s0 + per, nbin);
        int sum = 0;
        for (int b = s0; b < s1; ++b) sum += bins.get(b);
        const int inc = wscan_incl(sum, lane);
        if (lane == 31) sh.warp_tot[warp] = inc;
        __syncthreads();
        int wt = sh.warp_tot[lane];
        const int winc = wscan_incl(wt, lane);
        int excl = inc - sum + __shfl_sync(FULL, winc - wt, warp);
        for (int b = s0; b < s1; ++b) {
            const int c = bins.get(b);
            bins.set(b, excl);
            excl += c;
        }
        if (tid == 0) bins.set(nbin, n);
    }
    __syncthreads();
    if (tid <= NB) {
        const int s = bins.get(tid * nbb);
        sh.boff[tid] = s;
        if (tid < NB) {
            io.hit_offsets[(size_t)e * NB + tid] = rb + s;
            if (bins.get((tid + 1) * nbb) - s > BLOCK_SORT_MAX) {
                atomicOr(&sh.flagged, 1u << tid);
                atomicOr(io.status, LF_FLAG_BUCKET_OVERFLOW);
            }
        }
    }
    __syncthreads();

    const unsigned flagged = sh.flagged;
    if (n <= chunk && flagged == 0u) {
        // ---- the whole event in one piece: placed straight into shared memory
        for (int ib = 0; ib < n; ib += PACK_THREADS * UNROLL) {
            int pu[UNROLL];
            float xu[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int i = ib + u * PACK_THREADS + tid;
                pu[u] = -1;
                xu[u] = 0.0f;
                if (i < n) {
                    pu[u] = plane[rb + i];
                    xu[u] = x[rb + i];
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if (pu[u] < 0) continue;
                const int i = ib + u * PACK_THREADS + tid;
                bool bb = false;
                const int q = bucket_code(pu[u], bb);
                const float xv = xu[u] + 0.0f;
                const int pos = bins.add(q * nbb + bin_of(xv, lo, scale, nbb));
                xs[pos] = xv;
                ks[pos] = (K)i;
            }
        }
        __syncthreads();
        // bins[b] now holds the end of bin b; order each bin by (x, raw index)
        sort_bins(bins, xs, ks, 0, nbin, 0, sh, tid);
        // x, layer and perm straight from shared memory
        const size_t o0 = (size_t)rb;
        int qb = 0;   // bucket of position j (j only grows: the last q with boff[q] <= j)
        for (int j = tid; j < n; j += PACK_THREADS) {
            while (qb + 1 < NB && sh.boff[qb + 1] <= j) ++qb;
            io.ox[o0 + j] = xs[j];
            if (io.oc && ((o0 + j) & 31) == 0) io.oc[(o0 + j) >> 5] = xs[j];
            io.ol[o0 + j] = (uint8_t)(qb % NL);
            io.perm[o0 + j] = rb + (int)ks[j];
        }
        __syncthreads();
        // z, dxdy and w: each raw array is copied into shared memory (x's
        // area) with asynchronous 4-byte copies, all of them in flight at
        // once, and written in sorted order, gathered by raw index
        float* tmp = xs;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float* __restrict__ src = a == 0 ? io.z : (a == 1 ? io.dxdy : io.w);
            float* dst = a == 0 ? io.oz : (a == 1 ? io.od : io.ow);
            for (int i = tid; i < n; i += PACK_THREADS) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(tmp + i);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(src + rb + i) : "memory");
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
            for (int j = tid; j < n; j += PACK_THREADS) dst[o0 + j] = tmp[ks[j]];
            __syncthreads();
        }
        return;
    }

    // ---- a larger event (or one with a flagged bucket): chunks of consecutive
    // bins of at most `chunk` hits; per chunk one pass over the raw hits places
    // the chunk's hits in shared memory, and after the ordering and the x,
    // layer and perm writes, a second pass reads the payload coalesced and
    // stores each of the chunk's hits' z, dxdy and w at its position
    int b0 = 0;
    while (b0 < nbin) {
        const int q0 = b0 / nbb;
        if ((flagged >> q0) & 1u) {   // b0 is the bucket's first bin
            const int o0 = sh.boff[q0], o1 = sh.boff[q0 + 1];
            for (int j = o0 + tid; j < o1; j += PACK_THREADS) {
                const size_t o = (size_t)rb + j;
                io.perm[o] = -1;
                io.ox[o] = 0.0f;
                if (io.oc && (o & 31) == 0) io.oc[o >> 5] = 0.0f;
                io.oz[o] = 0.0f;
                io.od[o] = 0.0f;
                io.ow[o] = 0.0f;
                io.ol[o] = (uint8_t)(q0 % NL);
            }
            b0 = (q0 + 1) * nbb;
            continue;
        }
        const int base = bins.get(b0);
        if (tid == 0) {
            // the chunk stops before the next flagged bucket
            int limit = nbin;
            const unsigned later = flagged & ~((2u << q0) - 1u);
            if (later) limit = (__ffs(later) - 1) * nbb;
            // largest b1 in (b0, limit] with bins[b1] - base <= chunk (bins past
            // b0 still hold their starts, monotone in b; a single bin of an
            // unflagged bucket always fits)
            int l = b0 + 1, h = limit;
            while (l < h) {
                const int m = (l + h + 1) >> 1;
                if (bins.get(m) - base <= chunk) l = m; else h = m - 1;
            }
            sh.b1 = l;
            sh.n_big = 0;
        }
        __syncthreads();
        const int b1 = sh.b1;
        const int tot = bins.get(b1) - base;
        __syncthreads();   // every thread has read bins[b0], bins[b1]
        for (int ib = 0; ib < n; ib += PACK_THREADS * UNROLL) {
            int pu[UNROLL];
            float xu[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int i = ib + u * PACK_THREADS + tid;
                pu[u] = -1;
                xu[u] = 0.0f;
                if (i < n) {
                    pu[u] = plane[rb + i];
                    xu[u] = x[rb + i];
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if (pu[u] < 0) continue;
                const int i = ib + u * PACK_THREADS + tid;
                bool bb = false;
                const int q = bucket_code(pu[u], bb);
                const float xv = xu[u] + 0.0f;
                const int b = q * nbb + bin_of(xv, lo, scale, nbb);
                if (b >= b0 && b < b1) {
                    const int pos = bins.add(b) - base;
                    xs[pos] = xv;
                    ks[pos] = (K)i;
                }
            }
        }
        __syncthreads();
        // bins[b] now holds the end of bin b for b in [b0, b1)
        sort_bins(bins, xs, ks, b0, b1, base, sh, tid);
        const size_t o0 = (size_t)rb + base;
        int qb = 0;   // bucket of position base + j (grows with j)
        for (int j = tid; j < tot; j += PACK_THREADS) {
            while (qb + 1 < NB && sh.boff[qb + 1] <= base + j) ++qb;
            io.ox[o0 + j] = xs[j];
            if (io.oc && ((o0 + j) & 31) == 0) io.oc[(o0 + j) >> 5] = xs[j];
            io.ol[o0 + j] = (uint8_t)(qb % NL);
            io.perm[o0 + j] = rb + (int)ks[j];
        }
        for (int ib = 0; ib < n; ib += PACK_THREADS * UNROLL) {
            int pu[UNROLL];
            float xu[UNROLL], zu[UNROLL], du[UNROLL], wu[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int i = ib + u * PACK_THREADS + tid;
                pu[u] = -1;
                xu[u] = zu[u] = du[u] = wu[u] = 0.0f;
                if (i < n) {
                    pu[u] = plane[rb + i];
                    xu[u] = x[rb + i];
                    zu[u] = io.z[rb + i];
                    du[u] = io.dxdy[rb + i];
                    wu[u] = io.w[rb + i];
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if (pu[u] < 0) continue;
                const int i = ib + u * PACK_THREADS + tid;
                bool bb = false;
                const int q = bucket_code(pu[u], bb);
                const int b = q * nbb + bin_of(xu[u] + 0.0f, lo, scale, nbb);
                if (b < b0 || b >= b1) continue;
                const int en = bins.get(b) - base;
                int j = (b == b0 ? base : bins.get(b - 1)) - base;
                if (en - j > SMALL_BIN) continue;   // a big bin: gathered below
                while (j < en && (int)ks[j] != i) ++j;
                if (j < en) {
                    io.oz[o0 + j] = zu[u];
                    io.od[o0 + j] = du[u];
                    io.ow[o0 + j] = wu[u];
                }
            }
        }
        // hits of big bins (many hits at one x): their payload is gathered
        // through the raw index kept beside each x, so a big bin costs no
        // search per hit
        if (sh.n_big > 0) {
            const bool listed = sh.n_big <= BIG_BINS;
            const int nb_ = listed ? sh.n_big : b1 - b0;
            for (int q = 0; q < nb_; ++q) {
                const int b = listed ? sh.big[q] : b0 + q;
                const int s0 = (b == b0 ? base : bins.get(b - 1)) - base, s1 = bins.get(b) - base;
                if (s1 - s0 <= SMALL_BIN) continue;
                for (int j = s0 + tid; j < s1; j += PACK_THREADS) {
                    const int i = (int)ks[j];
                    io.oz[o0 + j] = __ldg(io.z + rb + i);
                    io.od[o0 + j] = __ldg(io.dxdy + rb + i);
                    io.ow[o0 + j] = __ldg(io.w + rb + i);
                }
            }
        }
        __syncthreads();
        b0 = b1;
    }
}

__global__ void __launch_bounds__(PACK_THREADS, 1) k_pack_event(
    const int* __restrict__ raw_offsets, const float* __restrict__ x, const float* __restrict__ z,
    const float* __restrict__ dxdy, const float* __restrict__ w, const uint8_t* __restrict__ plane, int n_events,
    int* hit_offsets, float* ox, float* oz, float* od, float* ow, uint8_t* ol, int* perm, int* cursor,
    int* status, const int* __restrict__ n_dev, const int* __restrict__ hit_src, float* ocoarse) {
    extern __shared__ __align__(16) char smem[];
    __shared__ EvShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    n_events = slot_events(n_dev, n_events);
    if (blockIdx.x == 0 && tid == 0) hit_offsets[(size_t)n_events * NB] = raw_offsets[n_events];
    if (tid == 0) sh.next = atomicAdd(cursor, 1);
    for (;;) {
        __syncthreads();   // the previous event is fully consumed
        if (tid == 0) {
            sh.event = sh.next;
            sh.next = sh.event < n_events ? atomicAdd(cursor, 1) : n_events;
            sh.flagged = 0u;
            sh.n_big = 0;
        }
        __syncthreads();
        const int e = sh.event;
        if (e >= n_events) break;
        // the event's place in the output (rb) and in the input (ib: the
        // same, or its gather source)
        const int rb = raw_offsets[e], n = raw_offsets[e + 1] - rb;
        const int ib = hit_src ? hit_src[e] : rb;
        // this event's payload and the next event's keys go to L2 while the
        // event is sorted (addresses inside the events' ranges only)
        if (n > 0) {
            prefetch_range(z + ib, (size_t)n * 4, tid);
            prefetch_range(dxdy + ib, (size_t)n * 4, tid);
            prefetch_range(w + ib, (size_t)n * 4, tid);
        }
        if (sh.next < n_events) {
            const int nb0 = raw_offsets[sh.next], nn = raw_offsets[sh.next + 1] - nb0;
            const int ni0 = hit_src ? hit_src[sh.next] : nb0;
            if (nn > 0) {
                prefetch_range(plane + ni0, (size_t)nn, tid);
                prefetch_range(x + ni0, (size_t)nn * 4, tid);
            }
        }
        if (n == 0) {
            if (tid < NB) hit_offsets[(size_t)e * NB + tid] = rb;
            continue;
        }
        if ((unsigned)n > ID_MASK) {
            // beyond the index field: nothing is sorted, every bucket flagged
            if (tid < NB) hit_offsets[(size_t)e * NB + tid] = rb;
            if (tid == 0) atomicOr(status, LF_FLAG_BUCKET_OVERFLOW);
            for (int i = tid; i < n; i += PACK_THREADS) perm[(size_t)rb + i] = -1;
            continue;
        }
        // input pointers shifted so that raw index rb + i reads input ib + i
        const ptrdiff_t d = (ptrdiff_t)ib - rb;
        const PackIO io{x + d, z + d, dxdy + d, w + d, plane + d, hit_offsets, ox, oz, od, ow, ol, perm, status,
                        ocoarse};
        if (n > 65535) sort_event<true>(io, sh, smem, e, rb, n, tid, lane, warp);
        else sort_event<false>(io, sh, smem, e, rb, n, tid, lane, warp);
    }
}

}  // namespace

cudaError_t launch_pack(const int* raw_offsets, const float* x, const float* z, const float* dxdy, const float* w,
                        const uint8_t* plane, int n_events, int n_hits, int* hit_offsets, float* ox, float* oz,
                        float* odxdy, float* ow, uint8_t* olayer, int* perm, int* cursor, int* status, int n_sm,
                        cudaStream_t s, const int* n_dev, const int* hit_src, float* ocoarse) {
    (void)n_hits;
    cudaError_t err =
        cudaFuncSetAttribute(k_pack_event, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AREA_BYTES);
    if (err != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(cursor, 0, sizeof(int), s)) != cudaSuccess) return err;
    int grid = n_sm;
    if (grid > n_events) grid = n_events > 0 ? n_events : 1;
    k_pack_event<<<grid, PACK_THREADS, AREA_BYTES, s>>>(raw_offsets, x, z, dxdy, w, plane, n_events, hit_offsets,
                                                        ox, oz, odxdy, ow, olayer, perm, cursor, status, n_dev,
                                                        hit_src, ocoarse);
    return cudaGetLastError();
}

}  // namespace lfk
