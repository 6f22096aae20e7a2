// Hit packing for sm_103a: per event, bucket the raw hits by (zone, layer),
// sort every bucket by x (ties by raw index) and write the SoA.
//
// Two kernels.  k_pack_event (persistent): a block takes one event at a
// time from a device work queue and sorts it in shared memory:
//   count     the plane codes of the event are counted per warp (peers by
//             __match_any_sync, warp-private counters); an exclusive scan of
//             the totals gives the bucket offsets, written to hit_offsets.
//   chunk     consecutive buckets are grouped into chunks of at most CHUNK
//             hits (one chunk for all but the largest events); per chunk:
//   scatter   the event's hits of the chunk's buckets are placed, bucket
//             by bucket, into shared memory as (x with -0 -> +0, raw index
//             inside the event): every warp owns a fixed share of the hits
//             and, from the counts, its own cursor per bucket (no shared
//             atomics); a warp per bucket then reduces the bucket's x range;
//   bin sort  every bucket is split into as many equal x bins as it has hits
//             (a monotone function of x), and the bins of all buckets of the
//             chunk are counted, scanned and filled by the whole block at
//             once; each bin is then ordered by (x, raw index) with an
//             insertion sort, so the result is the exact (x, raw index) order
//             whatever the data and whatever the order of the scatter;
//   write     the chunk's output range is contiguous: x, layer and perm are
//             written coalesced from shared memory.
// While an event is processed, the block has already taken its next event
// from the queue and prefetched that event's plane codes and x into L2.
// k_pack_payload then walks the packed positions in order (coalesced
// writes) and gathers z, dxdy and w through perm: scattered 4-byte reads
// want many loads in flight, i.e. a kernel at full occupancy rather than
// one large block per SM.
// A bucket above CHUNK hits cannot be sorted: it is flagged (status bit
// 0x1), its perm entries are set to -1 and its other outputs are not
// meaningful; a plane code >= 24 is flagged (0x2) and counted in the last
// bucket.
#include <cstdint>

#include "lf_internal.h"

namespace lfk {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PACK_THREADS = 1024;
constexpr int PACK_WARPS = PACK_THREADS / 32;
constexpr int CHUNK = BLOCK_SORT_MAX;  // hits sorted together in shared memory
constexpr int UNROLL = 4;              // hits per thread with loads in flight together

// shared memory per element: x, raw index, bin counter (16-bit halves of
// 32-bit words), slot inside the bin, element at each sorted position
constexpr size_t AREA_BYTES = (size_t)CHUNK * (4 + 4 + 2 + 2 + 2);

struct Area {
    float* xs;          // x of element k
    uint32_t* id;       // raw index of element k, relative to the event
    uint32_t* bins2;    // bin counters / starts, two 16-bit values per word
    uint16_t* slot;     // slot of element k inside its bin
    uint16_t* order;    // element at sorted position j
};

__device__ __forceinline__ Area area_at(char* p) {
    Area a;
    a.xs = reinterpret_cast<float*>(p);
    a.id = reinterpret_cast<uint32_t*>(p + (size_t)CHUNK * 4);
    a.bins2 = reinterpret_cast<uint32_t*>(p + (size_t)CHUNK * 8);
    a.slot = reinterpret_cast<uint16_t*>(p + (size_t)CHUNK * 10);
    a.order = reinterpret_cast<uint16_t*>(p + (size_t)CHUNK * 12);
    return a;
}

__device__ __forceinline__ int wscan_incl(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// x as an unsigned integer with the same order (-0 already turned into +0)
__device__ __forceinline__ unsigned ordered(float x) {
    unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ int bin_of(float x, float lo, float scale, int nb) {
    float f = (x - lo) * scale;   // monotone in x
    if (!(f > 0.0f)) return 0;
    if (!(f < (float)nb)) return nb - 1;
    return (int)f;
}

// 16-bit counter i of the packed bin array
__device__ __forceinline__ unsigned bin_add(uint32_t* bins2, int i) {
    unsigned old = atomicAdd(&bins2[i >> 1], (i & 1) ? 0x10000u : 1u);
    return (i & 1) ? (old >> 16) : (old & 0xffffu);
}
__device__ __forceinline__ unsigned bin_get(const uint32_t* bins2, int i) {
    unsigned v = bins2[i >> 1];
    return (i & 1) ? (v >> 16) : (v & 0xffffu);
}

struct EvShared {
    uint16_t wcur[PACK_WARPS][NB];   // per-warp scatter cursor inside each bucket
    int cnt[NB];                // bucket sizes
    int off[NB + 1];            // bucket offsets inside the event
    int coff[NB + 1];           // bucket offsets inside the chunk
    float blo[NB], bscale[NB];  // bin mapping of each bucket
    int warp_tot[PACK_WARPS];
    int event, next;
};

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

// bucket of chunk element k: the last bucket q in [qa, ql] with coff[q] <= k
// (an empty bucket shares its offset with the next one, so the last wins)
__device__ __forceinline__ int bucket_of(const EvShared& sh, int qa, int ql, int k) {
    int lo = qa, hi = ql;
#pragma unroll
    for (int it = 0; it < 5; ++it) {   // 2^5 >= 24 buckets
        const int mid = (lo + hi + 1) >> 1;
        if (lo < hi) {
            if (sh.coff[mid] <= k) lo = mid; else hi = mid - 1;
        }
    }
    return lo;
}

__global__ void __launch_bounds__(PACK_THREADS, 1) k_pack_event(
    const int* __restrict__ raw_offsets, const float* __restrict__ x, const uint8_t* __restrict__ plane,
    int n_events, int* hit_offsets, float* ox, uint8_t* ol, int* perm, int* cursor, int* status) {
    extern __shared__ __align__(16) char smem[];
    __shared__ EvShared sh;
    const Area a = area_at(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.x == 0 && tid == 0) hit_offsets[(size_t)n_events * NB] = raw_offsets[n_events];
    if (tid == 0) sh.next = atomicAdd(cursor, 1);
    for (;;) {
        __syncthreads();   // the previous event is fully consumed
        if (tid == 0) {
            sh.event = sh.next;
            sh.next = sh.event < n_events ? atomicAdd(cursor, 1) : n_events;
        }
        __syncthreads();
        const int e = sh.event;
        if (e >= n_events) break;
        const int rb = raw_offsets[e], n = raw_offsets[e + 1] - rb;
        // the next event's raw arrays go to L2 while this one is processed
        // (addresses inside the next event's range only)
        if (sh.next < n_events) {
            const int nb0 = raw_offsets[sh.next], nn = raw_offsets[sh.next + 1] - nb0;
            if (nn > 0) {
                prefetch_range(plane + nb0, (size_t)nn, tid);
                prefetch_range(x + nb0, (size_t)nn * 4, tid);
            }
        }

        // count into warp-private counters (in the element area, unused until
        // the scatter); the leader of each group of equal codes adds its size
        int* wcnt = reinterpret_cast<int*>(smem) + warp * NB;
        if (lane < NB) wcnt[lane] = 0;
        __syncwarp();
        bool bad = false;
        for (int base = warp * 32; base < n; base += PACK_THREADS * UNROLL) {
            int pu[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const int i = base + u * PACK_THREADS + lane;
                pu[u] = i < n ? (int)plane[rb + i] : -1;
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                int p = pu[u];
                if (p >= NB) {
                    bad = true;
                    p = NB - 1;
                }
                const unsigned peers = __match_any_sync(FULL, p);
                if (p >= 0 && lane == __ffs(peers) - 1) wcnt[p] += __popc(peers);
                __syncwarp();
            }
        }
        if (bad) atomicOr(status, 0x2);
        wcnt = reinterpret_cast<int*>(smem);
        __syncthreads();
        if (tid < 32) {
            // bucket totals; each warp's cursor starts after the earlier warps' hits
            int c = 0;
            if (lane < NB)
                for (int q = 0; q < PACK_WARPS; ++q) {
                    sh.wcur[q][lane] = (uint16_t)c;
                    c += wcnt[q * NB + lane];
                }
            const int inc = wscan_incl(c, lane);
            if (lane < NB) {
                sh.cnt[lane] = c;
                sh.off[lane] = inc - c;
                hit_offsets[(size_t)e * NB + lane] = rb + inc - c;
                if (c > CHUNK) atomicOr(status, 0x1);
            }
            if (lane == NB - 1) sh.off[NB] = inc;
        }
        __syncthreads();

        // chunks of consecutive buckets (every thread takes the same decisions)
        int qa = 0;
        while (qa < NB) {
            int qb = qa, tot = 0;
            while (qb < NB && tot + sh.cnt[qb] <= CHUNK) tot += sh.cnt[qb++];
            if (qb == qa) {   // a bucket above CHUNK hits: flagged above, not sorted
                const size_t o0 = (size_t)rb + sh.off[qa];
                for (int j = tid; j < sh.cnt[qa]; j += PACK_THREADS) perm[o0 + j] = -1;
                ++qa;
                continue;
            }
            if (tot == 0) {
                qa = qb;
                continue;
            }
            const int ql = qb - 1;
            // scatter the chunk's hits, bucket by bucket; a warp visits the
            // same hits as in the count and advances its own cursors
            if (tid < NB) sh.coff[tid] = (tid >= qa && tid < qb) ? sh.off[tid] - sh.off[qa] : 0;
            __syncthreads();
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
                const int i = base + u * PACK_THREADS + tid;
                int p = pu[u];
                if (p >= NB) p = NB - 1;
                if (p < qa || p >= qb) p = -1;
                const unsigned peers = __match_any_sync(FULL, p);
                const int cur = p >= 0 ? (int)sh.wcur[warp][p] : 0;
                __syncwarp();
                if (p >= 0) {
                    const int rank = __popc(peers & ((1u << lane) - 1u));
                    if (rank == 0) sh.wcur[warp][p] = (uint16_t)(cur + __popc(peers));
                    const int k = sh.coff[p] + cur + rank;
                    a.xs[k] = xu[u] + 0.0f;
                    a.id[k] = (uint32_t)i;
                }
                __syncwarp();
                }
            }
            for (int q = tid; q < (tot + 1) / 2; q += PACK_THREADS) a.bins2[q] = 0u;
            __syncthreads();
            // x range of bucket q, reduced by warp q - qa (buckets of a chunk <= 24 < 32 warps)
            {
                const int q = qa + warp;
                if (q < qb) {
                    const int m = sh.cnt[q], k0 = sh.coff[q];
                    unsigned mn = 0xffffffffu, mx = 0u;
                    for (int k = lane; k < m; k += 32) {
                        const unsigned ov = ordered(a.xs[k0 + k]);
                        mn = min(mn, ov);
                        mx = max(mx, ov);
                    }
                    mn = __reduce_min_sync(FULL, mn);
                    mx = __reduce_max_sync(FULL, mx);
                    if (lane == 0) {
                        float lo = 0.0f, scale = 0.0f;
                        if (m > 0) {
                            lo = unordered(mn);
                            const float hi = unordered(mx);
                            scale = hi > lo ? (float)m / (hi - lo) : 0.0f;
                        }
                        sh.blo[q] = lo;
                        sh.bscale[q] = scale;
                    }
                }
            }
            __syncthreads();

            // count: bin of element k = bucket offset + bin inside the bucket
            for (int k = tid; k < tot; k += PACK_THREADS) {
                const int q = bucket_of(sh, qa, ql, k);
                const int bn = sh.coff[q] + bin_of(a.xs[k], sh.blo[q], sh.bscale[q], sh.cnt[q]);
                a.slot[k] = (uint16_t)bin_add(a.bins2, bn);
            }
            __syncthreads();
            // exclusive scan of the tot counters; every thread's run starts
            // on an even counter, so each 32-bit word has a single writer
            {
                const int per = 2 * ((tot + 2 * PACK_THREADS - 1) / (2 * PACK_THREADS));
                const int s0 = min(tid * per, tot), s1 = min(s0 + per, tot);
                int sum = 0;
                for (int i = s0; i < s1; ++i) sum += (int)bin_get(a.bins2, i);
                const int inc = wscan_incl(sum, lane);
                if (lane == 31) sh.warp_tot[warp] = inc;
                __syncthreads();
                int excl = inc - sum;
                for (int q = 0; q < warp; ++q) excl += sh.warp_tot[q];
                for (int i = s0; i < s1; i += 2) {
                    const unsigned v = a.bins2[i >> 1];
                    const unsigned c0 = v & 0xffffu, c1 = v >> 16;
                    const unsigned st0 = (unsigned)excl, st1 = st0 + c0;
                    a.bins2[i >> 1] = st0 | (st1 << 16);
                    excl += (int)(c0 + c1);
                }
            }
            __syncthreads();
            // placement
            for (int k = tid; k < tot; k += PACK_THREADS) {
                const int q = bucket_of(sh, qa, ql, k);
                const int bn = sh.coff[q] + bin_of(a.xs[k], sh.blo[q], sh.bscale[q], sh.cnt[q]);
                a.order[bin_get(a.bins2, bn) + a.slot[k]] = (uint16_t)k;
            }
            __syncthreads();
            // order each bin by (x, raw index); bin b ends where b + 1 starts
            for (int bn = tid; bn < tot; bn += PACK_THREADS) {
                const int s = (int)bin_get(a.bins2, bn), en = bn + 1 < tot ? (int)bin_get(a.bins2, bn + 1) : tot;
                for (int i = s + 1; i < en; ++i) {
                    const int pv = a.order[i];
                    const float xv = a.xs[pv];
                    const uint32_t iv = a.id[pv];
                    int j = i - 1;
                    while (j >= s) {
                        const int pj = a.order[j];
                        const float xj = a.xs[pj];
                        if (!(xv < xj || (xv == xj && iv < a.id[pj]))) break;
                        a.order[j + 1] = (uint16_t)pj;
                        --j;
                    }
                    a.order[j + 1] = (uint16_t)pv;
                }
            }
            __syncthreads();
            // the chunk's output range is contiguous
            {
                const size_t o0 = (size_t)rb + sh.off[qa];
#pragma unroll 4
                for (int j = tid; j < tot; j += PACK_THREADS) {
                    const int q = bucket_of(sh, qa, ql, j);
                    const int k = a.order[j];
                    const size_t o = o0 + j;
                    ox[o] = a.xs[k];
                    ol[o] = (uint8_t)(q % NL);
                    perm[o] = rb + (int)a.id[k];
                }
            }
            __syncthreads();
            qa = qb;
        }
    }
}

// z, dxdy and w in packed order: position o takes raw hit perm[o].  Blocks
// take tiles of consecutive positions from a work queue, so the tiles in
// flight stay a narrow window of events whose raw lines L2 reuses (a grid
// stride lets warps drift apart over the batch and loses that reuse).
constexpr int PAYLOAD_THREADS = 256;
constexpr int PAYLOAD_PER_THREAD = 8;
constexpr int PAYLOAD_TILE = PAYLOAD_THREADS * PAYLOAD_PER_THREAD;

__global__ void __launch_bounds__(PAYLOAD_THREADS) k_pack_payload(
    const float* __restrict__ z, const float* __restrict__ dxdy, const float* __restrict__ w,
    const int* __restrict__ perm, int n_hits, float* __restrict__ oz, float* __restrict__ od,
    float* __restrict__ ow, int* cursor) {
    __shared__ int s_tile;
    const int n_tiles = (n_hits + PAYLOAD_TILE - 1) / PAYLOAD_TILE;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(cursor, 1);
        __syncthreads();
        const int tile = s_tile;
        __syncthreads();
        if (tile >= n_tiles) break;
        const int o0 = tile * PAYLOAD_TILE + threadIdx.x;
        int r[PAYLOAD_PER_THREAD];
#pragma unroll
        for (int u = 0; u < PAYLOAD_PER_THREAD; ++u) {
            const int o = o0 + u * PAYLOAD_THREADS;
            r[u] = o < n_hits ? perm[o] : -1;
        }
        float vz[PAYLOAD_PER_THREAD], vd[PAYLOAD_PER_THREAD], vw[PAYLOAD_PER_THREAD];
#pragma unroll
        for (int u = 0; u < PAYLOAD_PER_THREAD; ++u) {
            // r < 0: past the end, or a bucket the pack could not sort
            vz[u] = r[u] >= 0 ? __ldg(z + r[u]) : 0.0f;
            vd[u] = r[u] >= 0 ? __ldg(dxdy + r[u]) : 0.0f;
            vw[u] = r[u] >= 0 ? __ldg(w + r[u]) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < PAYLOAD_PER_THREAD; ++u) {
            const int o = o0 + u * PAYLOAD_THREADS;
            if (o < n_hits) {
                oz[o] = vz[u];
                od[o] = vd[u];
                ow[o] = vw[u];
            }
        }
    }
}

}  // namespace

cudaError_t launch_pack(const int* raw_offsets, const float* x, const float* z, const float* dxdy, const float* w,
                        const uint8_t* plane, int n_events, int n_hits, int* hit_offsets, float* ox, float* oz,
                        float* odxdy, float* ow, uint8_t* olayer, int* perm, int* cursor, int* status, int n_sm,
                        cudaStream_t s) {
    cudaError_t err =
        cudaFuncSetAttribute(k_pack_event, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AREA_BYTES);
    if (err != cudaSuccess) return err;
    int bps = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_pack_event, PACK_THREADS, AREA_BYTES);
    if (err != cudaSuccess) return err;
    if (bps < 1) bps = 1;
    if ((err = cudaMemsetAsync(cursor, 0, 2 * sizeof(int), s)) != cudaSuccess) return err;
    int grid = n_sm * bps;
    if (grid > n_events) grid = n_events > 0 ? n_events : 1;
    k_pack_event<<<grid, PACK_THREADS, AREA_BYTES, s>>>(raw_offsets, x, plane, n_events, hit_offsets, ox, olayer,
                                                        perm, cursor, status);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (n_hits > 0) {
        int bpp = 0;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpp, k_pack_payload, PAYLOAD_THREADS, 0);
        if (err != cudaSuccess) return err;
        const long tiles = ((long)n_hits + PAYLOAD_TILE - 1) / PAYLOAD_TILE;
        int gp = n_sm * (bpp > 0 ? bpp : 1);
        if (gp > tiles) gp = (int)tiles;
        k_pack_payload<<<gp, PAYLOAD_THREADS, 0, s>>>(z, dxdy, w, perm, n_hits, oz, odxdy, ow, cursor + 1);
    }
    return cudaGetLastError();
}

}  // namespace lfk
