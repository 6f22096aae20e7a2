// Hit packing for sm_103a: per event, bucket the raw hits by (zone, layer),
// then sort every bucket by x (ties by raw index) and write the SoA.
//
//   k_pack_bucket   one block per event (grid-stride): each warp counts the
//                   plane codes of its slice of the event (ranked with
//                   __match_any_sync), a per-bucket prefix over buckets and
//                   warps gives the bucket offsets and each warp's cursors,
//                   and each warp scatters its slice in order: a STABLE
//                   scatter, so inside a bucket raw indices stay ascending.
//   k_pack_sort     one block per event (grid-stride), so the event's raw
//                   hits stay hot in L1/L2 while all its buckets are sorted:
//                   buckets of at most 1024 hits by one warp each, larger
//                   ones (at most 8192) by the whole block; a bin sort in
//                   shared memory.
//                   Bins split [min, max] of the bucket into as many equal
//                   parts as hits (the bin is a monotone function of x); each
//                   bin is then ordered by (x, position) with an insertion
//                   sort; positions follow raw order, so the result is the
//                   exact (x, raw index) order whatever the data.
//   The sorted bucket is written out coalesced: x, z, dxdy, w, layer, perm.
#include <cstdint>

#include "lf_internal.h"

namespace lfk {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BUCKET_THREADS = 256;
constexpr int BUCKET_WARPS = BUCKET_THREADS / 32;
constexpr int WARP_MAX = 1024;      // bucket size sorted by one warp
constexpr int SORT_THREADS = 256;   // 8 warps: 8 warp areas of WARP_MAX == one block area of BLOCK_SORT_MAX

__device__ __forceinline__ int wscan_incl(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__global__ void __launch_bounds__(BUCKET_THREADS) k_pack_bucket(
    const int* __restrict__ raw_offsets, const uint8_t* __restrict__ plane, int n_events, int* hit_offsets,
    int* tmp, int* status) {
    __shared__ int wc[BUCKET_WARPS][NB];   // per-warp counts, then per-warp cursors
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = blockIdx.x; e < n_events; e += gridDim.x) {
        const int rb = raw_offsets[e], re = raw_offsets[e + 1];
        const int slice = ((re - rb + BUCKET_WARPS - 1) / BUCKET_WARPS + 31) & ~31;
        const int s0 = min(rb + warp * slice, re), s1 = min(s0 + slice, re);
        if (lane < NB) wc[warp][lane] = 0;
        __syncwarp();
        for (int base = s0; base < s1; base += 32) {
            int i = base + lane;
            int p = -1;
            if (i < s1) {
                p = plane[i];
                if (p >= NB) {
                    atomicOr(status, 0x2);
                    p = NB - 1;
                }
            }
            unsigned peers = __match_any_sync(FULL, p);
            if (p >= 0 && lane == __ffs(peers) - 1) wc[warp][p] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        if (tid < 32) {
            // bucket totals, their exclusive scan, then each warp's cursor
            int tot = 0;
            if (lane < NB)
                for (int w = 0; w < BUCKET_WARPS; ++w) tot += wc[w][lane];
            int inc = wscan_incl(tot, lane);
            int start = rb + inc - tot;
            if (lane < NB) {
                hit_offsets[(size_t)e * NB + lane] = start;
                if (tot > BLOCK_SORT_MAX) atomicOr(status, 0x1);
                int acc = start;
                for (int w = 0; w < BUCKET_WARPS; ++w) {
                    int c = wc[w][lane];
                    wc[w][lane] = acc;
                    acc += c;
                }
            }
        }
        __syncthreads();
        for (int base = s0; base < s1; base += 32) {
            int i = base + lane;
            int p = -1;
            if (i < s1) {
                p = plane[i];
                if (p >= NB) p = NB - 1;
            }
            unsigned peers = __match_any_sync(FULL, p);
            int rank = __popc(peers & ((1u << lane) - 1u));
            int cur = p >= 0 ? wc[warp][p] : 0;
            __syncwarp();
            if (p >= 0) {
                tmp[cur + rank] = i;
                if (rank == 0) wc[warp][p] = cur + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && tid == 0) hit_offsets[(size_t)n_events * NB] = raw_offsets[n_events];
}

__device__ __forceinline__ int bin_of(float x, float xmin, float scale, int nb) {
    float f = (x - xmin) * scale;   // monotone in x; NaN only when x == xmin and scale is infinite
    if (!(f > 0.0f)) return 0;
    if (!(f < (float)nb)) return nb - 1;
    return (int)f;
}

template <bool BLOCK>
__device__ __forceinline__ void gsync() {
    if (BLOCK) __syncthreads(); else __syncwarp();
}

// Work area of one bucket sort (m entries each): keys x, bin counters, and
// the positions (0..m-1, raw order inside the bucket) in sorted order.
struct SortArea {
    float* xa;
    int* bins;
    uint16_t* pos;
};

// Cooperative bin sort of one bucket by a warp (BLOCK = false) or a block.
template <bool BLOCK>
__device__ void sort_bucket(const float* __restrict__ x, const float* __restrict__ z, const float* __restrict__ dxdy,
                            const float* __restrict__ w, const int* __restrict__ tmp, int b0, int m, int layer,
                            float* ox, float* oz, float* od, float* ow, uint8_t* ol, int* perm, SortArea a,
                            int rank, int size, float* red_f, int* red_i) {
    const int lane = rank & 31, wid = rank >> 5, nw = size >> 5;
    float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
    for (int i = rank; i < m; i += size) {
        float xv = __ldg(x + tmp[b0 + i]) + 0.0f;
        a.xa[i] = xv;
        lo = fminf(lo, xv);
        hi = fmaxf(hi, xv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
    }
    if (BLOCK) {
        if (lane == 0) {
            red_f[wid] = lo;
            red_f[32 + wid] = hi;
        }
        __syncthreads();
        lo = red_f[0];
        hi = red_f[32];
        for (int q = 1; q < nw; ++q) {
            lo = fminf(lo, red_f[q]);
            hi = fmaxf(hi, red_f[32 + q]);
        }
    }
    const int nb = m;
    const float scale = hi > lo ? (float)nb / (hi - lo) : 0.0f;
    for (int i = rank; i < nb; i += size) a.bins[i] = 0;
    gsync<BLOCK>();
    for (int i = rank; i < m; i += size) atomicAdd(&a.bins[bin_of(a.xa[i], lo, scale, nb)], 1);
    gsync<BLOCK>();
    {
        // exclusive scan of the bin counts: a contiguous chunk per thread
        const int per = (nb + size - 1) / size;
        const int s0 = min(rank * per, nb), s1 = min(s0 + per, nb);
        int sum = 0;
        for (int i = s0; i < s1; ++i) sum += a.bins[i];
        int inc = wscan_incl(sum, lane);
        int excl = inc - sum;
        if (BLOCK) {
            if (lane == 31) red_i[wid] = inc;
            __syncthreads();
            int base = 0;
            for (int q = 0; q < wid; ++q) base += red_i[q];
            excl += base;
        }
        for (int i = s0; i < s1; ++i) {
            int c = a.bins[i];
            a.bins[i] = excl;
            excl += c;
        }
    }
    gsync<BLOCK>();
    for (int i = rank; i < m; i += size) a.pos[atomicAdd(&a.bins[bin_of(a.xa[i], lo, scale, nb)], 1)] = (uint16_t)i;
    gsync<BLOCK>();
    // bins[b] is now the end of bin b; order each bin by (x, position)
    for (int bn = rank; bn < nb; bn += size) {
        int s = bn ? a.bins[bn - 1] : 0, e = a.bins[bn];
        for (int i = s + 1; i < e; ++i) {
            int pv = a.pos[i];
            float xv = a.xa[pv];
            int j = i - 1;
            while (j >= s) {
                int pj = a.pos[j];
                float xj = a.xa[pj];
                if (!(xv < xj || (xv == xj && pv < pj))) break;
                a.pos[j + 1] = (uint16_t)pj;
                --j;
            }
            a.pos[j + 1] = (uint16_t)pv;
        }
    }
    gsync<BLOCK>();
    for (int i = rank; i < m; i += size) {
        int pv = a.pos[i];
        int r = tmp[b0 + pv];
        size_t o = (size_t)b0 + i;
        ox[o] = a.xa[pv];
        oz[o] = __ldg(z + r);
        od[o] = __ldg(dxdy + r);
        ow[o] = __ldg(w + r);
        ol[o] = (uint8_t)layer;
        perm[o] = r;
    }
    gsync<BLOCK>();
}

__host__ __device__ constexpr size_t area_bytes(int n) { return (size_t)n * 4 + (size_t)n * 4 + (((size_t)n * 2 + 15) & ~size_t(15)); }

__device__ __forceinline__ SortArea area_at(char* p, int n) {
    SortArea a;
    a.xa = reinterpret_cast<float*>(p);
    a.bins = reinterpret_cast<int*>(p + (size_t)n * 4);
    a.pos = reinterpret_cast<uint16_t*>(p + (size_t)n * 8);
    return a;
}

// One block per event: small buckets by the block's warps (each with its own
// shared-memory area), then the large ones by the whole block (the union of
// the warps' areas), so the event's raw hits are read while hot.
__global__ void __launch_bounds__(SORT_THREADS) k_pack_sort(
    const float* __restrict__ x, const float* __restrict__ z, const float* __restrict__ dxdy,
    const float* __restrict__ w, const int* __restrict__ hit_offsets, const int* __restrict__ tmp, int n_events,
    float* ox, float* oz, float* od, float* ow, uint8_t* ol, int* perm) {
    extern __shared__ __align__(16) char smem[];
    __shared__ float red_f[64];
    __shared__ int red_i[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SortArea wa = area_at(smem + (size_t)warp * area_bytes(WARP_MAX), WARP_MAX);
    const SortArea ba = area_at(smem, BLOCK_SORT_MAX);
    for (int e = blockIdx.x; e < n_events; e += gridDim.x) {
        const int* off = hit_offsets + (size_t)e * NB;
        for (int q = warp; q < NB; q += SORT_THREADS / 32) {
            int b0 = off[q], m = off[q + 1] - b0;
            if (m >= 1 && m <= WARP_MAX)
                sort_bucket<false>(x, z, dxdy, w, tmp, b0, m, q % NL, ox, oz, od, ow, ol, perm, wa, lane, 32,
                                   nullptr, nullptr);
        }
        __syncthreads();
        for (int q = 0; q < NB; ++q) {
            int b0 = off[q], m = off[q + 1] - b0;
            if (m > WARP_MAX && m <= BLOCK_SORT_MAX)
                sort_bucket<true>(x, z, dxdy, w, tmp, b0, m, q % NL, ox, oz, od, ow, ol, perm, ba, tid,
                                  SORT_THREADS, red_f, red_i);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_pack(const int* raw_offsets, const float* x, const float* z, const float* dxdy,
                        const float* w, const uint8_t* plane, int n_events, int n_hits,
                        int* hit_offsets, float* ox, float* oz, float* odxdy, float* ow, uint8_t* olayer,
                        int* perm, int* tmp, int* big_list, int* status, int n_sm, cudaStream_t s) {
    (void)n_hits;
    (void)big_list;
    if (n_events <= 0) return cudaMemsetAsync(hit_offsets, 0, sizeof(int), s);
    int grid = n_events < n_sm * 8 ? n_events : n_sm * 8;
    k_pack_bucket<<<grid, BUCKET_THREADS, 0, s>>>(raw_offsets, plane, n_events, hit_offsets, tmp, status);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const size_t sm = area_bytes(BLOCK_SORT_MAX);
    if ((err = cudaFuncSetAttribute(k_pack_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
        cudaSuccess)
        return err;
    int gs = n_events < n_sm * 2 ? n_events : n_sm * 2;
    k_pack_sort<<<gs, SORT_THREADS, sm, s>>>(x, z, dxdy, w, hit_offsets, tmp, n_events, ox, oz, odxdy, ow, olayer,
                                             perm);
    return cudaGetLastError();
}

}  // namespace lfk
