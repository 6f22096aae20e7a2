// Hit packing for sm_103a: per event, bucket the raw hits by (zone, layer),
// then sort every bucket by x (ties by raw index) and write the SoA.
//
//   k_pack_bucket   one block per event (grid-stride): shared-memory
//                   histogram of the plane codes, exclusive scan into the
//                   bucket offsets, scatter of raw indices into their bucket
//                   (order inside a bucket is fixed by the sort that follows).
//   k_pack_sort     one warp per bucket of at most WARP_SORT_MAX hits, one
//                   block per larger bucket: a bin sort in shared memory.
//                   Keys are the x values; bins split [min, max] of the bucket
//                   into as many equal parts as hits (the bin index is a
//                   monotone function of x), each bin is then ordered by
//                   (x, raw index) with an insertion sort, so the result is
//                   the exact (x, raw index) order whatever the data.
//   The sorted bucket is written out coalesced: x, z, dxdy, w, layer, perm.
#include <cstdint>

#include "lf_internal.h"

namespace lfk {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int wscan_incl(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__global__ void k_pack_bucket(const int* __restrict__ raw_offsets, const uint8_t* __restrict__ plane, int n_events,
                              int* hit_offsets, int* tmp, int* big_list, int* status) {
    __shared__ int cnt[NB], cur[NB];
    const int tid = threadIdx.x;
    for (int e = blockIdx.x; e < n_events; e += gridDim.x) {
        if (tid < NB) cnt[tid] = 0;
        __syncthreads();
        const int rb = raw_offsets[e], re = raw_offsets[e + 1];
        for (int i = rb + tid; i < re; i += blockDim.x) {
            int p = plane[i];
            if (p >= NB) {
                atomicOr(status, 0x2);
                p = NB - 1;
            }
            atomicAdd(&cnt[p], 1);
        }
        __syncthreads();
        if (tid == 0) {
            int acc = rb;
            for (int q = 0; q < NB; ++q) {
                hit_offsets[(size_t)e * NB + q] = acc;
                cur[q] = acc;
                int c = cnt[q];
                if (c > BLOCK_SORT_MAX) atomicOr(status, 0x1);
                else if (c > WARP_SORT_MAX) big_list[1 + atomicAdd(big_list, 1)] = e * NB + q;
                acc += c;
            }
        }
        __syncthreads();
        for (int i = rb + tid; i < re; i += blockDim.x) {
            int p = plane[i];
            if (p >= NB) p = NB - 1;
            int pos = atomicAdd(&cur[p], 1);
            tmp[pos] = i;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && tid == 0) hit_offsets[(size_t)n_events * NB] = raw_offsets[n_events];
}

// Work area of one bucket sort: keys (x), raw indices, their sorted copies
// and the bin counters, n entries each.
struct SortArea {
    float* xa;
    int* ra;
    float* xb;
    int* rb;
    int* bins;
};

__device__ __forceinline__ bool before(float xa, int ra, float xb, int rb) {
    return xa < xb || (xa == xb && ra < rb);
}

__device__ __forceinline__ int bin_of(float x, float xmin, float scale, int nb) {
    float f = (x - xmin) * scale;   // monotone in x; NaN only when x == xmin and scale is infinite
    if (!(f > 0.0f)) return 0;
    if (!(f < (float)nb)) return nb - 1;
    return (int)f;
}

// Group-cooperative bin sort; G is a warp (32 lanes, __syncwarp) or a block.
template <bool BLOCK>
__device__ __forceinline__ void gsync() {
    if (BLOCK) __syncthreads(); else __syncwarp();
}

template <bool BLOCK>
__device__ void sort_bucket(const float* __restrict__ x, const float* __restrict__ z, const float* __restrict__ dxdy,
                            const float* __restrict__ w, const int* __restrict__ tmp, int b0, int m, int layer,
                            float* ox, float* oz, float* od, float* ow, uint8_t* ol, int* perm, SortArea a,
                            int rank, int size, float* red_f, int* red_i) {
    const int lane = rank & 31, wid = rank >> 5, nw = size >> 5;
    // load keys, min / max
    float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
    for (int i = rank; i < m; i += size) {
        int r = tmp[b0 + i];
        float xv = __ldg(x + r) + 0.0f;
        a.xa[i] = xv;
        a.ra[i] = r;
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
    // exclusive scan of the bin counts: contiguous chunk per thread
    {
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
    for (int i = rank; i < m; i += size) {
        int pos = atomicAdd(&a.bins[bin_of(a.xa[i], lo, scale, nb)], 1);
        a.xb[pos] = a.xa[i];
        a.rb[pos] = a.ra[i];
    }
    gsync<BLOCK>();
    // bins[b] is now the end of bin b; order each bin by (x, raw index)
    for (int bn = rank; bn < nb; bn += size) {
        int s = bn ? a.bins[bn - 1] : 0, e = a.bins[bn];
        for (int i = s + 1; i < e; ++i) {
            float xv = a.xb[i];
            int rv = a.rb[i];
            int j = i - 1;
            while (j >= s && before(xv, rv, a.xb[j], a.rb[j])) {
                a.xb[j + 1] = a.xb[j];
                a.rb[j + 1] = a.rb[j];
                --j;
            }
            a.xb[j + 1] = xv;
            a.rb[j + 1] = rv;
        }
    }
    gsync<BLOCK>();
    for (int i = rank; i < m; i += size) {
        int r = a.rb[i];
        size_t o = (size_t)b0 + i;
        ox[o] = a.xb[i];
        oz[o] = __ldg(z + r);
        od[o] = __ldg(dxdy + r);
        ow[o] = __ldg(w + r);
        ol[o] = (uint8_t)layer;
        perm[o] = r;
    }
    gsync<BLOCK>();
}

constexpr int SORT_WARPS = 4;

__global__ void __launch_bounds__(SORT_WARPS * 32) k_pack_sort_warp(
    const float* __restrict__ x, const float* __restrict__ z, const float* __restrict__ dxdy,
    const float* __restrict__ w, const int* __restrict__ hit_offsets, const int* __restrict__ tmp, int n_buckets,
    float* ox, float* oz, float* od, float* ow, uint8_t* ol, int* perm) {
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    char* base = smem + (size_t)warp * WARP_SORT_MAX * 20;
    SortArea a;
    a.xa = reinterpret_cast<float*>(base);
    a.ra = reinterpret_cast<int*>(base + WARP_SORT_MAX * 4);
    a.xb = reinterpret_cast<float*>(base + WARP_SORT_MAX * 8);
    a.rb = reinterpret_cast<int*>(base + WARP_SORT_MAX * 12);
    a.bins = reinterpret_cast<int*>(base + WARP_SORT_MAX * 16);
    const int gw = blockIdx.x * SORT_WARPS + warp, nwarps = gridDim.x * SORT_WARPS;
    for (int q = gw; q < n_buckets; q += nwarps) {
        int b0 = hit_offsets[q], m = hit_offsets[q + 1] - b0;
        if (m == 0 || m > WARP_SORT_MAX) continue;
        sort_bucket<false>(x, z, dxdy, w, tmp, b0, m, (q % NB) % NL, ox, oz, od, ow, ol, perm, a, lane, 32, nullptr,
                           nullptr);
    }
}

__global__ void __launch_bounds__(BLOCK_SORT_THREADS) k_pack_sort_block(
    const float* __restrict__ x, const float* __restrict__ z, const float* __restrict__ dxdy,
    const float* __restrict__ w, const int* __restrict__ hit_offsets, const int* __restrict__ tmp,
    const int* __restrict__ big_list, float* ox, float* oz, float* od, float* ow, uint8_t* ol, int* perm) {
    extern __shared__ __align__(16) char smem[];
    __shared__ float red_f[64];
    __shared__ int red_i[32];
    SortArea a;
    a.xa = reinterpret_cast<float*>(smem);
    a.ra = reinterpret_cast<int*>(smem + BLOCK_SORT_MAX * 4);
    a.xb = reinterpret_cast<float*>(smem + BLOCK_SORT_MAX * 8);
    a.rb = reinterpret_cast<int*>(smem + BLOCK_SORT_MAX * 12);
    a.bins = reinterpret_cast<int*>(smem + BLOCK_SORT_MAX * 16);
    const int n_big = big_list[0];
    for (int k = blockIdx.x; k < n_big; k += gridDim.x) {
        int q = big_list[1 + k];
        int b0 = hit_offsets[q], m = hit_offsets[q + 1] - b0;
        sort_bucket<true>(x, z, dxdy, w, tmp, b0, m, (q % NB) % NL, ox, oz, od, ow, ol, perm, a, threadIdx.x,
                          blockDim.x, red_f, red_i);
    }
}

}  // namespace

cudaError_t launch_pack(const int* raw_offsets, const float* x, const float* z, const float* dxdy,
                        const float* w, const uint8_t* plane, int n_events, int n_hits,
                        int* hit_offsets, float* ox, float* oz, float* odxdy, float* ow, uint8_t* olayer,
                        int* perm, int* tmp, int* big_list, int* status, int n_sm, cudaStream_t s) {
    (void)n_hits;
    cudaError_t err = cudaMemsetAsync(big_list, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    if (n_events <= 0) {
        return cudaMemsetAsync(hit_offsets, 0, sizeof(int), s);
    }
    int grid = n_events < n_sm * 8 ? n_events : n_sm * 8;
    k_pack_bucket<<<grid, 256, 0, s>>>(raw_offsets, plane, n_events, hit_offsets, tmp, big_list, status);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int n_buckets = n_events * NB;
    size_t smw = (size_t)SORT_WARPS * WARP_SORT_MAX * 20;
    err = cudaFuncSetAttribute(k_pack_sort_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
    if (err != cudaSuccess) return err;
    int gw = (n_buckets + SORT_WARPS - 1) / SORT_WARPS;
    if (gw > n_sm * 16) gw = n_sm * 16;
    k_pack_sort_warp<<<gw, SORT_WARPS * 32, smw, s>>>(x, z, dxdy, w, hit_offsets, tmp, n_buckets, ox, oz, odxdy, ow,
                                                      olayer, perm);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    size_t smb = (size_t)BLOCK_SORT_MAX * 20;
    err = cudaFuncSetAttribute(k_pack_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    if (err != cudaSuccess) return err;
    k_pack_sort_block<<<n_sm, BLOCK_SORT_THREADS, smb, s>>>(x, z, dxdy, w, hit_offsets, tmp, big_list, ox, oz, odxdy,
                                                            ow, olayer, perm);
    return cudaGetLastError();
}

}  // namespace lfk
