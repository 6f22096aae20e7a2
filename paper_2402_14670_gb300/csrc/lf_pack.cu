// Hit packing for sm_103a: per event, bucket the raw hits by (zone, layer),
// then sort every bucket by x (ties by raw index) and write the SoA.
//
//   k_pack_bucket   one block per event (grid-stride): each warp counts the
//                   plane codes of its slice of the event (ranked with
//                   __match_any_sync), a per-bucket prefix over buckets and
//                   warps gives the bucket offsets and each warp's cursors,
//                   and each warp scatters its slice in order: a STABLE
//                   scatter of raw indices into bucket order, so inside a
//                   bucket raw indices stay ascending.
//   k_pack_gather   walks the packed positions in order and copies x (with
//                   -0 -> +0), z, dxdy, w into bucket order (coalesced
//                   writes; the raw reads stay inside the events in flight).
//   k_pack_sort_*   buckets of at most 1024 hits by one warp each, larger
//                   ones (at most 8192) by one block each; a bin sort in
//                   shared memory on the contiguous bucket-ordered copy.
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

// Staging of one batch in bucket order: raw index, x (with -0 -> +0), z,
// dxdy, w.
struct Staged {
    int* idx;
    float *x, *z, *d, *w;
};

__global__ void __launch_bounds__(BUCKET_THREADS) k_pack_bucket(
    const int* __restrict__ raw_offsets, const uint8_t* __restrict__ plane, int n_events, int* hit_offsets,
    int* tmp, int* big_list, int* status) {
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
                else if (tot > WARP_MAX) big_list[1 + atomicAdd(big_list, 1)] = e * NB + lane;
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

// Bucket-ordered copy of the hit data: packed positions are walked in order
// (coalesced writes); the raw reads stay inside the few events in flight, so
// they are served by L2.
__global__ void k_pack_gather(const float* __restrict__ x, const float* __restrict__ z,
                              const float* __restrict__ dxdy, const float* __restrict__ w, int n_hits, Staged sg) {
    const int stride = gridDim.x * blockDim.x;
#pragma unroll 4
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_hits; j += stride) {
        const int r = sg.idx[j];
        sg.x[j] = __ldg(x + r) + 0.0f;
        sg.z[j] = __ldg(z + r);
        sg.d[j] = __ldg(dxdy + r);
        sg.w[j] = __ldg(w + r);
    }
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
    uint16_t* pos;    // slot of each element inside its bin
    uint16_t* pos2;   // positions in sorted order
};

// Cooperative bin sort of one bucket by a warp (BLOCK = false) or a block.
template <bool BLOCK>
__device__ void sort_bucket(const Staged& sg, int b0, int m, int layer, float* ox, float* oz, float* od, float* ow,
                            uint8_t* ol, int* perm, SortArea a, int rank, int size, float* red_f, int* red_i) {
    const int lane = rank & 31, wid = rank >> 5, nw = size >> 5;
    float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
#pragma unroll 8
    for (int i = rank; i < m; i += size) {
        float xv = sg.x[b0 + i];
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
    // counting pass; the returned count is the element's slot inside its bin
    for (int i = rank; i < m; i += size) a.pos[i] = (uint16_t)atomicAdd(&a.bins[bin_of(a.xa[i], lo, scale, nb)], 1);
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
    // placement: bins[b] is the start of bin b; slot from the counting pass
    // (positions go to a second array: the first still holds the slots)
    for (int i = rank; i < m; i += size) {
        int d = a.bins[bin_of(a.xa[i], lo, scale, nb)] + a.pos[i];
        a.pos2[d] = (uint16_t)i;
    }
    gsync<BLOCK>();
    // order each bin by (x, position); bin b ends where bin b+1 starts
    for (int bn = rank; bn < nb; bn += size) {
        int s = a.bins[bn], e = bn + 1 < nb ? a.bins[bn + 1] : m;
        for (int i = s + 1; i < e; ++i) {
            int pv = a.pos2[i];
            float xv = a.xa[pv];
            int j = i - 1;
            while (j >= s) {
                int pj = a.pos2[j];
                float xj = a.xa[pj];
                if (!(xv < xj || (xv == xj && pv < pj))) break;
                a.pos2[j + 1] = (uint16_t)pj;
                --j;
            }
            a.pos2[j + 1] = (uint16_t)pv;
        }
    }
    gsync<BLOCK>();
#pragma unroll 4
    for (int i = rank; i < m; i += size) {
        int pv = a.pos2[i];
        size_t o = (size_t)b0 + i, q = (size_t)b0 + pv;
        ox[o] = a.xa[pv];
        oz[o] = sg.z[q];
        od[o] = sg.d[q];
        ow[o] = sg.w[q];
        ol[o] = (uint8_t)layer;
        perm[o] = sg.idx[q];
    }
    gsync<BLOCK>();
}

__host__ __device__ constexpr size_t area_bytes(int n) { return (size_t)n * 12; }

__device__ __forceinline__ SortArea area_at(char* p, int n) {
    SortArea a;
    a.xa = reinterpret_cast<float*>(p);
    a.bins = reinterpret_cast<int*>(p + (size_t)n * 4);
    a.pos = reinterpret_cast<uint16_t*>(p + (size_t)n * 8);
    a.pos2 = reinterpret_cast<uint16_t*>(p + (size_t)n * 10);
    return a;
}

constexpr int SMALL_WARPS = 4;   // warps per block of the small-bucket kernel

// Buckets of at most WARP_MAX hits: one warp each (grid-stride over buckets).
__global__ void __launch_bounds__(SMALL_WARPS * 32) k_pack_sort_small(
    const int* __restrict__ hit_offsets, Staged sg, int n_buckets, float* ox, float* oz, float* od, float* ow,
    uint8_t* ol, int* perm) {
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const SortArea wa = area_at(smem + (size_t)warp * area_bytes(WARP_MAX), WARP_MAX);
    for (int q = blockIdx.x * SMALL_WARPS + warp; q < n_buckets; q += gridDim.x * SMALL_WARPS) {
        int b0 = hit_offsets[q], m = hit_offsets[q + 1] - b0;
        if (m >= 1 && m <= WARP_MAX)
            sort_bucket<false>(sg, b0, m, (q % NB) % NL, ox, oz, od, ow, ol, perm, wa, lane, 32, nullptr, nullptr);
    }
}

// Buckets above WARP_MAX hits (listed by k_pack_bucket): one block each.
__global__ void __launch_bounds__(SORT_THREADS) k_pack_sort_large(
    const int* __restrict__ hit_offsets, const int* __restrict__ list, Staged sg, float* ox, float* oz, float* od,
    float* ow, uint8_t* ol, int* perm) {
    extern __shared__ __align__(16) char smem[];
    __shared__ float red_f[64];
    __shared__ int red_i[32];
    const SortArea ba = area_at(smem, BLOCK_SORT_MAX);
    const int n = list[0];
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        int q = list[1 + k];
        int b0 = hit_offsets[q], m = hit_offsets[q + 1] - b0;
        sort_bucket<true>(sg, b0, m, (q % NB) % NL, ox, oz, od, ow, ol, perm, ba, threadIdx.x, SORT_THREADS, red_f,
                          red_i);
    }
}

}  // namespace

cudaError_t launch_pack(const int* raw_offsets, const float* x, const float* z, const float* dxdy,
                        const float* w, const uint8_t* plane, int n_events, int n_hits,
                        int* hit_offsets, float* ox, float* oz, float* odxdy, float* ow, uint8_t* olayer,
                        int* perm, int* tmp, int* big_list, int* status, int n_sm, cudaStream_t s) {
    if (n_events <= 0) return cudaMemsetAsync(hit_offsets, 0, sizeof(int), s);
    // tmp holds 5 arrays of n_hits 4-byte words: the bucket-ordered staging
    Staged sg;
    sg.idx = tmp;
    sg.x = reinterpret_cast<float*>(tmp + (size_t)n_hits);
    sg.z = sg.x + (size_t)n_hits;
    sg.d = sg.z + (size_t)n_hits;
    sg.w = sg.d + (size_t)n_hits;
    cudaError_t err = cudaMemsetAsync(big_list, 0, sizeof(int), s);
    if (err != cudaSuccess) return err;
    int grid = n_events < n_sm * 8 ? n_events : n_sm * 8;
    k_pack_bucket<<<grid, BUCKET_THREADS, 0, s>>>(raw_offsets, plane, n_events, hit_offsets, tmp, big_list, status);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (n_hits > 0) {
        int gg = (int)(((long)n_hits + 255) / 256);
        if (gg > n_sm * 32) gg = n_sm * 32;
        k_pack_gather<<<gg, 256, 0, s>>>(x, z, dxdy, w, n_hits, sg);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    const int n_buckets = n_events * NB;
    const size_t sms = (size_t)SMALL_WARPS * area_bytes(WARP_MAX);
    if ((err = cudaFuncSetAttribute(k_pack_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms)) !=
        cudaSuccess)
        return err;
    int gsm = (n_buckets + SMALL_WARPS - 1) / SMALL_WARPS;
    if (gsm > n_sm * 32) gsm = n_sm * 32;
    k_pack_sort_small<<<gsm, SMALL_WARPS * 32, sms, s>>>(hit_offsets, sg, n_buckets, ox, oz, odxdy, ow, olayer,
                                                         perm);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const size_t sml = area_bytes(BLOCK_SORT_MAX);
    if ((err = cudaFuncSetAttribute(k_pack_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sml)) !=
        cudaSuccess)
        return err;
    k_pack_sort_large<<<n_sm * 2, SORT_THREADS, sml, s>>>(hit_offsets, big_list, sg, ox, oz, odxdy, ow, olayer,
                                                          perm);
    return cudaGetLastError();
}

}  // namespace lfk
