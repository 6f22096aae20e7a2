// Batch validation for debugging (lf_validate_batch): the input conventions
// the find kernels assume but do not check on the hot path.  Each kernel
// records the smallest index that breaks its rule with an atomic minimum, so
// the report names the first violation whatever the launch order.
#include <climits>
#include <cstdint>

#include "lf_internal.h"

namespace lfk {

namespace {

// off[0 .. n]: every entry within [0, total], non-decreasing; with exact_end
// the last entry equals total.  bad <- smallest i whose entry (or step from
// entry i to i + 1) breaks the rule.
__global__ void k_check_offsets(const int* __restrict__ off, int n, int total, bool exact_end, int* bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
        const int v = off[i];
        bool ok = v >= 0 && v <= total;
        if (i < n) ok = ok && v <= off[i + 1];
        if (i == n && exact_end) ok = ok && v == total;
        if (!ok) atomicMin(bad, i);
    }
}

// x ascending inside every bucket [off[q], off[q + 1]) (ties allowed, NaN
// breaks the order); a warp per bucket.  bad <- smallest packed index j with
// !(x[j] <= x[j + 1]) inside one bucket.  The offsets were checked first.
__global__ void k_check_sorted(const int* __restrict__ off, int n_buckets, const float* __restrict__ x, int* bad) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < n_buckets; q += warps) {
        const int s = off[q], e = off[q + 1];
        for (int j = s + lane; j + 1 < e; j += 32)
            if (!(x[j] <= x[j + 1])) atomicMin(bad, j);
    }
}

// x_coarse[i] holds x[32 i] bit for bit for every 32 i < n_hits
__global__ void k_check_coarse(const float* __restrict__ xc, const float* __restrict__ x, int n_hits, int* bad) {
    const int nc = (n_hits + 31) / 32;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
        if (__float_as_uint(xc[i]) != __float_as_uint(x[(size_t)32 * i])) atomicMin(bad, i);
}

int grid_for(long n, int per_block, int n_sm) {
    long g = (n + per_block - 1) / per_block;
    const long cap = 8L * n_sm;
    if (g > cap) g = cap;
    return g > 0 ? (int)g : 1;
}

}  // namespace

cudaError_t launch_validate_offsets(const KBatch& b, int* bad2, int n_sm, cudaStream_t s) {
    k_check_offsets<<<grid_for((long)NB * b.n_events + 1, 256, n_sm), 256, 0, s>>>(b.hit_offsets, NB * b.n_events,
                                                                                      b.n_hits, false, bad2);
    k_check_offsets<<<grid_for((long)b.n_events + 1, 256, n_sm), 256, 0, s>>>(b.trk_offsets, b.n_events, b.n_tracks,
                                                                              true, bad2 + 1);
    return cudaGetLastError();
}

cudaError_t launch_validate_hits(const KBatch& b, int* bad2, int n_sm, cudaStream_t s) {
    if (b.n_hits > 0) {
        k_check_sorted<<<grid_for((long)NB * b.n_events * 32, 256, n_sm), 256, 0, s>>>(b.hit_offsets,
                                                                                        NB * b.n_events, b.x, bad2);
        if (b.x_coarse)
            k_check_coarse<<<grid_for((b.n_hits + 31) / 32, 256, n_sm), 256, 0, s>>>(b.x_coarse, b.x, b.n_hits,
                                                                                     bad2 + 1);
    }
    return cudaGetLastError();
}

}  // namespace lfk
