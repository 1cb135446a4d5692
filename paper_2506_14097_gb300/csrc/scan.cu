// Device-wide exclusive prefix sum of int32 counts (two passes: tile sums,
// then a tile scan in which every block first adds up the sums of the tiles
// before it -- one load per thread -- so no separate pass scans the tile sums).  Used to turn
// per-item counts or 0/1 flags into output positions (pair lists, constraint
// compaction, incidence CSR) without atomics, so that every list the library
// builds has a deterministic order.
#include "relcp_internal.cuh"

namespace relcp {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kTile = kScanThreads * kScanItems;

// inclusive scan of one value per thread across the block; returns the
// inclusive prefix, *total gets the block total
__device__ int block_inclusive_scan(int v, int* total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    int r = x + (wid > 0 ? warp_sums[wid - 1] : 0);
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return r;
}

__global__ void tile_sums(const int* __restrict__ in, int64_t n, int* __restrict__ partial) {
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    int tot;
    block_inclusive_scan(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// tile scan plus offset; the offset of tile t is the sum of tile sums 0..t-1,
// reduced by this block; the last block writes the total to out[n]
__global__ void tile_scan(const int* __restrict__ in, int64_t n, const int* __restrict__ partial,
                          int* __restrict__ out) {
    int before = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += blockDim.x) before += partial[t];
    int offset;
    block_inclusive_scan(before, &offset);
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    int inc = block_inclusive_scan(s, &tot);
    int run = offset + inc - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = offset + tot;
}

}  // namespace

relcp_status exclusive_scan(const int* in, int* out, int64_t n, ScanScratch& sc, cudaStream_t s) {
    if (n < 0) return RELCP_ERR_INVALID_ARG;
    if (n == 0) {
        RELCP_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        return RELCP_OK;
    }
    const int64_t nparts = (n + kTile - 1) / kTile;
    RELCP_TRY(sc.partial.ensure((size_t)nparts, s));
    note_launch();
    tile_sums<<<(unsigned)nparts, kScanThreads, 0, s>>>(in, n, sc.partial.p);
    RELCP_CUDA(cudaGetLastError());
    note_launch();
    tile_scan<<<(unsigned)nparts, kScanThreads, 0, s>>>(in, n, sc.partial.p, out);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

}  // namespace relcp
