// Building blocks of the single-pass prefix sum (decoupled look-back), for the
// plain scan kernel (scan.cu) and for kernels that compute their counts and
// consume the positions in the same pass (the cached list's filter and
// compaction, broadphase.cu).
//
// Each block takes a tile ticket from a counter, so tile t is only ever
// processed by a block that started after the blocks of tiles 0..t-1: those
// are resident and never wait on later tiles, hence every wait ends.  A tile
// publishes its aggregate, then its inclusive prefix, as one 64-bit word
// (status in the high half, value in the low half); warp 0 walks back over the
// predecessors 32 at a time (one word per lane), adding aggregates up to the
// nearest inclusive prefix, so a look-back costs one L2 round trip per 32
// predecessors.  The spin on a predecessor is bounded: past the limit the
// block records DEV_TIMEOUT in the caller's status word and goes on.  The last
// block to finish clears the tile words and the counters, so the next call
// needs no memset (and a launch can be replayed inside a CUDA graph).
#pragma once

#include "relcp_internal.cuh"

namespace relcp {
namespace tile_scan {

constexpr long long kLookbackLimit = 1ll << 22;
constexpr unsigned long long kAggregate = 1ull << 32, kInclusive = 2ull << 32;

__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// inclusive scan of one value per thread across the block (blockDim.x a
// multiple of 32, at most 1024); returns the inclusive prefix, *total gets
// the block total
__device__ __forceinline__ int block_inclusive_scan(int v, int* total) {
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

// the block's tile (ctr[0]: ticket counter); every thread gets it
__device__ __forceinline__ int take_ticket(int* ctr) {
    __shared__ int sh_tile;
    if (threadIdx.x == 0) sh_tile = atomicAdd(&ctr[0], 1);
    __syncthreads();
    return sh_tile;
}

// the exclusive prefix of tile t, whose own total is tot (every thread gets it)
__device__ __forceinline__ int tile_prefix(int t, int tot, unsigned long long* tiles, int* status) {
    __shared__ int sh_excl;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int excl = 0;
        if (t == 0) {
            if (lane == 0) st_relaxed64(tiles, kInclusive | (unsigned)tot);
        } else {
            if (lane == 0) st_relaxed64(tiles + t, kAggregate | (unsigned)tot);
            long long spins = 0;
            bool timed_out = false;
            // window of predecessors top-lane; a lane before tile 0 reads an
            // inclusive zero
            for (int top = t - 1;;) {
                const int j = top - lane;
                const unsigned long long w = j >= 0 ? ld_relaxed64(tiles + j) : kInclusive;
                const unsigned long long st = w & (3ull << 32);
                if (__any_sync(0xffffffffu, st == 0)) {
                    // a predecessor has not published yet (warp-uniform decision)
                    if (++spins > kLookbackLimit) {
                        timed_out = true;
                        break;
                    }
                    if (spins > 64) __nanosleep(32);
                    continue;
                }
                const unsigned incl = __ballot_sync(0xffffffffu, st == kInclusive);
                const int upto = incl ? __ffs(incl) - 1 : 31;  // nearest inclusive prefix
                int c = lane <= upto ? (int)(unsigned)(w & 0xffffffffull) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                excl += c;
                if (incl) break;
                top -= 32;
            }
            if (lane == 0) {
                if (timed_out) atomicOr(status, DEV_TIMEOUT);
                st_relaxed64(tiles + t, kInclusive | (unsigned)(excl + tot));
            }
        }
        if (lane == 0) sh_excl = excl;
    }
    __syncthreads();
    return sh_excl;
}

// the end of every block: the last one to finish (ctr[1] counts them) clears
// the tile words and both counters for the next call
__device__ __forceinline__ void tile_finish(unsigned long long* tiles, int* ctr) {
    __shared__ int sh_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        sh_last = atomicAdd(&ctr[1], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (sh_last) {
        for (unsigned j = threadIdx.x; j < gridDim.x; j += blockDim.x) st_relaxed64(tiles + j, 0ull);
        if (threadIdx.x == 0) {
            ctr[0] = 0;
            ctr[1] = 0;
        }
        __threadfence();
    }
}

}  // namespace tile_scan
}  // namespace relcp
