// Device-wide exclusive prefix sum of int32 counts in ONE pass (decoupled
// look-back).  Used to turn per-item counts or 0/1 flags into output positions
// (pair lists, constraint compaction, incidence CSR) without atomics on the
// positions, so that every list the library builds has a deterministic order.
//
// Each block takes a tile ticket from a counter, so tile t is only ever
// processed by a block that started after the blocks of tiles 0..t-1: those
// are resident and never wait on later tiles, hence every wait below ends.
// A tile publishes its aggregate, then its inclusive prefix, as one 64-bit
// word (status in the high half, value in the low half); warp 0 walks back
// over the predecessors 32 at a time (one word per lane), adding aggregates up
// to the nearest inclusive prefix, so a look-back costs one L2 round trip per
// 32 predecessors rather than one per predecessor.
// The spin on a predecessor is bounded: past the limit the block records
// DEV_TIMEOUT in the caller's status word (or the scratch's own) and goes on.
// The last block to finish clears the tile words and the counters, so the next
// call needs no memset (and the launch can be replayed inside a CUDA graph).
#include "relcp_internal.cuh"

namespace relcp {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;
constexpr long long kLookbackLimit = 1ll << 22;
constexpr unsigned long long kAggregate = 1ull << 32, kInclusive = 2ull << 32;

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

__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ctr[0]: tile ticket, ctr[1]: finished blocks
__global__ void __launch_bounds__(kScanThreads) scan_lookback_kernel(const int* __restrict__ in, int64_t n,
                                                                     int* __restrict__ out,
                                                                     unsigned long long* tiles, int* ctr,
                                                                     int* status, int* total_copy) {
    pdl_wait();
    pdl_trigger();
    __shared__ int sh_tile, sh_excl, sh_last;
    if (threadIdx.x == 0) sh_tile = atomicAdd(&ctr[0], 1);
    __syncthreads();
    const int t = sh_tile;
    const int64_t base = (int64_t)t * kTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    const int inc = block_inclusive_scan(s, &tot);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int excl = 0;
        if (t == 0) {
            if (lane == 0) st_relaxed64(tiles, kInclusive | (unsigned)tot);
        } else {
            if (lane == 0) st_relaxed64(tiles + t, kAggregate | (unsigned)tot);
            long long spins = 0;
            bool timed_out = false;
            // window of predecessors t-1-32w-lane; a lane before tile 0 reads
            // an inclusive zero
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
    int run = sh_excl + inc - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (t == (int)gridDim.x - 1 && threadIdx.x == 0) {
        out[n] = sh_excl + tot;
        if (total_copy) *total_copy = sh_excl + tot;
    }
    // the last block to finish clears the tiles and counters for the next call
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

}  // namespace

relcp_status exclusive_scan(const int* in, int* out, int64_t n, ScanScratch& sc, cudaStream_t s, int* total_copy) {
    if (n < 0) return RELCP_ERR_INVALID_ARG;
    if (n == 0) {
        RELCP_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        if (total_copy) RELCP_CUDA(cudaMemsetAsync(total_copy, 0, sizeof(int), s));
        return RELCP_OK;
    }
    const int64_t ntiles = (n + kTile - 1) / kTile;
    if (ntiles > (int64_t)1 << 30) return RELCP_ERR_INVALID_ARG;
    RELCP_TRY(scan_reserve(sc, n, s));
    int* status = sc.status ? sc.status : sc.ctr.p + 2;  // ctr[2]: the scratch's own error word
    note_launch();
    launch_pdl(scan_lookback_kernel, dim3((unsigned)ntiles), dim3(kScanThreads), 0, s, in, n, out, sc.tiles.p,
               sc.ctr.p, status, total_copy);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status scan_reserve(ScanScratch& sc, int64_t n, cudaStream_t s) {
    const int64_t ntiles = (n + kTile - 1) / kTile;
    if (sc.tiles.cap < (size_t)ntiles || !sc.ctr.p) {
        // fresh words must start cleared; afterwards every call leaves them cleared
        RELCP_TRY(sc.tiles.ensure((size_t)(ntiles > 0 ? ntiles : 1), s));
        RELCP_TRY(sc.ctr.ensure(4, s));
        RELCP_CUDA(cudaMemsetAsync(sc.tiles.p, 0, sc.tiles.cap * sizeof(unsigned long long), s));
        RELCP_CUDA(cudaMemsetAsync(sc.ctr.p, 0, 4 * sizeof(int), s));
    }
    return RELCP_OK;
}

relcp_status scan_error(ScanScratch& sc, cudaStream_t s) {
    if (sc.status || !sc.ctr.p) return RELCP_OK;
    int bits = 0;
    RELCP_CUDA(cudaMemcpyAsync(&bits, sc.ctr.p + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    RELCP_CUDA(cudaStreamSynchronize(s));
    if (bits & DEV_TIMEOUT) {
        set_error("prefix-sum look-back timed out");
        return RELCP_ERR_TIMEOUT;
    }
    return RELCP_OK;
}

}  // namespace relcp
