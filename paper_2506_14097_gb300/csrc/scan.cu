// Device-wide exclusive prefix sum of int32 counts in ONE pass (decoupled
// look-back, scan_tile.cuh).  Used to turn per-item counts or 0/1 flags into
// output positions (pair lists, constraint compaction, incidence CSR) without
// atomics on the positions, so that every list the library builds has a
// deterministic order.
#include "relcp_internal.cuh"
#include "scan_tile.cuh"

namespace relcp {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;

// ctr[0]: tile ticket, ctr[1]: finished blocks
__global__ void __launch_bounds__(kScanThreads) scan_lookback_kernel(const int* __restrict__ in, int64_t n,
                                                                     int* __restrict__ out,
                                                                     unsigned long long* tiles, int* ctr,
                                                                     int* status, int* total_copy) {
    pdl_wait();
    pdl_trigger();
    const int t = tile_scan::take_ticket(ctr);
    const int64_t base = (int64_t)t * kTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    const int inc = tile_scan::block_inclusive_scan(s, &tot);
    const int excl = tile_scan::tile_prefix(t, tot, tiles, status);
    int run = excl + inc - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (t == (int)gridDim.x - 1 && threadIdx.x == 0) {
        out[n] = excl + tot;
        if (total_copy) *total_copy = excl + tot;
    }
    tile_scan::tile_finish(tiles, ctr);
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
    return scan_reserve_tiles(sc, (n + kTile - 1) / kTile, s);
}

relcp_status scan_reserve_tiles(ScanScratch& sc, int64_t ntiles, cudaStream_t s) {
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
