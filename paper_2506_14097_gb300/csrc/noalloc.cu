// Allocation-free SNSD evaluation (relcp_snsd_eval_noalloc).
//
// Same computation as relcp_snsd_eval, for callers that must not allocate
// device memory: a step running inside a host framework that has reserved the
// whole device pool for its own caching allocator, a real-time loop where an
// allocation (which may synchronise the device) is not allowed, or a plugin
// that may only allocate at initialisation.  Its scratch -- the per-body shape
// matrices and the device status word -- lives in one file-scope device array
// of fixed size instead of being allocated per call.
//
// The array is a per-device object: every GPU that loads this library holds
// RELCP_NOALLOC_SCRATCH_BYTES of it until the process exits.  Host code cannot
// use the array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current)
// and caches it; that first call should therefore happen before any stream
// capture.  All calls share the array and it keeps the last call's contents:
// the status word is cleared at the start of every call, and calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array and must be serialised by the caller.
#include <mutex>

#include "relcp_internal.cuh"

namespace relcp {

namespace {

constexpr int64_t kStatusBytes = 256;  // status word, padded to keep the shape matrices 256-byte aligned
constexpr int64_t kScratchBytes = kStatusBytes + 6 * 8 * (int64_t)RELCP_NOALLOC_MAX_BODIES;
static_assert(kScratchBytes == RELCP_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

relcp_status scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    RELCP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range for the allocation-free scratch table", dev);
        return RELCP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the allocation-free scratch failed: %s", cudaGetErrorString(e));
            return RELCP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return RELCP_OK;
}

}  // namespace

}  // namespace relcp

using namespace relcp;

extern "C" relcp_status relcp_snsd_eval_noalloc(int64_t npairs, const int32_t* pairs, int64_t n, const double* x,
                                                const double* q, const double* axes, const double* box3,
                                                int32_t precision, double* out, int32_t* iters, void* stream) {
    if (npairs < 0 || n < 0 || !box3 || (npairs > 0 && (!pairs || !x || !q || !axes || !out)))
        return set_error("bad argument"), RELCP_ERR_INVALID_ARG;
    if (precision != RELCP_FP64 && precision != RELCP_MIXED) return set_error("bad precision"), RELCP_ERR_INVALID_ARG;
    if (n > RELCP_NOALLOC_MAX_BODIES)
        return set_error("relcp_snsd_eval_noalloc: %lld bodies exceed the fixed scratch limit of %d bodies",
                         (long long)n, (int)RELCP_NOALLOC_MAX_BODIES),
               RELCP_ERR_CAPACITY;
    if (npairs == 0) return RELCP_OK;
    unsigned char* base = nullptr;
    RELCP_TRY(scratch_for_current_device(&base));
    int* status = reinterpret_cast<int*>(base);
    double* P = reinterpret_cast<double*>(base + kStatusBytes);
    cudaStream_t s = (cudaStream_t)stream;
    RELCP_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    RELCP_TRY(shape_launch(n, View<4, const double>::aos(q, 4), View<3, const double>::aos(axes, 3),
                           View<6, double>::soa(P, n), s));
    SnsdArgs a{};
    a.npairs = npairs;
    a.pa = pairs;
    a.pb = pairs + 1;
    a.pstride = 2;
    a.x = View<3, const double>::aos(x, 3);
    a.P = View<6, const double>::soa(P, n);
    for (int k = 0; k < 3; ++k) a.box[k] = box3[k];
    a.guess.c[0] = a.guess.c[1] = a.guess.c[2] = nullptr;
    a.guess.s = 1;
    a.mixed = precision == RELCP_MIXED;
    a.out.phi = out;
    a.out.phi_s = 10;
    a.out.n = View<3, double>::aos(out + 1, 10);
    a.out.ra = View<3, double>::aos(out + 4, 10);
    a.out.rb = View<3, double>::aos(out + 7, 10);
    a.out.iters = iters;
    a.status = status;
    a.maxov_bits = nullptr;
    a.newton_max = nullptr;
    a.iters_sum = nullptr;
    RELCP_TRY(snsd_launch(a, s));
    int bits = 0;
    RELCP_CUDA(cudaMemcpyAsync(&bits, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    RELCP_CUDA(cudaStreamSynchronize(s));
    return status_from_device(bits);
}
