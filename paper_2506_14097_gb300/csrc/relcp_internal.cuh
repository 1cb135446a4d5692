// Internal declarations of the GB300 ReLCP library (sm_103a).
//
// Data layout in HBM (structure of arrays throughout, one array per scalar
// component so that warps read contiguous 128-byte lines):
//   bodies  : x[3][N], q[4][N], axes[3][N], vel[6][N], fext[6][N] (FP64 state)
//             P[6][N]  shape matrix R diag(a^2) R^T, symmetric (xx,yy,zz,xy,xz,yz)
//             K[7][N]  body operator diag(k_t I, Kr), Kr symmetric
//             Ufree[6][N], Uc[6][N]
//   pairs   : pa[P], pb[P] int32, i-major / j ascending
//   rows    : ia[R], ib[R] int32; geometry n[3], r_a x n [3], r_b x n [3]
//             (FP64, plus an FP32 mirror for the mixed path); offset q[R] and
//             diagonal A_aa[R] in FP64; gamma and g double-buffered
//   incidence CSR: off[N+1], inc[2R] = (row << 1) | side, rows ascending.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "relcp.h"

namespace relcp {

// device status bits (OR-ed by kernels, read back by the host)
enum : int {
    DEV_LCP_NOT_CONVERGED = 1,
    DEV_NEWTON = 2,
    DEV_TIMEOUT = 4,
    DEV_CAPACITY = 8,
    DEV_RECURSION = 16,  // recursion limit reached with violators left (batched scenes)
};

void set_error(const char* fmt, ...);
relcp_status status_from_device(int bits);
// counts every kernel launch of the library (relcp_kernel_launches)
void note_launch();
void note_launches(long long k);  // k launches at once (a replayed graph; negative: captured, not run)

#define RELCP_CUDA(call)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            relcp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return RELCP_ERR_CUDA;                                                                    \
        }                                                                                             \
    } while (0)

#define RELCP_TRY(expr)                      \
    do {                                     \
        relcp_status s_ = (expr);            \
        if (s_ != RELCP_OK) return s_;       \
    } while (0)

// Stream-ordered device buffer owned by a context or a stateless call.
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t cap = 0;
    relcp_status ensure(size_t n, cudaStream_t s, bool keep = false) {
        if (n <= cap && p) return RELCP_OK;
        size_t nc = n < 16 ? 16 : n + n / 2;
        T* np_ = nullptr;
        RELCP_CUDA(cudaMallocAsync((void**)&np_, nc * sizeof(T), s));
        if (keep && p && cap) RELCP_CUDA(cudaMemcpyAsync(np_, p, cap * sizeof(T), cudaMemcpyDeviceToDevice, s));
        if (p) RELCP_CUDA(cudaFreeAsync(p, s));
        p = np_;
        cap = nc;
        return RELCP_OK;
    }
    void release(cudaStream_t s) {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        cap = 0;
    }
};

// Strided view of a K-component array: component k of item i at c[k][i*s].
template <int NC, class T>
struct View {
    T* c[NC];
    int64_t s;
    __host__ __device__ T& operator()(int k, int64_t i) const { return c[k][i * s]; }
    static View soa(T* base, int64_t n) {
        View v;
        for (int k = 0; k < NC; ++k) v.c[k] = base + (int64_t)k * n;
        v.s = 1;
        return v;
    }
    static View aos(T* base, int width) {
        View v;
        for (int k = 0; k < NC; ++k) v.c[k] = base + k;
        v.s = width;
        return v;
    }
};

// ---------------------------------------------------------------------------
// small device math
// ---------------------------------------------------------------------------
template <class T>
struct Sym3 {
    T xx, yy, zz, xy, xz, yz;
};

template <class T>
__device__ __forceinline__ void symv(const Sym3<T>& P, const T* n, T* v) {
    v[0] = P.xx * n[0] + P.xy * n[1] + P.xz * n[2];
    v[1] = P.xy * n[0] + P.yy * n[1] + P.yz * n[2];
    v[2] = P.xz * n[0] + P.yz * n[1] + P.zz * n[2];
}

template <class T>
__device__ __forceinline__ T dot3(const T* a, const T* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <class T>
__device__ __forceinline__ void cross3(const T* a, const T* b, T* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Rotation of the normalised quaternion (s, w), Hamilton, body -> world.
template <class T>
__device__ __forceinline__ void quat_to_R(T s, T x, T y, T z, T* R) {
    R[0] = T(1) - T(2) * (y * y + z * z);
    R[1] = T(2) * (x * y - s * z);
    R[2] = T(2) * (x * z + s * y);
    R[3] = T(2) * (x * y + s * z);
    R[4] = T(1) - T(2) * (x * x + z * z);
    R[5] = T(2) * (y * z - s * x);
    R[6] = T(2) * (x * z - s * y);
    R[7] = T(2) * (y * z + s * x);
    R[8] = T(1) - T(2) * (x * x + y * y);
}

// R diag(w) R^T as a symmetric matrix
template <class T>
__device__ __forceinline__ Sym3<T> rot_diag_rot(const T* R, T w0, T w1, T w2) {
    Sym3<T> P;
    P.xx = R[0] * R[0] * w0 + R[1] * R[1] * w1 + R[2] * R[2] * w2;
    P.yy = R[3] * R[3] * w0 + R[4] * R[4] * w1 + R[5] * R[5] * w2;
    P.zz = R[6] * R[6] * w0 + R[7] * R[7] * w1 + R[8] * R[8] * w2;
    P.xy = R[0] * R[3] * w0 + R[1] * R[4] * w1 + R[2] * R[5] * w2;
    P.xz = R[0] * R[6] * w0 + R[1] * R[7] * w1 + R[2] * R[8] * w2;
    P.yz = R[3] * R[6] * w0 + R[4] * R[7] * w1 + R[5] * R[8] * w2;
    return P;
}

// Periodic minimum image of one component, d - L * rint(d / L) (rint rounds
// half to even; L <= 0: open axis), every operation rounded separately.
// The image index k = rint(d / L) is decided by comparing |d| with L/2 and
// 3L/2, which gives the same k as the rounded quotient except within a
// relative 1e-12 of a tie; only there is the FP64 division evaluated (FP64
// division is slow on this part).  The result is bit-identical to the direct
// formula for every input.
__device__ __forceinline__ double min_image(double d, double L) {
    if (!(L > 0.0)) return d;
    const double ad = fabs(d);
    const double h = 0.5 * L;  // exact
    double k;
    if (ad < h * (1.0 - 1e-12)) {
        return d;  // k = 0
    } else if (ad > h * (1.0 + 1e-12) && ad < 3.0 * h * (1.0 - 1e-12)) {
        k = d > 0.0 ? 1.0 : -1.0;
    } else {
        k = rint(__ddiv_rn(d, L));
    }
    return __dsub_rn(d, __dmul_rn(L, k));
}

// The candidate test of the broad phase: |min_image(x_j - x_i)|^2 <=
// (rb_i + rb_j + skin)^2 as a fixed sequence of separately rounded FP64
// operations (no contraction), so the decision is reproducible bit for bit.
__device__ __forceinline__ bool near_pair_exact(double xi0, double xi1, double xi2, double xj0, double xj1,
                                                double xj2, double rbi, double rbj, double L0, double L1, double L2,
                                                double skin) {
    const double dx = min_image(__dsub_rn(xj0, xi0), L0);
    const double dy = min_image(__dsub_rn(xj1, xi1), L1);
    const double dz = min_image(__dsub_rn(xj2, xi2), L2);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double s = __dadd_rn(__dadd_rn(rbi, rbj), skin);
    return d2 <= __dmul_rn(s, s);
}

// A double truncated to FP32 by integer operations (FP64 conversions issue at
// the FP64 rate on this part): relative error below 2^-23 for a normal value in
// the FP32 range, exact for a widened float; other values by conversion.
__device__ __forceinline__ float trunc_f32(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ffull) - 1023 + 127;
    if (e <= 0 || e >= 255) return (float)d;
    return __uint_as_float(((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)e << 23) |
                           (unsigned)((b >> 29) & 0x7fffffull));
}

// near_pair_exact's decision, taken in FP32 where a rounding-error bound
// certifies it.  From the positions and radii truncated to FP32 (relative
// error < 2^-23 each), the per-axis difference, minimum image (the FP32 image
// may differ from the FP64 one only where |d| is near L/2, and the distance
// is continuous across that switch) and the sum of squares give a distance
// within 2^-22 (|x_i| + |x_j| + L) per axis of the FP64 one, and the radius sum
// within 2^-22 s.  m = 2^-19 (max |x_i| + max |x_j| + max L + s) exceeds the
// distance error more than fourfold: a pair further than s + m is out, one
// nearer than s - m is in, and only the pairs in between take the FP64 test.
__device__ __forceinline__ bool near_pair_fast(double xi0, double xi1, double xi2, double xj0, double xj1, double xj2,
                                               double rbi, double rbj, double L0, double L1, double L2, double skin,
                                               const float* Lf, const float* iLf, float Lmaxf, float skinf) {
    const float a0 = trunc_f32(xi0), a1 = trunc_f32(xi1), a2 = trunc_f32(xi2);
    const float b0 = trunc_f32(xj0), b1 = trunc_f32(xj1), b2 = trunc_f32(xj2);
    float d0 = b0 - a0, d1 = b1 - a1, d2 = b2 - a2;
    if (Lf[0] > 0.f) d0 -= Lf[0] * rintf(d0 * iLf[0]);
    if (Lf[1] > 0.f) d1 -= Lf[1] * rintf(d1 * iLf[1]);
    if (Lf[2] > 0.f) d2 -= Lf[2] * rintf(d2 * iLf[2]);
    const float dd = d0 * d0 + d1 * d1 + d2 * d2;
    const float sf = trunc_f32(rbi) + trunc_f32(rbj) + skinf;
    const float A = fmaxf(fabsf(a0), fmaxf(fabsf(a1), fabsf(a2))) + fmaxf(fabsf(b0), fmaxf(fabsf(b1), fabsf(b2)));
    const float m = 0x1p-19f * (A + Lmaxf + sf);
    const float hi = sf + m;
    if (dd > hi * hi) return false;
    const float lo = sf - m;
    if (lo > 0.f && dd < lo * lo) return true;
    return near_pair_exact(xi0, xi1, xi2, xj0, xj1, xj2, rbi, rbj, L0, L1, L2, skin);
}

// ---------------------------------------------------------------------------
// programmatic dependent launch: a kernel launched with launch_pdl may start
// while the previous kernel in the stream drains (its launch overlaps that
// kernel's tail); it executes pdl_wait() before touching anything earlier
// work in the stream wrote (the wait returns once that kernel has completed
// and its writes are visible), then pdl_trigger() to let its own dependents
// start launching.  Both are no-ops for a kernel launched the ordinary way.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---------------------------------------------------------------------------
// device-wide exclusive scan (int32) and helpers (scan.cu)
// ---------------------------------------------------------------------------
struct ScanScratch {
    DBuf<unsigned long long> tiles;  // per-tile look-back words (left cleared by every call)
    DBuf<int> ctr;                   // ticket, finished blocks, own error word
    int* status = nullptr;           // DEV_TIMEOUT goes here if set (else into ctr[2])
};
// out[i] = sum_{j<i} in[i]; out[n] = total.  `out` has n+1 entries.
// out[0..n] = exclusive prefix sums of in[0..n) and the total; the total is
// also written to *total_copy when that is not null
relcp_status exclusive_scan(const int* in, int* out, int64_t n, ScanScratch& sc, cudaStream_t s,
                            int* total_copy = nullptr);
// RELCP_ERR_TIMEOUT if a scan on this scratch (without a status word) timed
// out; synchronises s
relcp_status scan_error(ScanScratch& sc, cudaStream_t s);
// size the scratch for scans of up to n items (a later scan allocates nothing)
relcp_status scan_reserve(ScanScratch& sc, int64_t n, cudaStream_t s);
// the same for a kernel of its own with `ntiles` look-back tiles (scan_tile.cuh)
relcp_status scan_reserve_tiles(ScanScratch& sc, int64_t ntiles, cudaStream_t s);
inline void release(ScanScratch& sc, cudaStream_t s) {
    sc.tiles.release(s);
    sc.ctr.release(s);
}

// ---------------------------------------------------------------------------
// broad phase (broadphase.cu)
// ---------------------------------------------------------------------------
// What a step leaves for the next one about a pair of the cached candidate
// list: the step number, the pair's index in that step (its row of the SNSD
// output of the step's last overlap test) and the final gamma of its A_0 row
// (0 when it had none).
struct PairMemo {
    int stamp;
    int pidx;
    double gamma;
};

struct BroadphaseScratch {
    DBuf<int> cell_of, cell_count, cell_start, cell_cursor, cell_body, pair_count, pair_off;
    DBuf<float4> cell_xr;  // FP32 wrapped positions and radii in cell order (superset test)
    ScanScratch scan;
    // Verlet candidate list (context use): pairs within R_i + R_j + skin + delta
    // at the build positions xb in the build box Lb, sorted by (i, j)
    DBuf<int> vpa, vpb, vflag, vscan;
    // per-entry memo, carried to the new list (by pair key) when it is rebuilt
    DBuf<PairMemo> memo;
    DBuf<int> vpa_old, vpb_old;
    DBuf<PairMemo> memo_old;
    DBuf<int> pv;  // candidate pair p -> its entry of the cached list
    DBuf<double> xb;
    DBuf<unsigned long long> dmax;  // bits of the largest displacement since the build
    int64_t vn = 0, vn_bodies = -1;
    double Lb[3] = {0, 0, 0}, skin_b = -1.0, delta = 0.0;
    bool valid = false;
    int rebuilds = 0;
};
// Pairs of the bodies whose positions are given by x (any view) and bounding
// radii rb.  Writes pa/pb (grown as needed), *npairs (host; synchronises s).
// rbmax: the largest rb if known (> 0), else it is reduced on the device.
// superset: a list that may also hold pairs up to a small margin beyond the
// cutoff (FP32 test; cell-list path only), for the cached list's rebuild.
relcp_status broadphase(int64_t n, View<3, const double> x, const double* rb, double rbmax, const double box[3],
                        double skin, DBuf<int>& pa, DBuf<int>& pb, int64_t* npairs, BroadphaseScratch& sc,
                        cudaStream_t s, bool superset = false);
// The same pair list through a cached Verlet list (x in SoA layout, n bodies,
// rbmax known).  Rebuilds the cache when the displacement bound requires it;
// sc.pv maps each pair to its list entry, sc.memo is indexed by entry.
relcp_status broadphase_cached(int64_t n, const double* x_soa, const double* rb, double rbmax, const double box[3],
                               double skin, DBuf<int>& pa, DBuf<int>& pb, int64_t* npairs, BroadphaseScratch& sc,
                               cudaStream_t s);
// Whether the cached list is complete for positions whose largest displacement
// since the build is dmax, in the box `box` (the bound of broadphase_cached).
bool verlet_bound_holds(const BroadphaseScratch& sc, int64_t n, const double box[3], double rbmax, double skin,
                        double dmax);
// the scale factors of that check (false: no valid cached list), for kernels
// that fold the check into their own pass over the bodies (the trial pass)
bool broadphase_lookahead_params(const BroadphaseScratch& sc, int64_t n, const double box[3], double sfac[3]);
// The cached list's exact filter and compaction without a host round trip:
// pairs into pa, pb, sc.pv (capacity sc.vn), their count at sc.vscan.p[sc.vn].
// Valid only when the bound held for these positions (checked beforehand).
// box_dev (may be null): the box read on the device instead of `box`;
// np_copy (may be null): a second word that receives the count.  Its look-back
// tiles: broadphase_filter_tiles(sc.vn) words of sc.scan (scan_reserve_tiles)
int64_t broadphase_filter_tiles(int64_t nv);
relcp_status broadphase_filter_async(int64_t n, const double* x_soa, const double* rb, const double box[3],
                                     const double* box_dev, double skin, DBuf<int>& pa, DBuf<int>& pb,
                                     BroadphaseScratch& sc, cudaStream_t s, int* np_copy = nullptr);

// ---------------------------------------------------------------------------
// SNSD (snsd.cu)
// ---------------------------------------------------------------------------
struct SnsdOut {
    double* phi;
    int64_t phi_s;  // phi of pair p at phi[p * phi_s]
    View<3, double> n, ra, rb;
    int32_t* iters;  // may be null
};
// Per-step scalars read by the step's kernels from device memory, so that the
// kernels' arguments stay the same from step to step (CUDA-graph replay).
struct StepConst {
    double box0[3];  // box at C^k
    double box1[3];  // box at the trial configurations / C^{k+1}
    double sfac[3];  // box1 / the cached pair list's build box
    int stamp_prev;  // memo stamp of the previous step (-1: none)
    int pad;
};

struct SnsdArgs {
    int64_t npairs;
    const int32_t* pa;
    const int32_t* pb;
    int64_t pstride;                 // pair p: (pa[p*pstride], pb[p*pstride])
    View<3, const double> x;         // body centres
    View<6, const double> P;         // shape matrices
    double box[3];
    const double* box_dev;           // if set, the box is read here (device) instead
    View<3, const double> guess;     // per-pair start normal (c[0] == nullptr: cold start)
    const int* guess_on;             // if set, the start normals are used only when *guess_on != 0
    // optional pair subset: thread k < *count_dev evaluates pair idx[k] (its
    // start normal is guess(., k)); idx == nullptr: thread p evaluates pair p
    const int* idx;
    const int* count_dev;
    int mixed;                       // FP32 iterations + FP64 polish
    SnsdOut out;
    // optional overlap test (Phi < -eps): violator flags and the largest overlap
    double eps;
    int32_t* viol;                   // may be null
    unsigned long long* maxov_bits;  // may be null: atomicMax of the bits of max(0, -Phi) (>= 0 doubles
                                     // order like their bit patterns)
    int* nviol;                      // may be null: atomicAdd of the number of violators
    int* newton_max;                 // may be null: atomicMax of the Newton iteration counts
    unsigned long long* iters_sum;   // may be null: sum of the Newton iteration counts
    int* status;                     // DEV_NEWTON
    int newton_cap;                  // > 0: Newton iteration cap of every phase (fault injection)
    int shape;                       // RELCP_SHAPE_* (P holds the shape records of step_math::shape_record)
};
relcp_status snsd_launch(const SnsdArgs& a, cudaStream_t s);

// per-body shape matrices from (possibly unnormalised) quaternions and axes
relcp_status shape_launch(int64_t n, View<4, const double> q, View<3, const double> axes, View<6, double> P,
                          cudaStream_t s);

// ---------------------------------------------------------------------------
// LCP (lcp.cu)
// ---------------------------------------------------------------------------
struct LcpScratch {
    DBuf<int> inc_count;  // per body: incidence count, fill cursor; then the two grid-barrier counters
    DBuf<int> inc_off, inc_tmp, inc;
    DBuf<double> packd;              // FP64: packed (gamma, g) pairs x 2 buffers + contact-velocity records
    DBuf<float> packf;               // mixed: the same in FP32
    DBuf<double> g64;                // mixed: the FP64 offsets of the refinement's correction problem
    DBuf<double> partials;
    ScanScratch scan;
};
// Filled by the persistent kernel; read by the caller whenever it synchronises.
struct LcpDevResult {
    double iterations;
    double residual;
};
struct LcpProblem {
    int64_t m_cap;               // number of rows <= m_cap (grid sizing)
    const int* nrows_dev;        // device-side number of rows
    int64_t nbodies;
    const int32_t* ia;
    const int32_t* ib;
    const void* geom[9];         // SoA rows: n, r_a x n, r_b x n (double, or float when mixed)
    const double* q;             // offsets (FP64)
    const void* qr;              // offsets in the solve precision (== q on the FP64 path)
    const double* diag;          // A_aa
    const void* invd;            // 1 / A_aa in the solve precision: Jacobi-scaled steps, or null
    const double* K[7];          // SoA body operator (FP64)
    const void* Kr[7];           // the same in the solve precision (== K on the FP64 path)
    double c;
    int mixed;
    double tol;
    int max_iter;
    void* gamma;                 // SoA, solve precision: in = warm start (>= 0), out = solution
    double* uc[6];               // SoA output K D gamma (double)
    LcpDevResult* result;        // device
    int* status;                 // device status word (DEV_* bits OR-ed)
    cudaEvent_t ev_before;       // recorded right before / after the persistent launch (or null)
    cudaEvent_t ev_after;
    // every device wait of the launch gives up after this many nanoseconds
    // (0: kLcpWaitNs) and sets DEV_TIMEOUT
    unsigned long long wait_ns;
    int fault_skip_block;        // fault injection: the last block leaves before its first barrier arrival
    // mixed path: iterative refinement (FP32 iterations to kRefineFactor x tol,
    // an FP64 residual, an FP32 correction solve to tol); 0 turns it off
    int refine = 1;
};
#ifndef RELCP_REFINE_FACTOR
#define RELCP_REFINE_FACTOR 10.0
#endif
constexpr double kRefineFactor = RELCP_REFINE_FACTOR;
constexpr unsigned long long kLcpWaitNs = 2000000000ull;  // 2 s
constexpr unsigned long long kFaultWaitNs = 2000000ull;   // 2 ms (RELCP_FAULT_LCP_TIMEOUT)
// lcp_solve in two parts: the body incidence CSR of the rows, then the
// persistent solve (the second may be launched apart from the first, e.g.
// between timing events while the first is part of a captured graph)
relcp_status lcp_build_csr(const LcpProblem& pr, LcpScratch& sc, cudaStream_t s);
relcp_status lcp_run(const LcpProblem& pr, LcpScratch& sc, int* blocks, cudaStream_t s);
// size every buffer of lcp_solve for up to m_cap rows and nb bodies
relcp_status lcp_reserve(LcpScratch& sc, int64_t m_cap, int64_t nb, bool mixed, cudaStream_t s);
relcp_status lcp_solve(const LcpProblem& pr, LcpScratch& sc, int* blocks, float* kernel_ms, cudaStream_t s);
relcp_status lcp_diag_launch(int64_t nrows, const int32_t* ia, const int32_t* ib, View<9, const double> geom,
                             View<7, const double> K, double c, double* diag, cudaStream_t s);
// algorithmic bytes of one projected-gradient iteration: every row's
// geometry, offset, diagonal, gamma and g read once and gamma, g written once;
// every body's operator read once and its contact velocity written and read once
// Algorithmic bytes of one projected-gradient iteration: per row the ids
// (8 B), the row's 9 geometry scalars, its offset, gamma, the previous gamma
// and g read and gamma and g written (FP64: 136 B; FP32 geometry and iterates
// with an FP64 offset: 76 B); per body its operator K, the contact velocity
// written and read and the wrench (FP64: 150 B; FP32: 75 B).
inline double lcp_bytes_per_iter(int64_t nrows, int64_t nbodies, bool mixed) {
    return mixed ? 76.0 * nrows + 75.0 * nbodies : 136.0 * nrows + 150.0 * nbodies;
}
void release(LcpScratch& sc, cudaStream_t s);
int lcp_threads();  // threads per CTA of the persistent LCP kernel
relcp_status narrow_launch(const double* in, float* out, int64_t n, cudaStream_t s);
relcp_status widen_launch(const float* in, double* out, int64_t n, cudaStream_t s);

int device_sm_count();

}  // namespace relcp
