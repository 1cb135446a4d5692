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
};

void set_error(const char* fmt, ...);
relcp_status status_from_device(int bits);
// counts every kernel launch of the library (relcp_kernel_launches)
void note_launch();

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
__device__ __forceinline__ void quat_to_R(double s, double x, double y, double z, double* R) {
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - s * z);
    R[2] = 2.0 * (x * z + s * y);
    R[3] = 2.0 * (x * y + s * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - s * x);
    R[6] = 2.0 * (x * z - s * y);
    R[7] = 2.0 * (y * z + s * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// R diag(w) R^T as a symmetric matrix
__device__ __forceinline__ Sym3<double> rot_diag_rot(const double* R, double w0, double w1, double w2) {
    Sym3<double> P;
    P.xx = R[0] * R[0] * w0 + R[1] * R[1] * w1 + R[2] * R[2] * w2;
    P.yy = R[3] * R[3] * w0 + R[4] * R[4] * w1 + R[5] * R[5] * w2;
    P.zz = R[6] * R[6] * w0 + R[7] * R[7] * w1 + R[8] * R[8] * w2;
    P.xy = R[0] * R[3] * w0 + R[1] * R[4] * w1 + R[2] * R[5] * w2;
    P.xz = R[0] * R[6] * w0 + R[1] * R[7] * w1 + R[2] * R[8] * w2;
    P.yz = R[3] * R[6] * w0 + R[4] * R[7] * w1 + R[5] * R[8] * w2;
    return P;
}

// periodic minimum image of one component (L <= 0: open axis)
__device__ __forceinline__ double min_image(double d, double L) {
    if (L > 0.0) d = __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
    return d;
}

// ---------------------------------------------------------------------------
// device-wide exclusive scan (int32) and helpers (scan.cu)
// ---------------------------------------------------------------------------
struct ScanScratch {
    DBuf<int> partial;
};
// out[i] = sum_{j<i} in[i]; out[n] = total.  `out` has n+1 entries.
relcp_status exclusive_scan(const int* in, int* out, int64_t n, ScanScratch& sc, cudaStream_t s);

// ---------------------------------------------------------------------------
// broad phase (broadphase.cu)
// ---------------------------------------------------------------------------
struct BroadphaseScratch {
    DBuf<int> cell_of, cell_count, cell_start, cell_cursor, cell_body, pair_count, pair_off;
    ScanScratch scan;
};
// Pairs of the bodies whose positions are given by x (any view) and bounding
// radii rb.  Writes pa/pb (grown as needed), *npairs (host; synchronises s).
relcp_status broadphase(int64_t n, View<3, const double> x, const double* rb, const double box[3], double skin,
                        DBuf<int>& pa, DBuf<int>& pb, int64_t* npairs, BroadphaseScratch& sc, cudaStream_t s);

// ---------------------------------------------------------------------------
// SNSD (snsd.cu)
// ---------------------------------------------------------------------------
struct SnsdOut {
    double* phi;
    int64_t phi_s;  // phi of pair p at phi[p * phi_s]
    View<3, double> n, ra, rb;
    int32_t* iters;  // may be null
};
struct SnsdArgs {
    int64_t npairs;
    const int32_t* pa;
    const int32_t* pb;
    int64_t pstride;                 // pair p: (pa[p*pstride], pb[p*pstride])
    View<3, const double> x;         // body centres
    View<6, const double> P;         // shape matrices
    double box[3];
    View<3, const double> guess;     // per-pair start normal (c[0] == nullptr: cold start)
    int mixed;                       // FP32 iterations + FP64 polish
    SnsdOut out;
    // optional overlap test (Phi < -eps): violator flags and per-block max overlap
    double eps;
    int32_t* viol;                   // may be null
    double* block_maxov;             // may be null (one per block)
    int* status;                     // DEV_NEWTON
};
relcp_status snsd_launch(const SnsdArgs& a, int* nblocks_out, cudaStream_t s);

// per-body shape matrices from (possibly unnormalised) quaternions and axes
relcp_status shape_launch(int64_t n, View<4, const double> q, View<3, const double> axes, View<6, double> P,
                          cudaStream_t s);

// ---------------------------------------------------------------------------
// LCP (lcp.cu)
// ---------------------------------------------------------------------------
struct LcpScratch {
    DBuf<int> inc_count, inc_off, inc_cursor, inc;
    DBuf<double> gamma2, g2, partials;   // second gamma buffer, both g buffers
    DBuf<float> gammaf, gf, ucf, geomf;  // mixed-path buffers
    DBuf<unsigned> barrier;
    DBuf<int> status;
    DBuf<double> result;                 // [iters, residual]
    ScanScratch scan;
};
struct LcpProblem {
    int64_t nrows, nbodies;
    const int32_t* ia;
    const int32_t* ib;
    View<9, const double> geom;  // n, r_a x n, r_b x n
    const double* q;             // offsets
    const double* diag;          // A_aa (computed if null -> into scratch)
    View<7, const double> K;     // body operator
    double c;
    int mixed;
    double tol;
    int max_iter;
    double* gamma;               // in: warm start, out: solution (nrows)
    View<6, double> uc;          // out: K D gamma (nbodies)
    bool time_kernel;            // record CUDA events around the persistent launch
};
struct LcpResult {
    int iterations;
    double residual;
    int blocks;
    int dev_status;
    float kernel_ms;             // persistent-kernel time (time_kernel only)
};
// algorithmic bytes of one projected-gradient iteration: every row's
// geometry, offset, diagonal, gamma and g read once and gamma, g written once;
// every body's operator read once and its contact velocity written and read once
inline double lcp_bytes_per_iter(int64_t nrows, int64_t nbodies, bool mixed) {
    return mixed ? 68.0 * nrows + 104.0 * nbodies : 120.0 * nrows + 152.0 * nbodies;
}
relcp_status lcp_solve(const LcpProblem& pr, LcpScratch& sc, LcpResult* res, cudaStream_t s);
relcp_status lcp_diag_launch(int64_t nrows, const int32_t* ia, const int32_t* ib, View<9, const double> geom,
                             View<7, const double> K, double c, double* diag, cudaStream_t s);

int device_sm_count();

}  // namespace relcp
