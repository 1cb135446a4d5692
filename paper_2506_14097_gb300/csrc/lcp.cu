// Matrix-free LCP solve on the contact operator (Eq. cqpp; Lemma LCP <=> CQP):
//     find gamma >= 0 with g = q + c D^T K D gamma >= 0 and gamma . g = 0,
// i.e. the minimiser of 1/2 gamma^T A gamma + q^T gamma over gamma >= 0 with
// A = c D^T K D, by projected gradient with Barzilai-Borwein steps (the paper
// lists projected gradient among the admissible CQP solvers, Sec. 2.1.3).
//
// One persistent cooperative launch runs the whole solve.  Per iteration:
//   phase 1 (one thread per body, incidence CSR, no atomics): for every row
//     a incident to the body, gamma'_a = max(0, gamma_a - alpha g_a); the
//     body wrench w = sum (+-n, +-r x n) gamma'_a; contact velocity
//     Uc = K w.  The side-a thread stores gamma'_a.
//   grid barrier
//   phase 2 (one thread per row): g'_a = q_a + c d_a^T Uc, the BB inner
//     products s^T s, s^T y, y^T y (s = gamma' - gamma, y = g' - g = A s) and
//     the FP64 natural residual max |min(A_aa gamma'_a, g'_a)|, reduced per
//     block in a fixed order.
//   grid barrier; every block reduces the per-block partials in the same
//     fixed order, so all blocks take identical decisions and the result is
//     bit-for-bit reproducible.
// Steps alternate BB1 = s^T s / s^T y and BB2 = s^T y / y^T y.  The grid
// barrier spins a bounded number of times; a timeout sets DEV_TIMEOUT and the
// kernel returns.  Data written inside the launch is read with ld.global.cg
// (L2), never from a possibly stale L1 line.
#include <cooperative_groups.h>

#include "relcp_internal.cuh"

namespace relcp {

namespace {

constexpr int kThreads = 256;
constexpr int kNred = 4;  // ss, sy, yy, residual-or-maxdiag
constexpr long long kSpinLimit = 1ll << 24;

template <class R>
struct KArgs {
    int nrows, nbodies;
    const int* __restrict__ ia;
    const int* __restrict__ ib;
    const R* geom[9];
    const double* __restrict__ q;
    const double* __restrict__ diag;
    const double* K[7];
    const int* __restrict__ inc_off;
    const int* __restrict__ inc;
    R* gam[2];
    R* g[2];
    R* uc[6];
    int64_t uc_stride;
    double c, tol;
    int max_iter;
    double* partials;
    unsigned* bar;
    int* status;
    double* result;  // iterations, residual, final buffer
};

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

// bounded sense-free grid barrier (count + generation); false on timeout
__device__ bool grid_barrier(unsigned* bar, int* status) {
    __shared__ int timed_out;
    __syncthreads();
    if (threadIdx.x == 0) {
        timed_out = 0;
        volatile unsigned* vgen = bar + 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (++spins > kSpinLimit) {
                    atomicOr(status, DEV_TIMEOUT);
                    timed_out = 1;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*((volatile int*)status) & DEV_TIMEOUT) timed_out = 1;
    }
    __syncthreads();
    return timed_out == 0;
}

// deterministic block reduction of kNred values; slot k is a max when bit k
// of maxmask is set, a sum otherwise
__device__ void block_reduce_store(const double v[kNred], unsigned maxmask, double* out) {
    __shared__ double sh[kThreads / 32][kNred];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kNred; ++k) {
        double x = v[k];
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, o);
            x = ((maxmask >> k) & 1u) ? fmax(x, y) : x + y;
        }
        if (lane == 0) sh[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < kNred) {
        int k = threadIdx.x;
        double x = sh[0][k];
        for (int w = 1; w < kThreads / 32; ++w) x = ((maxmask >> k) & 1u) ? fmax(x, sh[w][k]) : x + sh[w][k];
        out[k] = x;
    }
    __syncthreads();
}

// every block: reduce all blocks' partials in a fixed order
__device__ void grid_reduce(const double* partials, unsigned maxmask, double tot[kNred]) {
    __shared__ double res[kNred];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double acc[kNred] = {0, 0, 0, 0};
        for (int b = lane; b < (int)gridDim.x; b += 32) {
#pragma unroll
            for (int k = 0; k < kNred; ++k) {
                double x = __ldcg(partials + (size_t)b * kNred + k);
                acc[k] = ((maxmask >> k) & 1u) ? fmax(acc[k], x) : acc[k] + x;
            }
        }
#pragma unroll
        for (int k = 0; k < kNred; ++k) {
            double x = acc[k];
            for (int o = 16; o > 0; o >>= 1) {
                double y = __shfl_down_sync(0xffffffffu, x, o);
                x = ((maxmask >> k) & 1u) ? fmax(x, y) : x + y;
            }
            if (lane == 0) res[k] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kNred; ++k) tot[k] = res[k];
    __syncthreads();
}

// phase 1: contact velocity of gamma' = P(src - alpha g) (alpha < 0: gamma' = src)
template <class R>
__device__ void scatter_phase(const KArgs<R>& a, const R* src, const R* gsrc, double alpha, R* dst) {
    const int stride = gridDim.x * blockDim.x;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < a.nbodies; b += stride) {
        R f0 = 0, f1 = 0, f2 = 0, t0 = 0, t1 = 0, t2 = 0;
        const int e0 = a.inc_off[b], e1 = a.inc_off[b + 1];
        for (int e = e0; e < e1; ++e) {
            const int code = a.inc[e];
            const int r = code >> 1;
            const bool sideb = code & 1;
            R gm = ldcg(src + r);
            if (alpha >= 0.0) {
                R v = gm - (R)alpha * ldcg(gsrc + r);
                gm = v > R(0) ? v : R(0);
                if (!sideb) dst[r] = gm;
            }
            const R n0 = a.geom[0][r], n1 = a.geom[1][r], n2 = a.geom[2][r];
            const int o = sideb ? 6 : 3;
            const R s0 = a.geom[o][r], s1 = a.geom[o + 1][r], s2 = a.geom[o + 2][r];
            const R sg = sideb ? gm : -gm;
            f0 += sg * n0;
            f1 += sg * n1;
            f2 += sg * n2;
            t0 += sg * s0;
            t1 += sg * s1;
            t2 += sg * s2;
        }
        const R kt = (R)a.K[0][b];
        const R kxx = (R)a.K[1][b], kyy = (R)a.K[2][b], kzz = (R)a.K[3][b];
        const R kxy = (R)a.K[4][b], kxz = (R)a.K[5][b], kyz = (R)a.K[6][b];
        const int64_t o = (int64_t)b * a.uc_stride;
        a.uc[0][o] = kt * f0;
        a.uc[1][o] = kt * f1;
        a.uc[2][o] = kt * f2;
        a.uc[3][o] = kxx * t0 + kxy * t1 + kxz * t2;
        a.uc[4][o] = kxy * t0 + kyy * t1 + kyz * t2;
        a.uc[5][o] = kxz * t0 + kyz * t1 + kzz * t2;
    }
}

// phase 2: g' for gamma' (gnew), BB products against (gold, gprev), residual
template <class R>
__device__ void gather_phase(const KArgs<R>& a, const R* gnew, const R* gold, const R* gprev, R* gout,
                             double v[kNred]) {
    const int stride = gridDim.x * blockDim.x;
    v[0] = v[1] = v[2] = v[3] = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.nrows; r += stride) {
        const int i = a.ia[r], j = a.ib[r];
        const int64_t oi = (int64_t)i * a.uc_stride, oj = (int64_t)j * a.uc_stride;
        const R n0 = a.geom[0][r], n1 = a.geom[1][r], n2 = a.geom[2][r];
        R du0 = ldcg(a.uc[0] + oj) - ldcg(a.uc[0] + oi);
        R du1 = ldcg(a.uc[1] + oj) - ldcg(a.uc[1] + oi);
        R du2 = ldcg(a.uc[2] + oj) - ldcg(a.uc[2] + oi);
        R rate = n0 * du0 + n1 * du1 + n2 * du2;
        rate += a.geom[6][r] * ldcg(a.uc[3] + oj) + a.geom[7][r] * ldcg(a.uc[4] + oj) + a.geom[8][r] * ldcg(a.uc[5] + oj);
        rate -= a.geom[3][r] * ldcg(a.uc[3] + oi) + a.geom[4][r] * ldcg(a.uc[4] + oi) + a.geom[5][r] * ldcg(a.uc[5] + oi);
        const double gd = a.q[r] + a.c * (double)rate;
        const double gm = (double)ldcg(gnew + r);
        gout[r] = (R)gd;
        if (gold) {
            const double s = gm - (double)ldcg(gold + r);
            const double y = gd - (double)ldcg(gprev + r);
            v[0] += s * s;
            v[1] += s * y;
            v[2] += y * y;
        }
        const double nat = fabs(fmin(a.diag[r] * gm, gd));
        v[3] = fmax(v[3], nat);
    }
}

template <class R>
__global__ void __launch_bounds__(kThreads) lcp_kernel(KArgs<R> a) {
    __shared__ double part[kNred];
    double v[kNred];
    double tot[kNred];
    // ---- init: Uc = K D gamma0, g0, residual, max diagonal
    scatter_phase(a, a.gam[0], (const R*)nullptr, -1.0, (R*)nullptr);
    if (!grid_barrier(a.bar, a.status)) return;
    gather_phase(a, a.gam[0], (const R*)nullptr, (const R*)nullptr, a.g[0], v);
    {
        // init reduces two maxima: slot 0 = largest A_aa, slot 3 = residual
        double md = 0.0;
        const int stride = gridDim.x * blockDim.x;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < a.nrows; r += stride) md = fmax(md, a.diag[r]);
        double w[kNred] = {md, 0.0, 0.0, v[3]};
        block_reduce_store(w, 0x9u, part);
        if (threadIdx.x == 0)
            for (int k = 0; k < kNred; ++k) a.partials[(size_t)blockIdx.x * kNred + k] = part[k];
    }
    if (!grid_barrier(a.bar, a.status)) return;
    grid_reduce(a.partials, 0x9u, tot);
    double resid = tot[3];
    const double maxdiag = tot[0];
    int cur = 0, it = 0;
    double alpha = maxdiag > 0.0 ? 1.0 / maxdiag : 1.0;
    if (!(resid <= a.tol)) {
        for (it = 1; it <= a.max_iter; ++it) {
            // all blocks have read partials before any block rewrites them:
            // the barrier after phase 1 separates the reads from the writes
            scatter_phase(a, a.gam[cur], a.g[cur], alpha, a.gam[1 - cur]);
            if (!grid_barrier(a.bar, a.status)) return;
            gather_phase(a, a.gam[1 - cur], a.gam[cur], a.g[cur], a.g[1 - cur], v);
            block_reduce_store(v, 0x8u, part);
            if (threadIdx.x == 0)
                for (int k = 0; k < kNred; ++k) a.partials[(size_t)blockIdx.x * kNred + k] = part[k];
            if (!grid_barrier(a.bar, a.status)) return;
            grid_reduce(a.partials, 0x8u, tot);
            cur = 1 - cur;
            resid = tot[3];
            if (resid <= a.tol) break;
            const double ss = tot[0], sy = tot[1], yy = tot[2];
            double na;
            if (it & 1) na = (sy > 0.0) ? ss / sy : alpha;
            else na = (yy > 0.0 && sy > 0.0) ? sy / yy : alpha;
            if (isfinite(na) && na > 0.0) alpha = na;
        }
        if (it > a.max_iter) it = a.max_iter;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.result[0] = (double)it;
        a.result[1] = resid;
        a.result[2] = (double)cur;
        if (!(resid <= a.tol)) atomicOr(a.status, DEV_LCP_NOT_CONVERGED);
    }
}

// ---- incidence CSR (rows ascending within each body)
__global__ void inc_count(int64_t nrows, const int* __restrict__ ia, const int* __restrict__ ib, int* __restrict__ cnt) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    atomicAdd(&cnt[ia[r]], 1);
    atomicAdd(&cnt[ib[r]], 1);
}

__global__ void inc_fill(int64_t nrows, const int* __restrict__ ia, const int* __restrict__ ib,
                         const int* __restrict__ off, int* __restrict__ cursor, int* __restrict__ inc) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int a = ia[r], b = ib[r];
    inc[off[a] + atomicAdd(&cursor[a], 1)] = (int)(r << 1);
    inc[off[b] + atomicAdd(&cursor[b], 1)] = (int)(r << 1) | 1;
}

__global__ void inc_sort(int64_t nbodies, const int* __restrict__ off, int* __restrict__ inc) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbodies) return;
    int e0 = off[b], e1 = off[b + 1];
    for (int k = e0 + 1; k < e1; ++k) {
        int v = inc[k];
        int m = k - 1;
        while (m >= e0 && inc[m] > v) {
            inc[m + 1] = inc[m];
            --m;
        }
        inc[m + 1] = v;
    }
}

__global__ void diag_kernel(int64_t nrows, const int* __restrict__ ia, const int* __restrict__ ib,
                            View<9, const double> g, View<7, const double> K, double c, double* __restrict__ diag) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int i = ia[r], j = ib[r];
    double nn = g(0, r) * g(0, r) + g(1, r) * g(1, r) + g(2, r) * g(2, r);
    double acc = (K(0, i) + K(0, j)) * nn;
    for (int side = 0; side < 2; ++side) {
        int b = side ? j : i;
        int o = side ? 6 : 3;
        double t0 = g(o, r), t1 = g(o + 1, r), t2 = g(o + 2, r);
        double kxx = K(1, b), kyy = K(2, b), kzz = K(3, b), kxy = K(4, b), kxz = K(5, b), kyz = K(6, b);
        acc += t0 * (kxx * t0 + kxy * t1 + kxz * t2) + t1 * (kxy * t0 + kyy * t1 + kyz * t2) +
               t2 * (kxz * t0 + kyz * t1 + kzz * t2);
    }
    diag[r] = c * acc;
}

template <class S, class D>
__global__ void convert_rows(int64_t n, View<9, const S> in, D* __restrict__ out) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
#pragma unroll
    for (int k = 0; k < 9; ++k) out[(int64_t)k * n + r] = (D)in(k, r);
}

template <class S, class D>
__global__ void convert_vec(int64_t n, const S* __restrict__ in, D* __restrict__ out) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[r] = (D)in[r];
}

__global__ void uc_to_double(int64_t n, const float* __restrict__ ucf, View<6, double> uc) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
#pragma unroll
    for (int k = 0; k < 6; ++k) uc(k, b) = (double)ucf[(int64_t)k * n + b];
}

__global__ void zero_uc(int64_t n, View<6, double> uc) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
#pragma unroll
    for (int k = 0; k < 6; ++k) uc(k, b) = 0.0;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <class R>
relcp_status launch_lcp(KArgs<R>& ka, int64_t work, LcpScratch& sc, cudaStream_t s, int* blocks_out,
                        bool timed, float* ms) {
    int dev = 0;
    RELCP_CUDA(cudaGetDevice(&dev));
    int sms = 0, coop = 0;
    RELCP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    RELCP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) {
        set_error("device does not support cooperative launch");
        return RELCP_ERR_CUDA;
    }
    int per_sm = 0;
    RELCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lcp_kernel<R>, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    int64_t want = (work + kThreads - 1) / kThreads;
    int64_t maxb = (int64_t)sms * per_sm;
    int blocks = (int)(want < 1 ? 1 : (want > maxb ? maxb : want));
    RELCP_TRY(sc.partials.ensure((size_t)blocks * kNred, s));
    ka.partials = sc.partials.p;
    void* args[] = {&ka};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        RELCP_CUDA(cudaEventCreate(&e0));
        RELCP_CUDA(cudaEventCreate(&e1));
        RELCP_CUDA(cudaEventRecord(e0, s));
    }
    note_launch();
    RELCP_CUDA(cudaLaunchCooperativeKernel((void*)lcp_kernel<R>, dim3(blocks), dim3(kThreads), args, 0, s));
    if (timed) {
        RELCP_CUDA(cudaEventRecord(e1, s));
        RELCP_CUDA(cudaEventSynchronize(e1));
        RELCP_CUDA(cudaEventElapsedTime(ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    *blocks_out = blocks;
    return RELCP_OK;
}

}  // namespace

relcp_status lcp_diag_launch(int64_t nrows, const int32_t* ia, const int32_t* ib, View<9, const double> geom,
                             View<7, const double> K, double c, double* diag, cudaStream_t s) {
    if (nrows == 0) return RELCP_OK;
    note_launch();
    diag_kernel<<<nblk(nrows), 256, 0, s>>>(nrows, ia, ib, geom, K, c, diag);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status lcp_solve(const LcpProblem& pr, LcpScratch& sc, LcpResult* res, cudaStream_t s) {
    res->iterations = 0;
    res->residual = 0.0;
    res->blocks = 0;
    res->dev_status = 0;
    res->kernel_ms = 0.f;
    const int64_t m = pr.nrows, nb = pr.nbodies;
    if (nb > 0) {
        note_launch();
        zero_uc<<<nblk(nb), 256, 0, s>>>(nb, pr.uc);
        RELCP_CUDA(cudaGetLastError());
    }
    if (m == 0) return RELCP_OK;
    if (m > (int64_t)1 << 29 || nb > (int64_t)1 << 30) return RELCP_ERR_INVALID_ARG;

    // incidence CSR
    RELCP_TRY(sc.inc_count.ensure((size_t)nb, s));
    RELCP_TRY(sc.inc_cursor.ensure((size_t)nb, s));
    RELCP_TRY(sc.inc_off.ensure((size_t)nb + 1, s));
    RELCP_TRY(sc.inc.ensure((size_t)(2 * m), s));
    RELCP_CUDA(cudaMemsetAsync(sc.inc_count.p, 0, nb * sizeof(int), s));
    RELCP_CUDA(cudaMemsetAsync(sc.inc_cursor.p, 0, nb * sizeof(int), s));
    note_launch();
    inc_count<<<nblk(m), 256, 0, s>>>(m, pr.ia, pr.ib, sc.inc_count.p);
    RELCP_CUDA(cudaGetLastError());
    RELCP_TRY(exclusive_scan(sc.inc_count.p, sc.inc_off.p, nb, sc.scan, s));
    note_launch();
    inc_fill<<<nblk(m), 256, 0, s>>>(m, pr.ia, pr.ib, sc.inc_off.p, sc.inc_cursor.p, sc.inc.p);
    RELCP_CUDA(cudaGetLastError());
    note_launch();
    inc_sort<<<nblk(nb), 256, 0, s>>>(nb, sc.inc_off.p, sc.inc.p);
    RELCP_CUDA(cudaGetLastError());

    const double* diag = pr.diag;
    DBuf<double> diag_tmp;
    if (!diag) {
        RELCP_TRY(diag_tmp.ensure((size_t)m, s));
        RELCP_TRY(lcp_diag_launch(m, pr.ia, pr.ib, pr.geom, pr.K, pr.c, diag_tmp.p, s));
        diag = diag_tmp.p;
    }
    RELCP_TRY(sc.barrier.ensure(2, s));
    RELCP_TRY(sc.status.ensure(1, s));
    RELCP_TRY(sc.result.ensure(3, s));
    RELCP_CUDA(cudaMemsetAsync(sc.barrier.p, 0, 2 * sizeof(unsigned), s));
    RELCP_CUDA(cudaMemsetAsync(sc.status.p, 0, sizeof(int), s));

    int blocks = 0;
    double hres[3] = {0, 0, 0};
    if (!pr.mixed) {
        RELCP_TRY(sc.gamma2.ensure((size_t)m, s));
        RELCP_TRY(sc.g2.ensure((size_t)(2 * m), s));
        KArgs<double> ka{};
        ka.nrows = (int)m;
        ka.nbodies = (int)nb;
        ka.ia = pr.ia;
        ka.ib = pr.ib;
        for (int k = 0; k < 9; ++k) ka.geom[k] = nullptr;
        // the FP64 kernel reads SoA rows: convert a strided view if needed
        DBuf<double> soa;
        bool is_soa = pr.geom.s == 1;
        for (int k = 1; k < 9 && is_soa; ++k) is_soa = pr.geom.c[k] == pr.geom.c[0] + k * m;
        if (is_soa) {
            for (int k = 0; k < 9; ++k) ka.geom[k] = pr.geom.c[k];
        } else {
            RELCP_TRY(soa.ensure((size_t)(9 * m), s));
            note_launch();
            convert_rows<double, double><<<nblk(m), 256, 0, s>>>(m, pr.geom, soa.p);
            RELCP_CUDA(cudaGetLastError());
            for (int k = 0; k < 9; ++k) ka.geom[k] = soa.p + k * m;
        }
        ka.q = pr.q;
        ka.diag = diag;
        for (int k = 0; k < 7; ++k) ka.K[k] = pr.K.c[k];
        // K view must be SoA-compatible: stride handled by pointer arithmetic below
        DBuf<double> ksoa;
        if (pr.K.s != 1) {
            RELCP_TRY(ksoa.ensure((size_t)(7 * nb), s));
            for (int k = 0; k < 7; ++k)
                RELCP_CUDA(cudaMemcpy2DAsync(ksoa.p + k * nb, sizeof(double), pr.K.c[k], pr.K.s * sizeof(double),
                                             sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
            for (int k = 0; k < 7; ++k) ka.K[k] = ksoa.p + k * nb;
        }
        ka.inc_off = sc.inc_off.p;
        ka.inc = sc.inc.p;
        ka.gam[0] = pr.gamma;
        ka.gam[1] = sc.gamma2.p;
        ka.g[0] = sc.g2.p;
        ka.g[1] = sc.g2.p + m;
        for (int k = 0; k < 6; ++k) ka.uc[k] = pr.uc.c[k];
        ka.uc_stride = pr.uc.s;
        ka.c = pr.c;
        ka.tol = pr.tol;
        ka.max_iter = pr.max_iter;
        ka.bar = sc.barrier.p;
        ka.status = sc.status.p;
        ka.result = sc.result.p;
        RELCP_TRY(launch_lcp(ka, m > nb ? m : nb, sc, s, &blocks, pr.time_kernel, &res->kernel_ms));
        RELCP_CUDA(cudaMemcpyAsync(hres, sc.result.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaMemcpyAsync(&res->dev_status, sc.status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaStreamSynchronize(s));
        if ((int)hres[2] == 1)
            RELCP_CUDA(cudaMemcpyAsync(pr.gamma, sc.gamma2.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
        soa.release(s);
        ksoa.release(s);
    } else {
        RELCP_TRY(sc.geomf.ensure((size_t)(9 * m), s));
        RELCP_TRY(sc.gammaf.ensure((size_t)(2 * m), s));
        RELCP_TRY(sc.gf.ensure((size_t)(2 * m), s));
        RELCP_TRY(sc.ucf.ensure((size_t)(6 * nb), s));
        note_launch();
        convert_rows<double, float><<<nblk(m), 256, 0, s>>>(m, pr.geom, sc.geomf.p);
        RELCP_CUDA(cudaGetLastError());
        note_launch();
        convert_vec<double, float><<<nblk(m), 256, 0, s>>>(m, pr.gamma, sc.gammaf.p);
        RELCP_CUDA(cudaGetLastError());
        KArgs<float> ka{};
        ka.nrows = (int)m;
        ka.nbodies = (int)nb;
        ka.ia = pr.ia;
        ka.ib = pr.ib;
        for (int k = 0; k < 9; ++k) ka.geom[k] = sc.geomf.p + k * m;
        ka.q = pr.q;
        ka.diag = diag;
        DBuf<double> ksoa;
        for (int k = 0; k < 7; ++k) ka.K[k] = pr.K.c[k];
        if (pr.K.s != 1) {
            RELCP_TRY(ksoa.ensure((size_t)(7 * nb), s));
            for (int k = 0; k < 7; ++k)
                RELCP_CUDA(cudaMemcpy2DAsync(ksoa.p + k * nb, sizeof(double), pr.K.c[k], pr.K.s * sizeof(double),
                                             sizeof(double), nb, cudaMemcpyDeviceToDevice, s));
            for (int k = 0; k < 7; ++k) ka.K[k] = ksoa.p + k * nb;
        }
        ka.inc_off = sc.inc_off.p;
        ka.inc = sc.inc.p;
        ka.gam[0] = sc.gammaf.p;
        ka.gam[1] = sc.gammaf.p + m;
        ka.g[0] = sc.gf.p;
        ka.g[1] = sc.gf.p + m;
        for (int k = 0; k < 6; ++k) ka.uc[k] = sc.ucf.p + k * nb;
        ka.uc_stride = 1;
        ka.c = pr.c;
        ka.tol = pr.tol;
        ka.max_iter = pr.max_iter;
        ka.bar = sc.barrier.p;
        ka.status = sc.status.p;
        ka.result = sc.result.p;
        RELCP_TRY(launch_lcp(ka, m > nb ? m : nb, sc, s, &blocks, pr.time_kernel, &res->kernel_ms));
        RELCP_CUDA(cudaMemcpyAsync(hres, sc.result.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaMemcpyAsync(&res->dev_status, sc.status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        RELCP_CUDA(cudaStreamSynchronize(s));
        int fin = (int)hres[2];
        note_launch();
        convert_vec<float, double><<<nblk(m), 256, 0, s>>>(m, sc.gammaf.p + fin * m, pr.gamma);
        RELCP_CUDA(cudaGetLastError());
        note_launch();
        uc_to_double<<<nblk(nb), 256, 0, s>>>(nb, sc.ucf.p, pr.uc);
        RELCP_CUDA(cudaGetLastError());
        ksoa.release(s);
    }
    diag_tmp.release(s);
    res->iterations = (int)hres[0];
    res->residual = hres[1];
    res->blocks = blocks;
    return RELCP_OK;
}

}  // namespace relcp
