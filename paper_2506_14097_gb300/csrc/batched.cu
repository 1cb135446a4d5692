// Batched scenes: many independent periodic scenes of up to kBatchMaxBodies
// bodies, each advanced by whole ReLCP time steps (Algorithm 1) inside ONE
// persistent launch.  A CTA pulls a scene from a device work counter (scenes
// are queued largest first) and runs every step of that scene by itself:
//
//   prep -> broad phase -> SNSD at C^k -> A_0 = {Phi <= phi_skin} ->
//   loop { body CSR -> LCP (projected gradient, BB steps) -> trial C_{n+1}
//          -> SNSD at C_{n+1} + overlap test -> stop if no Phi < -eps_NCP
//          -> append one pulled-back row per violating pair }
//   -> accept C^{k+1} -> keep the A_0 gammas for the next step's warm start
//
// Every phase is a loop of the CTA's threads over the scene's bodies, pairs or
// rows, separated by __syncthreads: no grid-wide barrier, no host round trip.
// The per-body, per-pair and per-row arithmetic is the single-scene path's
// (step_math.cuh, snsd_math.cuh); the LCP is the same projected gradient with
// alternating BB1/BB2 steps, solved in the precision R with the FP64 natural
// residual on every 4th iteration (R = float) or every iteration (R = double).
//
// Broad phase per scene: all pairs i < j, one warp per row i, 32 columns per
// ballot.  An FP32 distance test with a margin far above its rounding error
// discards far pairs; the survivors take the exact FP64 test of the
// single-scene broad phase, so the pair list is the same bit for bit.  The
// warp ballots keep the list i-major with j ascending.
//
// Memory: scene-major SoA.  Component k of body i of scene s sits at
// base[C * boff[s] + k * n_s + i] (C components); pairs and rows likewise with
// the per-scene capacities pcap_s and rcap_s at offsets poff[s] and roff[s].
// The scenes' scratch is L2/L1 resident while a CTA works on it.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "relcp_internal.cuh"
#include "snsd_math.cuh"
#include "step_math.cuh"

namespace relcp {

namespace {

constexpr int kBatchMaxBodies = RELCP_BATCH_MAX_BODIES;
constexpr int kBatchCheckEvery = 4;  // mixed path: FP64 residual every 4th iteration
constexpr unsigned kFull = 0xffffffffu;

struct SceneParams {
    double box[3];
    double dt, eps, skin, lcp_tol, phi_skin;
};
static_assert(sizeof(SceneParams) == 8 * sizeof(double), "scene parameter record");

template <class R>
struct Pair2;
template <>
struct Pair2<float> {
    using T = float2;
};
template <>
struct Pair2<double> {
    using T = double2;
};

struct BatchArgs {
    int nscenes;
    const int* order;  // processing order of the scenes
    const int* boff;   // body offsets [S + 1]
    const int* poff;   // pair capacity offsets [S + 1]
    const int* roff;   // row capacity offsets [S + 1]
    const SceneParams* sp;
    int dynamics;
    int shape;  // RELCP_SHAPE_* of every scene
    double drag_xi, density;
    int lcp_max_iter, max_recursion, nsteps;
    // body state
    double* x;           // 3
    double* q;           // 4
    const double* axes;  // 3
    double* vel;         // 6
    const double* fext;  // 6
    // body scratch
    double* P;      // 6
    double* K;      // 7
    float* Kf;      // 7
    double* rb;     // 1
    double* ufree;  // 6
    double* uc;     // 6  (K D gamma of the last LCP, FP64)
    double* ustep;  // 6
    double* xt;     // 3
    double* qt;     // 4
    double* Pt;     // 6
    void* ucp;      // 6 x R (contact velocity inside the LCP)
    // pair scratch
    int* pa;
    int* pb;
    int* flags;
    double* s0;  // 10
    double* s1;  // 10
    int* wkey;   // warm start: keys i * kBatchMaxBodies + j of the previous A_0 rows
    double* wgam;
    int* wcount;  // per scene
    // row scratch
    int* ia;
    int* ib;
    int* rrec;   // per row: recursion index that created it
    int* rpair;  // per row: its candidate pair (index in the scene's pair list)
    double* geom;  // 9
    float* geomf;  // 9
    double* qd;
    float* qf;
    double* diag;
    void* gamma;  // R
    void* gg;     // 2 buffers x rcap x (gamma, g) in R
    int* inc;     // 2
    int* inc_tmp; // 2
    // control
    int* work;
    relcp_scene_stats* stats;
    int* status;  // OR of all scenes' DEV_* bits
};

struct Scene {
    int s, n, pcap, rcap;
    int64_t boff, poff, roff;
    SceneParams p;
};

__device__ __forceinline__ double* bcomp(double* base, const Scene& S, int C, int k) {
    return base + (int64_t)C * S.boff + (int64_t)k * S.n;
}
__device__ __forceinline__ const double* bcomp(const double* base, const Scene& S, int C, int k) {
    return base + (int64_t)C * S.boff + (int64_t)k * S.n;
}
template <class T>
__device__ __forceinline__ T* pcomp(T* base, const Scene& S, int C, int k) {
    return base + (int64_t)C * S.poff + (int64_t)k * S.pcap;
}
template <class T>
__device__ __forceinline__ T* rcomp(T* base, const Scene& S, int C, int k) {
    return base + (int64_t)C * S.roff + (int64_t)k * S.rcap;
}

// ---------------------------------------------------------------------------
// CTA-wide primitives (blockDim.x a multiple of 32, at most 1024)
// ---------------------------------------------------------------------------
__device__ int cta_excl_scan(int v, int* total) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int y = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(kFull, y, o);
            if (lane >= o) y += z;
        }
        ws[lane] = y;
    }
    __syncthreads();
    const int excl = x - v + (wid > 0 ? ws[wid - 1] : 0);
    *total = ws[nw - 1];
    __syncthreads();
    return excl;
}

// in-place exclusive scan of a[0..n); returns the total (all threads)
__device__ int cta_scan_array(int* a, int n) {
    int carry = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < n ? a[i] : 0;
        int tot;
        const int e = cta_excl_scan(v, &tot);
        if (i < n) a[i] = carry + e;
        carry += tot;
    }
    return carry;
}

// fixed-order CTA reduction; every thread gets the result
template <class T>
__device__ T cta_sum(T v) {
    __shared__ T buf[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane == 0) buf[wid] = v;
    __syncthreads();
    T r = buf[0];
    for (int w = 1; w < nw; ++w) r += buf[w];
    __syncthreads();
    return r;
}

// maximum of non-negative doubles as the unsigned maximum of their bits (a
// NaN survives and fails later comparisons)
__device__ double cta_max_nonneg(double v) {
    __shared__ unsigned long long buf[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long m = (unsigned long long)__double_as_longlong(v);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_down_sync(kFull, m, o);
        m = y > m ? y : m;
    }
    if (lane == 0) buf[wid] = m;
    __syncthreads();
    unsigned long long r = buf[0];
    for (int w = 1; w < nw; ++w) r = buf[w] > r ? buf[w] : r;
    __syncthreads();
    return __longlong_as_double((long long)r);
}

__device__ int cta_or(int v) {
    __shared__ int buf[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_down_sync(kFull, v, o);
    if (lane == 0) buf[wid] = v;
    __syncthreads();
    int r = 0;
    for (int w = 0; w < nw; ++w) r |= buf[w];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// per-scene shared memory: FP32 positions and radii for the broad-phase
// filter, the row counts and the body CSR counters
// ---------------------------------------------------------------------------
struct SceneSmem {
    float xf[3][kBatchMaxBodies];
    float rbf[kBatchMaxBodies];
    int cnt[kBatchMaxBodies + 1];
    int cursor[kBatchMaxBodies];
};

__device__ __forceinline__ float min_image_f(float d, float L, float invL) {
    return L > 0.f ? d - L * rintf(d * invL) : d;
}

// FP32 test with a margin far above its rounding error (coordinates in
// [0, L), so every FP32 difference is off by a few ulp of L), then the exact test
struct NearTest {
    float L[3], invL[3], skinf, marg;
    double Ld[3], skin;
    __device__ bool operator()(const SceneSmem& sm, const double* x0, const double* x1, const double* x2,
                               const double* rb, int i, int j) const {
        const float dx = min_image_f(sm.xf[0][j] - sm.xf[0][i], L[0], invL[0]);
        const float dy = min_image_f(sm.xf[1][j] - sm.xf[1][i], L[1], invL[1]);
        const float dz = min_image_f(sm.xf[2][j] - sm.xf[2][i], L[2], invL[2]);
        const float c = sm.rbf[i] + sm.rbf[j] + skinf + marg;
        if (dx * dx + dy * dy + dz * dz > c * c) return false;
        return near_pair_exact(x0[i], x1[i], x2[i], x0[j], x1[j], x2[j], rb[i], rb[j], Ld[0], Ld[1], Ld[2], skin);
    }
};

// ---------------------------------------------------------------------------
// one step of one scene; returns the scene's DEV_* bits of this step
// ---------------------------------------------------------------------------
template <class R>
struct LcpOut {
    int iters;
    double resid;
};

template <class R>
__device__ void build_csr(const BatchArgs& a, const Scene& S, SceneSmem& sm, int nrows) {
    const int n = S.n;
    int* ia = a.ia + S.roff;
    int* ib = a.ib + S.roff;
    int* inc = a.inc + 2 * S.roff;
    int* tmp = a.inc_tmp + 2 * S.roff;
    for (int b = threadIdx.x; b <= n; b += blockDim.x) sm.cnt[b] = 0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) sm.cursor[b] = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        atomicAdd(&sm.cnt[ia[r]], 1);
        atomicAdd(&sm.cnt[ib[r]], 1);
    }
    __syncthreads();
    const int tot = cta_scan_array(sm.cnt, n);
    if (threadIdx.x == 0) sm.cnt[n] = tot;
    __syncthreads();
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        const int i = ia[r], j = ib[r];
        tmp[sm.cnt[i] + atomicAdd(&sm.cursor[i], 1)] = r << 1;
        tmp[sm.cnt[j] + atomicAdd(&sm.cursor[j], 1)] = (r << 1) | 1;
    }
    __syncthreads();
    // deterministic order: each code at its rank among its body's codes
    for (int e = threadIdx.x; e < 2 * nrows; e += blockDim.x) {
        const int v = tmp[e];
        const int r = v >> 1;
        const int b = (v & 1) ? ib[r] : ia[r];
        const int e0 = sm.cnt[b], e1 = sm.cnt[b + 1];
        int rank = 0;
        for (int k = e0; k < e1; ++k) rank += tmp[k] < v;
        inc[e0 + rank] = v;
    }
    __syncthreads();
}

// projected gradient with BB steps on the scene's rows (the single-scene
// solver's iteration, one CTA); writes gamma (R) and uc (FP64, K D gamma)
template <class R>
__device__ LcpOut<R> scene_lcp(const BatchArgs& a, const Scene& S, SceneSmem& sm, int nrows, int& bits) {
    using V2 = typename Pair2<R>::T;
    const int n = S.n;
    const int64_t rc = S.rcap;
    const int* ia = a.ia + S.roff;
    const int* ib = a.ib + S.roff;
    const int* inc = a.inc + 2 * S.roff;
    const R* geom[9];
    for (int k = 0; k < 9; ++k)
        geom[k] = sizeof(R) == sizeof(float) ? (const R*)rcomp(a.geomf, S, 9, k) : (const R*)rcomp(a.geom, S, 9, k);
    const R* qr = sizeof(R) == sizeof(float) ? (const R*)(a.qf + S.roff) : (const R*)(a.qd + S.roff);
    const double* qd = a.qd + S.roff;
    const double* diag = a.diag + S.roff;
    R* gamma = (R*)a.gamma + S.roff;
    V2* gg0 = (V2*)a.gg + 2 * S.roff;
    V2* gg1 = gg0 + rc;
    R* ucp = (R*)a.ucp + 6 * S.boff;
    const double c = S.p.dt;
    const R cr = (R)c;
    const int check_every = sizeof(R) == sizeof(double) ? 1 : kBatchCheckEvery;

    // body operator in the solve precision
    auto Kb = [&](int b, int k) -> R {
        return sizeof(R) == sizeof(float) ? (R)a.Kf[(int64_t)7 * S.boff + (int64_t)k * n + b]
                                          : (R)a.K[(int64_t)7 * S.boff + (int64_t)k * n + b];
    };
    // Uc = K D gamma' for every body (gamma' = projected step when project)
    auto scatter = [&](const V2* src, V2* dst, bool project, R alpha) {
        for (int b = threadIdx.x; b < n; b += blockDim.x) {
            R w[6] = {0, 0, 0, 0, 0, 0};
            const int e0 = sm.cnt[b], e1 = sm.cnt[b + 1];
            for (int e = e0; e < e1; ++e) {
                const int code = inc[e];
                const int r = code >> 1;
                const bool sideb = code & 1;
                const V2 pr = src[r];
                R gm = pr.x;
                if (project) {
                    const R v = gm - alpha * pr.y;
                    gm = v > R(0) ? v : R(0);
                    if (!sideb) dst[r].x = gm;
                }
                const R sg = sideb ? R(1) : R(-1);
                const int o = sideb ? 6 : 3;
                w[0] += sg * gm * geom[0][r];
                w[1] += sg * gm * geom[1][r];
                w[2] += sg * gm * geom[2][r];
                w[3] += sg * gm * geom[o][r];
                w[4] += sg * gm * geom[o + 1][r];
                w[5] += sg * gm * geom[o + 2][r];
            }
            const R k0 = Kb(b, 0), kxx = Kb(b, 1), kyy = Kb(b, 2), kzz = Kb(b, 3), kxy = Kb(b, 4), kxz = Kb(b, 5),
                    kyz = Kb(b, 6);
            ucp[0 * n + b] = k0 * w[0];
            ucp[1 * n + b] = k0 * w[1];
            ucp[2 * n + b] = k0 * w[2];
            ucp[3 * n + b] = kxx * w[3] + kxy * w[4] + kxz * w[5];
            ucp[4 * n + b] = kxy * w[3] + kyy * w[4] + kyz * w[5];
            ucp[5 * n + b] = kxz * w[3] + kyz * w[4] + kzz * w[5];
        }
    };
    // g' = q + c d^T Uc per row into dst.y; BB products against old; FP64 residual
    auto gather = [&](const V2* old, V2* dst, bool check, R acc[3], double& res, double& mdiag) {
        for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
            const int i = ia[r], j = ib[r];
            R rate = 0;
            for (int k = 0; k < 3; ++k) rate += geom[k][r] * (ucp[k * n + j] - ucp[k * n + i]);
            for (int k = 0; k < 3; ++k) rate += geom[6 + k][r] * ucp[(3 + k) * n + j] - geom[3 + k][r] * ucp[(3 + k) * n + i];
            const R g = qr[r] + cr * rate;
            const R gm = dst[r].x;
            dst[r].y = g;
            if (old) {
                const V2 po = old[r];
                const R s = gm - po.x, y = g - po.y;
                acc[0] += s * s;
                acc[1] += s * y;
                acc[2] += y * y;
            }
            if (check) res = fmax(res, fabs(fmin(diag[r] * (double)gm, qd[r] + c * (double)rate)));
            mdiag = fmax(mdiag, diag[r]);
        }
    };

    // init: gamma_0 from the warm start, Uc, g_0, residual, largest diagonal
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) gg0[r].x = gamma[r];
    __syncthreads();
    scatter(gg0, gg0, false, R(0));
    __syncthreads();
    R acc[3] = {0, 0, 0};
    double res = 0.0, mdiag = 0.0;
    gather(nullptr, gg0, true, acc, res, mdiag);
    res = cta_max_nonneg(res);
    mdiag = cta_max_nonneg(mdiag);
    R alpha = (R)(mdiag > 0.0 ? 1.0 / mdiag : 1.0);
    int it = 0;
    int cur = 0;
    V2* bufs[2] = {gg0, gg1};
    if (!(res <= S.p.lcp_tol)) {
        for (it = 1; it <= a.lcp_max_iter; ++it) {
            const bool check = (it % check_every) == 0 || it == a.lcp_max_iter;
            V2* src = bufs[cur];
            V2* dst = bufs[1 - cur];
            scatter(src, dst, true, alpha);
            __syncthreads();
            R ac[3] = {0, 0, 0};
            double rs = 0.0, md = 0.0;
            gather(src, dst, check, ac, rs, md);
            const R ss = cta_sum(ac[0]), sy = cta_sum(ac[1]), yy = cta_sum(ac[2]);
            if (check) res = cta_max_nonneg(rs);
            cur = 1 - cur;
            R na;
            if (it & 1) na = (sy > R(0)) ? ss / sy : alpha;
            else na = (yy > R(0) && sy > R(0)) ? sy / yy : alpha;
            if (isfinite(na) && na > R(0)) alpha = na;
            if (check && res <= S.p.lcp_tol) break;
        }
        if (it > a.lcp_max_iter) it = a.lcp_max_iter;
    }
    if (!(res <= S.p.lcp_tol)) bits |= DEV_LCP_NOT_CONVERGED;
    // outputs: gamma and the FP64 contact velocity
    const V2* fin = bufs[cur];
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) gamma[r] = fin[r].x;
    for (int b = threadIdx.x; b < n; b += blockDim.x)
        for (int k = 0; k < 6; ++k) a.uc[(int64_t)6 * S.boff + (int64_t)k * n + b] = (double)ucp[k * n + b];
    __syncthreads();
    LcpOut<R> o;
    o.iters = it;
    o.resid = res;
    return o;
}

// one row from a pair's SNSD output: geometry, offset (A_0: Phi + c d^T U_free;
// appended: Phi - c d^T uc, the pull-back), diagonal, warm-start gamma
template <class R>
__device__ void write_row(const BatchArgs& a, const Scene& S, int r, int i, int j, const double* so, int p,
                          bool appended, double g0, int rec) {
    const int64_t pc = S.pcap;
    const int n = S.n;
    double nn[3], ra[3], rb[3], ta[3], tb[3];
    for (int k = 0; k < 3; ++k) {
        nn[k] = so[(1 + k) * pc + p];
        ra[k] = so[(4 + k) * pc + p];
        rb[k] = so[(7 + k) * pc + p];
    }
    const double phi = so[p];
    step_math::row_torques(nn, ra, rb, ta, tb);
    if (a.dynamics == RELCP_OVERDAMPED_2D) step_math::planar_row(nn, ta, tb);
    a.ia[S.roff + r] = i;
    a.ib[S.roff + r] = j;
    a.rrec[S.roff + r] = rec;
    a.rpair[S.roff + r] = p;
    for (int k = 0; k < 3; ++k) {
        rcomp(a.geom, S, 9, k)[r] = nn[k];
        rcomp(a.geom, S, 9, 3 + k)[r] = ta[k];
        rcomp(a.geom, S, 9, 6 + k)[r] = tb[k];
        rcomp(a.geomf, S, 9, k)[r] = (float)nn[k];
        rcomp(a.geomf, S, 9, 3 + k)[r] = (float)ta[k];
        rcomp(a.geomf, S, 9, 6 + k)[r] = (float)tb[k];
    }
    const double* U = appended ? a.uc : a.ufree;
    double Ui[6], Uj[6], Ki[7], Kj[7];
    for (int k = 0; k < 6; ++k) {
        Ui[k] = U[(int64_t)6 * S.boff + (int64_t)k * n + i];
        Uj[k] = U[(int64_t)6 * S.boff + (int64_t)k * n + j];
    }
    for (int k = 0; k < 7; ++k) {
        Ki[k] = a.K[(int64_t)7 * S.boff + (int64_t)k * n + i];
        Kj[k] = a.K[(int64_t)7 * S.boff + (int64_t)k * n + j];
    }
    const double rate = step_math::row_rate(Ui, Uj, nn, ta, tb);
    const double c = S.p.dt;
    const double qv = appended ? phi - c * rate : phi + c * rate;
    a.qd[S.roff + r] = qv;
    a.qf[S.roff + r] = (float)qv;
    a.diag[S.roff + r] = c * step_math::row_dKd(Ki, Kj, nn, ta, tb);
    ((R*)a.gamma)[S.roff + r] = (R)g0;
}

// SNSD of every pair of the scene at the given configuration; returns the OR
// of DEV_NEWTON; optionally violator flags (Phi < -eps) and the largest overlap
__device__ int scene_snsd(const BatchArgs& a, const Scene& S, int np, const double* X, const double* Pm,
                          const double* guess_out, double* out, bool mixed, int* viol, double* maxov) {
    const int n = S.n;
    const int64_t pc = S.pcap;
    const int* pa = a.pa + S.poff;
    const int* pb = a.pb + S.poff;
    int bits = 0;
    double mo = 0.0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int i = pa[p], j = pb[p];
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = min_image(X[(int64_t)k * n + j] - X[(int64_t)k * n + i], S.p.box[k]);
        const Sym3<double> Pa{Pm[i], Pm[n + i], Pm[2 * n + i], Pm[3 * n + i], Pm[4 * n + i], Pm[5 * n + i]};
        const Sym3<double> Pb{Pm[j], Pm[n + j], Pm[2 * n + j], Pm[3 * n + j], Pm[4 * n + j], Pm[5 * n + j]};
        snsd_math::PairResult o;
        const bool hg = guess_out != nullptr;
        if (a.shape == RELCP_SHAPE_SPHEROCYLINDER)
            snsd_math::capsule_pair(d, Pa, Pb, o);
        else
            snsd_math::snsd_pair(d, Pa, Pb, hg, hg ? guess_out[1 * pc + p] : 0.0, hg ? guess_out[2 * pc + p] : 0.0,
                                 hg ? guess_out[3 * pc + p] : 0.0, mixed, o);
        if (!o.ok) bits |= DEV_NEWTON;
        out[p] = o.phi;
        for (int k = 0; k < 3; ++k) {
            out[(1 + k) * pc + p] = o.n[k];
            out[(4 + k) * pc + p] = o.ra[k];
            out[(7 + k) * pc + p] = o.rb[k];
        }
        if (viol) viol[p] = o.phi < -S.p.eps ? 1 : 0;
        if (o.phi < 0.0) mo = fmax(mo, -o.phi);
    }
    bits = cta_or(bits);
    if (maxov) *maxov = cta_max_nonneg(mo);
    return bits;
}

template <class R>
__device__ int scene_step(const BatchArgs& a, const Scene& S, SceneSmem& sm, relcp_scene_stats& st) {
    const int n = S.n;
    const int tid = threadIdx.x, T = blockDim.x;
    int bits = 0;
    const bool mixed = sizeof(R) == sizeof(float);

    // ---- prep: normalised q, P, K, bounding radius, U_free
    for (int i = tid; i < n; i += T) {
        double qin[4], ax[3], vel[6], f[6], x[3];
        for (int k = 0; k < 4; ++k) qin[k] = bcomp(a.q, S, 4, k)[i];
        for (int k = 0; k < 3; ++k) {
            ax[k] = bcomp(a.axes, S, 3, k)[i];
            x[k] = bcomp(a.x, S, 3, k)[i];
        }
        for (int k = 0; k < 6; ++k) {
            vel[k] = bcomp(a.vel, S, 6, k)[i];
            f[k] = bcomp(a.fext, S, 6, k)[i];
        }
        step_math::BodyPrep b;
        step_math::prep_body(qin, ax, vel, f, x, a.dynamics, S.p.dt, a.drag_xi, a.density, 0.0, S.p.box, b, a.shape);
        for (int k = 0; k < 4; ++k) bcomp(a.q, S, 4, k)[i] = b.q[k];
        const double Pv[6] = {b.P.xx, b.P.yy, b.P.zz, b.P.xy, b.P.xz, b.P.yz};
        for (int k = 0; k < 6; ++k) bcomp(a.P, S, 6, k)[i] = Pv[k];
        for (int k = 0; k < 7; ++k) {
            bcomp(a.K, S, 7, k)[i] = b.K[k];
            a.Kf[(int64_t)7 * S.boff + (int64_t)k * n + i] = (float)b.K[k];
        }
        a.rb[S.boff + i] = b.rb;
        for (int k = 0; k < 6; ++k) bcomp(a.ufree, S, 6, k)[i] = b.ufree[k];
        for (int k = 0; k < 3; ++k) sm.xf[k][i] = (float)x[k];
        sm.rbf[i] = (float)b.rb;
    }
    __syncthreads();

    // ---- broad phase: all pairs i < j, one warp per row, i-major with j ascending
    const double* x0 = bcomp(a.x, S, 3, 0);
    const double* x1 = bcomp(a.x, S, 3, 1);
    const double* x2 = bcomp(a.x, S, 3, 2);
    const double* rbv = a.rb + S.boff;
    NearTest nt;
    float Lmax = 0.f;
    for (int k = 0; k < 3; ++k) {
        nt.Ld[k] = S.p.box[k];
        nt.L[k] = (float)S.p.box[k];
        nt.invL[k] = S.p.box[k] > 0.0 ? (float)(1.0 / S.p.box[k]) : 0.f;
        Lmax = fmaxf(Lmax, nt.L[k]);
    }
    nt.skin = S.p.skin;
    nt.skinf = (float)S.p.skin;
    nt.marg = 1e-4f * (1.f + Lmax + nt.skinf);
    const int lane = tid & 31, warp = tid >> 5, nwarps = T >> 5;
    for (int i = warp; i < n; i += nwarps) {
        int cnt = 0;
        for (int j0 = i + 1; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const bool hit = j < n && nt(sm, x0, x1, x2, rbv, i, j);
            cnt += __popc(__ballot_sync(kFull, hit));
        }
        if (lane == 0) sm.cnt[i] = cnt;
    }
    __syncthreads();
    const int np = cta_scan_array(sm.cnt, n);
    if (np > S.pcap) return bits | DEV_CAPACITY;
    {
        int* pa = a.pa + S.poff;
        int* pb = a.pb + S.poff;
        for (int i = warp; i < n; i += nwarps) {
            int pos = sm.cnt[i];
            for (int j0 = i + 1; j0 < n; j0 += 32) {
                const int j = j0 + lane;
                const bool hit = j < n && nt(sm, x0, x1, x2, rbv, i, j);
                const unsigned m = __ballot_sync(kFull, hit);
                if (hit) {
                    const int p = pos + __popc(m & ((1u << lane) - 1u));
                    pa[p] = i;
                    pb[p] = j;
                }
                pos += __popc(m);
            }
        }
    }
    __syncthreads();
    st.n_pairs = np;

    // ---- SNSD at C^k (cold start)
    double* s0 = a.s0 + 10 * S.poff;
    double* s1 = a.s1 + 10 * S.poff;
    bits |= scene_snsd(a, S, np, a.x + 3 * S.boff, a.P + 6 * S.boff, nullptr, s0, mixed, nullptr, nullptr);

    // ---- A_0 rows: pairs with Phi(C^k) <= phi_skin, warm start by pair key
    int* fl = a.flags + S.poff;
    for (int p = tid; p < np; p += T) fl[p] = s0[p] <= S.p.phi_skin ? 1 : 0;
    __syncthreads();
    const int nrows0 = cta_scan_array(fl, np);
    if (nrows0 > S.rcap) return bits | DEV_CAPACITY;
    {
        const int wc = a.wcount[S.s];
        const int* wk = a.wkey + S.poff;
        const double* wg = a.wgam + S.poff;
        for (int p = tid; p < np; p += T) {
            if (!(s0[p] <= S.p.phi_skin)) continue;
            const int i = a.pa[S.poff + p], j = a.pb[S.poff + p];
            const int key = i * kBatchMaxBodies + j;
            int lo = 0, hi = wc;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (wk[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            const double g0 = (lo < wc && wk[lo] == key) ? wg[lo] : 0.0;
            write_row<R>(a, S, fl[p], i, j, s0, p, false, g0, 0);
        }
    }
    __syncthreads();

    // ---- recursion: LCP, trial, overlap test, augmentation
    int nrows = nrows0;
    int depth = 0;
    double maxov = 0.0;
    bool violated = false;  // an overlap test of this step found Phi < -eps (augmented or capped)
    for (;;) {
        if (nrows > 0) {
            build_csr<R>(a, S, sm, nrows);
            LcpOut<R> lo = scene_lcp<R>(a, S, sm, nrows, bits);
            st.lcp_iters += lo.iters;
            st.lcp_residual = lo.resid;
        } else {
            for (int b = tid; b < n; b += T)
                for (int k = 0; k < 6; ++k) bcomp(a.uc, S, 6, k)[b] = 0.0;
            __syncthreads();
        }
        // trial configuration C_{n+1}
        for (int i = tid; i < n; i += T) {
            double U[6], x[3], q[4], ax[3], xt[3], qt[4];
            for (int k = 0; k < 6; ++k) {
                U[k] = bcomp(a.ufree, S, 6, k)[i] + bcomp(a.uc, S, 6, k)[i];
                bcomp(a.ustep, S, 6, k)[i] = U[k];
            }
            for (int k = 0; k < 3; ++k) {
                x[k] = bcomp(a.x, S, 3, k)[i];
                ax[k] = bcomp(a.axes, S, 3, k)[i];
            }
            for (int k = 0; k < 4; ++k) q[k] = bcomp(a.q, S, 4, k)[i];
            Sym3<double> Pt;
            step_math::trial_body(x, q, U, ax, S.p.dt, xt, qt, Pt, a.shape);
            for (int k = 0; k < 3; ++k) bcomp(a.xt, S, 3, k)[i] = xt[k];
            for (int k = 0; k < 4; ++k) bcomp(a.qt, S, 4, k)[i] = qt[k];
            const double Pv[6] = {Pt.xx, Pt.yy, Pt.zz, Pt.xy, Pt.xz, Pt.yz};
            for (int k = 0; k < 6; ++k) bcomp(a.Pt, S, 6, k)[i] = Pv[k];
        }
        __syncthreads();
        // overlap test at C_{n+1}, warm-started from the C^k normals
        bits |= scene_snsd(a, S, np, a.xt + 3 * S.boff, a.Pt + 6 * S.boff, s0, s1, mixed, fl, &maxov);
        const int nv = cta_scan_array(fl, np);
        if (nv == 0) break;
        violated = true;
        if (depth >= a.max_recursion) {
            bits |= DEV_RECURSION;
            break;
        }
        if (nrows + nv > S.rcap) return bits | DEV_CAPACITY;
        // one frozen-normal row per violating pair, pulled back to C^k
        for (int p = tid; p < np; p += T) {
            if (!(s1[p] < -S.p.eps)) continue;
            write_row<R>(a, S, nrows + fl[p], a.pa[S.poff + p], a.pb[S.poff + p], s1, p, true, 0.0, depth + 1);
        }
        __syncthreads();
        nrows += nv;
        ++depth;
    }

    // ---- accept C^{k+1}; keep the A_0 gammas for the next step
    for (int i = tid; i < n; i += T) {
        for (int k = 0; k < 3; ++k) bcomp(a.x, S, 3, k)[i] = step_math::wrap_coord(bcomp(a.xt, S, 3, k)[i], S.p.box[k]);
        for (int k = 0; k < 4; ++k) bcomp(a.q, S, 4, k)[i] = bcomp(a.qt, S, 4, k)[i];
        if (a.dynamics == RELCP_INERTIAL)
            for (int k = 0; k < 6; ++k) bcomp(a.vel, S, 6, k)[i] = bcomp(a.ustep, S, 6, k)[i];
    }
    for (int r = tid; r < nrows0; r += T) {
        a.wkey[S.poff + r] = a.ia[S.roff + r] * kBatchMaxBodies + a.ib[S.roff + r];
        a.wgam[S.poff + r] = (double)((const R*)a.gamma)[S.roff + r];
    }
    if (tid == 0) a.wcount[S.s] = nrows0;
    __syncthreads();
    st.n_rows = nrows;
    st.depth_max = depth > st.depth_max ? depth : st.depth_max;
    st.max_overlap = maxov;
    if (maxov > st.max_overlap_all) st.max_overlap_all = maxov;
    if (violated) st.aug_steps += 1;
    return bits;
}

template <class R>
__global__ void batched_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char dyn[];
    SceneSmem& sm = *reinterpret_cast<SceneSmem*>(dyn);
    __shared__ int sh_w;
    for (;;) {
        if (threadIdx.x == 0) sh_w = atomicAdd(a.work, 1);
        __syncthreads();
        const int w = sh_w;
        __syncthreads();
        if (w >= a.nscenes) break;
        Scene S;
        S.s = a.order[w];
        S.boff = a.boff[S.s];
        S.n = a.boff[S.s + 1] - a.boff[S.s];
        S.poff = a.poff[S.s];
        S.pcap = a.poff[S.s + 1] - a.poff[S.s];
        S.roff = a.roff[S.s];
        S.rcap = a.roff[S.s + 1] - a.roff[S.s];
        S.p = a.sp[S.s];
        relcp_scene_stats st = a.stats[S.s];
        int acc_bits = 0;
        for (int k = 0; k < a.nsteps; ++k) {
            st.n_pairs = 0;
            const int b = scene_step<R>(a, S, sm, st);
            acc_bits |= b;
            if (b & (DEV_CAPACITY | DEV_TIMEOUT)) break;  // the scene keeps its last accepted state
            st.steps_done += 1;
        }
        if (threadIdx.x == 0) {
            st.status_bits |= acc_bits;
            a.stats[S.s] = st;
            if (acc_bits) atomicOr(a.status, acc_bits);
        }
        __syncthreads();
    }
}

}  // namespace

}  // namespace relcp

// ===========================================================================
// host side
// ===========================================================================
using namespace relcp;

namespace {

relcp_status batch_status(int bits) {
    if (bits & DEV_TIMEOUT) return RELCP_ERR_TIMEOUT;
    if (bits & DEV_CAPACITY) return RELCP_ERR_CAPACITY;
    if (bits & DEV_NEWTON) return RELCP_ERR_NEWTON;
    if (bits & DEV_RECURSION) return RELCP_ERR_RECURSION_LIMIT;
    if (bits & DEV_LCP_NOT_CONVERGED) return RELCP_ERR_NOT_CONVERGED;
    return RELCP_OK;
}

// per-scene capacities: candidate pairs and constraint rows
inline int pair_cap(int n) {
    const int64_t all = (int64_t)n * (n - 1) / 2;
    const int64_t c = 16 * (int64_t)n + 32;
    return (int)std::max<int64_t>(1, std::min(all, c));
}
inline int row_cap(int pcap) { return 2 * pcap + 32; }

struct GraphEntry {
    int nsteps = 0, threads = 0;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct relcp_batch {
    relcp_config cfg{};
    cudaStream_t s = nullptr;
    int S = 0;
    int64_t N = 0, Ptot = 0, Rtot = 0;
    std::vector<int> hoff;  // caller's scene offsets
    bool loaded = false;
    int threads = 0;
    // device
    DBuf<int> order, boff, poff, roff, work, status, wcount, pa, pb, flags, wkey, ia, ib, inc, inc_tmp, rrec, rpair;
    DBuf<SceneParams> sp;
    DBuf<double> x, q, axes, vel, fext, P, K, rb, ufree, uc, ustep, xt, qt, Pt, s0, s1, wgam, geom, qd, diag, gamma,
        gg, ucp;
    DBuf<float> Kf, geomf, qf;
    DBuf<relcp_scene_stats> stats;
    int* hstatus = nullptr;  // pinned
    std::vector<GraphEntry> graphs;
    bool own_stream = false;  // the legacy default stream cannot be captured: a blocking stream of our own
};

namespace {

BatchArgs batch_args(relcp_batch* b, int nsteps) {
    BatchArgs a{};
    a.nscenes = b->S;
    a.order = b->order.p;
    a.boff = b->boff.p;
    a.poff = b->poff.p;
    a.roff = b->roff.p;
    a.sp = b->sp.p;
    a.dynamics = b->cfg.dynamics;
    a.shape = b->cfg.shape;
    a.drag_xi = b->cfg.drag_xi;
    a.density = b->cfg.density;
    a.lcp_max_iter = b->cfg.lcp_max_iter;
    a.max_recursion = b->cfg.max_recursion;
    a.nsteps = nsteps;
    a.x = b->x.p;
    a.q = b->q.p;
    a.axes = b->axes.p;
    a.vel = b->vel.p;
    a.fext = b->fext.p;
    a.P = b->P.p;
    a.K = b->K.p;
    a.Kf = b->Kf.p;
    a.rb = b->rb.p;
    a.ufree = b->ufree.p;
    a.uc = b->uc.p;
    a.ustep = b->ustep.p;
    a.xt = b->xt.p;
    a.qt = b->qt.p;
    a.Pt = b->Pt.p;
    a.ucp = b->ucp.p;
    a.pa = b->pa.p;
    a.pb = b->pb.p;
    a.flags = b->flags.p;
    a.s0 = b->s0.p;
    a.s1 = b->s1.p;
    a.wkey = b->wkey.p;
    a.wgam = b->wgam.p;
    a.wcount = b->wcount.p;
    a.ia = b->ia.p;
    a.ib = b->ib.p;
    a.rrec = b->rrec.p;
    a.rpair = b->rpair.p;
    a.geom = b->geom.p;
    a.geomf = b->geomf.p;
    a.qd = b->qd.p;
    a.qf = b->qf.p;
    a.diag = b->diag.p;
    a.gamma = b->gamma.p;
    a.gg = b->gg.p;
    a.inc = b->inc.p;
    a.inc_tmp = b->inc_tmp.p;
    a.work = b->work.p;
    a.stats = b->stats.p;
    a.status = b->status.p;
    return a;
}

constexpr int kDefaultThreads = 128;

relcp_status launch_batch(relcp_batch* b, int nsteps, int threads) {
    const bool mixed = b->cfg.precision == RELCP_MIXED;
    const void* fn = mixed ? (const void*)batched_kernel<float> : (const void*)batched_kernel<double>;
    const size_t smem = sizeof(SceneSmem);
    int per_sm = 0, sms = device_sm_count();
    RELCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    if (per_sm < 1) {
        set_error("batched kernel does not fit with %d threads", threads);
        return RELCP_ERR_INVALID_ARG;
    }
    int64_t blocks = (int64_t)per_sm * (sms > 0 ? sms : 1);
    if (blocks > b->S) blocks = b->S;
    BatchArgs a = batch_args(b, nsteps);
    RELCP_CUDA(cudaMemsetAsync(b->work.p, 0, sizeof(int), b->s));
    note_launch();
    if (mixed) batched_kernel<float><<<(unsigned)blocks, threads, smem, b->s>>>(a);
    else batched_kernel<double><<<(unsigned)blocks, threads, smem, b->s>>>(a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

// the step as a replayable graph: work-counter reset, the persistent launch,
// the status word to pinned host memory
relcp_status graph_for(relcp_batch* b, int nsteps, int threads, cudaGraphExec_t* out) {
    for (auto& g : b->graphs)
        if (g.nsteps == nsteps && g.threads == threads) {
            *out = g.exec;
            return RELCP_OK;
        }
    cudaGraph_t graph = nullptr;
    RELCP_CUDA(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
    relcp_status st = launch_batch(b, nsteps, threads);
    if (st == RELCP_OK &&
        cudaMemcpyAsync(b->hstatus, b->status.p, sizeof(int), cudaMemcpyDeviceToHost, b->s) != cudaSuccess)
        st = RELCP_ERR_CUDA;
    cudaError_t e = cudaStreamEndCapture(b->s, &graph);
    if (st != RELCP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    RELCP_CUDA(e);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    RELCP_CUDA(e);
    b->graphs.push_back(GraphEntry{nsteps, threads, exec});
    *out = exec;
    return RELCP_OK;
}

void drop_graphs(relcp_batch* b) {
    for (auto& g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

relcp_status run_steps(relcp_batch* b, int nsteps, int threads) {
    cudaGraphExec_t exec = nullptr;
    RELCP_TRY(graph_for(b, nsteps, threads, &exec));
    RELCP_CUDA(cudaMemsetAsync(b->status.p, 0, sizeof(int), b->s));
    RELCP_CUDA(cudaGraphLaunch(exec, b->s));
    RELCP_CUDA(cudaStreamSynchronize(b->s));
    return batch_status(*b->hstatus);
}

template <class T>
relcp_status upload(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
    RELCP_TRY(d.ensure(h.size() > 0 ? h.size() : 1, s));
    if (!h.empty()) RELCP_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return RELCP_OK;
}

relcp_status fetch(const double* src, int64_t count, int32_t kind, std::vector<double>& out) {
    out.resize((size_t)count);
    if (count == 0) return RELCP_OK;
    if (kind == RELCP_PTR_DEVICE) RELCP_CUDA(cudaMemcpy(out.data(), src, count * sizeof(double), cudaMemcpyDeviceToHost));
    else std::memcpy(out.data(), src, count * sizeof(double));
    return RELCP_OK;
}

// caller's AoS rows (w columns) -> scene-major SoA
std::vector<double> to_scene_soa(const std::vector<double>& aos, int w, const std::vector<int>& off) {
    std::vector<double> out(aos.size());
    for (size_t s = 0; s + 1 < off.size(); ++s) {
        const int64_t b0 = off[s], n = off[s + 1] - off[s];
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < w; ++k) out[(size_t)(w * b0 + k * n + i)] = aos[(size_t)((b0 + i) * w + k)];
    }
    return out;
}

std::vector<double> from_scene_soa(const std::vector<double>& soa, int w, const std::vector<int>& off) {
    std::vector<double> out(soa.size());
    for (size_t s = 0; s + 1 < off.size(); ++s) {
        const int64_t b0 = off[s], n = off[s + 1] - off[s];
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < w; ++k) out[(size_t)((b0 + i) * w + k)] = soa[(size_t)(w * b0 + k * n + i)];
    }
    return out;
}

}  // namespace

extern "C" relcp_status relcp_batch_create(const relcp_config* cfg, void* cuda_stream, relcp_batch** out) {
    if (!cfg || !out) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->dynamics != RELCP_INERTIAL && cfg->dynamics != RELCP_OVERDAMPED && cfg->dynamics != RELCP_OVERDAMPED_2D)
        return set_error("dynamics must be RELCP_INERTIAL, RELCP_OVERDAMPED or RELCP_OVERDAMPED_2D"),
               RELCP_ERR_INVALID_ARG;
    if (cfg->precision != RELCP_FP64 && cfg->precision != RELCP_MIXED)
        return set_error("precision must be RELCP_FP64 or RELCP_MIXED"), RELCP_ERR_INVALID_ARG;
    if (cfg->guess != RELCP_GUESS_COLD) return set_error("batched scenes start the SNSD cold"), RELCP_ERR_INVALID_ARG;
    if (cfg->strain_rate != 0.0) return set_error("batched scenes have fixed boxes (strain_rate = 0)"), RELCP_ERR_INVALID_ARG;
    if (cfg->lcp_max_iter < 1 || cfg->max_recursion < 0 || cfg->max_recursion > 4096)
        return set_error("lcp_max_iter >= 1, 0 <= max_recursion <= 4096"), RELCP_ERR_INVALID_ARG;
    if (cfg->dynamics != RELCP_INERTIAL && !(cfg->drag_xi > 0)) return set_error("drag_xi must be > 0"), RELCP_ERR_INVALID_ARG;
    if (cfg->shape != RELCP_SHAPE_ELLIPSOID && cfg->shape != RELCP_SHAPE_SPHEROCYLINDER)
        return set_error("shape must be RELCP_SHAPE_ELLIPSOID or RELCP_SHAPE_SPHEROCYLINDER"), RELCP_ERR_INVALID_ARG;
    if (cfg->shape == RELCP_SHAPE_SPHEROCYLINDER && cfg->dynamics == RELCP_INERTIAL)
        return set_error("spherocylinders are stepped with the overdamped laws only"), RELCP_ERR_INVALID_ARG;
    if (cfg->dynamics == RELCP_INERTIAL && !(cfg->density > 0)) return set_error("density must be > 0"), RELCP_ERR_INVALID_ARG;
    relcp_batch* b = new relcp_batch();
    b->cfg = *cfg;
    b->s = (cudaStream_t)cuda_stream;
    if (!b->s) {
        if (cudaStreamCreate(&b->s) != cudaSuccess) {
            delete b;
            return set_error("stream creation failed"), RELCP_ERR_CUDA;
        }
        b->own_stream = true;
    }
    if (cudaMallocHost((void**)&b->hstatus, sizeof(int)) != cudaSuccess) {
        if (b->own_stream) cudaStreamDestroy(b->s);
        delete b;
        return set_error("pinned allocation failed"), RELCP_ERR_CUDA;
    }
    *b->hstatus = 0;
    *out = b;
    return RELCP_OK;
}

extern "C" relcp_status relcp_batch_set_scenes(relcp_batch* b, int32_t n_scenes, const int32_t* scene_offsets,
                                               const double* x, const double* q, const double* semi_axes,
                                               const double* vel, const double* f_ext, const double* scene_params,
                                               int32_t ptr_kind) {
    if (!b) return set_error("batch is NULL"), RELCP_ERR_INVALID_ARG;
    if (n_scenes < 1 || !scene_offsets || !scene_params) return set_error("n_scenes >= 1, offsets and params required"), RELCP_ERR_INVALID_ARG;
    if (ptr_kind != RELCP_PTR_HOST && ptr_kind != RELCP_PTR_DEVICE) return set_error("bad ptr_kind"), RELCP_ERR_INVALID_ARG;
    std::vector<int> off((size_t)n_scenes + 1);
    if (ptr_kind == RELCP_PTR_DEVICE)
        RELCP_CUDA(cudaMemcpy(off.data(), scene_offsets, off.size() * sizeof(int), cudaMemcpyDeviceToHost));
    else std::memcpy(off.data(), scene_offsets, off.size() * sizeof(int));
    if (off[0] != 0) return set_error("scene_offsets[0] must be 0"), RELCP_ERR_INVALID_ARG;
    for (int s = 0; s < n_scenes; ++s) {
        const int n = off[s + 1] - off[s];
        if (n < 0 || n > kBatchMaxBodies)
            return set_error("scene %d has %d bodies (0..%d allowed)", s, n, kBatchMaxBodies), RELCP_ERR_INVALID_ARG;
    }
    const int64_t N = off[n_scenes];
    if (N > 0 && (!x || !q || !semi_axes)) return set_error("x, q, semi_axes required"), RELCP_ERR_INVALID_ARG;
    std::vector<double> hx, hq, ha, hv, hf, hp;
    RELCP_TRY(fetch(x, 3 * N, ptr_kind, hx));
    RELCP_TRY(fetch(q, 4 * N, ptr_kind, hq));
    RELCP_TRY(fetch(semi_axes, 3 * N, ptr_kind, ha));
    if (vel) RELCP_TRY(fetch(vel, 6 * N, ptr_kind, hv));
    else hv.assign((size_t)(6 * N), 0.0);
    if (f_ext) RELCP_TRY(fetch(f_ext, 6 * N, ptr_kind, hf));
    else hf.assign((size_t)(6 * N), 0.0);
    RELCP_TRY(fetch(scene_params, (int64_t)RELCP_SCENE_PARAMS * n_scenes, ptr_kind, hp));
    std::vector<SceneParams> sp((size_t)n_scenes);
    for (int s = 0; s < n_scenes; ++s) {
        const double* p = &hp[(size_t)s * RELCP_SCENE_PARAMS];
        SceneParams& o = sp[(size_t)s];
        for (int k = 0; k < 3; ++k) o.box[k] = p[k];
        o.dt = p[3];
        o.eps = p[4];
        o.skin = p[5];
        o.lcp_tol = p[6];
        o.phi_skin = p[7];
        if (!(o.box[0] >= 0 && o.box[1] >= 0 && o.box[2] >= 0 && o.dt > 0 && o.eps > 0 && o.skin >= 0 &&
              o.lcp_tol > 0 && o.phi_skin >= 0))
            return set_error("scene %d: bad parameters", s), RELCP_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < N; ++i) {
        double qq = 0;
        for (int k = 0; k < 4; ++k) qq += hq[(size_t)(4 * i + k)] * hq[(size_t)(4 * i + k)];
        if (!(std::fabs(std::sqrt(qq) - 1.0) <= 1e-6)) return set_error("quaternion %lld not normalised", (long long)i), RELCP_ERR_INVALID_ARG;
        for (int k = 0; k < 3; ++k)
            if (!(ha[(size_t)(3 * i + k)] > 0)) return set_error("semi-axes must be > 0"), RELCP_ERR_INVALID_ARG;
    }
    // wrap positions into the scene boxes
    for (int s = 0; s < n_scenes; ++s)
        for (int64_t i = off[s]; i < off[s + 1]; ++i)
            for (int k = 0; k < 3; ++k) {
                const double L = sp[(size_t)s].box[k];
                double& v = hx[(size_t)(3 * i + k)];
                if (L > 0) v = v - L * std::floor(v / L);
            }
    // capacities and offsets
    std::vector<int> poff((size_t)n_scenes + 1, 0), roff((size_t)n_scenes + 1, 0);
    for (int s = 0; s < n_scenes; ++s) {
        const int pc = pair_cap(off[s + 1] - off[s]);
        poff[(size_t)s + 1] = poff[(size_t)s] + pc;
        roff[(size_t)s + 1] = roff[(size_t)s] + row_cap(pc);
    }
    const int64_t Pt = poff[(size_t)n_scenes], Rt = roff[(size_t)n_scenes];
    if (Pt > (int64_t)1 << 30 || Rt > (int64_t)1 << 30) return set_error("too many pairs / rows"), RELCP_ERR_CAPACITY;
    // largest scenes first
    std::vector<int> order((size_t)n_scenes);
    for (int s = 0; s < n_scenes; ++s) order[(size_t)s] = s;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c) { return off[(size_t)a + 1] - off[(size_t)a] > off[(size_t)c + 1] - off[(size_t)c]; });
    cudaStream_t st = b->s;
    drop_graphs(b);
    b->S = n_scenes;
    b->N = N;
    b->Ptot = Pt;
    b->Rtot = Rt;
    b->hoff = off;
    const size_t Na = (size_t)(N > 0 ? N : 1);
    RELCP_TRY(upload(b->boff, off, st));
    RELCP_TRY(upload(b->poff, poff, st));
    RELCP_TRY(upload(b->roff, roff, st));
    RELCP_TRY(upload(b->order, order, st));
    RELCP_TRY(upload(b->sp, sp, st));
    RELCP_TRY(upload(b->x, to_scene_soa(hx, 3, off), st));
    RELCP_TRY(upload(b->q, to_scene_soa(hq, 4, off), st));
    RELCP_TRY(upload(b->axes, to_scene_soa(ha, 3, off), st));
    RELCP_TRY(upload(b->vel, to_scene_soa(hv, 6, off), st));
    RELCP_TRY(upload(b->fext, to_scene_soa(hf, 6, off), st));
    RELCP_TRY(b->P.ensure(6 * Na, st));
    RELCP_TRY(b->K.ensure(7 * Na, st));
    RELCP_TRY(b->Kf.ensure(7 * Na, st));
    RELCP_TRY(b->rb.ensure(Na, st));
    RELCP_TRY(b->ufree.ensure(6 * Na, st));
    RELCP_TRY(b->uc.ensure(6 * Na, st));
    RELCP_TRY(b->ustep.ensure(6 * Na, st));
    RELCP_TRY(b->xt.ensure(3 * Na, st));
    RELCP_TRY(b->qt.ensure(4 * Na, st));
    RELCP_TRY(b->Pt.ensure(6 * Na, st));
    RELCP_TRY(b->ucp.ensure(6 * Na, st));
    RELCP_TRY(b->pa.ensure((size_t)Pt, st));
    RELCP_TRY(b->pb.ensure((size_t)Pt, st));
    RELCP_TRY(b->flags.ensure((size_t)Pt, st));
    RELCP_TRY(b->s0.ensure((size_t)(10 * Pt), st));
    RELCP_TRY(b->s1.ensure((size_t)(10 * Pt), st));
    RELCP_TRY(b->wkey.ensure((size_t)Pt, st));
    RELCP_TRY(b->wgam.ensure((size_t)Pt, st));
    RELCP_TRY(b->wcount.ensure((size_t)n_scenes, st));
    RELCP_TRY(b->ia.ensure((size_t)Rt, st));
    RELCP_TRY(b->ib.ensure((size_t)Rt, st));
    RELCP_TRY(b->rrec.ensure((size_t)Rt, st));
    RELCP_TRY(b->rpair.ensure((size_t)Rt, st));
    RELCP_TRY(b->geom.ensure((size_t)(9 * Rt), st));
    RELCP_TRY(b->geomf.ensure((size_t)(9 * Rt), st));
    RELCP_TRY(b->qd.ensure((size_t)Rt, st));
    RELCP_TRY(b->qf.ensure((size_t)Rt, st));
    RELCP_TRY(b->diag.ensure((size_t)Rt, st));
    RELCP_TRY(b->gamma.ensure((size_t)Rt, st));
    RELCP_TRY(b->gg.ensure((size_t)(4 * Rt), st));  // 2 buffers of (gamma, g)
    RELCP_TRY(b->inc.ensure((size_t)(2 * Rt), st));
    RELCP_TRY(b->inc_tmp.ensure((size_t)(2 * Rt), st));
    RELCP_TRY(b->work.ensure(1, st));
    RELCP_TRY(b->status.ensure(1, st));
    RELCP_TRY(b->stats.ensure((size_t)n_scenes, st));
    RELCP_CUDA(cudaMemsetAsync(b->wcount.p, 0, n_scenes * sizeof(int), st));
    RELCP_CUDA(cudaMemsetAsync(b->stats.p, 0, n_scenes * sizeof(relcp_scene_stats), st));
    RELCP_CUDA(cudaStreamSynchronize(st));  // host staging buffers go out of scope
    b->loaded = true;
    return RELCP_OK;
}

extern "C" relcp_status relcp_batch_set_threads(relcp_batch* b, int32_t threads) {
    if (!b) return set_error("batch is NULL"), RELCP_ERR_INVALID_ARG;
    if (threads != 0 && (threads < 32 || threads > 1024 || threads % 32))
        return set_error("threads must be 0 or a multiple of 32 in [32, 1024]"), RELCP_ERR_INVALID_ARG;
    b->threads = threads;
    return RELCP_OK;
}

extern "C" relcp_status relcp_batch_step(relcp_batch* b, int32_t nsteps) {
    if (!b) return set_error("batch is NULL"), RELCP_ERR_INVALID_ARG;
    if (!b->loaded) return set_error("relcp_batch_set_scenes has not been called"), RELCP_ERR_STATE;
    if (nsteps < 1) return set_error("nsteps must be >= 1"), RELCP_ERR_INVALID_ARG;
    return run_steps(b, nsteps, b->threads > 0 ? b->threads : kDefaultThreads);
}

extern "C" relcp_status relcp_batch_get_bodies(relcp_batch* b, double* x, double* q, double* vel, int32_t ptr_kind) {
    if (!b) return set_error("batch is NULL"), RELCP_ERR_INVALID_ARG;
    if (ptr_kind != RELCP_PTR_HOST && ptr_kind != RELCP_PTR_DEVICE) return set_error("bad ptr_kind"), RELCP_ERR_INVALID_ARG;
    RELCP_CUDA(cudaStreamSynchronize(b->s));
    const int64_t N = b->N;
    struct Item {
        double* dst;
        const double* src;
        int w;
    } items[3] = {{x, b->x.p, 3}, {q, b->q.p, 4}, {vel, b->ustep.p, 6}};
    for (auto& it : items) {
        if (!it.dst || N == 0) continue;
        std::vector<double> h((size_t)(it.w * N));
        RELCP_CUDA(cudaMemcpy(h.data(), it.src, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
        std::vector<double> a = from_scene_soa(h, it.w, b->hoff);
        if (ptr_kind == RELCP_PTR_DEVICE)
            RELCP_CUDA(cudaMemcpy(it.dst, a.data(), a.size() * sizeof(double), cudaMemcpyHostToDevice));
        else std::memcpy(it.dst, a.data(), a.size() * sizeof(double));
    }
    return RELCP_OK;
}

extern "C" relcp_status relcp_batch_get_scene_contacts(relcp_batch* b, int32_t scene, int32_t* pairs,
                                                       int64_t pair_cap, int64_t* n_pairs, int32_t* row_ids,
                                                       int64_t row_cap, int64_t* n_rows) {
    if (!b || !n_pairs || !n_rows) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    if (!b->loaded) return set_error("relcp_batch_set_scenes has not been called"), RELCP_ERR_STATE;
    if (scene < 0 || scene >= b->S) return set_error("scene %d out of range", (int)scene), RELCP_ERR_INVALID_ARG;
    RELCP_CUDA(cudaStreamSynchronize(b->s));
    relcp_scene_stats ss{};
    RELCP_CUDA(cudaMemcpy(&ss, b->stats.p + scene, sizeof(ss), cudaMemcpyDeviceToHost));
    int offs[2], roffs[2];
    RELCP_CUDA(cudaMemcpy(offs, b->poff.p + scene, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    RELCP_CUDA(cudaMemcpy(roffs, b->roff.p + scene, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    const int64_t np = ss.steps_done > 0 ? ss.n_pairs : 0, nr = ss.steps_done > 0 ? ss.n_rows : 0;
    if (np > offs[1] - offs[0] || nr > roffs[1] - roffs[0])
        return set_error("scene %d: counts beyond its capacities", (int)scene), RELCP_ERR_STATE;
    *n_pairs = np;
    *n_rows = nr;
    if ((pairs && pair_cap < np) || (row_ids && row_cap < nr))
        return set_error("need room for %lld pairs and %lld rows", (long long)np, (long long)nr),
               RELCP_ERR_CAPACITY;
    if (pairs && np > 0) {
        std::vector<int> a((size_t)np), c((size_t)np);
        RELCP_CUDA(cudaMemcpy(a.data(), b->pa.p + offs[0], np * sizeof(int), cudaMemcpyDeviceToHost));
        RELCP_CUDA(cudaMemcpy(c.data(), b->pb.p + offs[0], np * sizeof(int), cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < np; ++k) {
            pairs[2 * k] = a[(size_t)k];
            pairs[2 * k + 1] = c[(size_t)k];
        }
    }
    if (row_ids && nr > 0) {
        DBuf<int>* src[4] = {&b->ia, &b->ib, &b->rrec, &b->rpair};
        std::vector<int> v((size_t)nr);
        for (int f = 0; f < 4; ++f) {
            RELCP_CUDA(cudaMemcpy(v.data(), src[f]->p + roffs[0], nr * sizeof(int), cudaMemcpyDeviceToHost));
            for (int64_t k = 0; k < nr; ++k) row_ids[4 * k + f] = v[(size_t)k];
        }
    }
    return RELCP_OK;
}

extern "C" relcp_status relcp_batch_scene_stats(relcp_batch* b, relcp_scene_stats* out) {
    if (!b || !out) return set_error("NULL argument"), RELCP_ERR_INVALID_ARG;
    if (!b->loaded) return set_error("relcp_batch_set_scenes has not been called"), RELCP_ERR_STATE;
    RELCP_CUDA(cudaStreamSynchronize(b->s));
    RELCP_CUDA(cudaMemcpy(out, b->stats.p, b->S * sizeof(relcp_scene_stats), cudaMemcpyDeviceToHost));
    for (int s = 0; s < b->S; ++s) out[s].status = batch_status(out[s].status_bits);
    return RELCP_OK;
}

namespace {

// cache key: device, precision, dynamics and the scenes' size histogram
std::string tune_key(relcp_batch* b) {
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    int hist[11] = {0};
    for (int s = 0; s < b->S; ++s) {
        int n = b->hoff[(size_t)s + 1] - b->hoff[(size_t)s], k = 0;
        while (n > 1 && k < 10) {
            n >>= 1;
            ++k;
        }
        hist[k] += 1;
    }
    std::string key = "sm" + std::to_string(major) + std::to_string(minor) + "_" +
                      (b->cfg.precision == RELCP_MIXED ? "mixed" : "fp64") + "_" +
                      (b->cfg.dynamics == RELCP_INERTIAL ? "inertial" : "overdamped") + "_h";
    for (int k = 0; k < 11; ++k) key += "-" + std::to_string(hist[k]);
    return key;
}

// minimal JSON object of "key": integer entries
bool read_cache(const char* path, std::vector<std::pair<std::string, int>>& out) {
    out.clear();
    FILE* f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return false;
    std::string txt;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, r);
    std::fclose(f);
    size_t pos = 0;
    for (;;) {
        const size_t k0 = txt.find('"', pos);
        if (k0 == std::string::npos) break;
        const size_t k1 = txt.find('"', k0 + 1);
        if (k1 == std::string::npos) break;
        const size_t c = txt.find(':', k1);
        if (c == std::string::npos) break;
        out.emplace_back(txt.substr(k0 + 1, k1 - k0 - 1), std::atoi(txt.c_str() + c + 1));
        pos = c + 1;
    }
    return true;
}

bool write_cache(const char* path, const std::vector<std::pair<std::string, int>>& entries) {
    FILE* f = std::fopen(path, "w");
    if (!f) return false;
    std::fprintf(f, "{\n");
    for (size_t i = 0; i < entries.size(); ++i)
        std::fprintf(f, "  \"%s\": %d%s\n", entries[i].first.c_str(), entries[i].second, i + 1 < entries.size() ? "," : "");
    std::fprintf(f, "}\n");
    std::fclose(f);
    return true;
}

}  // namespace

extern "C" relcp_status relcp_batch_autotune(relcp_batch* b, const char* cache_path, int32_t* threads_out) {
    if (!b) return set_error("batch is NULL"), RELCP_ERR_INVALID_ARG;
    if (!b->loaded) return set_error("relcp_batch_set_scenes has not been called"), RELCP_ERR_STATE;
    const std::string key = tune_key(b);
    std::vector<std::pair<std::string, int>> cache;
    read_cache(cache_path, cache);
    for (auto& e : cache)
        if (e.first == key && e.second >= 32 && e.second <= 1024 && e.second % 32 == 0) {
            b->threads = e.second;
            if (threads_out) *threads_out = e.second;
            return RELCP_OK;
        }
    // time two steps per candidate from the same state, then restore it
    cudaStream_t st = b->s;
    const size_t N = (size_t)(b->N > 0 ? b->N : 1);
    DBuf<double> bx, bq, bv, bg;
    DBuf<int> bk, bc;
    DBuf<relcp_scene_stats> bs;
    relcp_status rs = RELCP_OK;
    auto save = [&](auto& dst, auto& src, size_t count) -> relcp_status {
        RELCP_TRY(dst.ensure(count, st));
        RELCP_CUDA(cudaMemcpyAsync(dst.p, src.p, count * sizeof(*src.p), cudaMemcpyDeviceToDevice, st));
        return RELCP_OK;
    };
    auto restore = [&](auto& dst, auto& src, size_t count) -> relcp_status {
        RELCP_CUDA(cudaMemcpyAsync(dst.p, src.p, count * sizeof(*src.p), cudaMemcpyDeviceToDevice, st));
        return RELCP_OK;
    };
    const size_t Pt = (size_t)(b->Ptot > 0 ? b->Ptot : 1);
    if (rs == RELCP_OK) rs = save(bx, b->x, 3 * N);
    if (rs == RELCP_OK) rs = save(bq, b->q, 4 * N);
    if (rs == RELCP_OK) rs = save(bv, b->vel, 6 * N);
    if (rs == RELCP_OK) rs = save(bg, b->wgam, Pt);
    if (rs == RELCP_OK) rs = save(bk, b->wkey, Pt);
    if (rs == RELCP_OK) rs = save(bc, b->wcount, (size_t)b->S);
    if (rs == RELCP_OK) rs = save(bs, b->stats, (size_t)b->S);
    const int cands[4] = {64, 128, 256, 512};
    int best = kDefaultThreads;
    float best_ms = 0.f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rs == RELCP_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rs = RELCP_ERR_CUDA;
    for (int c = 0; c < 4 && rs == RELCP_OK; ++c) {
        cudaGraphExec_t exec = nullptr;
        rs = graph_for(b, 2, cands[c], &exec);
        if (rs != RELCP_OK) {
            // a block size the kernel cannot run with is skipped
            rs = RELCP_OK;
            continue;
        }
        float ms = 0.f;
        if (cudaMemsetAsync(b->status.p, 0, sizeof(int), st) != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess ||
            cudaGraphLaunch(exec, st) != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rs = RELCP_ERR_CUDA;
            break;
        }
        if (best_ms == 0.f || ms < best_ms) {
            best_ms = ms;
            best = cands[c];
        }
        rs = restore(b->x, bx, 3 * N);
        if (rs == RELCP_OK) rs = restore(b->q, bq, 4 * N);
        if (rs == RELCP_OK) rs = restore(b->vel, bv, 6 * N);
        if (rs == RELCP_OK) rs = restore(b->wgam, bg, Pt);
        if (rs == RELCP_OK) rs = restore(b->wkey, bk, Pt);
        if (rs == RELCP_OK) rs = restore(b->wcount, bc, (size_t)b->S);
        if (rs == RELCP_OK) rs = restore(b->stats, bs, (size_t)b->S);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    bx.release(st);
    bq.release(st);
    bv.release(st);
    bg.release(st);
    bk.release(st);
    bc.release(st);
    bs.release(st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rs == RELCP_OK) rs = RELCP_ERR_CUDA;
    if (rs != RELCP_OK) return rs;
    b->threads = best;
    if (threads_out) *threads_out = best;
    if (cache_path) {
        cache.emplace_back(key, best);
        if (!write_cache(cache_path, cache)) return set_error("cannot write %s", cache_path), RELCP_ERR_INVALID_ARG;
    }
    return RELCP_OK;
}

extern "C" void relcp_batch_destroy(relcp_batch* b) {
    if (!b) return;
    cudaStream_t s = b->s;
    cudaStreamSynchronize(s);
    drop_graphs(b);
    DBuf<int>* ib[] = {&b->order, &b->boff, &b->poff, &b->roff, &b->work, &b->status, &b->wcount, &b->pa, &b->pb,
                       &b->flags, &b->wkey, &b->ia, &b->ib, &b->inc, &b->inc_tmp, &b->rrec, &b->rpair};
    for (auto* p : ib) p->release(s);
    DBuf<double>* db[] = {&b->x, &b->q, &b->axes, &b->vel, &b->fext, &b->P, &b->K, &b->rb, &b->ufree, &b->uc,
                          &b->ustep, &b->xt, &b->qt, &b->Pt, &b->s0, &b->s1, &b->wgam, &b->geom, &b->qd, &b->diag,
                          &b->gamma, &b->gg, &b->ucp};
    for (auto* p : db) p->release(s);
    b->Kf.release(s);
    b->geomf.release(s);
    b->qf.release(s);
    b->sp.release(s);
    b->stats.release(s);
    cudaStreamSynchronize(s);
    if (b->hstatus) cudaFreeHost(b->hstatus);
    if (b->own_stream) cudaStreamDestroy(s);
    delete b;
}
