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
// Steps alternate BB1 = s^T s / s^T y and BB2 = s^T y / y^T y.  On the mixed
// path the step length of iteration k+1 comes from the products of iteration
// k-1 (Barzilai-Borwein with one retard, Friedlander, Martinez, Molina and
// Raydan, SIAM J. Numer. Anal. 36, 1999): those partials are complete one
// barrier earlier, so every block folds them while it gathers and the
// iteration needs no grid-wide read after its second barrier except on the
// residual checks (every second iteration).  The FP64 path checks every
// iteration and keeps the plain alternation.
//
// On the mixed path, when every row has a thread of its own, the second grid
// barrier goes too (scatter_1b): phase 1 of iteration k waits, by polling,
// only for the records of the rows incident to its body, and the residual
// test is folded one iteration late like the step length.  There the FP64
// residual is certified from FP32 arithmetic with a rounding-error bound and
// evaluated in FP64 only for the rows within that bound of the tolerance
// (resid_certified): the same stop decisions at a fraction of the FP64 issue
// slots, which this part has few of.
//
// On the mixed path both loops hand over to an iterative refinement inside the
// launch (refine_solve): once the FP32 iterations are below 10 x tol and a few
// more have not reached tol, or when they stall, the residual of the iterate
// is taken in FP64 and the correction solved in FP32 (up to eight rounds), so
// the FP32 rounding of the nearly cancelling contact forces no longer bounds
// the attainable residual.
//
// The grid barrier spins a bounded number of times; a timeout sets
// DEV_TIMEOUT and the kernel returns.  Data written inside the launch is read
// with ld.global.cg or ld.relaxed.gpu (L2), never from a possibly stale L1
// line.
#include <cooperative_groups.h>

#include "relcp_internal.cuh"

namespace relcp {

namespace {

#ifndef RELCP_LCP_THREADS
#define RELCP_LCP_THREADS 640
#endif
#ifndef RELCP_LCP_INC_PER_LANE
#define RELCP_LCP_INC_PER_LANE 5
#endif
// 640 threads leave 96 registers per thread at one CTA per SM: the row and
// body slots and the 10 register-resident incidences per body fit, with a few
// spilled words in the mixed kernel (ptxas: 52 B of spill stores)
constexpr int kThreads = RELCP_LCP_THREADS;
constexpr int kMaxCtasPerSm = 1;
constexpr int kMixedCheckEvery = 2;  // mixed path: FP64 termination residual every 2nd iteration
#ifndef RELCP_REFINE_WAIT
#define RELCP_REFINE_WAIT 8
#endif
constexpr int kRefineWait = RELCP_REFINE_WAIT;  // iterations past tol_a before the refinement

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_status(const int* p) { return *(const volatile int*)p; }

#ifdef RELCP_LCP_TRACE
// optional phase timing of block 0 (nanoseconds summed over iterations):
// [0] scatter, [1] barrier 1, [2] gather, [3] block reduction + partials,
// [4] barrier 2, [5] grid reduction + step length, [6] iterations
__device__ unsigned long long g_lcp_trace[8];
#define TRACE_MARK(k)                                                            \
    do {                                                                         \
        if (blockIdx.x == 0 && threadIdx.x == 0) {                               \
            unsigned long long t_ = gtimer();                                    \
            g_lcp_trace[k] += t_ - t_prev;                                       \
            t_prev = t_;                                                         \
        }                                                                        \
    } while (0)
#else
#define TRACE_MARK(k) \
    do {              \
    } while (0)
#endif
constexpr int kNred = 4;  // ss, sy, yy, residual-or-maxdiag

template <class R>
struct Vec2;
template <>
struct Vec2<float> {
    using T = float2;
};
template <>
struct Vec2<double> {
    using T = double2;
};

template <class R>
struct KArgs {
    int nbodies;
    const int* nrows_dev;  // number of rows, read once at kernel start
    const int* __restrict__ ia;
    const int* __restrict__ ib;
    const R* geom[9];
    const double* __restrict__ q;     // offsets (FP64)
    const R* __restrict__ qr;          // offsets in the solve precision (== q when R = double)
    const double* __restrict__ diag;
    const R* __restrict__ invd;  // 1 / A_aa in the solve precision (Jacobi-scaled steps) or null
    const R* K[7];     // body operator in the solve precision
    const int* __restrict__ inc_off;
    const int* __restrict__ inc;
    R* gamma_io;         // caller's gamma (in: warm start, out: solution), SoA
    typename Vec2<R>::T* gg[2];  // (gamma, g) per row, double-buffered
    R* ucp;              // contact velocity, one 8-wide record per body (6 used)
    R* ucp2;             // the second such buffer (one-barrier iterations, mixed path) or null
    double* ucd[6];      // double output (SoA)
    double c, tol;
    int max_iter;
    int check_every;  // FP64 residual on every check_every-th iteration (and the first)
    unsigned long long* partials;  // two buffers of kMaxBlocks x kNred words (see block_partials)
    unsigned* bar;
    int* status;
    LcpDevResult* result;
    unsigned long long wait_ns;  // bound of every wait (grid barrier, row records)
    int skip_block;              // fault injection: the last block leaves before its first barrier arrival
    // iterative refinement (one-barrier mixed path): the one-barrier
    // iterations stop at tol_a (> tol when refinement is on), then an FP64
    // residual with the FP64 operator K64 (offsets g64, per row) and an FP32
    // correction solve to tol
    double tol_a;
    const double* K64[7];
    double* g64;
};

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier on a monotonic arrival counter (zeroed before the
// launch): barrier number e of the launch completes when the counter reaches
// e * gridDim.x.  After a __syncthreads, thread 0 of each block arrives with
// a release add (which publishes every write the block made before the
// __syncthreads) and polls with acquire loads (the block's later reads see
// every block's published writes).  It sleeps only after a short busy spin.
// Each poll also loads the status word (issued before the acquire load, so
// both are in flight together): a DEV_TIMEOUT set anywhere in the grid ends
// the wait, and so does a wait longer than wait_ns (globaltimer), which sets
// DEV_TIMEOUT.  Returns false on either; the caller returns from the kernel.
__device__ bool grid_barrier(unsigned* count, unsigned* epoch, int* status, unsigned long long wait_ns) {
    __shared__ int timed_out;
    __syncthreads();
    if (threadIdx.x == 0) {
        timed_out = 0;
        const unsigned target = (++(*epoch)) * gridDim.x;
        red_add_release(count, 1u);
        long long spins = 0;
        unsigned long long t0 = 0;
        for (;;) {
            const int st = ld_status(status);
            const unsigned cnt = ld_acquire(count);
            if (st & DEV_TIMEOUT) {
                timed_out = 1;
                break;
            }
            if (cnt >= target) break;
            if (++spins > 256) {
                __nanosleep(16);
                if ((spins & 63) == 0) {
                    const unsigned long long t = gtimer();
                    if (t0 == 0) {
                        t0 = t;
                    } else if (t - t0 > wait_ns) {
                        atomicOr(status, DEV_TIMEOUT);
                        timed_out = 1;
                        break;
                    }
                }
            }
        }
    }
    __syncthreads();
    return timed_out == 0;
}

// Deterministic block reduction of kNred values; slot k is a max when bit k
// of maxmask is set, a sum otherwise.  A is the accumulation type: the mixed
// path reduces its FP32 inner products in FP32 inside the block (FP64 is slow
// on this part); only the per-block results are widened to FP64.
template <class A>
__device__ void block_reduce_store(const A v[kNred], unsigned maxmask, double* out) {
    __shared__ A sh[kThreads / 32][kNred];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kNred; ++k) {
        A x = v[k];
        for (int o = 16; o > 0; o >>= 1) {
            A y = __shfl_down_sync(0xffffffffu, x, o);
            x = ((maxmask >> k) & 1u) ? (x > y ? x : y) : x + y;
        }
        if (lane == 0) sh[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < kNred) {
        int k = threadIdx.x;
        A x = sh[0][k];
        for (int w = 1; w < kThreads / 32; ++w) x = ((maxmask >> k) & 1u) ? (x > sh[w][k] ? x : sh[w][k]) : x + sh[w][k];
        out[k] = (double)x;
    }
    __syncthreads();
}

// Partials are 64-bit words, kNred per block.  A sum slot holds the bits of a
// value in the solve precision R (the mixed path sums in FP32: FP64 runs at a
// small fraction of the FP32 rate on this part); a max slot holds the bits of a
// non-negative double, whose maximum is the unsigned maximum of the bit
// patterns.  The integer max needs no FP64 unit, and a NaN residual (bits
// above +inf) survives it and fails the convergence test, where fmax would
// drop it.
__device__ __forceinline__ unsigned long long to_word(float x) { return (unsigned long long)__float_as_uint(x); }
__device__ __forceinline__ unsigned long long to_word(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
template <class R>
__device__ __forceinline__ R from_word(unsigned long long w);
template <>
__device__ __forceinline__ float from_word<float>(unsigned long long w) {
    return __uint_as_float((unsigned)w);
}
template <>
__device__ __forceinline__ double from_word<double>(unsigned long long w) {
    return __longlong_as_double((long long)w);
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long x, unsigned long long y) {
    return x > y ? x : y;
}

// Fold all blocks' partials (staged in shared memory, kNred words per block)
// in a fixed order: warp k folds slot k (lane-strided sums, then a shuffle
// tree), slot k a max when bit k of maxmask is set, a sum in the solve
// precision R otherwise; only the slots in `slots` are folded.  The results
// land in out[k] (shared); the caller's next __syncthreads publishes them.
constexpr int kMaxBlocks = 256;
template <class R>
__device__ __forceinline__ void fold_slots(const unsigned long long* buf, unsigned slots, unsigned maxmask,
                                           unsigned long long* out) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < kNred && ((slots >> w) & 1u)) {
        if ((maxmask >> w) & 1u) {
            unsigned long long m = 0;
            for (int b = lane; b < (int)gridDim.x; b += 32) m = umax64(m, buf[b * kNred + w]);
            for (int o = 16; o > 0; o >>= 1) m = umax64(m, __shfl_down_sync(0xffffffffu, m, o));
            if (lane == 0) out[w] = m;
        } else {
            R x = R(0);
            for (int b = lane; b < (int)gridDim.x; b += 32) x += from_word<R>(buf[b * kNred + w]);
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) out[w] = to_word(x);
        }
    }
}

// every block: reduce all blocks' partials in a fixed order.  All partials
// are fetched at once (one L2 round trip, one word per thread) into shared
// memory and folded one slot per warp; every thread gets the reduced words.
template <class R>
__device__ void grid_reduce(const unsigned long long* partials, unsigned maxmask, unsigned long long tot[kNred]) {
    __shared__ unsigned long long buf[kMaxBlocks * kNred];
    __shared__ unsigned long long red[kNred];
    const int n = gridDim.x * kNred;
    for (int t = threadIdx.x; t < n; t += blockDim.x) buf[t] = __ldcg(partials + t);
    __syncthreads();
    fold_slots<R>(buf, (1u << kNred) - 1u, maxmask, red);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kNred; ++k) tot[k] = red[k];
}

// the BB step length after an iteration with products ss, sy, yy (BB1 after
// odd iterations, BB2 after even ones); a non-positive or non-finite ratio
// keeps the previous step
template <class R>
__device__ __forceinline__ R bb_step(int it, R ss, R sy, R yy, R prev) {
    R na;
    if (it & 1) na = (sy > R(0)) ? ss / sy : prev;
    else na = (yy > R(0) && sy > R(0)) ? sy / yy : prev;
    return (isfinite(na) && na > R(0)) ? na : prev;
}

// per-block partials of an iteration: the three BB products (sums in the
// solve precision) and, on check iterations, the residual word resw (a max:
// the bits of a non-negative double, or on the one-barrier path those of a
// non-negative float in the low half; 0 otherwise).  Each
// warp reduces its threads' values by shuffles; then warp 0 folds the warps'
// values (all four slots at once) and writes the block's words, while warp 1
// (when `prev` is given) folds the previous iteration's partials of all
// blocks, staged in shared memory, and sets the next step length *alpha.
// Both folds run in a fixed order; the caller's next __syncthreads (the grid
// barrier's) publishes *alpha to the block.
template <class R>
__device__ void block_partials(const R v[3], unsigned long long resw, unsigned long long* out,
                               const unsigned long long* prev, int it, R* alpha, bool prev_res = false,
                               unsigned* prev_res_max = nullptr) {
    constexpr int kWarps = kThreads / 32;
    static_assert(kWarps <= 32, "one lane per warp in the fold");
    __shared__ R sh[kWarps][3];
    __shared__ unsigned long long shr[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    R x[3] = {v[0], v[1], v[2]};
    unsigned long long m = resw;
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] += __shfl_down_sync(0xffffffffu, x[k], o);
        m = umax64(m, __shfl_down_sync(0xffffffffu, m, o));
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) sh[wid][k] = x[k];
        shr[wid] = m;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = lane < kWarps ? sh[lane][k] : R(0);
        m = lane < kWarps ? shr[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) x[k] += __shfl_down_sync(0xffffffffu, x[k], o);
            m = umax64(m, __shfl_down_sync(0xffffffffu, m, o));
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) out[k] = to_word(x[k]);
            out[3] = m;
        }
    } else if (wid == 2 && prev && prev_res) {
        // the previous iteration's residual (FP32 bits, rounded up): max over
        // the blocks' low halves
        unsigned mm = 0u;
        for (int b = lane; b < (int)gridDim.x; b += 32) mm = max(mm, (unsigned)prev[b * kNred + 3]);
        for (int o = 16; o > 0; o >>= 1) mm = max(mm, __shfl_down_sync(0xffffffffu, mm, o));
        if (lane == 0) *prev_res_max = mm;
    } else if (wid == 1 && prev) {
        R y[3] = {R(0), R(0), R(0)};
        for (int b = lane; b < (int)gridDim.x; b += 32)
#pragma unroll
            for (int k = 0; k < 3; ++k) y[k] += from_word<R>(prev[b * kNred + k]);
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 3; ++k) y[k] += __shfl_down_sync(0xffffffffu, y[k], o);
        if (lane == 0) *alpha = bb_step<R>(it, y[0], y[1], y[2], *alpha);
    }
}

// ---------------------------------------------------------------------------
// Per-thread static data.  Every thread owns one body slot (two lanes per
// body, up to kIncPerLane incidences per lane kept in registers with their
// signed row coefficients) and one row slot (ids, geometry, offset, 1/A_aa in
// registers).  They are loaded once per solve; an iteration then only gathers
// the packed (gamma, g) pairs and the packed contact velocities.  Bodies and
// rows beyond one slot per thread, and incidences beyond
// kLanesPerBody x kIncPerLane per body, take the same path with loads.
//
// Packed layouts (fewer L2 sectors per access):
//   gg[buf][r] = (gamma_r, g_r)          one 8-byte (FP32) / 16-byte record
//   ucp[8 b .. 8 b + 5] = K D gamma of b one 32-byte (FP32) / 64-byte record
// ---------------------------------------------------------------------------
constexpr int kLanesPerBody = 2;
constexpr int kIncPerLane = RELCP_LCP_INC_PER_LANE;

template <class R>
struct BodySlot {
    int b;                   // body, or >= nbodies for none
    int e0, e1;              // CSR range of the body
    int code[kIncPerLane];   // (row << 1) | side, or -1
    R c[kIncPerLane][6];     // K times the signed row coefficients: side a (-n, -r_a x n), side b (n, r_b x n)
};

template <class R>
struct RowSlot {
    int r;                   // row, or -1
    int i, j;
    R g[9];
    R q, invd;
    R gm, gv;                // (gamma, g) of the current iterate, carried between iterations
};

template <class R>
__device__ __forceinline__ void load_coefs(const KArgs<R>& a, int code, R c[6]) {
    const int r = code >> 1;
    const bool sideb = code & 1;
    const R sg = sideb ? R(1) : R(-1);
    const int o = sideb ? 6 : 3;
    c[0] = sg * a.geom[0][r];
    c[1] = sg * a.geom[1][r];
    c[2] = sg * a.geom[2][r];
    c[3] = sg * a.geom[o][r];
    c[4] = sg * a.geom[o + 1][r];
    c[5] = sg * a.geom[o + 2][r];
}

template <class R>
__device__ __forceinline__ void load_K(const KArgs<R>& a, int b, R K[7]) {
#pragma unroll
    for (int kk = 0; kk < 7; ++kk) K[kk] = a.K[kk][b];
}

// c <- K c: the body operator applied to one row's coefficients, so that the
// body's contact velocity Uc = K sum_a c_a gamma_a is the plain sum of the
// premultiplied coefficients weighted by gamma (K is symmetric:
// K[0] scalar translation, rotation block (K1 K4 K5; K4 K2 K6; K5 K6 K3))
template <class R>
__device__ __forceinline__ void apply_K(const R K[7], R c[6]) {
    const R r3 = K[1] * c[3] + K[4] * c[4] + K[5] * c[5];
    const R r4 = K[4] * c[3] + K[2] * c[4] + K[6] * c[5];
    const R r5 = K[5] * c[3] + K[6] * c[4] + K[3] * c[5];
    c[0] *= K[0];
    c[1] *= K[0];
    c[2] *= K[0];
    c[3] = r3;
    c[4] = r4;
    c[5] = r5;
}

template <class R>
__device__ void load_body_slot(const KArgs<R>& a, int b, int lane, BodySlot<R>& S) {
    S.b = b;
    S.e0 = S.e1 = 0;
#pragma unroll
    for (int k = 0; k < kIncPerLane; ++k) S.code[k] = -1;
    if (b >= a.nbodies) return;
    S.e0 = a.inc_off[b];
    S.e1 = a.inc_off[b + 1];
    R K[7];
    load_K(a, b, K);
#pragma unroll
    for (int k = 0; k < kIncPerLane; ++k) {
        const int e = S.e0 + lane + kLanesPerBody * k;
        if (e < S.e1) {
            S.code[k] = a.inc[e];
            load_coefs(a, S.code[k], S.c[k]);
            apply_K(K, S.c[k]);
        }
    }
}

template <class R>
__device__ void load_row_slot(const KArgs<R>& a, int r, int nrows, RowSlot<R>& S) {
    S.r = r < nrows ? r : -1;
    if (S.r < 0) return;
    S.i = a.ia[r];
    S.j = a.ib[r];
#pragma unroll
    for (int k = 0; k < 9; ++k) S.g[k] = a.geom[k][r];
    S.q = a.qr[r];
    S.invd = a.invd ? a.invd[r] : R(1);
    S.gm = a.gamma_io[r];
    S.gv = R(0);
}

// the projected step of one row, gamma' = max(0, gamma - alpha g / A_aa), with
// explicit roundings: the body threads of the scatter and the row's own thread
// evaluate it on the same inputs and must agree bit for bit
__device__ __forceinline__ float proj_step(float gm, float g, float invd, float alpha) {
    const float v = __fmaf_rn(-alpha, __fmul_rn(g, invd), gm);
    return v > 0.f ? v : 0.f;
}
__device__ __forceinline__ double proj_step(double gm, double g, double invd, double alpha) {
    const double v = __fma_rn(-alpha, __dmul_rn(g, invd), gm);
    return v > 0.0 ? v : 0.0;
}

template <class R>
__device__ __forceinline__ typename Vec2<R>::T ld_pair(const typename Vec2<R>::T* p) {
    return __ldcg(p);
}

// one incidence: gamma' = P(gamma - alpha g/A_aa) (or gamma), accumulated
// wrench.  A row inside the row slots (r < threads in the grid) gets gamma'
// from its own thread; the side-a body thread stores it for the others.
template <class R>
__device__ __forceinline__ void incidence(const KArgs<R>& a, int code, const R c[6], int src, bool project,
                                          R alpha_r, int nslots, R w[6]) {
    const int r = code >> 1;
    const typename Vec2<R>::T p = ld_pair<R>(a.gg[src] + r);
    R gm = p.x;
    if (project) {
        const R inv = a.invd ? a.invd[r] : R(1);
        gm = proj_step(gm, p.y, inv, alpha_r);
        if (!(code & 1) && r >= nslots) a.gg[1 - src][r].x = gm;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] += gm * c[k];
}

// 8-wide contact-velocity record: vector load / store (16-byte accesses)
__device__ __forceinline__ void load_rec(const float* p, float u[6]) {
    const float4 a = __ldcg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldcg(reinterpret_cast<const float4*>(p) + 1);
    u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w; u[4] = b.x; u[5] = b.y;
}
__device__ __forceinline__ void load_rec(const double* p, double u[6]) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    const double2 c = __ldcg(reinterpret_cast<const double2*>(p) + 2);
    u[0] = a.x; u[1] = a.y; u[2] = b.x; u[3] = b.y; u[4] = c.x; u[5] = c.y;
}
__device__ __forceinline__ void store_rec(float* p, const float u[6]) {
    reinterpret_cast<float4*>(p)[0] = make_float4(u[0], u[1], u[2], u[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(u[4], u[5], 0.f, 0.f);
}
__device__ __forceinline__ void store_rec(double* p, const double u[6]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(u[0], u[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(u[2], u[3]);
    reinterpret_cast<double2*>(p)[2] = make_double2(u[4], u[5]);
}

template <class R>
__device__ __forceinline__ void reduce_lanes(R w[6]) {
#pragma unroll
    for (int sh = kLanesPerBody / 2; sh > 0; sh >>= 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] += __shfl_xor_sync(0xffffffffu, w[k], sh);
}

// phase 1: contact velocity Uc = K D gamma' for every body; gamma' read from
// buffer src (projected step when `project`), written to buffer 1 - src for
// rows outside the row slots.  The slot's coefficients already carry K;
// incidences read from memory are premultiplied on the fly.
template <class R>
__device__ void scatter_phase(const KArgs<R>& a, const BodySlot<R>& S, int src, bool project, R alpha_r) {
    const int lane = threadIdx.x & (kLanesPerBody - 1);
    const int nslots = gridDim.x * blockDim.x;
    {
        R w[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < kIncPerLane; ++k)
            if (S.code[k] >= 0) incidence(a, S.code[k], S.c[k], src, project, alpha_r, nslots, w);
        const int e_over = S.e0 + kLanesPerBody * kIncPerLane + lane;
        if (e_over < S.e1) {
            R K[7];
            load_K(a, S.b, K);
            for (int e = e_over; e < S.e1; e += kLanesPerBody) {
                const int code = a.inc[e];
                R c[6];
                load_coefs(a, code, c);
                apply_K(K, c);
                incidence(a, code, c, src, project, alpha_r, nslots, w);
            }
        }
        reduce_lanes(w);
        if (S.b < a.nbodies && lane == 0) store_rec(a.ucp + 8 * (int64_t)S.b, w);
    }
    // bodies beyond one slot per thread
    const int groups_total = nslots / kLanesPerBody;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / kLanesPerBody;
    const int warp_first = gid & ~(32 / kLanesPerBody - 1);
    for (int k = 1; warp_first + k * groups_total < a.nbodies; ++k) {
        const int b = gid + k * groups_total;
        R w[6] = {0, 0, 0, 0, 0, 0};
        if (b < a.nbodies) {
            R K[7];
            load_K(a, b, K);
            const int e0 = a.inc_off[b], e1 = a.inc_off[b + 1];
            for (int e = e0 + lane; e < e1; e += kLanesPerBody) {
                const int code = a.inc[e];
                R c[6];
                load_coefs(a, code, c);
                apply_K(K, c);
                incidence(a, code, c, src, project, alpha_r, nslots, w);
            }
        }
        reduce_lanes(w);
        if (b < a.nbodies && lane == 0) store_rec(a.ucp + 8 * (int64_t)b, w);
    }
}

// phase 2 for one row: g' = q + c d^T Uc in the solve precision, the BB
// products of s = gamma' - gamma, y = g' - g, and the FP64 natural residual on
// check iterations.  Every load is issued before the row's store.
template <class R>
__device__ __forceinline__ R row_rate(const R g9[9], const R ui[6], const R uj[6]) {
    R rate = g9[0] * (uj[0] - ui[0]) + g9[1] * (uj[1] - ui[1]) + g9[2] * (uj[2] - ui[2]);
    rate += g9[6] * uj[3] + g9[7] * uj[4] + g9[8] * uj[5];
    rate -= g9[3] * ui[3] + g9[4] * ui[4] + g9[5] * ui[5];
    return rate;
}

template <class R>
__device__ __forceinline__ void bb_accumulate(const KArgs<R>& a, R s, R y, R invd, R acc[3]) {
    if (a.invd) {
        // metric diag(A): s^T D s, s^T y, y^T D^-1 y
        acc[0] += s * s / invd;
        acc[1] += s * y;
        acc[2] += y * y * invd;
    } else {
        acc[0] += s * s;
        acc[1] += s * y;
        acc[2] += y * y;
    }
}

// a row outside the row slots: everything from memory; gamma' was stored by
// the side-a body thread of the scatter
template <class R>
__device__ __forceinline__ void row_update_mem(const KArgs<R>& a, int r, int nw, int old, bool check, R acc[3],
                                               double& res) {
    const int i = a.ia[r], j = a.ib[r];
    R g9[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g9[k] = a.geom[k][r];
    const R q = a.qr[r];
    const R invd = a.invd ? a.invd[r] : R(1);
    R ui[6], uj[6];
    load_rec(a.ucp + 8 * (int64_t)i, ui);
    load_rec(a.ucp + 8 * (int64_t)j, uj);
    const R gm = ldcg(&a.gg[nw][r].x);
    typename Vec2<R>::T po;
    if (old >= 0) po = ld_pair<R>(a.gg[old] + r);
    double qd = 0.0, dg = 0.0;
    if (check) {
        qd = a.q[r];
        dg = a.diag[r];
    }
    const R rate = row_rate(g9, ui, uj);
    const R g = q + (R)a.c * rate;
    a.gg[nw][r].y = g;
    if (old >= 0) bb_accumulate(a, gm - po.x, g - po.y, invd, acc);
    if (check) res = fmax(res, fabs(fmin(dg * (double)gm, qd + a.c * (double)rate)));
}

// the thread's own row: (gamma, g) of the current iterate are in registers,
// gamma' is recomputed here with the scatter's projected step, and the new
// pair is written with one store
template <class R>
__device__ __forceinline__ void row_update_slot(const KArgs<R>& a, RowSlot<R>& S, int nw, bool first, bool check,
                                                R alpha_r, R acc[3], double& res) {
    R ui[6], uj[6];
    load_rec(a.ucp + 8 * (int64_t)S.i, ui);
    load_rec(a.ucp + 8 * (int64_t)S.j, uj);
    double qd = 0.0, dg = 0.0;
    if (check) {
        qd = a.q[S.r];
        dg = a.diag[S.r];
    }
    const R gm = first ? S.gm : proj_step(S.gm, S.gv, S.invd, alpha_r);
    const R rate = row_rate(S.g, ui, uj);
    const R g = S.q + (R)a.c * rate;
    typename Vec2<R>::T p;
    p.x = gm;
    p.y = g;
    a.gg[nw][S.r] = p;
    if (!first) bb_accumulate(a, gm - S.gm, g - S.gv, S.invd, acc);
    if (check) res = fmax(res, fabs(fmin(dg * (double)gm, qd + a.c * (double)rate)));
    S.gm = gm;
    S.gv = g;
}

template <class R>
__device__ void gather_phase(const KArgs<R>& a, RowSlot<R>& S, const int nrows, int nw, int old, bool check,
                             R alpha_r, R v[3], double* resid) {
    R acc[3] = {0, 0, 0};
    double res = 0.0;
    if (S.r >= 0) row_update_slot(a, S, nw, old < 0, check, alpha_r, acc, res);
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x + stride; r < nrows; r += stride)
        row_update_mem(a, r, nw, old, check, acc, res);
    v[0] = acc[0];
    v[1] = acc[1];
    v[2] = acc[2];
    *resid = res;
}

// ---------------------------------------------------------------------------
// One grid barrier per iteration (mixed path, every row in a row slot).  A row
// record is one 64-bit word, g's FP32 bits in the high half and gamma's in the
// low half, written and read as a single 64-bit access, so a reader sees one
// iteration's (gamma, g) or another's, never a mix.  gamma >= 0, so its sign
// bit is free: it carries the record's phase, bit 1 of the iteration number,
// which tells the iteration k - 1 that the scatter of iteration k waits for
// from the k - 3 that the same buffer held before.  The scatter of iteration
// k polls only its own incident rows (bounded), so no grid barrier separates
// a gather from the next scatter; the contact-velocity records are
// double-buffered by iteration parity, and the hazards on both buffers are
// ordered by the one remaining barrier (a buffer is rewritten two iterations
// later, after every block has passed the barrier in between).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned rec_phase(int it) { return ((unsigned)it >> 1) & 1u; }
__device__ __forceinline__ unsigned long long ld_rel64(const unsigned long long* p) {
    // (no memory clobber: the loads of a body's incidences are issued together;
    // a stale word is caught by its phase bit)
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_rel64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long make_rec(float gm, float g, unsigned phase) {
    return ((unsigned long long)__float_as_uint(g) << 32) | (unsigned long long)(__float_as_uint(gm) | (phase << 31));
}
__device__ __forceinline__ bool rec_ok(unsigned long long w, unsigned phase) { return ((unsigned)w >> 31) == phase; }

// the row record of iteration `it` (phase rec_phase(it)), polled until it is
// there; a wait past wait_ns records DEV_TIMEOUT and takes the word as is
// (another thread's timeout ends the wait too), and the grid barrier that
// follows returns false in every block that sees the flag
__device__ __forceinline__ unsigned long long rec_wait(const unsigned long long* p, unsigned long long w,
                                                       unsigned phase, int* status, unsigned long long wait_ns) {
    long long spins = 0;
    unsigned long long t0 = 0;
    while (!rec_ok(w, phase)) {
        ++spins;
        if ((spins & 63) == 0) {
            if (ld_status(status) & DEV_TIMEOUT) break;
            const unsigned long long t = gtimer();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > wait_ns) {
                atomicOr(status, DEV_TIMEOUT);
                break;
            }
        }
        if (spins > 16) __nanosleep(20);
        w = ld_rel64(p);
    }
    return w;
}

__device__ __forceinline__ void incidence_1b(const KArgs<float>& a, int code, const float c[6],
                                             const unsigned long long* rec, unsigned phase, float alpha_r,
                                             unsigned long long w0, float w[6]) {
    const int r = code >> 1;
    const unsigned long long wv = rec_ok(w0, phase) ? w0 : rec_wait(rec + r, w0, phase, a.status, a.wait_ns);
    const float gm0 = fabsf(__uint_as_float((unsigned)wv));
    const float g0 = __uint_as_float((unsigned)(wv >> 32));
    const float inv = a.invd ? a.invd[r] : 1.f;
    const float gm = proj_step(gm0, g0, inv, alpha_r);
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] += gm * c[k];
}

// phase 1 of iteration it: Uc(it) = K D gamma(it) from the records of it - 1
__device__ void scatter_1b(const KArgs<float>& a, const BodySlot<float>& S, const unsigned long long* rec,
                           unsigned phase, float* ucp, float alpha_r) {
    const int lane = threadIdx.x & (kLanesPerBody - 1);
    float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    unsigned long long w0[kIncPerLane];
#pragma unroll
    for (int k = 0; k < kIncPerLane; ++k) w0[k] = S.code[k] >= 0 ? ld_rel64(rec + (S.code[k] >> 1)) : 0ull;
#pragma unroll
    for (int k = 0; k < kIncPerLane; ++k)
        if (S.code[k] >= 0) incidence_1b(a, S.code[k], S.c[k], rec, phase, alpha_r, w0[k], w);
    const int e_over = S.e0 + kLanesPerBody * kIncPerLane + lane;
    if (e_over < S.e1) {
        float K[7];
        load_K(a, S.b, K);
        for (int e = e_over; e < S.e1; e += kLanesPerBody) {
            const int code = a.inc[e];
            float c[6];
            load_coefs(a, code, c);
            apply_K(K, c);
            incidence_1b(a, code, c, rec, phase, alpha_r, ld_rel64(rec + (code >> 1)), w);
        }
    }
    reduce_lanes(w);
    if (S.b < a.nbodies && lane == 0) store_rec(ucp + 8 * (int64_t)S.b, w);
    // bodies beyond one slot per thread
    const int nslots = gridDim.x * blockDim.x;
    const int groups_total = nslots / kLanesPerBody;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / kLanesPerBody;
    const int warp_first = gid & ~(32 / kLanesPerBody - 1);
    for (int k = 1; warp_first + k * groups_total < a.nbodies; ++k) {
        const int b = gid + k * groups_total;
        float wb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (b < a.nbodies) {
            float K[7];
            load_K(a, b, K);
            const int e0 = a.inc_off[b], e1 = a.inc_off[b + 1];
            for (int e = e0 + lane; e < e1; e += kLanesPerBody) {
                const int code = a.inc[e];
                float c[6];
                load_coefs(a, code, c);
                apply_K(K, c);
                incidence_1b(a, code, c, rec, phase, alpha_r, ld_rel64(rec + (code >> 1)), wb);
            }
        }
        reduce_lanes(wb);
        if (b < a.nbodies && lane == 0) store_rec(ucp + 8 * (int64_t)b, wb);
    }
}

// The termination residual of one row, |min(A_aa gamma, q + c rate)| with q,
// A_aa and c in FP64 and gamma and the rate as the FP32 iterate holds them
// (the FP64 test), decided from FP32 arithmetic where FP32 suffices.  The FP32
// value r32 = |min(A32 gamma, q32 + c32 rate)| (q32 the FP32 offset) differs
// from the FP64 one by less than e = 2^-21 max(|q32| + |c32 rate|, A32 gamma)
// (the roundings of q, c, A_aa, the product and the sum, each at most 2^-24 or
// 2^-23 of its operands; min and abs are 1-Lipschitz; A32 is trunc_f32 of the
// FP64 A_aa).  The loop decides
// against two thresholds, tol and tol_a >= tol (th: tol and tol_a rounded
// down and up to FP32).  A row whose interval [r32 - e, r32 + e] lies below
// tol contributes r32 + e; above tol_a, r32 - e; strictly between them,
// r32 + e; only a row whose interval straddles a threshold evaluates the FP64
// expression, rounded up to FP32.  The fold's max then decides "<= tol" and
// "<= tol_a" exactly as the FP64 residuals rounded up to FP32 would, and
// bounds the FP64 residual from above when it stops.
__device__ __forceinline__ float resid_certified(const KArgs<float>& a, int r, double dg, float gm, float q32, float cr,
                                                 float g, float rate, const float* th) {
    const float p = trunc_f32(dg) * gm;  // (exact: the mixed rows' A_aa is a widened float)
    const float r32 = fabsf(fminf(p, g));
    const float e = 0x1p-21f * fmaxf(fabsf(q32) + fabsf(cr), p);
    const float up = __fadd_ru(r32, e);
    const float lo = __fsub_rd(r32, e);
    if (up <= th[0]) return up;                       // below tol
    if (lo > th[3]) return lo;                        // above tol_a
    if (lo > th[1] && up <= th[2]) return up;         // in (tol, tol_a]
    const double qd = a.q[r];
    return __double2float_ru(fabs(fmin(dg * (double)gm, qd + a.c * (double)rate)));
}

// phase 2 of iteration it for the thread's row: g(it) from Uc(it), the record
// of it, the BB products and (check) the residual as FP32 bits (resid_certified)
__device__ __forceinline__ void gather_1b(const KArgs<float>& a, RowSlot<float>& S, const float* ucp,
                                          unsigned long long* rec, unsigned phase, bool check, float alpha_r,
                                          const float* tol_lohi, float v[3], unsigned* resid_bits) {
    float acc[3] = {0.f, 0.f, 0.f};
    float res = 0.f;
    if (S.r >= 0) {
        float ui[6], uj[6];
        load_rec(ucp + 8 * (int64_t)S.i, ui);
        load_rec(ucp + 8 * (int64_t)S.j, uj);
        // (A_aa is loaded with the velocity records: the record store below is
        // a compiler barrier, and a load after it would be a second round trip)
        const double dg = check ? a.diag[S.r] : 0.0;
        const float gm = proj_step(S.gm, S.gv, S.invd, alpha_r);
        const float rate = row_rate(S.g, ui, uj);
        const float cr = (float)a.c * rate;
        const float g = S.q + cr;
        st_rel64(rec + S.r, make_rec(gm, g, phase));
        bb_accumulate(a, gm - S.gm, g - S.gv, S.invd, acc);
        if (check) res = resid_certified(a, S.r, dg, gm, S.q, cr, g, rate, tol_lohi);
        S.gm = gm;
        S.gv = g;
    }
    v[0] = acc[0];
    v[1] = acc[1];
    v[2] = acc[2];
    *resid_bits = __float_as_uint(res);
}

// ---------------------------------------------------------------------------
// Iterative refinement of the one-barrier solve.  FP32 iterates stall where
// the rounding of the wrench sums (relative 2^-24 of the summed contact
// forces, which nearly cancel on a body in a dense packing) reaches the stop;
// so the one-barrier iterations stop at tol_a, and then
//   (1) the FP64 residual of that iterate gamma1 (held in gamma_io): per body
//       U1 = K D gamma1 in FP64 (the rows' FP32 geometry widened, which is
//       exact, and the FP64 operator), kept in the FP64 output ucd; per row
//       g64 = q + c d^T (U1_j - U1_i) and |min(A_aa gamma1, g64)|;
//   (2) if that residual is above tol: projected Barzilai-Borwein in FP32 on
//       the correction delta >= -gamma1 of g = g64 + A delta, two grid
//       barriers per iteration (the records hold delta, which has no free
//       sign bit), the FP64 residual |min(A_aa (gamma1 + delta), g64 + c d^T
//       K D delta)| every second iteration.  The rounding of these iterations
//       scales with the correction, not with the forces;
//   (3) gamma = gamma1 + delta and Uc = U1 + K D delta.
// Mixed-precision iterative refinement (an FP64 residual, an FP32 solve of the
// correction), applied to the complementarity problem.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float proj_step_lb(float gm, float g, float invd, float alpha, float lb) {
    const float v = __fmaf_rn(-alpha, __fmul_rn(g, invd), gm);
    return v > lb ? v : lb;
}

// (1a) U1 = K D gamma1 per body in FP64 into ucd (two lanes per body)
__device__ void refine_scatter64(const KArgs<float>& a) {
    const int lane = threadIdx.x & (kLanesPerBody - 1);
    const int groups_total = (int)(gridDim.x * blockDim.x) / kLanesPerBody;
    const int gid = (int)(blockIdx.x * blockDim.x + threadIdx.x) / kLanesPerBody;
    const int warp_first = gid & ~(32 / kLanesPerBody - 1);
    for (int k = 0; warp_first + k * groups_total < a.nbodies; ++k) {
        const int b = gid + k * groups_total;
        double w[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (b < a.nbodies) {
            const int e0 = a.inc_off[b], e1 = a.inc_off[b + 1];
            for (int e = e0 + lane; e < e1; e += kLanesPerBody) {
                const int code = a.inc[e];
                const int r = code >> 1;
                const double gm = (double)__ldcg(a.gamma_io + r);
                const double sg = (code & 1) ? gm : -gm;
                const int o = (code & 1) ? 6 : 3;
                w[0] += sg * (double)a.geom[0][r];
                w[1] += sg * (double)a.geom[1][r];
                w[2] += sg * (double)a.geom[2][r];
                w[3] += sg * (double)a.geom[o][r];
                w[4] += sg * (double)a.geom[o + 1][r];
                w[5] += sg * (double)a.geom[o + 2][r];
            }
        }
        reduce_lanes(w);
        if (b < a.nbodies && lane == 0) {
            double K[7];
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) K[kk] = a.K64[kk][b];
            apply_K(K, w);
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) a.ucd[kk][b] = w[kk];
        }
    }
}

// (1b) the thread's row: g64 and its FP64 residual; the row slot and the
// record of buffer 0 become the correction problem's start (delta = 0, g = g64)
__device__ double refine_row64(const KArgs<float>& a, RowSlot<float>& S) {
    if (S.r < 0) return 0.0;
    double ui[6], uj[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        ui[k] = __ldcg(a.ucd[k] + S.i);
        uj[k] = __ldcg(a.ucd[k] + S.j);
    }
    double rate = (double)S.g[0] * (uj[0] - ui[0]) + (double)S.g[1] * (uj[1] - ui[1]) +
                  (double)S.g[2] * (uj[2] - ui[2]);
    rate += (double)S.g[6] * uj[3] + (double)S.g[7] * uj[4] + (double)S.g[8] * uj[5];
    rate -= (double)S.g[3] * ui[3] + (double)S.g[4] * ui[4] + (double)S.g[5] * ui[5];
    const double g64 = a.q[S.r] + a.c * rate;
    a.g64[S.r] = g64;
    const double g1 = (double)__ldcg(a.gamma_io + S.r);
    S.q = trunc_f32(g64);
    S.gm = 0.f;
    S.gv = S.q;
    a.gg[0][S.r] = make_float2(0.f, S.q);
    return fabs(fmin(a.diag[S.r] * g1, g64));
}

// (1b) a row beyond the row slots: g64 and its FP64 residual, the record of
// buffer 0 = (0, g64 truncated to FP32, as for the slot rows)
__device__ double refine_row64_mem(const KArgs<float>& a, int r) {
    const int i = a.ia[r], j = a.ib[r];
    double g9[9], ui[6], uj[6];
#pragma unroll
    for (int k = 0; k < 9; ++k) g9[k] = (double)a.geom[k][r];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        ui[k] = __ldcg(a.ucd[k] + i);
        uj[k] = __ldcg(a.ucd[k] + j);
    }
    double rate = g9[0] * (uj[0] - ui[0]) + g9[1] * (uj[1] - ui[1]) + g9[2] * (uj[2] - ui[2]);
    rate += g9[6] * uj[3] + g9[7] * uj[4] + g9[8] * uj[5];
    rate -= g9[3] * ui[3] + g9[4] * ui[4] + g9[5] * ui[5];
    const double g64 = a.q[r] + a.c * rate;
    a.g64[r] = g64;
    a.gg[0][r] = make_float2(0.f, trunc_f32(g64));
    return fabs(fmin(a.diag[r] * (double)__ldcg(a.gamma_io + r), g64));
}

// (2) a row beyond the row slots: delta' (stored by the side-a body thread of
// the scatter), g = g64 + c d^T K D delta', the BB products, the residual
__device__ __forceinline__ void refine_gather_mem(const KArgs<float>& a, int r, int nw, int old, bool check,
                                                  float acc[3], double& res) {
    const int i = a.ia[r], j = a.ib[r];
    float g9[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g9[k] = a.geom[k][r];
    float ui[6], uj[6];
    load_rec(a.ucp + 8 * (int64_t)i, ui);
    load_rec(a.ucp + 8 * (int64_t)j, uj);
    const double g64 = a.g64[r];
    const float dl = __ldcg(&a.gg[nw][r].x);
    const float2 po = __ldcg(a.gg[old] + r);
    const float invd = a.invd ? a.invd[r] : 1.f;
    const float rate = row_rate(g9, ui, uj);
    const float g = trunc_f32(g64) + (float)a.c * rate;
    a.gg[nw][r].y = g;
    bb_accumulate(a, dl - po.x, g - po.y, invd, acc);
    if (check)
        res = fmax(res, fabs(fmin(a.diag[r] * ((double)__ldcg(a.gamma_io + r) + (double)dl), g64 + a.c * (double)rate)));
}

// (2) scatter: K D delta' with delta' = max(-gamma1, delta - alpha g / A_aa)
// from the records gg[src] (every row has a row slot on this path)
__device__ void refine_scatter(const KArgs<float>& a, const BodySlot<float>& S, int src, float alpha_r) {
    const int lane = threadIdx.x & (kLanesPerBody - 1);
    const int nslots = gridDim.x * blockDim.x;
    auto inc = [&](int code, const float c[6], float w[6]) {
        const int r = code >> 1;
        const float2 p = __ldcg(a.gg[src] + r);
        const float inv = a.invd ? a.invd[r] : 1.f;
        const float dl = proj_step_lb(p.x, p.y, inv, alpha_r, -__ldcg(a.gamma_io + r));
        if (!(code & 1) && r >= nslots) a.gg[1 - src][r].x = dl;  // rows beyond the row slots
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] += dl * c[k];
    };
    {
        float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kIncPerLane; ++k)
            if (S.code[k] >= 0) inc(S.code[k], S.c[k], w);
        const int e_over = S.e0 + kLanesPerBody * kIncPerLane + lane;
        if (e_over < S.e1) {
            float K[7];
            load_K(a, S.b, K);
            for (int e = e_over; e < S.e1; e += kLanesPerBody) {
                const int code = a.inc[e];
                float c[6];
                load_coefs(a, code, c);
                apply_K(K, c);
                inc(code, c, w);
            }
        }
        reduce_lanes(w);
        if (S.b < a.nbodies && lane == 0) store_rec(a.ucp + 8 * (int64_t)S.b, w);
    }
    const int groups_total = nslots / kLanesPerBody;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / kLanesPerBody;
    const int warp_first = gid & ~(32 / kLanesPerBody - 1);
    for (int k = 1; warp_first + k * groups_total < a.nbodies; ++k) {
        const int b = gid + k * groups_total;
        float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (b < a.nbodies) {
            float K[7];
            load_K(a, b, K);
            const int e0 = a.inc_off[b], e1 = a.inc_off[b + 1];
            for (int e = e0 + lane; e < e1; e += kLanesPerBody) {
                const int code = a.inc[e];
                float c[6];
                load_coefs(a, code, c);
                apply_K(K, c);
                inc(code, c, w);
            }
        }
        reduce_lanes(w);
        if (b < a.nbodies && lane == 0) store_rec(a.ucp + 8 * (int64_t)b, w);
    }
}

// (2) gather for the thread's row: the same projected step, g = g64 + c d^T
// K D delta', the record of buffer nw, the BB products and (check) the FP64
// residual of gamma1 + delta'
__device__ __forceinline__ void refine_gather(const KArgs<float>& a, RowSlot<float>& S, int nw, bool check,
                                              float alpha_r, float v[3], double* resid) {
    float acc[3] = {0.f, 0.f, 0.f};
    double res = 0.0;
    if (S.r >= 0) {
        float ui[6], uj[6];
        load_rec(a.ucp + 8 * (int64_t)S.i, ui);
        load_rec(a.ucp + 8 * (int64_t)S.j, uj);
        const float g1 = __ldcg(a.gamma_io + S.r);
        const float dl = proj_step_lb(S.gm, S.gv, S.invd, alpha_r, -g1);
        const float rate = row_rate(S.g, ui, uj);
        const float g = S.q + (float)a.c * rate;
        a.gg[nw][S.r] = make_float2(dl, g);
        bb_accumulate(a, dl - S.gm, g - S.gv, S.invd, acc);
        if (check)
            res = fabs(fmin(a.diag[S.r] * ((double)g1 + (double)dl), a.g64[S.r] + a.c * (double)rate));
        S.gm = dl;
        S.gv = g;
    }
    v[0] = acc[0];
    v[1] = acc[1];
    v[2] = acc[2];
    *resid = res;
}

constexpr int kRefineRounds = 8;        // FP64 residual passes per solve at most
constexpr int kStallIters = 128;        // FP32 iterations: no 10% residual decrease in this many is a stall
constexpr int kStallItersRefine = 256;  // the same for a correction solve

// The residual history of a loop: a stall is `window` iterations in which the
// smallest checked residual has not fallen by 10% (BB is not monotone, and a
// near-singular LCP converges slowly without stalling; a stalled one stops
// improving altogether).  Every thread of every block updates its own copy
// from the same folded residuals, so all take the same decisions.
struct StallWatch {
    double best = 1e300;
    int it_best = 0;
    __device__ bool stalled(double rsd, int it, int window) {
        if (rsd < 0.9 * best) {
            best = rsd;
            it_best = it;
        }
        return it - it_best > window;
    }
};

// Iterative refinement of the mixed solve from the iterate in gamma_io (and
// its velocity in ucd): up to kRefineRounds rounds of (1) the FP64 residual
// and (2) the FP32 correction solve, which ends on tol, on a stall or when the
// rounds' shared budget of max_iter iterations is spent; (3) gamma_io and ucd
// then hold gamma1 + delta and U1 + K D delta, the next round's start.  resid:
// the last residual; it: incremented by the correction iterations.  Returns
// false when a grid barrier timed out (the caller returns from the kernel).
__device__ bool refine_solve(const KArgs<float>& a, const BodySlot<float>& bs, RowSlot<float>& rs, int nrows,
                             unsigned* epoch, float alpha0, unsigned long long* pbuf, double& resid, int& it) {
    __shared__ double sh_part[kNred];
    __shared__ double sh_res;
    __shared__ float sh_alpha;
    constexpr size_t kBuf = (size_t)kMaxBlocks * kNred;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    unsigned long long tot[kNred];
    int budget = a.max_iter;  // correction iterations, all rounds together
    for (int round = 0; round < kRefineRounds && budget > 0; ++round) {
        // (1) gamma1 is complete in gamma_io after this barrier
        if (!grid_barrier(a.bar, epoch, a.status, a.wait_ns)) return false;
        refine_scatter64(a);
        if (!grid_barrier(a.bar, epoch, a.status, a.wait_ns)) return false;
        double r64 = refine_row64(a, rs);
        for (int r = tid + stride; r < nrows; r += stride) r64 = fmax(r64, refine_row64_mem(a, r));
        {
            double w4[kNred] = {0.0, 0.0, 0.0, r64};
            block_reduce_store<double>(w4, 0x8u, sh_part);
            if (threadIdx.x == 0) {
                unsigned long long* o = a.partials + (size_t)blockIdx.x * kNred;
                o[0] = to_word(0.f);
                o[1] = to_word(0.f);
                o[2] = to_word(0.f);
                o[3] = to_word(sh_part[3]);
            }
        }
        if (!grid_barrier(a.bar, epoch, a.status, a.wait_ns)) return false;
        grid_reduce<float>(a.partials, 0x8u, tot);
        resid = from_word<double>(tot[3]);
        if (resid <= a.tol) return true;
        // (2) the correction solve, two grid barriers per iteration; buffer 0
        // holds its start (delta = 0, g = g64)
        float alpha_r = alpha0;
        if (threadIdx.x == 0) sh_alpha = alpha0;
        int cur = 0, itc;
        bool conv = false;
        StallWatch sw;
        for (itc = 1; itc <= budget; ++itc) {
            const bool check = (itc % kMixedCheckEvery) == 0 || itc == budget;
            unsigned long long* pc = a.partials + (size_t)(itc & 1) * kBuf;
            refine_scatter(a, bs, cur, alpha_r);
            if (!grid_barrier(a.bar, epoch, a.status, a.wait_ns)) return false;
            const int npw = (int)gridDim.x * kNred;
            unsigned pf = 0u;
            if (itc >= 2 && (int)threadIdx.x < npw)
                pf = __ldcg(reinterpret_cast<const unsigned*>(a.partials + (size_t)((itc - 1) & 1) * kBuf + threadIdx.x));
            float v[3];
            double res_t;
            refine_gather(a, rs, 1 - cur, check, alpha_r, v, &res_t);
            {
                float acc[3] = {0.f, 0.f, 0.f};
                for (int r = tid + stride; r < nrows; r += stride) refine_gather_mem(a, r, 1 - cur, cur, check, acc, res_t);
                v[0] += acc[0];
                v[1] += acc[1];
                v[2] += acc[2];
            }
            if (itc >= 2) {
                if ((int)threadIdx.x < npw) pbuf[threadIdx.x] = pf;
                for (int t = threadIdx.x + kThreads; t < npw; t += kThreads)
                    pbuf[t] = (unsigned)__ldcg(a.partials + (size_t)((itc - 1) & 1) * kBuf + t);
            }
            block_partials<float>(v, check ? (unsigned long long)__double_as_longlong(res_t) : 0ull,
                                  pc + (size_t)blockIdx.x * kNred, itc >= 2 ? pbuf : nullptr, itc, &sh_alpha);
            if (!grid_barrier(a.bar, epoch, a.status, a.wait_ns)) return false;
            cur = 1 - cur;
            alpha_r = sh_alpha;
            if (check) {
                grid_reduce<float>(pc, 0x8u, tot);
                if (threadIdx.x == 0) sh_res = from_word<double>(tot[3]);
                __syncthreads();
                const double rsd = sh_res;
                if (rsd <= a.tol) {
                    conv = true;
                    break;
                }
                if (sw.stalled(rsd, itc, kStallItersRefine)) break;
            }
        }
        if (itc > budget) itc = budget;
        it += itc;
        budget -= itc;
        resid = sh_res;
        // (3) gamma = gamma1 + delta (buffer cur), Uc = U1 + K D delta
        for (int r = tid; r < nrows; r += stride) a.gamma_io[r] = __ldcg(a.gamma_io + r) + __ldcg(&a.gg[cur][r].x);
        for (int b = tid; b < a.nbodies; b += stride) {
            float u[6];
            load_rec(a.ucp + 8 * (int64_t)b, u);
#pragma unroll
            for (int k = 0; k < 6; ++k) a.ucd[k][b] = __ldcg(a.ucd[k] + b) + (double)u[k];
        }
        if (conv) return true;
    }
    return true;
}

template <class R>
__global__ void __launch_bounds__(kThreads) lcp_kernel(KArgs<R> a) {
    __shared__ double part[kNred];
    const int nrows = *a.nrows_dev;
    unsigned epoch = 0;  // used by thread 0 only
    R v[3];
    double res_t;
    unsigned long long tot[kNred];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    // warm start into the packed buffer
    for (int r = tid; r < nrows; r += stride) a.gg[0][r].x = a.gamma_io[r];
    BodySlot<R> bs;
    RowSlot<R> rs;
    load_body_slot(a, tid / kLanesPerBody, threadIdx.x & (kLanesPerBody - 1), bs);
    load_row_slot(a, tid, nrows, rs);
    // fault injection: a block that never arrives; every other block's wait
    // at the barrier below runs out (wait_ns) and the launch reports DEV_TIMEOUT
    if (a.skip_block && blockIdx.x == gridDim.x - 1) return;
    if (!grid_barrier(a.bar, &epoch, a.status, a.wait_ns)) return;
    // ---- init: Uc = K D gamma0, g0, residual, max diagonal
    scatter_phase(a, bs, 0, false, R(0));
    if (!grid_barrier(a.bar, &epoch, a.status, a.wait_ns)) return;
    gather_phase(a, rs, nrows, 0, -1, true, R(0), v, &res_t);
    // one grid barrier per iteration (mixed path): every row has its own
    // thread, whose records start as the phase-0 record of the initial
    // iterate (buffer 0) and a phase-1 placeholder (buffer 1, which iteration
    // 1 writes with phase 0)
    const bool one_bar = sizeof(R) == sizeof(float) && a.ucp2 != nullptr && nrows <= stride;
    if constexpr (sizeof(R) == sizeof(float)) {
        if (one_bar && rs.r >= 0) {
            rs.gm = fabsf(rs.gm);
            st_rel64(reinterpret_cast<unsigned long long*>(a.gg[0]) + rs.r, make_rec(rs.gm, rs.gv, 0u));
            st_rel64(reinterpret_cast<unsigned long long*>(a.gg[1]) + rs.r, make_rec(0.f, 0.f, 1u));
        }
    }
    {
        // init reduces two maxima: slot 0 = largest A_aa, slot 3 = residual
        double md = 0.0;
        for (int r = tid; r < nrows; r += stride) md = fmax(md, a.diag[r]);
        double w[kNred] = {md, 0.0, 0.0, res_t};
        block_reduce_store<double>(w, 0x9u, part);
        if (threadIdx.x == 0) {
            unsigned long long* o = a.partials + (size_t)blockIdx.x * kNred;
            o[0] = to_word(part[0]);
            o[1] = to_word(R(0));
            o[2] = to_word(R(0));
            o[3] = to_word(part[3]);
        }
    }
    if (!grid_barrier(a.bar, &epoch, a.status, a.wait_ns)) return;
    grid_reduce<R>(a.partials, 0x9u, tot);
    // the step length, the residual and the stop decision are computed by
    // thread 0 of each block (identically in every block: same reduced values)
    // and broadcast through shared memory, so FP64 scalar work is not repeated
    // by every thread
    __shared__ double sh_resid;
    __shared__ R sh_alpha_r, sh_alpha0;
    __shared__ int sh_stop;
    double resid = 0.0;
    if (threadIdx.x == 0) {
        resid = from_word<double>(tot[3]);
        const double md = from_word<double>(tot[0]);
        const double alpha = a.invd ? 1.0 : (md > 0.0 ? 1.0 / md : 1.0);
        sh_alpha_r = (R)alpha;
        sh_alpha0 = (R)alpha;
        sh_resid = resid;
        sh_stop = resid <= a.tol;
    }
    __syncthreads();
    R alpha_r = sh_alpha_r;
    int cur = 0, it = 0;
    // both loops end in one call of refine_solve below (one inlined copy)
    bool to_refine = false, done_1b = false;
    __shared__ unsigned long long pbuf_g[kMaxBlocks * kNred];
    if constexpr (sizeof(R) == sizeof(float)) {
        if (one_bar) {
            // ---- one grid barrier per iteration (see scatter_1b), to tol, or
            // to tol_a and kRefineWait iterations more before the refinement
            int fin = 0;  // the iterate returned
            __shared__ float sh_tol[4];  // tol and tol_a, each rounded down and up to FP32
            constexpr size_t kBuf = (size_t)kMaxBlocks * kNred;
            unsigned long long* pbuf1 = pbuf_g;
            if (threadIdx.x == 0) {
                sh_tol[0] = __double2float_rd(a.tol);
                sh_tol[1] = __double2float_ru(a.tol);
                sh_tol[2] = __double2float_rd(a.tol_a);
                sh_tol[3] = __double2float_ru(a.tol_a);
            }
            __syncthreads();
            resid = sh_resid;
            if (!(resid <= a.tol)) {
#ifdef RELCP_LCP_TRACE
                unsigned long long t_prev = gtimer();
#endif
                __shared__ unsigned sh_rmax;
                fin = -1;
                int it_a = resid <= a.tol_a ? 0 : -1;  // the first iterate at or below tol_a
                const bool refine = a.tol_a > a.tol;    // the FP32 iterations hand over to refine_solve
                // the stall watch, block-uniform in shared memory (no per-thread
                // registers in this loop): thread 0 updates it at check k and
                // writes its verdict to slot (k + 1) & 1, which every thread reads
                // at check k + 1, after the barriers in between
                __shared__ double sh_best;
                __shared__ int sh_itbest, sh_stall[2];
                if (threadIdx.x == 0) {
                    sh_best = 1e300;
                    sh_itbest = 0;
                    sh_stall[0] = sh_stall[1] = 0;
                }
                int ncheck = 0;
                for (it = 1; it <= a.max_iter; ++it) {
                    const bool check = (it % a.check_every) == 0 || it == a.max_iter;
                    const bool prev_check = it >= 2 && ((it - 1) % a.check_every) == 0;
                    unsigned long long* part = a.partials + (size_t)(it & 1) * kBuf;
                    R* uc_it = (it & 1) ? a.ucp2 : a.ucp;
                    scatter_1b(a, bs, reinterpret_cast<const unsigned long long*>(a.gg[(it - 1) & 1]), rec_phase(it - 1),
                               uc_it, alpha_r);
                    TRACE_MARK(0);
                    if (!grid_barrier(a.bar, &epoch, a.status, a.wait_ns)) return;
                    TRACE_MARK(1);
                    // the previous iteration's partials, complete since this
                    // barrier: loaded before the gather, staged after it (the
                    // FP32 sums and the rounded-up residual are low halves)
                    const int npw = (int)gridDim.x * kNred;
                    unsigned pf = 0u;
                    if (it >= 2 && (int)threadIdx.x < npw)
                        pf = __ldcg(reinterpret_cast<const unsigned*>(a.partials + (size_t)((it - 1) & 1) * kBuf +
                                                                      threadIdx.x));
                    unsigned rbits;
                    gather_1b(a, rs, uc_it, reinterpret_cast<unsigned long long*>(a.gg[it & 1]), rec_phase(it), check,
                              alpha_r, sh_tol, v, &rbits);
                    TRACE_MARK(2);
                    if (it >= 2) {
                        if ((int)threadIdx.x < npw) pbuf1[threadIdx.x] = pf;
                        for (int t = threadIdx.x + kThreads; t < npw; t += kThreads)
                            pbuf1[t] = (unsigned)__ldcg(a.partials + (size_t)((it - 1) & 1) * kBuf + t);
                    }
                    block_partials<R>(v, check ? (unsigned long long)rbits : 0ull, part + (size_t)blockIdx.x * kNred,
                                      it >= 2 ? pbuf1 : nullptr, it, &sh_alpha_r, prev_check, &sh_rmax);
                    __syncthreads();
                    alpha_r = sh_alpha_r;
                    TRACE_MARK(3);
#ifdef RELCP_LCP_TRACE
                    if (blockIdx.x == 0 && threadIdx.x == 0) g_lcp_trace[6] += 1;
#endif
                    if (prev_check) {
                        // every block folds the same words: the same decision.
                        // Below tol_a the iterations go on towards tol for up to
                        // kRefineWait more; only a solve still above tol then is
                        // refined (a light solve usually gets there first, and
                        // the refinement's FP64 pass would cost it more).  A
                        // stall hands over at once.
                        const double rsd = (double)__uint_as_float(sh_rmax);
                        if (rsd <= a.tol_a && it_a < 0) it_a = it - 1;
                        const bool stall = refine && sh_stall[ncheck & 1];
                        if (threadIdx.x == 0) {
                            if (rsd < 0.9 * sh_best) {
                                sh_best = rsd;
                                sh_itbest = it - 1;
                            }
                            sh_stall[(ncheck + 1) & 1] = it - 1 - sh_itbest > kStallIters;
                        }
                        ++ncheck;
                        if (rsd <= a.tol || (refine && it_a >= 0 && it - 1 >= it_a + kRefineWait) || stall) {
                            resid = rsd;
                            fin = it - 1;
                            break;
                        }
                    }
                }
                if (fin < 0) {
                    // the cap: the last iterate's residual, after every block's partials
                    it = a.max_iter;
                    fin = it;
                    if (!grid_barrier(a.bar, &epoch, a.status, a.wait_ns)) return;
                    const unsigned long long* part = a.partials + (size_t)(it & 1) * kBuf;
                    if (threadIdx.x < 32) {
                        unsigned mm = 0u;
                        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) mm = max(mm, (unsigned)__ldcg(part + b * kNred + 3));
                        for (int o = 16; o > 0; o >>= 1) mm = max(mm, __shfl_down_sync(0xffffffffu, mm, o));
                        if (threadIdx.x == 0) sh_rmax = mm;
                    }
                    __syncthreads();
                    resid = (double)__uint_as_float(sh_rmax);
                }
            }
            // outputs: gamma and the contact velocity of the returned iterate
            // (its record buffer and velocity buffer are intact: iteration
            // fin + 1 wrote the other ones)
            const unsigned long long* rf = reinterpret_cast<const unsigned long long*>(a.gg[fin & 1]);
            for (int r = tid; r < nrows; r += stride) a.gamma_io[r] = fabsf(__uint_as_float((unsigned)ld_rel64(rf + r)));
            const R* uf = (fin & 1) ? a.ucp2 : a.ucp;
            for (int b = tid; b < a.nbodies; b += stride) {
                R u[6];
                load_rec(uf + 8 * (int64_t)b, u);
#pragma unroll
                for (int k = 0; k < 6; ++k) a.ucd[k][b] = (double)u[k];
            }
            done_1b = true;
        }
    }
    if (!done_1b) {
    if (!sh_stop) {
#ifdef RELCP_LCP_TRACE
        unsigned long long t_prev = gtimer();
#endif
        constexpr bool kRetard = sizeof(R) == sizeof(float);
        constexpr size_t kBuf = (size_t)kMaxBlocks * kNred;
        unsigned long long* pbuf = pbuf_g;
        // mixed path: hand over to refine_solve below tol_a (after kRefineWait
        // more iterations) or on a stall, as the one-barrier loop does
        const bool refine = kRetard && a.tol_a > a.tol;
        int it_a = sh_resid <= a.tol_a ? 0 : -1;
        StallWatch sw;
        for (it = 1; it <= a.max_iter; ++it) {
            // all blocks have read partials before any block rewrites them:
            // the barrier after phase 1 separates the reads from the writes
            const bool check = (it % a.check_every) == 0 || it == a.max_iter;
            unsigned long long* part = a.partials + (kRetard ? (size_t)(it & 1) * kBuf : 0);
            scatter_phase(a, bs, cur, true, alpha_r);
            TRACE_MARK(0);
            if (!grid_barrier(a.bar, &epoch, a.status, a.wait_ns)) return;
            TRACE_MARK(1);
            // the previous iteration's partials (complete since its second
            // barrier) are loaded before this iteration gathers and stored to
            // shared memory after it, so the two sets of loads overlap
            // (the FP32 sums are the low halves of their words)
            const int npw = (int)gridDim.x * kNred;
            unsigned pf = 0u;
            if (kRetard && it >= 2 && (int)threadIdx.x < npw)
                pf = __ldcg(reinterpret_cast<const unsigned*>(a.partials + (size_t)((it - 1) & 1) * kBuf +
                                                              threadIdx.x));
            gather_phase(a, rs, nrows, 1 - cur, cur, check, alpha_r, v, &res_t);
            TRACE_MARK(2);
            if (kRetard && it >= 2) {
                if ((int)threadIdx.x < npw) pbuf[threadIdx.x] = pf;
                // (only a grid of more than kThreads / kNred blocks has words left)
                for (int t = threadIdx.x + kThreads; t < npw; t += kThreads)
                    pbuf[t] = __ldcg(a.partials + (size_t)((it - 1) & 1) * kBuf + t);
            }
            block_partials<R>(v, check ? (unsigned long long)__double_as_longlong(res_t) : 0ull,
                              part + (size_t)blockIdx.x * kNred, (kRetard && it >= 2) ? pbuf : nullptr, it,
                              &sh_alpha_r);
            TRACE_MARK(3);
            if (!grid_barrier(a.bar, &epoch, a.status, a.wait_ns)) return;
            TRACE_MARK(4);
            cur = 1 - cur;
            if (!kRetard || check) {
                grid_reduce<R>(part, 0x8u, tot);
                if (threadIdx.x == 0) {
                    int stop = 0;
                    if (check) {
                        const double rs = from_word<double>(tot[3]);
                        sh_resid = rs;
                        stop = rs <= a.tol;
                    }
                    if (!kRetard)
                        sh_alpha_r = bb_step<R>(it, from_word<R>(tot[0]), from_word<R>(tot[1]),
                                                from_word<R>(tot[2]), sh_alpha_r);
                    sh_stop = stop;
                }
                __syncthreads();
            }
            alpha_r = sh_alpha_r;
            TRACE_MARK(5);
#ifdef RELCP_LCP_TRACE
            if (blockIdx.x == 0 && threadIdx.x == 0) g_lcp_trace[6] += 1;
#endif
            if (sh_stop) break;
            if (refine && check) {
                const double rsd = sh_resid;
                if (rsd <= a.tol_a && it_a < 0) it_a = it;
                if ((it_a >= 0 && it >= it_a + kRefineWait) || sw.stalled(rsd, it, kStallIters)) {
                    to_refine = true;
                    break;
                }
            }
        }
        if (it > a.max_iter) it = a.max_iter;
    }
    resid = sh_resid;
    // outputs: gamma of the last iterate (buffer cur) and the contact velocity
    // in double; every write of the last iteration happened before the last
    // grid barrier
    for (int r = tid; r < nrows; r += stride) a.gamma_io[r] = ldcg(&a.gg[cur][r].x);
    for (int b = tid; b < a.nbodies; b += stride) {
        R u[6];
        load_rec(a.ucp + 8 * (int64_t)b, u);
#pragma unroll
        for (int k = 0; k < 6; ++k) a.ucd[k][b] = (double)u[k];
    }
    }
    if constexpr (sizeof(R) == sizeof(float)) {
        // ---- iterative refinement of either loop's result (see refine_solve);
        // a solve that reached max_iter above tol hands over too
        if ((to_refine || (a.tol_a > a.tol && !(resid <= a.tol))) &&
            !refine_solve(a, bs, rs, nrows, &epoch, sh_alpha0, pbuf_g, resid, it))
            return;
    }
    pdl_trigger();  // the next kernel in the stream may start launching
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.result->iterations = (double)it;
        a.result->residual = resid;
        if (!(resid <= a.tol)) atomicOr(a.status, DEV_LCP_NOT_CONVERGED);
    }
}

// ---- incidence CSR (rows ascending within each body)
__global__ void inc_count(const int* __restrict__ nrows_dev, const int* __restrict__ ia, const int* __restrict__ ib,
                          int* __restrict__ cnt) {
    pdl_wait();
    pdl_trigger();
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= *nrows_dev) return;
    atomicAdd(&cnt[ia[r]], 1);
    atomicAdd(&cnt[ib[r]], 1);
}

__global__ void inc_fill(const int* __restrict__ nrows_dev, const int* __restrict__ ia, const int* __restrict__ ib,
                         const int* __restrict__ off, int* __restrict__ cursor, int* __restrict__ inc) {
    pdl_wait();
    pdl_trigger();
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= *nrows_dev) return;
    int a = ia[r], b = ib[r];
    inc[off[a] + atomicAdd(&cursor[a], 1)] = (int)(r << 1);
    inc[off[b] + atomicAdd(&cursor[b], 1)] = (int)(r << 1) | 1;
}

// deterministic order inside each body's segment: incidence codes sorted
// ascending (row order), each placed at its rank among its body's codes
// (the atomic fill above leaves the order of a segment to the scheduler)
__global__ void inc_rank(const int* __restrict__ nrows_dev, const int* __restrict__ ia, const int* __restrict__ ib,
                         const int* __restrict__ off, const int* __restrict__ unsorted, int* __restrict__ inc) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * (int64_t)*nrows_dev) return;
    const int v = unsorted[e];
    const int r = v >> 1;
    const int b = (v & 1) ? ib[r] : ia[r];
    const int e0 = off[b], e1 = off[b + 1];
    int rank = 0;
    for (int k = e0; k < e1; ++k) rank += unsorted[k] < v;
    inc[e0 + rank] = v;
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

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <class R>
relcp_status launch_lcp(KArgs<R>& ka, int64_t work, LcpScratch& sc, cudaStream_t s, int* blocks_out,
                        cudaEvent_t ev0, cudaEvent_t ev1) {
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
    // one CTA per SM: fewest arrivals per grid barrier
    int64_t maxb = (int64_t)sms * (per_sm < kMaxCtasPerSm ? per_sm : kMaxCtasPerSm);
    if (maxb > kMaxBlocks) maxb = kMaxBlocks;  // the grid reduction stages kMaxBlocks blocks' partials
    int blocks = (int)(want < 1 ? 1 : (want > maxb ? maxb : want));
    RELCP_TRY(sc.partials.ensure((size_t)2 * kMaxBlocks * kNred, s));
    ka.partials = reinterpret_cast<unsigned long long*>(sc.partials.p);
    void* args[] = {&ka};
    if (ev0) RELCP_CUDA(cudaEventRecord(ev0, s));
    note_launch();
    RELCP_CUDA(cudaLaunchCooperativeKernel((void*)lcp_kernel<R>, dim3(blocks), dim3(kThreads), args, 0, s));
    if (ev1) RELCP_CUDA(cudaEventRecord(ev1, s));
    *blocks_out = blocks;
    return RELCP_OK;
}

template <class R>
relcp_status solve_typed(const LcpProblem& pr, LcpScratch& sc, DBuf<R>& pack, int* blocks, float* kernel_ms,
                         cudaStream_t s) {
    using V2 = typename Vec2<R>::T;
    const int64_t mc = pr.m_cap > 0 ? pr.m_cap : 1, nb = pr.nbodies, nba = nb > 0 ? nb : 1;
    // (gamma, g) pairs for both buffers, then the 8-wide contact-velocity records
    const size_t pair_elems = (size_t)(2 * mc) * 2;
    // mixed path: a second contact-velocity buffer for the one-barrier iterations
    const bool two_uc = sizeof(R) == sizeof(float);
    RELCP_TRY(pack.ensure(pair_elems + (size_t)((two_uc ? 16 : 8) * nba), s));
    KArgs<R> ka{};
    ka.nrows_dev = pr.nrows_dev;
    ka.nbodies = (int)nb;
    ka.ia = pr.ia;
    ka.ib = pr.ib;
    for (int k = 0; k < 9; ++k) ka.geom[k] = (const R*)pr.geom[k];
    ka.q = pr.q;
    ka.qr = (const R*)pr.qr;
    ka.diag = pr.diag;
    for (int k = 0; k < 7; ++k) ka.K[k] = (const R*)pr.Kr[k];
    ka.invd = (const R*)pr.invd;
    ka.inc_off = sc.inc_off.p;
    ka.inc = sc.inc.p;
    ka.gamma_io = (R*)pr.gamma;
    ka.gg[0] = reinterpret_cast<V2*>(pack.p);
    ka.gg[1] = reinterpret_cast<V2*>(pack.p) + mc;
    ka.ucp = pack.p + pair_elems;
    ka.ucp2 = two_uc ? pack.p + pair_elems + (size_t)(8 * nba) : nullptr;
    for (int k = 0; k < 6; ++k) ka.ucd[k] = pr.uc[k];
    ka.c = pr.c;
    ka.tol = pr.tol;
    ka.max_iter = pr.max_iter;
    ka.check_every = sizeof(R) == sizeof(double) ? 1 : kMixedCheckEvery;
    ka.bar = reinterpret_cast<unsigned*>(sc.inc_count.p + 2 * (nb > 0 ? nb : 1));  // zeroed with the counts
    ka.status = pr.status;
    ka.result = pr.result;
    ka.wait_ns = pr.wait_ns ? pr.wait_ns : kLcpWaitNs;
    ka.skip_block = pr.fault_skip_block;
    ka.tol_a = pr.tol;
    if (sizeof(R) == sizeof(float) && pr.refine) {
        RELCP_TRY(sc.g64.ensure((size_t)mc, s));
        ka.tol_a = kRefineFactor * pr.tol;
        ka.g64 = sc.g64.p;
        for (int k = 0; k < 7; ++k) ka.K64[k] = pr.K[k];
    }
    int64_t work = pr.m_cap > kLanesPerBody * nb ? pr.m_cap : kLanesPerBody * nb;
    (void)kernel_ms;
    return launch_lcp(ka, work, sc, s, blocks, pr.ev_before, pr.ev_after);
}

}  // namespace

int lcp_threads() { return kThreads; }

relcp_status lcp_diag_launch(int64_t nrows, const int32_t* ia, const int32_t* ib, View<9, const double> geom,
                             View<7, const double> K, double c, double* diag, cudaStream_t s) {
    if (nrows == 0) return RELCP_OK;
    note_launch();
    diag_kernel<<<nblk(nrows), 256, 0, s>>>(nrows, ia, ib, geom, K, c, diag);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

// Every buffer lcp_solve uses for up to m_cap rows and nb bodies, so that a
// later solve of that size allocates nothing.
relcp_status lcp_reserve(LcpScratch& sc, int64_t m_cap, int64_t nb, bool mixed, cudaStream_t s) {
    const int64_t mc = m_cap > 0 ? m_cap : 1, nba = nb > 0 ? nb : 1;
    RELCP_TRY(sc.inc_count.ensure((size_t)(2 * nba + 2), s));
    RELCP_TRY(sc.inc_off.ensure((size_t)nba + 1, s));
    RELCP_TRY(sc.inc_tmp.ensure((size_t)(2 * mc), s));
    RELCP_TRY(sc.inc.ensure((size_t)(2 * mc), s));
    const size_t pack = (size_t)(2 * mc) * 2 + (size_t)((mixed ? 16 : 8) * nba);
    if (mixed) {
        RELCP_TRY(sc.packf.ensure(pack, s));
        RELCP_TRY(sc.g64.ensure((size_t)mc, s));
    } else {
        RELCP_TRY(sc.packd.ensure(pack, s));
    }
    RELCP_TRY(sc.partials.ensure((size_t)2 * kMaxBlocks * kNred, s));
    RELCP_TRY(scan_reserve(sc.scan, nba, s));
    return RELCP_OK;
}

// Incidence CSR of the current rows (device row count), then the persistent
// solve.  Nothing here synchronises the stream.
relcp_status lcp_build_csr(const LcpProblem& pr, LcpScratch& sc, cudaStream_t s) {
    const int64_t mc = pr.m_cap > 0 ? pr.m_cap : 1, nb = pr.nbodies;
    if (pr.m_cap > (int64_t)1 << 29 || nb > (int64_t)1 << 30) return RELCP_ERR_INVALID_ARG;
    const int64_t nba = nb > 0 ? nb : 1;
    // one zeroed block: counts [0, nb), fill cursors [nb, 2 nb), barrier counters [2 nb, 2 nb + 2)
    RELCP_TRY(sc.inc_count.ensure((size_t)(2 * nba + 2), s));
    RELCP_TRY(sc.inc_off.ensure((size_t)nba + 1, s));
    RELCP_TRY(sc.inc_tmp.ensure((size_t)(2 * mc), s));
    RELCP_TRY(sc.inc.ensure((size_t)(2 * mc), s));
    int* cnt = sc.inc_count.p;
    int* cursor = cnt + nba;
    RELCP_CUDA(cudaMemsetAsync(cnt, 0, (2 * nba + 2) * sizeof(int), s));
    note_launch();
    launch_pdl(inc_count, dim3(nblk(mc)), dim3(256), 0, s, pr.nrows_dev, pr.ia, pr.ib, cnt);
    RELCP_CUDA(cudaGetLastError());
    RELCP_TRY(exclusive_scan(cnt, sc.inc_off.p, nb, sc.scan, s));
    note_launch();
    launch_pdl(inc_fill, dim3(nblk(mc)), dim3(256), 0, s, pr.nrows_dev, pr.ia, pr.ib, sc.inc_off.p, cursor,
               sc.inc_tmp.p);
    RELCP_CUDA(cudaGetLastError());
    note_launch();
    launch_pdl(inc_rank, dim3(nblk(2 * mc)), dim3(256), 0, s, pr.nrows_dev, pr.ia, pr.ib, sc.inc_off.p, sc.inc_tmp.p,
               sc.inc.p);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status lcp_run(const LcpProblem& pr, LcpScratch& sc, int* blocks, cudaStream_t s) {
    *blocks = 0;
    float kernel_ms = 0.f;
    if (pr.mixed) return solve_typed<float>(pr, sc, sc.packf, blocks, &kernel_ms, s);
    return solve_typed<double>(pr, sc, sc.packd, blocks, &kernel_ms, s);
}

relcp_status lcp_solve(const LcpProblem& pr, LcpScratch& sc, int* blocks, float* kernel_ms, cudaStream_t s) {
    *kernel_ms = 0.f;
    RELCP_TRY(lcp_build_csr(pr, sc, s));
    return lcp_run(pr, sc, blocks, s);
}

void release(LcpScratch& sc, cudaStream_t s) {
    sc.inc_count.release(s);
    sc.inc_off.release(s);
    sc.inc_tmp.release(s);
    sc.inc.release(s);
    sc.packd.release(s);
    sc.packf.release(s);
    sc.g64.release(s);
    sc.partials.release(s);
    release(sc.scan, s);
}

}  // namespace relcp

#ifdef RELCP_LCP_TRACE
extern "C" int relcp_debug_lcp_trace(unsigned long long* out, int reset) {
    if (cudaMemcpyFromSymbol(out, relcp::g_lcp_trace, 8 * sizeof(unsigned long long)) != cudaSuccess) return 1;
    if (reset) {
        unsigned long long z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (cudaMemcpyToSymbol(relcp::g_lcp_trace, z, sizeof(z)) != cudaSuccess) return 1;
    }
    return 0;
}
#endif
