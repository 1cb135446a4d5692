// Learned SNSD initial guess (the learned part of the method's Newton start;
// Newton on the sphere decides every result).
//
// Network: features (16, 13 used) -> 128 -> 128 -> 128 -> outputs (8, 5 used),
// ReLU, BF16 operands on the tensor cores, FP32 accumulation: inference with
// mma.sync.m16n8k16 fragments chained through registers, training GEMMs with
// tcgen05.mma into tensor memory (the 8-wide output layer with mma.sync).
//   features : d = c_b - c_a (minimum image) in a's frame divided by
//              s = max(a_a) + max(a_b); q_rel = conj(q_a) (x) q_b with s >= 0;
//              a's and b's semi-axes; the analytic seed (P_a + P_b)^-1 d,
//              normalised, in a's frame.
//   outputs  : the correction from the seed to the shared normal (in a's
//              frame, scaled by RELCP_MLP_CORR_SCALE), Phi / s, and a trust
//              logit (positive: the corrected seed is the Newton start; else
//              the cold start is used).
// Inference: the four weight matrices live in shared memory (BF16, row =
// output unit, packed once per parameter set and bulk-copied in per CTA), each
// warp carries 16 pairs through all four layers in registers -- the FP32
// accumulator fragment of one layer is exactly the A-operand fragment of the
// next (same rows, same columns per thread), so activations never leave the
// registers.  Inside a step one kernel does the whole start for a list of
// pairs (features, network, rotated normal); relcp_mlp_forward runs the
// network alone on given features.
// Training is layer by layer with a tensor-core GEMM C = A B^T (both operands
// K-contiguous BF16), transposes, the loss, bias sums and Adam (Kingma & Ba)
// on FP32 master parameters.
#include <cuda_bf16.h>

#include <vector>

#include "mlp.cuh"

namespace relcp {

namespace {

// ---------------------------------------------------------------------------
// tensor-core primitives
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// D = A B + D with A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate.
// Fragment ownership (g = lane / 4, t = lane % 4):
//   a0: A[g][2t..2t+1]   a1: A[g+8][2t..2t+1]   a2: A[g][2t+8..]   a3: A[g+8][2t+8..]
//   b0: B[2t..2t+1][g]   b1: B[2t+8..2t+9][g]
//   c0,c1: C[g][2t..2t+1]   c2,c3: C[g+8][2t..2t+1]
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
// T = double when training targets are written (the targets resolve the SNSD
// normal to FP64 accuracy); T = float for inference, whose outputs are FP32
// features (FP64 runs at a small fraction of the FP32 rate on this part).  The
// minimum image of the centres is always taken in FP64 (exact, like the SNSD).
template <class T>
__device__ void compute_features(const MlpFeatArgs& a, int64_t row, int64_t p, float* f, float* targ) {
    const int i = a.pa[p * a.pstride], j = a.pb[p * a.pstride];
    T d[3];
    for (int k = 0; k < 3; ++k) d[k] = (T)min_image(a.x(k, j) - a.x(k, i), a.box_dev ? a.box_dev[k] : a.box[k]);
    T qa[4], qb[4];
    T la = 0, lb = 0;
    for (int k = 0; k < 4; ++k) {
        qa[k] = (T)a.q(k, i);
        qb[k] = (T)a.q(k, j);
        la += qa[k] * qa[k];
        lb += qb[k] * qb[k];
    }
    la = sqrt(la);
    lb = sqrt(lb);
    for (int k = 0; k < 4; ++k) {
        qa[k] /= la;
        qb[k] /= lb;
    }
    T R[9];
    quat_to_R(qa[0], qa[1], qa[2], qa[3], R);
    const T aa[3] = {(T)a.axes(0, i), (T)a.axes(1, i), (T)a.axes(2, i)};
    const T ab[3] = {(T)a.axes(0, j), (T)a.axes(1, j), (T)a.axes(2, j)};
    const T sc = fmax(aa[0], fmax(aa[1], aa[2])) + fmax(ab[0], fmax(ab[1], ab[2]));
    for (int k = 0; k < 3; ++k) f[k] = (float)((R[k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2]) / sc);
    // q_rel = conj(q_a) (x) q_b
    const T s1 = qa[0], x1 = -qa[1], y1 = -qa[2], z1 = -qa[3];
    const T s2 = qb[0], x2 = qb[1], y2 = qb[2], z2 = qb[3];
    T qr[4] = {s1 * s2 - (x1 * x2 + y1 * y2 + z1 * z2), s1 * x2 + s2 * x1 + (y1 * z2 - z1 * y2),
               s1 * y2 + s2 * y1 + (z1 * x2 - x1 * z2), s1 * z2 + s2 * z1 + (x1 * y2 - y1 * x2)};
    const T sg = qr[0] < T(0) ? T(-1) : T(1);
    for (int k = 0; k < 4; ++k) f[3 + k] = (float)(sg * qr[k]);
    for (int k = 0; k < 3; ++k) {
        f[7 + k] = (float)aa[k];
        f[10 + k] = (float)ab[k];
    }
    // analytic seed (P_a + P_b)^-1 d (world), normalised, in a's frame: the
    // network predicts the correction from this seed to the shared normal
    T sd[3];
    {
        T Rb[9];
        quat_to_R(qb[0], qb[1], qb[2], qb[3], Rb);
        Sym3<T> Pa = rot_diag_rot(R, aa[0] * aa[0], aa[1] * aa[1], aa[2] * aa[2]);
        Sym3<T> Pb = rot_diag_rot(Rb, ab[0] * ab[0], ab[1] * ab[1], ab[2] * ab[2]);
        const T xx = Pa.xx + Pb.xx, yy = Pa.yy + Pb.yy, zz = Pa.zz + Pb.zz;
        const T xy = Pa.xy + Pb.xy, xz = Pa.xz + Pb.xz, yz = Pa.yz + Pb.yz;
        // adjugate of the symmetric sum times d (same direction as the inverse)
        const T A00 = yy * zz - yz * yz, A11 = xx * zz - xz * xz, A22 = xx * yy - xy * xy;
        const T A01 = xz * yz - xy * zz, A02 = xy * yz - yy * xz, A12 = xy * xz - xx * yz;
        T w[3] = {A00 * d[0] + A01 * d[1] + A02 * d[2], A01 * d[0] + A11 * d[1] + A12 * d[2],
                  A02 * d[0] + A12 * d[1] + A22 * d[2]};
        T lw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (!(lw > T(0))) {
            w[0] = 1;
            w[1] = w[2] = 0;
            lw = 1;
        }
        for (int k = 0; k < 3; ++k) sd[k] = (R[k] * w[0] + R[3 + k] * w[1] + R[6 + k] * w[2]) / lw;
    }
    for (int k = 0; k < 3; ++k) f[13 + k] = (float)sd[k];
    if (targ && a.snsd) {
        const double* o = a.snsd + p * a.snsd_s;
        const T n[3] = {(T)o[1 * a.snsd_c], (T)o[2 * a.snsd_c], (T)o[3 * a.snsd_c]};
        float* t = targ;
        for (int k = 0; k < 3; ++k)
            t[k] = (float)(T(RELCP_MLP_CORR_SCALE) * ((R[k] * n[0] + R[3 + k] * n[1] + R[6 + k] * n[2]) - sd[k]));
        t[3] = (float)((T)o[0] / sc);
    }
}

template <class T>
__global__ void features_kernel(MlpFeatArgs a) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (a.count_dev ? (int64_t)*a.count_dev : a.npairs)) return;
    const int64_t p = a.idx ? (int64_t)a.idx[row] : row;
    compute_features<T>(a, row, p, a.feat + 16 * row, a.targets ? a.targets + 4 * row : nullptr);
}

// ---------------------------------------------------------------------------
// fused inference
// ---------------------------------------------------------------------------
constexpr int kFwdWarps = 4;
constexpr int kKs1 = kMlpIn + 8;   // padded row stride (BF16 elements) of W1
constexpr int kKs = kMlpHid + 8;   // padded row stride of W2, W3, W4
constexpr int kSmemW1 = kMlpHid * kKs1;
constexpr int kSmemW = kMlpHid * kKs;
constexpr int kSmemW4 = kMlpOut * kKs;
constexpr size_t kFwdSmem = (size_t)(kSmemW1 + 2 * kSmemW + kSmemW4) * 2 + (3 * kMlpHid + kMlpOut) * 4;

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// The forward kernel's shared-memory image of the network, built once per
// parameter set: BF16 weight rows padded to the strides above, then the FP32
// biases b1 | b2 | b3 | b4.  kFwdSmem is a multiple of 16 bytes (bulk copies).
static_assert(kFwdSmem % 16 == 0, "image size must be a multiple of 16 bytes");
constexpr unsigned kBulkChunk = 16384;
constexpr long long kBulkWaitLimit = 1ll << 22;

__global__ void mlp_pack_kernel(const float* __restrict__ params, unsigned char* __restrict__ image) {
    __nv_bfloat16* W1 = reinterpret_cast<__nv_bfloat16*>(image);
    __nv_bfloat16* W2 = W1 + kSmemW1;
    __nv_bfloat16* W3 = W2 + kSmemW;
    __nv_bfloat16* W4 = W3 + kSmemW;
    float* bias = reinterpret_cast<float*>(W4 + kSmemW4);
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int e = t0; e < kSmemW1; e += stride) {
        const int r = e / kKs1, c = e % kKs1;
        W1[e] = __float2bfloat16_rn(c < kMlpIn ? params[kOffW1 + r * kMlpIn + c] : 0.f);
    }
    for (int e = t0; e < kSmemW; e += stride) {
        const int r = e / kKs, c = e % kKs;
        W2[e] = __float2bfloat16_rn(c < kMlpHid ? params[kOffW2 + r * kMlpHid + c] : 0.f);
        W3[e] = __float2bfloat16_rn(c < kMlpHid ? params[kOffW3 + r * kMlpHid + c] : 0.f);
    }
    for (int e = t0; e < kSmemW4; e += stride) {
        const int r = e / kKs, c = e % kKs;
        W4[e] = __float2bfloat16_rn(c < kMlpHid ? params[kOffW4 + r * kMlpHid + c] : 0.f);
    }
    for (int e = t0; e < kMlpHid; e += stride) {
        bias[e] = params[kOffB1 + e];
        bias[kMlpHid + e] = params[kOffB2 + e];
        bias[2 * kMlpHid + e] = params[kOffB3 + e];
    }
    if (t0 < kMlpOut) bias[3 * kMlpHid + t0] = params[kOffB4 + t0];
}

// Copy `bytes` (multiple of 16) from global memory into this block's shared
// memory with the bulk asynchronous copy engine (cp.async.bulk), completion
// tracked by an mbarrier.  Every thread waits a bounded number of polls; on
// a timeout the block records DEV_TIMEOUT, waits once more (bounded) for its
// copies and returns false.
__device__ bool bulk_copy_to_smem(unsigned char* dst, const unsigned char* src, unsigned bytes,
                                  unsigned long long* mbar, int* status) {
    const unsigned bar = (unsigned)__cvta_generic_to_shared(mbar);
    const unsigned dsts = (unsigned)__cvta_generic_to_shared(dst);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        for (unsigned off = 0; off < bytes; off += kBulkChunk) {
            const unsigned sz = bytes - off < kBulkChunk ? bytes - off : kBulkChunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    dsts + off),
                "l"(src + off), "r"(sz), "r"(bar)
                : "memory");
        }
    }
    __syncthreads();  // the barrier is initialised before anyone polls it
    auto wait = [&]() {
        unsigned done = 0;
        for (long long it = 0; it < kBulkWaitLimit && !done; ++it)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(bar)
                : "memory");
        return done != 0;
    };
    if (wait()) return true;
    if (status) atomicOr(status, DEV_TIMEOUT);
    wait();
    return false;
}

// one hidden layer: acc (16 n-tiles) = A (8 k-tiles) x W^T, then bias + ReLU
// and repack as the next layer's A fragments
__device__ __forceinline__ void hidden_layer(uint32_t A[8][4], const __nv_bfloat16* W, const float* bias, int g, int t) {
    float acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        const __nv_bfloat16* wr = W + (8 * j + g) * kKs + 2 * t;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) mma_bf16(acc[j], A[kk], lds32(wr + 16 * kk), lds32(wr + 16 * kk + 8));
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
        acc[j][0] = fmaxf(acc[j][0] + b0, 0.f);
        acc[j][1] = fmaxf(acc[j][1] + b1, 0.f);
        acc[j][2] = fmaxf(acc[j][2] + b0, 0.f);
        acc[j][3] = fmaxf(acc[j][3] + b1, 0.f);
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        A[kk][0] = pack_bf16(acc[2 * kk][0], acc[2 * kk][1]);
        A[kk][1] = pack_bf16(acc[2 * kk][2], acc[2 * kk][3]);
        A[kk][2] = pack_bf16(acc[2 * kk + 1][0], acc[2 * kk + 1][1]);
        A[kk][3] = pack_bf16(acc[2 * kk + 1][2], acc[2 * kk + 1][3]);
    }
}

// One warp carries 16 rows through the network: rows g and g + 8 of the warp
// (g = lane / 4) come from feature rows f0 and f1 (16 floats each, null: a
// zero row) and their 8 outputs go to o0 and o1 (null: dropped); each thread
// writes outputs 2t and 2t + 1 (t = lane % 4).  `img` is the network image in
// shared memory.
__device__ __forceinline__ void mlp_warp_rows(const unsigned char* img, const float* f0p, const float* f1p, float* o0,
                                              float* o1) {
    const __nv_bfloat16* W1 = reinterpret_cast<const __nv_bfloat16*>(img);
    const __nv_bfloat16* W2 = W1 + kSmemW1;
    const __nv_bfloat16* W3 = W2 + kSmemW;
    const __nv_bfloat16* W4 = W3 + kSmemW;
    const float* bias = reinterpret_cast<const float*>(W4 + kSmemW4);  // b1 | b2 | b3 | b4
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    // layer 1: A = features (16 x 16)
    uint32_t A[8][4];
    {
        float f0[4] = {0, 0, 0, 0}, f1[4] = {0, 0, 0, 0};
        if (f0p) {
            f0[0] = f0p[2 * t];
            f0[1] = f0p[2 * t + 1];
            f0[2] = f0p[2 * t + 8];
            f0[3] = f0p[2 * t + 9];
        }
        if (f1p) {
            f1[0] = f1p[2 * t];
            f1[1] = f1p[2 * t + 1];
            f1[2] = f1p[2 * t + 8];
            f1[3] = f1p[2 * t + 9];
        }
        uint32_t X[4] = {pack_bf16(f0[0], f0[1]), pack_bf16(f1[0], f1[1]), pack_bf16(f0[2], f0[3]),
                         pack_bf16(f1[2], f1[3])};
        float acc[16][4];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
            const __nv_bfloat16* wr = W1 + (8 * j + g) * kKs1 + 2 * t;
            mma_bf16(acc[j], X, lds32(wr), lds32(wr + 8));
            const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
            acc[j][0] = fmaxf(acc[j][0] + b0, 0.f);
            acc[j][1] = fmaxf(acc[j][1] + b1, 0.f);
            acc[j][2] = fmaxf(acc[j][2] + b0, 0.f);
            acc[j][3] = fmaxf(acc[j][3] + b1, 0.f);
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            A[kk][0] = pack_bf16(acc[2 * kk][0], acc[2 * kk][1]);
            A[kk][1] = pack_bf16(acc[2 * kk][2], acc[2 * kk][3]);
            A[kk][2] = pack_bf16(acc[2 * kk + 1][0], acc[2 * kk + 1][1]);
            A[kk][3] = pack_bf16(acc[2 * kk + 1][2], acc[2 * kk + 1][3]);
        }
    }
    hidden_layer(A, W2, bias + kMlpHid, g, t);
    hidden_layer(A, W3, bias + 2 * kMlpHid, g, t);
    // layer 4: 8 outputs
    float o[4] = {0, 0, 0, 0};
    const __nv_bfloat16* wr = W4 + g * kKs + 2 * t;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) mma_bf16(o, A[kk], lds32(wr + 16 * kk), lds32(wr + 16 * kk + 8));
    const float b0 = bias[3 * kMlpHid + 2 * t], b1 = bias[3 * kMlpHid + 2 * t + 1];
    if (o0) {
        o0[2 * t] = o[0] + b0;
        o0[2 * t + 1] = o[1] + b1;
    }
    if (o1) {
        o1[2 * t] = o[2] + b0;
        o1[2 * t + 1] = o[3] + b1;
    }
}

__global__ void __launch_bounds__(kFwdWarps * 32) mlp_forward_kernel(int64_t nmax, const unsigned char* __restrict__ image,
                                                                     const float* __restrict__ feat,
                                                                     float* __restrict__ out,
                                                                     const int* __restrict__ count_dev,
                                                                     int* __restrict__ status) {
    const int64_t npairs = count_dev ? (int64_t)*count_dev : nmax;
    if ((int64_t)blockIdx.x * 16 * kFwdWarps >= npairs) return;  // no tile for this block
    extern __shared__ __align__(16) unsigned char smem[];
    // the packed network (weights and biases) in one bulk copy; the mbarrier
    // sits right after it
    if (!bulk_copy_to_smem(smem, image, (unsigned)kFwdSmem, reinterpret_cast<unsigned long long*>(smem + kFwdSmem),
                           status))
        return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (npairs + 16 * kFwdWarps - 1) / (16 * kFwdWarps);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * 16 * kFwdWarps + 16 * warp + (lane >> 2), r1 = r0 + 8;
        mlp_warp_rows(smem, r0 < npairs ? feat + 16 * r0 : nullptr, r1 < npairs ? feat + 16 * r1 : nullptr,
                      r0 < npairs ? out + 8 * r0 : nullptr, r1 < npairs ? out + 8 * r1 : nullptr);
    }
}

// network output -> world-frame start normal (zero when the trust logit is
// negative: the Newton solve then starts cold).  FP32: it only seeds the FP32
// Newton iterations.
__device__ __forceinline__ void guess_from(const float* f, const float* o, float s, float x, float y, float z,
                                           double g[3]) {
    const float inv = 1.f / (float)RELCP_MLP_CORR_SCALE;
    const float n[3] = {f[13] + inv * o[0], f[14] + inv * o[1], f[15] + inv * o[2]};
    const float l = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(o[4] > 0.f) || !(l > 1e-6f)) {
        g[0] = g[1] = g[2] = 0.0;
        return;
    }
    const float lq = sqrtf(s * s + x * x + y * y + z * z);
    float R[9];
    quat_to_R(s / lq, x / lq, y / lq, z / lq, R);
    for (int k = 0; k < 3; ++k) g[k] = (double)((R[3 * k] * n[0] + R[3 * k + 1] * n[1] + R[3 * k + 2] * n[2]) / l);
}

__device__ __forceinline__ bool g_zero(const View<3, double>& guess, int64_t k, int64_t pair) {
    return pair >= 0 && guess(0, k) == 0.0 && guess(1, k) == 0.0 && guess(2, k) == 0.0;
}

// The learned start in one kernel for a list of pairs: per tile of 64 pairs,
// FP32 features into shared memory, the BF16 network on the tensor cores (one
// warp per 16 pairs, weights bulk-copied into shared memory once per CTA),
// the outputs back into shared memory, then the rotated start normals.
constexpr int kGuessTile = 16 * kFwdWarps;
constexpr size_t kGuessSmem = kFwdSmem + 16 + (size_t)kGuessTile * (16 + 8) * sizeof(float);

__global__ void __launch_bounds__(kFwdWarps * 32) mlp_guess_kernel(MlpFeatArgs fa, const unsigned char* __restrict__ image,
                                                                   View<3, double> guess, int* __restrict__ status,
                                                                   int64_t min_count, int* __restrict__ ran,
                                                                   int* __restrict__ declined) {
    pdl_wait();
    pdl_trigger();
    const int64_t count = fa.count_dev ? (int64_t)*fa.count_dev : fa.npairs;
    const bool run = count >= min_count;
    if (ran && blockIdx.x == 0 && threadIdx.x == 0) *ran = run ? 1 : 0;
    if (!run || (int64_t)blockIdx.x * kGuessTile >= count) return;  // no tile for this block
    extern __shared__ __align__(16) unsigned char smem[];
    if (!bulk_copy_to_smem(smem, image, (unsigned)kFwdSmem, reinterpret_cast<unsigned long long*>(smem + kFwdSmem),
                           status))
        return;
    float* feat = reinterpret_cast<float*>(smem + kFwdSmem + 16);  // kGuessTile x 16
    float* outs = feat + kGuessTile * 16;                          // kGuessTile x 8
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (count + kGuessTile - 1) / kGuessTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t row0 = tile * kGuessTile;
        const int r = threadIdx.x;  // one pair per thread (kGuessTile <= blockDim.x)
        int64_t pair = -1;
        if (r < kGuessTile && row0 + r < count) {
            pair = fa.idx ? (int64_t)fa.idx[row0 + r] : row0 + r;
            compute_features<float>(fa, row0 + r, pair, feat + 16 * r, nullptr);
        }
        __syncthreads();
        const int rr = 16 * warp + (lane >> 2);
        mlp_warp_rows(smem, row0 + rr < count ? feat + 16 * rr : nullptr,
                      row0 + rr + 8 < count ? feat + 16 * (rr + 8) : nullptr,
                      row0 + rr < count ? outs + 8 * rr : nullptr, row0 + rr + 8 < count ? outs + 8 * (rr + 8) : nullptr);
        __syncthreads();
        if (pair >= 0) {
            const int i = fa.pa[pair * fa.pstride];
            double g[3];
            guess_from(feat + 16 * r, outs + 8 * r, (float)fa.q(0, i), (float)fa.q(1, i), (float)fa.q(2, i),
                       (float)fa.q(3, i), g);
            for (int k = 0; k < 3; ++k) guess(k, row0 + r) = g[k];
        }
        // pairs the network declined (zero start: Newton starts cold)
        const unsigned dm = __ballot_sync(0xffffffffu, pair >= 0 && g_zero(guess, row0 + r, pair));
        if (declined && lane == 0 && dm) atomicAdd(declined, __popc(dm));
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// training GEMM on the fifth-generation tensor cores (tcgen05):
//     C[M x N] (+)= A[M x K] B[N x K]^T,  BF16 operands, FP32 accumulation
// in tensor memory, for N a multiple of 16 in [16, 128] and K a multiple of
// 16 (the hidden and input layers of the network; the 8-wide output layer
// takes gemm_nt_kernel below).  One CTA of 128 threads per 128-row tile of C:
// the threads stage 64-wide K chunks of A and B into shared memory in the
// no-swizzle K-major core-matrix layout, one thread issues the chunk's
// 128 x N x 16 MMAs (tcgen05.mma.cta_group::1.kind::f16) into a 128-lane x
// 128-column FP32 accumulator in tensor memory and commits them to an
// mbarrier, and after the last chunk each warp reads its 32 lanes back
// (tcgen05.ld.32x32b).  Every wait is bounded: a timeout records DEV_TIMEOUT,
// waits once more (bounded) for the MMAs in flight, frees the tensor memory
// and skips the store.
// ---------------------------------------------------------------------------
constexpr int kTcM = 128;              // rows of a tile (the MMA's M)
constexpr int kTcK = 64;               // K staged per chunk
constexpr int kTcMaxN = 128;           // widest N handled (one tile, 128 TMEM columns)
constexpr int kTcThreads = 128;
constexpr unsigned kTcCols = 128;      // TMEM columns allocated per CTA
// 4 CTAs per SM at most (4 x 128 = all 512 TMEM columns): the dynamic shared
// memory request keeps a fifth CTA off the SM, so no allocation ever waits
constexpr size_t kTcSmem = 56 * 1024;
constexpr long long kTcWaitLimit = 1ll << 20;

// byte offset of element (r, k) in a [rows x kTcK] K-major chunk: core
// matrices of 8 rows x 16 bytes (8 BF16 along K), consecutive along K 128 bytes
// apart (the descriptor's leading-dimension byte offset), 8-row groups
// kTcK / 8 x 128 = 1024 bytes apart (its stride-dimension byte offset)
__device__ __forceinline__ uint32_t tc_core_off(int r, int k) {
    return (uint32_t)((((r >> 3) * (kTcK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), the fixed value
// 0b001 in bits 46-48, base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, unsigned parity) {
    unsigned done = 0;
    for (long long it = 0; it < kTcWaitLimit && !done; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
    }
    return done != 0;
}

__global__ void __launch_bounds__(kTcThreads) gemm_nt_tc_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                                int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                                                                float* __restrict__ C, int ldc, int accumulate,
                                                                int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sA = tc_smem;                    // kTcM x kTcK BF16 (16 KB)
    unsigned char* sB = tc_smem + kTcM * kTcK * 2;  // kTcMaxN x kTcK BF16 (16 KB)
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int m0 = blockIdx.x * kTcM;
    // split K: CTA y takes the K range [kbeg, kend) and adds its partial
    // product to C with atomics (the caller has C initialised: accumulate)
    const int kper = ((K + (int)gridDim.y - 1) / (int)gridDim.y + kTcK - 1) / kTcK * kTcK;
    const int kbeg = (int)blockIdx.y * kper, kend = kbeg + kper < K ? kbeg + kper : K;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
    const uint32_t a_s = (uint32_t)__cvta_generic_to_shared(sA), b_s = (uint32_t)__cvta_generic_to_shared(sB);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc_idesc(N);
    unsigned parity = 0;
    bool issued = false;  // MMAs of this CTA may be in flight
    for (int k0 = kbeg; k0 < kend; k0 += kTcK) {
        const int kc = kend - k0 < kTcK ? kend - k0 : kTcK;  // a multiple of 16
        // stage the chunk: 16-byte units of 8 BF16 along K; rows past M and
        // units past the chunk's K are zero
        for (int e = threadIdx.x; e < kTcM * (kTcK / 8); e += kTcThreads) {
            const int r = e / (kTcK / 8), c = e % (kTcK / 8);
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + r < M && 8 * c < kc) v = *reinterpret_cast<const uint4*>(A + (int64_t)(m0 + r) * lda + k0 + 8 * c);
            *reinterpret_cast<uint4*>(sA + tc_core_off(r, 8 * c)) = v;
        }
        for (int e = threadIdx.x; e < N * (kTcK / 8); e += kTcThreads) {
            const int r = e / (kTcK / 8), c = e % (kTcK / 8);
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (8 * c < kc) v = *reinterpret_cast<const uint4*>(B + (int64_t)r * ldb + k0 + 8 * c);
            *reinterpret_cast<uint4*>(sB + tc_core_off(r, 8 * c)) = v;
        }
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int j = 0; j < kc / 16; ++j) {
                // K = 16 per MMA: two core matrices along K, 256 bytes per step
                const uint64_t da = tc_smem_desc(a_s + 256u * j), db = tc_smem_desc(b_s + 256u * j);
                const uint32_t acc = (k0 > kbeg || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        issued = true;
        // the next chunk overwrites the operands: wait for this chunk's MMAs
        const bool ok = tc_wait(bar, parity);
        parity ^= 1u;
        if (!ok && threadIdx.x == 0) failed = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (failed) break;
        issued = false;
    }
    if (failed) {
        if (threadIdx.x == 0) atomicOr(status, DEV_TIMEOUT);
        if (issued) tc_wait(bar, parity ^ 1u);  // once more, bounded, for the MMAs in flight
    } else if (kbeg < kend) {
        // epilogue: warp w holds rows m0 + 32 w + lane in TMEM lanes 32 w .. 32 w + 31
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                float* d = C + (int64_t)row * ldc + c0;
                if (gridDim.y > 1) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) atomicAdd(d + j, __uint_as_float(v[j]));
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float x = __uint_as_float(v[j]);
                        d[j] = accumulate ? d[j] + x : x;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// ---------------------------------------------------------------------------
// training: generic tensor-core GEMM C[M x N] (+)= A[M x K] B[N x K]^T
// ---------------------------------------------------------------------------
constexpr int kGT = 64;  // tile M and N
__global__ void __launch_bounds__(128) gemm_nt_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                                                      const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ C,
                                                      int ldc, int accumulate) {
    __shared__ __align__(16) __nv_bfloat16 As[kGT][16 + 8];
    __shared__ __align__(16) __nv_bfloat16 Bs[kGT][16 + 8];
    const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < kGT * 16; e += blockDim.x) {
            const int r = e / 16, c = e % 16;
            const int gm = m0 + r, gn = n0 + r, gk = k0 + c;
            As[r][c] = (gm < M && gk < K) ? A[(int64_t)gm * lda + gk] : zero;
            Bs[r][c] = (gn < N && gk < K) ? B[(int64_t)gn * ldb + gk] : zero;
        }
        __syncthreads();
        uint32_t a[4] = {lds32(&As[16 * warp + g][2 * t]), lds32(&As[16 * warp + g + 8][2 * t]),
                         lds32(&As[16 * warp + g][2 * t + 8]), lds32(&As[16 * warp + g + 8][2 * t + 8])};
#pragma unroll
        for (int j = 0; j < 8; ++j) mma_bf16(acc[j], a, lds32(&Bs[8 * j + g][2 * t]), lds32(&Bs[8 * j + g][2 * t + 8]));
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int col = n0 + 8 * j + 2 * t;
        const int row0 = m0 + 16 * warp + g, row1 = row0 + 8;
        const float v[4] = {acc[j][0], acc[j][1], acc[j][2], acc[j][3]};
        const int rr[4] = {row0, row0, row1, row1};
        const int cc[4] = {col, col + 1, col, col + 1};
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (rr[e] < M && cc[e] < N) {
                float* d = C + (int64_t)rr[e] * ldc + cc[e];
                *d = accumulate ? *d + v[e] : v[e];
            }
    }
}

// dst (BF16) [rows x cols] from src (FP32) [rows x cols] (ld = cols), optionally transposed
__global__ void cast_kernel(int64_t rows, int cols, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                            int transpose) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    const int64_t r = e / cols, c = e % cols;
    const __nv_bfloat16 v = __float2bfloat16_rn(src[e]);
    if (transpose) dst[c * rows + r] = v;
    else dst[e] = v;
}

// H = relu(Z + b) in place on Z (FP32), plus the BF16 copy
__global__ void bias_relu_kernel(int64_t rows, int cols, float* __restrict__ Z, const float* __restrict__ b, int relu) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    float v = Z[e] + b[e % cols];
    Z[e] = relu ? fmaxf(v, 0.f) : v;
}

// dZ = dH * (H > 0)
__global__ void relu_back_kernel(int64_t n, float* __restrict__ dH, const float* __restrict__ H) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && !(H[e] > 0.f)) dH[e] = 0.f;
}

struct LossCfg {
    float w_phi, w_trust, trust_tol;
};

// loss of one sample and dL/dO (batch mean); partial loss sums per block
__global__ void loss_kernel(int64_t B, const float* __restrict__ O, const float* __restrict__ T, LossCfg lc,
                            float* __restrict__ dO, double* __restrict__ part) {
    __shared__ double sh[256 / 32];
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double L = 0.0;
    if (b < B) {
        const float* o = O + 8 * b;
        const float* t = T + 4 * b;
        float* d = dO + 8 * b;
        const float inv = 1.0f / (float)B;
        float en = 0.f;
        for (int k = 0; k < 3; ++k) {
            const float r = o[k] - t[k];
            en += r * r;
            d[k] = 2.f * r * inv;
        }
        const float rp = o[3] - t[3];
        d[3] = 2.f * lc.w_phi * rp * inv;
        const float e0 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];  // squared error of the seed alone
        const float y = en < lc.trust_tol * e0 ? 1.f : 0.f;
        const float z = o[4];
        const float p = 1.f / (1.f + expf(-z));
        d[4] = lc.w_trust * (p - y) * inv;
        d[5] = d[6] = d[7] = 0.f;
        // BCE with logits, written stably
        const float bce = fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
        L = (double)en + (double)lc.w_phi * rp * rp + (double)lc.w_trust * bce;
    }
    for (int o = 16; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = L;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

// column sums of dZ [rows x cols] -> out[cols] (fixed order)
__global__ void colsum_kernel(int64_t rows, int cols, const float* __restrict__ dZ, float* __restrict__ out) {
    const int c = blockIdx.x;
    __shared__ float sh[256];
    float s = 0.f;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += dZ[r * cols + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0];
}

__global__ void adam_kernel(int n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ gr, float lr, float b1, float b2, float eps, float c1, float c2) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float g = gr[e];
    const float mm = b1 * m[e] + (1.f - b1) * g;
    const float vv = b2 * v[e] + (1.f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// padded entries of the parameter vector are kept at zero
__global__ void mask_grad_kernel(float* __restrict__ grad) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kMlpOut * kMlpHid) {
        if (e / kMlpHid >= 5) grad[kOffW4 + e] = 0.f;
    }
    if (e < kMlpOut && e >= 5) grad[kOffB4 + e] = 0.f;
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// tcgen05 kernel when the shape and the 16-byte alignment of the operand rows
// allow it (N a multiple of 16 in [16, 128], K a multiple of 16, row strides a
// multiple of 8 elements, 16-byte aligned bases), else the mma.sync kernel
relcp_status gemm_nt(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C,
                     int ldc, bool accumulate, cudaStream_t s, int* status) {
    if (M <= 0 || N <= 0) return RELCP_OK;
    const bool tc = status != nullptr && N % 16 == 0 && N >= 16 && N <= kTcMaxN && K % 16 == 0 && K >= 16 &&
                    lda % 8 == 0 && ldb % 8 == 0 && ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0;
    note_launch();
    if (tc) {
        static bool attr_set[64] = {false};
        int dev = 0;
        RELCP_CUDA(cudaGetDevice(&dev));
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            RELCP_CUDA(cudaFuncSetAttribute(gemm_nt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
            attr_set[dev] = true;
        }
        // a long K with few row tiles (the weight gradients, K = batch) is
        // split over CTAs that add into C (which then must hold its initial
        // value: only with accumulate)
        const int mt = (M + kTcM - 1) / kTcM;
        int ks = 1;
        if (accumulate && mt < 32 && K >= 8 * kTcK) {
            ks = K / (8 * kTcK);
            if (ks > 64) ks = 64;
        }
        gemm_nt_tc_kernel<<<dim3((unsigned)mt, (unsigned)ks), kTcThreads, kTcSmem, s>>>(M, N, K, A, lda, B, ldb, C, ldc,
                                                                                       accumulate ? 1 : 0, status);
    } else {
        dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT);
        gemm_nt_kernel<<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, accumulate ? 1 : 0);
    }
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status cast(int64_t rows, int cols, const float* src, __nv_bfloat16* dst, bool transpose, cudaStream_t s) {
    if (rows * cols == 0) return RELCP_OK;
    note_launch();
    cast_kernel<<<nb(rows * cols), 256, 0, s>>>(rows, cols, src, dst, transpose ? 1 : 0);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

}  // namespace

relcp_status mlp_features_launch(const MlpFeatArgs& a, cudaStream_t s) {
    if (a.npairs == 0) return RELCP_OK;
    note_launch();
    // small blocks: a short pair list still spreads over many SMs
    if (a.targets) features_kernel<double><<<nb(a.npairs, 64), 64, 0, s>>>(a);
    else features_kernel<float><<<nb(a.npairs, 64), 64, 0, s>>>(a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

size_t mlp_image_bytes() { return kFwdSmem; }

relcp_status mlp_pack_launch(const float* params, unsigned char* image, cudaStream_t s) {
    note_launch();
    mlp_pack_kernel<<<64, 256, 0, s>>>(params, image);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status mlp_forward_launch(int64_t npairs, const unsigned char* image, const float* feat, float* out,
                                cudaStream_t s, const int* count_dev, int* status) {
    if (npairs == 0) return RELCP_OK;
    constexpr size_t smem = kFwdSmem + 16;  // image + mbarrier
    static bool attr_set[64] = {false};
    int dev = 0;
    RELCP_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        RELCP_CUDA(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set[dev] = true;
    }
    const int64_t ntiles = (npairs + 16 * kFwdWarps - 1) / (16 * kFwdWarps);
    const int sms = device_sm_count();
    int64_t blocks = (int64_t)(sms > 0 ? sms : 1) * 2;
    if (blocks > ntiles) blocks = ntiles;
    note_launch();
    mlp_forward_kernel<<<(unsigned)blocks, kFwdWarps * 32, smem, s>>>(npairs, image, feat, out, count_dev, status);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status mlp_guess(MlpState& m, int64_t npairs, const int* pa, const int* pb, View<3, const double> x,
                       View<4, const double> q, View<3, const double> axes, const double box[3], cudaStream_t s,
                       const int* idx, const int* count_dev, int* status, const double* box_dev, int64_t min_count,
                       int* ran, int* declined) {
    if (!m.loaded) {
        set_error("learned guess not loaded");
        return RELCP_ERR_STATE;
    }
    if (npairs == 0) return RELCP_OK;
    RELCP_TRY(m.guess.ensure((size_t)(3 * npairs), s));
    MlpFeatArgs fa{};
    fa.npairs = npairs;
    fa.pa = pa;
    fa.pb = pb;
    fa.pstride = 1;
    fa.x = x;
    fa.q = q;
    fa.axes = axes;
    for (int k = 0; k < 3; ++k) fa.box[k] = box[k];
    fa.box_dev = box_dev;
    fa.snsd = nullptr;
    fa.feat = nullptr;
    fa.targets = nullptr;
    fa.idx = idx;
    fa.count_dev = count_dev;
    static bool attr_set[64] = {false};
    int dev = 0;
    RELCP_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        RELCP_CUDA(cudaFuncSetAttribute(mlp_guess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGuessSmem));
        attr_set[dev] = true;
    }
    const int64_t ntiles = (npairs + kGuessTile - 1) / kGuessTile;
    const int sms = device_sm_count();
    int64_t blocks = (int64_t)(sms > 0 ? sms : 1) * 2;
    if (blocks > ntiles) blocks = ntiles;
    note_launch();
    launch_pdl(mlp_guess_kernel, dim3((unsigned)blocks), dim3(kFwdWarps * 32), kGuessSmem, s, fa, m.image.p,
               View<3, double>::soa(m.guess.p, npairs), status, min_count, ran, declined);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

void mlp_release(MlpState& m, cudaStream_t s) {
    m.params.release(s);
    m.image.release(s);
    m.guess.release(s);
    m.loaded = false;
}

// one training step (see relcp_mlp_train_step)
relcp_status mlp_train_step(int64_t B, float* params, float* am, float* av, const float* feat, const float* targets,
                            const relcp_mlp_train_config& tc, float* grad_out, double* loss_out, cudaStream_t s) {
    if (B <= 0 || B > (1 << 24)) {
        set_error("batch must be in [1, 2^24]");
        return RELCP_ERR_INVALID_ARG;
    }
    const int H = kMlpHid;
    DBuf<float> Z1, Z2, Z3, O, dO, dH, grad, dH2;
    DBuf<__nv_bfloat16> Xb, H1b, H2b, H3b, Wb, Wtb, T1, T2;
    DBuf<double> part;
    DBuf<int> tstat;  // DEV_* bits of the tensor-core GEMMs
    relcp_status st = RELCP_OK;
    auto R = [&](relcp_status e) {
        if (st == RELCP_OK) st = e;
        return st != RELCP_OK;
    };
    do {
        if (R(Z1.ensure(B * H, s)) || R(Z2.ensure(B * H, s)) || R(Z3.ensure(B * H, s)) || R(O.ensure(B * 8, s)) ||
            R(dO.ensure(B * 8, s)) || R(dH.ensure(B * H, s)) || R(dH2.ensure(B * H, s)) ||
            R(grad.ensure(kMlpParams, s)) || R(Xb.ensure(B * 16, s)) || R(H1b.ensure(B * H, s)) ||
            R(H2b.ensure(B * H, s)) || R(H3b.ensure(B * H, s)) || R(Wb.ensure(H * H, s)) ||
            R(Wtb.ensure(H * H, s)) || R(T1.ensure(B * H, s)) || R(T2.ensure(B * H, s)) ||
            R(part.ensure(nb(B), s)) || R(tstat.ensure(1, s)))
            break;
        cudaError_t ce = cudaMemsetAsync(grad.p, 0, kMlpParams * sizeof(float), s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(tstat.p, 0, sizeof(int), s);
        if (ce != cudaSuccess) {
            set_error("%s", cudaGetErrorString(ce));
            st = RELCP_ERR_CUDA;
            break;
        }
        // ---- forward
        if (R(cast(B, 16, feat, Xb.p, false, s))) break;
        struct L {
            int in, out, offw, offb;
        };
        const L layers[4] = {{16, H, kOffW1, kOffB1}, {H, H, kOffW2, kOffB2}, {H, H, kOffW3, kOffB3}, {H, 8, kOffW4, kOffB4}};
        float* Zs[4] = {Z1.p, Z2.p, Z3.p, O.p};
        const __nv_bfloat16* Ins[4] = {Xb.p, H1b.p, H2b.p, H3b.p};
        __nv_bfloat16* Outs[3] = {H1b.p, H2b.p, H3b.p};
        for (int l = 0; l < 4 && st == RELCP_OK; ++l) {
            const L& ly = layers[l];
            if (R(cast(ly.out, ly.in, params + ly.offw, Wb.p, false, s))) break;
            if (R(gemm_nt((int)B, ly.out, ly.in, Ins[l], ly.in, Wb.p, ly.in, Zs[l], ly.out, false, s, tstat.p))) break;
            note_launch();
            bias_relu_kernel<<<nb(B * ly.out), 256, 0, s>>>(B, ly.out, Zs[l], params + ly.offb, l < 3 ? 1 : 0);
            if (l < 3 && R(cast(B, ly.out, Zs[l], Outs[l], false, s))) break;
        }
        if (st != RELCP_OK) break;
        // ---- loss and dO
        LossCfg lc{tc.w_phi, tc.w_trust, tc.trust_tol};
        note_launch();
        loss_kernel<<<nb(B), 256, 0, s>>>(B, O.p, targets, lc, dO.p, part.p);
        // ---- backward: for l = 3..0: dW_l = dZ_l^T H_{l-1}, db_l = colsum dZ_l, dH_{l-1} = dZ_l W_l
        float* dZ = dO.p;  // dZ of layer 3 (output layer, no activation)
        int dzcols = 8;
        for (int l = 3; l >= 0 && st == RELCP_OK; --l) {
            const L& ly = layers[l];
            // transposes: dZ^T [out x B], H_{l-1}^T [in x B]
            if (R(cast(B, dzcols, dZ, T1.p, true, s))) break;
            const float* Hprev = l == 0 ? feat : Zs[l - 1];
            if (R(cast(B, ly.in, Hprev, T2.p, true, s))) break;
            // (grad is zeroed above and each weight block receives one product:
            // accumulating lets the tensor-core GEMM split its long K = batch)
            if (R(gemm_nt(ly.out, ly.in, (int)B, T1.p, (int)B, T2.p, (int)B, grad.p + ly.offw, ly.in, true, s,
                          tstat.p)))
                break;
            note_launch();
            colsum_kernel<<<ly.out, 256, 0, s>>>(B, dzcols, dZ, grad.p + ly.offb);
            if (l == 0) break;
            // dH_{l-1} [B x in] = dZ [B x out] W_l [out x in]: NT form with B-operand W^T [in x out]
            // (T1 is free again: the dW GEMM that read it precedes this cast on the stream)
            if (R(cast(B, dzcols, dZ, T1.p, false, s))) break;
            const __nv_bfloat16* dZb = T1.p;
            if (R(cast(ly.out, ly.in, params + ly.offw, Wtb.p, true, s))) break;
            float* dHn = (l % 2 == 1) ? dH.p : dH2.p;
            if (R(gemm_nt((int)B, ly.in, ly.out, dZb, ly.out, Wtb.p, ly.out, dHn, ly.in, false, s, tstat.p))) break;
            note_launch();
            relu_back_kernel<<<nb(B * ly.in), 256, 0, s>>>(B * ly.in, dHn, Zs[l - 1]);
            dZ = dHn;
            dzcols = ly.in;
        }
        if (st != RELCP_OK) break;
        note_launch();
        mask_grad_kernel<<<nb(kMlpHid * kMlpIn), 256, 0, s>>>(grad.p);
        if (grad_out) {
            ce = cudaMemcpyAsync(grad_out, grad.p, kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice, s);
            if (ce != cudaSuccess) {
                set_error("%s", cudaGetErrorString(ce));
                st = RELCP_ERR_CUDA;
                break;
            }
        }
        if (tc.lr > 0.f) {
            const float c1 = 1.f - powf(tc.beta1, (float)tc.step), c2 = 1.f - powf(tc.beta2, (float)tc.step);
            note_launch();
            adam_kernel<<<nb(kMlpParams), 256, 0, s>>>(kMlpParams, params, am, av, grad.p, tc.lr, tc.beta1, tc.beta2,
                                                       tc.eps, c1, c2);
        }
        std::vector<double> hp(nb(B));
        int hstat = 0;
        ce = cudaMemcpyAsync(hp.data(), part.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hstat, tstat.p, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce == cudaSuccess && (hstat & DEV_TIMEOUT)) {
            set_error("a tensor-core GEMM's wait for its MMAs timed out");
            st = RELCP_ERR_TIMEOUT;
            break;
        }
        if (ce != cudaSuccess) {
            set_error("%s", cudaGetErrorString(ce));
            st = RELCP_ERR_CUDA;
            break;
        }
        double L = 0;
        for (double v : hp) L += v;
        if (loss_out) *loss_out = L / (double)B;
    } while (0);
    DBuf<float>* fb[] = {&Z1, &Z2, &Z3, &O, &dO, &dH, &grad, &dH2};
    for (auto* b : fb) b->release(s);
    DBuf<__nv_bfloat16>* bb[] = {&Xb, &H1b, &H2b, &H3b, &Wb, &Wtb, &T1, &T2};
    for (auto* b : bb) b->release(s);
    part.release(s);
    tstat.release(s);
    return st;
}

}  // namespace relcp

using namespace relcp;

extern "C" relcp_status relcp_mlp_features(int64_t npairs, const int32_t* pairs, int64_t n, const double* x,
                                           const double* q, const double* axes, const double* box3,
                                           const double* snsd_out, float* feat, float* targets, void* stream) {
    if (npairs < 0 || n < 0 || !box3 || (npairs > 0 && (!pairs || !x || !q || !axes || !feat)))
        return set_error("bad argument"), RELCP_ERR_INVALID_ARG;
    if (targets && !snsd_out) return set_error("targets need snsd_out"), RELCP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    MlpFeatArgs a{};
    a.npairs = npairs;
    a.pa = pairs;
    a.pb = pairs + 1;
    a.pstride = 2;
    a.x = View<3, const double>::aos(x, 3);
    a.q = View<4, const double>::aos(q, 4);
    a.axes = View<3, const double>::aos(axes, 3);
    for (int k = 0; k < 3; ++k) a.box[k] = box3[k];
    a.snsd = snsd_out;
    a.snsd_s = 10;
    a.snsd_c = 1;
    a.feat = feat;
    a.targets = targets;
    RELCP_TRY(mlp_features_launch(a, s));
    RELCP_CUDA(cudaStreamSynchronize(s));
    return RELCP_OK;
}

extern "C" relcp_status relcp_mlp_forward(int64_t npairs, const float* params, const float* feat, float* out,
                                          void* stream) {
    if (npairs < 0 || !params || (npairs > 0 && (!feat || !out))) return set_error("bad argument"), RELCP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (npairs == 0) return RELCP_OK;
    DBuf<unsigned char> image;
    DBuf<int> status;
    relcp_status st = image.ensure(kFwdSmem, s);
    if (st == RELCP_OK) st = status.ensure(1, s);
    if (st == RELCP_OK && cudaMemsetAsync(status.p, 0, sizeof(int), s) != cudaSuccess) st = RELCP_ERR_CUDA;
    if (st == RELCP_OK) st = mlp_pack_launch(params, image.p, s);
    if (st == RELCP_OK) st = mlp_forward_launch(npairs, image.p, feat, out, s, nullptr, status.p);
    int bits = 0;
    if (st == RELCP_OK && cudaMemcpyAsync(&bits, status.p, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = RELCP_ERR_CUDA;
    image.release(s);
    status.release(s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == RELCP_OK) st = RELCP_ERR_CUDA;
    if (st == RELCP_OK) st = status_from_device(bits);
    return st;
}

extern "C" relcp_status relcp_mlp_train_step(int64_t batch, float* params, float* adam_m, float* adam_v,
                                             const float* feat, const float* targets,
                                             const relcp_mlp_train_config* cfg, float* grad_out, double* loss_out,
                                             void* stream) {
    if (!params || !feat || !targets || !cfg) return set_error("bad argument"), RELCP_ERR_INVALID_ARG;
    if (cfg->lr > 0.f && (!adam_m || !adam_v || cfg->step < 1))
        return set_error("Adam needs m, v and step >= 1"), RELCP_ERR_INVALID_ARG;
    return mlp_train_step(batch, params, adam_m, adam_v, feat, targets, *cfg, grad_out, loss_out, (cudaStream_t)stream);
}
