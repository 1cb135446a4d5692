// Shared-normal signed distance (SNSD) of ellipsoid pairs, one thread per pair.
//
// For a unit direction n (from body a to body b) the gap between the two
// support slabs is
//     G(n) = n.d - sqrt(n.Pa n) - sqrt(n.Pb n),   d = c_b - c_a (minimum image),
// with Pa = R_a diag(a^2) R_a^T.  Its gradient is y_b(n) - y_a(n) (support
// points y_a = c_a + Pa n/|.|, y_b = c_b - Pb n/|.|), so a stationary point on
// the sphere is a pair of surface points with opposite normals whose
// difference is parallel to n -- the shared-normal points of Sec. 2.1.4, with
// y_b - y_a = Phi n as in the interior tangent-ball lemma -- and the signed
// distance is Phi = max_n G(n) (distance when separated, minus the
// penetration depth when overlapping).
//
// Newton ascent on the sphere: tangent-plane gradient and Hessian
// (G is 1-homogeneous, so the Riemannian Hessian is T^T H T - G I), shifted
// to be negative definite when it is not, with step halving until G does not
// fall.  Start: a supplied normal (warm start from an earlier evaluation or the
// learned guess) or the best of four seeds d, Pa^-1 d, Pb^-1 d,
// (Pa + Pb)^-1 d.  The mixed path iterates in FP32 and finishes with FP64
// Newton steps (the polish); the plain path is FP64 throughout.
#include "snsd_math.cuh"

namespace relcp {

namespace {

using namespace snsd_math;

constexpr int kThreads = 128;

__device__ __forceinline__ Sym3<double> load_P(View<6, const double> P, int64_t i) {
    return Sym3<double>{P(0, i), P(1, i), P(2, i), P(3, i), P(4, i), P(5, i)};
}

// A grid-stride loop over the pairs: a subset launch is sized to one wave of
// resident blocks, not to the capacity, so a C^k evaluation of the few pairs
// new to the list costs one wave of blocks that mostly find no work.
__global__ void __launch_bounds__(kThreads) snsd_kernel(SnsdArgs a) {
    pdl_wait();
    pdl_trigger();
    const int64_t count = a.count_dev ? (int64_t)*a.count_dev : a.npairs;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // a subset launch has no violator flags; a capacity-sized one clears the
    // flags of the slots past the count
    const int64_t kend = (a.viol && !a.idx) ? a.npairs : count;
    double maxov = 0.0;
    int it_max = 0;
    long long it_sum = 0;
    int nvl = 0;
    for (int64_t k_thr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k_thr < kend; k_thr += stride) {
        if (k_thr >= count) {
            a.viol[k_thr] = 0;  // (a.viol set: kend is the capacity only then)
            continue;
        }
        const int64_t p = a.idx ? (int64_t)a.idx[k_thr] : k_thr;  // the pair
        const int64_t gk = k_thr;                                  // its start-normal slot
        const int i = a.pa[p * a.pstride];
        const int j = a.pb[p * a.pstride];
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = min_image(a.x(k, j) - a.x(k, i), a.box_dev ? a.box_dev[k] : a.box[k]);
        const Sym3<double> Pa = load_P(a.P, i), Pb = load_P(a.P, j);
        const bool hg = a.guess.c[0] != nullptr && (!a.guess_on || *a.guess_on != 0);
        snsd_math::PairResult o;
        if (a.shape == RELCP_SHAPE_SPHEROCYLINDER)
            snsd_math::capsule_pair(d, Pa, Pb, o);
        else
            snsd_math::snsd_pair(d, Pa, Pb, hg, hg ? a.guess(0, gk) : 0.0, hg ? a.guess(1, gk) : 0.0,
                                 hg ? a.guess(2, gk) : 0.0, a.mixed != 0, o, a.newton_cap);
        if (!o.ok) atomicOr(a.status, DEV_NEWTON);
        const double G = o.phi;
        const int iters = o.iters;
        a.out.phi[p * a.out.phi_s] = G;
        for (int k = 0; k < 3; ++k) {
            a.out.n(k, p) = o.n[k];
            a.out.ra(k, p) = o.ra[k];
            a.out.rb(k, p) = o.rb[k];
        }
        if (a.out.iters) a.out.iters[p] = iters;
        const int itabs = iters < 0 ? -iters : iters;
        it_max = max(it_max, itabs);
        it_sum += itabs;
        const bool viol_here = G < -a.eps;
        if (a.viol) a.viol[p] = viol_here ? 1 : 0;
        nvl += viol_here ? 1 : 0;
        if (G < 0.0 && -G > maxov) maxov = -G;
    }
    // one atomic per block (skipped when it would change nothing) for the
    // largest overlap, the iteration counts and the violators; the overlap
    // maximum is taken on the bits of non-negative doubles (integer max, no
    // FP64 unit)
    __shared__ unsigned long long sh_ov[kThreads / 32];
    __shared__ int sh_it[kThreads / 32];
    __shared__ long long sh_is[kThreads / 32];
    __shared__ int sh_nv[kThreads / 32];
    unsigned long long ovb = (unsigned long long)__double_as_longlong(maxov);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, ovb, o);
        ovb = y > ovb ? y : ovb;
        it_max = max(it_max, __shfl_xor_sync(0xffffffffu, it_max, o));
        it_sum += __shfl_xor_sync(0xffffffffu, it_sum, o);
        nvl += __shfl_xor_sync(0xffffffffu, nvl, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh_ov[threadIdx.x >> 5] = ovb;
        sh_it[threadIdx.x >> 5] = it_max;
        sh_is[threadIdx.x >> 5] = it_sum;
        sh_nv[threadIdx.x >> 5] = nvl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        int mi = 0, nv = 0;
        long long ms = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            m = sh_ov[w] > m ? sh_ov[w] : m;
            mi = max(mi, sh_it[w]);
            ms += sh_is[w];
            nv += sh_nv[w];
        }
        if (a.maxov_bits && m) atomicMax(a.maxov_bits, m);
        if (a.newton_max && mi) atomicMax(a.newton_max, mi);
        if (a.iters_sum && ms) atomicAdd(a.iters_sum, (unsigned long long)ms);
        if (a.nviol && nv) atomicAdd(a.nviol, nv);
    }
}

__global__ void shape_kernel(int64_t n, View<4, const double> q, View<3, const double> axes, View<6, double> P) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = q(0, i), x = q(1, i), y = q(2, i), z = q(3, i);
    double l = sqrt(s * s + x * x + y * y + z * z);
    double R[9];
    quat_to_R(s / l, x / l, y / l, z / l, R);
    double a0 = axes(0, i), a1 = axes(1, i), a2 = axes(2, i);
    Sym3<double> S = rot_diag_rot(R, a0 * a0, a1 * a1, a2 * a2);
    P(0, i) = S.xx;
    P(1, i) = S.yy;
    P(2, i) = S.zz;
    P(3, i) = S.xy;
    P(4, i) = S.xz;
    P(5, i) = S.yz;
}

}  // namespace

relcp_status snsd_launch(const SnsdArgs& a, cudaStream_t s) {
    if (a.npairs == 0) return RELCP_OK;
    // blocks resident at once per SM (register-limited)
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        RELCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, snsd_kernel, kThreads, 0));
        per_sm = b > 0 ? b : 1;
    }
    // a subset launch (a few new pairs against the list's capacity) takes
    // one wave of blocks that loop; a full evaluation one thread per pair
    const int64_t need = (a.npairs + kThreads - 1) / kThreads;
    int64_t nb = need;
    if (a.idx) {
        const int sms = device_sm_count();
        nb = (int64_t)(sms > 0 ? sms : 1) * per_sm;
        if (nb > need) nb = need;
    }
    note_launch();
    launch_pdl(snsd_kernel, dim3((unsigned)nb), dim3(kThreads), 0, s, a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status shape_launch(int64_t n, View<4, const double> q, View<3, const double> axes, View<6, double> P,
                          cudaStream_t s) {
    if (n == 0) return RELCP_OK;
    note_launch();
    shape_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, q, axes, P);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

}  // namespace relcp
