// Per-body and per-row kernels of one ReLCP time step (Algorithm 1).
//
//   prep      : normalised q, shape matrix P = R diag(a^2) R^T, the body
//               operator K (overdamped: the local-drag mobility of Eq.
//               ellipsoid_mobility, (1/xi) diag(I/L, 12 I/L^3), L = twice the
//               largest semi-axis; inertial: dt M^-1 with m = 4/3 pi abc rho
//               and I_body = m/5 (b^2+c^2, a^2+c^2, a^2+b^2), rotated to the
//               world frame at C^k), bounding radius, and
//               U_free = vel + K F_ext (+ the affine background velocity).
//   rows      : one constraint row per flagged pair, written at position
//               base + exclusive-scan(flags): the Jacobian row
//               [-n, -(r_a x n), n, (r_b x n)] (Appendix, proof of the
//               stopping rule), its diagonal A_aa = c d^T K d and its offset:
//                 A_0 rows       q = Phi(C^k) + c d^T U_free      (Eq. relcp, n = 0)
//                 appended rows  q = Phi(C_n) - c d^T K D gamma_{n-1}
//               (the pull-back of Sec. 3.1.3: retained rows keep their q).
//   trial     : C_{n+1} = C^k + dt G^k (U_free + K D gamma_n), the telescoped
//               trial configuration of Eq. relcp; q normalised.
//   accept    : C^{k+1} = the last trial, positions wrapped into the box.
#include "relcp_internal.cuh"
#include "step_kernels.cuh"
#include "step_math.cuh"

namespace relcp {

namespace {

constexpr int kT = 256;
inline unsigned nb(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

__device__ __forceinline__ void prep_one(const PrepArgs& a, int64_t i) {
    const int64_t n = a.n;
    double qin[4], ax[3], vel[6], f[6], x[3];
    for (int k = 0; k < 4; ++k) qin[k] = a.q[k * n + i];
    for (int k = 0; k < 3; ++k) {
        ax[k] = a.axes[k * n + i];
        x[k] = a.x[k * n + i];
    }
    for (int k = 0; k < 6; ++k) {
        vel[k] = a.vel[k * n + i];
        f[k] = a.fext[k * n + i];
    }
    step_math::BodyPrep b;
    step_math::prep_body(qin, ax, vel, f, x, a.dynamics, a.dt, a.drag_xi, a.density, a.strain_rate, a.box, b,
                         a.shape);
    for (int k = 0; k < 4; ++k) a.q[k * n + i] = b.q[k];
    a.P[i] = b.P.xx;
    a.P[n + i] = b.P.yy;
    a.P[2 * n + i] = b.P.zz;
    a.P[3 * n + i] = b.P.xy;
    a.P[4 * n + i] = b.P.xz;
    a.P[5 * n + i] = b.P.yz;
    a.rb[i] = b.rb;
    for (int k = 0; k < 7; ++k) a.K[k * n + i] = b.K[k];
    if (a.Kf)
        for (int k = 0; k < 7; ++k) a.Kf[k * n + i] = (float)b.K[k];
    for (int k = 0; k < 6; ++k) a.ufree[k * n + i] = b.ufree[k];
    if (a.ufreef)
        for (int k = 0; k < 6; ++k) a.ufreef[k * n + i] = (float)b.ufree[k];
}

// the next step's prep after an accepted trial (overdamped): q was normalised
// by the trial and P at that orientation is Pt; K, Kf and rb depend on the
// semi-axes and the config only, so they hold; U_free = vel + K F_ext (+ the
// affine background velocity at the accepted position)
__device__ __forceinline__ void prep_keep(const PrepArgs& a, const double* __restrict__ Pt, int64_t i) {
    const int64_t n = a.n;
#pragma unroll
    for (int k = 0; k < 6; ++k) a.P[k * n + i] = Pt[k * n + i];
    double K[7], u[6], f[6];
#pragma unroll
    for (int k = 0; k < 7; ++k) K[k] = a.K[k * n + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        u[k] = a.vel[k * n + i];
        f[k] = a.fext[k * n + i];
    }
    // the same operations, in the same order, as prep_body
    u[0] += K[0] * f[0];
    u[1] += K[0] * f[1];
    u[2] += K[0] * f[2];
    u[3] += K[1] * f[3] + K[4] * f[4] + K[5] * f[5];
    u[4] += K[4] * f[3] + K[2] * f[4] + K[6] * f[5];
    u[5] += K[5] * f[3] + K[6] * f[4] + K[3] * f[5];
    if (a.strain_rate != 0.0)
        for (int k = 0; k < 3; ++k)
            if (a.box[k] > 0.0) u[k] += a.strain_rate * (a.x[k * n + i] - 0.5 * a.box[k]);
    if (a.dynamics == RELCP_OVERDAMPED_2D) step_math::planar_velocity(u);
#pragma unroll
    for (int k = 0; k < 6; ++k) a.ufree[k * n + i] = u[k];
    if (a.ufreef)
#pragma unroll
        for (int k = 0; k < 6; ++k) a.ufreef[k * n + i] = (float)u[k];
}

__global__ void prep_kernel(PrepArgs a) {
    pdl_wait();
    pdl_trigger();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) prep_one(a, i);
}

__global__ void flag_le_kernel(int64_t cap, const int* __restrict__ np_dev, const double* __restrict__ phi, double thr,
                               int* __restrict__ flags) {
    pdl_wait();
    pdl_trigger();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < cap) flags[p] = (p < *np_dev && phi[p] <= thr) ? 1 : 0;
}

__device__ __forceinline__ double body_rate(const double* U, int64_t n, int i, int j, const double* nn,
                                            const double* ta, const double* tb) {
    double Ui[6], Uj[6];
    for (int k = 0; k < 6; ++k) {
        Ui[k] = U[k * n + i];
        Uj[k] = U[k * n + j];
    }
    return step_math::row_rate(Ui, Uj, nn, ta, tb);
}

// One row on the mixed path: the Jacobian row, its rate and its diagonal in
// FP32 (the LCP iterates on FP32 geometry anyway, and the lever arms come from
// the FP32 Newton phase); the offset q = Phi + c d^T U keeps Phi in FP64 and
// adds the FP32 rate term, whose rounding (relative 1e-7 of c |d^T U|) is far
// below the LCP tolerance.  The FP64 geometry written for read-outs is the
// widened FP32 one.  The periodic-image correction of the affine background
// velocity needs only which image the pair uses: decided from the FP64
// separation, as in the FP64 path.
__device__ __forceinline__ void rows_mixed(const RowsArgs& a, int64_t p, int64_t r, int i, int j) {
    const int64_t P = a.npairs, C = a.cap, n = a.nbodies;
    float nn[3], ra[3], rb[3], ta[3], tb[3];
    for (int k = 0; k < 3; ++k) {
        nn[k] = (float)a.snsd[(1 + k) * P + p];
        ra[k] = (float)a.snsd[(4 + k) * P + p];
        rb[k] = (float)a.snsd[(7 + k) * P + p];
    }
    const double phi = a.snsd[p];
    ta[0] = ra[1] * nn[2] - ra[2] * nn[1];
    ta[1] = ra[2] * nn[0] - ra[0] * nn[2];
    ta[2] = ra[0] * nn[1] - ra[1] * nn[0];
    tb[0] = rb[1] * nn[2] - rb[2] * nn[1];
    tb[1] = rb[2] * nn[0] - rb[0] * nn[2];
    tb[2] = rb[0] * nn[1] - rb[1] * nn[0];
    if (a.planar) step_math::planar_row(nn, ta, tb);
    a.ia[r] = i;
    a.ib[r] = j;
    a.rec[r] = a.rec_index;
    a.pair[r] = (int)p;
    for (int k = 0; k < 3; ++k) {
        a.geomf[k * C + r] = nn[k];
        a.geomf[(3 + k) * C + r] = ta[k];
        a.geomf[(6 + k) * C + r] = tb[k];
        a.geom[k * C + r] = (double)nn[k];
        a.geom[(3 + k) * C + r] = (double)ta[k];
        a.geom[(6 + k) * C + r] = (double)tb[k];
    }
    float Ui[6], Uj[6];
    if (a.rec_index == 0) {
        for (int k = 0; k < 6; ++k) {
            Ui[k] = a.ufreef[k * n + i];
            Uj[k] = a.ufreef[k * n + j];
        }
    } else {
        for (int k = 0; k < 6; ++k) {
            Ui[k] = (float)a.uc[k * n + i];
            Uj[k] = (float)a.uc[k * n + j];
        }
    }
    float rate = 0.f;
    for (int k = 0; k < 3; ++k) rate += nn[k] * (Uj[k] - Ui[k]);
    for (int k = 0; k < 3; ++k) rate += tb[k] * Uj[3 + k] - ta[k] * Ui[3 + k];
    double qv;
    if (a.rec_index == 0) {
        if (a.strain_rate != 0.0) {
            const double* L = a.box_dev ? a.box_dev : a.box;
            float corr = 0.f;
            for (int k = 0; k < 3; ++k) {
                const double raw = a.x[k * n + j] - a.x[k * n + i];
                corr += nn[k] * (float)(min_image(raw, L[k]) - raw);  // 0 or a multiple of the box side
            }
            rate += (float)a.strain_rate * corr;
        }
        qv = phi + a.c * (double)rate;
    } else {
        qv = phi - a.c * (double)rate;
    }
    a.q[r] = qv;
    if (a.qf) a.qf[r] = (float)qv;
    // diagonal c d^T K d
    float acc = (a.Kf[i] + a.Kf[j]) * (nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    for (int side = 0; side < 2; ++side) {
        const int b = side ? j : i;
        const float* t = side ? tb : ta;
        const float kxx = a.Kf[n + b], kyy = a.Kf[2 * n + b], kzz = a.Kf[3 * n + b], kxy = a.Kf[4 * n + b],
                    kxz = a.Kf[5 * n + b], kyz = a.Kf[6 * n + b];
        acc += t[0] * (kxx * t[0] + kxy * t[1] + kxz * t[2]) + t[1] * (kxy * t[0] + kyy * t[1] + kyz * t[2]) +
               t[2] * (kxz * t[0] + kyz * t[1] + kzz * t[2]);
    }
    const float cf = (float)a.c;
    a.diag[r] = (double)(cf * acc);
    if (a.invdf) a.invdf[r] = 1.f / (cf * acc);
    if (a.gammaf) a.gammaf[r] = (a.rec_index == 0 && a.gamma0) ? (float)a.gamma0[p] : 0.f;
    if (a.gamma) a.gamma[r] = (a.rec_index == 0 && a.gamma0) ? a.gamma0[p] : 0.0;
}

__global__ void rows_kernel(RowsArgs a) {
    pdl_wait();
    pdl_trigger();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {
        int64_t total = a.base + a.scan[a.npairs];
        *a.nrows_dev = (int)(total < a.cap ? total : a.cap);
        if (a.nrows0_dev) *a.nrows0_dev = (int)(total < a.cap ? total : a.cap);
        if (a.clear3) a.clear3[0] = a.clear3[1] = a.clear3[2] = 0ull;
    }
    if (p >= a.npairs) return;
    int64_t r = a.flags[p] ? a.base + a.scan[p] : -1;
    if (r >= a.cap) {
        atomicOr(a.status, DEV_CAPACITY);
        r = -1;
    }
    if (a.rowof) a.rowof[p] = (int)r;
    if (r < 0) return;
    int i = a.pa[p], j = a.pb[p];
    const int64_t P = a.npairs;
    if (a.geomf && a.ufreef && a.Kf) {
        rows_mixed(a, p, r, i, j);
        return;
    }
    double nn[3], ra[3], rb[3], ta[3], tb[3];
    for (int k = 0; k < 3; ++k) {
        nn[k] = a.snsd[(1 + k) * P + p];
        ra[k] = a.snsd[(4 + k) * P + p];
        rb[k] = a.snsd[(7 + k) * P + p];
    }
    double phi = a.snsd[p];
    step_math::row_torques(nn, ra, rb, ta, tb);
    if (a.planar) step_math::planar_row(nn, ta, tb);
    const int64_t C = a.cap;
    a.ia[r] = i;
    a.ib[r] = j;
    a.rec[r] = a.rec_index;
    a.pair[r] = (int)p;
    for (int k = 0; k < 3; ++k) {
        a.geom[k * C + r] = nn[k];
        a.geom[(3 + k) * C + r] = ta[k];
        a.geom[(6 + k) * C + r] = tb[k];
    }
    if (a.geomf)
        for (int k = 0; k < 3; ++k) {
            a.geomf[k * C + r] = (float)nn[k];
            a.geomf[(3 + k) * C + r] = (float)ta[k];
            a.geomf[(6 + k) * C + r] = (float)tb[k];
        }
    // offset
    double qv;
    if (a.rec_index == 0) {
        double rate = body_rate(a.ufree, a.nbodies, i, j, nn, ta, tb);
        if (a.strain_rate != 0.0) {
            double xi[3], xj[3];
            for (int k = 0; k < 3; ++k) {
                xi[k] = a.x[k * a.nbodies + i];
                xj[k] = a.x[k * a.nbodies + j];
            }
            rate += a.strain_rate * step_math::affine_image_corr(xi, xj, nn, a.box_dev ? a.box_dev : a.box);
        }
        qv = phi + a.c * rate;
    } else {
        qv = phi - a.c * body_rate(a.uc, a.nbodies, i, j, nn, ta, tb);
    }
    a.q[r] = qv;
    if (a.qf) a.qf[r] = (float)qv;
    // diagonal c d^T K d
    double Ki[7], Kj[7];
    for (int k = 0; k < 7; ++k) {
        Ki[k] = a.K[k * a.nbodies + i];
        Kj[k] = a.K[k * a.nbodies + j];
    }
    const double acc = step_math::row_dKd(Ki, Kj, nn, ta, tb);
    a.diag[r] = a.c * acc;
    if (a.invd) a.invd[r] = 1.0 / (a.c * acc);
    if (a.invdf) a.invdf[r] = (float)(1.0 / (a.c * acc));
    const double g0 = (a.rec_index == 0 && a.gamma0) ? a.gamma0[p] : 0.0;
    if (a.gamma) a.gamma[r] = g0;
    if (a.gammaf) a.gammaf[r] = (float)g0;
}

__global__ void reuse_kernel(ReuseArgs a) {
    pdl_wait();
    pdl_trigger();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool need = false;
    if (p < a.npairs && p < *a.np_dev) {
        const PairMemo m = a.memo[a.pv[p]];
        const int sp = a.stamp_prev_dev ? *a.stamp_prev_dev : a.stamp_prev;
        const bool hit = sp >= 0 && m.stamp == sp && m.pidx >= 0;
        a.gamma0[p] = (hit && a.use_gamma) ? m.gamma : 0.0;
        const bool take = hit && a.reuse_snsd;
        if (take) {
#pragma unroll
            for (int k = 0; k < 10; ++k) a.s0[k * a.npairs + p] = a.sprev[k * a.sprev_stride + m.pidx];
            a.it0[p] = 0;
        }
        need = !take;
    }
    // warp-aggregated append to the list of pairs to evaluate
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    if (mask) {
        const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(a.count, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (need) a.list[base + __popc(mask & ((1u << lane) - 1u))] = (int)p;
    }
}

__global__ void memo_save_kernel(MemoSaveArgs a) {
    pdl_wait();
    pdl_trigger();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npairs || p >= *a.np_dev) return;
    const int r = a.rowof[p];
    double g = 0.0;
    if (r >= 0) g = a.gamma ? a.gamma[r] : (double)a.gammaf[r];
    PairMemo m;
    m.stamp = a.stamp;
    m.pidx = (int)p;
    m.gamma = g;
    a.memo[a.pv[p]] = m;
}

__global__ void trial_kernel(TrialArgs a) {
    pdl_wait();
    pdl_trigger();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d2max = 0.0;  // squared look-ahead displacement of this body
    if (i < a.n) {
    const int64_t n = a.n;
    double U[6], x[3], q[4], ax[3], xt[3], qt[4];
    for (int k = 0; k < 6; ++k) {
        U[k] = a.ufree[k * n + i] + a.uc[k * n + i];
        a.ustep[k * n + i] = U[k];
    }
    for (int k = 0; k < 3; ++k) {
        x[k] = a.x[k * n + i];
        ax[k] = a.axes[k * n + i];
    }
    for (int k = 0; k < 4; ++k) q[k] = a.q[k * n + i];
    Sym3<double> P;
    step_math::trial_body(x, q, U, ax, a.dt, xt, qt, P, a.shape);
    for (int k = 0; k < 3; ++k) a.xt[k * n + i] = xt[k];
    for (int k = 0; k < 4; ++k) a.qt[k * n + i] = qt[k];
    a.Pt[i] = P.xx;
    a.Pt[n + i] = P.yy;
    a.Pt[2 * n + i] = P.zz;
    a.Pt[3 * n + i] = P.xy;
    a.Pt[4 * n + i] = P.xz;
    a.Pt[5 * n + i] = P.yz;
    if (a.xb) {
        // the same arithmetic as the broad phase's displacement check
        double d2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double sf = a.sfac_dev ? a.sfac_dev[k] : a.sfac[k];
            const double lb = a.la_box_dev ? a.la_box_dev[k] : a.la_box[k];
            const double d = min_image(xt[k] - sf * a.xb[k * n + i], lb);
            d2 += d * d;
        }
        d2max = d2;
    }
    }
    if (a.xb) {
        // the largest squared displacement (the host takes its square root):
        // integer max of the non-negative doubles' bits
        unsigned long long b = (unsigned long long)__double_as_longlong(d2max);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
            b = y > b ? y : b;
        }
        if ((threadIdx.x & 31) == 0 && b) atomicMax(a.la_dmax, b);
    }
}

__global__ void accept_kernel(AcceptArgs a) {
    pdl_wait();
    pdl_trigger();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int64_t n = a.n;
    for (int k = 0; k < 3; ++k) a.x[k * n + i] = step_math::wrap_coord(a.xt[k * n + i], a.box[k]);
    for (int k = 0; k < 4; ++k) a.q[k * n + i] = a.qt[k * n + i];
    if (a.inertial)
        for (int k = 0; k < 6; ++k) a.vel[k * n + i] = a.ustep[k * n + i];
    if (a.next.n == n) {  // reads back this thread's own writes
        if (a.keep) prep_keep(a.next, a.Pt, i);
        else prep_one(a.next, i);
    }
}


}  // namespace

relcp_status prep_launch(const PrepArgs& a, cudaStream_t s) {
    if (a.n == 0) return RELCP_OK;
    note_launch();
    launch_pdl(prep_kernel, dim3(nb(a.n)), dim3(kT), 0, s, a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}
relcp_status flag_le_launch(int64_t cap, const int* np_dev, const double* phi, double thr, int* flags, cudaStream_t s) {
    if (cap == 0) return RELCP_OK;
    note_launch();
    launch_pdl(flag_le_kernel, dim3(nb(cap)), dim3(kT), 0, s, cap, np_dev, phi, thr, flags);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}
relcp_status rows_launch(const RowsArgs& a, cudaStream_t s) {
    if (a.npairs == 0) return RELCP_OK;
    note_launch();
    launch_pdl(rows_kernel, dim3(nb(a.npairs)), dim3(kT), 0, s, a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}
relcp_status trial_launch(const TrialArgs& a, cudaStream_t s) {
    if (a.n == 0) return RELCP_OK;
    note_launch();
    launch_pdl(trial_kernel, dim3(nb(a.n)), dim3(kT), 0, s, a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}
relcp_status accept_launch(const AcceptArgs& a, cudaStream_t s) {
    if (a.n == 0) return RELCP_OK;
    note_launch();
    launch_pdl(accept_kernel, dim3(nb(a.n)), dim3(kT), 0, s, a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}
relcp_status reuse_launch(const ReuseArgs& a, cudaStream_t s) {
    if (a.npairs == 0) return RELCP_OK;
    note_launch();
    launch_pdl(reuse_kernel, dim3(nb(a.npairs)), dim3(kT), 0, s, a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}
relcp_status memo_save_launch(const MemoSaveArgs& a, cudaStream_t s) {
    if (a.npairs == 0) return RELCP_OK;
    note_launch();
    launch_pdl(memo_save_kernel, dim3(nb(a.npairs)), dim3(kT), 0, s, a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

__global__ void load_bodies_kernel(LoadArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int ch = 0;
    if (i < a.n) {
        const double* r = a.stage + 22 * i;
        const int64_t n = a.n;
        auto put = [&](double* dst, int k, double v, int bit) {
            if (a.compare && __double_as_longlong(dst[k * n + i]) != __double_as_longlong(v)) ch |= bit;
            dst[k * n + i] = v;
        };
        for (int k = 0; k < 3; ++k) put(a.x, k, step_math::wrap_coord(r[k], a.box[k]), 1);
        for (int k = 0; k < 4; ++k) put(a.q, k, r[3 + k], 1);
        for (int k = 0; k < 3; ++k) put(a.axes, k, r[7 + k], 2);
        for (int k = 0; k < 6; ++k) put(a.vel, k, r[10 + k], 1);
        for (int k = 0; k < 6; ++k) put(a.fext, k, r[16 + k], 1);
    }
    if (a.compare) {
        for (int o = 16; o > 0; o >>= 1) ch |= __shfl_xor_sync(0xffffffffu, ch, o);
        if ((threadIdx.x & 31) == 0 && ch) atomicOr(a.changed, ch);
    }
}

__global__ void store_bodies_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ q,
                                    const double* __restrict__ vel, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double* r = out + 13 * i;
    if (x)
        for (int k = 0; k < 3; ++k) r[k] = x[k * n + i];
    if (q)
        for (int k = 0; k < 4; ++k) r[3 + k] = q[k * n + i];
    if (vel)
        for (int k = 0; k < 6; ++k) r[7 + k] = vel[k * n + i];
}

__global__ void check_bodies_kernel(CheckArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bad = 0, ch = 0;
    double amax = 0.0;
    if (i < a.n) {
        const int64_t n = a.n;
        double x[3], q[4], ax[3], v[6], f[6];
        for (int k = 0; k < 3; ++k) {
            x[k] = a.in.x[3 * i + k];
            ax[k] = a.in.axes[3 * i + k];
        }
        for (int k = 0; k < 4; ++k) q[k] = a.in.q[4 * i + k];
        for (int k = 0; k < 6; ++k) {
            v[k] = a.in.vel ? a.in.vel[6 * i + k] : 0.0;
            f[k] = a.in.fext ? a.in.fext[6 * i + k] : 0.0;
        }
        const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
        if (!(fabs(sqrt(qq) - 1.0) <= 1e-6)) bad |= 1;
        for (int k = 0; k < 3; ++k) {
            if (!isfinite(x[k])) bad |= 2;
            if (!(ax[k] > 0) || !isfinite(ax[k])) bad |= 4;
            amax = fmax(amax, ax[k]);
        }
        for (int k = 0; k < 6; ++k)
            if (!isfinite(v[k]) || !isfinite(f[k])) bad |= 8;
        double* r = a.stage + 22 * i;
        for (int k = 0; k < 3; ++k) {
            r[k] = x[k];
            r[7 + k] = ax[k];
        }
        for (int k = 0; k < 4; ++k) r[3 + k] = q[k];
        for (int k = 0; k < 6; ++k) {
            r[10 + k] = v[k];
            r[16 + k] = f[k];
        }
        if (a.compare && !bad) {
            auto diff = [](double u, double w) { return __double_as_longlong(u) != __double_as_longlong(w); };
            for (int k = 0; k < 3; ++k)
                if (diff(a.x[k * n + i], step_math::wrap_coord(x[k], a.box[k]))) ch |= 1;
            for (int k = 0; k < 4; ++k)
                if (diff(a.q[k * n + i], q[k])) ch |= 1;
            for (int k = 0; k < 3; ++k)
                if (diff(a.axes[k * n + i], ax[k])) ch |= 2;
            for (int k = 0; k < 6; ++k)
                if (diff(a.vel[k * n + i], v[k]) || diff(a.fext[k * n + i], f[k])) ch |= 1;
        }
        if (bad) atomicMin(&a.out->bad_key, ((unsigned long long)i << 4) | (unsigned long long)bad);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ch |= __shfl_xor_sync(0xffffffffu, ch, o);
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (ch) atomicOr(&a.out->changed, ch);
        if (amax > 0.0) atomicMax(&a.out->rbmax_bits, (unsigned long long)__double_as_longlong(amax));
    }
}

__global__ void store_direct_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ q,
                                    const double* __restrict__ vel, double* ox, double* oq, double* ov) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (ox)
        for (int k = 0; k < 3; ++k) ox[3 * i + k] = x[k * n + i];
    if (oq)
        for (int k = 0; k < 4; ++k) oq[4 * i + k] = q[k * n + i];
    if (ov)
        for (int k = 0; k < 6; ++k) ov[6 * i + k] = vel[k * n + i];
}

relcp_status check_bodies_launch(const CheckArgs& a, cudaStream_t s) {
    if (a.n == 0) return RELCP_OK;
    note_launch();
    check_bodies_kernel<<<nb(a.n), kT, 0, s>>>(a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status store_direct_launch(int64_t n, const double* x, const double* q, const double* vel, double* ox,
                                 double* oq, double* ov, cudaStream_t s) {
    if (n == 0) return RELCP_OK;
    note_launch();
    store_direct_kernel<<<nb(n), kT, 0, s>>>(n, x, q, vel, ox, oq, ov);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status load_bodies_launch(const LoadArgs& a, cudaStream_t s) {
    if (a.n == 0) return RELCP_OK;
    note_launch();
    load_bodies_kernel<<<nb(a.n), kT, 0, s>>>(a);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}

relcp_status store_bodies_launch(int64_t n, const double* x, const double* q, const double* vel, double* out,
                                 cudaStream_t s) {
    if (n == 0) return RELCP_OK;
    note_launch();
    store_bodies_kernel<<<nb(n), kT, 0, s>>>(n, x, q, vel, out);
    RELCP_CUDA(cudaGetLastError());
    return RELCP_OK;
}


}  // namespace relcp
