// Per-body and per-row arithmetic of one ReLCP time step (Algorithm 1),
// shared by the single-scene kernels (step_kernels.cu) and the batched-scene
// step (batched.cu), so both compute the same values the same way.
#pragma once

#include "relcp_internal.cuh"

namespace relcp {
namespace step_math {

// prep of one body at C^k: normalised q, P = R diag(a^2) R^T, the body
// operator K = (kt, Kr) (overdamped: the local-drag mobility
// (1/xi) diag(I/L, 12 I/L^3), L = twice the largest semi-axis; inertial:
// dt M^-1 with m = 4/3 pi abc rho and I_body = m/5 (b^2+c^2, a^2+c^2, a^2+b^2)
// rotated to the world frame), bounding radius, and U_free = vel + K F_ext
// (+ the affine background velocity strain_rate (x - L/2) on periodic axes).
// K[0] = kt, K[1..6] = Kr (xx, yy, zz, xy, xz, yz).
struct BodyPrep {
    double q[4];
    Sym3<double> P;
    double K[7];
    double rb;
    double ufree[6];
};

// planar dynamics (RELCP_OVERDAMPED_2D): only u_x, u_y and omega_z
template <class T>
__device__ __forceinline__ void planar_velocity(T u[6]) {
    u[2] = T(0);
    u[3] = T(0);
    u[4] = T(0);
}
// a row of the planar problem keeps its entries on u_x, u_y and omega_z
template <class T>
__device__ __forceinline__ void planar_row(T nn[3], T ta[3], T tb[3]) {
    nn[2] = T(0);
    ta[0] = ta[1] = T(0);
    tb[0] = tb[1] = T(0);
}

// The per-body shape record the SNSD kernels read (six doubles).  Ellipsoid:
// P = R diag(a^2) R^T.  Spherocylinder (semi-axes (h + rho, rho, rho)): the
// unit axis u = R e_x, then h and rho, then 0.
__device__ __forceinline__ Sym3<double> shape_record(const double R[9], const double ax[3], int shape) {
    if (shape == RELCP_SHAPE_SPHEROCYLINDER) {
        const double rho = ax[1];
        const double h = ax[0] > rho ? ax[0] - rho : 0.0;
        return Sym3<double>{R[0], R[3], R[6], h, rho, 0.0};
    }
    return rot_diag_rot(R, ax[0] * ax[0], ax[1] * ax[1], ax[2] * ax[2]);
}

__device__ __forceinline__ void prep_body(const double qin[4], const double ax[3], const double vel[6],
                                          const double fext[6], const double x[3], int dynamics, double dt,
                                          double drag_xi, double density, double strain_rate, const double box[3],
                                          BodyPrep& b, int shape = RELCP_SHAPE_ELLIPSOID) {
    double s = qin[0], x1 = qin[1], y1 = qin[2], z1 = qin[3];
    // one FP64 reciprocal square root (no separate division), four products
    const double il = rsqrt(s * s + x1 * x1 + y1 * y1 + z1 * z1);
    s *= il;
    x1 *= il;
    y1 *= il;
    z1 *= il;
    b.q[0] = s;
    b.q[1] = x1;
    b.q[2] = y1;
    b.q[3] = z1;
    double R[9];
    quat_to_R(s, x1, y1, z1, R);
    const double a0 = ax[0], a1 = ax[1], a2 = ax[2];
    b.P = shape_record(R, ax, shape);
    const double amax = fmax(a0, fmax(a1, a2));
    b.rb = amax;
    double kt;
    Sym3<double> Kr;
    if (dynamics == RELCP_OVERDAMPED || dynamics == RELCP_OVERDAMPED_2D) {
        const double L = 2.0 * amax;
        kt = 1.0 / (drag_xi * L);
        const double kr = 12.0 / (drag_xi * L * L * L);
        Kr = Sym3<double>{kr, kr, kr, 0.0, 0.0, 0.0};
    } else {
        const double pi = 3.14159265358979323846;
        const double m = density * 4.0 / 3.0 * pi * a0 * a1 * a2;
        const double I0 = m / 5.0 * (a1 * a1 + a2 * a2), I1 = m / 5.0 * (a0 * a0 + a2 * a2),
                     I2 = m / 5.0 * (a0 * a0 + a1 * a1);
        kt = dt / m;
        Kr = rot_diag_rot(R, dt / I0, dt / I1, dt / I2);
    }
    b.K[0] = kt;
    b.K[1] = Kr.xx;
    b.K[2] = Kr.yy;
    b.K[3] = Kr.zz;
    b.K[4] = Kr.xy;
    b.K[5] = Kr.xz;
    b.K[6] = Kr.yz;
    double u[6];
    for (int k = 0; k < 6; ++k) u[k] = vel[k];
    u[0] += kt * fext[0];
    u[1] += kt * fext[1];
    u[2] += kt * fext[2];
    u[3] += Kr.xx * fext[3] + Kr.xy * fext[4] + Kr.xz * fext[5];
    u[4] += Kr.xy * fext[3] + Kr.yy * fext[4] + Kr.yz * fext[5];
    u[5] += Kr.xz * fext[3] + Kr.yz * fext[4] + Kr.zz * fext[5];
    if (strain_rate != 0.0)
        for (int k = 0; k < 3; ++k)
            if (box[k] > 0.0) u[k] += strain_rate * (x[k] - 0.5 * box[k]);
    if (dynamics == RELCP_OVERDAMPED_2D) planar_velocity(u);
    for (int k = 0; k < 6; ++k) b.ufree[k] = u[k];
}

// Jacobian row of a pair, [-n, -(r_a x n), n, (r_b x n)]: returns ta = r_a x n
// and tb = r_b x n
__device__ __forceinline__ void row_torques(const double nn[3], const double ra[3], const double rb[3], double ta[3],
                                            double tb[3]) {
    cross3(ra, nn, ta);
    cross3(rb, nn, tb);
}

// d^T U for the row: n.(U_j - U_i) + tb.w_j - ta.w_i
__device__ __forceinline__ double row_rate(const double Ui[6], const double Uj[6], const double nn[3],
                                           const double ta[3], const double tb[3]) {
    double r = 0.0;
    for (int k = 0; k < 3; ++k) r += nn[k] * (Uj[k] - Ui[k]);
    for (int k = 0; k < 3; ++k) r += tb[k] * Uj[3 + k] - ta[k] * Ui[3 + k];
    return r;
}

// A_aa / c = d^T K d
__device__ __forceinline__ double row_dKd(const double Ki[7], const double Kj[7], const double nn[3],
                                          const double ta[3], const double tb[3]) {
    double acc = (Ki[0] + Kj[0]) * (nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    for (int side = 0; side < 2; ++side) {
        const double* K = side ? Kj : Ki;
        const double* t = side ? tb : ta;
        const double kxx = K[1], kyy = K[2], kzz = K[3], kxy = K[4], kxz = K[5], kyz = K[6];
        acc += t[0] * (kxx * t[0] + kxy * t[1] + kxz * t[2]) + t[1] * (kxy * t[0] + kyy * t[1] + kyz * t[2]) +
               t[2] * (kxz * t[0] + kyz * t[1] + kzz * t[2]);
    }
    return acc;
}

// n . (min_image(x_j - x_i) - (x_j - x_i)): the background-velocity correction
// of a pair that interacts across the periodic boundary
__device__ __forceinline__ double affine_image_corr(const double xi[3], const double xj[3], const double nn[3],
                                                    const double box[3]) {
    double corr = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double raw = xj[k] - xi[k];
        corr += nn[k] * (min_image(raw, box[k]) - raw);
    }
    return corr;
}

// trial configuration of one body: x + dt v, q + dt/2 (0, w) (x) q normalised,
// and P at the new orientation
__device__ __forceinline__ void trial_body(const double x[3], const double q[4], const double U[6], const double ax[3],
                                           double dt, double xt[3], double qt[4], Sym3<double>& Pt,
                                           int shape = RELCP_SHAPE_ELLIPSOID) {
    for (int k = 0; k < 3; ++k) xt[k] = x[k] + dt * U[k];
    const double s = q[0], x1 = q[1], y1 = q[2], z1 = q[3];
    const double h = 0.5 * dt;
    const double w0 = U[3], w1 = U[4], w2 = U[5];
    double ns = s - h * (w0 * x1 + w1 * y1 + w2 * z1);
    double nx = x1 + h * (s * w0 + (w1 * z1 - w2 * y1));
    double ny = y1 + h * (s * w1 + (w2 * x1 - w0 * z1));
    double nz = z1 + h * (s * w2 + (w0 * y1 - w1 * x1));
    const double il = rsqrt(ns * ns + nx * nx + ny * ny + nz * nz);
    ns *= il;
    nx *= il;
    ny *= il;
    nz *= il;
    qt[0] = ns;
    qt[1] = nx;
    qt[2] = ny;
    qt[3] = nz;
    double R[9];
    quat_to_R(ns, nx, ny, nz, R);
    Pt = shape_record(R, ax, shape);
}

// position wrapped into [0, L) on a periodic axis
// (v itself when already inside, without the division)
__device__ __forceinline__ double wrap_coord(double v, double L) {
    if (!(L > 0.0) || (v >= 0.0 && v < L)) return v;
    return v - L * floor(v / L);
}

}  // namespace step_math
}  // namespace relcp
