// SNSD of one ellipsoid pair: the signed distance Phi = max over unit n of
//     G(n) = n.d - sqrt(n.Pa n) - sqrt(n.Pb n)
// by Newton ascent on the sphere (see snsd.cu for the derivation), with the
// shared normal and the lever arms.  Device functions shared by the
// per-pair SNSD kernel and the batched-scene step.
#pragma once

#include "relcp_internal.cuh"

namespace relcp {
namespace snsd_math {

template <class T>
struct Tol;
template <>
struct Tol<double> {
    static constexpr double grad = 1e-13;   // tangent-gradient stop, x (1 + |d|)
    static constexpr double drop = 1e-15;   // admissible G decrease per step from rounding
    static constexpr double kappa = 1e-6;
};
template <>
struct Tol<float> {
    static constexpr float grad = 2e-6f;
    static constexpr float drop = 1e-6f;
    static constexpr float kappa = 1e-4f;
};

template <class T>
__device__ __forceinline__ T g_value(const T* n, const T* d, const Sym3<T>& Pa, const Sym3<T>& Pb) {
    T va[3], vb[3];
    symv(Pa, n, va);
    symv(Pb, n, vb);
    return dot3(n, d) - sqrt(dot3(n, va)) - sqrt(dot3(n, vb));
}

template <class T>
__device__ __forceinline__ void normalize3(T* v) {
    T l = sqrt(dot3(v, v));
    v[0] /= l;
    v[1] /= l;
    v[2] /= l;
}

template <class T>
__device__ __forceinline__ void tangent_basis(const T* n, T* t1, T* t2) {
    T ax = fabs(n[0]), ay = fabs(n[1]), az = fabs(n[2]);
    T e0 = 0, e1 = 0, e2 = 0;
    if (ax <= ay && ax <= az) e0 = 1;
    else if (ay <= az) e1 = 1;
    else e2 = 1;
    T en = e0 * n[0] + e1 * n[1] + e2 * n[2];
    t1[0] = e0 - en * n[0];
    t1[1] = e1 - en * n[1];
    t1[2] = e2 - en * n[2];
    normalize3(t1);
    cross3(n, t1, t2);
}

// adj(P) v  (P symmetric positive definite: same direction as P^-1 v)
template <class T>
__device__ __forceinline__ void adj_solve(const Sym3<T>& P, const T* v, T* o) {
    T A00 = P.yy * P.zz - P.yz * P.yz, A11 = P.xx * P.zz - P.xz * P.xz, A22 = P.xx * P.yy - P.xy * P.xy;
    T A01 = P.xz * P.yz - P.xy * P.zz, A02 = P.xy * P.yz - P.yy * P.xz, A12 = P.xy * P.xz - P.xx * P.yz;
    o[0] = A00 * v[0] + A01 * v[1] + A02 * v[2];
    o[1] = A01 * v[0] + A11 * v[1] + A12 * v[2];
    o[2] = A02 * v[0] + A12 * v[1] + A22 * v[2];
}

template <class T>
__device__ void cold_start(const T* d, const Sym3<T>& Pa, const Sym3<T>& Pb, T* n) {
    T l = sqrt(dot3(d, d));
    n[0] = 1;
    n[1] = 0;
    n[2] = 0;
    if (!(l > 0)) return;
    const Sym3<T> S{Pa.xx + Pb.xx, Pa.yy + Pb.yy, Pa.zz + Pb.zz, Pa.xy + Pb.xy, Pa.xz + Pb.xz, Pa.yz + Pb.yz};
    T best = -INFINITY;
    // seeds d, Pa^-1 d, Pb^-1 d, (Pa + Pb)^-1 d, each normalised; the best G wins
    // (unrolled: the candidate stays in registers)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        T v[3];
        if (c == 0) {
            v[0] = d[0];
            v[1] = d[1];
            v[2] = d[2];
        } else {
            adj_solve(c == 1 ? Pa : (c == 2 ? Pb : S), d, v);
        }
        const T lc = sqrt(dot3(v, v));
        if (!(lc > 0)) continue;
        for (int k = 0; k < 3; ++k) v[k] /= lc;
        const T g = g_value(v, d, Pa, Pb);
        if (g > best) {
            best = g;
            n[0] = v[0];
            n[1] = v[1];
            n[2] = v[2];
        }
    }
}

// Newton ascent of G on the unit sphere from n (updated in place).
// Returns the iteration count when the tangent gradient falls to tol, or
// -(count+1) otherwise.  *Gout = G at the returned n.  tol_mult scales the
// stop (0: take maxit steps whatever the gradient).
template <class T>
__device__ int newton_sphere(T* n, const T* d, const Sym3<T>& Pa, const Sym3<T>& Pb, T scale, int maxit, T* Gout,
                             T tol_mult = T(1)) {
    const T tol = Tol<T>::grad * scale * tol_mult;
    const T gfloor = Tol<T>::drop * scale;
    const T kappa = Tol<T>::kappa * scale;
    T G = 0;
    int it;
    for (it = 0; it < maxit; ++it) {
        T va[3], vb[3];
        symv(Pa, n, va);
        symv(Pb, n, vb);
        T sa = sqrt(dot3(n, va)), sb = sqrt(dot3(n, vb));
        G = dot3(n, d) - sa - sb;
        T t1[3], t2[3];
        tangent_basis(n, t1, t2);
        T Pa1[3], Pa2[3], Pb1[3], Pb2[3];
        symv(Pa, t1, Pa1);
        symv(Pa, t2, Pa2);
        symv(Pb, t1, Pb1);
        symv(Pb, t2, Pb2);
        T ia = T(1) / sa, ib = T(1) / sb;
        T a1 = dot3(n, Pa1), a2 = dot3(n, Pa2);
        T b1 = dot3(n, Pb1), b2 = dot3(n, Pb2);
        T g1 = dot3(t1, d) - a1 * ia - b1 * ib;
        T g2 = dot3(t2, d) - a2 * ia - b2 * ib;
        T gn = sqrt(g1 * g1 + g2 * g2);
        if (gn <= tol) {
            *Gout = G;
            return it;
        }
        T ia3 = ia * ia * ia, ib3 = ib * ib * ib;
        T h11 = -(dot3(t1, Pa1) * ia - a1 * a1 * ia3) - (dot3(t1, Pb1) * ib - b1 * b1 * ib3) - G;
        T h22 = -(dot3(t2, Pa2) * ia - a2 * a2 * ia3) - (dot3(t2, Pb2) * ib - b2 * b2 * ib3) - G;
        T h12 = -(dot3(t1, Pa2) * ia - a1 * a2 * ia3) - (dot3(t1, Pb2) * ib - b1 * b2 * ib3);
        T tr = T(0.5) * (h11 + h22), df = T(0.5) * (h11 - h22);
        T lmax = tr + sqrt(df * df + h12 * h12);
        if (lmax > -kappa) {
            T sh = lmax + kappa;
            h11 -= sh;
            h22 -= sh;
        }
        T det = h11 * h22 - h12 * h12;
        T d1 = -(h22 * g1 - h12 * g2) / det;
        T d2 = -(-h12 * g1 + h11 * g2) / det;
        T step = 1;
        bool acc = false;
        for (int bt = 0; bt < 40; ++bt) {
            T m[3];
            for (int k = 0; k < 3; ++k) m[k] = n[k] + step * (d1 * t1[k] + d2 * t2[k]);
            normalize3(m);
            T Gm = g_value(m, d, Pa, Pb);
            if (Gm >= G - gfloor) {
                n[0] = m[0];
                n[1] = m[1];
                n[2] = m[2];
                acc = true;
                break;
            }
            step *= T(0.5);
        }
        if (!acc) break;
    }
    *Gout = G;
    return -(it + 1);
}

// Result of one pair: Phi, the shared normal n (a -> b), the lever arms
// r_a = Pa n / sqrt(n.Pa n) and r_b = -Pb n / sqrt(n.Pb n) (support points
// relative to the centres), the Newton iteration count (negative: not
// converged) and ok = converged.
struct PairResult {
    double phi;
    double n[3], ra[3], rb[3];
    int iters;
    bool ok;
};

// d = c_b - c_a (minimum image); with has_guess the start normal is
// (g0, g1, g2) when its length is in (0.5, 2), else the cold start; mixed:
// FP32 iterations + FP64 polish, else FP64 throughout
__device__ __forceinline__ void snsd_pair(const double d[3], const Sym3<double>& Pa, const Sym3<double>& Pb,
                                          bool has_guess, double g0, double g1, double g2, bool mixed,
                                          PairResult& o, int cap = 0) {
    // cap > 0 bounds every Newton phase (fault injection: RELCP_FAULT_NEWTON_ITERS)
    const int cap32 = cap > 0 ? cap : 30, cap64 = cap > 0 ? cap : 50;
    double n[3];
    int iters = 0;
    double G = 0.0;
    int r;
    double va[3], vb[3], sa, sb;
    float raf[3], rbf[3];
    bool arms_f = false;  // lever arms from the FP32 phase
    if (mixed) {
        // FP32 iterations.  FP64 runs at a small fraction of the FP32 rate
        // on this part, so everything but the polish (G in FP64 at the FP32
        // maximiser) stays in FP32: the start, the Newton steps, the scale
        // of the stopping test and the lever arms.
        float df[3] = {(float)d[0], (float)d[1], (float)d[2]};
        Sym3<float> Pfa{(float)Pa.xx, (float)Pa.yy, (float)Pa.zz, (float)Pa.xy, (float)Pa.xz, (float)Pa.yz};
        Sym3<float> Pfb{(float)Pb.xx, (float)Pb.yy, (float)Pb.zz, (float)Pb.xy, (float)Pb.xz, (float)Pb.yz};
        const float scalef = 1.f + sqrtf(dot3(df, df));
        float nf[3];
        bool have = false;
        if (has_guess) {
            nf[0] = (float)g0;
            nf[1] = (float)g1;
            nf[2] = (float)g2;
            const float l = sqrtf(dot3(nf, nf));
            if (l > 0.5f && l < 2.f) {
                normalize3(nf);
                have = true;
            }
        }
        if (!have) cold_start(df, Pfa, Pfb, nf);
        float Gf;
        int rf = newton_sphere(nf, df, Pfa, Pfb, scalef, cap32, &Gf);
        iters = rf >= 0 ? rf : -rf;
        // one more FP32 Newton step past the stop: the stop leaves the normal
        // within ~2e-6 (1 + |d|) / |H| of the maximiser, one step takes it to
        // the FP32 rounding level (~1e-7), and the rows built from it (normal,
        // lever arms) perturb the LCP that much less
        if (rf >= 0) newton_sphere(nf, df, Pfa, Pfb, scalef, 1, &Gf, 0.f);
        n[0] = nf[0];
        n[1] = nf[1];
        n[2] = nf[2];
        const double e = dot3(n, n) - 1.0;
        if (rf >= 0 && fabs(e) < 1e-4) {
            // FP64 polish.  At the FP32 maximiser the tangent gradient is
            // below 2e-6 (1 + |d|), so by stationarity G evaluated there in
            // FP64 is within O(1e-12) of the maximum: that evaluation (below)
            // is the polish.  n is brought to unit length in FP64 with
            // 1/sqrt(1 + e) = 1 - e/2 + 3e^2/8 + O(e^3), exact to rounding
            // for |e| ~ 1e-7 (FP32 normalisation).
            const double f = 1.0 + e * (-0.5 + 0.375 * e);
            n[0] *= f;
            n[1] *= f;
            n[2] *= f;
            r = 0;
            float vaf[3], vbf[3];
            symv(Pfa, nf, vaf);
            symv(Pfb, nf, vbf);
            const float ia = 1.f / sqrtf(dot3(nf, vaf)), ib = 1.f / sqrtf(dot3(nf, vbf));
            for (int k = 0; k < 3; ++k) {
                raf[k] = vaf[k] * ia;
                rbf[k] = -vbf[k] * ib;
            }
            arms_f = true;
        } else {
            // the FP32 phase failed: FP64 Newton from its last iterate
            normalize3(n);
            const double scale = 1.0 + sqrt(dot3(d, d));
            r = newton_sphere(n, d, Pa, Pb, scale, cap64, &G);
        }
    } else {
        const double scale = 1.0 + sqrt(dot3(d, d));
        bool have = false;
        if (has_guess) {
            n[0] = g0;
            n[1] = g1;
            n[2] = g2;
            const double l = sqrt(dot3(n, n));
            if (l > 0.5 && l < 2.0) {
                normalize3(n);
                have = true;
            }
        }
        if (!have) cold_start(d, Pa, Pb, n);
        r = newton_sphere(n, d, Pa, Pb, scale, cap64, &G);
    }
    o.ok = r >= 0;
    if (r < 0) iters = -(iters + (-r));
    else iters += r;
    symv(Pa, n, va);
    symv(Pb, n, vb);
    sa = sqrt(dot3(n, va));
    sb = sqrt(dot3(n, vb));
    G = dot3(n, d) - sa - sb;
    o.phi = G;
    if (arms_f) {
        for (int k = 0; k < 3; ++k) {
            o.n[k] = n[k];
            o.ra[k] = (double)raf[k];
            o.rb[k] = (double)rbf[k];
        }
    } else {
        const double ia = 1.0 / sa, ib = 1.0 / sb;
        for (int k = 0; k < 3; ++k) {
            o.n[k] = n[k];
            o.ra[k] = va[k] * ia;
            o.rb[k] = -vb[k] * ib;
        }
    }
    o.iters = iters;
}

// Spherocylinder pair (RELCP_SHAPE_SPHEROCYLINDER records: unit axis u, half-
// length h, radius rho).  The closest points A + s u, B + t v of the two
// segments (B - A = d) minimise |d + t v - s u|^2 over the rectangle; the
// minimiser is the first minimal one among the interior stationary point
// (when it lies inside) and the edge minimisers at s = -h_a, +h_a, t = -h_b,
// +h_b.  Phi = |Q - P| - rho_a - rho_b, n = (Q - P)/|Q - P|, support points
// P + rho_a n and Q - rho_b n.  FP64 in closed form on both precision paths
// (no iteration); intersecting segments give ok = false.
__device__ __forceinline__ void capsule_pair(const double d[3], const Sym3<double>& A, const Sym3<double>& B,
                                             PairResult& o) {
    const double u[3] = {A.xx, A.yy, A.zz}, v[3] = {B.xx, B.yy, B.zz};
    const double ha = A.xy, ra = A.xz, hb = B.xy, rb = B.xz;
    const double uv = dot3(u, v), wu = dot3(d, u), wv = dot3(d, v);
    double best_s = 0.0, best_t = 0.0, best_f = 0.0;
    bool have = false;
    auto consider = [&](double s_, double t_) {
        double r[3];
        for (int k = 0; k < 3; ++k) r[k] = d[k] + t_ * v[k] - s_ * u[k];
        const double f = dot3(r, r);
        if (!have || f < best_f) {
            best_s = s_;
            best_t = t_;
            best_f = f;
            have = true;
        }
    };
    const double det = 1.0 - uv * uv;
    if (det > 1e-14) {
        const double s0 = (wu - uv * wv) / det, t0 = (uv * wu - wv) / det;
        if (fabs(s0) <= ha && fabs(t0) <= hb) consider(s0, t0);
    }
    consider(-ha, fmin(fmax(-ha * uv - wv, -hb), hb));
    consider(ha, fmin(fmax(ha * uv - wv, -hb), hb));
    consider(fmin(fmax(wu - hb * uv, -ha), ha), -hb);
    consider(fmin(fmax(wu + hb * uv, -ha), ha), hb);
    double w[3];
    for (int k = 0; k < 3; ++k) w[k] = d[k] + best_t * v[k] - best_s * u[k];
    const double dist = sqrt(dot3(w, w));
    o.iters = 0;
    if (!(dist > 1e-12)) {
        o.ok = false;
        o.phi = -(ra + rb);
        for (int k = 0; k < 3; ++k) o.n[k] = o.ra[k] = o.rb[k] = 0.0;
        return;
    }
    o.ok = true;
    o.phi = dist - ra - rb;
    for (int k = 0; k < 3; ++k) {
        const double nk = w[k] / dist;
        o.n[k] = nk;
        o.ra[k] = best_s * u[k] + ra * nk;
        o.rb[k] = best_t * v[k] - rb * nk;
    }
}

}  // namespace snsd_math
}  // namespace relcp
