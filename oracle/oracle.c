/*
 * ReLCP oracle, numerical core: plain, single-threaded FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library; it is written from the paper ("Smooth-Rigid-Body Contact as a
 * ReLCP", arXiv 2506.14097) and from textbook definitions.
 *
 * Compile with -ffp-contract=off: every threshold decision (candidate pairs)
 * is a sequence of separately rounded IEEE operations.
 *
 * Contents
 *   orc_pairs       candidate pairs by brute force (all i<j), periodic
 *                   minimum image (the "near-contacting pairs" of Sec. 3.1,
 *                   Algorithm 1 initialisation).
 *   orc_snsd        shared-normal signed distance of two ellipsoids
 *                   (Sec. 2.1.4 surface points with n_a = -n_b; Lemma
 *                   "uniform interior tangent ball": y_b - y_a = Phi n),
 *                   by multi-start damped Riemannian Newton on the unit sphere.
 *   orc_lemke       Lemke's complementary pivoting for 0 <= Mz + q _|_ z >= 0
 *                   (the LCP of Eq. cqpp / Lemma "LCP <=> CQP"), covering
 *                   vector e, lexicographic ratio test, basis re-solve polish.
 *
 * Conventions (shared with the paper's notation, Sec. 2.1.1):
 *   quaternion q = (s, w1, w2, w3), Hamilton product, R(q) maps body to world;
 *   ellipsoid E = { c + R S u : |u| <= 1 }, S = diag(semi-axes);
 *   P = R S^2 R^T ("shape matrix"); support function h(n) = n.c + sqrt(n.P n).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* small vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void matvec3(const double* M, const double* v, double* o) {
    o[0] = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
    o[1] = M[3] * v[0] + M[4] * v[1] + M[5] * v[2];
    o[2] = M[6] * v[0] + M[7] * v[1] + M[8] * v[2];
}

/* Rotation matrix of the normalised quaternion (s, w), Hamilton convention,
 * body -> world (Sec. 2.1.1: orientation as a unit quaternion). */
void orc_quat_rot(const double* qin, double* R) {
    double nq = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    double s = qin[0] / nq, x = qin[1] / nq, y = qin[2] / nq, z = qin[3] / nq;
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

/* P = R diag(a^2) R^T */
void orc_shape_matrix(const double* q, const double* ax, double* P) {
    double R[9];
    orc_quat_rot(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * ax[k] * ax[k] * R[3 * j + k];
            P[3 * i + j] = acc;
        }
}

/* Periodic minimum image of one component; L <= 0 means not periodic. */
static double min_image(double dx, double L) {
    if (L > 0.0) {
        double k = rint(dx / L); /* round half to even */
        double t = L * k;
        dx = dx - t;
    }
    return dx;
}

/* ------------------------------------------------------------------ */
/* O1: candidate pairs                                                  */
/* ------------------------------------------------------------------ */
/*
 * All pairs i<j whose bounding spheres, grown by `skin`, overlap:
 *   |min_image(x_j - x_i)|^2 <= (rb_i + rb_j + skin)^2,
 * with the squared length summed as ((dx*dx + dy*dy) + dz*dz) and the cutoff
 * as ((rb_i + rb_j) + skin)^2, every operation rounded separately.
 * Output is i-major, j ascending.  Returns the number of pairs (which may
 * exceed cap: then only the first cap are written).
 */
int64_t orc_pairs(int64_t n, const double* x, const double* rb, const double* box, double skin,
                  int32_t* pairs, int64_t cap) {
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = min_image(x[3 * j + 0] - x[3 * i + 0], box[0]);
            double dy = min_image(x[3 * j + 1] - x[3 * i + 1], box[1]);
            double dz = min_image(x[3 * j + 2] - x[3 * i + 2], box[2]);
            double xx = dx * dx;
            double yy = dy * dy;
            double zz = dz * dz;
            double d2 = xx + yy;
            d2 = d2 + zz;
            double s = rb[i] + rb[j];
            s = s + skin;
            double c2 = s * s;
            if (d2 <= c2) {
                if (np < cap) {
                    pairs[2 * np + 0] = (int32_t)i;
                    pairs[2 * np + 1] = (int32_t)j;
                }
                ++np;
            }
        }
    }
    return np;
}

/* Same decision for one pair, returning also the margin d2 - c2 (used by the
 * tests to flag pairs whose decision sits on the threshold). */
double orc_pair_margin(const double* xi, const double* xj, double rbi, double rbj, const double* box, double skin) {
    double dx = min_image(xj[0] - xi[0], box[0]);
    double dy = min_image(xj[1] - xi[1], box[1]);
    double dz = min_image(xj[2] - xi[2], box[2]);
    double xx = dx * dx;
    double yy = dy * dy;
    double zz = dz * dz;
    double d2 = xx + yy;
    d2 = d2 + zz;
    double s = rbi + rbj;
    s = s + skin;
    return d2 - s * s;
}

/* ------------------------------------------------------------------ */
/* O2: shared-normal signed distance                                    */
/* ------------------------------------------------------------------ */
/*
 * For unit n (pointing from a to b) the gap between the slabs that contain
 * the two ellipsoids is
 *     G(n) = n.d - sqrt(n.Pa n) - sqrt(n.Pb n),     d = c_b - c_a,
 * and its gradient is  d - Pa n/|.| - Pb n/|.| = y_b(n) - y_a(n)  with the
 * support points y_a = c_a + Pa n/sqrt(n.Pa n), y_b = c_b - Pb n/sqrt(n.Pb n).
 * A stationary point of G on the unit sphere is therefore a pair of surface
 * points with opposite normals whose difference is parallel to n (Sec. 2.1.4,
 * n_a = -n_b; y_b - y_a = Phi n of the interior tangent-ball lemma), and the
 * signed distance is the maximum:  Phi = max_{|n|=1} G(n).  For separated
 * bodies this is the Euclidean distance, for overlapping bodies it is minus
 * the penetration depth.
 */
typedef struct {
    double G;
    double grad[3];
    double H[9];
    double va[3], vb[3];
    double sa, sb;
} gval_t;

static void G_full(const double* n, const double* d, const double* Pa, const double* Pb, gval_t* o) {
    matvec3(Pa, n, o->va);
    matvec3(Pb, n, o->vb);
    o->sa = sqrt(dot3(n, o->va));
    o->sb = sqrt(dot3(n, o->vb));
    o->G = dot3(n, d) - o->sa - o->sb;
    for (int i = 0; i < 3; ++i) o->grad[i] = d[i] - o->va[i] / o->sa - o->vb[i] / o->sb;
    double ia = 1.0 / o->sa, ib = 1.0 / o->sb;
    double ia3 = ia * ia * ia, ib3 = ib * ib * ib;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            o->H[3 * i + j] = -(Pa[3 * i + j] * ia - o->va[i] * o->va[j] * ia3) -
                              (Pb[3 * i + j] * ib - o->vb[i] * o->vb[j] * ib3);
}

double orc_G(const double* n, const double* d, const double* Pa, const double* Pb) {
    double va[3], vb[3];
    matvec3(Pa, n, va);
    matvec3(Pb, n, vb);
    return dot3(n, d) - sqrt(dot3(n, va)) - sqrt(dot3(n, vb));
}

static void tangent_basis(const double* n, double* t1, double* t2) {
    /* pick the coordinate axis least aligned with n */
    double ax = fabs(n[0]), ay = fabs(n[1]), az = fabs(n[2]);
    double e[3] = {0, 0, 0};
    if (ax <= ay && ax <= az) e[0] = 1;
    else if (ay <= az) e[1] = 1;
    else e[2] = 1;
    double en = dot3(e, n);
    for (int i = 0; i < 3; ++i) t1[i] = e[i] - en * n[i];
    double l = norm3(t1);
    for (int i = 0; i < 3; ++i) t1[i] /= l;
    cross3(n, t1, t2);
}

/* Icosphere directions (icosahedron subdivided three times: 642 vertices),
 * built once.  Used only as multi-start seeds. */
#define ICO_MAXV 700
static double g_ico[ICO_MAXV][3];
static int g_ico_n = 0;

static int ico_mid(int a, int b, int* em_a, int* em_b, int* em_v, int* nem, int* nv) {
    if (a > b) { int t = a; a = b; b = t; }
    for (int i = 0; i < *nem; ++i)
        if (em_a[i] == a && em_b[i] == b) return em_v[i];
    double m[3];
    for (int k = 0; k < 3; ++k) m[k] = 0.5 * (g_ico[a][k] + g_ico[b][k]);
    double l = norm3(m);
    int v = (*nv)++;
    for (int k = 0; k < 3; ++k) g_ico[v][k] = m[k] / l;
    em_a[*nem] = a; em_b[*nem] = b; em_v[*nem] = v; ++(*nem);
    return v;
}

static void ico_build(void) {
    if (g_ico_n) return;
    double t = (1.0 + sqrt(5.0)) / 2.0;
    double base[12][3] = {{-1, t, 0}, {1, t, 0}, {-1, -t, 0}, {1, -t, 0}, {0, -1, t}, {0, 1, t},
                          {0, -1, -t}, {0, 1, -t}, {t, 0, -1}, {t, 0, 1}, {-t, 0, -1}, {-t, 0, 1}};
    static const int f0[20][3] = {{0, 11, 5}, {0, 5, 1}, {0, 1, 7}, {0, 7, 10}, {0, 10, 11},
                                  {1, 5, 9}, {5, 11, 4}, {11, 10, 2}, {10, 7, 6}, {7, 1, 8},
                                  {3, 9, 4}, {3, 4, 2}, {3, 2, 6}, {3, 6, 8}, {3, 8, 9},
                                  {4, 9, 5}, {2, 4, 11}, {6, 2, 10}, {8, 6, 7}, {9, 8, 1}};
    int nv = 12;
    for (int i = 0; i < 12; ++i) {
        double l = norm3(base[i]);
        for (int k = 0; k < 3; ++k) g_ico[i][k] = base[i][k] / l;
    }
    int* faces = (int*)malloc(sizeof(int) * 3 * 1280);
    int* nf = (int*)malloc(sizeof(int) * 3 * 1280);
    int nfaces = 20;
    memcpy(faces, f0, sizeof(f0));
    int* em_a = (int*)malloc(sizeof(int) * 2000);
    int* em_b = (int*)malloc(sizeof(int) * 2000);
    int* em_v = (int*)malloc(sizeof(int) * 2000);
    for (int level = 0; level < 3; ++level) {
        int nem = 0, k = 0;
        for (int f = 0; f < nfaces; ++f) {
            int a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
            int ab = ico_mid(a, b, em_a, em_b, em_v, &nem, &nv);
            int bc = ico_mid(b, c, em_a, em_b, em_v, &nem, &nv);
            int ca = ico_mid(c, a, em_a, em_b, em_v, &nem, &nv);
            int tri[4][3] = {{a, ab, ca}, {b, bc, ab}, {c, ca, bc}, {ab, bc, ca}};
            for (int u = 0; u < 4; ++u) { nf[3 * k] = tri[u][0]; nf[3 * k + 1] = tri[u][1]; nf[3 * k + 2] = tri[u][2]; ++k; }
        }
        nfaces = k;
        memcpy(faces, nf, sizeof(int) * 3 * nfaces);
    }
    free(faces); free(nf); free(em_a); free(em_b); free(em_v);
    g_ico_n = nv;
}

int orc_icosphere(double* out) {
    ico_build();
    for (int i = 0; i < g_ico_n; ++i)
        for (int k = 0; k < 3; ++k) out[3 * i + k] = g_ico[i][k];
    return g_ico_n;
}

/*
 * Damped Riemannian Newton ascent of G on the unit sphere from n0.
 * Tangent-plane gradient gt and Hessian Ht = T^T H T - G I (G is positively
 * homogeneous of degree one, so n.grad = G).  If Ht is not negative definite
 * it is shifted until it is; the step is then halved until G does not fall.
 * Returns iterations used; *gnorm gets the final tangent-gradient norm and
 * *hmax the largest eigenvalue of the final (unshifted) tangent Hessian.
 */
static int newton_sphere(const double* n0, const double* d, const double* Pa, const double* Pb, double tol,
                         double* nout, double* Gout, double* gnorm, double* hmax) {
    double n[3] = {n0[0], n0[1], n0[2]};
    double l = norm3(n);
    for (int i = 0; i < 3; ++i) n[i] /= l;
    gval_t gv;
    int it;
    const int maxit = 200;
    double scale = 1.0 + norm3(d);
    for (it = 0; it < maxit; ++it) {
        G_full(n, d, Pa, Pb, &gv);
        double t1[3], t2[3];
        tangent_basis(n, t1, t2);
        double g1 = dot3(t1, gv.grad), g2 = dot3(t2, gv.grad);
        double Ht1[3], Ht2[3];
        matvec3(gv.H, t1, Ht1);
        matvec3(gv.H, t2, Ht2);
        double h11 = dot3(t1, Ht1) - gv.G, h22 = dot3(t2, Ht2) - gv.G, h12 = dot3(t1, Ht2);
        double tr = 0.5 * (h11 + h22), df = 0.5 * (h11 - h22);
        double lmax = tr + sqrt(df * df + h12 * h12);
        *gnorm = sqrt(g1 * g1 + g2 * g2);
        *hmax = lmax;
        if (*gnorm <= tol) break;
        double kappa = 1e-6 * scale;
        if (lmax > -kappa) {
            double shift = lmax + kappa;
            h11 -= shift;
            h22 -= shift;
        }
        double det = h11 * h22 - h12 * h12;
        double d1 = -(h22 * g1 - h12 * g2) / det;
        double d2 = -(-h12 * g1 + h11 * g2) / det;
        double step = 1.0;
        int accepted = 0;
        for (int bt = 0; bt < 60; ++bt) {
            double m[3];
            for (int i = 0; i < 3; ++i) m[i] = n[i] + step * (d1 * t1[i] + d2 * t2[i]);
            double lm = norm3(m);
            for (int i = 0; i < 3; ++i) m[i] /= lm;
            double Gm = orc_G(m, d, Pa, Pb);
            if (Gm >= gv.G - 1e-15 * scale) {
                for (int i = 0; i < 3; ++i) n[i] = m[i];
                accepted = 1;
                break;
            }
            step *= 0.5;
        }
        if (!accepted) break; /* no ascent possible at this precision */
    }
    G_full(n, d, Pa, Pb, &gv);
    {
        double t1[3], t2[3];
        tangent_basis(n, t1, t2);
        double g1 = dot3(t1, gv.grad), g2 = dot3(t2, gv.grad);
        double Ht1[3], Ht2[3];
        matvec3(gv.H, t1, Ht1);
        matvec3(gv.H, t2, Ht2);
        double h11 = dot3(t1, Ht1) - gv.G, h22 = dot3(t2, Ht2) - gv.G, h12 = dot3(t1, Ht2);
        double tr = 0.5 * (h11 + h22), df = 0.5 * (h11 - h22);
        *hmax = tr + sqrt(df * df + h12 * h12);
        *gnorm = sqrt(g1 * g1 + g2 * g2);
    }
    for (int i = 0; i < 3; ++i) nout[i] = n[i];
    *Gout = gv.G;
    return it;
}

/* flags returned by orc_snsd */
#define ORC_SNSD_TIE 1          /* two distinct maxima agree to 1e-12 (set-valued contact) */
#define ORC_SNSD_NOT_NEGDEF 2   /* tangent Hessian at the maximiser is not negative definite */
#define ORC_SNSD_NOT_CONVERGED 4

/*
 * SNSD of one ellipsoid pair.  d = minimum-image c_b - c_a.
 * out[0] = Phi, out[1..3] = n (unit, from a to b), out[4..6] = r_a = y_a - c_a,
 * out[7..9] = r_b = y_b - c_b.  Multi-start: G on the 642 icosphere directions
 * plus 8 seeds (+-d/|d| and +-the coordinate axes... the first two are the
 * important ones); the three best seeds that are mutually more than 0.2 rad
 * apart are refined by newton_sphere; the best result is kept, ties broken by
 * the smaller seed index.
 */
int orc_snsd_d(const double* d, const double* Pa, const double* Pb, double* out) {
    ico_build();
    int nseed = g_ico_n + 8;
    double dl = norm3(d);
    double dh[3] = {0, 0, 1};
    if (dl > 0) for (int i = 0; i < 3; ++i) dh[i] = d[i] / dl;
    double (*seeds)[3] = malloc(sizeof(double) * 3 * nseed);
    for (int i = 0; i < 3; ++i) { seeds[0][i] = dh[i]; seeds[1][i] = -dh[i]; }
    for (int a = 0; a < 3; ++a)
        for (int sgn = 0; sgn < 2; ++sgn) {
            int k = 2 + 2 * a + sgn;
            for (int i = 0; i < 3; ++i) seeds[k][i] = (i == a) ? (sgn ? -1.0 : 1.0) : 0.0;
        }
    for (int v = 0; v < g_ico_n; ++v)
        for (int i = 0; i < 3; ++i) seeds[8 + v][i] = g_ico[v][i];
    double* Gs = malloc(sizeof(double) * nseed);
    for (int s = 0; s < nseed; ++s) Gs[s] = orc_G(seeds[s], d, Pa, Pb);
    int best[3] = {-1, -1, -1};
    int nb = 0;
    char* used = calloc(nseed, 1);
    while (nb < 3) {
        int arg = -1;
        for (int s = 0; s < nseed; ++s) {
            if (used[s]) continue;
            int far = 1;
            for (int b = 0; b < nb; ++b)
                if (dot3(seeds[s], seeds[best[b]]) > cos(0.2)) { far = 0; break; }
            if (!far) { used[s] = 1; continue; }
            if (arg < 0 || Gs[s] > Gs[arg]) arg = s;
        }
        if (arg < 0) break;
        used[arg] = 1;
        best[nb++] = arg;
    }
    double scale = 1.0 + dl;
    double tol = 1e-14 * scale;
    double bestG = -HUGE_VAL, bestn[3] = {0, 0, 0}, bgn = 0, bhm = 0;
    int flags = 0, bidx = -1;
    double candG[3], candn[3][3];
    for (int b = 0; b < nb; ++b) {
        double n1[3], G1, gn, hm;
        newton_sphere(seeds[best[b]], d, Pa, Pb, tol, n1, &G1, &gn, &hm);
        candG[b] = G1;
        for (int i = 0; i < 3; ++i) candn[b][i] = n1[i];
        if (G1 > bestG) { bestG = G1; for (int i = 0; i < 3; ++i) bestn[i] = n1[i]; bgn = gn; bhm = hm; bidx = b; }
    }
    for (int b = 0; b < nb; ++b) {
        if (b == bidx) continue;
        double dn[3] = {candn[b][0] - bestn[0], candn[b][1] - bestn[1], candn[b][2] - bestn[2]};
        if (fabs(candG[b] - bestG) <= 1e-12 * scale && norm3(dn) > 1e-6) flags |= ORC_SNSD_TIE;
    }
    if (bhm >= 0) flags |= ORC_SNSD_NOT_NEGDEF;
    if (bgn > 1e-10 * scale) flags |= ORC_SNSD_NOT_CONVERGED;
    double va[3], vb[3];
    matvec3(Pa, bestn, va);
    matvec3(Pb, bestn, vb);
    double sa = sqrt(dot3(bestn, va)), sb = sqrt(dot3(bestn, vb));
    out[0] = bestG;
    for (int i = 0; i < 3; ++i) {
        out[1 + i] = bestn[i];
        out[4 + i] = va[i] / sa;
        out[7 + i] = -vb[i] / sb;
    }
    free(seeds); free(Gs); free(used);
    return flags;
}

/* SNSD of pair (a, b) from positions, quaternions and semi-axes (n x 3 / n x 4
 * row-major), periodic box (0 = open axis).  Writes 10 doubles per pair. */
int64_t orc_snsd_pairs(int64_t npairs, const int32_t* pairs, const double* x, const double* q, const double* axes,
                       const double* box, double* out, int32_t* flags) {
    int64_t nflag = 0;
    for (int64_t p = 0; p < npairs; ++p) {
        int a = pairs[2 * p], b = pairs[2 * p + 1];
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = min_image(x[3 * b + k] - x[3 * a + k], box[k]);
        double Pa[9], Pb[9];
        orc_shape_matrix(q + 4 * a, axes + 3 * a, Pa);
        orc_shape_matrix(q + 4 * b, axes + 3 * b, Pb);
        int f = orc_snsd_d(d, Pa, Pb, out + 10 * p);
        if (flags) flags[p] = f;
        if (f) ++nflag;
    }
    return nflag;
}

/* ------------------------------------------------------------------ */
/* O7: Lemke's complementary pivoting                                   */
/* ------------------------------------------------------------------ */
/*
 * Solve  w = M z + q,  w >= 0, z >= 0, w.z = 0  (n x n, row-major M).
 * Artificial variable z0 with covering vector e = 1; tableau columns
 * [w (n) | z (n) | z0 | rhs] of  w - M z - e z0 = q.  Lexicographic
 * minimum-ratio rule (rows compared by rhs, then by the columns of the basis
 * inverse, i.e. the w block).  At termination the basic system is re-solved
 * from the original data (Gaussian elimination with partial pivoting plus one
 * round of iterative refinement) to remove the accumulated pivoting error.
 * Returns 0 on success, 1 on ray termination, 2 when the pivot cap is hit.
 */
static int solve_dense(int n, double* A, double* b) {
    /* in-place partial-pivot Gaussian elimination, A row-major n x n */
    int* piv = malloc(sizeof(int) * n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double mx = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[(size_t)i * n + k]) > mx) { mx = fabs(A[(size_t)i * n + k]); p = i; }
        if (mx == 0.0) { free(piv); return 1; }
        if (p != k) {
            for (int j = 0; j < n; ++j) { double t = A[(size_t)k * n + j]; A[(size_t)k * n + j] = A[(size_t)p * n + j]; A[(size_t)p * n + j] = t; }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            if (f == 0.0) continue;
            for (int j = k; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[(size_t)i * n + j] * b[j];
        b[i] = s / A[(size_t)i * n + i];
    }
    free(piv);
    return 0;
}

int orc_lemke(int n, const double* M, const double* q, double* z, double* w, int max_pivots, int* npivots) {
    for (int i = 0; i < n; ++i) { z[i] = 0.0; w[i] = q[i]; }
    if (npivots) *npivots = 0;
    if (n == 0) return 0;
    int rmin = 0;
    for (int i = 1; i < n; ++i)
        if (q[i] < q[rmin]) rmin = i;
    if (q[rmin] >= 0.0) return 0;
    const int W = 2 * n + 2; /* tableau width */
    const int Z0 = 2 * n, RHS = 2 * n + 1;
    double* T = malloc(sizeof(double) * (size_t)n * W);
    int* basis = malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) {
        double* row = T + (size_t)i * W;
        for (int j = 0; j < n; ++j) row[j] = (i == j) ? 1.0 : 0.0;
        for (int j = 0; j < n; ++j) row[n + j] = -M[(size_t)i * n + j];
        row[Z0] = -1.0;
        row[RHS] = q[i];
        basis[i] = i;
    }
    double qscale = 0.0;
    for (int i = 0; i < n; ++i) qscale = fmax(qscale, fabs(q[i]));
    const double ptol = 1e-12;
    int status = 2, piv_count = 0;
    int entering = Z0, prow = rmin;
    for (;;) {
        /* pivot on (prow, entering) */
        double* pr = T + (size_t)prow * W;
        double pv = pr[entering];
        for (int j = 0; j < W; ++j) pr[j] /= pv;
        for (int i = 0; i < n; ++i) {
            if (i == prow) continue;
            double* ri = T + (size_t)i * W;
            double f = ri[entering];
            if (f == 0.0) continue;
            for (int j = 0; j < W; ++j) ri[j] -= f * pr[j];
        }
        int leaving = basis[prow];
        basis[prow] = entering;
        ++piv_count;
        if (leaving == Z0) { status = 0; break; }
        if (piv_count >= max_pivots) { status = 2; break; }
        entering = (leaving < n) ? leaving + n : leaving - n; /* complement */
        /* lexicographic ratio test */
        int best = -1;
        for (int i = 0; i < n; ++i) {
            double* ri = T + (size_t)i * W;
            double c = ri[entering];
            if (c <= ptol) continue;
            if (best < 0) { best = i; continue; }
            double* rb = T + (size_t)best * W;
            double cb = rb[entering];
            double ra = ri[RHS] / c, rbv = rb[RHS] / cb;
            double sc = 1e-13 * (1.0 + fabs(ra) + fabs(rbv));
            if (ra < rbv - sc) { best = i; continue; }
            if (ra > rbv + sc) continue;
            /* tie: prefer the row holding z0, then compare the w columns */
            if (basis[i] == Z0) { best = i; continue; }
            if (basis[best] == Z0) continue;
            for (int j = 0; j < n; ++j) {
                double ea = ri[j] / c, eb = rb[j] / cb;
                if (ea < eb - 1e-15) { best = i; break; }
                if (ea > eb + 1e-15) break;
            }
        }
        if (best < 0) { status = 1; break; }
        prow = best;
    }
    if (npivots) *npivots = piv_count;
    if (status == 0) {
        /* re-solve the final basis from the original data: B xB = q, with
         * column j of B = e_j for basic w_j and -M[:, j] for basic z_j. */
        double* B = calloc((size_t)n * n, sizeof(double));
        double* xb = malloc(sizeof(double) * n);
        double* B0 = malloc(sizeof(double) * (size_t)n * n);
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < n; ++c) {
                int v = basis[c];
                double e = (v < n) ? ((i == v) ? 1.0 : 0.0) : -M[(size_t)i * n + (v - n)];
                B[(size_t)i * n + c] = e;
            }
        memcpy(B0, B, sizeof(double) * (size_t)n * n);
        for (int i = 0; i < n; ++i) xb[i] = q[i];
        int bad = solve_dense(n, B, xb);
        if (!bad) {
            /* one round of iterative refinement */
            double* r = malloc(sizeof(double) * n);
            for (int i = 0; i < n; ++i) {
                double s = q[i];
                for (int c = 0; c < n; ++c) s -= B0[(size_t)i * n + c] * xb[c];
                r[i] = s;
            }
            memcpy(B, B0, sizeof(double) * (size_t)n * n);
            if (!solve_dense(n, B, r))
                for (int i = 0; i < n; ++i) xb[i] += r[i];
            free(r);
        } else {
            for (int i = 0; i < n; ++i) xb[i] = T[(size_t)i * W + RHS];
        }
        for (int i = 0; i < n; ++i) z[i] = 0.0;
        for (int c = 0; c < n; ++c) {
            int v = basis[c];
            if (v >= n && v < 2 * n) z[v - n] = xb[c] > 0.0 ? xb[c] : 0.0;
        }
        for (int i = 0; i < n; ++i) {
            double s = q[i];
            for (int j = 0; j < n; ++j) s += M[(size_t)i * n + j] * z[j];
            w[i] = s;
        }
        free(B); free(B0); free(xb);
    }
    free(T);
    free(basis);
    (void)qscale;
    return status;
}
