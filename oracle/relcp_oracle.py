"""ReLCP oracle: one time step of the recursive constraint augmentation, FP64.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this module; the product path never does.  It
shares no code with the CUDA library.  The heavy numerics (brute-force pairs,
multi-start SNSD Newton, Lemke pivoting) are plain C in oracle.c; this file
takes the steps of Algorithm 1 in the paper's order with numpy.

Readings of the paper used here (all FP64):
  * contact Jacobian row (Appendix, proof of the geometric stopping rule):
        [-n, -(r_a x n), n, (r_b x n)]  on the (u, omega) blocks of bodies a, b;
  * with c = dt and K = M (overdamped, Eq. law_overdamped) or K = dt M^-1
    (inertial, Eq. law_inertia), the n-th LCP of Eq. relcp / relcp_inertial is
        g = q + c D^T K D gamma >= 0  _|_  gamma >= 0,   A = c D^T K D,
    with fixed per-row offsets q: for rows of A_0, q = Phi(C^k) + c d^T U_free;
    for a row appended at recursion j, q = Phi(C_j) - c d^T K D_{j-1} gamma_{j-1}
    (the pull-back Psi of Sec. 3.1.3; retained rows keep their q, Eq. qn_scaled
    and the identity q_{m+1}|A_m = q_m of the small-dt proof);
  * U_free = vel + K F_ext (+ an affine background velocity when the box is
    compacted), the trial configuration telescopes to
        C_{n+1} = C^k + dt G^k (U_free + K D_n gamma_n),
    with x' = x + dt u and q' = normalise(q + dt/2 (0, omega) (x) q);
  * a pair violates when Phi < -eps_NCP and the recursion stops when
    max overlap <= eps_NCP (Eq. gap_stopping_rule).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

INERTIAL = 0
OVERDAMPED = 1
OVERDAMPED_2D = 2  # bodies confined to the z = 0 plane: three DOFs (u_x, u_y, omega_z)

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        L.orc_pairs.restype = ctypes.c_int64
        L.orc_pairs.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_double, ip, ctypes.c_int64]
        L.orc_pair_margin.restype = ctypes.c_double
        L.orc_pair_margin.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp, ctypes.c_double]
        L.orc_snsd_pairs.restype = ctypes.c_int64
        L.orc_snsd_pairs.argtypes = [ctypes.c_int64, ip, dp, dp, dp, dp, dp, ip]
        L.orc_snsd_d.restype = ctypes.c_int
        L.orc_snsd_d.argtypes = [dp, dp, dp, dp]
        L.orc_G.restype = ctypes.c_double
        L.orc_G.argtypes = [dp, dp, dp, dp]
        L.orc_quat_rot.restype = None
        L.orc_quat_rot.argtypes = [dp, dp]
        L.orc_shape_matrix.restype = None
        L.orc_shape_matrix.argtypes = [dp, dp, dp]
        L.orc_icosphere.restype = ctypes.c_int
        L.orc_icosphere.argtypes = [dp]
        L.orc_lemke.restype = ctypes.c_int
        L.orc_lemke.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


# ---------------------------------------------------------------------------
# geometry and kinematics (Sec. 2.1.1)
# ---------------------------------------------------------------------------
def quat_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrices (n, 3, 3) of (s, w) quaternions, body -> world."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    s, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - s * z)
    R[..., 0, 2] = 2 * (x * z + s * y)
    R[..., 1, 0] = 2 * (x * y + s * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - s * x)
    R[..., 2, 0] = 2 * (x * z - s * y)
    R[..., 2, 1] = 2 * (y * z + s * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product of (..., 4) quaternions (s, w)."""
    s1, v1 = a[..., :1], a[..., 1:]
    s2, v2 = b[..., :1], b[..., 1:]
    s = s1 * s2 - np.sum(v1 * v2, axis=-1, keepdims=True)
    v = s1 * v2 + s2 * v1 + np.cross(v1, v2)
    return np.concatenate([s, v], axis=-1)


def quat_step(q: np.ndarray, omega: np.ndarray, dt: float) -> np.ndarray:
    """Linear kinematic update with G^k (Eq. law_inertia, 'implicit (linear)';
    Eq. law_overdamped): q + dt * 1/2 (0, omega) (x) q, then normalised."""
    w4 = np.concatenate([np.zeros(omega.shape[:-1] + (1,)), omega], axis=-1)
    qn = q / np.linalg.norm(q, axis=-1, keepdims=True)
    q1 = qn + dt * 0.5 * quat_mul(w4, qn)
    return q1 / np.linalg.norm(q1, axis=-1, keepdims=True)


def mass_properties(axes: np.ndarray, density: float = 1.0):
    """Mass and principal inertia of solid ellipsoids: m = 4/3 pi a b c rho,
    I = m/5 (b^2 + c^2, a^2 + c^2, a^2 + b^2)."""
    a, b, c = axes[:, 0], axes[:, 1], axes[:, 2]
    m = density * 4.0 / 3.0 * np.pi * a * b * c
    I = np.stack([m / 5 * (b * b + c * c), m / 5 * (a * a + c * c), m / 5 * (a * a + b * b)], axis=1)
    return m, I


def operator_K(dynamics: int, dt: float, q: np.ndarray, axes: np.ndarray, density: float = 1.0,
               drag_xi: float = 1.0):
    """Per-body operator K of the LCP  g = q + dt D^T K D gamma.

    Overdamped: K = M, the local-drag mobility of Eq. ellipsoid_mobility,
    (1/xi) diag(I/L, 12 I/L^3) with L = 2 x (largest semi-axis).
    Inertial: K = dt M^-1 with M = diag(m I, R I_body R^T) (Eq. law_inertia),
    evaluated at C^k and held fixed over the step.
    Returns kt (n,) and Kr (n, 3, 3)."""
    n = axes.shape[0]
    if dynamics in (OVERDAMPED, OVERDAMPED_2D):
        L = 2.0 * axes.max(axis=1)
        kt = 1.0 / (drag_xi * L)
        Kr = np.zeros((n, 3, 3))
        for k in range(3):
            Kr[:, k, k] = 12.0 / (drag_xi * L ** 3)
        return kt, Kr
    m, I = mass_properties(axes, density)
    R = quat_rot(q)
    Kr = dt * np.einsum("nij,nj,nkj->nik", R, 1.0 / I, R)
    return dt / m, Kr


# ---------------------------------------------------------------------------
# candidate pairs and SNSD (C core)
# ---------------------------------------------------------------------------
def candidate_pairs(x: np.ndarray, rb: np.ndarray, box: np.ndarray, skin: float) -> np.ndarray:
    """All i<j with periodic centre distance <= rb_i + rb_j + skin (brute
    force, i-major, j ascending)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    rb = np.ascontiguousarray(rb, dtype=np.float64)
    box = np.ascontiguousarray(box, dtype=np.float64)
    n = x.shape[0]
    cap = max(16, 64 * n)
    while True:
        out = np.zeros((cap, 2), dtype=np.int32)
        npairs = lib().orc_pairs(n, _dp(x), _dp(rb), _dp(box), float(skin), _ip(out), cap)
        if npairs <= cap:
            return out[:npairs].copy()
        cap = int(npairs)


def snsd(pairs: np.ndarray, x: np.ndarray, q: np.ndarray, axes: np.ndarray, box: np.ndarray):
    """SNSD of every listed pair: returns (phi (P,), n (P,3), r_a (P,3),
    r_b (P,3), flags (P,))."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    P = pairs.shape[0]
    out = np.zeros((max(P, 1), 10))
    flags = np.zeros(max(P, 1), dtype=np.int32)
    if P:
        lib().orc_snsd_pairs(P, _ip(pairs), _dp(np.ascontiguousarray(x, dtype=np.float64)),
                             _dp(np.ascontiguousarray(q, dtype=np.float64)),
                             _dp(np.ascontiguousarray(axes, dtype=np.float64)),
                             _dp(np.ascontiguousarray(box, dtype=np.float64)), _dp(out), _ip(flags))
    out = out[:P]
    return out[:, 0].copy(), out[:, 1:4].copy(), out[:, 4:7].copy(), out[:, 7:10].copy(), flags[:P].copy()


# ---------------------------------------------------------------------------
# spherocylinders (Sec. 5.4 colony cells): a segment of half-length h along
# the body x axis, swept by a ball of radius rho; semi-axes row (h + rho, rho, rho)
# ---------------------------------------------------------------------------
SHAPE_ELLIPSOID = 0
SHAPE_SPHEROCYLINDER = 1


def capsule_geometry(q, axes):
    """Per body: unit axis u = R(q) e_x, segment half-length h, radius rho."""
    R = quat_rot(q)
    u = R[:, :, 0]
    rho = np.asarray(axes, dtype=np.float64)[:, 1]
    h = np.asarray(axes, dtype=np.float64)[:, 0] - rho
    return u, h, rho


def segment_closest_params(w, u, ha, v, hb):
    """Parameters (s, t) of the closest points A + s u, B + t v (s in
    [-ha, ha], t in [-hb, hb]) of two segments with B - A = w, u and v unit:
    the minimiser of f(s, t) = |w + t v - s u|^2 over the rectangle, taken as
    the best of the candidates (the interior stationary point when it lies
    inside, then the edge minimisers at s = -ha, +ha, t = -hb, +hb); the first
    minimal candidate in that order wins a tie (parallel segments).  Plain
    loop, one pair at a time."""
    uv = float(u @ v)
    wu, wv = float(w @ u), float(w @ v)
    cands = []
    det = 1.0 - uv * uv
    if det > 1e-14:
        s0 = (wu - uv * wv) / det
        t0 = (uv * wu - wv) / det
        if abs(s0) <= ha and abs(t0) <= hb:
            cands.append((s0, t0))
    for s_ in (-ha, ha):
        cands.append((s_, min(max(s_ * uv - wv, -hb), hb)))
    for t_ in (-hb, hb):
        cands.append((min(max(wu + t_ * uv, -ha), ha), t_))
    best, bf = None, None
    for s_, t_ in cands:
        r = w + t_ * v - s_ * u
        f = float(r @ r)
        if bf is None or f < bf:
            best, bf = (s_, t_), f
    return best


def snsd_capsules(pairs, x, q, axes, box):
    """Shared-normal signed distance of spherocylinder pairs: Phi = |Q - P| -
    rho_a - rho_b with P, Q the closest points of the two segments (minimum
    image), n = (Q - P)/|Q - P| from a to b, support points y_a = P + rho_a n,
    y_b = Q - rho_b n, lever arms r = y - c.  Segments that intersect (no
    normal) are flagged.  Returns (phi, n, r_a, r_b, flags)."""
    pairs = np.asarray(pairs)
    P_ = pairs.shape[0]
    u, h, rho = capsule_geometry(q, axes)
    phi = np.zeros(P_)
    nrm = np.zeros((P_, 3))
    ra = np.zeros((P_, 3))
    rb = np.zeros((P_, 3))
    fl = np.zeros(P_, dtype=np.int32)
    box = np.asarray(box, dtype=np.float64)
    for k in range(P_):
        i, j = int(pairs[k, 0]), int(pairs[k, 1])
        w = min_image(x[j] - x[i], box)
        s_, t_ = segment_closest_params(w, u[i], h[i], u[j], h[j])
        dv = w + t_ * u[j] - s_ * u[i]
        dist = float(np.linalg.norm(dv))
        if dist <= 1e-12:
            fl[k] = 1
            continue
        nn = dv / dist
        phi[k] = dist - rho[i] - rho[j]
        nrm[k] = nn
        ra[k] = s_ * u[i] + rho[i] * nn
        rb[k] = t_ * u[j] - rho[j] * nn
    return phi, nrm, ra, rb, fl


def snsd_shape(shape, pairs, x, q, axes, box):
    if shape == SHAPE_SPHEROCYLINDER:
        return snsd_capsules(pairs, x, q, axes, box)
    return snsd(pairs, x, q, axes, box)


def snsd_from_d(d, Pa, Pb):
    """SNSD for a given minimum-image centre offset d and shape matrices."""
    out = np.zeros(10)
    d = np.ascontiguousarray(d, dtype=np.float64)
    Pa = np.ascontiguousarray(Pa, dtype=np.float64)
    Pb = np.ascontiguousarray(Pb, dtype=np.float64)
    f = lib().orc_snsd_d(_dp(d), _dp(Pa), _dp(Pb), _dp(out))
    return out[0], out[1:4].copy(), out[4:7].copy(), out[7:10].copy(), int(f)


def shape_matrices(q: np.ndarray, axes: np.ndarray) -> np.ndarray:
    R = quat_rot(q)
    return np.einsum("nij,nj,nkj->nik", R, axes ** 2, R)


def min_image(d: np.ndarray, box: np.ndarray) -> np.ndarray:
    d = np.array(d, dtype=np.float64, copy=True)
    for k in range(3):
        if box[k] > 0:
            d[..., k] = d[..., k] - box[k] * np.rint(d[..., k] / box[k])
    return d


def lemke(A: np.ndarray, qv: np.ndarray, max_pivots: int | None = None):
    """Lemke's method on 0 <= A z + q _|_ z >= 0.  Returns (z, w, status,
    pivots); status 0 = solved, 1 = ray termination, 2 = pivot cap."""
    n = qv.shape[0]
    A = np.ascontiguousarray(A, dtype=np.float64)
    qv = np.ascontiguousarray(qv, dtype=np.float64)
    z = np.zeros(max(n, 1))
    w = np.zeros(max(n, 1))
    piv = ctypes.c_int(0)
    if max_pivots is None:
        max_pivots = 50 * n + 100
    st = lib().orc_lemke(n, _dp(A if n else np.zeros(1)), _dp(qv if n else np.zeros(1)), _dp(z), _dp(w),
                         int(max_pivots), ctypes.byref(piv))
    return z[:n].copy(), w[:n].copy(), int(st), int(piv.value)


# ---------------------------------------------------------------------------
# contact operator pieces
# ---------------------------------------------------------------------------
def rows_dot_U(ia, ib, nrm, ta, tb, U):
    """d_alpha^T U for rows (ia, ib, n, t_a = r_a x n, t_b = r_b x n)."""
    return (np.einsum("ij,ij->i", nrm, U[ib, :3] - U[ia, :3]) + np.einsum("ij,ij->i", tb, U[ib, 3:])
            - np.einsum("ij,ij->i", ta, U[ia, 3:]))


def wrench(nbody, ia, ib, nrm, ta, tb, gamma):
    """D gamma: per-body force and torque (Eq. collision_ft)."""
    W = np.zeros((nbody, 6))
    np.add.at(W, ia, np.concatenate([-nrm * gamma[:, None], -ta * gamma[:, None]], axis=1))
    np.add.at(W, ib, np.concatenate([nrm * gamma[:, None], tb * gamma[:, None]], axis=1))
    return W


def apply_K(kt, Kr, W):
    out = np.empty_like(W)
    out[:, :3] = kt[:, None] * W[:, :3]
    out[:, 3:] = np.einsum("nij,nj->ni", Kr, W[:, 3:])
    return out


def dense_D(nbody, ia, ib, nrm, ta, tb):
    """D^T as a dense (rows, 6 nbody) matrix."""
    m = ia.shape[0]
    Dt = np.zeros((m, 6 * nbody))
    r = np.arange(m)
    for k in range(3):
        Dt[r, 6 * ia + k] = -nrm[:, k]
        Dt[r, 6 * ia + 3 + k] = -ta[:, k]
        Dt[r, 6 * ib + k] = nrm[:, k]
        Dt[r, 6 * ib + 3 + k] = tb[:, k]
    return Dt


def dense_A(c, kt, Kr, ia, ib, nrm, ta, tb):
    """A = c D^T K D (dense)."""
    nbody = kt.shape[0]
    Dt = dense_D(nbody, ia, ib, nrm, ta, tb)
    Kd = np.zeros((6 * nbody, 6 * nbody))
    for b in range(nbody):
        Kd[6 * b:6 * b + 3, 6 * b:6 * b + 3] = kt[b] * np.eye(3)
        Kd[6 * b + 3:6 * b + 6, 6 * b + 3:6 * b + 6] = Kr[b]
    return c * Dt @ Kd @ Dt.T


def sparse_A(c, kt, Kr, ia, ib, nrm, ta, tb):
    """A = c D^T K D assembled body by body (same values as dense_A without
    the 6N x 6N intermediate; used for the larger snapshots)."""
    m = ia.shape[0]
    nbody = kt.shape[0]
    A = np.zeros((m, m))
    # coefficient vectors of each row on each of its two bodies
    ca = np.concatenate([-nrm, -ta], axis=1)
    cb = np.concatenate([nrm, tb], axis=1)
    inc = [[] for _ in range(nbody)]
    for r in range(m):
        inc[ia[r]].append((r, 0))
        inc[ib[r]].append((r, 1))
    for b in range(nbody):
        if not inc[b]:
            continue
        idx = np.array([r for r, _ in inc[b]])
        C = np.stack([ca[r] if s == 0 else cb[r] for r, s in inc[b]])
        KC = C.copy()
        KC[:, :3] *= kt[b]
        KC[:, 3:] = C[:, 3:] @ Kr[b].T
        A[np.ix_(idx, idx)] += c * (C @ KC.T)
    return A


# ---------------------------------------------------------------------------
# one ReLCP time step (Algorithm 1; inertial variant Eq. relcp_inertial)
# ---------------------------------------------------------------------------
@dataclass
class Config:
    dynamics: int = INERTIAL
    dt: float = 1e-3
    eps_ncp: float = 1e-3
    box: tuple = (0.0, 0.0, 0.0)
    skin: float = 0.05
    phi_skin: float | None = None  # None: equal to skin
    drag_xi: float = 1.0
    density: float = 1.0
    strain_rate: float = 0.0
    max_recursion: int = 64
    shape: int = SHAPE_ELLIPSOID


@dataclass
class StepResult:
    x: np.ndarray
    q: np.ndarray
    vel: np.ndarray
    box: np.ndarray
    pairs: np.ndarray
    phi0: np.ndarray
    rows_ia: np.ndarray
    rows_ib: np.ndarray
    rows_pair: np.ndarray
    rows_rec: np.ndarray
    rows_n: np.ndarray
    rows_ta: np.ndarray
    rows_tb: np.ndarray
    rows_q: np.ndarray
    gamma: np.ndarray
    g: np.ndarray
    U_contact: np.ndarray
    depth: int
    status: int
    max_overlap: float
    W: list = field(default_factory=list)
    gammas: list = field(default_factory=list)
    gs: list = field(default_factory=list)
    U_contacts: list = field(default_factory=list)
    trial_phi: list = field(default_factory=list)
    ambiguous: int = 0
    snsd_flags: int = 0
    lcp_status: list = field(default_factory=list)
    n_rows_per_rec: list = field(default_factory=list)


def free_velocity(cfg: Config, x, vel, fext, kt, Kr, box):
    """U_free = vel + K F_ext, plus the affine background velocity
    strain_rate * (x - L/2) on periodic axes when the box is compacted.  In the
    plane (OVERDAMPED_2D) only u_x, u_y and omega_z are kept."""
    U = np.array(vel, dtype=np.float64, copy=True)
    U += apply_K(kt, Kr, np.asarray(fext, dtype=np.float64))
    if cfg.strain_rate != 0.0:
        for k in range(3):
            if box[k] > 0:
                U[:, k] += cfg.strain_rate * (x[:, k] - 0.5 * box[k])
    if cfg.dynamics == OVERDAMPED_2D:
        U[:, 2] = 0.0
        U[:, 3] = 0.0
        U[:, 4] = 0.0
    return U


def planar_rows(nrm, ta, tb):
    """Rows of the planar problem (OVERDAMPED_2D): the generalised velocity
    has the three components (u_x, u_y, omega_z) with the SPD mobility
    diag(k_t, k_t, k_r) of Eq. ellipsoid_mobility; embedded in the six-DOF
    layout, a row keeps its entries on those components and has none on
    u_z, omega_x, omega_y."""
    nrm = np.array(nrm, dtype=np.float64, copy=True)
    ta = np.array(ta, dtype=np.float64, copy=True)
    tb = np.array(tb, dtype=np.float64, copy=True)
    nrm[:, 2] = 0.0
    ta[:, :2] = 0.0
    tb[:, :2] = 0.0
    return nrm, ta, tb


def step(cfg: Config, x, q, axes, vel=None, fext=None, band: float = 1e-9, lcp_solver=None) -> StepResult:
    """One ReLCP time step from C^k = (x, q).  Returns the accepted C^{k+1},
    the velocity of the step (inertial: U^{k+1}), every constraint row with the
    recursion index that created it, and per-recursion diagnostics.

    status: 0 ok, 5 recursion limit, 4 LCP failure.
    `band`: decisions within band * (1 + |eps|) of a threshold are counted as
    ambiguous (reported, not changed).  `lcp_solver(A, q) -> gamma` replaces
    Lemke's method (the tests pass a brute-force enumeration)."""
    x = np.array(x, dtype=np.float64)
    q = np.array(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    axes = np.asarray(axes, dtype=np.float64)
    n = x.shape[0]
    vel = np.zeros((n, 6)) if vel is None else np.asarray(vel, dtype=np.float64)
    fext = np.zeros((n, 6)) if fext is None else np.asarray(fext, dtype=np.float64)
    box0 = np.asarray(cfg.box, dtype=np.float64)
    box1 = np.where(box0 > 0, box0 * (1.0 + cfg.strain_rate * cfg.dt), 0.0)
    dt = cfg.dt
    c = dt
    phi_skin = cfg.skin if cfg.phi_skin is None else cfg.phi_skin

    if cfg.shape == SHAPE_SPHEROCYLINDER and cfg.dynamics == INERTIAL:
        raise NotImplementedError("spherocylinders are stepped with the overdamped laws only")
    kt, Kr = operator_K(cfg.dynamics, dt, q, axes, cfg.density, cfg.drag_xi)
    U_free = free_velocity(cfg, x, vel, fext, kt, Kr, box0)

    # Initialise: near-contacting pairs and their SNSD constraints at C^k
    rb = axes.max(axis=1)
    pairs = candidate_pairs(x, rb, box0, cfg.skin)
    phi0, n0, ra0, rb0, fl0 = snsd_shape(cfg.shape, pairs, x, q, axes, box0)
    ambiguous = int(np.sum(np.abs(phi0 - phi_skin) <= band * (1.0 + abs(phi_skin))))
    keep = np.nonzero(phi0 <= phi_skin)[0]
    ia = pairs[keep, 0].astype(np.int64)
    ib = pairs[keep, 1].astype(np.int64)
    nrm = n0[keep]
    ta = np.cross(ra0[keep], nrm)
    tb = np.cross(rb0[keep], nrm)
    if cfg.dynamics == OVERDAMPED_2D:
        nrm, ta, tb = planar_rows(nrm, ta, tb)
    # offset of A_0 rows: Phi_0 + c d^T U_free; the affine part of the relative
    # free velocity uses the minimum-image offset
    dU = rows_dot_U(ia, ib, nrm, ta, tb, U_free - _affine(cfg, x, box0))
    if cfg.strain_rate != 0.0:
        dmin = min_image(x[ib] - x[ia], box0)
        dU = dU + cfg.strain_rate * np.einsum("ij,ij->i", nrm, dmin)
    qv = phi0[keep] + c * dU
    rec = np.zeros(keep.shape[0], dtype=np.int64)
    rpair = keep.astype(np.int64)
    snsd_flags = int(np.count_nonzero(fl0))

    res = StepResult(x=x, q=q, vel=vel, box=box1, pairs=pairs, phi0=phi0, rows_ia=ia, rows_ib=ib,
                     rows_pair=rpair, rows_rec=rec, rows_n=nrm, rows_ta=ta, rows_tb=tb, rows_q=qv,
                     gamma=np.zeros(0), g=np.zeros(0), U_contact=np.zeros((n, 6)), depth=0, status=0,
                     max_overlap=0.0)
    depth = 0
    while True:
        m = ia.shape[0]
        if m:
            A = sparse_A(c, kt, Kr, ia, ib, nrm, ta, tb) if n > 256 else dense_A(c, kt, Kr, ia, ib, nrm, ta, tb)
            if lcp_solver is not None:
                gamma = lcp_solver(A, qv)
                st = 0
            else:
                gamma, _, st, _ = lemke(A, qv)
            res.lcp_status.append(st)
            if st != 0:
                res.status = 4
            g = A @ gamma + qv
            res.W.append(float(gamma @ A @ gamma))
        else:
            gamma = np.zeros(0)
            g = np.zeros(0)
            res.lcp_status.append(0)
            res.W.append(0.0)
        Wb = wrench(n, ia, ib, nrm, ta, tb, gamma)
        Uc = apply_K(kt, Kr, Wb)
        res.gammas.append(gamma.copy())
        res.gs.append(g.copy())
        res.U_contacts.append(Uc.copy())
        res.n_rows_per_rec.append(m)
        # trial configuration C_{n+1} = C^k + dt G^k (U_free + K D_n gamma_n)
        U = U_free + Uc
        x1 = x + dt * U[:, :3]
        q1 = quat_step(q, U[:, 3:], dt)
        phi1, n1, ra1, rb1, fl1 = snsd_shape(cfg.shape, pairs, x1, q1, axes, box1)
        snsd_flags += int(np.count_nonzero(fl1))
        res.trial_phi.append(phi1.copy())
        ambiguous += int(np.sum(np.abs(phi1 + cfg.eps_ncp) <= band * (1.0 + cfg.eps_ncp)))
        viol = np.nonzero(phi1 < -cfg.eps_ncp)[0]
        max_ov = float(max(0.0, -phi1.min())) if phi1.size else 0.0
        if viol.size == 0:
            break
        if depth >= cfg.max_recursion:
            res.status = 5
            break
        depth += 1
        # append one frozen-normal row per violating pair, pulled back to C^k
        nn = n1[viol]
        tan = np.cross(ra1[viol], nn)
        tbn = np.cross(rb1[viol], nn)
        if cfg.dynamics == OVERDAMPED_2D:
            nn, tan, tbn = planar_rows(nn, tan, tbn)
        iav = pairs[viol, 0].astype(np.int64)
        ibv = pairs[viol, 1].astype(np.int64)
        qnew = phi1[viol] - c * rows_dot_U(iav, ibv, nn, tan, tbn, Uc)
        ia = np.concatenate([ia, iav])
        ib = np.concatenate([ib, ibv])
        nrm = np.concatenate([nrm, nn])
        ta = np.concatenate([ta, tan])
        tb = np.concatenate([tb, tbn])
        qv = np.concatenate([qv, qnew])
        rec = np.concatenate([rec, np.full(viol.size, depth, dtype=np.int64)])
        rpair = np.concatenate([rpair, viol.astype(np.int64)])
    # accept
    xw = x1.copy()
    for k in range(3):
        if box1[k] > 0:
            xw[:, k] = xw[:, k] - box1[k] * np.floor(xw[:, k] / box1[k])
    res.x = xw
    res.q = q1
    res.vel = U
    res.rows_ia, res.rows_ib, res.rows_n, res.rows_ta, res.rows_tb = ia, ib, nrm, ta, tb
    res.rows_q, res.rows_rec, res.rows_pair = qv, rec, rpair
    res.gamma, res.g, res.U_contact = gamma, g, Uc
    res.depth = depth
    res.max_overlap = max_ov
    res.ambiguous = ambiguous
    res.snsd_flags = snsd_flags
    return res


def _affine(cfg: Config, x, box):
    A = np.zeros((x.shape[0], 6))
    if cfg.strain_rate != 0.0:
        for k in range(3):
            if box[k] > 0:
                A[:, k] = cfg.strain_rate * (x[:, k] - 0.5 * box[k])
    return A


def run(cfg: Config, x, q, axes, vel=None, fext=None, steps: int = 1):
    """Several steps; the box follows the compaction schedule."""
    results = []
    box = np.asarray(cfg.box, dtype=np.float64)
    for _ in range(steps):
        c2 = Config(**{**cfg.__dict__, "box": tuple(box)})
        r = step(c2, x, q, axes, vel, fext)
        results.append(r)
        x, q = r.x, r.q
        if cfg.dynamics == INERTIAL:
            vel = r.vel
        box = r.box
    return results
