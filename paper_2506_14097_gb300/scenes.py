"""Seeded synthetic scenes (inputs only).

This module produces arrays -- positions, unit quaternions (s, w1, w2, w3),
semi-axes, velocities, box sides, time steps -- for the workloads the ReLCP
paper exercises (Sec. 5: ellipsoid suspensions, two-ellipsoid collisions) and
their restated sizes.  It contains none of the contact method's arithmetic and
is the only code that both the CUDA path and the CPU oracle consume.

Every generator takes an explicit seed and uses numpy's PCG64 generator, so a
scene is a pure function of its arguments.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Scene:
    """One periodic (or open) scene.  Arrays are float64, row-major.

    x: (n, 3) centres; q: (n, 4) unit quaternions (s, w); axes: (n, 3)
    semi-axes; vel: (n, 6) (u, omega) with omega in the world frame;
    fext: (n, 6) external force and torque; box: (3,) periodic box sides
    (0 = open axis); dt: time step.
    """

    x: np.ndarray
    q: np.ndarray
    axes: np.ndarray
    vel: np.ndarray
    fext: np.ndarray
    box: np.ndarray
    dt: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations by Shoemake's subgroup method (Graphics Gems
    III, "Uniform random rotations"), returned as (s, w1, w2, w3)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                  a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def lattice_scene(seed: int = 0, n: int = 64, spacing: float = 2.5, box: float | None = None,
                  axes_range=(0.5, 1.0), vel_sigma: float = 1.0, omega_sigma: float = 0.5,
                  dt: float = 1e-3) -> Scene:
    """Ellipsoids on a cubic lattice in a periodic box.

    The smallest m with m^3 >= n gives an m x m x m lattice of spacing
    `spacing` (box side m * spacing unless given); the first n sites in
    i-major order are occupied.  Semi-axes U[axes_range], uniform random
    orientations, u ~ N(0, vel_sigma^2) per component and
    omega ~ N(0, omega_sigma^2) per component, no external force.
    With the defaults this is the 64-body, side-10 scene of the small
    inertial workload.
    """
    rng = np.random.default_rng(seed)
    m = 1
    while m ** 3 < n:
        m += 1
    side = m * spacing if box is None else box
    sites = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)], dtype=np.float64)
    x = (sites[:n] + 0.5) * spacing
    axes = rng.uniform(axes_range[0], axes_range[1], size=(n, 3))
    q = random_quaternions(rng, n)
    vel = np.concatenate([rng.normal(0.0, vel_sigma, size=(n, 3)),
                          rng.normal(0.0, omega_sigma, size=(n, 3))], axis=1)
    return Scene(x=x, q=q, axes=axes, vel=vel, fext=np.zeros((n, 6)), box=np.array([side] * 3, dtype=np.float64),
                 dt=float(dt), meta={"kind": "lattice", "seed": seed, "m": m})


def _rsa_positions(rng: np.random.Generator, radii: np.ndarray, side: float, max_attempts: int) -> np.ndarray:
    """Random sequential addition of spheres of the given radii (largest
    first) into a periodic cube, rejecting any overlap with earlier spheres."""
    n = radii.shape[0]
    rmax = float(radii.max())
    ncell = max(1, int(side // (2.0 * rmax)))
    csz = side / ncell
    grid: dict[tuple, list] = {}
    pos = np.zeros((n, 3))
    order = np.argsort(-radii, kind="stable")
    attempts = 0
    for idx in order:
        r = radii[idx]
        while True:
            attempts += 1
            if attempts > max_attempts:
                raise RuntimeError("random sequential addition did not finish")
            p = rng.random(3) * side
            c = (p // csz).astype(int) % ncell
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        key = ((c[0] + dx) % ncell, (c[1] + dy) % ncell, (c[2] + dz) % ncell)
                        for j in grid.get(key, ()):
                            d = pos[j] - p
                            d -= side * np.rint(d / side)
                            if d @ d < (r + radii[j]) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pos[idx] = p
                grid.setdefault((c[0], c[1], c[2]), []).append(idx)
                break
    return pos


def suspension_scene(seed: int = 1, n: int = 32768, phi: float = 0.1, axes_range=(0.4, 1.0),
                     dt: float = 5e-3, phi_final: float = 0.55, steps: int = 2000) -> Scene:
    """Compacting ellipsoid suspension (overdamped).

    n ellipsoids, semi-axes U[axes_range], uniform random orientations, placed
    by random sequential addition of their bounding spheres into a periodic
    cube whose side gives ellipsoid volume fraction `phi`.  meta carries the
    affine compaction schedule: box side shrinking geometrically so that the
    volume fraction reaches `phi_final` after `steps` steps of size dt, i.e. a
    constant strain rate  (r - 1)/dt  with  r = (phi/phi_final)^(1/(3 steps)).
    """
    rng = np.random.default_rng(seed)
    axes = rng.uniform(axes_range[0], axes_range[1], size=(n, 3))
    vol = float(np.sum(4.0 / 3.0 * np.pi * np.prod(axes, axis=1)))
    side = (vol / phi) ** (1.0 / 3.0)
    radii = axes.max(axis=1)
    x = _rsa_positions(rng, radii, side, max_attempts=200 * n)
    q = random_quaternions(rng, n)
    ratio = (phi / phi_final) ** (1.0 / (3.0 * steps))
    strain_rate = (ratio - 1.0) / dt
    return Scene(x=x, q=q, axes=axes, vel=np.zeros((n, 6)), fext=np.zeros((n, 6)),
                 box=np.array([side] * 3), dt=float(dt),
                 meta={"kind": "suspension", "seed": seed, "phi": phi, "phi_final": phi_final,
                       "steps": steps, "strain_rate": strain_rate, "volume": vol})


def batched_scenes(n_scenes: int = 2048, seed0: int = 1000, nmin: int = 2, nmax: int = 512,
                   dt_range=(1e-3, 1e-2)) -> list:
    """Independent lattice scenes of uneven size: scene s uses seed seed0+s,
    body count floor(exp(U[ln nmin, ln(nmax+1)))), box side 2.5 m with m the
    smallest integer with m^3 >= n, and dt ~ U[dt_range]."""
    out = []
    for s in range(n_scenes):
        rng = np.random.default_rng(seed0 + s)
        n = int(math.floor(math.exp(rng.uniform(math.log(nmin), math.log(nmax + 1)))))
        n = max(nmin, min(nmax, n))
        dt = float(rng.uniform(dt_range[0], dt_range[1]))
        out.append(lattice_scene(seed=seed0 + s, n=n, dt=dt))
    return out


def pack_scenes(scenes: list, precision_fp64: bool = False, eps_factor: float = 1e-3, skin_factor: float = 0.1):
    """Concatenate scenes for the batched entry points: (offsets, x, q, axes,
    vel, params) with params[s] = (box x, y, z, dt, eps_ncp, skin, lcp_tol,
    phi_skin).  Per scene, with a_min its smallest semi-axis: eps_ncp =
    eps_factor a_min, skin = phi_skin = skin_factor a_min, lcp_tol = 1e-12
    (FP64) or 1e-7 (mixed) times a_min."""
    offsets = np.zeros(len(scenes) + 1, dtype=np.int32)
    params = np.zeros((len(scenes), 8))
    for s, sc in enumerate(scenes):
        offsets[s + 1] = offsets[s] + sc.n
        amin = float(sc.axes.min()) if sc.n else 1.0
        params[s, 0:3] = sc.box
        params[s, 3] = sc.dt
        params[s, 4] = eps_factor * amin
        params[s, 5] = skin_factor * amin
        params[s, 6] = (1e-12 if precision_fp64 else 1e-7) * amin
        params[s, 7] = skin_factor * amin
    cat = lambda f, w: (np.concatenate([getattr(sc, f) for sc in scenes if sc.n]) if offsets[-1] else np.zeros((0, w)))
    return offsets, cat("x", 3), cat("q", 4), cat("axes", 3), cat("vel", 6), params


def two_ellipsoid_scene(offset_y: float = 2.5, force: float = 1.0) -> Scene:
    """Two identical ellipsoids with radii (1, 1, 2) rotated so that the long
    axis lies in the x-y plane at 45 degrees, centres one unit apart in x and
    separated in y, pushed together by equal and opposite unit forces along y
    (the refinement study of Sec. 5.2; the paper does not give the vertical
    offset, which is a parameter here).  Open (non-periodic) box."""
    # long axis (body z) rotated into the x-y plane at 45 degrees: rotate by
    # 90 degrees about x (body z -> world -y), then 45 degrees about z.
    def qmul(a, b):
        s1, v1 = a[0], np.array(a[1:])
        s2, v2 = b[0], np.array(b[1:])
        return np.concatenate([[s1 * s2 - v1 @ v2], s1 * v2 + s2 * v1 + np.cross(v1, v2)])

    qx = np.array([math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0])
    qz = np.array([math.cos(math.pi / 8), 0.0, 0.0, math.sin(math.pi / 8)])
    q0 = qmul(qz, qx)
    q = np.stack([q0, q0])
    x = np.array([[0.0, offset_y / 2, 0.0], [1.0, -offset_y / 2, 0.0]])
    axes = np.array([[1.0, 1.0, 2.0], [1.0, 1.0, 2.0]])
    fext = np.zeros((2, 6))
    fext[0, 1] = -force
    fext[1, 1] = force
    return Scene(x=x, q=q, axes=axes, vel=np.zeros((2, 6)), fext=fext, box=np.zeros(3), dt=1e-2,
                 meta={"kind": "two_ellipsoids"})


def sphere_scene(seed: int, n: int, side: float, radius_range=(0.5, 1.0), vel_sigma: float = 1.0) -> Scene:
    """Spheres (equal semi-axes) by random sequential addition; used for the
    sphere-only pins."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(radius_range[0], radius_range[1], size=n)
    x = _rsa_positions(rng, r, side, max_attempts=500 * n)
    axes = np.repeat(r[:, None], 3, axis=1)
    q = random_quaternions(rng, n)
    vel = np.concatenate([rng.normal(0.0, vel_sigma, size=(n, 3)), np.zeros((n, 3))], axis=1)
    return Scene(x=x, q=q, axes=axes, vel=vel, fext=np.zeros((n, 6)), box=np.array([side] * 3), dt=1e-3,
                 meta={"kind": "spheres", "seed": seed})


def planar_quaternions(theta: np.ndarray) -> np.ndarray:
    """(s, w) quaternions of rotations by theta about the z axis."""
    theta = np.asarray(theta, dtype=np.float64)
    return np.stack([np.cos(0.5 * theta), np.zeros_like(theta), np.zeros_like(theta), np.sin(0.5 * theta)], axis=1)


def planar_angle(q: np.ndarray) -> np.ndarray:
    """Rotation angle about z of (s, w) quaternions that rotate about z."""
    q = np.asarray(q, dtype=np.float64)
    return 2.0 * np.arctan2(q[:, 3], q[:, 0])


class Colony:
    """Growing colony of prolate ellipsoidal cells in the z = 0 plane (the
    paper's Sec. 5.4 colony, restated with ellipsoids).

    Cell i has length L_i and semi-axes (L_i/2, 0.5, 0.5), its long axis the
    body x axis, in the plane.  Each cell draws its growth rate once, at birth,
    from N(rate, rate_sd) (length per unit time).  After every time step the
    host loop advances L_i by rate_i dt; a cell that reaches L_div divides along
    its axis into two daughters of length L_i / 2 centred at c +- (L_i / 4) e,
    each turned by its own N(0, jitter) angle.  All random numbers come from
    the colony's own seeded generator, so a colony is a pure function of its
    seed and of the positions and angles the solver returns.  This is input
    preparation (the scene), not the contact method."""

    def __init__(self, seed: int = 0, rate: float = 0.01, rate_sd: float = 0.001, jitter: float = 0.05,
                 L0: float = 1.0, L_div: float = 2.0, dt: float = 0.05):
        self.rng = np.random.default_rng(seed)
        self.rate, self.rate_sd, self.jitter = rate, rate_sd, jitter
        self.L_div, self.dt = L_div, dt
        self.x = np.zeros((1, 3))
        self.theta = np.zeros(1)
        self.L = np.array([L0], dtype=np.float64)
        self.g = self._rates(1)
        self.divisions = 0

    def _rates(self, k: int) -> np.ndarray:
        return np.maximum(self.rng.normal(self.rate, self.rate_sd, size=k), 0.0)

    @property
    def n(self) -> int:
        return int(self.L.shape[0])

    def axes(self) -> np.ndarray:
        a = np.full((self.n, 3), 0.5)
        a[:, 0] = 0.5 * self.L
        return a

    def q(self) -> np.ndarray:
        return planar_quaternions(self.theta)

    def advance(self, x: np.ndarray, q: np.ndarray) -> int:
        """Take the solver's accepted positions and orientations, grow every
        cell by one step and divide those at L_div.  Returns the number of
        divisions."""
        self.x = np.array(x, dtype=np.float64, copy=True)
        self.x[:, 2] = 0.0
        self.theta = planar_angle(q)
        self.L = self.L + self.g * self.dt
        idx = np.nonzero(self.L >= self.L_div)[0]
        if idx.size == 0:
            return 0
        e = np.stack([np.cos(self.theta[idx]), np.sin(self.theta[idx]), np.zeros(idx.size)], axis=1)
        off = (0.25 * self.L[idx])[:, None] * e
        Ld = 0.5 * self.L[idx]
        jit = self.rng.normal(0.0, self.jitter, size=(idx.size, 2))
        # daughter 1 replaces the mother, daughter 2 is appended
        x2 = self.x[idx] + off
        self.x[idx] = self.x[idx] - off
        th2 = self.theta[idx] + jit[:, 1]
        self.theta[idx] = self.theta[idx] + jit[:, 0]
        self.L[idx] = Ld
        self.g[idx] = self._rates(idx.size)
        self.x = np.concatenate([self.x, x2])
        self.theta = np.concatenate([self.theta, th2])
        self.L = np.concatenate([self.L, Ld])
        self.g = np.concatenate([self.g, self._rates(idx.size)])
        self.divisions += int(idx.size)
        return int(idx.size)
