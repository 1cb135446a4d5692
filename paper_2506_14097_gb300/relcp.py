"""Python binding of the ReLCP C ABI (include/relcp.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all steps run in librelcp.so's CUDA kernels.
Host arrays are numpy float64 / int32; device arrays are torch CUDA tensors
(PyTorch provides device memory and the stream).  There is no CPU fallback:
load() raises when the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int32, c_int64, c_uint32, c_uint64, c_void_p

import numpy as np

from . import build as _build

RELCP_OK = 0
RELCP_ERR_INVALID_ARG = 1
RELCP_ERR_CUDA = 2
RELCP_ERR_CAPACITY = 3
RELCP_ERR_NOT_CONVERGED = 4
RELCP_ERR_RECURSION_LIMIT = 5
RELCP_ERR_NEWTON = 6
RELCP_ERR_TIMEOUT = 7
RELCP_ERR_STATE = 8
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "CAPACITY", 4: "NOT_CONVERGED", 5: "RECURSION_LIMIT",
                6: "NEWTON", 7: "TIMEOUT", 8: "STATE"}

RELCP_INERTIAL, RELCP_OVERDAMPED, RELCP_OVERDAMPED_2D = 0, 1, 2
RELCP_FP64, RELCP_MIXED = 0, 1
RELCP_GUESS_COLD, RELCP_GUESS_MLP = 0, 1
RELCP_PTR_HOST, RELCP_PTR_DEVICE = 0, 1
RELCP_SHAPE_ELLIPSOID, RELCP_SHAPE_SPHEROCYLINDER = 0, 1
RELCP_FAULT_ROW_CAPACITY, RELCP_FAULT_LCP_ITERS, RELCP_FAULT_LCP_TIMEOUT, RELCP_FAULT_NEWTON_ITERS = 1, 2, 4, 8
RELCP_FLAG_PHASE_TIMING = 1
RELCP_FLAG_NO_WARM_START = 2
RELCP_FLAG_JACOBI = 4
RELCP_FLAG_NO_SNSD_REUSE = 8
RELCP_FLAG_LCP_TIMING = 16
RELCP_FLAG_GRAPH = 32
RELCP_FLAG_HOST_STAGING = 64
RELCP_FLAG_LEARNED_ALWAYS = 128
RELCP_FLAG_NO_LCP_REFINE = 256
MAX_DEPTH_STATS = 64


class relcp_config(ctypes.Structure):
    _fields_ = [("dynamics", c_int32), ("precision", c_int32), ("guess", c_int32), ("lcp_max_iter", c_int32),
                ("max_recursion", c_int32), ("n_scenes", c_int32), ("dt", c_double), ("eps_ncp", c_double),
                ("box", c_double * 3), ("skin", c_double), ("phi_skin", c_double), ("drag_xi", c_double),
                ("density", c_double), ("strain_rate", c_double), ("lcp_tol", c_double), ("seed", c_uint64),
                ("fault_inject", c_uint32), ("flags", c_uint32), ("shape", c_int32), ("reserved", c_int32)]


class relcp_step_stats(ctypes.Structure):
    _fields_ = [("n_bodies", c_int64), ("n_pairs", c_int64), ("n_rows", c_int64), ("n_rows0", c_int64),
                ("depth", c_int32), ("status", c_int32), ("lcp_iters_total", c_int32), ("newton_iters_max", c_int32),
                ("lcp_iters", c_int32 * MAX_DEPTH_STATS), ("rows_per_rec", c_int32 * MAX_DEPTH_STATS),
                ("lcp_residual", c_double), ("max_overlap", c_double), ("box", c_double * 3),
                ("ms_broadphase", c_double), ("ms_snsd", c_double), ("ms_lcp", c_double), ("ms_augment", c_double),
                ("ms_total", c_double), ("steps_done", c_int64), ("guess_used", c_int32),
                ("newton_fallbacks", c_int32), ("ms_lcp_kernel", c_double), ("lcp_alg_bytes", c_double),
                ("ms_snsd_kernel", c_double), ("snsd_evals", c_int64), ("lcp_launches", c_int32),
                ("snsd_launches", c_int32), ("pair_list_rebuilt", c_int32), ("graph_replayed", c_int32),
                ("newton_iters_c0", c_int64), ("snsd_c0_evaluated", c_int64),
                ("host_ms", c_double), ("host_wait_ms", c_double)]


class relcp_lcp_info(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("status", c_int32), ("residual", c_double), ("grid_blocks", c_int32),
                ("one_barrier", c_int32)]


MLP_IN, MLP_HID, MLP_OUT = 16, 128, 8
MLP_CORR_SCALE = 32.0
MLP_NPARAMS = 128 * 16 + 128 + 128 * 128 + 128 + 128 * 128 + 128 + 8 * 128 + 8


class relcp_mlp_train_config(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("w_phi", ctypes.c_float), ("w_trust", ctypes.c_float), ("trust_tol", ctypes.c_float),
                ("step", c_int32)]


class RelcpError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({msg})")
        self.status = status


_lib = None
EXPORTS = ["relcp_last_error", "relcp_kernel_launches", "relcp_version", "relcp_create", "relcp_set_config", "relcp_set_bodies",
           "relcp_step", "relcp_get_bodies", "relcp_get_box", "relcp_stats", "relcp_get_pairs", "relcp_get_rows",
           "relcp_get_contact_velocity", "relcp_destroy", "relcp_broadphase", "relcp_snsd_eval", "relcp_lcp_solve",
           "relcp_snsd_eval_noalloc", "relcp_mlp_features", "relcp_mlp_forward", "relcp_mlp_train_step",
           "relcp_load_mlp", "relcp_batch_create", "relcp_batch_set_scenes", "relcp_batch_step",
           "relcp_batch_get_bodies", "relcp_batch_scene_stats", "relcp_batch_get_scene_contacts",
           "relcp_batch_autotune", "relcp_batch_set_threads", "relcp_batch_destroy"]


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load librelcp.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"librelcp.so not found at {path}: build it with paper_2506_14097_gb300.build")
    L = ctypes.CDLL(path)
    L.relcp_last_error.restype = c_char_p
    L.relcp_last_error.argtypes = []
    sigs = {
        "relcp_version": [POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)],
        "relcp_create": [POINTER(relcp_config), c_void_p, POINTER(c_void_p)],
        "relcp_set_config": [c_void_p, POINTER(relcp_config)],
        "relcp_set_bodies": [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                             c_int32],
        "relcp_step": [c_void_p, c_int32],
        "relcp_get_bodies": [c_void_p, c_void_p, c_void_p, c_void_p, c_int32],
        "relcp_get_box": [c_void_p, c_void_p],
        "relcp_stats": [c_void_p, POINTER(relcp_step_stats)],
        "relcp_get_pairs": [c_void_p, c_void_p, c_void_p, c_int64, POINTER(c_int64), c_int32],
        "relcp_get_rows": [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, POINTER(c_int64), c_int32],
        "relcp_get_contact_velocity": [c_void_p, c_void_p, c_int32],
        "relcp_broadphase": [c_int64, c_void_p, c_void_p, c_void_p, c_double, c_void_p, c_int64, POINTER(c_int64),
                             c_void_p],
        "relcp_snsd_eval": [c_int64, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                            c_void_p, c_void_p],
        "relcp_lcp_solve": [c_int64, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int32,
                            c_double, c_int32, c_void_p, c_void_p, POINTER(relcp_lcp_info), c_void_p],
        "relcp_snsd_eval_noalloc": [c_int64, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                    c_void_p, c_void_p, c_void_p],
        "relcp_mlp_features": [c_int64, c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p],
        "relcp_mlp_forward": [c_int64, c_void_p, c_void_p, c_void_p, c_void_p],
        "relcp_mlp_train_step": [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                 POINTER(relcp_mlp_train_config), c_void_p, POINTER(c_double), c_void_p],
        "relcp_load_mlp": [c_void_p, c_void_p, c_int32],
        "relcp_batch_create": [POINTER(relcp_config), c_void_p, POINTER(c_void_p)],
        "relcp_batch_set_scenes": [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_int32],
        "relcp_batch_step": [c_void_p, c_int32],
        "relcp_batch_get_bodies": [c_void_p, c_void_p, c_void_p, c_void_p, c_int32],
        "relcp_batch_scene_stats": [c_void_p, c_void_p],
        "relcp_batch_get_scene_contacts": [c_void_p, c_int32, c_void_p, c_int64, POINTER(c_int64), c_void_p, c_int64,
                                           POINTER(c_int64)],
        "relcp_batch_autotune": [c_void_p, c_char_p, POINTER(c_int32)],
        "relcp_batch_set_threads": [c_void_p, c_int32],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = c_int32
    L.relcp_destroy.argtypes = [c_void_p]
    L.relcp_destroy.restype = None
    L.relcp_batch_destroy.argtypes = [c_void_p]
    L.relcp_batch_destroy.restype = None
    L.relcp_kernel_launches.argtypes = []
    L.relcp_kernel_launches.restype = c_int64
    _lib = L
    return L


def relcp_kernel_launches() -> int:
    return int(load().relcp_kernel_launches())


def last_error() -> str:
    return load().relcp_last_error().decode()


def _check(st: int, where: str, allow=()):
    if st != RELCP_OK and st not in allow:
        raise RelcpError(st, where, last_error())
    return st


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _kind(a):
    return RELCP_PTR_DEVICE if (a is not None and hasattr(a, "is_cuda") and a.is_cuda) else RELCP_PTR_HOST


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def make_config(dynamics=RELCP_INERTIAL, precision=RELCP_FP64, guess=RELCP_GUESS_COLD, dt=1e-3, eps_ncp=1e-3,
                box=(0.0, 0.0, 0.0), skin=0.05, phi_skin=None, drag_xi=1.0, density=1.0, strain_rate=0.0,
                lcp_tol=None, lcp_max_iter=20000, max_recursion=64, seed=0, fault_inject=0, flags=0, length_scale=None,
                shape=RELCP_SHAPE_ELLIPSOID):
    """A relcp_config.  lcp_tol defaults to `length_scale` (default:
    eps_ncp / 1e-3, i.e. the smallest semi-axis when eps_ncp = 1e-3 x a_min)
    times 1e-12 on the FP64 path; on the mixed path times 1e-8 for the
    overdamped laws and 1e-7 for inertial dynamics.  Those are the stops at
    which each path's step meets its error bound against the exact LCP
    solution (relative 1e-9 and 1e-5): the error of a stopped
    projected-gradient iterate follows the stop, not the arithmetic, and in an
    overdamped compaction the contact velocity is the whole non-affine motion
    (a stop of 1e-7 a_min leaves up to 4e-5 there, in FP64 as in FP32).  Under
    inertia the velocity is mostly free motion, 1e-7 a_min meets the bound, and
    FP32 iterates cannot resolve 1e-8 a_min when the bodies move far per step
    (the solve stalls at its rounding floor and reports NOT_CONVERGED); an
    overdamped step with a large strain per step stalls the same way and needs
    an explicit lcp_tol."""
    c = relcp_config()
    c.dynamics, c.precision, c.guess = dynamics, precision, guess
    c.lcp_max_iter, c.max_recursion, c.n_scenes = lcp_max_iter, max_recursion, 1
    c.dt, c.eps_ncp = dt, eps_ncp
    for k in range(3):
        c.box[k] = float(box[k])
    c.skin = skin
    c.phi_skin = skin if phi_skin is None else phi_skin
    c.drag_xi, c.density, c.strain_rate = drag_xi, density, strain_rate
    scale = (eps_ncp / 1e-3) if length_scale is None else length_scale
    c.lcp_tol = lcp_tol if lcp_tol is not None else (1e-12 if precision == RELCP_FP64 else (1e-7 if dynamics == RELCP_INERTIAL else 1e-8)) * scale
    c.seed, c.fault_inject, c.flags = seed, fault_inject, flags
    c.shape, c.reserved = shape, 0
    return c


# ---------------------------------------------------------------------------
# context API (same names as the C ABI)
# ---------------------------------------------------------------------------
def relcp_create(cfg: relcp_config, stream=None) -> c_void_p:
    L = load()
    h = c_void_p()
    _check(L.relcp_create(byref(cfg), c_void_p(_stream(stream)), byref(h)), "relcp_create")
    return h


def relcp_set_config(ctx, cfg: relcp_config):
    _check(load().relcp_set_config(ctx, byref(cfg)), "relcp_set_config")


def relcp_set_bodies(ctx, x, q, semi_axes, vel=None, f_ext=None):
    n = int(x.shape[0])
    kind = _kind(x)
    _check(load().relcp_set_bodies(ctx, n, None, _ptr(x), _ptr(q), _ptr(semi_axes), _ptr(vel), _ptr(f_ext), None,
                                   kind), "relcp_set_bodies")


def relcp_step(ctx, nsteps: int = 1, allow=()):
    return _check(load().relcp_step(ctx, int(nsteps)), "relcp_step", allow)


def relcp_get_bodies(ctx, x=None, q=None, vel=None):
    kind = _kind(x if x is not None else (q if q is not None else vel))
    _check(load().relcp_get_bodies(ctx, _ptr(x), _ptr(q), _ptr(vel), kind), "relcp_get_bodies")


def relcp_get_box(ctx) -> np.ndarray:
    b = np.zeros(3)
    _check(load().relcp_get_box(ctx, _ptr(b)), "relcp_get_box")
    return b


def relcp_stats(ctx) -> relcp_step_stats:
    s = relcp_step_stats()
    _check(load().relcp_stats(ctx, byref(s)), "relcp_stats")
    return s


def relcp_get_pairs(ctx):
    """(pairs (P, 2) int32, phi0 (P,)) of the last step, host arrays."""
    n = c_int64(0)
    L = load()
    st = L.relcp_get_pairs(ctx, None, None, 0, byref(n), RELCP_PTR_HOST)
    _check(st, "relcp_get_pairs", allow=(RELCP_ERR_CAPACITY,))
    P = n.value
    pairs = np.zeros((max(P, 1), 2), dtype=np.int32)
    phi = np.zeros(max(P, 1))
    _check(L.relcp_get_pairs(ctx, _ptr(pairs), _ptr(phi), P, byref(n), RELCP_PTR_HOST), "relcp_get_pairs")
    return pairs[:P], phi[:P]


def relcp_get_rows(ctx):
    """(ids (m, 4) int32 [a, b, recursion, pair], geom (m, 11), gamma (m,))."""
    n = c_int64(0)
    L = load()
    _check(L.relcp_get_rows(ctx, None, None, None, 0, byref(n), RELCP_PTR_HOST), "relcp_get_rows",
           allow=(RELCP_ERR_CAPACITY,))
    m = n.value
    ids = np.zeros((max(m, 1), 4), dtype=np.int32)
    geom = np.zeros((max(m, 1), 11))
    gam = np.zeros(max(m, 1))
    _check(L.relcp_get_rows(ctx, _ptr(ids), _ptr(geom), _ptr(gam), m, byref(n), RELCP_PTR_HOST), "relcp_get_rows")
    return ids[:m], geom[:m], gam[:m]


def relcp_get_contact_velocity(ctx, n: int) -> np.ndarray:
    uc = np.zeros((max(n, 1), 6))
    _check(load().relcp_get_contact_velocity(ctx, _ptr(uc), RELCP_PTR_HOST), "relcp_get_contact_velocity")
    return uc[:n]


def relcp_destroy(ctx):
    if ctx:
        load().relcp_destroy(ctx)


# ---------------------------------------------------------------------------
# stateless entry points (device tensors)
# ---------------------------------------------------------------------------
def relcp_broadphase(x, rb, box, skin: float, cap: int | None = None, stream=None):
    """x (n,3), rb (n,) float64 CUDA tensors -> pairs (P, 2) int32 CUDA tensor."""
    import torch

    n = int(x.shape[0])
    box_h = np.ascontiguousarray(box, dtype=np.float64)
    cap = max(16, 64 * n) if cap is None else cap
    L = load()
    while True:
        pairs = torch.empty((cap, 2), dtype=torch.int32, device=x.device)
        npairs = c_int64(0)
        st = L.relcp_broadphase(n, _ptr(x), _ptr(rb), _ptr(box_h), float(skin), _ptr(pairs), cap, byref(npairs),
                                c_void_p(_stream(stream)))
        if st == RELCP_ERR_CAPACITY:
            cap = int(npairs.value)
            continue
        _check(st, "relcp_broadphase")
        return pairs[: npairs.value]


def relcp_snsd_eval(pairs, x, q, axes, box, precision=RELCP_FP64, stream=None, allow=()):
    """SNSD of every pair: returns (out (P, 10) = phi, n, r_a, r_b; iters (P,))
    as CUDA tensors."""
    import torch

    P = int(pairs.shape[0])
    out = torch.empty((max(P, 1), 10), dtype=torch.float64, device=x.device)
    iters = torch.empty(max(P, 1), dtype=torch.int32, device=x.device)
    box_h = np.ascontiguousarray(box, dtype=np.float64)
    st = load().relcp_snsd_eval(P, _ptr(pairs), int(x.shape[0]), _ptr(x), _ptr(q), _ptr(axes), _ptr(box_h),
                                int(precision), _ptr(out), _ptr(iters), c_void_p(_stream(stream)))
    _check(st, "relcp_snsd_eval", allow)
    return out[:P], iters[:P]


NOALLOC_MAX_BODIES = 65536


def relcp_snsd_eval_noalloc(pairs, x, q, axes, box, out, iters=None, precision=RELCP_FP64, stream=None, allow=()):
    """Allocation-free SNSD evaluation into caller-provided device buffers
    `out` (P, 10) float64 and `iters` (P,) int32 (or None).  Same results as
    relcp_snsd_eval; see include/relcp.h for the scratch rules."""
    P = int(pairs.shape[0])
    box_h = np.ascontiguousarray(box, dtype=np.float64)
    st = load().relcp_snsd_eval_noalloc(P, _ptr(pairs), int(x.shape[0]), _ptr(x), _ptr(q), _ptr(axes), _ptr(box_h),
                                        int(precision), _ptr(out), _ptr(iters), c_void_p(_stream(stream)))
    return _check(st, "relcp_snsd_eval_noalloc", allow)


def relcp_lcp_solve(ia, ib, geom, qv, K, c: float, gamma=None, precision=RELCP_FP64, tol=1e-12, max_iter=100000,
                    stream=None, allow=()):
    """Matrix-free LCP; returns (gamma, uc, info).  Inputs are CUDA tensors:
    ia, ib (m,) int32; geom (m, 9); qv (m,); K (nbodies, 7) float64."""
    import torch

    m = int(ia.shape[0])
    nb = int(K.shape[0])
    if gamma is None:
        gamma = torch.zeros(max(m, 1), dtype=torch.float64, device=K.device)
    else:
        gamma = gamma.clone()
    uc = torch.empty((max(nb, 1), 6), dtype=torch.float64, device=K.device)
    info = relcp_lcp_info()
    st = load().relcp_lcp_solve(m, nb, _ptr(ia), _ptr(ib), _ptr(geom), _ptr(qv), _ptr(K), float(c), int(precision),
                                float(tol), int(max_iter), _ptr(gamma), _ptr(uc), byref(info),
                                c_void_p(_stream(stream)))
    _check(st, "relcp_lcp_solve", allow)
    return gamma[:m], uc[:nb], info


# ---------------------------------------------------------------------------
# learned SNSD guess (device tensors)
# ---------------------------------------------------------------------------
def relcp_mlp_features(pairs, x, q, axes, box, snsd_out=None, stream=None):
    """(feat (P, 16) float32, targets (P, 4) float32 or None) on the device."""
    import torch

    P = int(pairs.shape[0])
    feat = torch.empty((max(P, 1), MLP_IN), dtype=torch.float32, device=x.device)
    targets = torch.empty((max(P, 1), 4), dtype=torch.float32, device=x.device) if snsd_out is not None else None
    box_h = np.ascontiguousarray(box, dtype=np.float64)
    st = load().relcp_mlp_features(P, _ptr(pairs), int(x.shape[0]), _ptr(x), _ptr(q), _ptr(axes), _ptr(box_h),
                                   _ptr(snsd_out), _ptr(feat), _ptr(targets), c_void_p(_stream(stream)))
    _check(st, "relcp_mlp_features")
    return feat[:P], (targets[:P] if targets is not None else None)


def relcp_mlp_forward(params, feat, stream=None):
    import torch

    P = int(feat.shape[0])
    out = torch.empty((max(P, 1), MLP_OUT), dtype=torch.float32, device=feat.device)
    _check(load().relcp_mlp_forward(P, _ptr(params), _ptr(feat), _ptr(out), c_void_p(_stream(stream))),
           "relcp_mlp_forward")
    return out[:P]


def relcp_mlp_train_step(params, m, v, feat, targets, cfg: relcp_mlp_train_config, grad=None, stream=None) -> float:
    loss = c_double(0.0)
    st = load().relcp_mlp_train_step(int(feat.shape[0]), _ptr(params), _ptr(m), _ptr(v), _ptr(feat), _ptr(targets),
                                     byref(cfg), _ptr(grad), byref(loss), c_void_p(_stream(stream)))
    _check(st, "relcp_mlp_train_step")
    return float(loss.value)


def relcp_load_mlp(ctx, params):
    _check(load().relcp_load_mlp(ctx, _ptr(params), _kind(params)), "relcp_load_mlp")


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Simulation:
    """A context holding one scene: create, set bodies, step, read back."""

    def __init__(self, cfg: relcp_config, stream=None):
        self.cfg = cfg
        self.ctx = relcp_create(cfg, stream)
        self.n = 0

    def set_bodies(self, x, q, axes, vel=None, fext=None):
        self.n = int(x.shape[0])
        relcp_set_bodies(self.ctx, x, q, axes, vel, fext)

    def step(self, nsteps=1, allow=()):
        return relcp_step(self.ctx, nsteps, allow)

    def bodies(self):
        x = np.zeros((self.n, 3))
        q = np.zeros((self.n, 4))
        v = np.zeros((self.n, 6))
        relcp_get_bodies(self.ctx, x, q, v)
        return x, q, v

    def stats(self):
        return relcp_stats(self.ctx)

    def close(self):
        if self.ctx:
            relcp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# batched scenes
# ---------------------------------------------------------------------------
BATCH_MAX_BODIES = 1024
SCENE_PARAMS = 8


class relcp_scene_stats(ctypes.Structure):
    _fields_ = [("status", c_int32), ("status_bits", c_int32), ("steps_done", c_int32), ("depth_max", c_int32),
                ("lcp_iters", c_int32), ("n_pairs", c_int32), ("n_rows", c_int32), ("aug_steps", c_int32),
                ("max_overlap", c_double), ("lcp_residual", c_double), ("max_overlap_all", c_double)]


def relcp_batch_create(cfg: relcp_config, stream=None):
    h = c_void_p()
    _check(load().relcp_batch_create(byref(cfg), c_void_p(_stream(stream)), byref(h)), "relcp_batch_create")
    return h


def relcp_batch_set_scenes(b, offsets, x, q, axes, vel, fext, params):
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    x, q, axes, params = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, q, axes, params))
    vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
    fext = None if fext is None else np.ascontiguousarray(fext, dtype=np.float64)
    _check(load().relcp_batch_set_scenes(b, int(offsets.shape[0] - 1), _ptr(offsets), _ptr(x), _ptr(q), _ptr(axes),
                                         _ptr(vel), _ptr(fext), _ptr(params), RELCP_PTR_HOST),
           "relcp_batch_set_scenes")


def relcp_batch_step(b, nsteps=1, allow=()):
    return _check(load().relcp_batch_step(b, int(nsteps)), "relcp_batch_step", allow)


def relcp_batch_get_bodies(b, x, q, vel):
    _check(load().relcp_batch_get_bodies(b, _ptr(x), _ptr(q), _ptr(vel), RELCP_PTR_HOST), "relcp_batch_get_bodies")


def relcp_batch_scene_stats(b, n_scenes):
    out = (relcp_scene_stats * n_scenes)()
    _check(load().relcp_batch_scene_stats(b, ctypes.cast(out, c_void_p)), "relcp_batch_scene_stats")
    return list(out)


def relcp_batch_get_scene_contacts(b, scene):
    """(pairs (P, 2) int32, row ids (m, 4) int32 = a, b, recursion, pair) of
    the scene's last step, host arrays."""
    L = load()
    n_p, n_r = c_int64(0), c_int64(0)
    _check(L.relcp_batch_get_scene_contacts(b, int(scene), None, 0, byref(n_p), None, 0, byref(n_r)),
           "relcp_batch_get_scene_contacts")
    pairs = np.zeros((max(n_p.value, 1), 2), dtype=np.int32)
    ids = np.zeros((max(n_r.value, 1), 4), dtype=np.int32)
    _check(L.relcp_batch_get_scene_contacts(b, int(scene), _ptr(pairs), n_p.value, byref(n_p), _ptr(ids), n_r.value,
                                            byref(n_r)), "relcp_batch_get_scene_contacts")
    return pairs[:n_p.value], ids[:n_r.value]


def relcp_batch_autotune(b, cache_path=None):
    t = c_int32(0)
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(load().relcp_batch_autotune(b, path, byref(t)), "relcp_batch_autotune")
    return int(t.value)


def relcp_batch_set_threads(b, threads):
    _check(load().relcp_batch_set_threads(b, int(threads)), "relcp_batch_set_threads")


def relcp_batch_destroy(b):
    load().relcp_batch_destroy(b)


class Batch:
    """Many independent scenes stepped by one persistent launch."""

    def __init__(self, cfg: relcp_config, stream=None):
        self.cfg = cfg
        self.h = relcp_batch_create(cfg, stream)
        self.offsets = None

    def set_scenes(self, offsets, x, q, axes, params, vel=None, fext=None):
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int32)
        relcp_batch_set_scenes(self.h, self.offsets, x, q, axes, vel, fext, params)

    def step(self, nsteps=1, allow=()):
        return relcp_batch_step(self.h, nsteps, allow)

    def bodies(self):
        n = int(self.offsets[-1])
        x, q, v = np.zeros((n, 3)), np.zeros((n, 4)), np.zeros((n, 6))
        relcp_batch_get_bodies(self.h, x, q, v)
        return x, q, v

    def scene_stats(self):
        return relcp_batch_scene_stats(self.h, len(self.offsets) - 1)

    def contacts(self, scene):
        return relcp_batch_get_scene_contacts(self.h, scene)

    def autotune(self, cache_path=None):
        return relcp_batch_autotune(self.h, cache_path)

    def set_threads(self, threads):
        relcp_batch_set_threads(self.h, threads)

    def close(self):
        if self.h:
            relcp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
