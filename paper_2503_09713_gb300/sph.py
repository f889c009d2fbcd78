"""Python binding of the C ABI in ``include/sph.h`` (ctypes; argument marshalling only).

Every computation runs in ``libsph_gb300.so``.  The module refuses to work without it: there is no
CPU fallback.  Device memory comes from PyTorch tensors (``DeviceState``); the library receives their
raw pointers and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsph_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "sph.h")

SPH_OK = 0
SPH_ERR_INVALID_ARG = -1
SPH_ERR_OOM = -2
SPH_ERR_CAPACITY = -3
SPH_ERR_CACHE_STALE = -4
SPH_ERR_H_NOT_CONVERGED = -5
SPH_ERR_TIMEOUT = -6
SPH_ERR_CUDA = -7
SPH_ERR_ORDER = -8
SPH_ERR_NONFINITE = -9
SPH_KERNEL_M4 = 0
SPH_KERNEL_M5 = 1
SPH_KERNEL_M6 = 2
SPH_KERNEL_C2 = 3
SPH_KERNEL_C4 = 4
SPH_KERNEL_C6 = 5
SPH_FP64 = 0
SPH_MIXED = 1

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho", "omega", "vsig")

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


class sph_params(ctypes.Structure):
    _fields_ = [("kernel", _i), ("precision", _i), ("hfact", _d), ("gamma", _d), ("alpha_av", _d),
                ("beta_av", _d), ("alpha_u", _d), ("c_cour", _d), ("c_force", _d), ("h_tol", _d),
                ("h_clamp", _d), ("cache_tol", _d), ("h_max_iter", _i), ("reduction_level", _i),
                ("periodic", _i), ("max_outer", _i), ("box_lo", _d * 3), ("box_hi", _d * 3),
                ("morton_bits", _i), ("av_switch", _i), ("max_corr", _i), ("alpha_min", _d),
                ("sigma_decay", _d), ("eps_v", _d), ("lambda_stiff", _d)]


class sph_state(ctypes.Structure):
    _fields_ = [("n", _i64), ("mass", _d)] + [(f, _p) for f in FIELDS] + [("id", _p), ("alpha", _p)]


class sph_tree_view(ctypes.Structure):
    _fields_ = [(f, _p) for f in ("mu", "perm", "leaf_first", "mu_leaf", "lchild", "rchild", "lflag", "rflag",
                                  "endrange", "bmin", "bmax", "hmax", "group_start")]


class sph_stats(ctypes.Structure):
    _fields_ = [("n", _i64), ("n_leaves", _i64), ("n_groups", _i64), ("n_pairs", _i64), ("cache_slots", _i64),
                ("cand_chunks", _i64),
                ("density_iters_max", _i), ("outer_passes", _i), ("n_red", _i), ("dt_next", _d), ("dv_ratio", _d),
                ("kernel_launches", _i64), ("density_pair_evals", _i64), ("density_inrange", _i64), ("force_pairs", _i64), ("stage_ms", _d * 8),
                ("cfl_multiplier", _d), ("corrector_passes", _i), ("graph_replays", _i64),
                ("graph_captures", _i64), ("graph_fallbacks", _i64)]

class sph_launch(ctypes.Structure):
    _fields_ = [("density_block", _i), ("forces_block", _i), ("walk_block", _i), ("stage2_warps", _i),
                ("reduction_level", _i)]


STAGES = ("predict", "tree", "neighbours", "density", "force_prep", "forces", "correct", "switch")


class SPHError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lib = None


def load():
    """Load the CUDA library (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(the SPH path has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "sph_default_params": (None, [P(sph_params)]),
        "sph_create": (_i, [P(sph_params), _i64, _i64, _p, P(_p)]),
        "sph_destroy": (_i, [_p]),
        "sph_batch_create": (_i, [P(sph_params), _i, _p, _p, _p, _i64, _p, P(_p)]),
        "sph_batch_dt": (_i, [_p, _p]),
        "sph_set_params": (_i, [_p, P(sph_params)]),
        "sph_build_tree": (_i, [_p, P(sph_state)]),
        "sph_find_neighbours": (_i, [_p, P(sph_state), P(_i64)]),
        "sph_compute_density_h": (_i, [_p, P(sph_state), P(_i)]),
        "sph_compute_forces": (_i, [_p, P(sph_state)]),
        "sph_step": (_i, [_p, P(sph_state), _d, P(_d), P(_d)]),
        "sph_step_host": (_i, [_p, P(sph_state), _d, P(_d), P(_d)]),
        "sph_tree_sizes": (_i, [_p, P(_i64), P(_i64)]),
        "sph_export_tree": (_i, [_p, P(sph_tree_view)]),
        "sph_export_neighbours": (_i, [_p, _p, _p]),
        "sph_get_stats": (_i, [_p, P(sph_stats)]),
        "sph_set_timing": (_i, [_p, _i]),
        "sph_set_graph": (_i, [_p, _i]),
        "sph_reset_timing": (_i, [_p]),
        "sph_get_launch": (_i, [_p, P(sph_launch)]),
        "sph_set_launch": (_i, [_p, P(sph_launch)]),
        "sph_autotune": (_i, [_p, P(sph_state), P(sph_launch), P(_d)]),
        "sph_sort_morton_noalloc": (_i, [_i64, _p, _p, _p, P(_d * 3), P(_d * 3), _p, _p, _p]),
        "sph_debug_wait_timeout": (_i, [_p, P(sph_state), _i, ctypes.c_uint32]),
        "sph_last_error": (ctypes.c_char_p, [_p]),
        "sph_error_string": (ctypes.c_char_p, [_i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def header_functions() -> list:
    """Names of the functions declared in include/sph.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sph_\w+)\s*\(", txt, flags=re.M)))


def default_params(**kw) -> sph_params:
    p = sph_params()
    load().sph_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("box_lo", "box_hi"):
            setattr(p, k, (_d * 3)(*v))
        else:
            setattr(p, k, v)
    return p


# ---------------------------------------------------------------- thin wrappers with the ABI names
def _check(ctx, code):
    if code != SPH_OK:
        lib = load()
        msg = lib.sph_last_error(ctx).decode() if ctx else ""
        raise SPHError(code, f"{lib.sph_error_string(code).decode()}: {msg}")


def sph_create(params: sph_params, n_cap: int, neigh_cap: int = 0, stream: int | None = None):
    ctx = _p()
    code = load().sph_create(ctypes.byref(params), int(n_cap), int(neigh_cap), _p(stream or 0), ctypes.byref(ctx))
    _check(None, code)
    return ctx


def sph_batch_create(params: sph_params, box_offsets, box_mass, box_gamma=None, neigh_cap: int = 0,
                     stream: int | None = None):
    off = np.ascontiguousarray(box_offsets, dtype=np.int64)
    mass = np.ascontiguousarray(box_mass, dtype=np.float64)
    gam = None if box_gamma is None else np.ascontiguousarray(box_gamma, dtype=np.float64)
    ctx = _p()
    code = load().sph_batch_create(ctypes.byref(params), len(off) - 1, off.ctypes.data, mass.ctypes.data,
                                   gam.ctypes.data if gam is not None else None, int(neigh_cap), _p(stream or 0),
                                   ctypes.byref(ctx))
    _check(None, code)
    return ctx


def sph_batch_dt(ctx, n_boxes: int) -> np.ndarray:
    out = np.zeros(n_boxes)
    _check(ctx, load().sph_batch_dt(ctx, out.ctypes.data))
    return out


def sph_destroy(ctx):
    load().sph_destroy(ctx)


def sph_build_tree(ctx, st: sph_state):
    _check(ctx, load().sph_build_tree(ctx, ctypes.byref(st)))


def sph_find_neighbours(ctx, st: sph_state) -> int:
    n = _i64()
    _check(ctx, load().sph_find_neighbours(ctx, ctypes.byref(st), ctypes.byref(n)))
    return n.value


def sph_compute_density_h(ctx, st: sph_state) -> int:
    it = _i()
    _check(ctx, load().sph_compute_density_h(ctx, ctypes.byref(st), ctypes.byref(it)))
    return it.value


def sph_compute_forces(ctx, st: sph_state):
    _check(ctx, load().sph_compute_forces(ctx, ctypes.byref(st)))


def sph_step(ctx, st: sph_state, dt: float = 0.0):
    used, nxt = _d(), _d()
    _check(ctx, load().sph_step(ctx, ctypes.byref(st), float(dt), ctypes.byref(used), ctypes.byref(nxt)))
    return used.value, nxt.value


def sph_step_host(ctx, st: sph_state, dt: float = 0.0):
    used, nxt = _d(), _d()
    _check(ctx, load().sph_step_host(ctx, ctypes.byref(st), float(dt), ctypes.byref(used), ctypes.byref(nxt)))
    return used.value, nxt.value


def sph_get_stats(ctx) -> dict:
    s = sph_stats()
    _check(ctx, load().sph_get_stats(ctx, ctypes.byref(s)))
    out = {f: getattr(s, f) for f, _ in sph_stats._fields_}
    out["stage_ms"] = {k: s.stage_ms[i] for i, k in enumerate(STAGES)}
    return out


def sph_set_timing(ctx, on: bool):
    _check(ctx, load().sph_set_timing(ctx, 1 if on else 0))


def sph_set_graph(ctx, on: bool):
    _check(ctx, load().sph_set_graph(ctx, 1 if on else 0))


def sph_reset_timing(ctx):
    _check(ctx, load().sph_reset_timing(ctx))


def sph_debug_wait_timeout(ctx, st, which: int, spins: int) -> int:
    """Failure-detection probe: returns the status code (SPH_ERR_TIMEOUT is the expected result)."""
    return int(load().sph_debug_wait_timeout(ctx, ctypes.byref(st) if st is not None else None, int(which),
                                             int(spins)))


def sph_sort_morton_noalloc(n: int, x_ptr: int, y_ptr: int, z_ptr: int, box_lo, box_hi, codes_ptr: int,
                            perm_ptr: int, stream: int | None = None) -> None:
    """Morton codes + stable sort into caller buffers, without device allocation (see sph.h)."""
    lo, hi = (_d * 3)(*box_lo), (_d * 3)(*box_hi)
    code = load().sph_sort_morton_noalloc(int(n), _p(x_ptr), _p(y_ptr), _p(z_ptr), ctypes.byref(lo),
                                          ctypes.byref(hi), _p(codes_ptr), _p(perm_ptr), _p(stream or 0))
    if code != SPH_OK:
        raise SPHError(code, load().sph_error_string(code).decode())


def sph_export_tree(ctx) -> dict:
    lib = load()
    n, L = _i64(), _i64()
    _check(ctx, lib.sph_tree_sizes(ctx, ctypes.byref(n), ctypes.byref(L)))
    n, L = n.value, L.value
    nin, nodes = max(L - 1, 0), 2 * L - 1
    out = {"mu": np.zeros(n, np.uint64), "perm": np.zeros(n, np.uint32), "leaf_first": np.zeros(L + 1, np.int64),
           "mu_leaf": np.zeros(L, np.uint64), "lchild": np.zeros(nin, np.int32), "rchild": np.zeros(nin, np.int32),
           "lflag": np.zeros(nin, np.uint8), "rflag": np.zeros(nin, np.uint8), "endrange": np.zeros(nin, np.int32),
           "bmin": np.zeros((nodes, 3)), "bmax": np.zeros((nodes, 3)), "hmax": np.zeros(nodes)}
    st = sph_stats()
    _check(ctx, lib.sph_get_stats(ctx, ctypes.byref(st)))
    out["group_start"] = np.zeros(st.n_groups + 1, np.int64)
    v = sph_tree_view(**{k: (a.ctypes.data if a.size else None) for k, a in out.items()})
    _check(ctx, lib.sph_export_tree(ctx, ctypes.byref(v)))
    return out


def sph_get_launch(ctx) -> dict:
    l = sph_launch()
    _check(ctx, load().sph_get_launch(ctx, ctypes.byref(l)))
    return {f: getattr(l, f) for f, _ in sph_launch._fields_}


def sph_set_launch(ctx, **shape):
    l = sph_launch(**{**sph_get_launch(ctx), **shape})
    _check(ctx, load().sph_set_launch(ctx, ctypes.byref(l)))


def sph_autotune(ctx, st: sph_state) -> tuple:
    l, ms = sph_launch(), _d()
    _check(ctx, load().sph_autotune(ctx, ctypes.byref(st), ctypes.byref(l), ctypes.byref(ms)))
    return {f: getattr(l, f) for f, _ in sph_launch._fields_}, ms.value


def sph_export_neighbours(ctx, n: int, n_pairs: int):
    off = np.zeros(n + 1, np.int64)
    ids = np.zeros(max(n_pairs, 1), np.uint32)
    _check(ctx, load().sph_export_neighbours(ctx, off.ctypes.data, ids.ctypes.data))
    return off, ids[:off[-1]].copy()


# ---------------------------------------------------------------- device state (PyTorch memory)
class DeviceState:
    """Particle arrays as float64 CUDA tensors (id: int32 holding the uint32 original index; alpha:
    per-particle viscosity for the shock switch, present only when requested)."""

    def __init__(self, n: int, mass: float, device: str = "cuda", alpha: bool = False):
        import torch
        self.n = int(n)
        self.mass = float(mass)
        self.t = {f: torch.zeros(self.n, dtype=torch.float64, device=device) for f in FIELDS}
        self.t["id"] = torch.arange(self.n, dtype=torch.int32, device=device)
        if alpha:
            self.t["alpha"] = torch.ones(self.n, dtype=torch.float64, device=device)

    @classmethod
    def from_numpy(cls, d: dict, device: str = "cuda"):
        import torch
        s = cls(len(d["x"]), d["mass"], device, alpha="alpha" in d)
        for f in FIELDS + ("alpha",):
            if f in d:
                s.t[f].copy_(torch.from_numpy(np.ascontiguousarray(d[f], dtype=np.float64)))
        return s

    def to_numpy(self) -> dict:
        out = {f: self.t[f].cpu().numpy() for f in FIELDS}
        out["id"] = self.t["id"].cpu().numpy().view(np.uint32)
        if "alpha" in self.t:
            out["alpha"] = self.t["alpha"].cpu().numpy()
        out["mass"] = self.mass
        return out

    def c(self) -> sph_state:
        return sph_state(self.n, self.mass, *[self.t[f].data_ptr() for f in FIELDS], self.t["id"].data_ptr(),
                         self.t["alpha"].data_ptr() if "alpha" in self.t else None)


def host_state(d: dict) -> tuple:
    """sph_state over host numpy arrays (kept alive by the returned dict) for sph_step_host."""
    arrs = {f: np.ascontiguousarray(d[f], dtype=np.float64) for f in FIELDS}
    arrs["id"] = np.ascontiguousarray(d.get("id", np.arange(len(arrs["x"]))), dtype=np.uint32)
    if "alpha" in d:
        arrs["alpha"] = np.ascontiguousarray(d["alpha"], dtype=np.float64)
    st = sph_state(len(arrs["x"]), float(d["mass"]), *[arrs[f].ctypes.data for f in FIELDS], arrs["id"].ctypes.data,
                   arrs["alpha"].ctypes.data if "alpha" in arrs else None)
    return st, arrs


class Solver:
    """Owns one context; methods mirror the ABI on a DeviceState."""

    def __init__(self, params: sph_params, n_cap: int, neigh_cap: int = 0, stream: int | None = None, _ctx=None):
        if _ctx is not None:
            self.ctx = _ctx
            return
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.ctx = sph_create(params, n_cap, neigh_cap, stream)
        self.n_boxes = 1

    @classmethod
    def batch(cls, params: sph_params, box_offsets, box_mass, box_gamma=None, neigh_cap: int = 0,
              stream: int | None = None):
        """Context over an ensemble of independent boxes (sph_batch_create)."""
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        s = cls(params, 0, _ctx=sph_batch_create(params, box_offsets, box_mass, box_gamma, neigh_cap, stream))
        s.n_boxes = len(box_offsets) - 1
        return s

    def batch_dt(self) -> np.ndarray:
        return sph_batch_dt(self.ctx, self.n_boxes)

    def close(self):
        if self.ctx:
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_tree(self, s: DeviceState):
        st = s.c()
        sph_build_tree(self.ctx, st)

    def find_neighbours(self, s: DeviceState) -> int:
        return sph_find_neighbours(self.ctx, s.c())

    def compute_density_h(self, s: DeviceState) -> int:
        return sph_compute_density_h(self.ctx, s.c())

    def compute_forces(self, s: DeviceState):
        sph_compute_forces(self.ctx, s.c())

    def step(self, s: DeviceState, dt: float = 0.0):
        return sph_step(self.ctx, s.c(), dt)

    def converge(self, s: DeviceState, max_outer: int = 16) -> int:
        """Initial ("white") step: tree, cache and density until h stays inside the cache tolerance,
        then forces (sets a, du and the first CFL step)."""
        self.build_tree(s)
        total = 0
        for _ in range(max_outer):
            self.find_neighbours(s)
            try:
                total += self.compute_density_h(s)
                break
            except SPHError as e:
                if e.code != SPH_ERR_CACHE_STALE:
                    raise
        else:
            raise SPHError(SPH_ERR_CACHE_STALE, "initial h did not settle")
        self.compute_forces(s)
        return total

    def stats(self) -> dict:
        return sph_get_stats(self.ctx)

    def launch(self) -> dict:
        return sph_get_launch(self.ctx)

    def set_launch(self, **shape):
        sph_set_launch(self.ctx, **shape)

    def autotune(self, s: DeviceState) -> tuple:
        """Pick the fastest launch shapes / reduction level on state s (see sph_autotune)."""
        return sph_autotune(self.ctx, s.c())

    def set_timing(self, on: bool):
        sph_set_timing(self.ctx, on)

    def set_graph(self, on: bool):
        """Replay sph_step as one captured CUDA graph (see sph_set_graph)."""
        sph_set_graph(self.ctx, on)

    def reset_timing(self):
        sph_reset_timing(self.ctx)

    def step_host(self, host_st, dt: float = 0.0):
        return sph_step_host(self.ctx, host_st, dt)

    def export_tree(self) -> dict:
        return sph_export_tree(self.ctx)

    def export_neighbours(self, n: int) -> tuple:
        st = self.stats()
        return sph_export_neighbours(self.ctx, n, st["n_pairs"])
