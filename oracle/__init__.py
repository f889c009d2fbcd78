"""CPU oracle for the SPH hot path of arXiv 2503.09713 (Shamrock) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this
package.  The product library (``paper_2503_09713_gb300``) never imports it, and this package imports
nothing from the product library.  The arithmetic lives in ``sph_oracle.c`` (plain C, FP64,
``-ffp-contract=off``); this module only compiles it and marshals numpy arrays through ctypes.

Every function names the passage of the paper it follows in ``sph_oracle.c``.  Parity pins for each
function are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "libsph_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _setup(_lib)
    return _lib


_d = ctypes.c_double
_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_p = ctypes.c_void_p


class OrcParams(ctypes.Structure):
    _fields_ = [("hfact", _d), ("gamma", _d), ("alpha_av", _d), ("beta_av", _d), ("alpha_u", _d),
                ("c_cour", _d), ("c_force", _d), ("h_tol", _d), ("h_clamp", _d), ("cache_tol", _d),
                ("lo", _d * 3), ("hi", _d * 3), ("periodic", _i32), ("h_max_iter", _i32),
                ("av_switch", _i32), ("max_corr", _i32), ("alpha_min", _d), ("sigma_decay", _d), ("eps_v", _d),
                ("lambda_stiff", _d)]


@dataclass
class Params:
    """Hydro parameters (Sect. 2.1, App. F, App. G); defaults are the paper's / the workloads'."""
    hfact: float = 1.2
    gamma: float = 5.0 / 3.0
    alpha_av: float = 1.0
    beta_av: float = 2.0
    alpha_u: float = 1.0
    c_cour: float = 0.3
    c_force: float = 0.25
    h_tol: float = 1e-6
    h_clamp: float = 1.2
    cache_tol: float = 1.1
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    periodic: int = 1
    h_max_iter: int = 200
    kernel: int = 0          # 0 M4, 1 M5, 2 M6, 3 Wendland C2, 4 C4, 5 C6 (Sect. 2.1)
    av_switch: int = 0       # 1: alpha evolves per particle (App. G "Shock detection"), alpha_av = max
    max_corr: int = 4        # most corrector passes per step
    alpha_min: float = 0.0
    sigma_decay: float = 0.1
    eps_v: float = 0.0       # epsilon_v of Eq. cvleapfrog (the paper: 1e-2); 0: no corrector re-run
    lambda_stiff: float = 1.0

    def c(self) -> OrcParams:
        return OrcParams(self.hfact, self.gamma, self.alpha_av, self.beta_av, self.alpha_u, self.c_cour,
                         self.c_force, self.h_tol, self.h_clamp, self.cache_tol, (_d * 3)(*self.lo),
                         (_d * 3)(*self.hi), int(self.periodic), int(self.h_max_iter), int(self.av_switch),
                         int(self.max_corr), float(self.alpha_min), float(self.sigma_decay), float(self.eps_v),
                         float(self.lambda_stiff))


def _setup(lib):
    P = ctypes.POINTER(OrcParams)
    sig = {
        "orc_quantise": (ctypes.c_uint64, [_d, _d, _d, _i32]),
        "orc_interleave": (ctypes.c_uint64, [ctypes.c_uint64] * 3 + [_i32]),
        "orc_deinterleave": (None, [ctypes.c_uint64, _i32, _p, _p, _p]),
        "orc_morton": (None, [_i64, _p, _p, _p, _p, _p, _i32, _p]),
        "orc_delta": (_i32, [ctypes.c_uint64, ctypes.c_uint64, _i32]),
        "orc_sort_by_key": (None, [_i64, _p, _p, _p]),
        "orc_keep_mask": (None, [_i64, _p, _i32, _i32, _p]),
        "orc_compact": (_i64, [_i64, _p, _p, _p, _p]),
        "orc_radix_tree": (None, [_i64, _p, _i32, _p, _p, _p, _p, _p]),
        "orc_cell_boxes": (None, [_i64, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
        "orc_set_kernel": (None, [_i32]),
        "orc_kernel_R": (_d, [_i32]),
        "orc_kernel_C": (_d, [_i32]),
        "orc_kernel_f": (_d, [_i32, _d]),
        "orc_kernel_df": (_d, [_i32, _d]),
        "orc_m4_f": (_d, [_d]),
        "orc_m4_df": (_d, [_d]),
        "orc_W": (_d, [_d, _d]),
        "orc_dWdh": (_d, [_d, _d]),
        "orc_F": (_d, [_d, _d]),
        "orc_neighbours": (_i64, [_i64, _p, _p, _p, _p, _d, _p, _p, _i32, _i32]),
        "orc_neighbours_copy": (None, [_p, _p]),
        "orc_density_root": (_i64, [_i64, _p, _p, _p, _d, _d, _p, _p, _i32, _i32, _p]),
        "orc_density_algF": (_i32, [_i64, _d, P, _p, _p, _p, _p, _p, _p, _i32, ctypes.POINTER(_i32)]),
        "orc_density_at": (None, [_i64, _d, _d, _p, _p, _p, _p, _p, _p, _i32, _i32, _p, _p]),
        "orc_forces": (None, [_i64, _d, P, _p, _p, _p, _p, _p, _p, _p, _p, _p, _i32, _p, _p, _p, _p, _p]),
        "orc_cfl": (_d, [_i64, P, _p, _p, _p, _p, _p]),
        "orc_step": (_d, [_i64, _d, P, _d] + [_p] * 15 + [_i32, ctypes.POINTER(_i32), ctypes.POINTER(_d)]),
        "orc_step_ext": (_d, [_i64, _d, P, _d] + [_p] * 17 + [_i32, ctypes.POINTER(_i32), ctypes.POINTER(_d),
                                                             ctypes.POINTER(_i32)]),
        "orc_forces_alpha": (None, [_i64, _d, P] + [_p] * 10 + [_i32] + [_p] * 5),
        "orc_alpha_update": (None, [_i64, _d, P] + [_p] * 12 + [_d, _i32, _p]),
        "orc_num_threads": (_i32, []),
        "orc_subset_forces": (_i64, [_i64, _d, P] + [_p] * 7 + [_d, _i64, _p] + [_p] * 7),
        "orc_subset_neighbours": (_i64, [_i64, _p, _p, _p, _p, _d, _p, _p, _i32, _i64, _p, _p, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _box(lo, hi):
    return np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)


def num_threads() -> int:
    return _load().orc_num_threads()


# ---- Morton codes / prefixes (App. B) ----
def quantise(x, lo, hi, bits):
    return _load().orc_quantise(float(x), float(lo), float(hi), int(bits))


def interleave(X, Y, Z, bits):
    return _load().orc_interleave(int(X), int(Y), int(Z), int(bits))


def deinterleave(m, bits):
    X, Y, Z = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _load().orc_deinterleave(int(m), int(bits), ctypes.byref(X), ctypes.byref(Y), ctypes.byref(Z))
    return X.value, Y.value, Z.value


def morton(x, y, z, lo=(0, 0, 0), hi=(1, 1, 1), bits=21):
    x, y, z = _f64(x), _f64(y), _f64(z)
    lo, hi = _box(lo, hi)
    out = np.empty(len(x), dtype=np.uint64)
    _load().orc_morton(len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(lo), _ptr(hi), int(bits), _ptr(out))
    return out


def delta(a, b, nbits):
    return _load().orc_delta(int(a), int(b), int(nbits))


# ---- Sort, mask, compaction (App. C) ----
def sort_by_key(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    s = np.empty_like(keys)
    perm = np.empty(len(keys), dtype=np.uint32)
    _load().orc_sort_by_key(len(keys), _ptr(keys), _ptr(s), _ptr(perm))
    return s, perm


def keep_mask(mu, nbits, n_red):
    mu = np.ascontiguousarray(mu, dtype=np.uint64)
    xi = np.zeros(len(mu), dtype=np.uint8)
    _load().orc_keep_mask(len(mu), _ptr(mu), int(nbits), int(n_red), _ptr(xi))
    return xi


def compact(mu, xi):
    mu = np.ascontiguousarray(mu, dtype=np.uint64)
    xi = np.ascontiguousarray(xi, dtype=np.uint8)
    idv = np.zeros(len(mu) + 1, dtype=np.int64)
    ml = np.zeros(max(len(mu), 1), dtype=np.uint64)
    L = _load().orc_compact(len(mu), _ptr(mu), _ptr(xi), _ptr(idv), _ptr(ml))
    return idv[:L + 1].copy(), ml[:L].copy()


@dataclass
class RadixTree:
    lchild: np.ndarray
    rchild: np.ndarray
    lflag: np.ndarray
    rflag: np.ndarray
    endrange: np.ndarray


def radix_tree(mu_leaf, nbits):
    mu_leaf = np.ascontiguousarray(mu_leaf, dtype=np.uint64)
    L = len(mu_leaf)
    m = max(L - 1, 1)
    t = RadixTree(np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(m, np.uint8),
                  np.zeros(m, np.uint8), np.zeros(m, np.int32))
    _load().orc_radix_tree(L, _ptr(mu_leaf), int(nbits), _ptr(t.lchild), _ptr(t.rchild), _ptr(t.lflag),
                           _ptr(t.rflag), _ptr(t.endrange))
    if L < 2:
        t = RadixTree(*(a[:0] for a in (t.lchild, t.rchild, t.lflag, t.rflag, t.endrange)))
    return t


def cell_boxes(idv, endrange, x, y, z, h):
    """Tight boxes and h_max per node (internal 0..L-2, leaf j at L-1+j), positions in sorted order."""
    idv = np.ascontiguousarray(idv, dtype=np.int64)
    L = len(idv) - 1
    endrange = np.ascontiguousarray(endrange, dtype=np.int32)
    if len(endrange) == 0:
        endrange = np.zeros(1, np.int32)
    x, y, z, h = _f64(x), _f64(y), _f64(z), _f64(h)
    nodes = 2 * L - 1
    bmin = np.zeros((nodes, 3))
    bmax = np.zeros((nodes, 3))
    hmax = np.zeros(nodes)
    _load().orc_cell_boxes(L, _ptr(idv), _ptr(endrange), _ptr(x), _ptr(y), _ptr(z), _ptr(h), _ptr(bmin),
                           _ptr(bmax), _ptr(hmax))
    return bmin, bmax, hmax


# ---- Kernel (Sect. 2.1) ----
def m4_f(q):
    return _load().orc_m4_f(float(q))


def m4_df(q):
    return _load().orc_m4_df(float(q))


KERNELS = {"M4": 0, "M5": 1, "M6": 2, "C2": 3, "C4": 4, "C6": 5}


def _kernel(kind):
    """Select the smoothing kernel every oracle function uses (a module setting of the C oracle)."""
    _load().orc_set_kernel(int(kind))


def kernel_f(kind, q):
    return _load().orc_kernel_f(int(kind), float(q))


def kernel_df(kind, q):
    return _load().orc_kernel_df(int(kind), float(q))


def kernel_R(kind):
    return _load().orc_kernel_R(int(kind))


def kernel_C(kind):
    return _load().orc_kernel_C(int(kind))


def W(r, h, kernel=0):
    _kernel(kernel)
    return _load().orc_W(float(r), float(h))


def dWdh(r, h, kernel=0):
    _kernel(kernel)
    return _load().orc_dWdh(float(r), float(h))


def F(r, h, kernel=0):
    _kernel(kernel)
    return _load().orc_F(float(r), float(h))


# ---- Neighbour sets (App. C/D) ----
def neighbours(x, y, z, hc, s, lo=(0, 0, 0), hi=(1, 1, 1), periodic=1, method=None):
    """CSR neighbour lists: b != a with r_ab^2 < (s*max(hc_a,hc_b))^2 (minimum image).  method 0 =
    brute force (the definition), 1 = uniform grid (same set); default brute force below 4096."""
    x, y, z, hc = _f64(x), _f64(y), _f64(z), _f64(hc)
    lo, hi = _box(lo, hi)
    n = len(x)
    if method is None:
        method = 0 if n <= 4096 else 1
    lib = _load()
    npairs = lib.orc_neighbours(n, _ptr(x), _ptr(y), _ptr(z), _ptr(hc), float(s), _ptr(lo), _ptr(hi),
                                int(periodic), int(method))
    off = np.zeros(n + 1, np.int64)
    ids = np.zeros(max(npairs, 1), np.int32)
    lib.orc_neighbours_copy(_ptr(off), _ptr(ids))
    return off, ids[:npairs].copy()


# ---- Density / smoothing length (App. F) ----
def density_root(x, y, z, hfact, h_hi, lo=(0, 0, 0), hi=(1, 1, 1), periodic=1, method=None, kernel=0):
    """Unique root h_a of sum_b m W(r_ab,h_a) = m (hfact/h_a)^3 by bisection (equal masses)."""
    _kernel(kernel)
    x, y, z = _f64(x), _f64(y), _f64(z)
    lo, hi = _box(lo, hi)
    n = len(x)
    if method is None:
        method = 0 if n <= 4096 else 1
    h = np.zeros(n)
    bad = _load().orc_density_root(n, _ptr(x), _ptr(y), _ptr(z), float(hfact), float(h_hi), _ptr(lo),
                                   _ptr(hi), int(periodic), int(method), _ptr(h))
    if bad:
        raise ValueError(f"{bad} particles without an upper bracket at h_hi={h_hi}")
    return h


def density_algF(x, y, z, h, mass, params: Params, method=None):
    """App. F iteration.  Returns (h, rho, omega, inner_iterations, outer_passes)."""
    _kernel(params.kernel)
    x, y, z = _f64(x), _f64(y), _f64(z)
    h = _f64(h).copy()
    n = len(x)
    if method is None:
        method = 0 if n <= 4096 else 1
    rho = np.zeros(n)
    om = np.zeros(n)
    outer = _i32(0)
    p = params.c()
    it = _load().orc_density_algF(n, float(mass), ctypes.byref(p), _ptr(x), _ptr(y), _ptr(z), _ptr(h),
                                  _ptr(rho), _ptr(om), int(method), ctypes.byref(outer))
    if it < 0:
        raise RuntimeError("oracle h iteration exceeded h_max_iter")
    return h, rho, om, it, outer.value


def density_at(x, y, z, h, mass, hfact, lo=(0, 0, 0), hi=(1, 1, 1), periodic=1, method=None, kernel=0):
    """(rho_sum, Omega) at fixed h."""
    _kernel(kernel)
    x, y, z, h = _f64(x), _f64(y), _f64(z), _f64(h)
    lo, hi = _box(lo, hi)
    n = len(x)
    if method is None:
        method = 0 if n <= 4096 else 1
    rs = np.zeros(n)
    om = np.zeros(n)
    _load().orc_density_at(n, float(mass), float(hfact), _ptr(x), _ptr(y), _ptr(z), _ptr(h), _ptr(lo),
                           _ptr(hi), int(periodic), int(method), _ptr(rs), _ptr(om))
    return rs, om


# ---- Forces, CFL, step (Sect. 2.1, App. G) ----
def forces(x, y, z, vx, vy, vz, u, h, omega, mass, params: Params, method=None):
    """Returns (ax, ay, az, du, vsig)."""
    _kernel(params.kernel)
    arrs = [_f64(a) for a in (x, y, z, vx, vy, vz, u, h, omega)]
    n = len(arrs[0])
    if method is None:
        method = 0 if n <= 4096 else 1
    outs = [np.zeros(n) for _ in range(5)]
    p = params.c()
    _load().orc_forces(n, float(mass), ctypes.byref(p), *[_ptr(a) for a in arrs], int(method),
                       *[_ptr(o) for o in outs])
    return tuple(outs)


def cfl(h, vsig, ax, ay, az, params: Params):
    _kernel(params.kernel)
    arrs = [_f64(a) for a in (h, vsig, ax, ay, az)]
    p = params.c()
    return _load().orc_cfl(len(arrs[0]), ctypes.byref(p), *[_ptr(a) for a in arrs])


_STATE_KEYS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "ax", "ay", "az", "du", "rho", "omega", "vsig")


def step(state: dict, mass, params: Params, dt, method=None):
    """One KDK step on a dict of float64 arrays (keys x..vsig), in place.  Returns
    (dt_next, inner_iterations, dv_ratio).  With params.av_switch the dict needs "alpha" (per
    particle, updated in place); with params.eps_v > 0 it may hold "lambda_cfl" (the CFL multiplier,
    1 when absent, updated) and receives "corrector_passes"."""
    _kernel(params.kernel)
    for k in _STATE_KEYS:
        state[k] = _f64(state[k])
    n = len(state["x"])
    if method is None:
        method = 0 if n <= 4096 else 1
    it = _i32(0)
    dvr = _d(0.0)
    passes = _i32(0)
    p = params.c()
    alpha = None
    if params.av_switch:
        state["alpha"] = _f64(state["alpha"])
        alpha = _ptr(state["alpha"])
    lam = _d(float(state.get("lambda_cfl", 1.0)))
    dtn = _load().orc_step_ext(n, float(mass), ctypes.byref(p), float(dt), *[_ptr(state[k]) for k in _STATE_KEYS],
                               alpha, ctypes.byref(lam), int(method), ctypes.byref(it), ctypes.byref(dvr),
                               ctypes.byref(passes))
    if dtn < 0:
        raise RuntimeError("oracle h iteration exceeded h_max_iter")
    state["lambda_cfl"] = lam.value
    state["corrector_passes"] = passes.value
    return dtn, it.value, dvr.value


def alpha_update(x, y, z, vx, vy, vz, ax, ay, az, u, h, omega, mass, params: Params, dt, alpha, method=None):
    """The shock-switch step of alpha (orc_alpha_update) on copies; returns the new alpha."""
    _kernel(params.kernel)
    arrs = [_f64(a) for a in (x, y, z, vx, vy, vz, ax, ay, az, u, h, omega)]
    n = len(arrs[0])
    if method is None:
        method = 0 if n <= 4096 else 1
    out = _f64(alpha).copy()
    p = params.c()
    _load().orc_alpha_update(n, float(mass), ctypes.byref(p), *[_ptr(a) for a in arrs], float(dt), int(method),
                             _ptr(out))
    return out


def forces_alpha(x, y, z, vx, vy, vz, u, h, omega, alpha, mass, params: Params, method=None):
    """forces() with a per-particle alpha (v_sig,a = alpha_a c_s,a + beta |v_ab . rhat|)."""
    _kernel(params.kernel)
    arrs = [_f64(a) for a in (x, y, z, vx, vy, vz, u, h, omega, alpha)]
    n = len(arrs[0])
    if method is None:
        method = 0 if n <= 4096 else 1
    outs = [np.zeros(n) for _ in range(5)]
    p = params.c()
    _load().orc_forces_alpha(n, float(mass), ctypes.byref(p), *[_ptr(a) for a in arrs], int(method),
                             *[_ptr(o) for o in outs])
    return tuple(outs)


# ---- sampled evaluation for full-size inputs ----
def subset_forces(x, y, z, vx, vy, vz, u, mass, params: Params, idx, h_hi):
    """Root h, Omega and (ax, ay, az, du, vsig) of the particles idx, by brute force over all n.
    Returns a dict of arrays aligned with idx."""
    _kernel(params.kernel)
    arrs = [_f64(a) for a in (x, y, z, vx, vy, vz, u)]
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = len(idx)
    outs = [np.zeros(m) for _ in range(7)]
    p = params.c()
    bad = _load().orc_subset_forces(len(arrs[0]), float(mass), ctypes.byref(p), *[_ptr(a) for a in arrs],
                                    float(h_hi), m, _ptr(idx), *[_ptr(o) for o in outs])
    if bad:
        raise ValueError(f"{bad} roots not bracketed below h_hi={h_hi}")
    return dict(zip(("h", "omega", "ax", "ay", "az", "du", "vsig"), outs))


def subset_neighbours(x, y, z, hc, s, idx, lo=(0, 0, 0), hi=(1, 1, 1), periodic=1):
    """Neighbour lists (definition of ``neighbours``) of the particles idx only."""
    x, y, z, hc = _f64(x), _f64(y), _f64(z), _f64(hc)
    lo, hi = _box(lo, hi)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    lib = _load()
    args = (len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(hc), float(s), _ptr(lo), _ptr(hi), int(periodic), len(idx),
            _ptr(idx))
    tot = lib.orc_subset_neighbours(*args, None, None)
    off = np.zeros(len(idx) + 1, np.int64)
    ids = np.zeros(max(tot, 1), np.int32)
    lib.orc_subset_neighbours(*args, _ptr(off), _ptr(ids))
    return off, ids[:tot].copy()
