"""The C-ABI library loads and exports every function declared in include/sph.h (no GPU needed)."""
import ctypes

import pytest

from paper_2503_09713_gb300 import sph


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build_library()
    return sph.load()


def test_header_declares_the_boundary():
    names = sph.header_functions()
    for required in ("sph_build_tree", "sph_find_neighbours", "sph_compute_density_h", "sph_compute_forces",
                     "sph_step", "sph_create", "sph_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in sph.header_functions():
        assert hasattr(lib, name), name


def test_host_only_entry_points(lib):
    p = sph.default_params()
    assert p.hfact == 1.2 and p.h_clamp == 1.2 and p.cache_tol == 1.1 and p.kernel == sph.SPH_KERNEL_M4
    assert abs(p.gamma - 5.0 / 3.0) < 1e-15 and p.c_cour == 0.3 and p.c_force == 0.25
    assert lib.sph_error_string(sph.SPH_ERR_CACHE_STALE).startswith(b"neighbour cache stale")
    assert lib.sph_error_string(12345) == b"unknown status"
    # argument checks run before any device call
    ctx = ctypes.c_void_p()
    bad = sph.default_params(hfact=-1.0)
    assert lib.sph_create(ctypes.byref(bad), 100, 0, None, ctypes.byref(ctx)) == sph.SPH_ERR_INVALID_ARG
    assert lib.sph_create(ctypes.byref(p), 100, 0, None, None) == sph.SPH_ERR_INVALID_ARG
    assert lib.sph_build_tree(None, None) == sph.SPH_ERR_INVALID_ARG
    assert lib.sph_destroy(None) == sph.SPH_OK


def test_degenerate_sizes_are_refused_before_any_device_call(lib):
    """An empty particle set, an empty or oversized batch and malformed box tables are argument
    errors found on the host (the context pointer stays NULL)."""
    import numpy as np
    p = sph.default_params()
    ctx = ctypes.c_void_p(1)
    assert lib.sph_create(ctypes.byref(p), 0, 0, None, ctypes.byref(ctx)) == sph.SPH_ERR_INVALID_ARG
    assert ctx.value is None
    assert lib.sph_create(ctypes.byref(p), (1 << 30) + 1, 0, None, ctypes.byref(ctx)) == sph.SPH_ERR_INVALID_ARG

    def batch(off, mass, gamma=None, n_boxes=None):
        off = np.ascontiguousarray(off, dtype=np.int64)
        mass = np.ascontiguousarray(mass, dtype=np.float64)
        g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
        out = ctypes.c_void_p(1)
        nb = len(off) - 1 if n_boxes is None else n_boxes
        r = lib.sph_batch_create(ctypes.byref(p), nb, off.ctypes.data, mass.ctypes.data,
                                 None if g is None else g.ctypes.data, 0, None, ctypes.byref(out))
        assert out.value is None
        return r

    bad = sph.SPH_ERR_INVALID_ARG
    assert batch([0, 0, 0], [1.0, 1.0]) == bad                 # every box empty
    assert batch([5, 10], [1.0]) == bad                        # offsets do not start at 0
    assert batch([0, 10, 5], [1.0, 1.0]) == bad                # negative box size
    assert batch([0, 10], [0.0]) == bad                        # mass not positive
    assert batch([0, 10], [1.0], gamma=[1.0]) == bad           # gamma not above 1
    assert batch([0, 10], [1.0], n_boxes=0) == bad             # no box
    assert batch(np.arange(4098) * 4, np.ones(4097)) == bad    # more than 4096 boxes


def _c_layout(struct, fields):
    """sizeof and offsetof of a struct of include/sph.h, from the C compiler (gcc, host)."""
    import os
    import subprocess
    import tempfile
    inc = os.path.join(os.path.dirname(sph.HEADER))
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sph.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        with open(src, "w") as fh:
            fh.write("\n".join(lines))
        subprocess.run(["gcc", "-I", inc, src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("name", ["sph_params", "sph_state", "sph_tree_view", "sph_stats", "sph_launch"])
def test_struct_layouts_match_header(name):
    """Every ctypes mirror of an ABI struct has the C compiler's size and field offsets."""
    cls = getattr(sph, name)
    fields = [f for f, _ in cls._fields_]
    size, offs = _c_layout(name, fields)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs
