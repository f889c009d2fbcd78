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


def test_struct_layouts_match_header():
    # sph_params: 2 ints, 10 doubles, 4 ints, 6 doubles
    assert ctypes.sizeof(sph.sph_params) == 8 + 80 + 16 + 48
    assert ctypes.sizeof(sph.sph_state) == 8 + 8 + 16 * 8
