"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU, and exports
every function declared in include/*.h (no compute calls are made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_0811_4446_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_0811_4446_gb300 import mg, unet
    assert _declared() == set(mg.SIGNATURES) | set(unet.SIGNATURES)


def test_unet_param_count_matches_oracle(lib):
    from oracle import unet as ou
    from paper_0811_4446_gb300 import unet
    assert unet.param_count() == ou.param_count()
    assert unet.init_params(0).size == ou.param_count()


def test_workspace_sizing_without_gpu(lib):
    import workloads as W
    from paper_0811_4446_gb300 import mg
    mg.load()
    p = mg.default_params()
    z = W.z_nodes(256, 1e-2)
    g = mg.mg_grid(256, 256, 1e-2, z.ctypes.data_as(mg._dp))
    n256 = mg.load().mg_workspace_bytes(ctypes.byref(g), ctypes.byref(p))
    assert 10e6 < n256 < 60e6
    bad = mg.mg_grid(255, 256, 1e-2, z.ctypes.data_as(mg._dp))
    assert mg.load().mg_workspace_bytes(ctypes.byref(bad), ctypes.byref(p)) == 0
    # parameters of the later forms are validated before any allocation (0 bytes = invalid)
    for kw in (dict(full_jacobian=2), dict(max_corrections=0), dict(max_corrections=101), dict(line_smoother=4),
               dict(newton_tol_rel=1.0), dict(newton_tol_rel=-0.1), dict(pdl=32), dict(wall_dirichlet=2)):
        pb = mg.default_params(**kw)
        assert mg.load().mg_workspace_bytes(ctypes.byref(g), ctypes.byref(pb)) == 0, kw
    # r-lines (2) and alternating lines (3): rows of at most 512 unknowns
    z512 = W.z_nodes(512, 1e-2)
    g512 = mg.mg_grid(512, 512, 1e-2, z512.ctypes.data_as(mg._dp))
    for line in (2, 3):
        assert mg.load().mg_workspace_bytes(ctypes.byref(g), ctypes.byref(mg.default_params(line_smoother=line))) > 0
        assert mg.load().mg_workspace_bytes(ctypes.byref(g512), ctypes.byref(mg.default_params(line_smoother=line))) == 0
        assert mg.load().mg_workspace_bytes(ctypes.byref(g512), ctypes.byref(
            mg.default_params(line_smoother=line, wall_dirichlet=1))) > 0
    # the line smoother's column scratch is allocated only when it is enabled
    nl = mg.load().mg_workspace_bytes(ctypes.byref(g), ctypes.byref(mg.default_params(line_smoother=1)))
    assert 0 <= nl - n256 - 8 * 12 * 257 * 129 < 256     # plus its 256-byte alignment


def test_params_default_values(lib):
    from paper_0811_4446_gb300 import mg
    p = mg.default_params()
    assert (p.dt1, p.dt_growth, p.max_newton, p.nu1, p.nu2) == (1e-9, 5.0, 10, 4, 4)
    assert (p.nu_coarse_n, p.nu_coarse1, p.nu_coarse2, p.chain_from) == (64, 2, 2, 1)
    assert (p.nu_tiny_n, p.nu_tiny1, p.nu_tiny2, p.pdl, p.wall_dirichlet) == (8, 1, 1, 9, 0)
    assert p.newton_tol_rel == 0.1 and p.newton_tol == 0.0
    assert (p.full_jacobian, p.max_corrections, p.line_smoother) == (0, 20, 0)
    assert np.isclose(p.mu_p, 0.15) and np.isclose(p.D_p, 0.0038)
