"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/pmeft.h declares (no device needed; nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(pm_\w+|poisson_solve|scalar_mg_solve\w*|force_interp)\s*\(",
                             txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2604_15434_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ("pm_deposit_cic", "poisson_solve", "scalar_mg_solve", "force_interp", "pm_step", "pm_create"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2604_15434_gb300 import api

    assert _declared() <= set(api.SIGNATURES), _declared() - set(api.SIGNATURES)


def test_coefficients_through_the_abi_match_the_oracle(lib):
    """Host-only entry point: no device is touched."""
    import oracle as O
    from paper_2604_15434_gb300 import api

    for args in ((-0.5, 0.0, 1.0), (-1.0, 0.2, 0.6), (-2.0, 0.5, 0.35)):
        got = api.coefficients(*args)
        want = O.coefficients(*args)
        for k in ("nu", "xi", "kappa", "C2", "C4", "geff", "src"):
            assert got[k] == pytest.approx(want[k], rel=1e-14, abs=1e-15)


def test_product_path_refuses_host_tensors(lib):
    """No CPU fallback: the binding accepts only CUDA tensors, and every entry point called
    with host tensors raises instead of computing anything."""
    import torch

    from paper_2604_15434_gb300 import api

    x = torch.zeros((8, 8, 8), dtype=torch.float64)
    with pytest.raises(TypeError):
        api._ptr(x)
    calls = (lambda: api.scalar_mg_solve(x, -0.5, 0.0, 1.0, 1e-8),
             lambda: api.pm_deposit_cic(torch.zeros((3, 8), dtype=torch.float64), 8),
             lambda: api.poisson_solve(x, 1.0, 0.0),
             lambda: api.pm_mg_sweep(x, x, 0.0, 0.475, 0.5, 0.35))
    for call in calls:
        with pytest.raises(Exception):
            call()
