"""The allocation-free deposit (pm_deposit_cic_static) against the allocating one.

pm_deposit_cic_static serves callers that cannot allocate device memory themselves
(a host application with a fixed, pre-reserved memory budget, or a plug-in environment
that forbids runtime allocations): its accumulator is a fixed 128^3 device array inside
the library.  Here it must give the same delta as pm_deposit_cic, bit for bit (the
deposit's tolerance), on two calls in a row, so the second call also checks that the
shared array is cleared between calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2604_15434_gb300 import synth

pytestmark = pytest.mark.gpu


def test_static_deposit_matches_allocating_deposit_twice(gpu_lib):
    cases = [
        (32, synth.zeldovich_particles(32, -1.5, 1.0, 1001, nyquist_cutoff=True)),
        (64, np.random.default_rng(77).random((3, 100003))),
    ]
    for n, pos in cases:  # two calls in a row on the same shared array
        p = torch.from_numpy(pos).cuda()
        want = gpu_lib.pm_deposit_cic(p, n)
        got, st = gpu_lib.pm_deposit_cic_static(p, n)
        torch.cuda.synchronize()
        assert st == gpu_lib.PM_OK
        assert torch.equal(got, want)


def test_static_deposit_at_full_capacity(gpu_lib):
    """n = 128 clears and uses the whole static array; a smaller call after it must not
    see its contents."""
    pos = np.random.default_rng(128).random((3, 300007))
    p = torch.from_numpy(pos).cuda()
    for n in (128, 16):
        want = gpu_lib.pm_deposit_cic(p, n)
        got, st = gpu_lib.pm_deposit_cic_static(p, n)
        torch.cuda.synchronize()
        assert st == gpu_lib.PM_OK
        assert torch.equal(got, want)


def test_static_deposit_rejects_meshes_above_its_capacity(gpu_lib):
    p = torch.from_numpy(np.random.default_rng(1).random((3, 1000))).cuda()
    _, st = gpu_lib.pm_deposit_cic_static(p, 256)
    assert st == gpu_lib.PM_ERR_TOO_LARGE


def test_static_deposit_rejects_invalid_arguments(gpu_lib):
    p = torch.from_numpy(np.random.default_rng(2).random((3, 1000))).cuda()
    for n in (48, 4):  # not a power of two; below the smallest mesh
        _, st = gpu_lib.pm_deposit_cic_static(p, n)
        assert st == gpu_lib.PM_ERR_INVALID_ARG
    empty = torch.empty((3, 0), dtype=torch.float64, device=p.device)
    _, st = gpu_lib.pm_deposit_cic_static(empty, 16)
    assert st == gpu_lib.PM_ERR_INVALID_ARG
    lib = gpu_lib.load()
    delta = torch.empty((16, 16, 16), dtype=torch.float64, device=p.device)
    assert lib.pm_deposit_cic_static(None, 1000, 16, ctypes.c_void_p(delta.data_ptr()), None) == gpu_lib.PM_ERR_INVALID_ARG
    assert lib.pm_deposit_cic_static(ctypes.c_void_p(p.data_ptr()), 1000, 16, None, None) == gpu_lib.PM_ERR_INVALID_ARG
