"""The allocation-free deposit (pm_deposit_cic_static) against the allocating one.

pm_deposit_cic_static serves callers that cannot allocate device memory themselves
(a host application with a fixed, pre-reserved memory budget, or a plug-in environment
that forbids runtime allocations): its accumulator is a fixed 128^3 device array inside
the library.  Here it must give the same delta as pm_deposit_cic, bit for bit (the
deposit's tolerance), on two calls in a row, so the second call also checks that the
shared array is cleared between calls.  This file is collected last on purpose.
"""
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


def test_static_deposit_rejects_meshes_above_its_capacity(gpu_lib):
    p = torch.from_numpy(np.random.default_rng(1).random((3, 1000))).cuda()
    _, st = gpu_lib.pm_deposit_cic_static(p, 256)
    assert st == gpu_lib.PM_ERR_TOO_LARGE
