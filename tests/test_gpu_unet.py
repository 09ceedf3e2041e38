"""The warm-start network on the GPU (BF16 tensor cores, FP32 accumulation) against the
FP64 reference, its training, and what it gains over starting the solve without it."""
import os

import numpy as np
import pytest
import torch

import oracle as O
from oracle import unet as U
from paper_2604_15434_gb300 import synth

pytestmark = pytest.mark.gpu


def cu(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(7)
    n = 16
    delta = synth.lognormal_delta(n, -2.0, 1.2, 11)
    target = delta + 0.3 * rng.standard_normal((n, n, n))
    p = U.init_params(5)
    p[-1] = 0.1
    return n, delta, target, p


@pytest.mark.parametrize("path", [0, 1])
def test_forward_matches_reference(gpu_lib, case, path):
    """path 0: mma.sync convolutions; path 1: tcgen05 convolutions (the 16^3 level; the
    smaller levels keep path 0)."""
    n, delta, target, p = case
    net = gpu_lib.UNet()
    net.set_conv_path(path)
    net.set_params(p)
    got = net.forward(cu(delta), -0.8, 0.4, 0.9).cpu().numpy()
    want, _ = U.forward(p, delta, -0.8, 0.4, 0.9)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 3e-2  # BF16 activations and weights


@pytest.mark.parametrize("path", [0, 1])
def test_forward_matches_reference_64(gpu_lib, path):
    """At 64^3 every level takes the tiled convolution kernel (levels 64, 32, 16), with path 1
    the tcgen05 kernel on every level."""
    n = 64
    delta = synth.lognormal_delta(n, -2.0, 1.2, 21)
    p = U.init_params(9)
    p[-1] = 0.1
    net = gpu_lib.UNet()
    net.set_conv_path(path)
    net.set_params(p)
    got = net.forward(cu(delta), -1.2, 0.3, 0.7).cpu().numpy()
    want, _ = U.forward(p, delta, -1.2, 0.3, 0.7)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 3e-2


@pytest.mark.slow
@pytest.mark.parametrize("path", [0, 1])
def test_forward_at_512_matches_reference_on_a_crop(gpu_lib, path):
    """The network applied at 512^3 (the size the warm start runs at; some of its
    activation tensors hold more than 2^31 values) against the reference evaluated on a
    64^3 crop: outputs farther from the crop's faces than the receptive field (about 23
    voxels through the coarsest level) do not see the crop's wrap-around, so the central
    8^3 must agree."""
    n, s0, w = 512, 196, 64
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    delta = (torch.randn((n, n, n), generator=g, device="cuda", dtype=torch.float64) * 0.8).exp() - 1.0
    p = U.init_params(4)
    p[-1] = 0.1
    net = gpu_lib.UNet()
    net.set_conv_path(path)
    net.set_params(p)
    got = net.forward(delta, -1.0, 0.2, 0.9)[s0 + 28:s0 + 36, s0 + 28:s0 + 36, s0 + 28:s0 + 36].cpu().numpy()
    crop = delta[s0:s0 + w, s0:s0 + w, s0:s0 + w].cpu().numpy()
    want, _ = U.forward(p, crop, -1.0, 0.2, 0.9)
    want = want[28:36, 28:36, 28:36]
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 3e-2


@pytest.mark.parametrize("path", [0, 1])
def test_gradients_match_reference(gpu_lib, case, path):
    n, delta, target, p = case
    net = gpu_lib.UNet()
    net.set_conv_path(path)
    net.set_params(p)
    net.zero_grad()
    loss = net.loss_grad(cu(delta), cu(target, torch.float32), -0.8, 0.4, 0.9)
    g = net.get_params(grads=True).astype(np.float64)
    loss_o, g_o = U.loss_grad(p, delta, target, -0.8, 0.4, 0.9)
    assert loss == pytest.approx(loss_o, rel=3e-2)
    offs = np.cumsum([0] + [27 * ci * co + co for ci, co in U.CONVS] + [17])
    for k in range(11):
        a, b = g[offs[k]:offs[k + 1]], g_o[offs[k]:offs[k + 1]]
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        assert cos > 0.99, (k, cos)
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 0.1, k


def test_tensor_core_paths_agree_at_128(gpu_lib):
    """The tcgen05 and the mma.sync convolutions on the same network and field (128^3, every
    level on the tensor-core path): the same BF16 products with FP32 sums in another order, so
    the outputs agree to the BF16 rounding of the activations."""
    n = 128
    delta = synth.lognormal_delta(n, -2.0, 1.5, 31)
    p = U.init_params(6)
    p[-1] = 0.1
    out = []
    for path in (0, 1):
        net = gpu_lib.UNet()
        net.set_conv_path(path)
        net.set_params(p)
        out.append(net.forward(cu(delta), -2.0, 0.5, 1.0).cpu().numpy())
        net.close()
    assert np.linalg.norm(out[1] - out[0]) / np.linalg.norm(out[0]) < 1e-2


def test_target_and_linear_start(gpu_lib):
    n = 32
    d = synth.lognormal_delta(n, -2.0, 1.5, 3)
    c = O.coefficients(-0.5, 0.0, 1.0)
    chi, _, st = O.scalar_solve(d, -0.5, 0.0, 1.0, 1e-12)
    T = gpu_lib.unet_target(cu(chi), -0.5, 0.0, 1.0).cpu().numpy()
    want = c["nu"] * O.apply_N(chi, 1.0, 0.0) / c["src"]
    assert np.abs(T - want).max() <= 1e-5 * np.abs(want).max()
    lin = gpu_lib.linear_start(cu(d), -0.5, 0.0, 1.0).cpu().numpy()
    f = O.source(d, c)
    chi_lin, _, st = O.mg_solve(f, c["nu"], 0.0, 1e-13)
    # the start fields come from an FP32 FFT solve (they are guesses): FP32 accuracy
    assert np.linalg.norm(lin - chi_lin) / np.linalg.norm(chi_lin) < 2e-6


def test_training_reduces_the_loss(gpu_lib):
    from paper_2604_15434_gb300 import learned

    ctx = gpu_lib.Context(precision=1)
    net = gpu_lib.UNet(ctx)
    net.set_params(learned.init_params(1))
    pairs = learned.make_pairs(8, 32, 99, ctx, log=None)
    first = sum(net.loss_grad(d, T, *p) for d, p, T in pairs) / len(pairs)
    net.zero_grad()
    assert len(pairs) >= 6
    learned.train(net, pairs, epochs=8, lr=3e-3, batch=2, log=None, decay=1.0)  # >= 24 Adam steps
    last = sum(net.loss_grad(d, T, *p) for d, p, T in pairs) / len(pairs)
    net.zero_grad()
    assert last < 0.7 * first


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2604_15434_gb300",
                       "weights", "unet_128")


@pytest.mark.skipif(not os.path.exists(WEIGHTS + ".bin"), reason="trained weights not present")
def test_trained_warm_start(gpu_lib):
    """On held-out fields (seeds outside the training range) the learned initial guess has a
    smaller residual than chi = 0 and than the paper's linear start, and the solve from it
    converges to the same chi as the cold start, in no more outer iterations in total.  On the
    benchmark's field at 128^3 (the lognormal recipe, seed 1003, the resolution the network was
    trained at) the learned start takes fewer outer iterations in total over the four benchmark
    pairs than the cold start.  (At 256^3 and 512^3 this does not hold for the nu < 0 pairs:
    their iteration counts are a performance figure measured by the benchmark.)"""
    from paper_2604_15434_gb300 import learned

    ctx = gpu_lib.Context(precision=1, max_cycles=100)
    net = gpu_lib.UNet(ctx)
    net.set_params(learned.load_params(WEIGHTS))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77777)
    cycles_cold = cycles_warm = 0
    for kind, aB, aM, a in (("lognormal", -0.5, 0.0, 1.0), ("lognormal", -2.0, 0.0, 1.0),
                            ("zeldovich", -1.0, 0.2, 1.0), ("zeldovich", -0.8, 0.6, 0.7)):
        d = learned.gpu_field(128, kind, 1.5, gen, torch.device("cuda"), ctx)
        chi_cold, cold = gpu_lib.scalar_mg_solve(d, aB, aM, a, 1e-8, ctx=ctx)
        phi = net.warm_start(d, aB, aM, a)
        chi_warm, warm = gpu_lib.scalar_mg_solve(d, aB, aM, a, 1e-8, phi=phi, ctx=ctx)
        phl = gpu_lib.linear_start(d, aB, aM, a)
        _, lin = gpu_lib.scalar_mg_solve(d, aB, aM, a, 1e-8, phi=phl, ctx=ctx)
        assert not warm["guess_rejected"]
        assert warm["guess_rel_res"] < cold["hist"][0]
        assert warm["guess_rel_res"] < lin["guess_rel_res"]
        err = (chi_warm - chi_cold).norm() / chi_cold.norm()
        assert err < 1e-6, (kind, aB, aM, a, float(err))
        cycles_cold += cold["cycles"]
        cycles_warm += warm["cycles"]
    assert cycles_warm <= cycles_cold, (cycles_warm, cycles_cold)
    d = torch.from_numpy(synth.lognormal_delta(128, -2.0, 1.5, 1003)).cuda()
    cycles_cold = cycles_warm = 0
    for aB, aM in ((-2.0, 0.0), (-2.0, 0.5), (-0.5, 0.0), (-0.5, 0.5)):
        _, cold = gpu_lib.scalar_mg_solve(d, aB, aM, 1.0, 1e-8, ctx=ctx)
        _, warm = gpu_lib.scalar_mg_solve(d, aB, aM, 1.0, 1e-8, phi=net.warm_start(d, aB, aM, 1.0), ctx=ctx)
        cycles_cold += cold["cycles"]
        cycles_warm += warm["cycles"]
    assert cycles_warm < cycles_cold, (cycles_warm, cycles_cold)
