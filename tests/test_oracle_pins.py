"""Pins of the CPU oracle against the paper's closed forms and against mathematics.

Every test here fixes a part of the oracle to something other than the oracle itself:
an exact identity, a closed form, an independent FFT computation, a brute-force
Newton solve, or an invariance.  Each names the passage of arXiv 2604.15434 it pins.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
from oracle import sphere
from paper_2604_15434_gb300 import synth

# ---------------------------------------------------------------- coefficients


@pytest.mark.parametrize("a", [0.3, 0.55, 1.0])
def test_C2_vanishes_without_modification(a):
    """Sec. 2.2: with all alphas zero the chi equation must disappear (C2 = 0)."""
    c = O.coefficients(0.0, 0.0, a)
    assert abs(c["C2"]) < 1e-15
    assert c["geff"] == 1.0 and c["nu"] == pytest.approx(0.0, abs=1e-15)


def test_coefficients_config_c1_by_hand():
    """alpha_B0=-0.5, alpha_M0=0, a=1, Omega_m0=0.3, worked by hand from Sec. 2.2 and 2.5:
    C2 = -0.5 + 0.55*(-0.45) - 0.45 + 0.45 = -0.725, nu = 0.725 - 0.25 = 0.475,
    xi = -0.5, C4 = 2, kappa = 2/4 = 0.5."""
    c = O.coefficients(-0.5, 0.0, 1.0)
    assert c["C2"] == pytest.approx(-0.725, abs=1e-15)
    assert c["nu"] == pytest.approx(0.475, abs=1e-15)
    assert c["xi"] == -0.5 and c["C4"] == 2.0 and c["kappa"] == pytest.approx(0.5, abs=1e-15)
    assert c["mu_chi"] == pytest.approx(-0.5 / 0.475, rel=1e-15)


@pytest.mark.parametrize("aB0,aM0", [(-0.5, 0.0), (-1.0, 0.2), (-0.24, -0.2), (-2.0, 0.5)])
def test_alpha_today_and_nu_is_laplacian_prefactor(aB0, aM0):
    """Eq. alpha-a at a=1 returns alpha_I0; nu (Eq. linearised) equals Eq. chi's
    Laplacian prefactor 2 aB aM - aB^2 - C2; mu_Psi = 1 + xi^2/nu."""
    c = O.coefficients(aB0, aM0, 1.0)
    assert c["alpha_B"] == pytest.approx(aB0, rel=1e-15) and c["alpha_M"] == pytest.approx(aM0, rel=1e-15)
    assert c["nu"] == pytest.approx(2 * aB0 * aM0 - aB0 ** 2 - c["C2"], abs=1e-14)
    assert c["mu_psi"] == pytest.approx(1 + c["xi"] ** 2 / c["nu"], rel=1e-14)
    assert c["E2"] == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("aM0", [0.2, -0.2, 0.5])
def test_geff_matches_definition_by_quadrature(aM0):
    """Sec. 2.4: G_eff/G = exp(-int_0^a alpha_M(a')/a' da'), checked by quadrature
    against the closed form Omega_m(a)^(alpha_M0/(3(1-Omega_m0)))."""
    om0 = 0.3
    for a in (0.4, 0.8, 1.0):
        def am(x):
            return O.coefficients(0.0, aM0, x)["alpha_M"] / x
        integ, _ = quad(am, 1e-8, a, epsabs=1e-14, epsrel=1e-13, limit=200)
        assert O.coefficients(0.0, aM0, a)["geff"] == pytest.approx(math.exp(-integ), rel=1e-10)


def test_alphaB_dot_is_log_derivative():
    """Reading of alpha_B-dot/H as d alpha_B / d ln a (Sec. 2.2), checked by central differences."""
    for a in (0.35, 0.7, 1.0):
        e = 1e-5
        up = O.coefficients(-0.8, 0.0, a * math.exp(e))["alpha_B"]
        dn = O.coefficients(-0.8, 0.0, a * math.exp(-e))["alpha_B"]
        num = (up - dn) / (2 * e)
        assert O.coefficients(-0.8, 0.0, a)["alphaB_dot_over_h"] == pytest.approx(num, rel=1e-8)
        assert O.coefficients(-0.8, 0.0, a, include_dot=False)["alphaB_dot_over_h"] == 0.0


def test_hdot_matches_background():
    """H-dot/H^2 = d ln E / d ln a for E^2 = Omega_m0 a^-3 + 1 - Omega_m0."""
    for a in (0.4, 1.0):
        e = 1e-5
        lnE = lambda x: 0.5 * math.log(O.coefficients(0, 0, x)["E2"])
        num = (lnE(a * math.exp(e)) - lnE(a * math.exp(-e))) / (2 * e)
        assert O.coefficients(0, 0, a)["hdot_over_h2"] == pytest.approx(num, rel=1e-8)


# ---------------------------------------------------------------- discrete operator


def _padded_quadratic(n, A, b, c0, h):
    idx = (np.arange(-1, n + 1) + 0.5) * h
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    X = np.stack([x, y, z])
    quadf = 0.5 * np.einsum("i...,ij,j...->...", X, A, X)
    return quadf + np.einsum("i,i...->...", b, X) + c0


def test_operator_exact_on_quadratic_polynomials():
    """Sec. 3.2.1 stencils are exact on quadratics: L = tr A and the bracket of Eq. chi_scm
    (L chi)^2 - chi_ij chi^ij = (tr A)^2 - |A|_F^2.  A sign error, a dropped cross term or
    a transposed index in q2 changes this value."""
    rng = np.random.default_rng(7)
    n, h = 6, 1.0 / 6
    for _ in range(5):
        M = rng.standard_normal((3, 3))
        A = M + M.T
        p = _padded_quadratic(n, A, rng.standard_normal(3), 0.3, h)
        nu, kap = 0.7, 0.0
        L = O.apply_N_padded(p, h, 1.0, 0.0)
        assert np.allclose(L, np.trace(A), rtol=1e-9, atol=1e-9)
        q2 = -O.apply_N_padded(p, h, 0.0, 1.0)
        exact = np.trace(A) ** 2 - np.sum(A * A)
        assert np.allclose(q2, exact, rtol=1e-8, atol=1e-8 * max(1, abs(exact)))
        N = O.apply_N_padded(p, h, nu, 0.37)
        assert np.allclose(N, nu * np.trace(A) - 0.37 * exact, rtol=1e-8, atol=1e-8)


def test_laplacian_matches_fft_eigenvalues():
    """The 7-point Laplacian has eigenvalues -(4/h^2) sum sin^2(pi m/n) on a periodic grid."""
    rng = np.random.default_rng(3)
    n = 16
    u = rng.standard_normal((n, n, n))
    got = O.apply_N(u, 1.0, 0.0)
    m = np.fft.fftfreq(n) * n
    s = np.sin(np.pi * m / n) ** 2
    lam = -(4.0 * n * n) * (s[:, None, None] + s[None, :, None] + s[None, None, :])
    want = np.real(np.fft.ifftn(lam * np.fft.fftn(u)))
    assert np.allclose(got, want, atol=1e-9 * np.abs(want).max())


def test_operator_plane_parallel_has_no_screening():
    """For a field that varies along one axis only the discrete bracket vanishes exactly."""
    n = 16
    x = (np.arange(n) + 0.5) / n
    u = np.broadcast_to((np.sin(2 * np.pi * x) + 0.3 * np.cos(6 * np.pi * x))[None, None, :], (n, n, n)).copy()
    assert np.array_equal(O.apply_N(u, 0.0, 1.0), np.zeros_like(u))


def test_operator_commutes_with_axis_permutation_and_shift():
    rng = np.random.default_rng(11)
    n = 8
    u = rng.standard_normal((n, n, n))
    N = O.apply_N(u, 0.4, 0.9)
    assert np.allclose(O.apply_N(np.transpose(u, (1, 2, 0)), 0.4, 0.9), np.transpose(N, (1, 2, 0)), atol=1e-9)
    assert np.allclose(O.apply_N(np.roll(u, 3, axis=1), 0.4, 0.9), np.roll(N, 3, axis=1), atol=1e-9)


def test_local_update_solves_the_cell_equation():
    """Eq. quadratic: after a red half-sweep each red cell, with only its own value changed,
    zeroes its residual (real root) or sits on the floored root (Sec. 3.3)."""
    rng = np.random.default_rng(5)
    n = 8
    u = 0.002 * rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    nu, kap, eta = 0.475, 0.5, 0.35
    u1 = O.smooth_sweep(u, f, 0.0, nu, kap, eta)
    red = (np.indices(u.shape).sum(0) % 2) == 0
    checked = 0
    for cell in zip(*np.nonzero(red)):
        uc = u.copy()
        uc[cell] = u1[cell]
        r, sat = O.residual(uc, f, 0.0, nu, kap, eta)
        scale = 6 * nu * n * n * max(abs(uc[cell]), 1e-3)
        assert abs(r[cell]) < 1e-11 * scale, (cell, r[cell], sat[cell])
        checked += 1
    assert checked == n ** 3 // 2


@pytest.mark.parametrize("nu,kap", [(0.475, 0.5), (-1.1, 2.0)])
def test_method_ii_update_solves_the_cell_equation(nu, kap):
    """Method II (Sec. 3.2.2, Eq. opsplit): after its red half-sweep each red cell, with only
    its own value changed, zeroes the residual of the operator of Sec. 3.2.1 (real root), or
    of the floored piece of R-res (floored cells, exercised by the nu < 0 case)."""
    rng = np.random.default_rng(6)
    n = 8
    u = 0.002 * rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    eta = 0.35
    u1 = O.smooth_sweep_opsplit(u, f, 0.0, nu, kap, eta)
    red = (np.indices(u.shape).sum(0) % 2) == 0
    floored = 0
    for cell in zip(*np.nonzero(red)):
        uc = u.copy()
        uc[cell] = u1[cell]
        r, sat = O.residual(uc, f, 0.0, nu, kap, eta)
        scale = 6 * abs(nu) * n * n * max(abs(uc[cell]), 1e-3)
        assert abs(r[cell]) < 1e-10 * scale, (cell, r[cell], sat[cell])
        floored += int(sat[cell])
    if nu < 0:
        assert floored > 0


@pytest.mark.parametrize("aB0,aM0,masked", [(-0.5, 0.0, False), (-2.0, 0.0, False), (-2.0, 0.5, True)])
def test_method_ii_sweep_equals_method_i(aB0, aM0, masked):
    """The squared traceless Hessian holds no centre value and q2 = (2/3) L^2 - T2, so Method II's
    local solve in the Laplacian and Method I's in the cell value (Eq. quadratic) are one
    equation: a whole sweep agrees to rounding, floored and partly screened cells included."""
    n = 16
    d = synth.lognormal_delta(n, -2.0, 1.5, 1003)
    c = O.coefficients(aB0, aM0, 1.0)
    f = O.source(d, c)
    u = 1e-3 * np.random.default_rng(2).standard_normal((n, n, n))
    km = np.random.default_rng(4).integers(0, 10, (n, n, n)).astype(np.uint8) if masked else None
    a = O.smooth_sweep(u, f, 0.013, c["nu"], c["kappa"], 0.35, kmask=km)
    b = O.smooth_sweep_opsplit(u, f, 0.013, c["nu"], c["kappa"], 0.35, kmask=km)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    _, fl = O.residual(a, f, 0.013, c["nu"], c["kappa"], 0.35)
    if c["nu"] < 0:
        assert fl.sum() > 0


def test_method_ii_fas_solve_matches_method_i():
    """The FAS cycle with Method II sweeps reaches the solution of the Method I cycle."""
    n = 16
    d = synth.lognormal_delta(n, -2.0, 1.5, 1003)
    c = O.coefficients(-2.0, 0.0, 1.0)
    f = O.source(d, c)
    chi1, i1, s1 = O.mg_solve(f, c["nu"], c["kappa"], 1e-11)
    chi2, i2, s2 = O.mg_solve(f, c["nu"], c["kappa"], 1e-11, smoother=1)
    assert s1 == 0 and s2 == 0
    assert np.abs(chi1 - chi2).max() <= 1e-10 * np.abs(chi1).max()


def test_restriction_keeps_block_constants_and_the_mean():
    """R-mg restriction: a field constant on every 2x2x2 block restricts to those constants,
    and any field keeps its mean."""
    rng = np.random.default_rng(12)
    nc = 8
    blocks = rng.standard_normal((nc, nc, nc))
    fine = np.repeat(np.repeat(np.repeat(blocks, 2, 0), 2, 1), 2, 2)
    assert np.allclose(O.restrict(fine), blocks, rtol=1e-15, atol=1e-15)  # 8 equal terms summed, then / 8
    u = rng.standard_normal((16, 16, 16))
    assert abs(O.restrict(u).mean() - u.mean()) < 1e-15


def _centres(n):
    x = (np.arange(n) + 0.5) / n
    return np.meshgrid(x, x, x, indexing="ij")


def test_periodic_prolongation_is_second_order_and_keeps_constants_and_mean():
    """R-mg prolongation (trilinear, cell-centred, periodic): it adds a constant exactly, it
    keeps the mean, and for a smooth periodic field its error falls 4x per halving of h."""
    assert np.allclose(O.prolong_add(np.full((4, 4, 4), 2.5), np.zeros((8, 8, 8))), 2.5, rtol=0, atol=1e-15)
    u = np.random.default_rng(13).standard_normal((8, 8, 8))
    assert abs(O.prolong_add(u, np.zeros((16, 16, 16))).mean() - u.mean()) < 1e-15
    errs = []
    for nc in (8, 16, 32):
        g = lambda x, y, z: np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.sin(2 * np.pi * (z + 0.1))
        coarse = g(*_centres(nc))
        want = g(*_centres(2 * nc))
        errs.append(np.abs(O.prolong_add(coarse, np.zeros_like(want)) - want).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_dirichlet_prolongation_is_second_order_for_fields_vanishing_on_the_faces():
    """The fixed-boundary form (outside neighbours take minus their mirror cell) is second
    order for a field that vanishes on the box faces."""
    errs = []
    for nc in (8, 16, 32):
        g = lambda x, y, z: np.sin(np.pi * x) * np.sin(2 * np.pi * y) * np.sin(np.pi * z)
        coarse = g(*_centres(nc))
        want = g(*_centres(2 * nc))
        errs.append(np.abs(O.prolong_add(coarse, np.zeros_like(want), periodic=False) - want).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


@pytest.mark.parametrize("k", [0, 3, 8, 11])
def test_partial_screening_mask_scales_kappa(k):
    """The mask byte k of a cell keeps (8 - k)/8 of the screening term (none for k >= 8):
    a sweep with k everywhere equals the unmasked sweep with kappa scaled by that weight."""
    rng = np.random.default_rng(9)
    n = 8
    u = 0.002 * rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    nu, kap, eta = 0.475, 0.5, 0.35
    w = 0.0 if k >= 8 else (8 - k) / 8
    got = O.smooth_sweep(u, f, 0.01, nu, kap, eta, kmask=np.full((n, n, n), k, np.uint8))
    want = O.smooth_sweep(u, f, 0.01, nu, kap * w, eta)
    assert np.array_equal(got, want)
    r1, s1 = O.residual(u, f, 0.01, nu, kap, eta, kmask=np.full((n, n, n), k, np.uint8))
    r2, s2 = O.residual(u, f, 0.01, nu, kap * w, eta)
    assert np.array_equal(r1, r2) and np.array_equal(s1, s2)


def test_strongly_floored_draw_converges():
    """A draw with most cells floored (alpha = (-1.5, 0.3, 0.8): kappa/nu = 3.8, about 80% of
    the cells on the floor at sigma_ln = 1.5) converges; with coarse cells screened all or
    nothing it stalled near 1e-5 at 64^3, with the children's mean fraction it converges."""
    d = synth.lognormal_delta(64, -2.0, 1.5, 1003)
    chi, info, st = O.scalar_solve(d, -1.5, 0.3, 0.8, 1e-8, max_cycles=60, coarse_sweeps=8)
    assert st == 0 and info["rel_res"] <= 1e-8


def test_root_branch_is_linear_continuation():
    """Eq. quadratic picks the root that continues the linearised solution: for tiny kappa a
    sweep must agree with the kappa = 0 (linear Gauss-Seidel) sweep to O(kappa)."""
    rng = np.random.default_rng(9)
    n = 8
    u = 0.01 * rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    for nu in (0.475, -1.1):
        lin = O.smooth_sweep(u, f, 0.0, nu, 0.0, 0.2)
        nl = O.smooth_sweep(u, f, 0.0, nu, 1e-9, 0.2)
        assert np.abs(nl - lin).max() < 1e-8 * np.abs(lin).max()


# ---------------------------------------------------------------- multigrid solutions


def _fft_linear_solve(f, nu):
    n = f.shape[0]
    m = np.fft.fftfreq(n) * n
    s = np.sin(np.pi * m / n) ** 2
    lam = -(4.0 * n * n) * (s[:, None, None] + s[None, :, None] + s[None, None, :])
    fk = np.fft.fftn(f)
    lam[0, 0, 0] = 1.0
    uk = fk / (nu * lam)
    uk[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(uk))


def test_linear_limit_matches_fft_solve():
    """Screening off (kappa = 0): the FAS solve equals the FFT solve of nu L chi = f - <f>
    to 1e-10 relative (Eq. linearised)."""
    pos = synth.zeldovich_particles(32, -1.5, 1.0, 1001, nyquist_cutoff=True)
    d = O.density(O.deposit_cic(pos, 32), pos.shape[1])
    c = O.coefficients(-0.5, 0.0, 1.0)
    f = O.source(d, c)
    chi, info, st = O.mg_solve(f, c["nu"], 0.0, 1e-13)
    assert st == 0
    ref = _fft_linear_solve(f, c["nu"])
    assert np.linalg.norm(chi - ref) / np.linalg.norm(ref) < 1e-10


def test_plane_parallel_nonlinear_equals_linear():
    """With kappa != 0 but a source varying along z only, q2 vanishes exactly, so the
    nonlinear solve must return the FFT linear solution (no floor triggered)."""
    n = 32
    z = (np.arange(n) + 0.5) / n
    prof = 0.5 * np.sin(2 * np.pi * z) + 0.2 * np.cos(4 * np.pi * z + 0.4)
    d = np.broadcast_to(prof[:, None, None], (n, n, n)).copy()
    c = O.coefficients(-0.5, 0.0, 1.0)
    f = O.source(d, c)
    chi, info, st = O.mg_solve(f, c["nu"], c["kappa"], 1e-13)
    assert st == 0 and info["sat_cells"] == 0
    ref = _fft_linear_solve(f, c["nu"])
    assert np.linalg.norm(chi - ref) / np.linalg.norm(ref) < 1e-10


def _newton_dense(f, nu, kap, eta, chi0):
    """Brute force: damped Newton on the residual map (r(chi, lambda), <chi>) of the whole grid.
    The residual is piecewise quadratic, so central differences give its Jacobian exactly
    (up to rounding) wherever no cell changes piece; a backtracking line search on |F|
    globalises the iteration."""
    n = f.shape[0]
    m = n ** 3
    chi = chi0.copy()
    lam = 0.0
    fnorm = np.linalg.norm(f - f.mean())

    def F_of(chi, lam):
        r, _ = O.residual(chi, f, lam, nu, kap, eta)
        return np.concatenate([r.ravel(), [chi.mean() * 6 * abs(nu) * n * n]])

    F = F_of(chi, lam)
    for it in range(200):
        if np.linalg.norm(F) < 1e-14 * fnorm:
            return chi, lam, it
        J = np.zeros((m + 1, m + 1))
        t = 1e-6 * max(np.abs(chi).max(), 1e-6)
        for j in range(m):
            e = np.zeros(m)
            e[j] = t
            J[:, j] = (F_of(chi + e.reshape(chi.shape), lam) - F_of(chi - e.reshape(chi.shape), lam)) / (2 * t)
        tl = 1e-6 * max(abs(lam), np.abs(f).max())
        J[:, m] = (F_of(chi, lam + tl) - F_of(chi, lam - tl)) / (2 * tl)
        dx = np.linalg.solve(J, -F)
        step = 1.0
        while step > 1e-4:
            chi_t = chi + step * dx[:m].reshape(chi.shape)
            lam_t = lam + step * dx[m]
            Ft = F_of(chi_t, lam_t)
            if np.linalg.norm(Ft) < (1 - 1e-4 * step) * np.linalg.norm(F):
                break
            step *= 0.5
        chi, lam, F = chi_t, lam_t, Ft
    raise AssertionError("dense Newton did not converge")


@pytest.mark.parametrize("amp", [0.5, 3.0])
def test_fas_matches_dense_newton_8cubed(amp):
    """A full Newton solve of the discrete system on an
    8^3 grid agrees with the FAS multigrid to 1e-12 (amp = 3 exercises the screening term)."""
    rng = np.random.default_rng(21)
    n = 8
    g = rng.standard_normal((n, n, n))
    d = amp * (g - g.mean())
    c = O.coefficients(-0.5, 0.0, 1.0)
    f = O.source(d, c)
    chi_mg, info, st = O.mg_solve(f, c["nu"], c["kappa"], 1e-14, coarsest_n=4)
    assert st == 0
    chi_lin = _fft_linear_solve(f, c["nu"])
    chi_nt, lam, it = _newton_dense(f, c["nu"], c["kappa"], O.ETA_DEFAULT, chi_lin)
    assert np.linalg.norm(chi_mg - chi_nt) / np.linalg.norm(chi_nt) < 1e-12
    assert info["lambda"] == pytest.approx(lam, abs=1e-10 * np.abs(f).max())


@pytest.mark.parametrize("amp", [0.5, 3.0])
def test_exact_coarse_solve_matches_dense_newton_8cubed(amp):
    """The exact coarsest-level solve (Newton, analytic dense Jacobian, LU; Sec. 3.4 FAS reading)
    run as the only level of an 8^3 grid is the whole discrete problem: it must land on the
    brute-force Newton solution (finite-difference Jacobian) to 1e-12, with the same lambda."""
    rng = np.random.default_rng(21)
    n = 8
    g = rng.standard_normal((n, n, n))
    d = amp * (g - g.mean())
    c = O.coefficients(-0.5, 0.0, 1.0)
    f = O.source(d, c)
    chi_ex, info, st = O.mg_solve(f, c["nu"], c["kappa"], 1e-14, coarsest_n=8, coarse_exact=True)
    assert st == 0 and info["cycles"] <= 4
    chi_nt, lam, _ = _newton_dense(f, c["nu"], c["kappa"], O.ETA_DEFAULT, _fft_linear_solve(f, c["nu"]))
    assert np.linalg.norm(chi_ex - chi_nt) / np.linalg.norm(chi_nt) < 1e-12
    assert info["lambda"] == pytest.approx(lam, abs=1e-10 * np.abs(f).max())
    if amp == 3.0:
        assert info["sat_cells"] > 0  # the floored pieces are part of the solved system


def test_exact_coarse_solve_alone_zeroes_the_residual_with_a_mask():
    """One exact solve of a 4^3 level with partial screening weights: every residual piece of
    R-res vanishes to 1e-12 of |f| at the returned lambda, and the mean of the start is kept."""
    rng = np.random.default_rng(31)
    n = 4
    c = O.coefficients(-2.0, 0.5, 1.0)
    f = O.source(2.0 * rng.standard_normal((n, n, n)), c)
    km = rng.integers(0, 9, size=(n, n, n)).astype(np.uint8)
    u0 = 1e-3 * rng.standard_normal((n, n, n))
    u, lam = O.coarse_exact(u0, f, c["nu"], c["kappa"], kmask=km)
    r, sat = O.residual(u, f, lam, c["nu"], c["kappa"], O.ETA_DEFAULT, kmask=km)
    assert np.abs(r).max() < 1e-12 * np.abs(f).max()
    assert u.mean() == pytest.approx(u0.mean(), abs=1e-15)


@pytest.mark.parametrize("aB0,aM0", [(-0.5, 0.0), (-2.0, 0.0), (-2.0, 0.5)])
def test_exact_coarsest_level_keeps_the_solution(aB0, aM0):
    """The coarse solve only changes how the FAS cycle converges: with the exact coarsest solve
    the 32^3 lognormal problems (floored, nu < 0 included) reach the same chi to 1e-10 in no more
    cycles than with sweeps."""
    d = synth.lognormal_delta(32, -2.0, 1.5, 1003)
    c = O.coefficients(aB0, aM0, 1.0)
    f = O.source(d, c)
    a, ia, sa = O.mg_solve(f, c["nu"], c["kappa"], 1e-12)
    b, ib, sb = O.mg_solve(f, c["nu"], c["kappa"], 1e-12, coarse_exact=True)
    assert sa == 0 and sb == 0
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-10
    assert ib["cycles"] <= ia["cycles"]


def test_solution_commutes_with_axis_permutation():
    pos = synth.zeldovich_particles(16, -1.5, 1.0, 1234, nyquist_cutoff=True)
    d = O.density(O.deposit_cic(pos, 16), pos.shape[1])
    chi, _, st = O.scalar_solve(d, -0.5, 0.0, 1.0, 1e-13)
    chi2, _, st2 = O.scalar_solve(np.transpose(d, (2, 0, 1)), -0.5, 0.0, 1.0, 1e-13)
    assert st == 0 and st2 == 0
    assert np.linalg.norm(np.transpose(chi, (2, 0, 1)) - chi2) / np.linalg.norm(chi) < 1e-11


@pytest.mark.parametrize("aB0,aM0", [(-0.5, 0.0), (-2.0, 0.0), (-2.0, 0.5)])
def test_floored_solution_is_unique(aB0, aM0):
    """Reading R-sat (Sec. 3.3): with the floored discriminant the discrete problem has one
    solution.  Two different starting points (zero and the linear FFT solution) and two
    cycle shapes must land on the same field, including strongly floored cases (nu < 0)."""
    d = synth.lognormal_delta(32, -2.0, 1.5, 1003)
    c = O.coefficients(aB0, aM0, 1.0)
    f = O.source(d, c)
    a, ia, sa = O.mg_solve(f, c["nu"], c["kappa"], 1e-13)
    b, ib, sb = O.mg_solve(f, c["nu"], c["kappa"], 1e-13, chi0=_fft_linear_solve(f, c["nu"]), npre=3, npost=1)
    assert sa == 0 and sb == 0 and ia["sat_cells"] > 0
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-10


def test_void_floor_sensitivity_on_the_benchmark_pairs():
    """Reading R-sat (Sec. 3.3: the discriminant of void cells without a real root is set to
    'a very low value close to zero'): how much the floor value eta decides the solution, on a
    32^3 field of the benchmark recipe (lognormal, P ~ k^-2, sigma_ln 1.5).  eta = 0 is the
    literal reading: only cells with D < 0 are floored, and they sit at the parabola's vertex
    L = 3 nu / (4 kappa).  The nu > 0 pairs are barely touched: (-0.5, 0.5) has no floored cell,
    so every eta gives the same chi, and (-0.5, 0) moves by at most 4% in chi and 1.5% in the
    force from eta = 0.35 down to the literal floor.  For the nu < 0 pair (-2, 0) the floor
    covers more than half of the box and eta decides the solution at the 10-30% level."""
    n = 32
    d = synth.lognormal_delta(n, -2.0, 1.5, 1003)
    res = {}
    for aB0, aM0 in ((-0.5, 0.5), (-0.5, 0.0), (-2.0, 0.0)):
        c = O.coefficients(aB0, aM0, 1.0)
        f = O.source(d, c)
        psi = O.poisson_fft(d, c, 1.0)
        ref, iref, st = O.mg_solve(f, c["nu"], c["kappa"], 1e-11)
        assert st == 0
        gref = O.accel_grid(psi, ref, c["xi"], n)
        rows = [(O.ETA_DEFAULT, iref["sat_cells"] / n ** 3, 0.0, 0.0)]
        for eta in (0.25, 0.05, 0.0):
            x, info, st = O.mg_solve(f, c["nu"], c["kappa"], 1e-11, eta=eta, max_cycles=400)
            assert st == 0
            g = O.accel_grid(psi, x, c["xi"], n)
            rows.append((eta, info["sat_cells"] / n ** 3, np.linalg.norm(x - ref) / np.linalg.norm(ref),
                         np.linalg.norm(g - gref) / np.linalg.norm(gref)))
            if eta == 0.0:
                # the literal floor: floored cells exactly at the vertex, the rest with D >= 0 and
                # a zero residual
                r, sat = O.residual(x, f, info["lambda"], c["nu"], c["kappa"], 0.0)
                w = sat == 0
                r = r - w * (r.sum() / max(w.sum(), 1))
                assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(f - f.mean())
        res[(aB0, aM0)] = rows
    assert all(r[1] == 0.0 and r[2] < 1e-9 for r in res[(-0.5, 0.5)])
    rows = res[(-0.5, 0.0)]
    assert all(rows[k + 1][1] < rows[k][1] for k in range(3))  # a lower floor floors fewer cells
    assert all(rows[k + 1][2] > rows[k][2] for k in range(3))  # and moves chi further from eta = 0.35
    assert rows[-1][2] < 0.045 and rows[-1][3] < 0.016
    rows = res[(-2.0, 0.0)]
    assert all(r[1] > 0.5 for r in rows)
    assert rows[1][2] > 0.05 and rows[-1][2] > 0.2


# ---------------------------------------------------------------- spherical closed form


def _sphere_setup(n, kind, nu, kap, xi, S0, R):
    h = 1.0 / n
    levels = []
    nl = n
    while nl >= 4:
        levels.append(nl)
        nl //= 2
    ghosts = []
    for nl in levels:
        hl = 1.0 / nl
        idx = (np.arange(-1, nl + 1) + 0.5) * hl - 0.5
        z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
        r = np.sqrt(x * x + y * y + z * z)
        prof = sphere.tophat_profile(r, S0, R, nu, kap, xi) if kind == "tophat" else \
            sphere.gauss_profile(r, S0, R, nu, kap, xi)
        ghosts.append(prof)
    idx = (np.arange(n) + 0.5) * h - 0.5
    z, y, x = np.meshgrid(idx, idx, idx, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    if kind == "tophat":
        # cell average of the top-hat (volume fraction from 8^3 sub-samples per cell), the
        # consistent finite-volume source for the sharp-edged closed form
        sub = (np.arange(8) + 0.5) / 8 - 0.5
        frac = np.zeros_like(r)
        for dz in sub:
            for dy in sub:
                for dx in sub:
                    frac += ((x + dx * h) ** 2 + (y + dy * h) ** 2 + (z + dz * h) ** 2) <= R * R
        S = S0 * frac / 512.0
    else:
        S = S0 * np.exp(-0.5 * (r / R) ** 2)
    return r, xi * S, ghosts


def test_tophat_sphere_matches_closed_form():
    """Sec. 3.6.1 / Fig. grids analogue: top-hat source, Dirichlet faces from the closed form,
    config-1 coefficients, strongly screened (nu^2 << 8 kappa |xi| y_N).  The paper reports
    chi within 0.2% at 32^3 and 64^3; here chi is within 0.5% (32^3) and 0.25% (64^3) of
    the central value, and the error falls with resolution."""
    c = O.coefficients(-0.5, 0.0, 1.0)
    nu, kap, xi = c["nu"], c["kappa"], c["xi"]
    S0, R = 6.0, 0.2
    assert 8 * kap * abs(xi) * S0 / 3 > 10 * nu ** 2  # deep in the screened regime
    errs = []
    for n in (32, 64):
        r, f, ghosts = _sphere_setup(n, "tophat", nu, kap, xi, S0, R)
        chi, info, st = O.mg_solve(f, nu, kap, 1e-11, ghosts=ghosts)
        assert st == 0 and info["sat_cells"] == 0
        ref = sphere.tophat_profile(r, S0, R, nu, kap, xi)
        errs.append(np.abs(chi - ref).max() / np.abs(ref).max())
    assert errs[0] < 5e-3 and errs[1] < 2.5e-3 and errs[1] < errs[0] / 1.8, errs


def test_gaussian_sphere_converges_second_order():
    """Same closed form with a smooth source: the discretisation error at 16^3 -> 32^3 falls
    by about 4 (the 7-point and 4h^2 cross stencils are second order)."""
    c = O.coefficients(-0.5, 0.0, 1.0)
    nu, kap, xi = c["nu"], c["kappa"], c["xi"]
    S0, s = 8.0, 0.07
    errs = []
    for n in (16, 32):
        r, f, ghosts = _sphere_setup(n, "gauss", nu, kap, xi, S0, s)
        chi, info, st = O.mg_solve(f, nu, kap, 1e-12, ghosts=ghosts)
        assert st == 0
        ref = sphere.gauss_profile(r, S0, s, nu, kap, xi)
        errs.append(np.abs(chi - ref).max() / np.abs(ref).max())
    assert errs[1] < 4e-3
    assert 3.3 < errs[0] / errs[1] < 4.7, errs


def test_spherical_ratio_limits():
    """Fig. spher-ana: Psi'/Psi'_GR -> mu_Psi far from the mass and -> 1 deep inside the
    screening radius (Eq. analytical)."""
    c = O.coefficients(-0.5, 0.0, 1.0)
    far = sphere.radial_derivative_ratio(1e-9, c["nu"], c["kappa"], c["xi"])
    near = sphere.radial_derivative_ratio(1e9, c["nu"], c["kappa"], c["xi"])
    assert far == pytest.approx(c["mu_psi"], rel=1e-6)
    assert near == pytest.approx(1.0, abs=2e-4)


# ---------------------------------------------------------------- particle-mesh steps


def test_cic_mass_and_single_particle():
    """CIC (Sec. 3.6.2): weights sum to one per particle; a particle at a cell centre
    lands in one cell; one at a quarter-cell offset splits 3/4 : 1/4 exactly."""
    n = 8
    pos = np.array([[0.5 / n], [1.5 / n], [2.5 / n]])
    acc = O.deposit_cic(pos, n)
    assert acc[2, 1, 0] == 2 ** 40 and np.count_nonzero(acc) == 1
    pos = np.array([[0.75 / n], [1.5 / n], [2.5 / n]])
    acc = O.deposit_cic(pos, n)
    assert acc[2, 1, 0] == 3 * 2 ** 38 and acc[2, 1, 1] == 2 ** 38 and np.count_nonzero(acc) == 2
    pos = np.array([[0.1 / n], [7.9 / n], [0.0]])  # wraps on every axis
    acc = O.deposit_cic(pos, n)
    assert acc.sum() == 2 ** 40 and acc[7, 7, 7] > 0


def test_cic_is_permutation_invariant_and_mass_exact():
    pos = synth.zeldovich_particles(16, -1.5, 2.0, 77)
    acc = O.deposit_cic(pos, 16)
    perm = np.random.default_rng(1).permutation(pos.shape[1])
    assert np.array_equal(acc, O.deposit_cic(pos[:, perm], 16))
    assert abs(int(acc.sum()) - pos.shape[1] * 2 ** 40) <= 8 * pos.shape[1]


def test_interp_is_adjoint_of_deposit():
    """Same weights for assignment and interpolation (no self-force): sum_p W g = sum_c rho g."""
    rng = np.random.default_rng(2)
    n = 8
    pos = rng.random((3, 50))
    grid = rng.standard_normal((3, n, n, n))
    at_p = O.interp_cic(grid, pos)
    acc = O.deposit_cic(pos, n).astype(np.float64) / 2 ** 40
    for d in range(3):
        assert at_p[d].sum() == pytest.approx((acc * grid[d]).sum(), rel=1e-9)
    const = np.ones((3, n, n, n)) * 2.5
    assert np.allclose(O.interp_cic(const, pos), 2.5, rtol=1e-15)


def test_poisson_fft_solves_the_7pt_equation():
    """Eq. phipsi_mod: L_7pt Psi_N = (3/2)(G_eff/G) a Omega_m0 delta (zero-mean part)."""
    d = synth.lognormal_delta(16, -2.0, 1.0, 4)
    c = O.coefficients(-1.0, 0.2, 0.8)
    psi = O.poisson_fft(d, c, 0.8)
    lap = O.apply_N(psi, 1.0, 0.0)
    rhs = 1.5 * c["geff"] * 0.8 * 0.3 * d
    assert np.allclose(lap, rhs - rhs.mean(), atol=1e-10 * np.abs(rhs).max())
    assert abs(psi.mean()) < 1e-14


def test_five_point_gradient_spectral_factor():
    """Sec. 3.5.2 five-point stencil on a sinusoid: derivative times (8 sin t - sin 2t)/(6 t),
    t = k h, which is 1 - t^4/30 + O(t^6) (fourth order)."""
    n = 32
    x = (np.arange(n) + 0.5) / n
    for m in (1, 3):
        k = 2 * np.pi * m
        psi = np.broadcast_to(np.sin(k * x)[None, None, :], (n, n, n)).copy()
        g = O.accel_grid(psi, None, 0.0, n)
        t = k / n
        fac = (8 * np.sin(t) - np.sin(2 * t)) / (6 * t)
        want = -k * np.cos(k * x) * fac
        assert np.allclose(g[0, 0, 0, :], want, atol=1e-12 * k)
        assert np.allclose(g[1], 0.0, atol=1e-9) and np.allclose(g[2], 0.0, atol=1e-9)
        assert abs(fac - (1 - t ** 4 / 30)) < t ** 6


def test_two_point_gradient_spectral_factor():
    """The grad_order = 2 option: the two-point central difference on a sinusoid gives the
    derivative times sin(t)/t, t = k h, which is 1 - t^2/6 + O(t^4) (second order); each axis
    sees only its own variation."""
    n = 32
    x = (np.arange(n) + 0.5) / n
    for m, axis in ((1, 0), (3, 2)):
        k = 2 * np.pi * m
        prof = np.sin(k * x)
        psi = np.broadcast_to(prof[None, None, :] if axis == 0 else prof[:, None, None], (n, n, n)).copy()
        g = O.accel_grid(psi, None, 0.0, n, order=2)
        t = k / n
        fac = np.sin(t) / t
        want = -k * np.cos(k * x) * fac
        line = g[0, 0, 0, :] if axis == 0 else g[2, :, 0, 0]
        assert np.allclose(line, want, atol=1e-12 * k)
        others = [d for d in range(3) if d != axis]
        assert all(np.allclose(g[d], 0.0, atol=1e-9) for d in others)
        assert abs(fac - (1 - t ** 2 / 6)) < t ** 4 / 100


def test_force_adds_fifth_force_with_coupling():
    """Eq. force / Eq. phipsi_mod: the grid force is -grad(Psi_N + (alpha_B - alpha_M) chi)."""
    rng = np.random.default_rng(4)
    n = 8
    psi = rng.standard_normal((n, n, n))
    chi = rng.standard_normal((n, n, n))
    g = O.accel_grid(psi, chi, -0.7, n)
    assert np.allclose(g, O.accel_grid(psi, None, 0.0, n) - 0.7 * O.accel_grid(chi, None, 0.0, n), atol=1e-10)


def test_kick_drift_closed_form_and_wrap():
    pos = np.array([[0.95], [0.1], [0.5]])
    vel = np.array([[1.0], [-2.0], [0.0]])
    acc = np.array([[10.0], [0.0], [-4.0]])
    p2, v2 = O.kick_drift(pos, vel, acc, 0.01)
    assert np.allclose(v2[:, 0], [1.1, -2.0, -0.04])
    assert np.allclose(p2[:, 0], [(0.95 + 0.011) % 1.0, 0.08, 0.5 - 0.0004])


# ---------------------------------------------------------------- several steps and linear growth


def test_lcdm_growth_matches_heath_integral():
    """Eq. delta_mod_a with mu_Psi = G_eff/G = 1 is the LCDM growth equation, whose growing mode
    is D(a) = (5 Omega_m0 / 2) E(a) int_0^a da' / (a' E(a'))^3 (normalised to D -> a early)."""
    from scipy.integrate import quad

    om = O.OMEGA_M0
    E = lambda a: math.sqrt(om / a ** 3 + 1.0 - om)  # noqa: E731
    a_ev = [0.2, 0.5, 1.0]
    D, dD = O.growth_factor(0.0, 0.0, a_ev)
    for a, d in zip(a_ev, D):
        want = 2.5 * om * E(a) * quad(lambda x: 1.0 / (x * E(x)) ** 3, 0.0, a, epsrel=1e-12)[0]
        assert d == pytest.approx(want, rel=2e-7)


def test_supercomoving_schedule_einstein_de_sitter():
    """With Omega_m0 = 1, dt~/da = a^(-3/2): the run lasts 2 (a0^-1/2 - a1^-1/2) and the step
    starts satisfy a_n^-1/2 = a0^-1/2 - n dt / 2."""
    a_n, dt = O.step_schedule(0.25, 1.0, 8, omega_m0=1.0)
    assert dt * 8 == pytest.approx(2.0 * (0.25 ** -0.5 - 1.0), rel=1e-12)
    want = (0.25 ** -0.5 - 0.5 * dt * np.arange(8)) ** -2
    assert np.allclose(a_n, want, rtol=1e-10)


def test_multistep_run_reproduces_linear_growth_ratio():
    """Several PM steps from Zel'dovich initial conditions at a = 0.1 to a = 1 (16^3, 30 steps):
    on the largest scales the EFT / LCDM ratio of the density modes follows the ratio of the
    growth factors of Eq. delta_mod_a (the paper's large-scale check of Sec. 4.2)."""
    n, a_i, a_f = 16, 0.1, 1.0
    x0 = synth.zeldovich_particles(n, -1.5, 1.0, 4242)
    q = (np.indices((n, n, n))[::-1].reshape(3, -1) + 0.5) / n
    psi = (x0 - q + 0.5) % 1.0 - 0.5
    D, dD = O.growth_factor(0.0, 0.0, [a_i, a_f])
    s = 0.1 / D[1]
    pos = (q + s * D[0] * psi) % 1.0
    vel = s * a_i ** 3 * math.sqrt(0.3 / a_i ** 3 + 0.7) * dD[0] * psi

    def fundamental(p):
        F = np.fft.rfftn(O.density(O.deposit_cic(p, n), p.shape[1]))
        return np.array([F[0, 0, 1], F[0, 1, 0], F[1, 0, 0]])

    m = {}
    for name, ab in (("lcdm", (0.0, 0.0)), ("eft", (-0.5, 0.0))):
        p, v, chi = O.pm_run(pos, vel, n, ab[0], ab[1], a_i, a_f, 30, 1e-9)
        m[name] = fundamental(p)
    De, _ = O.growth_factor(-0.5, 0.0, [a_f], a_init=a_i, y_init=(D[0], dD[0]))
    ratio = np.real(m["eft"] / m["lcdm"])
    assert np.all(np.abs(ratio / (De[0] / D[1]) - 1.0) < 5e-3), ratio


def test_linearised_mode_equals_unscreened_solve_and_mu_factors():
    """Eq. linearised: with the screening term dropped, nu L chi = xi S, so the linear-mode chi =
    (xi/nu) Psi_N is the kappa = 0 multigrid solution of the same source; and
    then Psi = Psi_N + (alpha_B - alpha_M) chi = mu_Psi Psi_N, Phi = mu_Phi Psi_N with
    mu_Psi = 1 + xi^2/nu and mu_Phi = 1 + xi alpha_B / nu."""
    n = 16
    pos = synth.zeldovich_particles(n, -1.5, 0.5, 31)
    vel = np.zeros_like(pos)
    aB0, aM0, a = -0.5, 0.2, 0.8
    c = O.coefficients(aB0, aM0, a)
    out = O.pm_step(pos, vel, n, aB0, aM0, a, 1e-3, 1e-12, linear=True)
    psiN, chi = out["psiN"], out["chi"]
    f = O.source(out["delta"], c)
    chi_mg, info, st = O.mg_solve(f, c["nu"], 0.0, 1e-13)
    assert st == 0
    chi_mg = chi_mg - chi_mg.mean()
    assert np.linalg.norm(chi - chi_mg) < 1e-9 * np.linalg.norm(chi_mg)
    psi = psiN + c["xi"] * chi
    assert np.allclose(psi, (1.0 + c["xi"] ** 2 / c["nu"]) * psiN, rtol=0, atol=1e-14 * np.abs(psiN).max())
    assert c["mu_psi"] == pytest.approx(1.0 + c["xi"] ** 2 / c["nu"], rel=1e-14)
    Phi = O.lensing_potential(psiN, chi, aB0, aM0, a)
    assert np.allclose(Phi, (1.0 + c["xi"] * c["alpha_B"] / c["nu"]) * psiN, rtol=0,
                       atol=1e-14 * np.abs(psiN).max())
