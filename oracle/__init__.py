"""Plain FP64 CPU oracle for the screened EFTofDE particle-mesh path (arXiv 2604.15434).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library in ``paper_2604_15434_gb300``; the two meet only through the
seeded synthetic inputs of ``paper_2604_15434_gb300.synth``.

The stencil, multigrid and particle parts live in ``pm_oracle.c`` (plain loops,
compiled with ``-O2 -ffp-contract=off``); the FFT Poisson solve (Sec. 3.1,
Eq. phipsi_mod) and the spherical closed form (Sec. 2.7, Eq. analytical) are
numpy.  Every function cites the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .sphere import tophat_profile  # noqa: F401  (re-export)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pm_oracle.c")
_LIB = os.path.join(_HERE, "_pm_oracle.so")
_lock = threading.Lock()
_handle = None

OMEGA_M0 = 0.3  # the paper's Omega_m0 for the static sphere (Sec. 3.6.1); used as the default
ETA_DEFAULT = 0.35  # void floor sqrt(D_floor) = eta 6|nu|/h^2 (reading R-sat of Sec. 3.3)


def build(force: bool = False) -> str:
    """Compile ``pm_oracle.c`` into ``_pm_oracle.so`` (portable flags, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            h = ctypes.CDLL(_LIB)
            D, I, LL, P = ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
            h.orc_coefficients.argtypes = [D, D, D, D, I, P]
            h.orc_apply_N.argtypes = [P, I, D, D, D, P]
            h.orc_apply_N_padded.argtypes = [P, I, D, D, D, P]
            h.orc_smooth_sweep.argtypes = [P, P, D, I, D, D, D, D, P]
            h.orc_smooth_sweep_opsplit.argtypes = [P, P, D, I, D, D, D, D, P]
            h.orc_residual.argtypes = [P, P, D, I, D, D, D, D, P, P, P]
            h.orc_residual.restype = LL
            h.orc_coarse_exact.argtypes = [P, P, I, D, D, D, D, P]
            h.orc_coarse_exact.restype = D
            h.orc_restrict.argtypes = [P, I, P]
            h.orc_prolong_add.argtypes = [P, I, P, I]
            h.orc_mg_solve.argtypes = [P, I, P, D, P, P]
            h.orc_mg_solve.restype = I
            h.orc_deposit_cic.argtypes = [P, LL, I, P]
            h.orc_density.argtypes = [P, I, LL, P]
            h.orc_accel_grid.argtypes = [P, P, D, I, I, P]
            h.orc_interp_cic.argtypes = [P, I, P, LL, P]
            h.orc_kick_drift.argtypes = [P, P, P, LL, D]
            _handle = h
    return _handle


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Coeffs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "omega_m_a", "alpha_B", "alpha_M", "geff", "E2", "hdot_over_h2", "alphaB_dot_over_h",
        "rho_term", "C2", "C4", "nu", "xi", "kappa", "mu_chi", "mu_psi", "src")]


def coefficients(alpha_B0: float, alpha_M0: float, a: float, omega_m0: float = OMEGA_M0,
                 include_dot: bool = True) -> dict:
    """EFT coefficients at scale factor a (Sec. 2.2, Eq. alpha-a, G_eff/G, Eq. linearised, Eq. chi_scm)."""
    c = _Coeffs()
    _lib().orc_coefficients(alpha_B0, alpha_M0, a, omega_m0, int(bool(include_dot)), ctypes.byref(c))
    return {n: getattr(c, n) for n, _ in _Coeffs._fields_}


def apply_N(u, nu, kappa):
    """N(u) = nu L(u) - kappa q2(u) on a periodic n^3 grid, h = 1/n (Sec. 3.2.1)."""
    u = _f64(u)
    n = u.shape[0]
    out = np.empty_like(u)
    _lib().orc_apply_N(_p(u), n, 1.0 / n, nu, kappa, _p(out))
    return out


def apply_N_padded(p, h, nu, kappa):
    """N(u) on the interior of a padded (n+2)^3 array whose ghost layer is given (Sec. 3.2.1)."""
    p = _f64(p)
    n = p.shape[0] - 2
    out = np.empty((n, n, n))
    _lib().orc_apply_N_padded(_p(p), n, h, nu, kappa, _p(out))
    return out


def smooth_sweep(u, f, lam, nu, kappa, eta, kmask=None):
    """One red-black Newton-Gauss-Seidel sweep on a periodic grid (Sec. 3.2.1, 3.3, 3.4).
    kmask (uint8, optional): per cell, the eighths of the screening term switched off
    (0 keeps kappa, 8 or more removes it)."""
    u = _f64(u).copy()
    f = _f64(f)
    n = u.shape[0]
    km = None if kmask is None else np.ascontiguousarray(kmask, dtype=np.uint8)
    _lib().orc_smooth_sweep(_p(u), _p(f), lam, n, 1.0 / n, nu, kappa, eta, _p(km))
    return u


def smooth_sweep_opsplit(u, f, lam, nu, kappa, eta, kmask=None):
    """One red-black sweep of Method II, operator splitting (Sec. 3.2.2, Eq. opsplit): each
    cell solves its equation as a quadratic in its Laplacian, with the squared traceless
    Hessian taken from the neighbours, then moves its value so its discrete Laplacian equals
    that root.  Same arguments and snapshot semantics as smooth_sweep."""
    u = _f64(u).copy()
    f = _f64(f)
    n = u.shape[0]
    km = None if kmask is None else np.ascontiguousarray(kmask, dtype=np.uint8)
    _lib().orc_smooth_sweep_opsplit(_p(u), _p(f), lam, n, 1.0 / n, nu, kappa, eta, _p(km))
    return u


def residual(u, f, lam, nu, kappa, eta, kmask=None):
    """Residual (unsaturated: f + lam - N(u); floored: nu (L_sat - L)) and the floored-cell mask."""
    u = _f64(u)
    f = _f64(f)
    n = u.shape[0]
    r = np.empty_like(u)
    sat = np.empty(u.shape, dtype=np.uint8)
    km = None if kmask is None else np.ascontiguousarray(kmask, dtype=np.uint8)
    _lib().orc_residual(_p(u), _p(f), lam, n, 1.0 / n, nu, kappa, eta, _p(km), _p(r), _p(sat))
    return r, sat


def coarse_exact(u, f, nu, kappa, eta=ETA_DEFAULT, kmask=None):
    """The exact coarsest-level solve alone (Sec. 3.4 FAS, reading of the coarse solve): Newton
    with a dense Jacobian and LU on the residual pieces of a periodic grid, the gauge multiplier
    as an extra unknown and the mean of u kept.  Returns (u, lambda)."""
    u = _f64(u).copy()
    f = _f64(f)
    n = u.shape[0]
    km = None if kmask is None else np.ascontiguousarray(kmask, dtype=np.uint8)
    lam = _lib().orc_coarse_exact(_p(u), _p(f), n, 1.0 / n, nu, kappa, eta, _p(km))
    return u, lam


def restrict(u):
    """Average of the 8 children."""
    u = _f64(u)
    n = u.shape[0]
    out = np.empty((n // 2,) * 3)
    _lib().orc_restrict(_p(u), n, _p(out))
    return out


def prolong_add(corr, fine, periodic=True):
    """fine + trilinear cell-centred prolongation of corr."""
    corr = _f64(corr)
    fine = _f64(fine).copy()
    _lib().orc_prolong_add(_p(corr), corr.shape[0], _p(fine), int(periodic))
    return fine


class _MGParams(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("kappa", ctypes.c_double), ("eta", ctypes.c_double),
                ("npre", ctypes.c_int), ("npost", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("coarsest_n", ctypes.c_int), ("coarse_sweeps", ctypes.c_int),
                ("dirichlet", ctypes.c_int), ("ghosts", ctypes.c_void_p), ("smoother", ctypes.c_int),
                ("coarse_exact", ctypes.c_int)]


class _MGInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("rel_res", ctypes.c_double), ("lam", ctypes.c_double),
                ("sat_cells", ctypes.c_longlong), ("hist", ctypes.c_double * 256)]



def mg_solve(f, nu, kappa, tol, chi0=None, eta=ETA_DEFAULT, npre=2, npost=2, max_cycles=200,
             coarsest_n=4, coarse_sweeps=100, ghosts=None, smoother=0, coarse_exact=False):
    """FAS multigrid solve of nu L(chi) - kappa q2(chi) = f (+ lambda) (Sec. 3.4).

    Periodic by default (with the gauge multiplier and <chi> = 0); with ``ghosts`` (a
    list of padded ghost arrays, finest level first) the faces are Dirichlet.  smoother 0
    is Method I (Sec. 3.2.1), 1 Method II (Sec. 3.2.2).  coarse_exact: the coarsest grid is
    solved by Newton with a dense Jacobian and LU (gauge multiplier and mean constraint as
    the extra unknown and row) instead of coarse_sweeps sweeps.
    Returns (chi, info dict, status) with status 0 = converged, 2 = not converged.
    """
    f = _f64(f)
    n = f.shape[0]
    chi = np.zeros_like(f) if chi0 is None else _f64(chi0).copy()
    gbuf = None
    if ghosts is not None:
        gbuf = np.concatenate([_f64(g).ravel() for g in ghosts])
    prm = _MGParams(nu, kappa, eta, npre, npost, max_cycles, coarsest_n, coarse_sweeps,
                    int(ghosts is not None), _p(gbuf) if gbuf is not None else None, int(smoother),
                    int(bool(coarse_exact)))
    info = _MGInfo()
    st = _lib().orc_mg_solve(_p(f), n, ctypes.byref(prm), tol, _p(chi), ctypes.byref(info))
    d = {"cycles": info.cycles, "rel_res": info.rel_res, "lambda": info.lam, "sat_cells": info.sat_cells,
         "hist": list(info.hist[: info.cycles + 1])}
    return chi, d, st


def source(delta, coeffs):
    """f = xi (3/2) (G_eff/G) a Omega_m0 delta (Eq. chi_scm moved to nu L - kappa q2 = f)."""
    return coeffs["src"] * _f64(delta)


def scalar_solve(delta, alpha_B0, alpha_M0, a, tol, omega_m0=OMEGA_M0, include_dot=True, chi0=None, **kw):
    """chi for a density contrast grid: coefficients, source and the FAS solve (Sec. 3.2-3.4)."""
    c = coefficients(alpha_B0, alpha_M0, a, omega_m0, include_dot)
    f = source(delta, c)
    if c["xi"] == 0.0:
        return np.zeros_like(f), {"cycles": 0, "rel_res": 0.0, "lambda": 0.0, "sat_cells": 0, "hist": [0.0]}, 0
    return mg_solve(f, c["nu"], c["kappa"], tol, chi0=chi0, **kw)


def deposit_cic(pos, n):
    """CIC assignment into a 2^40 fixed-point int64 grid (Sec. 3.6.2); pos is [3][np]."""
    pos = _f64(pos)
    npart = pos.shape[1]
    acc = np.empty((n, n, n), dtype=np.int64)
    _lib().orc_deposit_cic(_p(pos), npart, n, _p(acc))
    return acc


def density(acc, npart):
    """delta = rho / rho_bar - 1 from the fixed-point grid."""
    acc = np.ascontiguousarray(acc, dtype=np.int64)
    n = acc.shape[0]
    out = np.empty(acc.shape)
    _lib().orc_density(_p(acc), n, npart, _p(out))
    return out


def poisson_fft(delta, coeffs, a, omega_m0=OMEGA_M0):
    """Psi_N with L_7pt Psi_N = (3/2)(G_eff/G) a Omega_m0 delta, periodic, zero mean (Eq. phipsi_mod).

    The 7-point Laplacian's eigenvalues -(4/h^2) sum sin^2(pi m_i / n) are used so that
    this solves the same discrete equation as the multigrid Laplacian.
    """
    d = _f64(delta)
    n = d.shape[0]
    h = 1.0 / n
    rhs = 1.5 * coeffs["geff"] * a * omega_m0 * d
    m = np.fft.fftfreq(n) * n
    mr = np.fft.rfftfreq(n) * n
    s = (np.sin(np.pi * m / n) ** 2)
    sr = (np.sin(np.pi * mr / n) ** 2)
    lam = -(4.0 / h ** 2) * (s[:, None, None] + s[None, :, None] + sr[None, None, :])
    rk = np.fft.rfftn(rhs)
    lam[0, 0, 0] = 1.0
    pk = rk / lam
    pk[0, 0, 0] = 0.0
    return np.fft.irfftn(pk, s=(n, n, n), axes=(0, 1, 2))


def accel_grid(psiN, chi, xi_force, n, order=4):
    """g = -grad(Psi_N + xi_force chi) with the 5-point stencil (Eq. force, Sec. 3.5.2), or with
    the 2-point central difference for order 2; [3][n^3]."""
    psiN = _f64(psiN)
    chi = None if chi is None else _f64(chi)
    out = np.empty((3, n, n, n))
    _lib().orc_accel_grid(_p(psiN), _p(chi), xi_force, n, int(order), _p(out))
    return out


def interp_cic(grid, pos):
    """CIC gather of a [3][n^3] grid at the particles, same weights as the deposit."""
    grid = _f64(grid)
    pos = _f64(pos)
    n = grid.shape[1]
    out = np.empty_like(pos)
    _lib().orc_interp_cic(_p(grid), n, _p(pos), pos.shape[1], _p(out))
    return out


def kick_drift(pos, vel, acc, dt):
    """v += g dt; x = frac(x + v dt), in place on copies; returns (pos, vel)."""
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    acc = _f64(acc)
    _lib().orc_kick_drift(_p(pos), _p(vel), _p(acc), pos.shape[1], dt)
    return pos, vel


def pm_step(pos, vel, n, alpha_B0, alpha_M0, a, dt, tol, chi0=None, omega_m0=OMEGA_M0, include_dot=True,
            linear=False, grad_order=4, **kw):
    """One particle-mesh step: deposit, Poisson, chi solve, force, kick-drift (Sec. 3.5.1 step order).
    linear: the linearised equations (Sec. 2.5, Eq. linearised): nu L chi = xi S with L Psi_N = S,
    so chi = (xi / nu) Psi_N, with no screening term and no multigrid solve."""
    c = coefficients(alpha_B0, alpha_M0, a, omega_m0, include_dot)
    acc_grid_i = deposit_cic(pos, n)
    delta = density(acc_grid_i, pos.shape[1])
    psiN = poisson_fft(delta, c, a, omega_m0)
    if linear:
        chi = (c["xi"] / c["nu"]) * psiN if c["xi"] != 0.0 else np.zeros_like(psiN)
        info, st = {"cycles": 0}, 0
    else:
        chi, info, st = scalar_solve(delta, alpha_B0, alpha_M0, a, tol, omega_m0, include_dot, chi0=chi0, **kw)
    g = accel_grid(psiN, chi, c["xi"], n, grad_order)
    accp = interp_cic(g, pos)
    pos2, vel2 = kick_drift(pos, vel, accp, dt)
    return {"acc_fixed": acc_grid_i, "delta": delta, "psiN": psiN, "chi": chi, "info": info, "status": st,
            "acc": accp, "pos": pos2, "vel": vel2}


# ---------------------------------------------------------------- several steps and linear growth

def supercomoving_time(a0, a1, omega_m0=OMEGA_M0):
    """Supercomoving time elapsed from a0 to a1: dt~ = H0 dt / a^2, i.e. dt~/da = 1 / (a^3 E(a)) with
    E^2 = Omega_m0 a^-3 + 1 - Omega_m0 (the code units of Sec. 3.1, flat background)."""
    from scipy.integrate import quad

    val, _ = quad(lambda a: 1.0 / (a ** 3 * np.sqrt(omega_m0 / a ** 3 + 1.0 - omega_m0)), a0, a1,
                  epsabs=0.0, epsrel=1e-13, limit=200)
    return val


def step_schedule(a_start, a_end, nsteps, omega_m0=OMEGA_M0):
    """(a_n, dt) of nsteps equal supercomoving-time steps from a_start to a_end: a_n is the scale
    factor at the start of step n, from da/dt~ = a^3 E(a) integrated to 1e-12 (reading R-kd)."""
    from scipy.integrate import solve_ivp

    T = supercomoving_time(a_start, a_end, omega_m0)
    dt = T / nsteps
    ts = dt * np.arange(nsteps)
    sol = solve_ivp(lambda t, y: [y[0] ** 3 * np.sqrt(omega_m0 / y[0] ** 3 + 1.0 - omega_m0)], (0.0, T),
                    [a_start], t_eval=ts, rtol=1e-12, atol=0.0, method="DOP853")
    return sol.y[0], dt


def pm_run(pos, vel, n, alpha_B0, alpha_M0, a_start, a_end, nsteps, tol, omega_m0=OMEGA_M0, **kw):
    """nsteps particle-mesh steps (Sec. 3.5.1) at equal supercomoving-time steps from a_start to
    a_end, each warm-started from the previous chi (the paper's choice for every step after the
    first, Sec. 3.5.1).  Returns the final positions, velocities and chi."""
    a_n, dt = step_schedule(a_start, a_end, nsteps, omega_m0)
    pos, vel, chi = _f64(pos), _f64(vel), None
    for a in a_n:
        out = pm_step(pos, vel, n, alpha_B0, alpha_M0, float(a), dt, tol, chi0=chi, omega_m0=omega_m0, **kw)
        if out["status"] != 0:
            raise RuntimeError(f"oracle solve did not converge at a = {a}")
        pos, vel, chi = out["pos"], out["vel"], out["chi"]
    return pos, vel, chi


def growth_factor(alpha_B0, alpha_M0, a_eval, omega_m0=OMEGA_M0, include_dot=True, a_init=1e-3, y_init=None):
    """Linear growth D(a) and dD/da of Eq. delta_mod_a:
        D'' + (3/a + dlnH/da) D' - 3/(2 a^2) Omega_m(a) (G_eff/G) mu_Psi D = 0,
    mu_Psi = 1 + xi^2/nu (Sec. 2.5), from the matter-era growing mode D = a at a_init (the EFT
    couplings scale with 1 - Omega_m(a) and vanish there), or from y_init = (D, D') at a_init."""
    from scipy.integrate import solve_ivp

    def rhs(a, y):
        c = coefficients(alpha_B0, alpha_M0, a, omega_m0, include_dot)
        e2 = omega_m0 / a ** 3 + 1.0 - omega_m0
        dlnh = -1.5 * omega_m0 / a ** 4 / e2
        mu = c["mu_psi"] if c["xi"] != 0.0 else 1.0
        return [y[1], -(3.0 / a + dlnh) * y[1] + 1.5 / a ** 2 * c["omega_m_a"] * c["geff"] * mu * y[0]]

    y0 = [a_init, 1.0] if y_init is None else list(y_init)
    a_eval = np.atleast_1d(np.asarray(a_eval, dtype=np.float64))
    sol = solve_ivp(rhs, (a_init, float(a_eval.max())), y0, t_eval=a_eval, rtol=1e-11, atol=1e-14, method="DOP853")
    return sol.y[0], sol.y[1]


def lensing_potential(psiN, chi, alpha_B0, alpha_M0, a, omega_m0=OMEGA_M0, include_dot=True):
    """Phi = Psi_N + alpha_B chi (Eq. phipsi_mod, second line: L Phi = S + alpha_B L chi)."""
    c = coefficients(alpha_B0, alpha_M0, a, omega_m0, include_dot)
    return _f64(psiN) + c["alpha_B"] * _f64(chi)
