"""Pins for the oracle's Cattaneo step (Eq. 14, Sec. 5): tau d2C/dt2 + dC/dt = R(C), written as
dC/dt = Q, tau dQ/dt = R(C) - Q and advanced by the midpoint rule of Eq. 8-9.

What fixes the result independently of the oracle's code:
  * a lattice Fourier mode is an eigenvector of R (R = -lam C, lam from one rate evaluation), so
    (C, Q) = (A, B) cos(2 pi k.x0) stays a mode and the midpoint rule on the linear system
    y' = M y, M = [[0, 1], [-lam/tau, -1/tau]], multiplies (A, B) by I + dt M + dt^2 M^2 / 2;
  * the mode's amplitude solves the telegraph equation tau A'' + A' + lam A = 0 exactly in closed
    form, and the scheme converges to it at second order in dt;
  * as tau -> 0 (with Q(0) = R(C(0))) the solution tends to the parabolic one of Eq. 1;
  * sum m C is conserved when sum Q(0) = 0 (the pair terms of R are antisymmetric).
"""
import math

import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

V = np.array([0.1, 0.1]) / math.sqrt(2)
THETA = (1e-2, 1e-3, 1e-6)
SIDE, H_DX = 48, 3.005


def _mode(orc, k=(3, 2)):
    x = inputs.lattice_positions(2, SIDE)
    box = np.ones(2)
    H = H_DX / SIDE
    m = 1.0 / SIDE ** 2
    C = np.cos(2 * math.pi * (x @ np.array(k)))
    r, _ = orc.rate(x, V, C, m, 1.0, box, 0, H, 4.0, *THETA)
    i = np.argmax(C)
    lam = -r[i] / C[i]
    assert np.max(np.abs(r + lam * C)) < 1e-10 * lam          # an eigenvector
    return x, box, H, m, C, lam


def _mstep(lam, tau, dt):
    M = np.array([[0.0, 1.0], [-lam / tau, -1.0 / tau]])
    return np.eye(2) + dt * M + 0.5 * dt * dt * M @ M


@pytest.mark.parametrize("tau_factor", [0.1, 1.0, 10.0])
def test_cattaneo_mode_amplification_matrix(orc, tau_factor):
    """After s steps the mode's (A, B) equals (I + dt M + dt^2 M^2/2)^s (1, B0), for Q(0) = R(C(0))
    (B0 = -lam) and Q(0) = 0; tau below, at and above 1/lam."""
    x, box, H, m, C, lam = _mode(orc)
    tau = tau_factor / lam
    dt = 0.3 * min(tau, 1.0 / lam)
    s = 12
    for B0 in (-lam, 0.0):
        _, Cs, Qs, pairs = orc.step_cattaneo(x, V, C, B0 * C, m, 1.0, box, 0, H, 4.0, *THETA, dt, tau,
                                             nsteps=s)
        A, B = np.linalg.matrix_power(_mstep(lam, tau, dt), s) @ np.array([1.0, B0])
        assert np.max(np.abs(Cs - A * C)) < 1e-12
        assert np.max(np.abs(Qs - B * C)) < 1e-12 * max(lam, 1.0)
        assert pairs == 2 * s * SIDE * SIDE * 28
    # forward Euler on the system is a different matrix
    assert abs(np.linalg.matrix_power(np.eye(2) + dt * np.array([[0, 1], [-lam / tau, -1 / tau]]), s)[0, 0]
               - np.linalg.matrix_power(_mstep(lam, tau, dt), s)[0, 0]) > 1e-8


def test_cattaneo_converges_to_the_telegraph_solution(orc):
    """The mode amplitude against the exact solution of tau A'' + A' + lam A = 0, A(0) = 1,
    A'(0) = -lam (over-damped and oscillatory tau): second-order convergence in dt."""
    x, box, H, m, C, lam = _mode(orc)
    for tau in (0.1 / lam, 2.0 / lam):
        disc = complex(1.0 - 4.0 * lam * tau) ** 0.5
        mp, mm = (-1.0 + disc) / (2 * tau), (-1.0 - disc) / (2 * tau)
        cp = (-lam - mm) / (mp - mm)            # A(0) = cp + cm = 1, A'(0) = cp mp + cm mm = -lam
        cm = 1.0 - cp
        T = 3.0 / lam
        errs = []
        for s in (30, 60):
            dt = T / s
            _, Cs, _, _ = orc.step_cattaneo(x, V, C, -lam * C, m, 1.0, box, 0, H, 4.0, *THETA, dt, tau,
                                            nsteps=s)
            A_exact = (cp * np.exp(mp * T) + cm * np.exp(mm * T)).real
            errs.append(abs(Cs[np.argmax(C)] / C[np.argmax(C)] - A_exact))
        assert 3.2 < errs[0] / errs[1] < 4.8


def test_cattaneo_tends_to_the_parabolic_solution(orc):
    """Q(0) = R(C(0)): the difference to the parabolic run of Eq. 8-9 over the same time shrinks
    in proportion to tau (a Gaussian plume, not a single mode)."""
    p = inputs.Plume(dim=2, side=32, h_over_dx=1.5)
    x = inputs.lattice_positions(2, p.side)
    C = inputs.gaussian_plume(x, p.boxv, np.array([0.5, 0.5]), 0.08)
    args = (p.velocity, C, p.mass, p.rho, p.boxv, p.kernel, p.support, 4.0, p.alpha_L, p.alpha_T, p.D_m)
    r0, _ = orc.rate(x, *args)
    D = orc.dispersion_tensor(p.velocity, p.alpha_L, p.alpha_T, p.D_m)
    T = 10 * orc.dt_rule(D, p.h)
    diffs = []
    for tau in (T / 40, T / 160):
        s = int(round(T / (tau / 2)))
        dt = T / s
        _, Cp, _ = orc.step(x, p.velocity, C, p.mass, p.rho, p.boxv, p.kernel, p.support, 4.0, p.alpha_L,
                            p.alpha_T, p.D_m, dt, nsteps=s)
        _, Cc, _, _ = orc.step_cattaneo(x, p.velocity, C, r0, p.mass, p.rho, p.boxv, p.kernel, p.support,
                                        4.0, p.alpha_L, p.alpha_T, p.D_m, dt, tau, nsteps=s)
        diffs.append(np.max(np.abs(Cc - Cp)) / np.max(np.abs(Cp - C)))
    assert diffs[0] < 0.05
    assert 3.0 < diffs[0] / diffs[1] < 5.0


def test_cattaneo_conserves_mass(orc):
    """sum Q(0) = 0 (Q(0) = R(C(0))) keeps sum m C constant; Q(0) with a non-zero sum changes it by
    the integral of sum Q, which decays with time constant tau."""
    p = inputs.Plume(dim=2, side=32, h_over_dx=1.5, jitter=0.3, seed=2)
    x = inputs.lattice_positions(2, p.side, jitter=0.3, seed=2)
    C = inputs.gaussian_plume(x, p.boxv, np.array([0.4, 0.6]), 0.07)
    args = (p.velocity, C, p.mass, p.rho, p.boxv, p.kernel, p.support, 4.0, p.alpha_L, p.alpha_T, p.D_m)
    r0, _ = orc.rate(x, *args)
    D = orc.dispersion_tensor(p.velocity, p.alpha_L, p.alpha_T, p.D_m)
    dt = orc.dt_rule(D, p.h)
    tau = 2 * dt
    _, Cc, Qc, _ = orc.step_cattaneo(x, p.velocity, C, r0, p.mass, p.rho, p.boxv, p.kernel, p.support, 4.0,
                                     p.alpha_L, p.alpha_T, p.D_m, dt, tau, nsteps=20)
    assert abs(Cc.sum() - C.sum()) <= 1e-12 * C.sum()
    assert abs(Qc.sum()) <= 1e-12 * np.abs(Qc).sum()
    q0 = np.full(C.size, 1e-3)
    _, Cq, Qq, _ = orc.step_cattaneo(x, p.velocity, C, q0, p.mass, p.rho, p.boxv, p.kernel, p.support, 4.0,
                                     p.alpha_L, p.alpha_T, p.D_m, dt, tau, nsteps=20)
    # sum Q evolves exactly as the scalar midpoint rule of q' = -q / tau
    g = (1 - dt / tau + 0.5 * (dt / tau) ** 2) ** 20
    assert Qq.sum() == pytest.approx(q0.sum() * g, rel=1e-10)
