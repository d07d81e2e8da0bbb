"""Pins for the oracle's misfit gradient (the reference for the GPU adjoint): the tangent-linear
gradient against central finite differences in FP64, and the linear dependence of Eq. 4 on
(alpha_L, alpha_T, D_m)."""
import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs


def _setup(side=24, steps=12):
    p = inputs.Plume(dim=2, side=side, h_over_dx=1.6, alpha_L=1e-2, alpha_T=1e-3, D_m=1e-6)
    xq, C = p.initial_state()
    x = inputs.from_fixed(xq, p.boxv)
    return p, x, C.astype(np.float64)


def test_rate_is_linear_in_theta(orc):
    p, x, C = _setup()
    args = (x, p.velocity, C, p.mass, 1.0, p.boxv, 0, p.support, 4.0)
    th = (0.02, 0.003, 1e-4)
    r = orc.rate(*args, *th)[0]
    rk = [orc.rate(*args, *np.eye(3)[k])[0] for k in range(3)]
    assert np.max(np.abs(r - sum(t * q for t, q in zip(th, rk)))) <= 1e-12 * np.max(np.abs(r))


def test_tlm_gradient_equals_central_differences(orc):
    p, x, C = _setup()
    dt = 2.0e-3
    th = np.array([1e-2, 1e-3, 1e-6])
    kw = dict(m=p.mass, rho=1.0, box=p.boxv, kind=0, H=p.support, gamma=4.0, dt=dt, nsteps=12)
    _, target = orc.misfit(x, p.velocity, C, theta=np.array([2e-2, 2e-3, 1e-6]),
                           target=np.zeros_like(C), **kw)
    J, g = orc.misfit_gradient_tlm(x, p.velocity, C, theta=th, target=target, **kw)
    for k in range(3):
        eps = 1e-4 * th[k]
        tp = th.copy(); tp[k] += eps
        tm = th.copy(); tm[k] -= eps
        Jp, _ = orc.misfit(x, p.velocity, C, theta=tp, target=target, **kw)
        Jm, _ = orc.misfit(x, p.velocity, C, theta=tm, target=target, **kw)
        fd = (Jp - Jm) / (2 * eps)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-12 * abs(J) / th[k])
