"""The hand-written adjoint (ade_adjoint) against the FP64 oracle: the misfit, its gradient with
respect to (alpha_L, alpha_T, D_m) against the oracle's tangent-linear gradient and central finite
differences, and dJ/dC0 along random directions against finite differences; the configured
inversion problem (512^2, 400 steps, checkpoints every 40) against stored FP64 oracle values;
bitwise independence of the checkpoint interval; an adjoint dot-product identity at the full
size; the torch.autograd.Function wrapper."""
import importlib.util
import os

import numpy as np
import pytest

from paper_2108_09488_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))

pytestmark = pytest.mark.gpu

THETA = np.array([1e-2, 1e-3, 1e-6])
THETA_STAR = np.array([2e-2, 2e-3, 1e-6])
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _problem(lib, orc, side, nsteps, h_dx=1.3):
    p = inputs.Plume(dim=2, side=side, h_over_dx=h_dx, alpha_L=THETA[0], alpha_T=THETA[1], D_m=THETA[2])
    xq, C = p.initial_state()
    sim = lib.Simulation(lib.params_for(p), xq, C)
    dt = sim.info.dt
    x = inputs.from_fixed(xq, p.boxv)
    kw = dict(m=p.mass, rho=1.0, box=p.boxv, kind=0, H=p.support, gamma=4.0, dt=dt, nsteps=nsteps)
    _, target = orc.misfit(x, p.velocity, C.astype(np.float64), theta=THETA_STAR,
                           target=np.zeros(p.n), **kw)
    return p, sim, x, C, target, kw


def test_adjoint_against_oracle_tlm_and_fd(adelib, orc, torch_cuda):
    p, sim, x, C, target, kw = _problem(adelib, orc, 64, 40)
    J, g, dC0, _ = sim.adjoint(target.astype(np.float32), 40, 8)
    Jo, go = orc.misfit_gradient_tlm(x, p.velocity, C.astype(np.float64), theta=THETA,
                                     target=target, **kw)
    assert J == pytest.approx(Jo, rel=1e-5)
    for k in range(3):
        assert g[k] == pytest.approx(go[k], rel=GRAD_TOL)
    # alpha_L by FP64 central differences (eps = 1e-4 relative)
    eps = 1e-4 * THETA[0]
    Jp, _ = orc.misfit(x, p.velocity, C.astype(np.float64), theta=THETA + [eps, 0, 0], target=target, **kw)
    Jm, _ = orc.misfit(x, p.velocity, C.astype(np.float64), theta=THETA - [eps, 0, 0], target=target, **kw)
    assert g[0] == pytest.approx((Jp - Jm) / (2 * eps), rel=GRAD_TOL)
    # dJ/dC0 along two random directions
    d0 = dC0.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(2):
        delta = rng.normal(size=p.n)
        e = 1e-3
        Jp, _ = orc.misfit(x, p.velocity, C + e * delta, theta=THETA, target=target, **kw)
        Jm, _ = orc.misfit(x, p.velocity, C - e * delta, theta=THETA, target=target, **kw)
        assert np.dot(d0, delta) == pytest.approx((Jp - Jm) / (2 * e), rel=GRAD_TOL)


def test_adjoint_checkpoint_interval_is_bitwise_irrelevant(adelib, orc, torch_cuda):
    p, sim, x, C, target, kw = _problem(adelib, orc, 48, 23)
    res = [sim.adjoint(target.astype(np.float32), 23, ck) for ck in (1, 5, 23, 40)]
    for J, g, d, _ in res[1:]:
        assert J == res[0][0] and np.array_equal(g, res[0][1])
        assert np.array_equal(d.cpu().numpy(), res[0][2].cpu().numpy())


def test_adjoint_512_theta_gradient(adelib, orc, torch_cuda):
    """The 512^2 plume of the inversion problem over 20 steps against the oracle TLM."""
    p, sim, x, C, target, kw = _problem(adelib, orc, 512, 20)
    J, g, _, _ = sim.adjoint(target.astype(np.float32), 20, 40)
    Jo, go = orc.misfit_gradient_tlm(x, p.velocity, C.astype(np.float64), theta=THETA, target=target, **kw)
    assert J == pytest.approx(Jo, rel=1e-5)
    for k in range(3):
        assert g[k] == pytest.approx(go[k], rel=GRAD_TOL)


def _adjoint_golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "adjoint_512_400.txt")) as f:
        for line in f:
            if not line.startswith("#"):
                key, *v = line.split()
                vals[key] = [float(t) for t in v]
    return vals


def test_adjoint_configured_problem_against_stored_oracle(adelib, orc, torch_cuda):
    """The inversion problem at its configured size: 512^2 lattice, 400 steps, checkpoints every
    40, target from the oracle at theta* = (2e-2, 2e-3, 1e-6).  J within 1e-5 and each component of
    dJ/d(alpha_L, alpha_T, D_m) within 1e-4 of the FP64 oracle's tangent-linear gradient and of its
    FP64 central differences (eps = 1e-4 theta_k), stored by tests/golden/make_adjoint_golden.py;
    the target is recomputed here by the same function of that script."""
    spec = importlib.util.spec_from_file_location("make_adjoint_golden",
                                                  os.path.join(HERE, "golden", "make_adjoint_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    gold = _adjoint_golden()
    p, x, C, kw, target = mk.problem()
    assert kw["dt"] == pytest.approx(gold["dt"][0], rel=1e-14)
    sim = adelib.Simulation(adelib.params_for(p, dt=gold["dt"][0]), *p.initial_state())
    J, g, _, _ = sim.adjoint(target.astype(np.float32), mk.NSTEPS, 40, want_dC0=False)
    rel = lambda a, b: abs(a - b) / abs(b)
    print(f"\n512^2 x 400: J rel err {rel(J, gold['J'][0]):.2e}; dJ/dtheta rel err vs TLM "
          + ", ".join(f"{rel(g[k], gold['grad_tlm'][k]):.2e}" for k in range(3)) + "; vs FD "
          + ", ".join(f"{rel(g[k], gold['grad_fd'][k]):.2e}" for k in range(3)))
    assert J == pytest.approx(gold["J"][0], rel=1e-5)
    for k in range(3):
        assert g[k] == pytest.approx(gold["grad_tlm"][k], rel=GRAD_TOL)
        assert g[k] == pytest.approx(gold["grad_fd"][k], rel=GRAD_TOL)


def test_adjoint_dot_product_identity_full_size(adelib, torch_cuda):
    """512^2, 400 steps, checkpoints every 40: with C* = 0, dJ/dC0 = (S^N)^T S^N C0, so
    <dJ/dC0(delta), w> = <S^N delta, S^N w> for any w."""
    torch = torch_cuda
    p = inputs.Plume(dim=2, side=512, h_over_dx=1.3, alpha_L=THETA[0], alpha_T=THETA[1], D_m=THETA[2])
    xq, C = p.initial_state()
    rng = np.random.default_rng(5)
    delta = C + 0.1 * rng.normal(size=p.n).astype(np.float32)
    w = rng.normal(size=p.n).astype(np.float32)
    zero = np.zeros(p.n, np.float32)
    s1 = adelib.Simulation(adelib.params_for(p), xq, delta)
    _, _, g, Nd = s1.adjoint(zero, 400, 40, want_final=True)
    s2 = adelib.Simulation(adelib.params_for(p), xq, w)
    _, _, _, Nw = s2.adjoint(zero, 400, 40, want_final=True)
    lhs = float(np.dot(g.cpu().numpy().astype(np.float64), w.astype(np.float64)))
    rhs = float(np.dot(Nd.cpu().numpy().astype(np.float64), Nw.cpu().numpy().astype(np.float64)))
    assert lhs == pytest.approx(rhs, rel=GRAD_TOL)


def test_autograd_function(adelib, orc, torch_cuda):
    torch = torch_cuda
    from paper_2108_09488_gb300.autograd import misfit
    p, sim, x, C, target, kw = _problem(adelib, orc, 32, 10)
    C0 = torch.tensor(C, device="cuda", requires_grad=True)
    theta = torch.tensor(THETA, dtype=torch.float64, requires_grad=True)
    tgt = torch.tensor(target, dtype=torch.float32, device="cuda")
    J = misfit(sim, C0, theta, tgt, 10, 4)
    J.backward()
    J2, g2, d2, _ = sim.adjoint(target.astype(np.float32), 10, 4)
    assert float(J.detach()) == J2
    assert np.array_equal(theta.grad.numpy(), g2)
    assert torch.equal(C0.grad, d2)
    # a few gradient steps on alpha_L lower the misfit
    th = THETA.copy()
    Js = []
    for _ in range(3):
        sim.set_dispersivity(*th)
        Jk, gk, _, _ = sim.adjoint(target.astype(np.float32), 10, 4, want_dC0=False)
        Js.append(Jk)
        th[0] -= 0.5 * Jk / gk[0] if gk[0] != 0 else 0.0
    assert Js[-1] < Js[0]
