"""Pins for the oracle's SPH rate (Eq. 4-5), update (Eq. 8-9) and closed form (Eq. 12-13).

What fixes each result independently of the oracle:
  * constant fields, pair antisymmetry, conservation of sum m C, translation invariance: exact
    properties of the symmetric pair form;
  * isotropic D = d I: the textbook Brookshaw Laplacian 2 d sum V (C_a - C_b) W'(r)/r;
  * a Fourier mode on a lattice is an eigenvector, and as h -> 0 its eigenvalue tends to
    4 pi^2 k^T D k, the eigenvalue of the continuous operator div(D grad) (this fixes Gamma, the
    factor 4 of the harmonic mean, the 1/2, the kernel normalisation and the sign of D_xy);
  * a linear velocity field: the convective term equals -C div v (Eq. 1);
  * Eq. 8-9 read as the midpoint rule: a mode's amplitude is multiplied by 1 - dt L + dt^2 L^2/2;
  * the closed form against scipy's multivariate normal, its t = 0 limit (Eq. 11), its mass and
    the advection-dispersion PDE by finite differences.
"""
import math

import numpy as np
import pytest
from scipy import stats as sps

from paper_2108_09488_gb300 import inputs


def _lattice_setup(dim, side, H_dx):
    x = inputs.lattice_positions(dim, side)
    box = np.ones(dim)
    dx = 1.0 / side
    return x, box, H_dx * dx, dx ** dim


def test_constant_field_rate_is_zero(orc):
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(600, 2))
    C = np.full(600, 0.731)
    r, pairs = orc.rate(x, [0.07, -0.02], C, 1.0 / 600, 1.0, np.ones(2), 0, 0.12, 4.0, 0.01, 0.001, 1e-6)
    assert pairs > 0
    assert np.all(r == 0.0)


def test_pair_antisymmetry_and_even_tensor(orc):
    """P(a,b) = -P(b,a) bit for bit, and Dcal_ab is even in x_ab."""
    rng = np.random.default_rng(11)
    for dim in (2, 3):
        for _ in range(20):
            xab = rng.normal(size=dim) * 0.05
            va, vb = rng.normal(size=dim), rng.normal(size=dim)
            Da = orc.dispersion_tensor(va, 0.03, 0.004, 1e-5)
            Db = orc.dispersion_tensor(vb, 0.03, 0.004, 1e-5)
            Ca, Cb = rng.uniform(size=2)
            H = 0.2
            g = dim + 2.0
            ab, _ = orc.pair_term(xab, Da, Db, Ca, Cb, va, vb, 1e-3, 1.0, 1.0, 0, H, g)
            ba, _ = orc.pair_term(-xab, Db, Da, Cb, Ca, vb, va, 1e-3, 1.0, 1.0, 0, H, g)
            assert ab == -ba
            # even in x_ab (same C difference, same tensors)
            ab2, _ = orc.pair_term(-xab, Da, Db, Ca, Cb, va, vb, 1e-3, 1.0, 1.0, 0, H, g)
            assert ab2 == ab


def test_isotropic_reduces_to_brookshaw(orc):
    """aL = aT: D = d I, Dcal = 2d (Gamma - m) = 4d, and Eq. 4 is the Brookshaw Laplacian."""
    rng = np.random.default_rng(5)
    for dim, n, H in ((2, 900, 0.1), (3, 1500, 0.22)):
        x = rng.uniform(size=(n, dim))
        box = np.ones(dim)
        C = rng.uniform(size=n)
        v = np.zeros(dim)
        v[0] = 0.3
        aL = aT = 0.02
        Dm = 1e-4
        d = aT * 0.3 + Dm
        V = 1.0 / n
        r, _ = orc.rate(x, v, C, V, 1.0, box, 0, H, dim + 2.0, aL, aT, Dm)
        ptr, idx = orc.neighbours(x, box, H)
        ref = np.zeros(n)
        for a in range(n):
            b = idx[ptr[a]:ptr[a + 1]]
            dd = x[a] - x[b]
            dd -= np.rint(dd)
            rr = np.sqrt((dd * dd).sum(1))
            ref[a] = 2.0 * d * np.sum(V * (C[a] - C[b]) * orc.kernel_dwdr(0, dim, H, rr) / rr)
        assert np.max(np.abs(r - ref)) <= 1e-12 * np.max(np.abs(ref))


def _mode_rate(orc, dim, side, H_dx, k, v, aL, aT, Dm, kind=0):
    x, box, H, V = _lattice_setup(dim, side, H_dx)
    C = np.cos(2 * math.pi * (x @ np.asarray(k, dtype=float)))
    r, _ = orc.rate(x, v, C, V, 1.0, box, kind, H, dim + 2.0, aL, aT, Dm)
    return x, C, r


@pytest.mark.parametrize("k", [(1, 0), (1, 1), (1, -1), (2, 1)])
def test_fourier_mode_eigenvalue_2d(orc, k):
    """r = -lam C exactly on the lattice, and lam -> 4 pi^2 k^T D k as the neighbour count grows
    (Eq. 6: part of the error falls only with n, not with h)."""
    v = np.array([0.1, 0.1]) / math.sqrt(2)
    aL, aT, Dm = 1e-2, 1e-3, 1e-6
    D = orc.dispersion_tensor(v, aL, aT, Dm)
    exact = 4 * math.pi ** 2 * (np.asarray(k) @ D @ np.asarray(k))
    errs = []
    for H_dx in (3.005, 4.245, 6.085):                     # 28, 60, 120 neighbours
        x, C, r = _mode_rate(orc, 2, 192, H_dx, k, v, aL, aT, Dm)
        big = np.abs(C) > 0.5
        lam = -r[big] / C[big]
        assert np.ptp(lam) <= 1e-9 * abs(lam.mean())          # eigenvector on the lattice
        errs.append(abs(lam.mean() - exact) / exact)
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.05


def test_fourier_mode_h_convergence(orc):
    """At fixed neighbour count the error of the axis mode falls as the lattice is refined."""
    v = np.array([0.1, 0.1]) / math.sqrt(2)
    aL, aT, Dm = 1e-2, 1e-3, 1e-6
    D = orc.dispersion_tensor(v, aL, aT, Dm)
    k = (1, 0)
    exact = 4 * math.pi ** 2 * D[0, 0]
    errs = []
    for side in (64, 128, 256):
        x, C, r = _mode_rate(orc, 2, side, 6.085, k, v, aL, aT, Dm)
        i = np.argmax(C)
        errs.append(abs(-r[i] / C[i] - exact) / exact)
    assert errs[0] > 2.5 * errs[1] > 2.5 * 2.5 * errs[2]
    assert errs[2] < 1e-3


def test_fourier_mode_eigenvalue_3d(orc):
    """3D (Gamma = 5): lattice eigenvector; the axis-mode error falls with h, the transverse-mode
    error falls with the neighbour count."""
    v = np.full(3, 0.1 / math.sqrt(3))
    aL, aT, Dm = 1e-2, 1e-3, 1e-6
    D = orc.dispersion_tensor(v, aL, aT, Dm)

    def err(k, side, H_dx):
        exact = 4 * math.pi ** 2 * (np.asarray(k) @ D @ np.asarray(k))
        x, C, r = _mode_rate(orc, 3, side, H_dx, k, v, aL, aT, Dm)
        big = np.abs(C) > 0.5
        lam = -r[big] / C[big]
        assert np.ptp(lam) <= 1e-9 * abs(lam.mean())
        return abs(lam.mean() - exact) / exact

    e24, e32 = err((1, 0, 0), 24, 4.0), err((1, 0, 0), 32, 4.0)
    assert e32 < e24 / 1.6 and e32 < 1.2e-2
    t = [err((1, -1, 0), 32, H_dx) for H_dx in (3.0, 4.0, 5.0)]
    assert t[2] < t[1] < t[0] and t[2] < 0.035


def test_wendland_c4_fourier_mode(orc):
    """The paper's kernel (Eq. 7, support h) gives the same continuum operator."""
    v = np.array([0.1, 0.0])
    aL, aT, Dm = 1e-2, 1e-3, 0.0
    D = orc.dispersion_tensor(v, aL, aT, Dm)
    k = (1, 1)
    exact = 4 * math.pi ** 2 * (np.asarray(k) @ D @ np.asarray(k))
    x, C, r = _mode_rate(orc, 2, 128, 6.085, k, v, aL, aT, Dm, kind=1)
    i = np.argmax(C)
    assert -r[i] / C[i] == pytest.approx(exact, rel=5e-3)


def test_conservation_translation_and_sign(orc):
    """sum m r = 0 to round-off; a uniform shift leaves r unchanged; r < 0 at the plume peak."""
    p = inputs.ladder_2d(256, 10)
    p = inputs.Plume(**{**p.__dict__, "side": 96})
    xq, C = p.initial_state()
    x = inputs.from_fixed(xq, p.boxv)
    C = C.astype(np.float64)
    args = (p.velocity, C, p.mass, 1.0, p.boxv, 0, p.support, 4.0, p.alpha_L, p.alpha_T, p.D_m)
    r, rd, rc, _ = orc.rate(x, *args, split=True)
    assert np.all(rc == 0.0)                                 # uniform v: convective term vanishes
    assert abs(np.sum(p.mass * r)) <= 1e-13 * np.sum(p.mass * np.abs(r))
    assert r[np.argmax(C)] < 0.0
    xs = np.mod(x + np.array([0.123456, -0.0421]), 1.0)
    r2, _ = orc.rate(xs, *args)
    assert np.max(np.abs(r2 - r)) <= 1e-9 * np.max(np.abs(r))


def test_convective_term_is_minus_c_div_v(orc):
    """Eq. 1 convective term -C div v: with v = (a x, b y) the SPH sum gives -C (a + b) away from
    the periodic seam (the velocity field jumps there)."""
    side = 64
    x, box, H, V = _lattice_setup(2, side, 4.245)
    a, b = 0.3, -0.1
    v = np.stack([a * x[:, 0], b * x[:, 1]], 1)
    C = 1.0 + 0.5 * np.sin(2 * math.pi * x[:, 0])
    _, _, rc, _ = orc.rate(x, v, C, V, 1.0, box, 0, H, 4.0, 0.0, 0.0, 0.0, split=True)
    inner = np.all((x > 2 * H) & (x < 1 - 2 * H), axis=1)
    assert np.max(np.abs(rc[inner] + C[inner] * (a + b))) < 1e-3 * np.max(np.abs(C * (a + b)))


def test_midpoint_update_amplification(orc):
    """Eq. 8-9 as the midpoint rule: after s steps a lattice mode is scaled by
    (1 - dt lam + dt^2 lam^2 / 2)^s, with lam measured from one rate evaluation; forward Euler's
    (1 - dt lam)^s is rejected.  dt is a stable step (dt * lam_max < 2 for every lattice mode)."""
    v = np.array([0.1, 0.1]) / math.sqrt(2)
    aL, aT, Dm = 1e-2, 1e-3, 1e-6
    side, H_dx = 48, 3.005
    x, box, H, V = _lattice_setup(2, side, H_dx)
    k = np.array([3, 2])
    C = np.cos(2 * math.pi * (x @ k))
    r, _ = orc.rate(x, v, C, V, 1.0, box, 0, H, 4.0, aL, aT, Dm)
    i = np.argmax(C)
    lam = -r[i] / C[i]
    D = orc.dispersion_tensor(v, aL, aT, Dm)
    dt = orc.dt_rule(D, H / 2.0) * 3.0
    s = 20
    x1, C1, pairs = orc.step(x, v, C, V, 1.0, box, 0, H, 4.0, aL, aT, Dm, dt, nsteps=s)
    g = (1 - dt * lam + 0.5 * (dt * lam) ** 2) ** s
    # particles carry the mode with the flow, so each particle's value is scaled by g
    assert np.max(np.abs(C1 - g * C)) < 1e-12
    assert abs((1 - dt * lam) ** s - g) > 1e-6
    assert np.max(np.abs(np.mod(x1 - x - v * s * dt + 0.5, 1.0) - 0.5)) < 1e-13
    assert pairs == 2 * s * side * side * 28


def test_closed_form_matches_multivariate_normal(orc):
    """Eq. 12-13 (2D, with the 2 w^4 denominator) and the 3D form against scipy's Gaussian pdf:
    C/C0 = (2 pi)^(d/2) w^d N(x; x0 + v t, w^2 I + 2 t D)."""
    rng = np.random.default_rng(2)
    for dim in (2, 3):
        box = np.full(dim, 50.0)                            # no image contributes
        x0 = np.full(dim, 20.0)
        v = rng.normal(size=dim) * 0.3
        D = orc.dispersion_tensor(v, 0.4, 0.05, 0.01)
        w = 0.8
        for t in (0.0, 0.7, 3.0):
            x = x0 + v * t + rng.normal(size=(50, dim)) * 1.5
            C = orc.closed_form(x, box, x0, v, D, w, 2.0, t, nimg=0)
            S = w * w * np.eye(dim) + 2 * t * D
            ref = 2.0 * (2 * math.pi) ** (dim / 2) * w ** dim * sps.multivariate_normal(x0 + v * t, S).pdf(x)
            assert np.max(np.abs(C - ref)) <= 1e-12 * ref.max()


def test_closed_form_initial_condition_and_mass(orc):
    """t = 0 gives Eq. 11; sum over a fine lattice of C dA stays 2 pi w^2 C0 for t > 0."""
    p = inputs.lattice_2d_64()
    x = p.positions()
    D = orc.dispersion_tensor(p.velocity, p.alpha_L, p.alpha_T, p.D_m)
    C_t0 = orc.closed_form(x, p.boxv, p.x0[:2], p.velocity, D, p.w, 1.0, 0.0)
    assert np.max(np.abs(C_t0 - inputs.gaussian_plume(x, p.boxv, p.x0[:2], p.w))) < 1e-13
    xf = inputs.lattice_positions(2, 400)
    for t in (1.0, 8.244):
        Cf = orc.closed_form(xf, p.boxv, p.x0[:2], p.velocity, D, p.w, 1.0, t, nimg=3)
        assert np.sum(Cf) / 400 ** 2 == pytest.approx(2 * math.pi * p.w ** 2, rel=1e-9)


def test_closed_form_solves_the_ade(orc):
    """dC/dt = div(D grad C) - v . grad C (Eulerian form of Eq. 1-2) by central differences."""
    box = np.array([10.0, 10.0])
    x0 = np.array([4.0, 5.0])
    v = np.array([0.3, -0.2])
    D = orc.dispersion_tensor(v, 0.5, 0.07, 0.02)
    w, t = 0.6, 1.3
    pts = np.array([[4.5, 4.9], [3.8, 5.6], [4.1, 4.2]])
    e = 1e-3
    f = lambda X, T: orc.closed_form(X, box, x0, v, D, w, 1.0, T, nimg=1)
    dCdt = (f(pts, t + e) - f(pts, t - e)) / (2 * e)
    g = np.zeros((3, 2))
    hess = np.zeros((3, 2, 2))
    for i in range(2):
        ei = np.eye(2)[i] * e
        g[:, i] = (f(pts + ei, t) - f(pts - ei, t)) / (2 * e)
        for j in range(2):
            ej = np.eye(2)[j] * e
            hess[:, i, j] = (f(pts + ei + ej, t) - f(pts + ei - ej, t) - f(pts - ei + ej, t)
                             + f(pts - ei - ej, t)) / (4 * e * e)
    rhs = np.einsum("ij,pij->p", D, hess) - g @ v
    assert np.max(np.abs(dCdt - rhs)) < 1e-5 * np.max(np.abs(dCdt))


def test_run_converges_to_closed_form(orc):
    """Runs to t = 0.3 on the 45-degree plume approach the closed form in the joint limit of
    Sec. 2.3 (h -> 0 with the neighbour count n growing); at fixed n = 20 the error stalls, which
    is the fixed-n term of Eq. 6."""
    def run(side, h_dx):
        p = inputs.Plume(dim=2, side=side, h_over_dx=h_dx)
        xq, C = p.initial_state()
        x = inputs.from_fixed(xq, p.boxv)
        D = orc.dispersion_tensor(p.velocity, p.alpha_L, p.alpha_T, p.D_m)
        T = 0.3
        ns = int(np.ceil(T / orc.dt_rule(D, 1.3 / 192)))
        x1, C1, _ = orc.step(x, p.velocity, C.astype(np.float64), p.mass, 1.0, p.boxv, 0,
                             p.support, 4.0, p.alpha_L, p.alpha_T, p.D_m, T / ns, nsteps=ns)
        Ca = orc.closed_form(x1, p.boxv, p.x0[:2], p.velocity, D, p.w, 1.0, T)
        return np.max(np.abs(C1 - Ca))

    joint = [run(48, 1.3), run(96, 2.1225), run(192, 3.0425)]
    assert joint[0] > 1.5 * joint[1] > 1.5 * 1.5 * joint[2]
    assert joint[2] < 3e-3
    fixed_n = run(96, 1.3)
    assert fixed_n > 1.5 * joint[1]
