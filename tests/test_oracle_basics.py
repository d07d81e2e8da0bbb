"""Pins for the oracle's building blocks: kernels, dispersion tensor, time step, scaling relations,
neighbour search and the fixed-point cell list.  Every check compares the oracle with something
other than itself: quadrature, finite differences, an eigen-decomposition, the paper's Table 1,
brute force or a numpy library routine."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from paper_2108_09488_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_normalised(orc, kind, dim):
    """Both Wendland kernels integrate to 1 over their support (2D: 2 pi r dr, 3D: 4 pi r^2 dr)."""
    H = 0.37
    f = (lambda r: 2 * math.pi * r * orc.kernel_w(kind, dim, H, r)[0]) if dim == 2 else \
        (lambda r: 4 * math.pi * r * r * orc.kernel_w(kind, dim, H, r)[0])
    val, _ = integrate.quad(f, 0.0, H, epsabs=1e-13, epsrel=1e-12)
    assert abs(val - 1.0) < 1e-10


def test_kernel_c4_matches_eq7(orc):
    """Eq. 7 as printed (2D): W = 9/(pi h^2) (1-q)^6 (1 + 6q + 35 q^2 / 3), q = r/h, support h."""
    h = 0.8
    for q in (0.0, 0.1, 0.5, 0.93):
        ref = 9.0 / (math.pi * h * h) * (1 - q) ** 6 * (1 + 6 * q + 35.0 * q * q / 3.0)
        assert orc.kernel_w(1, 2, h, q * h)[0] == pytest.approx(ref, rel=1e-14)
    assert orc.kernel_w(1, 2, h, h)[0] == 0.0
    assert orc.kernel_w(1, 2, h, 1.2 * h)[0] == 0.0


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_derivative_finite_difference(orc, kind, dim):
    """dW/dr against a central difference of W; both vanish at the support radius."""
    H = 1.3
    eps = 1e-6
    for r in np.linspace(0.02, 0.98, 13) * H:
        fd = (orc.kernel_w(kind, dim, H, r + eps)[0] - orc.kernel_w(kind, dim, H, r - eps)[0]) / (2 * eps)
        an = orc.kernel_dwdr(kind, dim, H, r)[0]
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9)
        assert an < 0.0
    assert orc.kernel_dwdr(kind, dim, H, H)[0] == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_dispersion_tensor_eigenstructure(orc, dim):
    """Eq. 3: v is an eigenvector with eigenvalue aL|v| + Dm; every direction normal to v has
    eigenvalue aT|v| + Dm; D is symmetric."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        v = rng.normal(size=dim)
        aL, aT, Dm = 0.7, 0.05, 1e-3
        D = orc.dispersion_tensor(v, aL, aT, Dm)
        assert np.array_equal(D, D.T)
        s = np.linalg.norm(v)
        assert D @ v == pytest.approx((aL * s + Dm) * v, rel=1e-13)
        ev = np.sort(np.linalg.eigvalsh(D))
        expect = np.sort([aL * s + Dm] + [aT * s + Dm] * (dim - 1))
        assert ev == pytest.approx(expect, rel=1e-12)


def test_dispersion_tensor_zero_velocity(orc):
    D = orc.dispersion_tensor([0.0, 0.0], 0.5, 0.1, 2e-3)
    assert np.array_equal(D, 2e-3 * np.eye(2))


def test_time_step_rules(orc):
    """64^2 lattice workload: dt = 0.1 h^2 / (aL |v| + Dm) with h = 1.3/64, |v| = 0.1, and
    Eq. 10 (trace form) = 0.1 h^2 / ((aL + aT)|v| + 2 Dm)."""
    p = inputs.lattice_2d_64()
    D = orc.dispersion_tensor(p.velocity, p.alpha_L, p.alpha_T, p.D_m)
    h = 1.3 / 64
    assert orc.dt_rule(D, h) == pytest.approx(0.1 * h * h / (1e-2 * 0.1 + 1e-6), rel=1e-12)
    assert orc.dt_rule(D, h) == pytest.approx(0.04122, abs=5e-6)
    assert orc.dt_rule(D, h, "trace") == pytest.approx(0.1 * h * h / (1.1e-2 * 0.1 + 2e-6), rel=1e-12)


def test_scaling_relations_reproduce_table1(orc):
    """Sec. 2.3 scaling relations against Table 1 (golden/table1.txt)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1.txt"))
    for N, n, dx, h, _ in rows:
        n_s, h_s = orc.scaling_relations(N)
        assert abs(n_s - n) <= 1.0                  # printed neighbour counts are rounded
        assert abs(h_s - h) <= 0.0015               # printed h/L has two significant digits
        assert abs(1.0 / math.sqrt(N) - dx) <= 0.02 * dx


# ---------------------------------------------------------------------------------------------
# Neighbour search
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,box", [(2, (1.0, 1.0)), (2, (1.0, 0.6)), (3, (1.0, 0.8, 1.0))])
def test_cell_list_equals_brute_force(orc, dim, box):
    rng = np.random.default_rng(7)
    n = 700 if dim == 2 else 900
    box = np.array(box)
    x = rng.uniform(size=(n, dim)) * box
    H = 0.11 if dim == 2 else 0.19
    p1, i1 = orc.neighbours(x, box, H, brute=True)
    p2, i2 = orc.neighbours(x, box, H, brute=False)
    assert np.array_equal(p1, p2) and np.array_equal(i1, i2)
    # independent minimum-image check of a few lists
    for a in (0, 17, n - 1):
        d = x - x[a]
        d -= box * np.rint(d / box)
        r = np.sqrt((d * d).sum(1))
        want = np.nonzero((r > 0) & (r < H))[0]
        assert np.array_equal(np.sort(i1[p1[a]:p1[a + 1]]), want)


def _lattice_count(dim, R):
    """Number of nonzero integer offsets with |o| < R (brute enumeration)."""
    m = int(math.ceil(R))
    rng = np.arange(-m, m + 1)
    g = np.stack(np.meshgrid(*([rng] * dim), indexing="ij"), -1).reshape(-1, dim)
    r2 = (g * g).sum(1)
    return int(np.sum((r2 > 0) & (r2 < R * R)))


@pytest.mark.parametrize("dim,side,H_dx,expect", [
    (2, 64, 2.6, 20), (2, 48, 3.005, 28), (2, 48, 4.245, 60), (2, 48, 6.085, 120),
    (3, 32, 4.0, 250)])
def test_lattice_neighbour_counts(orc, dim, side, H_dx, expect):
    """Neighbour counts of the lattice workloads (20; 28/60/120; 3D with h = 2dx)."""
    x = inputs.lattice_positions(dim, side)
    box = np.ones(dim)
    ptr, _ = orc.neighbours(x, box, H_dx / side)
    cnt = np.diff(ptr)
    want = _lattice_count(dim, H_dx) if expect is None else expect
    assert _lattice_count(dim, H_dx) == want
    assert cnt.min() == want and cnt.max() == want


def test_fixed_point_cell_sort_matches_lexsort(orc):
    """Stable counting sort of fixed-point cell keys against numpy lexsort / searchsorted."""
    rng = np.random.default_rng(3)
    for dim, nc in ((2, (37, 23, 1)), (3, (9, 11, 7))):
        n = 5000
        xq = rng.integers(0, 2 ** 32, size=(dim, n), dtype=np.uint64).astype(np.uint32)
        key = orc.cell_keys(xq, np.array(nc))
        c = [((xq[i].astype(np.uint64) * np.uint64(nc[i])) >> np.uint64(32)).astype(np.int64)
             for i in range(dim)]
        ref = c[0] + nc[0] * (c[1] + (nc[1] * c[2] if dim == 3 else 0))
        assert np.array_equal(key.astype(np.int64), ref)
        ncells = int(np.prod(nc[:dim]))
        perm, start = orc.sort_cells(key, ncells)
        assert np.array_equal(perm, np.lexsort((np.arange(n), key)).astype(np.uint32))
        assert np.array_equal(start, np.searchsorted(np.sort(key), np.arange(ncells + 1), "left"))


def test_fixed_point_roundtrip():
    x = inputs.lattice_positions(2, 64)
    xq = inputs.to_fixed(x, np.ones(2))
    assert np.array_equal(inputs.from_fixed(xq, np.ones(2)), x)
    # minimum image: difference words as int32
    d = (xq[0, 1].astype(np.int64) - xq[0, 0].astype(np.int64))
    assert d == 2 ** 32 // 64


def test_stats_hand_computed(orc):
    """Sec. 4 metrics on three particles worked by hand: C = (1, -0.5, 2), m = 0.25, reference
    (1, 0, 1), C0 = 2.  Mass 0.25 * 2.5 = 0.625; min -0.5; max 2; errors (0, -0.5, 1):
    L2 = sqrt(0.25 * 1.25) = sqrt(0.3125), Linf = 1, RMSE of e / C0 = sqrt((0.0625 + 0.25) / 3)."""
    out = orc.stats([1.0, -0.5, 2.0], 0.25, C_ref=[1.0, 0.0, 1.0], C0=2.0)
    assert out["mass"] == 0.625
    assert out["c_min"] == -0.5 and out["c_max"] == 2.0
    assert out["l2"] == pytest.approx(0.5590169943749474, rel=1e-15)
    assert out["linf"] == 1.0
    assert out["rmse"] == pytest.approx(0.3227486121839514, rel=1e-15)
    # an explicit volume per particle replaces m in L2
    assert orc.stats([3.0], 1.0, C_ref=[1.0], vol=4.0)["l2"] == 4.0
