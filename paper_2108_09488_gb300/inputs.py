"""Seeded synthetic inputs shared by the GPU path, the oracle and the benchmark.

This module holds no arithmetic of the SPH method (no kernel, no dispersion tensor, no rate, no
update).  It only produces the workload: particle positions in the fixed-point format that the
library consumes, the initial concentration field of the test model (Sec. 3, Eq. 11) and the
parameter sets of the workloads, all from a seed.

Fixed-point positions: a coordinate u in [0, L) is stored as ``round(u / L * 2**32) mod 2**32``
(uint32).  Differences of two such words, read as int32, are the minimum-image separation in
units of L / 2**32, and a uniform translation adds the same word to every particle.

Workload recipes (all in a periodic unit square or cube, rho = 1, m = rho * dx**dim):
  * ``lattice_2d_64``: 64 x 64 lattice, h = 1.3 dx, Wendland C2 (support 2h), v = 0.1 (1,1)/sqrt2,
    alpha_L = 1e-2, alpha_T = 1e-3, D_m = 1e-6, Gaussian sigma0 = 0.05 at (0.3, 0.3), 200 steps.
  * ``ladder_2d``: the same plume on 256^2 / 512^2 / 1024^2 lattices with support radius
    H = 3.005 / 4.245 / 6.085 dx (28 / 60 / 120 neighbours), alpha_T = 1e-3,
    alpha_L / alpha_T in {1, 10, 100}, flow at 45 degrees, 1000 steps.
  * ``cube_3d_128``: 128^3 lattice, h = 2 dx, v = 0.1 (1,1,1)/sqrt3, 500 steps.
  * ``batched_2d``: 64 plumes, side s = round(exp U(ln 32, ln 512)), h/dx ~ U[1.2, 2.5],
    alpha_L/alpha_T log-uniform in [1, 100] with alpha_T = 1e-3, angle ~ U[0, 2 pi), |v| = 0.1,
    D_m = 1e-6, sigma0 = 0.05 at (0.3, 0.3); numpy PCG64 seed 20210821.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WENDLAND_C2 = 0
WENDLAND_C4 = 1

_TWO32 = 2.0 ** 32


def to_fixed(x, box):
    """FP64 positions [n][dim] -> uint32 fixed point [dim][n]."""
    x = np.asarray(x, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    dim = x.shape[1]
    u = x / box[None, :dim]
    u = u - np.floor(u)
    q = np.rint(u * _TWO32).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    return np.ascontiguousarray(q.T.astype(np.uint32))


def from_fixed(xq, box):
    """uint32 fixed point [dim][n] -> FP64 positions [n][dim] (exact)."""
    xq = np.asarray(xq, dtype=np.uint32)
    box = np.asarray(box, dtype=np.float64)
    dim = xq.shape[0]
    return np.ascontiguousarray((xq.astype(np.float64) * (box[:dim, None] / _TWO32)).T)


def lattice_positions(dim, side, box=1.0, jitter=0.0, seed=0):
    """Cell-centred lattice in [0, box)^dim, particle index with x fastest.

    With ``jitter > 0`` every coordinate is displaced by U(-jitter, jitter) * dx (seeded), which
    gives an irregular particle set of the same density."""
    dx = box / side
    idx = np.arange(side ** dim, dtype=np.int64)
    # index = ((k * side) + j) * side + i, x fastest
    cell = np.stack([(idx // side ** d) % side for d in range(dim)], axis=1)
    x = (cell.astype(np.float64) + 0.5) * dx
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        x = x + rng.uniform(-jitter, jitter, size=x.shape) * dx
        x = np.mod(x, box)
    return x


def gaussian_plume(x, box, x0, w, C0=1.0):
    """Initial condition of the test model (Sec. 3, Eq. 11): C0 exp(-|x - x0|^2 / (2 w^2)),
    with |x - x0| the minimum-image distance in the periodic box."""
    x = np.asarray(x, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    dim = x.shape[1]
    d = x - np.asarray(x0, dtype=np.float64)[None, :dim]
    d = d - box[None, :dim] * np.rint(d / box[None, :dim])
    return C0 * np.exp(-np.sum(d * d, axis=1) / (2.0 * w * w))


@dataclasses.dataclass
class Plume:
    """One plume: geometry, kernel, transport parameters and run length."""
    dim: int
    side: int
    h_over_dx: float
    kernel: int = WENDLAND_C2
    alpha_L: float = 1e-2
    alpha_T: float = 1e-3
    D_m: float = 1e-6
    speed: float = 0.1
    angle: float = math.pi / 4.0          # 2D flow angle from the x axis
    x0: tuple = (0.3, 0.3, 0.3)
    w: float = 0.05
    C0: float = 1.0
    rho: float = 1.0
    steps: int = 200
    box: float = 1.0
    jitter: float = 0.0
    seed: int = 0
    name: str = ""
    dt: float = 0.0                       # 0: the library's time-step rule

    @property
    def n(self):
        return self.side ** self.dim

    @property
    def dx(self):
        return self.box / self.side

    @property
    def h(self):
        return self.h_over_dx * self.dx

    @property
    def support(self):
        return 2.0 * self.h if self.kernel == WENDLAND_C2 else self.h

    @property
    def mass(self):
        return self.rho * self.dx ** self.dim

    @property
    def velocity(self):
        if self.dim == 2:
            return np.array([self.speed * math.cos(self.angle), self.speed * math.sin(self.angle)])
        return np.full(3, self.speed / math.sqrt(3.0))

    @property
    def boxv(self):
        return np.full(self.dim, self.box)

    def positions(self):
        return lattice_positions(self.dim, self.side, self.box, self.jitter, self.seed)

    def fixed_positions(self):
        return to_fixed(self.positions(), self.boxv)

    def initial_state(self):
        """(xq uint32 [dim][n], C float32 [n]): fixed-point lattice and the Eq. 11 plume,
        evaluated at the positions the fixed-point words represent."""
        xq = self.fixed_positions()
        x = from_fixed(xq, self.boxv)
        C = gaussian_plume(x, self.boxv, np.asarray(self.x0[: self.dim]), self.w, self.C0)
        return xq, C.astype(np.float32)


def lattice_2d_64():
    return Plume(dim=2, side=64, h_over_dx=1.3, steps=200, name="2d-64x64-h1.3dx-C2")


LADDER_SUPPORT_OVER_DX = {256: 3.005, 512: 4.245, 1024: 6.085}
LADDER_NEIGHBOURS = {256: 28, 512: 60, 1024: 120}


def ladder_2d(side, ratio, steps=1000):
    """One rung of the 2D convergence ladder (support radius chosen for 28/60/120 neighbours)."""
    H_dx = LADDER_SUPPORT_OVER_DX[side]
    return Plume(dim=2, side=side, h_over_dx=H_dx / 2.0, alpha_T=1e-3, alpha_L=1e-3 * ratio,
                 steps=steps, name=f"2d-ladder-{side}^2-n{LADDER_NEIGHBOURS[side]}-ratio{ratio}")


def cube_3d_128(side=128, steps=500):
    return Plume(dim=3, side=side, h_over_dx=2.0, alpha_L=1e-2, alpha_T=1e-3, steps=steps,
                 name=f"3d-{side}^3-h2dx-C2")


def batched_2d(nplumes=64, seed=20210821, steps=500, side_lo=32, side_hi=512):
    """Uneven batch of independent 2D plumes (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for p in range(nplumes):
        side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        h_dx = float(rng.uniform(1.2, 2.5))
        ratio = float(math.exp(rng.uniform(0.0, math.log(100.0))))
        angle = float(rng.uniform(0.0, 2.0 * math.pi))
        out.append(Plume(dim=2, side=side, h_over_dx=h_dx, alpha_T=1e-3, alpha_L=1e-3 * ratio,
                         angle=angle, steps=steps, name=f"batch{p}-{side}^2"))
    return out


def velocity_field(x, box, speed=0.1, amplitude=0.5, modes=3, seed=2108):
    """Seeded smooth, periodic, non-uniform velocity field at positions x [n][dim] (float32
    [dim][n], axis-major like the positions): a uniform drift of the given speed along the
    diagonal plus `modes` random Fourier modes per component with relative amplitude `amplitude`
    (it has a nonzero divergence, so the convective term of Eq. 4 is exercised)."""
    x = np.asarray(x, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    n, dim = x.shape
    rng = np.random.Generator(np.random.PCG64(seed))
    u = x / box[None, :dim]
    v = np.zeros((dim, n))
    base = speed / math.sqrt(dim)
    for d in range(dim):
        v[d] = base
        for _ in range(modes):
            k = rng.integers(-2, 3, size=dim)
            if not np.any(k):
                k[d] = 1
            a = rng.uniform(-1.0, 1.0) * amplitude * base
            ph = rng.uniform(0.0, 2.0 * math.pi)
            v[d] += a * np.sin(2.0 * math.pi * (u @ k) + ph)
    return np.ascontiguousarray(v.astype(np.float32))


def velocity_noise(n, dim, vmax, seed=7):
    """Seeded white-noise velocity field (float32 [dim][n]): independent directions, speeds
    uniform in [0, vmax).  Neighbours move apart at up to 2 vmax, the case the cell-grid skin of
    velocity-field mode has to cover."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((dim, n))
    d /= np.maximum(np.linalg.norm(d, axis=0), 1e-30)
    s = rng.uniform(0.0, vmax, size=n) * (1.0 - 1e-6)
    return np.ascontiguousarray((d * s).astype(np.float32))


# The test model of Sec. 3 in physical units: periodic square of side 2000 m, alpha_L = 10 m,
# D_m = 0, |v| = 1.16e-5 m/s at 45 degrees, Gaussian plume C0 = 0.32 kg/m^3, w = 44 m at the
# centre, 300 days; Table 1 runs of 1, 2 and 4 million irregular particles.
PAPER_SIDE_M = 2000.0
PAPER_DAY_S = 86400.0
PAPER_CPU_TIME_S = {1000000: 98766.54, 2000000: 495064.78, 4000000: 1773900.15}


def paper_plume(side, ratio, jitter=0.45, seed=3, steps=300):
    """The Sec. 3 test model in units of the box side L = 2000 m and of seconds, on side^2
    irregular particles (a jittered lattice, displacements U(-jitter, jitter) dx): the number of
    neighbours and the smoothing length follow the scaling relations of Sec. 2.3,
    n = 2.81 N^0.675 and h = 1.29 n^-0.247 L, with the Wendland C4 kernel (Eq. 7, support h);
    alpha_T = ratio * alpha_L.  The paper does not state its time step; dt = 1 day here, so 300
    steps cover its 300 days."""
    N = side * side
    n = 2.81 * N ** 0.675
    h_over_L = 1.29 * n ** -0.247
    L = PAPER_SIDE_M
    return Plume(dim=2, side=side, h_over_dx=h_over_L * side, kernel=WENDLAND_C4,
                 alpha_L=10.0 / L, alpha_T=ratio * 10.0 / L, D_m=0.0, speed=1.16e-5 / L,
                 angle=math.pi / 4.0, x0=(0.5, 0.5, 0.5), w=44.0 / L, C0=0.32, steps=steps,
                 jitter=jitter, seed=seed, dt=PAPER_DAY_S,
                 name=f"paper-2d-{N}-n{round(n)}-c4-aT_over_aL{ratio:g}")
