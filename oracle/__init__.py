"""FP64 CPU oracle for the SPH advection-dispersion path (Klapp et al., arXiv 2108.09488).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The GPU library shares no code with it and never
calls it.

The arithmetic lives in ``ade_oracle.c`` (plain C, FP64), compiled by :func:`build` with gcc and
loaded through ctypes.  This module only marshals numpy arrays and adds a few helpers written
directly from the paper:

* :func:`dt_rule` -- Sec. 2.4, Eq. 10 and the largest-eigenvalue variant;
* :func:`scaling_relations` -- Sec. 2.3, n ~ 2.81 N^0.675 and h ~ 1.29 n^-0.247 (Table 1);
* :func:`stats` -- mass, extrema and error norms against the closed form (Sec. 4, Table 2).

Function-level citations are in the C source.  Parity status of every function: pinned by
``tests/test_oracle_*.py`` (see each test's docstring for the pin it uses).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ade_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_ade_oracle.so")
_lib = None
_lock = threading.Lock()

WENDLAND_C2 = 0
WENDLAND_C4 = 1

_d = ctypes.c_double
_i = ctypes.c_int
_ll = ctypes.c_longlong
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP over particles)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.orc_dispersion_tensor.argtypes = [_i, _p, _d, _d, _d, _p]
            lib.orc_kernel_w.argtypes = [_i, _i, _d, _d]
            lib.orc_kernel_w.restype = _d
            lib.orc_kernel_dwdr.argtypes = [_i, _i, _d, _d]
            lib.orc_kernel_dwdr.restype = _d
            lib.orc_pair_term.argtypes = [_i, _p, _p, _p, _d, _d, _p, _p, _d, _d, _d, _i, _d, _d,
                                          _p, _p]
            lib.orc_neighbours_brute.argtypes = [_i, _i, _p, _p, _d, _p, _p, _ll]
            lib.orc_neighbours_brute.restype = _ll
            lib.orc_neighbours_cells.argtypes = [_i, _i, _p, _p, _d, _p, _p, _ll]
            lib.orc_neighbours_cells.restype = _ll
            lib.orc_rate.argtypes = [_i, _i, _p, _p, _p, _p, _p, _p, _i, _d, _d, _d, _d, _d, _i,
                                     _p, _p, _p]
            lib.orc_rate.restype = _ll
            lib.orc_rate_sel.argtypes = [_i, _i, _p, _p, _p, _p, _p, _p, _i, _d, _d, _d, _d, _d,
                                         _i, _i, _p, _p, _p, _p]
            lib.orc_rate_sel.restype = _ll
            lib.orc_step.argtypes = [_i, _i, _p, _p, _p, _p, _p, _p, _i, _d, _d, _d, _d, _d, _d, _i]
            lib.orc_step.restype = _ll
            lib.orc_step_cattaneo.argtypes = [_i, _i, _p, _p, _p, _p, _p, _p, _p, _i, _d, _d, _d, _d,
                                              _d, _d, _d, _i]
            lib.orc_step_cattaneo.restype = _ll
            lib.orc_cell_keys.argtypes = [_i, _i, _p, _p, _p]
            lib.orc_sort_cells.argtypes = [_i, _p, _i, _p, _p]
            lib.orc_sort_cells.restype = _i
            lib.orc_closed_form.argtypes = [_i, _i, _p, _p, _p, _p, _p, _d, _d, _d, _i, _p]
            lib.orc_set_threads.argtypes = [_i]
            lib.orc_set_threads.restype = None
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = _i
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------------------------
# Eq. 3
# --------------------------------------------------------------------------------------------
def dispersion_tensor(v, alpha_L, alpha_T, D_m):
    """Eq. 3: D = (aT|v| + Dm) I + (aL - aT) v v^T / |v|  (dim x dim, FP64)."""
    v = _f64(v).ravel()
    dim = v.size
    D = np.zeros((dim, dim))
    _load().orc_dispersion_tensor(dim, _ptr(v), alpha_L, alpha_T, D_m, _ptr(D))
    return D


# --------------------------------------------------------------------------------------------
# Kernels (Eq. 7 and the Wendland C2 member of the same family)
# --------------------------------------------------------------------------------------------
def kernel_w(kind, dim, H, r):
    """Kernel value W(r) for support radius H."""
    lib = _load()
    return np.array([lib.orc_kernel_w(kind, dim, H, float(x)) for x in np.ravel(r)])


def kernel_dwdr(kind, dim, H, r):
    """dW/dr for support radius H."""
    lib = _load()
    return np.array([lib.orc_kernel_dwdr(kind, dim, H, float(x)) for x in np.ravel(r)])


def support_radius(kind, h):
    """Support radius H: 2h for Wendland C2, h for the paper's Wendland C4 (Eq. 7)."""
    return 2.0 * h if kind == WENDLAND_C2 else h


def pair_term(xab, Da, Db, Ca, Cb, va, vb, mb, rhoa, rhob, kind, H, gamma):
    """One ordered pair of Eq. 4-5: returns (dispersive part, convective part)."""
    xab = _f64(xab).ravel()
    dim = xab.size
    Da = _f64(Da).ravel()
    Db = _f64(Db).ravel()
    va = _f64(va).ravel()
    vb = _f64(vb).ravel()
    out = np.zeros(2)
    _load().orc_pair_term(dim, _ptr(xab), _ptr(Da), _ptr(Db), Ca, Cb, _ptr(va), _ptr(vb), mb,
                          rhoa, rhob, kind, H, gamma, _ptr(out[0:]), _ptr(out[1:]))
    return out[0], out[1]


# --------------------------------------------------------------------------------------------
# Neighbour search
# --------------------------------------------------------------------------------------------
def neighbours(x, box, H, brute=False, cap=None):
    """CSR neighbour lists (ptr, idx): all b != a with 0 < |x_ab| < H (minimum image)."""
    x = _f64(x)
    n, dim = x.shape
    box = _f64(box).ravel()
    if cap is None:
        cap = max(16, int(n * 1.5 * _expected_n(dim, box, H, n)) + 64)
    ptr = np.zeros(n + 1, dtype=np.int64)
    idx = np.zeros(cap, dtype=np.int32)
    fn = _load().orc_neighbours_brute if brute else _load().orc_neighbours_cells
    k = fn(dim, n, _ptr(x), _ptr(box), H, _ptr(ptr), _ptr(idx), cap)
    if k < 0:
        return neighbours(x, box, H, brute, cap * 4)
    return ptr, idx[:k].copy()


def _expected_n(dim, box, H, n):
    vol = float(np.prod(box[:dim]))
    ball = np.pi * H * H if dim == 2 else 4.0 / 3.0 * np.pi * H ** 3
    return max(1.0, n * ball / vol)


# --------------------------------------------------------------------------------------------
# Eq. 4-5 and Eq. 8-9
# --------------------------------------------------------------------------------------------
def _per_particle(a, n, dim=None):
    a = np.asarray(a, dtype=np.float64)
    if dim is None:
        return np.ascontiguousarray(np.broadcast_to(a, (n,)), dtype=np.float64)
    return np.ascontiguousarray(np.broadcast_to(a, (n, dim)), dtype=np.float64)


def rate(x, v, C, m, rho, box, kind, H, gamma, alpha_L, alpha_T, D_m, brute=False,
         split=False):
    """Eq. 4 for every particle (FP64).  Returns (rate, pairs) or, with split=True,
    (rate, dispersive part, convective part, pairs)."""
    x = _f64(x)
    n, dim = x.shape
    v = _per_particle(v, n, dim)
    C = _f64(C).ravel()
    m = _per_particle(m, n)
    rho = _per_particle(rho, n)
    box = _f64(box).ravel()
    r = np.zeros(n)
    rd = np.zeros(n)
    rc = np.zeros(n)
    pairs = _load().orc_rate(dim, n, _ptr(x), _ptr(v), _ptr(C), _ptr(m), _ptr(rho), _ptr(box),
                             kind, H, gamma, alpha_L, alpha_T, D_m, int(brute), _ptr(r), _ptr(rd),
                             _ptr(rc))
    if split:
        return r, rd, rc, pairs
    return r, pairs


def rate_at(sel, x, v, C, m, rho, box, kind, H, gamma, alpha_L, alpha_T, D_m):
    """Eq. 4 for the selected particles only (same arithmetic as :func:`rate`)."""
    x = _f64(x)
    n, dim = x.shape
    v = _per_particle(v, n, dim)
    C = _f64(C).ravel()
    m = _per_particle(m, n)
    rho = _per_particle(rho, n)
    box = _f64(box).ravel()
    sel = np.ascontiguousarray(sel, dtype=np.int32)
    r = np.zeros(sel.size)
    pairs = _load().orc_rate_sel(dim, n, _ptr(x), _ptr(v), _ptr(C), _ptr(m), _ptr(rho),
                                 _ptr(box), kind, H, gamma, alpha_L, alpha_T, D_m, 0, sel.size,
                                 _ptr(sel), _ptr(r), None, None)
    return r, pairs


def step(x, v, C, m, rho, box, kind, H, gamma, alpha_L, alpha_T, D_m, dt, nsteps=1,
         brute=False):
    """Eq. 8-9: nsteps predictor-corrector steps.  Returns new (x, C, pairs)."""
    x = _f64(x).copy()
    n, dim = x.shape
    v = _per_particle(v, n, dim)
    C = _f64(C).ravel().copy()
    m = _per_particle(m, n)
    rho = _per_particle(rho, n)
    box = _f64(box).ravel()
    pairs = 0
    lib = _load()
    for _ in range(nsteps):
        pairs += lib.orc_step(dim, n, _ptr(x), _ptr(v), _ptr(C), _ptr(m), _ptr(rho), _ptr(box),
                              kind, H, gamma, alpha_L, alpha_T, D_m, dt, int(brute))
    return x, C, pairs


def step_cattaneo(x, v, C, Q, m, rho, box, kind, H, gamma, alpha_L, alpha_T, D_m, dt, tau,
                  nsteps=1, brute=False):
    """Eq. 14 (Cattaneo's hyperbolic form) as the system dC/dt = Q, tau dQ/dt = R(C) - Q, advanced
    by the midpoint rule of Eq. 8-9.  Returns new (x, C, Q, pairs)."""
    x = _f64(x).copy()
    n, dim = x.shape
    v = _per_particle(v, n, dim)
    C = _f64(C).ravel().copy()
    Q = _f64(Q).ravel().copy()
    m = _per_particle(m, n)
    rho = _per_particle(rho, n)
    box = _f64(box).ravel()
    pairs = 0
    lib = _load()
    for _ in range(nsteps):
        pairs += lib.orc_step_cattaneo(dim, n, _ptr(x), _ptr(v), _ptr(C), _ptr(Q), _ptr(m), _ptr(rho),
                                       _ptr(box), kind, H, gamma, alpha_L, alpha_T, D_m, dt, tau,
                                       int(brute))
    return x, C, Q, pairs


# --------------------------------------------------------------------------------------------
# Cell list on fixed-point positions (bit-exact reference for the GPU cell build)
# --------------------------------------------------------------------------------------------
def cell_keys(xq, nc):
    """Linear cell key of each particle; xq is uint32 [dim][n], nc cells per axis."""
    xq = np.ascontiguousarray(xq, dtype=np.uint32)
    dim, n = xq.shape
    ncv = np.ones(3, dtype=np.int32)
    ncv[:dim] = nc[:dim]
    key = np.zeros(n, dtype=np.uint32)
    _load().orc_cell_keys(dim, n, _ptr(xq), _ptr(ncv), _ptr(key))
    return key


def sort_cells(key, ncells):
    """Stable counting sort by key: (perm, cell_start[ncells+1])."""
    key = np.ascontiguousarray(key, dtype=np.uint32)
    perm = np.zeros(key.size, dtype=np.uint32)
    start = np.zeros(ncells + 1, dtype=np.uint32)
    if _load().orc_sort_cells(key.size, _ptr(key), ncells, _ptr(perm), _ptr(start)) != 0:
        raise ValueError("key out of range")
    return perm, start


# --------------------------------------------------------------------------------------------
# Closed form (Eq. 12-13) and metrics
# --------------------------------------------------------------------------------------------
def closed_form(x, box, x0, v, D, w, C0, t, nimg=2):
    """Eq. 12-13 (2D) or the 3D Gaussian of the same family, summed over periodic images."""
    x = _f64(x)
    n, dim = x.shape
    box = _f64(box).ravel()
    x0 = _f64(x0).ravel()
    v = _f64(v).ravel()
    D = _f64(D)
    C = np.zeros(n)
    _load().orc_closed_form(dim, n, _ptr(x), _ptr(box), _ptr(x0), _ptr(v), _ptr(D), w, C0, t,
                            nimg, _ptr(C))
    return C


def set_threads(n):
    """Host threads of the oracle's OpenMP loops (n <= 0 leaves the setting)."""
    _load().orc_set_threads(int(n))


def max_threads():
    return int(_load().orc_max_threads())


def dt_rule(D, h, rule="lambda_max", coef=0.1):
    """Time step.  'trace': Eq. 10, coef * h^2 / (D_xx + D_yy [+ D_zz]) (uniform D, so the min over
    particles is that one value).  'lambda_max': coef * h^2 / lambda_max(D), the largest-eigenvalue
    form used for the lattice workloads."""
    D = np.asarray(D, dtype=np.float64)
    if rule == "trace":
        return coef * h * h / float(np.trace(D))
    return coef * h * h / float(np.max(np.linalg.eigvalsh(D)))


def scaling_relations(N):
    """Sec. 2.3: n ~ 2.81 N^0.675 and h ~ 1.29 n^-0.247 (h in units of L)."""
    n = 2.81 * N ** 0.675
    return n, 1.29 * n ** -0.247


def stats(C, m, C_ref=None, C0=1.0, vol=None):
    """Mass sum(m C), min, max; with C_ref: L2 = sqrt(sum V (C-C_ref)^2), Linf, RMSE of C/C0."""
    C = np.asarray(C, dtype=np.float64)
    m = np.broadcast_to(np.asarray(m, dtype=np.float64), C.shape)
    out = {"mass": float(np.sum(m * C)), "c_min": float(C.min()), "c_max": float(C.max())}
    if C_ref is not None:
        e = C - np.asarray(C_ref, dtype=np.float64)
        V = m if vol is None else np.broadcast_to(vol, C.shape)
        out["l2"] = float(np.sqrt(np.sum(V * e * e)))
        out["linf"] = float(np.max(np.abs(e)))
        out["rmse"] = float(np.sqrt(np.mean((e / C0) ** 2)))
    return out


# --------------------------------------------------------------------------------------------
# Misfit and its gradient (checks for the adjoint; FP64)
# --------------------------------------------------------------------------------------------
def _R(x, v, C, m, rho, box, kind, H, gamma, theta):
    """Eq. 4 with theta = (alpha_L, alpha_T, D_m) at fixed positions."""
    return rate(x, v, C, m, rho, box, kind, H, gamma, theta[0], theta[1], theta[2])[0]


def misfit(x, v, C0, m, rho, box, kind, H, gamma, theta, dt, nsteps, target):
    """J = 1/2 sum (C^N - C*)^2 for nsteps of Eq. 8-9 at fixed positions (a uniform drift leaves
    every separation, hence the rate, unchanged), dt fixed.  Returns (J, C^N)."""
    C = np.asarray(C0, dtype=np.float64).copy()
    for _ in range(nsteps):
        a = _R(x, v, C, m, rho, box, kind, H, gamma, theta)
        C = C + dt * _R(x, v, C + 0.5 * dt * a, m, rho, box, kind, H, gamma, theta)
    e = C - np.asarray(target, dtype=np.float64)
    return 0.5 * float(np.dot(e, e)), C


def misfit_gradient_tlm(x, v, C0, m, rho, box, kind, H, gamma, theta, dt, nsteps, target):
    """dJ/dtheta by the tangent-linear model: with S(theta) C = C + dt R(C + dt/2 R(C)),
    dC^{l+1}/dtheta_k = S dC^l/dtheta_k + (dS/dtheta_k) C^l, where (dS/dtheta_k) C =
    dt R_k(C) + dt^2/2 (R_k(R(C)) + R(R_k(C))) and R_k is Eq. 4 with theta = e_k (D of Eq. 3 is
    linear in theta).  Returns (J, gradient[3])."""
    ek = [np.eye(3)[k] for k in range(3)]
    args = (x, v)
    kw = (m, rho, box, kind, H, gamma)
    R = lambda C, th: _R(*args, C, *kw, th)
    C = np.asarray(C0, dtype=np.float64).copy()
    dC = [np.zeros_like(C) for _ in range(3)]
    for _ in range(nsteps):
        RC = R(C, theta)
        for k in range(3):
            Rk = R(C, ek[k])
            dSk = dt * Rk + 0.5 * dt * dt * (R(RC, ek[k]) + R(Rk, theta))
            d = dC[k]
            Sd = d + dt * R(d + 0.5 * dt * R(d, theta), theta)
            dC[k] = Sd + dSk
        C = C + dt * R(C + 0.5 * dt * RC, theta)
    e = C - np.asarray(target, dtype=np.float64)
    return 0.5 * float(np.dot(e, e)), np.array([float(np.dot(e, dC[k])) for k in range(3)])
