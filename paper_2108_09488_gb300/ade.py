"""Thin ctypes binding of libade_sph.so (include/ade_sph.h).

Every function here marshals arguments and calls the C entry point of the same name; all
computation happens in the library's CUDA kernels.  ``Simulation`` additionally owns the device
buffers (allocated through PyTorch) that the C API expects from its caller.

Loading fails loudly (``RuntimeError``) when the library has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libade_sph.so")

ADE_OK = 0
ERRORS = {-1: "ADE_ERR_ARG", -2: "ADE_ERR_CUDA", -3: "ADE_ERR_NUMERIC", -4: "ADE_ERR_TIMEOUT",
          -5: "ADE_ERR_CAPACITY", -6: "ADE_ERR_STATE"}
WENDLAND_C2 = 0
WENDLAND_C4 = 1
# interaction walks (ADE_FLAG_* of ade_sph.h); info.variant reports the one in use:
# 0 branch-free direct, 1 tiled, 2 branched direct, 3 / 4 = 0 / 2 over trimmed rows,
# 5 / 6 / 7 / 8 = 0 / 3 / 2 / 4 with two particles per thread (FLAG_PAIRED, packed FP32x2)
FLAG_DIRECT = 1
FLAG_TILED = 2
FLAG_BRANCHED = 4
FLAG_TRIMMED = 8
FLAG_PAIRED = 16
DT_LAMBDA_MAX = 0
DT_TRACE = 1

# every symbol declared in include/ade_sph.h
EXPORTS = ("ade_workspace_bytes", "ade_init_particles", "ade_get_info", "ade_build_cells",
           "ade_get_cells", "ade_dispersion_rate", "ade_count_pairs", "ade_step", "ade_run",
           "ade_get_stats", "ade_closed_form_error", "ade_destroy", "ade_last_error",
           "ade_step_timed", "ade_launches_per_step", "ade_build_cells_noalloc",
           "ade_batch_workspace_bytes", "ade_batch_init", "ade_batch_step", "ade_batch_run",
           "ade_batch_stats", "ade_batch_count_pairs", "ade_batch_get_plume_info",
           "ade_batch_autotune", "ade_batch_launches_per_step", "ade_batch_destroy",
           "ade_batch_get_config", "ade_batch_set_config",
           "ade_batch_step_timed", "ade_set_dispersivity", "ade_adjoint_workspace_bytes",
           "ade_adjoint", "ade_autotune", "ade_set_velocity_field", "ade_alu_peaks",
           "ade_sweep_workspace_bytes", "ade_sweep_init", "ade_sweep_get_info", "ade_sweep_rate",
           "ade_sweep_count_pairs", "ade_sweep_step", "ade_sweep_run", "ade_sweep_step_timed",
           "ade_sweep_launches_per_step", "ade_sweep_stats", "ade_sweep_destroy", "ade_set_flux",
           "ade_get_flux", "ade_checkpoint_bytes", "ade_checkpoint_save", "ade_checkpoint_load")
NOALLOC_MAX_PARTICLES = 1 << 20
NOALLOC_MAX_CELLS = 1 << 20


class AdeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("kernel", ctypes.c_int), ("box", ctypes.c_double * 3),
                ("h", ctypes.c_double), ("alpha_L", ctypes.c_double), ("alpha_T", ctypes.c_double),
                ("D_m", ctypes.c_double), ("v", ctypes.c_double * 3), ("mass", ctypes.c_double),
                ("rho", ctypes.c_double), ("gamma", ctypes.c_double), ("dt", ctypes.c_double),
                ("dt_rule", ctypes.c_int), ("dt_coef", ctypes.c_double),
                ("cell_subdiv", ctypes.c_int), ("flags", ctypes.c_uint), ("vmax", ctypes.c_double),
                ("tau", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("c_min", ctypes.c_double), ("c_max", ctypes.c_double),
                ("t", ctypes.c_double), ("step", ctypes.c_longlong), ("pairs", ctypes.c_longlong),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("support", ctypes.c_double), ("dt", ctypes.c_double), ("D", ctypes.c_double * 9),
                ("nc", ctypes.c_int * 3), ("ncells", ctypes.c_int), ("cell_subdiv", ctypes.c_int),
                ("stencil_rows", ctypes.c_int), ("sort_passes", ctypes.c_int),
                ("variant", ctypes.c_int), ("tile", ctypes.c_int * 3),
                ("tile_capacity", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t),
                ("skin", ctypes.c_double)]


_lib = None


def load():
    """Load libade_sph.so (raises RuntimeError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2108_09488_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, V, SZ, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_longlong
    sig = {
        "ade_workspace_bytes": (I, [ctypes.POINTER(Params), I, ctypes.POINTER(SZ)]),
        "ade_init_particles": (I, [ctypes.POINTER(P), ctypes.POINTER(Params), I, P, P, P, SZ]),
        "ade_get_info": (I, [P, ctypes.POINTER(Info)]),
        "ade_build_cells": (I, [P, V]),
        "ade_get_cells": (I, [P, P, P, V]),
        "ade_dispersion_rate": (I, [P, P, V]),
        "ade_count_pairs": (I, [P, ctypes.POINTER(LL), V]),
        "ade_step": (I, [P, I, V]),
        "ade_run": (I, [P, I, ctypes.POINTER(Stats), V]),
        "ade_get_stats": (I, [P, ctypes.POINTER(Stats), V]),
        "ade_closed_form_error": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                      ctypes.c_double, I, ctypes.POINTER(ctypes.c_double), V]),
        "ade_step_timed": (I, [P, ctypes.POINTER(ctypes.c_double), V]),
        "ade_launches_per_step": (I, [P, ctypes.POINTER(I)]),
        "ade_build_cells_noalloc": (I, [I, I, P, P, ctypes.POINTER(I), P, P, P, V]),
        "ade_batch_workspace_bytes": (I, [I, P, P, ctypes.POINTER(SZ)]),
        "ade_batch_init": (I, [ctypes.POINTER(P), I, P, P, P, P, P, SZ, V]),
        "ade_batch_step": (I, [P, I, V]),
        "ade_batch_run": (I, [P, I, V]),
        "ade_batch_stats": (I, [P, P, V]),
        "ade_batch_count_pairs": (I, [P, ctypes.POINTER(LL), V]),
        "ade_batch_get_plume_info": (I, [P, I, ctypes.POINTER(Info)]),
        "ade_batch_autotune": (I, [P, ctypes.POINTER(ctypes.c_double), V]),
        "ade_batch_get_config": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "ade_batch_set_config": (I, [P, I, I, I, I, V]),
        "ade_batch_launches_per_step": (I, [P, ctypes.POINTER(I)]),
        "ade_batch_step_timed": (I, [P, ctypes.POINTER(ctypes.c_double), V]),
        "ade_set_dispersivity": (I, [P, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "ade_set_velocity_field": (I, [P, P, V]),
        "ade_set_flux": (I, [P, P, V]),
        "ade_checkpoint_bytes": (I, [P, ctypes.POINTER(SZ)]),
        "ade_checkpoint_save": (I, [P, P, SZ, V]),
        "ade_checkpoint_load": (I, [P, P, SZ, V]),
        "ade_get_flux": (I, [P, P, V]),
        "ade_alu_peaks": (I, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), V]),
        "ade_sweep_workspace_bytes": (I, [ctypes.POINTER(Params), I, I, ctypes.POINTER(SZ)]),
        "ade_sweep_init": (I, [ctypes.POINTER(P), ctypes.POINTER(Params), I, I,
                               ctypes.POINTER(ctypes.c_double), P, P, P, SZ]),
        "ade_sweep_get_info": (I, [P, ctypes.POINTER(Info)]),
        "ade_sweep_rate": (I, [P, P, V]),
        "ade_sweep_count_pairs": (I, [P, ctypes.POINTER(LL), V]),
        "ade_sweep_step": (I, [P, I, V]),
        "ade_sweep_run": (I, [P, I, V]),
        "ade_sweep_step_timed": (I, [P, ctypes.POINTER(ctypes.c_double), V]),
        "ade_sweep_launches_per_step": (I, [P, ctypes.POINTER(I)]),
        "ade_sweep_stats": (I, [P, P, V]),
        "ade_sweep_destroy": (None, [P]),
        "ade_autotune": (I, [P, ctypes.POINTER(ctypes.c_double), V]),
        "ade_adjoint_workspace_bytes": (I, [P, I, I, ctypes.POINTER(SZ)]),
        "ade_adjoint": (I, [P, P, I, I, P, SZ, P, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), P, V]),
        "ade_batch_destroy": (None, [P]),
        "ade_destroy": (None, [P]),
        "ade_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != ADE_OK:
        raise AdeError(rc, load().ade_last_error().decode())
    return rc


def params(dim, h, alpha_L, alpha_T, D_m, v, mass, rho=1.0, box=1.0, kernel=WENDLAND_C2,
           gamma=0.0, dt=0.0, dt_rule=DT_LAMBDA_MAX, dt_coef=0.0, cell_subdiv=0, flags=0, vmax=0.0,
           tau=0.0):
    p = Params()
    p.dim = dim
    p.kernel = kernel
    b = np.ravel(np.asarray(box, dtype=np.float64))
    vv = np.ravel(np.asarray(v, dtype=np.float64))
    for i in range(3):
        p.box[i] = float(b[min(i, b.size - 1)]) if i < dim else 1.0
        p.v[i] = float(vv[i]) if i < min(dim, vv.size) else 0.0
    p.h, p.alpha_L, p.alpha_T, p.D_m = h, alpha_L, alpha_T, D_m
    p.mass, p.rho, p.gamma, p.dt = mass, rho, gamma, dt
    p.dt_rule, p.dt_coef, p.cell_subdiv, p.flags = dt_rule, dt_coef, cell_subdiv, flags
    p.vmax = vmax
    p.tau = tau
    return p


def params_for(plume, **over):
    """Params of an ``inputs.Plume`` workload (keyword overrides allowed)."""
    kw = dict(dim=plume.dim, h=plume.h, alpha_L=plume.alpha_L, alpha_T=plume.alpha_T,
              D_m=plume.D_m, v=plume.velocity, mass=plume.mass, rho=plume.rho, box=plume.box,
              kernel=plume.kernel, dt=plume.dt)
    kw.update(over)
    return params(**kw)


# ---- entry points (same names as the C ABI, without the ade_ prefix) --------------------------
def workspace_bytes(p, n):
    out = ctypes.c_size_t(0)
    _check(load().ade_workspace_bytes(ctypes.byref(p), n, ctypes.byref(out)))
    return out.value


def init_particles(p, n, xq_ptr, C_ptr, ws_ptr, ws_bytes):
    ctx = ctypes.c_void_p()
    _check(load().ade_init_particles(ctypes.byref(ctx), ctypes.byref(p), n, xq_ptr, C_ptr, ws_ptr,
                                     ws_bytes))
    return ctx


def get_info(ctx):
    info = Info()
    _check(load().ade_get_info(ctx, ctypes.byref(info)))
    return info


def build_cells(ctx, stream=None):
    _check(load().ade_build_cells(ctx, stream))


def get_cells(ctx, perm_ptr, cell_start_ptr, stream=None):
    _check(load().ade_get_cells(ctx, perm_ptr, cell_start_ptr, stream))


def dispersion_rate(ctx, out_ptr, stream=None):
    _check(load().ade_dispersion_rate(ctx, out_ptr, stream))


def count_pairs(ctx, stream=None):
    v = ctypes.c_longlong(0)
    _check(load().ade_count_pairs(ctx, ctypes.byref(v), stream))
    return v.value


def step(ctx, nsteps=1, stream=None):
    _check(load().ade_step(ctx, nsteps, stream))


def run(ctx, nsteps, stream=None, stats=True):
    st = Stats() if stats else None
    _check(load().ade_run(ctx, nsteps, ctypes.byref(st) if stats else None, stream))
    return st


def step_timed(ctx, stream=None):
    out = (ctypes.c_double * 4)()
    _check(load().ade_step_timed(ctx, out, stream))
    return list(out)


def launches_per_step(ctx):
    v = ctypes.c_int(0)
    _check(load().ade_launches_per_step(ctx, ctypes.byref(v)))
    return v.value


def get_stats(ctx, stream=None):
    st = Stats()
    rc = load().ade_get_stats(ctx, ctypes.byref(st), stream)
    if rc not in (ADE_OK, -3):
        _check(rc)
    return st


def closed_form_error(ctx, x0, w, C0=1.0, nimg=2, stream=None):
    x = (ctypes.c_double * 3)(*([float(u) for u in x0] + [0.0] * (3 - len(x0))))
    out = (ctypes.c_double * 4)()
    _check(load().ade_closed_form_error(ctx, x, w, C0, nimg, out, stream))
    return {"l2": out[0], "linf": out[1], "rmse": out[2], "c_an_max": out[3]}


def build_cells_noalloc(dim, n, xq_ptr, C_ptr, nc, perm_ptr, cell_start_ptr, sorted_ptr,
                        stream=None):
    """Cell build with the library's static scratch (no allocation); see include/ade_sph.h."""
    ncv = (ctypes.c_int * 3)(*([int(c) for c in nc[:dim]] + [1] * (3 - dim)))
    _check(load().ade_build_cells_noalloc(dim, n, xq_ptr, C_ptr, ncv, perm_ptr, cell_start_ptr,
                                          sorted_ptr, stream))


def alu_peaks(stream=None):
    """(FFMA/s, RSQRT/s) measured on the current device (ade_alu_peaks)."""
    f = ctypes.c_double(0.0)
    r = ctypes.c_double(0.0)
    _check(load().ade_alu_peaks(ctypes.byref(f), ctypes.byref(r), stream))
    return f.value, r.value


def checkpoint_save(ctx, stream=None):
    nb = ctypes.c_size_t(0)
    _check(load().ade_checkpoint_bytes(ctx, ctypes.byref(nb)))
    buf = ctypes.create_string_buffer(nb.value)
    _check(load().ade_checkpoint_save(ctx, buf, nb.value, stream))
    return buf.raw


def checkpoint_load(ctx, blob, stream=None):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    _check(load().ade_checkpoint_load(ctx, buf, len(blob), stream))


def destroy(ctx):
    if ctx:
        load().ade_destroy(ctx)


# ---- device-memory owner ----------------------------------------------------------------------
class Simulation:
    """Particle state + workspace on the current CUDA device, bound to one library context.

    ``xq`` (int32 [dim][n], the uint32 fixed-point words) and ``C`` (float32 [n]) are torch CUDA
    tensors in the caller's particle order; the library updates them in place."""

    def __init__(self, p, xq, C, device="cuda"):
        import torch
        self.torch = torch
        self.p = p
        xq = np.ascontiguousarray(xq, dtype=np.uint32)
        self.dim, self.n = xq.shape
        self.xq = torch.from_numpy(xq.view(np.int32)).to(device).contiguous()
        self.C = torch.as_tensor(np.ascontiguousarray(C, dtype=np.float32)).to(device).contiguous()
        nbytes = workspace_bytes(p, self.n)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        self.ws_bytes = nbytes
        self.ctx = init_particles(p, self.n, self.xq.data_ptr(), self.C.data_ptr(), self.ws_ptr, nbytes)
        self.info = get_info(self.ctx)

    @property
    def stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def build_cells(self):
        build_cells(self.ctx, self.stream)

    def cells(self):
        """(perm uint32 [n], cell_start uint32 [ncells+1]) of the last cell build, as numpy."""
        t = self.torch
        perm = t.empty(max(self.n, 1), dtype=t.int32, device=self.C.device)
        cs = t.empty(self.info.ncells + 1, dtype=t.int32, device=self.C.device)
        get_cells(self.ctx, perm.data_ptr(), cs.data_ptr(), self.stream)
        t.cuda.synchronize()
        return (perm.cpu().numpy().view(np.uint32)[: self.n], cs.cpu().numpy().view(np.uint32))

    def rate(self):
        out = self.torch.empty(max(self.n, 1), dtype=self.torch.float32, device=self.C.device)
        dispersion_rate(self.ctx, out.data_ptr(), self.stream)
        return out[: self.n]

    def count_pairs(self):
        return count_pairs(self.ctx, self.stream)

    def step(self, nsteps=1):
        step(self.ctx, nsteps, self.stream)

    def run(self, nsteps, stats=True):
        return run(self.ctx, nsteps, self.stream, stats)

    def step_timed(self):
        return step_timed(self.ctx, self.stream)

    def stats(self):
        return get_stats(self.ctx, self.stream)

    def closed_form_error(self, x0, w, C0=1.0, nimg=2):
        return closed_form_error(self.ctx, x0, w, C0, nimg, self.stream)

    def autotune(self):
        """Pick the cell subdivision and interaction walk (variants 0-8) by timing a cell build
        and two evaluations per configuration (ade_autotune); returns that time in ms."""
        ms = ctypes.c_double(0.0)
        _check(load().ade_autotune(self.ctx, ctypes.byref(ms), self.stream))
        self.info = get_info(self.ctx)
        return ms.value

    def set_dispersivity(self, alpha_L, alpha_T, D_m):
        _check(load().ade_set_dispersivity(self.ctx, alpha_L, alpha_T, D_m))

    def checkpoint(self):
        """Snapshot of the state (ade_checkpoint_save) as bytes."""
        return checkpoint_save(self.ctx, self.stream)

    def restore(self, blob):
        """Resume from a snapshot taken of a context with the same parameters (ade_checkpoint_load)."""
        checkpoint_load(self.ctx, blob, self.stream)

    def set_flux(self, Q=None):
        """Cattaneo form (tau > 0): set the flux Q = dC/dt (float32 [n], caller order), or with
        None the Fickian flux R(C) of the current state (ade_set_flux)."""
        t = self.torch
        if Q is None:
            _check(load().ade_set_flux(self.ctx, None, self.stream))
            return
        q = t.as_tensor(np.ascontiguousarray(Q, dtype=np.float32) if not t.is_tensor(Q) else Q,
                        dtype=t.float32, device=self.C.device).contiguous()
        _check(load().ade_set_flux(self.ctx, q.data_ptr() if self.n else None, self.stream))
        t.cuda.current_stream().synchronize()

    def flux(self):
        """The current flux Q (Cattaneo form) as a torch tensor [n]."""
        out = self.torch.empty(max(self.n, 1), dtype=self.torch.float32, device=self.C.device)
        _check(load().ade_get_flux(self.ctx, out.data_ptr(), self.stream))
        return out[: self.n]

    def set_velocity_field(self, v):
        """Per-particle velocities (float32 [dim][n], caller order) of a context created with
        vmax > 0 (ade_set_velocity_field); the library keeps its own copy."""
        t = self.torch
        vt = t.as_tensor(np.ascontiguousarray(v, dtype=np.float32) if not t.is_tensor(v) else v,
                         dtype=t.float32, device=self.C.device).contiguous()
        if tuple(vt.shape) != (self.dim, self.n):
            raise ValueError(f"velocity field must be [{self.dim}][{self.n}], got {tuple(vt.shape)}")
        _check(load().ade_set_velocity_field(self.ctx, vt.data_ptr() if self.n else None, self.stream))

    def adjoint(self, C_target, nsteps, ckpt_every=40, want_dC0=True, want_final=False):
        """Misfit J = 1/2 |C^N - C*|^2 and its gradients (adjoint of Eq. 8-9, see ade_adjoint).
        Returns (J, dJ/d(alpha_L, alpha_T, D_m) as a numpy array, dJ/dC0 tensor or None,
        C^N tensor or None)."""
        t = self.torch
        tgt = t.as_tensor(C_target, dtype=t.float32, device=self.C.device).contiguous()
        nbytes = ctypes.c_size_t(0)
        _check(load().ade_adjoint_workspace_bytes(self.ctx, nsteps, ckpt_every, ctypes.byref(nbytes)))
        aws = t.empty(nbytes.value + 256, dtype=t.uint8, device=self.C.device)
        aws_ptr = (aws.data_ptr() + 255) // 256 * 256
        dC0 = t.empty(max(self.n, 1), dtype=t.float32, device=self.C.device) if want_dC0 else None
        fin = t.empty(max(self.n, 1), dtype=t.float32, device=self.C.device) if want_final else None
        g = (ctypes.c_double * 3)()
        J = ctypes.c_double(0.0)
        _check(load().ade_adjoint(self.ctx, tgt.data_ptr(), nsteps, ckpt_every, aws_ptr, nbytes.value,
                                  dC0.data_ptr() if dC0 is not None else None, g, ctypes.byref(J),
                                  fin.data_ptr() if fin is not None else None, self.stream))
        return (J.value, np.array(list(g)), dC0[: self.n] if dC0 is not None else None,
                fin[: self.n] if fin is not None else None)

    def state(self):
        """(xq uint32 [dim][n], C float32 [n]) copied to the host."""
        self.torch.cuda.synchronize()
        return self.xq.cpu().numpy().view(np.uint32), self.C.cpu().numpy()

    def close(self):
        if self.ctx:
            destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched plumes ---------------------------------------------------------------------------
def _params_array(plist):
    arr = (Params * len(plist))()
    for i, p in enumerate(plist):
        arr[i] = p
    return arr


def batch_workspace_bytes(plist, ns):
    arr = _params_array(plist)
    nn = (ctypes.c_int * len(ns))(*[int(v) for v in ns])
    out = ctypes.c_size_t(0)
    _check(load().ade_batch_workspace_bytes(len(plist), arr, nn, ctypes.byref(out)))
    return out.value


class Batch:
    """Many plumes stepped together through the ade_batch_* entry points.

    ``xq_list[p]`` (uint32 [dim][n_p]) and ``C_list[p]`` (float32 [n_p]) are copied into one
    concatenated device state (plume p's position block starts at element dim * off_p)."""

    def __init__(self, plist, xq_list, C_list, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.P = len(plist)
        self.dim = plist[0].dim
        self.ns = [int(np.asarray(x).shape[1]) for x in xq_list]
        self.offsets = np.concatenate([[0], np.cumsum(self.ns)]).astype(np.int64)
        xq = np.concatenate([np.ascontiguousarray(x, dtype=np.uint32).ravel() for x in xq_list])
        C = np.concatenate([np.asarray(c, dtype=np.float32).ravel() for c in C_list])
        self.xq = torch.from_numpy(xq.view(np.int32)).to(device).contiguous()
        self.C = torch.from_numpy(C).to(device).contiguous()
        self._params = _params_array(plist)
        self._n = (ctypes.c_int * self.P)(*self.ns)
        nbytes = batch_workspace_bytes(plist, self.ns)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        self.ws_ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self.ctx = ctypes.c_void_p()
        _check(load().ade_batch_init(ctypes.byref(self.ctx), self.P, self._params, self._n,
                                     self.xq.data_ptr(), self.C.data_ptr(), self.ws_ptr, nbytes,
                                     self.stream))

    @property
    def stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def step(self, nsteps=1):
        _check(load().ade_batch_step(self.ctx, nsteps, self.stream))

    def run(self, nsteps):
        _check(load().ade_batch_run(self.ctx, nsteps, self.stream))

    def stats(self):
        st = (Stats * self.P)()
        rc = load().ade_batch_stats(self.ctx, st, self.stream)
        if rc not in (ADE_OK, -3):
            _check(rc)
        return list(st)

    def count_pairs(self):
        v = ctypes.c_longlong(0)
        _check(load().ade_batch_count_pairs(self.ctx, ctypes.byref(v), self.stream))
        return v.value

    def plume_info(self, p):
        info = Info()
        _check(load().ade_batch_get_plume_info(self.ctx, p, ctypes.byref(info)))
        return info

    def autotune(self):
        ms = ctypes.c_double(0.0)
        _check(load().ade_batch_autotune(self.ctx, ctypes.byref(ms), self.stream))
        return ms.value

    def config(self):
        """(subdivision policy, work-item size, persistent grid, paired walk) in use."""
        m, t, g, w = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(load().ade_batch_get_config(self.ctx, ctypes.byref(m), ctypes.byref(t), ctypes.byref(g),
                                           ctypes.byref(w)))
        return m.value, t.value, g.value, w.value

    def set_config(self, cfg):
        """Apply a (subdivision policy, work-item size, persistent grid, paired walk) tuple, e.g.
        another batch's config() after its autotune."""
        _check(load().ade_batch_set_config(self.ctx, int(cfg[0]), int(cfg[1]), int(cfg[2]), int(cfg[3]),
                                           self.stream))

    def launches_per_step(self):
        v = ctypes.c_int(0)
        _check(load().ade_batch_launches_per_step(self.ctx, ctypes.byref(v)))
        return v.value

    def step_timed(self):
        out = (ctypes.c_double * 4)()
        _check(load().ade_batch_step_timed(self.ctx, out, self.stream))
        return list(out)

    def state(self, p):
        """(xq uint32 [dim][n_p], C float32 [n_p]) of plume p, copied to the host."""
        self.torch.cuda.synchronize()
        lo, hi = int(self.offsets[p]), int(self.offsets[p + 1])
        xq = self.xq[self.dim * lo:self.dim * hi].cpu().numpy().view(np.uint32).reshape(self.dim, hi - lo)
        return xq, self.C[lo:hi].cpu().numpy()

    def close(self):
        if self.ctx:
            load().ade_batch_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- parameter sweep ----------------------------------------------------------------------------
def sweep_workspace_bytes(p, n, ntheta):
    out = ctypes.c_size_t(0)
    _check(load().ade_sweep_workspace_bytes(ctypes.byref(p), n, ntheta, ctypes.byref(out)))
    return out.value


class Sweep:
    """P dispersivity sets theta[k] = (alpha_L, alpha_T, D_m) on one particle set through the
    ade_sweep_* entry points.  ``C`` is a float32 [P][n] torch CUDA tensor (set k's field in row k),
    ``xq`` the shared int32 [dim][n] positions; both are updated in place."""

    def __init__(self, p, xq, C_sets, theta, device="cuda"):
        import torch
        self.torch = torch
        self.p = p
        xq = np.ascontiguousarray(xq, dtype=np.uint32)
        self.dim, self.n = xq.shape
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 3)
        self.P = th.shape[0]
        C = np.array(np.broadcast_to(np.asarray(C_sets, dtype=np.float32), (self.P, self.n)))
        self.xq = torch.from_numpy(xq.view(np.int32)).to(device).contiguous()
        self.C = torch.from_numpy(C).to(device).contiguous()
        nbytes = sweep_workspace_bytes(p, self.n, self.P)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        self.ws_ptr = (self.ws.data_ptr() + 255) // 256 * 256
        self._theta = (ctypes.c_double * th.size)(*th.ravel().tolist())
        self.ctx = ctypes.c_void_p()
        _check(load().ade_sweep_init(ctypes.byref(self.ctx), ctypes.byref(p), self.n, self.P,
                                     self._theta, self.xq.data_ptr(), self.C.data_ptr(), self.ws_ptr,
                                     nbytes))
        self.info = Info()
        _check(load().ade_sweep_get_info(self.ctx, ctypes.byref(self.info)))

    @property
    def stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def rate(self):
        out = self.torch.empty((self.P, max(self.n, 1)), dtype=self.torch.float32, device=self.C.device)
        _check(load().ade_sweep_rate(self.ctx, out.data_ptr(), self.stream))
        return out[:, : self.n]

    def count_pairs(self):
        v = ctypes.c_longlong(0)
        _check(load().ade_sweep_count_pairs(self.ctx, ctypes.byref(v), self.stream))
        return v.value

    def step(self, nsteps=1):
        _check(load().ade_sweep_step(self.ctx, nsteps, self.stream))

    def run(self, nsteps):
        _check(load().ade_sweep_run(self.ctx, nsteps, self.stream))

    def step_timed(self):
        out = (ctypes.c_double * 4)()
        _check(load().ade_sweep_step_timed(self.ctx, out, self.stream))
        return list(out)

    def launches_per_step(self):
        v = ctypes.c_int(0)
        _check(load().ade_sweep_launches_per_step(self.ctx, ctypes.byref(v)))
        return v.value

    def stats(self):
        st = (Stats * self.P)()
        rc = load().ade_sweep_stats(self.ctx, st, self.stream)
        if rc not in (ADE_OK, -3):
            _check(rc)
        return list(st)

    def state(self):
        self.torch.cuda.synchronize()
        return self.xq.cpu().numpy().view(np.uint32), self.C.cpu().numpy()

    def close(self):
        if self.ctx:
            load().ade_sweep_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
