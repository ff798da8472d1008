"""Thin ctypes binding of the C ABI in include/pf.h (argument marshalling only).

Every step of the computation runs in the CUDA library ``libpf.so``; this
module only converts Python arguments to the C structs and pointers.  Arrays
may be numpy arrays (host memory, ``mem=PF_MEM_HOST``) or torch CUDA tensors
(device memory, ``mem=PF_MEM_DEVICE``; their ``data_ptr()`` is passed).
Importing it does not need a GPU; creating a handle does.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ENOCONV, PF_ENAN, PF_ETIMEOUT, PF_ECHECK = 0, -1, -2, -3, -4, -5, -6, -7
PF_FP64, PF_FP32, PF_MIXED = 0, 1, 2
PF_MEM_HOST, PF_MEM_DEVICE = 0, 1
PF_C0_PER_STEP, PF_C0_FIXED = 0, 1
PF_LOAD_STRAIN, PF_LOAD_UNIAXIAL = 0, 1

# every entry point declared in include/pf.h
EXPORTS = ("pf_config_default", "pf_create", "pf_create_batch", "pf_destroy", "pf_set_fields", "pf_set_plastic_strain",
           "pf_get_fields", "pf_set_mobility",
           "pf_step", "pf_stress", "pf_energy", "pf_timing", "pf_timing_get",
           "pf_launch_count", "pf_strerror", "pf_ms_residual_static", "pf_fma_peak")


class PfConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("n_variants", ctypes.c_int),
        ("variant_ids", ctypes.c_int * 6),
        ("precision", ctypes.c_int),
        ("c1", ctypes.c_double), ("c2", ctypes.c_double), ("c3", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma_tw", ctypes.c_double),
        ("c_over_a", ctypes.c_double),
        ("twin_angle_deg", ctypes.c_double),
        ("C_hex", ctypes.c_double * 5),
        ("twin_stiffness", ctypes.c_int),
        ("ms_tol", ctypes.c_double),
        ("ms_max_it", ctypes.c_int),
        ("c0_mode", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("n_grains", ctypes.c_int),
        ("grain_R", ctypes.POINTER(ctypes.c_double)),
        ("stream", ctypes.c_void_p),
        ("load_mode", ctypes.c_int),
        ("load_dir", ctypes.c_double * 3),
        ("warm_degree", ctypes.c_int),
        ("c2_aniso", ctypes.c_double * 3),
        ("mob_corr", ctypes.c_int),
        ("pic_iters", ctypes.c_int),
        ("clamp", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("warm_points", ctypes.c_int),
    ]


class PfStepInfo(ctypes.Structure):
    _fields_ = [
        ("n_ms_last", ctypes.c_int),
        ("n_ms_total", ctypes.c_int),
        ("resid", ctypes.c_double),
        ("status", ctypes.c_int),
        ("mean_sigma", ctypes.c_double * 6),
        ("mean_strain", ctypes.c_double * 6),
        ("mob_change", ctypes.c_double),
        ("pic_change", ctypes.c_double),
    ]


_LIB = None


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libpf.so (building it first when needed); raises if it cannot.
    With PF_CHECK_BUILD=1 in the environment the PF_CHECK variant
    (libpf_check.so) is built and loaded instead."""
    global _LIB
    if _LIB is not None:
        return _LIB
    check = os.environ.get("PF_CHECK_BUILD", "0") == "1"
    path = _build.LIB_CHECK if check else _build.LIB
    if build_if_missing:
        path = _build.build_library(check=check)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run the build first")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.pf_config_default.argtypes = [ctypes.POINTER(PfConfig)]
    lib.pf_config_default.restype = None
    lib.pf_create.argtypes = [ctypes.POINTER(PfConfig), ip, ctypes.POINTER(vp)]
    lib.pf_create.restype = ip
    lib.pf_create_batch.argtypes = [ctypes.POINTER(PfConfig), ip, ctypes.POINTER(vp)]
    lib.pf_create_batch.restype = ip
    lib.pf_destroy.argtypes = [vp]
    lib.pf_destroy.restype = None
    lib.pf_set_fields.argtypes = [vp, ip, vp, vp, vp, vp, ip]
    lib.pf_set_fields.restype = ip
    lib.pf_set_plastic_strain.argtypes = [vp, ip, vp, ip]
    lib.pf_set_plastic_strain.restype = ip
    lib.pf_get_fields.argtypes = [vp, ip, vp, vp, ip]
    lib.pf_get_fields.restype = ip
    lib.pf_step.argtypes = [vp, ip, ctypes.POINTER(dp), ctypes.POINTER(PfStepInfo)]
    lib.pf_step.restype = ip
    lib.pf_stress.argtypes = [vp, ip, ctypes.POINTER(dp), vp, ip]
    lib.pf_stress.restype = ip
    lib.pf_energy.argtypes = [vp, ip, ctypes.POINTER(dp)]
    lib.pf_energy.restype = ip
    lib.pf_timing.argtypes = [vp, ip]
    lib.pf_timing.restype = ip
    lib.pf_timing_get.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(dp),
                                  ctypes.POINTER(ctypes.c_longlong)]
    lib.pf_timing_get.restype = ip
    lib.pf_launch_count.argtypes = [vp]
    lib.pf_launch_count.restype = ctypes.c_longlong
    lib.pf_ms_residual_static.argtypes = [vp, vp, ctypes.c_longlong, ip, ctypes.POINTER(dp), vp]
    lib.pf_ms_residual_static.restype = ip
    lib.pf_fma_peak.argtypes = [ip, ctypes.POINTER(dp), vp]
    lib.pf_fma_peak.restype = ip
    lib.pf_strerror.argtypes = [ip]
    lib.pf_strerror.restype = ctypes.c_char_p
    _LIB = lib
    return lib


class PfError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load_library(False).pf_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")


def _check(code, where, allow=()):
    if code != PF_OK and code not in allow:
        raise PfError(code, where)
    return code


def config_default() -> PfConfig:
    c = PfConfig()
    load_library().pf_config_default(ctypes.byref(c))
    return c


def _ptr(a):
    """(pointer, keep-alive) for a numpy array, a torch tensor or None."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(a)
    return a.ctypes.data_as(ctypes.c_void_p), a


class Handle:
    """pf_create / pf_destroy around one handle; methods mirror the C calls.

    `cfg` is one PfConfig (pf_create with n_instances copies) or a list of
    them (pf_create_batch, one per instance; grain_R then is a list too)."""

    def __init__(self, cfg, n_instances: int = 1, grain_R=None):
        self.lib = load_library()
        cfgs = list(cfg) if isinstance(cfg, (list, tuple)) else [cfg]
        Rs = list(grain_R) if isinstance(cfg, (list, tuple)) and grain_R is not None else [grain_R] * len(cfgs)
        self._R = []
        for c, R in zip(cfgs, Rs):
            if R is not None:
                r = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(-1, 9))
                self._R.append(r)
                c.grain_R = r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                c.n_grains = r.shape[0]
        h = ctypes.c_void_p()
        if isinstance(cfg, (list, tuple)):
            arr = (PfConfig * len(cfgs))(*cfgs)
            self._arr = arr
            n_instances = len(cfgs)
            _check(self.lib.pf_create_batch(arr, n_instances, ctypes.byref(h)), "pf_create_batch")
        else:
            _check(self.lib.pf_create(ctypes.byref(cfg), n_instances, ctypes.byref(h)), "pf_create")
            cfgs = cfgs * n_instances
        self.h = h
        self.cfg = cfgs[0]
        self.cfgs = cfgs
        self.n_instances = n_instances
        self.dtype = np.float64 if cfgs[0].precision == PF_FP64 else np.float32
        self.Ns = [c.nx * c.ny * c.nz for c in cfgs]
        self.Vs = [c.n_variants for c in cfgs]
        self.N = self.Ns[0]
        self.V = self.Vs[0]

    def close(self):
        if getattr(self, "h", None):
            self.lib.pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, inst, f, eps_p=None, grain=None, eps0=None, mem=PF_MEM_HOST):
        if mem == PF_MEM_HOST:
            f = np.ascontiguousarray(f, dtype=self.dtype)
            eps_p = None if eps_p is None else np.ascontiguousarray(eps_p, dtype=self.dtype)
            grain = None if grain is None else np.ascontiguousarray(grain, dtype=np.uint16)
            eps0 = None if eps0 is None else np.ascontiguousarray(eps0, dtype=self.dtype)
        pf_, k1 = _ptr(f)
        pe, k2 = _ptr(eps_p)
        pg, k3 = _ptr(grain)
        p0, k4 = _ptr(eps0)
        _check(self.lib.pf_set_fields(self.h, inst, pf_, pe, pg, p0, mem), "pf_set_fields")

    def set_plastic_strain(self, inst, eps_p, mem=PF_MEM_HOST):
        if mem == PF_MEM_HOST and eps_p is not None:
            eps_p = np.ascontiguousarray(eps_p, dtype=self.dtype)
        pe, k = _ptr(eps_p)
        _check(self.lib.pf_set_plastic_strain(self.h, inst, pe, mem), "pf_set_plastic_strain")

    def set_mobility(self, inst, M, mem=PF_MEM_HOST):
        """Pad-layer mobility factor M [N] in [0, 1] (None removes it)."""
        if mem == PF_MEM_HOST and M is not None:
            M = np.ascontiguousarray(M, dtype=self.dtype)
        pm, k = _ptr(M)
        _check(self.lib.pf_set_mobility(self.h, inst, pm, mem), "pf_set_mobility")

    def get_fields(self, inst, f=None, eps=None, mem=PF_MEM_HOST, want_f=True, want_eps=True):
        """Host mode: returns (f [V][N], eps [6][N]) numpy arrays (None where
        not wanted); device mode fills the given tensors."""
        if mem == PF_MEM_HOST:
            f = np.empty((self.Vs[inst], self.Ns[inst]), dtype=self.dtype) if want_f else None
            eps = np.empty((6, self.Ns[inst]), dtype=self.dtype) if want_eps else None
        pf_, k1 = _ptr(f)
        pe, k2 = _ptr(eps)
        _check(self.lib.pf_get_fields(self.h, inst, pf_, pe, mem), "pf_get_fields")
        return f, eps

    def step(self, E, nsteps=None, allow=(PF_ENOCONV,)):
        """E: [n_instances][nsteps][6] (or [nsteps][6] for one instance)."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        if E.ndim == 1:
            E = E[None, None, :]
        elif E.ndim == 2:
            E = E[None]
        nsteps = E.shape[1] if nsteps is None else nsteps
        info = (PfStepInfo * self.n_instances)()
        code = self.lib.pf_step(self.h, nsteps, E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), info)
        _check(code, "pf_step", allow)
        return code, [info[i] for i in range(self.n_instances)]

    def stress(self, inst, field=True, out=None, mem=PF_MEM_HOST):
        mean = (ctypes.c_double * 6)()
        if field and mem == PF_MEM_HOST:
            out = np.empty((6, self.Ns[inst]), dtype=self.dtype)
        po, k = _ptr(out if field else None)
        _check(self.lib.pf_stress(self.h, inst, mean, po, mem), "pf_stress")
        return np.array(mean[:]), out

    def energy(self, inst):
        parts = (ctypes.c_double * 4)()
        _check(self.lib.pf_energy(self.h, inst, parts), "pf_energy")
        return np.array(parts[:])

    def timing(self, enable):
        _check(self.lib.pf_timing(self.h, 1 if enable else 0), "pf_timing")

    def timing_table(self):
        n = self.lib.pf_timing_get(self.h, 0, None, None, None)
        out = {}
        for k in range(n):
            name = ctypes.c_char_p()
            ms = ctypes.c_double()
            cnt = ctypes.c_longlong()
            _check(self.lib.pf_timing_get(self.h, k, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(cnt)),
                   "pf_timing_get")
            if cnt.value:
                out[name.value.decode()] = (ms.value, cnt.value)
        return out

    def launch_count(self):
        return int(self.lib.pf_launch_count(self.h))


def ms_residual_static(eps_new, eps_old, n_voxels, precision, stream=None):
    """pf_ms_residual_static on two device tensors [6][n]; returns (code, out[2])."""
    out = (ctypes.c_double * 2)()
    code = load_library().pf_ms_residual_static(ctypes.c_void_p(eps_new.data_ptr()),
                                                 ctypes.c_void_p(eps_old.data_ptr()), n_voxels, precision,
                                                 out, stream)
    return code, (out[0], out[1])


def fma_peak(kind, stream=None):
    """pf_fma_peak: measured multiply-add rate in flop/s (kind 0 FP32, 1 paired
    FP32, 2 FP64)."""
    out = ctypes.c_double()
    _check(load_library().pf_fma_peak(kind, ctypes.byref(out), stream), "pf_fma_peak")
    return out.value


def config_for(workload, precision=None, stream=None, ms_tol=None, ms_max_it=None, c0_mode=PF_C0_PER_STEP,
               twin_angle_deg=0.0, use_graph=0, load_dir=None, warm_degree=0, c2_nst=None,
               mob_corr=3, pic_iters=1, clamp=0, autotune=0, warm_points=0) -> PfConfig:
    """pf_config for an inputs.Workload; load_dir selects uniaxial loading along it,
    warm_degree (0..5) the extrapolated start of each step's passes (fitted by
    least squares to warm_points held solutions when warm_points > warm_degree + 1),
    c2_nst the anisotropic gradient coefficients (c2_n, c2_s, c2_t) of a single
    crystal."""
    c = config_default()
    nz, ny, nx = workload.shape
    c.nx, c.ny, c.nz = nx, ny, nz
    c.n_variants = workload.V
    for i, v in enumerate(workload.variant_ids):
        c.variant_ids[i] = v
    prec = precision or workload.precision
    c.precision = {"fp64": PF_FP64, "fp32": PF_FP32, "mixed": PF_MIXED}[prec]
    c.c1, c.c2, c.c3, c.dt = workload.c1, workload.c2, workload.c3, workload.dt
    c.gamma_tw = workload.gamma_tw
    c.c_over_a = workload.c_over_a
    c.twin_angle_deg = twin_angle_deg
    for i in range(5):
        c.C_hex[i] = workload.C_hex[i]
    c.twin_stiffness = workload.twin_stiffness
    c.ms_tol = workload.ms_tol if ms_tol is None else ms_tol
    c.ms_max_it = workload.ms_max_it if ms_max_it is None else ms_max_it
    c.c0_mode = c0_mode
    c.use_graph = use_graph
    c.n_grains = len(workload.grain_R)
    c.stream = stream
    c.warm_degree = warm_degree
    c.mob_corr = mob_corr
    c.pic_iters = pic_iters
    c.clamp = clamp
    c.autotune = autotune
    c.warm_points = warm_points
    if c2_nst is not None:
        for i in range(3):
            c.c2_aniso[i] = float(c2_nst[i])
    if load_dir is not None:
        c.load_mode = PF_LOAD_UNIAXIAL
        for i in range(3):
            c.load_dir[i] = float(load_dir[i])
    return c


def _set_workload(h, i, w):
    N = w.nvox
    h.set_fields(i, w.f.reshape(w.V, N), None if w.eps_p is None else w.eps_p.reshape(6, N),
                 None if w.grain is None else w.grain.reshape(N))
    if getattr(w, "mobility", None) is not None:
        h.set_mobility(i, w.mobility.reshape(N))


def handle_for(workload, **kw) -> Handle:
    """Create a handle for a workload and set its fields from host memory."""
    cfg = config_for(workload, **kw)
    h = Handle(cfg, 1, grain_R=workload.grain_R)
    _set_workload(h, 0, workload)
    return h


def handle_for_device(workload, precision, kw, f, eps_p=None, grain=None) -> Handle:
    """A handle for a workload whose fields are already device tensors."""
    cfg = config_for(workload, precision=precision, **kw)
    h = Handle(cfg, 1, grain_R=workload.grain_R)
    h.set_fields(0, f, eps_p, grain, None, mem=PF_MEM_DEVICE)
    return h


def batch_handle_for(workloads, **kw) -> Handle:
    """One pf_create_batch handle over several workloads (grids may differ)."""
    cfgs = [config_for(w, **kw) for w in workloads]
    h = Handle(cfgs, grain_R=[w.grain_R for w in workloads])
    for i, w in enumerate(workloads):
        _set_workload(h, i, w)
    return h
