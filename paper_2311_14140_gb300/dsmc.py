"""ctypes binding of the sm_103a DSMC library (``include/dsmc.h``).

Argument marshalling only: every step of the DSMC runs in the library's CUDA
kernels.  PyTorch, when present, provides the device workspace (a uint8 tensor) and
the CUDA stream (the current stream); without it the library allocates its own
memory and uses the legacy default stream.  There is no CPU path: if the library is
missing, loading raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdsmc.so")
NMOM = 13

DSMC_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
          4: "device limit reached", 5: "invalid state"}


class DsmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Gas(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("d_ref", ctypes.c_double),
                ("omega", ctypes.c_double), ("T_ref", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("dt_factor", ctypes.c_double), ("dt", ctypes.c_double),
                ("sample_start", ctypes.c_longlong), ("group_size", ctypes.c_int),
                ("collisions", ctypes.c_int), ("profile", ctypes.c_int),
                ("span_particles", ctypes.c_int), ("cta_warps", ctypes.c_int),
                ("span_rows", ctypes.c_int), ("graph", ctypes.c_int),
                ("accum", ctypes.c_int), ("stream", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_longlong), ("n_cells", ctypes.c_int),
                ("ppc", ctypes.c_int), ("step", ctypes.c_longlong),
                ("n_samples", ctypes.c_longlong), ("Kn", ctypes.c_double),
                ("omega", ctypes.c_double), ("body_force", ctypes.c_double),
                ("nsigma", ctypes.c_double), ("dt", ctypes.c_double),
                ("dt_f", ctypes.c_float), ("F_f", ctypes.c_float), ("coef", ctypes.c_float),
                ("cvhs", ctypes.c_float), ("vexp", ctypes.c_float), ("vinv", ctypes.c_float), ("lncv", ctypes.c_float),
                ("smax0", ctypes.c_float), ("device_bytes", ctypes.c_size_t),
                ("n_instances", ctypes.c_int), ("span_particles", ctypes.c_int),
                ("cta_warps", ctypes.c_int), ("span_rows", ctypes.c_int),
                ("cells_per_span", ctypes.c_int), ("n_spans", ctypes.c_int),
                ("total_spans", ctypes.c_int), ("first_slot", ctypes.c_int),
                ("first_cell", ctypes.c_int)]


class Instance(ctypes.Structure):
    _fields_ = [("gas", Gas), ("Kn", ctypes.c_double), ("wall_T", ctypes.c_double),
                ("body_force", ctypes.c_double), ("n_cells", ctypes.c_int),
                ("ppc", ctypes.c_int), ("seed", ctypes.c_uint64)]


class PoolLimits(ctypes.Structure):
    _fields_ = [("max_particles", ctypes.c_longlong), ("max_cells", ctypes.c_int),
                ("max_instances", ctypes.c_int), ("max_cells_per_instance", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("instance", Instance), ("arrival", ctypes.c_double),
                ("target_se", ctypes.c_double), ("max_steps", ctypes.c_longlong)]


class ServeOptions(ctypes.Structure):
    _fields_ = [("epoch_steps", ctypes.c_int), ("batches", ctypes.c_int),
                ("max_active", ctypes.c_int), ("time_limit", ctypes.c_double)]


class RequestResult(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_double), ("finished", ctypes.c_double),
                ("steps", ctypes.c_longlong), ("u_mean", ctypes.c_double),
                ("u_se", ctypes.c_double), ("count", ctypes.c_double),
                ("sum_vx", ctypes.c_double), ("converged", ctypes.c_int), ("id", ctypes.c_int)]


class SurrogateFit(ctypes.Structure):
    D = ctypes.c_double
    _fields_ = [("n_samples", ctypes.c_longlong), ("n_v", D), ("n_c", D),
                ("log_evidence_v", D * 2), ("prob_v", D * 2), ("alpha_v", D * 2),
                ("beta_v", D * 2), ("sigma_p", D), ("sigma_p_var", D),
                ("iterations_v", ctypes.c_int), ("log_evidence_c", D * 4), ("prob_c", D * 4),
                ("alpha_c", D * 4), ("beta_c", D * 4), ("m_c", (D * 3) * 4),
                ("S_c", (D * 9) * 4), ("iterations_c", ctypes.c_int * 4),
                ("sel_v", ctypes.c_int), ("sel_c", ctypes.c_int), ("b", D * 3)]


MMS_MAX_ITER = 64


class MmsParams(ctypes.Structure):
    _fields_ = [("gas", Gas), ("Kn", ctypes.c_double), ("body_force", ctypes.c_double),
                ("wall_T", ctypes.c_double), ("dy", ctypes.c_double), ("ppc", ctypes.c_int),
                ("buffer", ctypes.c_int), ("iterations", ctypes.c_int), ("steps", ctypes.c_int),
                ("window", ctypes.c_int), ("warmup", ctypes.c_int), ("n_cfd", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("group_size", ctypes.c_int)]


class MmsResult(ctypes.Structure):
    _fields_ = [("n_train", ctypes.c_int), ("n_sub", ctypes.c_int), ("L_d", ctypes.c_double),
                ("b", ctypes.c_double * 3), ("iterations_done", ctypes.c_int),
                ("u_interface", ctypes.c_double * MMS_MAX_ITER),
                ("p_interface", ctypes.c_double * MMS_MAX_ITER),
                ("samples", ctypes.c_longlong), ("fit", SurrogateFit)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load ``libdsmc.so`` and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    L = ctypes.CDLL(path)
    c = ctypes
    H = c.c_void_p
    st = c.c_int
    sig = {
        "dsmc_default_options": (st, [c.POINTER(Options)]),
        "dsmc_workspace_bytes": (c.c_size_t, [c.c_int, c.c_int]),
        "dsmc_create": (st, [c.POINTER(Gas), c.c_double, c.c_double, c.c_double, c.c_int,
                             c.c_int, c.c_uint64, c.POINTER(H)]),
        "dsmc_create_in": (st, [c.POINTER(Gas), c.c_double, c.c_double, c.c_double, c.c_int,
                                c.c_int, c.c_uint64, c.POINTER(Options), c.c_void_p,
                                c.c_size_t, c.POINTER(H)]),
        "dsmc_set_options": (st, [H, c.POINTER(Options)]),
        "dsmc_step": (st, [H, c.c_int]),
        "dsmc_sync": (st, [H]),
        "dsmc_sample_moments": (st, [H, c.c_void_p, c.POINTER(c.c_longlong)]),
        "dsmc_cell_fields": (st, [c.c_void_p, c.c_longlong, c.c_int, c.c_int, c.c_void_p]),
        "dsmc_cell_fields_of": (st, [H, c.c_int, c.c_void_p]),
        "dsmc_reset_samples": (st, [H]),
        "dsmc_copy_state": (st, [H, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]),
        "dsmc_copy_cells": (st, [H, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]),
        "dsmc_load_state": (st, [H, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p,
                                 c.c_void_p, c.c_longlong]),
        "dsmc_get_info": (st, [H, c.POINTER(Info)]),
        "dsmc_batch_workspace_bytes": (c.c_size_t, [c.POINTER(Instance), c.c_int]),
        "dsmc_create_batch": (st, [c.POINTER(Instance), c.c_int, c.POINTER(Options), c.c_void_p,
                                   c.c_size_t, c.POINTER(H)]),
        "dsmc_batch_size": (c.c_int, [H]),
        "dsmc_sample_moments_of": (st, [H, c.c_int, c.c_void_p, c.POINTER(c.c_longlong)]),
        "dsmc_sample_moments_all": (st, [H, c.c_void_p, c.c_void_p]),
        "dsmc_reset_samples_of": (st, [H, c.c_int]),
        "dsmc_copy_state_of": (st, [H, c.c_int, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]),
        "dsmc_copy_cells_of": (st, [H, c.c_int, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]),
        "dsmc_load_state_of": (st, [H, c.c_int, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p,
                                    c.c_void_p, c.c_longlong]),
        "dsmc_get_info_of": (st, [H, c.c_int, c.POINTER(Info)]),
        "dsmc_autotune": (st, [H, c.c_int, c.POINTER(c.c_int), c.POINTER(c.c_double)]),
        "dsmc_sort_cells_static": (st, [c.c_void_p] * 9 + [c.c_int, c.c_int, c.c_void_p]),
        "dsmc_id_bound": (c.c_int, [H]),
        "dsmc_channel_sums": (st, [H, c.c_void_p]),
        "dsmc_pool_workspace_bytes": (c.c_size_t, [c.POINTER(PoolLimits)]),
        "dsmc_pool_create": (st, [c.POINTER(PoolLimits), c.POINTER(Options), c.c_void_p,
                                  c.c_size_t, c.POINTER(H)]),
        "dsmc_pool_add": (st, [H, c.POINTER(Instance), c.POINTER(c.c_int)]),
        "dsmc_pool_remove": (st, [H, c.c_int]),
        "dsmc_default_serve_options": (st, [c.POINTER(ServeOptions)]),
        "dsmc_serve": (st, [H, c.POINTER(Request), c.c_int, c.POINTER(ServeOptions),
                            c.POINTER(RequestResult)]),
        "dsmc_solve": (st, [c.POINTER(Request), c.POINTER(Options), c.POINTER(ServeOptions),
                            c.POINTER(RequestResult)]),
        "dsmc_device_moments_of": (st, [H, c.c_int, c.POINTER(c.c_void_p)]),
        "dsmc_set_open_top": (st, [H, c.c_int, c.c_double, c.c_double]),
        "dsmc_gp_fit": (st, [c.c_void_p, c.c_void_p, c.c_int, c.c_int, c.c_void_p, c.c_int,
                             c.c_void_p, c.POINTER(H), c.c_void_p, c.POINTER(c.c_int)]),
        "dsmc_gp_predict": (st, [H, c.c_void_p, c.c_int, c.c_void_p]),
        "dsmc_gp_hyper": (st, [H, c.POINTER(c.c_double), c.POINTER(c.c_double),
                               c.POINTER(c.c_double)]),
        "dsmc_gp_destroy": (st, [H]),
        "dsmc_surrogate_correction": (st, [c.POINTER(SurrogateFit), c.c_int, c.c_void_p,
                                           c.c_void_p]),
        "dsmc_cfd_faces": (st, [c.c_double, c.c_double, c.c_int, c.c_int, c.c_double,
                                c.c_void_p, c.c_void_p, c.c_void_p]),
        "dsmc_surrogate_create_region": (st, [c.c_double, c.c_double, c.c_int, c.c_int,
                                              c.c_double, c.c_int, c.c_void_p, c.c_void_p,
                                              c.POINTER(H)]),
        "dsmc_default_mms_params": (st, [c.POINTER(MmsParams)]),
        "dsmc_mms_run": (st, [c.POINTER(MmsParams), c.c_void_p, c.c_void_p, c.c_void_p, c.c_int,
                              c.c_void_p, c.POINTER(MmsResult)]),
        "dsmc_surrogate_exponents": (st, [c.c_double, c.c_void_p]),
        "dsmc_surrogate_create": (st, [c.c_double, c.c_double, c.c_int, c.c_int, c.c_void_p,
                                       c.c_void_p, c.POINTER(H)]),
        "dsmc_surrogate_destroy": (st, [H]),
        "dsmc_surrogate_reset": (st, [H]),
        "dsmc_surrogate_add_window": (st, [H, c.c_void_p, c.c_longlong]),
        "dsmc_surrogate_add_run": (st, [H, H, c.c_int]),
        "dsmc_surrogate_train": (st, [H, c.POINTER(SurrogateFit)]),
        "dsmc_surrogate_profile": (st, [H, c.POINTER(SurrogateFit), c.c_int, c.c_void_p, c.c_int,
                                        c.c_void_p, c.c_void_p]),
        "dsmc_kernel_count": (c.c_int, []),
        "dsmc_kernel_name": (c.c_char_p, [c.c_int]),
        "dsmc_kernel_times": (st, [H, c.c_void_p, c.c_void_p]),
        "dsmc_reset_kernel_times": (st, [H]),
        "dsmc_destroy": (st, [H]),
        "dsmc_last_error": (c.c_char_p, []),
        "dsmc_status_string": (c.c_char_p, [c.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int) -> None:
    if status != DSMC_OK:
        raise DsmcError(status, load_library().dsmc_last_error().decode())


def _ptr(a) -> Optional[int]:
    """Address of a contiguous numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def default_options() -> Options:
    o = Options()
    _check(load_library().dsmc_default_options(ctypes.byref(o)))
    return o


# Argon: mass, VHS reference diameter (Bird's table) and reference temperature.
ARGON = dict(mass=6.63e-26, d_ref=4.17e-10, T_ref=273.0)


class Dsmc:
    """One DSMC run on the current CUDA device (see ``include/dsmc.h``).

    ``workspace``: "torch" (a torch uint8 tensor on the device owns the memory; the
    current torch stream is used unless ``stream`` is given) or "library" (the
    library calls cudaMalloc).
    """

    def __init__(self, Kn: float, n_cells: int, ppc: int, *, omega: float = 0.5,
                 body_force: float = 0.0, seed: int = 0, wall_T: float = 273.0,
                 dt_factor: float = 0.2, dt: float = 0.0, sample_start: int = 0,
                 group_size: int = 256, collisions: bool = True, profile: bool = False,
                 span_particles: int = 0, cta_warps: int = 0, span_rows: int = 0,
                 graph: bool = False, accum: int = 0, stream=None, workspace: str = "torch",
                 gas: Optional[dict] = None):
        L = load_library()
        self._lib = L
        self.n_cells, self.ppc = int(n_cells), int(ppc)
        self.N = self.n_cells * self.ppc
        g = dict(ARGON)
        g.update(gas or {})
        self._gas = Gas(g["mass"], g["d_ref"], float(omega), g["T_ref"])
        o = default_options()
        o.dt_factor, o.dt, o.sample_start = float(dt_factor), float(dt), int(sample_start)
        o.group_size, o.collisions, o.profile = int(group_size), int(bool(collisions)), int(bool(profile))
        o.span_particles, o.cta_warps, o.graph = int(span_particles), int(cta_warps), int(bool(graph))
        o.span_rows, o.accum = int(span_rows), int(accum)
        self._ws = None
        if workspace == "torch":
            import torch
            nbytes = L.dsmc_workspace_bytes(self.n_cells, self.ppc)
            self._ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            ws_ptr, ws_bytes = self._ws.data_ptr(), nbytes
        elif workspace == "library":
            ws_ptr, ws_bytes = None, 0
        else:
            raise ValueError("workspace must be 'torch' or 'library'")
        o.stream = int(stream) if stream is not None else None
        self._opt = o
        h = ctypes.c_void_p()
        _check(L.dsmc_create_in(ctypes.byref(self._gas), float(Kn), float(wall_T),
                                float(body_force), self.n_cells, self.ppc,
                                int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o), ws_ptr,
                                ws_bytes, ctypes.byref(h)))
        self._h = h

    # lifetime -------------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.dsmc_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # stepping -------------------------------------------------------------------
    def step(self, n: int = 1) -> None:
        _check(self._lib.dsmc_step(self._h, int(n)))

    def sync(self) -> None:
        _check(self._lib.dsmc_sync(self._h))

    def set_options(self, **kw) -> None:
        o = Options.from_buffer_copy(self._opt)
        for k, v in kw.items():
            if k == "stream":
                v = int(v) if v is not None else None
            setattr(o, k, v)
        _check(self._lib.dsmc_set_options(self._h, ctypes.byref(o)))
        self._opt = o

    # outputs --------------------------------------------------------------------
    def moments(self, out=None):
        """(raw sums [n_cells, 13] float64, sampled steps); ``out`` may be a pinned or
        device buffer of that shape."""
        if out is None:
            out = np.empty((self.n_cells, NMOM), np.float64)
        ns = ctypes.c_longlong()
        _check(self._lib.dsmc_sample_moments(self._h, _ptr(out), ctypes.byref(ns)))
        return out, int(ns.value)

    def reset_samples(self) -> None:
        _check(self._lib.dsmc_reset_samples(self._h))

    def fields(self) -> dict:
        """Cell fields of the samples so far, computed by the library on the device
        (see ``fields``)."""
        out = np.empty((self.n_cells, NFIELD), np.float64)
        _check(self._lib.dsmc_cell_fields_of(self._h, 0, _ptr(out)))
        return _field_dict(out)

    def state(self):
        arrs = [np.empty(self.N, np.float32) for _ in range(4)]
        _check(self._lib.dsmc_copy_state(self._h, *[_ptr(a) for a in arrs]))
        return tuple(arrs)

    def state_into(self, y=None, vx=None, vy=None, vz=None) -> None:
        _check(self._lib.dsmc_copy_state(self._h, _ptr(y), _ptr(vx), _ptr(vy), _ptr(vz)))

    def set_open_top(self, u: float, P: float) -> None:
        """Makes y = 1 an open Chapman-Enskog interface (velocity u, stress P)."""
        _check(self._lib.dsmc_set_open_top(self._h, 0, float(u), float(P)))

    def device_moments(self) -> int:
        """Device address of the moment sums (n_cells x 13 binary64)."""
        p = ctypes.c_void_p()
        _check(self._lib.dsmc_device_moments_of(self._h, 0, ctypes.byref(p)))
        return p.value

    def cells(self):
        off = np.empty(self.n_cells + 1, np.int32)
        smax = np.empty(self.n_cells, np.float32)
        nc = np.empty(self.n_cells, np.uint64)
        na = np.empty(self.n_cells, np.uint64)
        _check(self._lib.dsmc_copy_cells(self._h, _ptr(off), _ptr(smax), _ptr(nc), _ptr(na)))
        return off, smax, nc, na

    def load_state(self, y, vx, vy, vz, smax=None, step: int = 0) -> None:
        arrs = [np.ascontiguousarray(a, np.float32) if isinstance(a, np.ndarray) else a
                for a in (y, vx, vy, vz)]
        sm = None if smax is None else np.ascontiguousarray(smax, np.float32)
        _check(self._lib.dsmc_load_state(self._h, *[_ptr(a) for a in arrs], _ptr(sm),
                                         int(step)))

    def info(self) -> dict:
        i = Info()
        _check(self._lib.dsmc_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}

    def kernel_times(self) -> dict:
        n = self._lib.dsmc_kernel_count()
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.int64)
        _check(self._lib.dsmc_kernel_times(self._h, _ptr(ms), _ptr(cnt)))
        return {self._lib.dsmc_kernel_name(k).decode(): (float(ms[k]), int(cnt[k]))
                for k in range(n)}

    def reset_kernel_times(self) -> None:
        _check(self._lib.dsmc_reset_kernel_times(self._h))


def make_instance(Kn: float, n_cells: int, ppc: int, *, omega: float = 0.5,
                  body_force: float = 0.0, seed: int = 0, wall_T: float = 273.0,
                  gas: Optional[dict] = None) -> Instance:
    g = dict(ARGON)
    g.update(gas or {})
    return Instance(Gas(g["mass"], g["d_ref"], float(omega), g["T_ref"]), float(Kn),
                    float(wall_T), float(body_force), int(n_cells), int(ppc),
                    int(seed) & 0xFFFFFFFFFFFFFFFF)


def _options(dt_factor=0.2, dt=0.0, sample_start=0, group_size=256, collisions=True,
             profile=False, span_particles=0, cta_warps=0, span_rows=0, graph=False,
             accum=0) -> Options:
    o = default_options()
    o.dt_factor, o.dt, o.sample_start = float(dt_factor), float(dt), int(sample_start)
    o.group_size, o.collisions, o.profile = int(group_size), int(bool(collisions)), int(bool(profile))
    o.span_particles, o.cta_warps, o.graph = int(span_particles), int(cta_warps), int(bool(graph))
    o.span_rows, o.accum = int(span_rows), int(accum)
    return o


class _Multi:
    """Accessors of a handle with several instances, by instance id."""

    _lib = None
    _h = None
    _opt = None
    _ws = None

    def _alloc(self, workspace: str, nbytes: int, stream):
        """(workspace pointer, bytes, stream) for a torch-owned or library-owned handle."""
        if workspace == "torch":
            import torch
            if nbytes == 0:
                raise DsmcError(1, "invalid sizes")
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            return self._ws.data_ptr(), nbytes, stream
        if workspace == "library":
            return None, 0, stream
        raise ValueError("workspace must be 'torch' or 'library'")

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.dsmc_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n: int = 1) -> None:
        _check(self._lib.dsmc_step(self._h, int(n)))

    def sync(self) -> None:
        _check(self._lib.dsmc_sync(self._h))

    def set_options(self, **kw) -> None:
        o = Options.from_buffer_copy(self._opt)
        for k, v in kw.items():
            if k == "stream":
                v = int(v) if v is not None else None
            setattr(o, k, v)
        _check(self._lib.dsmc_set_options(self._h, ctypes.byref(o)))
        self._opt = o

    def autotune(self, steps_per_trial: int = 4):
        best = ctypes.c_int()
        ms = ctypes.c_double()
        _check(self._lib.dsmc_autotune(self._h, int(steps_per_trial), ctypes.byref(best),
                                       ctypes.byref(ms)))
        self._opt.span_particles = best.value
        inf = self.info(self._first_id())
        self._opt.cta_warps = inf["cta_warps"]
        self._opt.span_rows = inf["span_rows"]
        return best.value, ms.value

    def _first_id(self) -> int:
        for i in range(max(1, self._lib.dsmc_id_bound(self._h))):
            try:
                self.info(i)
                return i
            except DsmcError:
                continue
        return 0

    def size(self) -> int:
        return self._lib.dsmc_batch_size(self._h)

    def set_open_top(self, i: int, u: float, P: float) -> None:
        _check(self._lib.dsmc_set_open_top(self._h, int(i), float(u), float(P)))

    def moments(self, i: int, out=None):
        if out is None:
            out = np.empty((self.info(i)["n_cells"], NMOM), np.float64)
        ns = ctypes.c_longlong()
        _check(self._lib.dsmc_sample_moments_of(self._h, int(i), _ptr(out), ctypes.byref(ns)))
        return out, int(ns.value)

    def fields(self, i: int) -> dict:
        """Cell fields of instance i's samples (``dsmc_cell_fields_of``)."""
        out = np.empty((self.info(i)["n_cells"], NFIELD), np.float64)
        _check(self._lib.dsmc_cell_fields_of(self._h, int(i), _ptr(out)))
        return _field_dict(out)

    def channel_sums(self):
        """[id bound, 2]: sampled particle count and sum of vx per instance id."""
        out = np.zeros((max(1, self._lib.dsmc_id_bound(self._h)), 2), np.float64)
        _check(self._lib.dsmc_channel_sums(self._h, _ptr(out)))
        return out

    def reset_samples(self, i: Optional[int] = None) -> None:
        if i is None:
            _check(self._lib.dsmc_reset_samples(self._h))
        else:
            _check(self._lib.dsmc_reset_samples_of(self._h, int(i)))

    def state(self, i: int):
        n = self.info(i)["n_particles"]
        arrs = [np.empty(n, np.float32) for _ in range(4)]
        _check(self._lib.dsmc_copy_state_of(self._h, int(i), *[_ptr(a) for a in arrs]))
        return tuple(arrs)

    def cells(self, i: int):
        nc = self.info(i)["n_cells"]
        off = np.empty(nc + 1, np.int32)
        smax = np.empty(nc, np.float32)
        cand = np.empty(nc, np.uint64)
        acc = np.empty(nc, np.uint64)
        _check(self._lib.dsmc_copy_cells_of(self._h, int(i), _ptr(off), _ptr(smax), _ptr(cand),
                                            _ptr(acc)))
        return off, smax, cand, acc

    def load_state(self, i: int, y, vx, vy, vz, smax=None, step: int = 0) -> None:
        arrs = [np.ascontiguousarray(a, np.float32) if isinstance(a, np.ndarray) else a
                for a in (y, vx, vy, vz)]
        sm = None if smax is None else np.ascontiguousarray(smax, np.float32)
        _check(self._lib.dsmc_load_state_of(self._h, int(i), *[_ptr(a) for a in arrs],
                                            _ptr(sm), int(step)))

    def info(self, i: int = 0) -> dict:
        inf = Info()
        _check(self._lib.dsmc_get_info_of(self._h, int(i), ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    def kernel_times(self) -> dict:
        n = self._lib.dsmc_kernel_count()
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.int64)
        _check(self._lib.dsmc_kernel_times(self._h, _ptr(ms), _ptr(cnt)))
        return {self._lib.dsmc_kernel_name(k).decode(): (float(ms[k]), int(cnt[k]))
                for k in range(n)}

    def reset_kernel_times(self) -> None:
        _check(self._lib.dsmc_reset_kernel_times(self._h))


class DsmcBatch(_Multi):
    """Many independent DSMC runs advanced by the same launches (``dsmc_create_batch``).

    ``instances``: a sequence of dicts with the keyword arguments of ``make_instance``
    (Kn, n_cells, ppc, omega, body_force, seed, wall_T).  Options are shared.  Instance
    i evolves exactly as ``Dsmc(**instances[i], ...)`` with the same options.
    """

    def __init__(self, instances, *, stream=None, workspace: str = "torch", **opts):
        L = load_library()
        self._lib = L
        self._defs = [dict(d) for d in instances]
        arr = (Instance * len(self._defs))(*[make_instance(**d) for d in self._defs])
        self.n = len(self._defs)
        self.n_cells = [int(d["n_cells"]) for d in self._defs]
        self.ppc = [int(d["ppc"]) for d in self._defs]
        self.cell_base = np.concatenate([[0], np.cumsum(self.n_cells)]).astype(np.int64)
        o = _options(**opts)
        ws_ptr, ws_bytes, stream = self._alloc(
            workspace, L.dsmc_batch_workspace_bytes(arr, self.n) if workspace == "torch" else 0,
            stream)
        o.stream = int(stream) if stream is not None else None
        self._opt = o
        h = ctypes.c_void_p()
        _check(L.dsmc_create_batch(arr, self.n, ctypes.byref(o), ws_ptr, ws_bytes,
                                   ctypes.byref(h)))
        self._h = h

    def moments_all(self, out=None):
        """(raw sums [sum n_cells, 13], sampled steps per instance); rows of instance i
        are ``cell_base[i]:cell_base[i+1]``."""
        if out is None:
            out = np.empty((int(self.cell_base[-1]), NMOM), np.float64)
        ns = np.empty(self.n, np.int64)
        _check(self._lib.dsmc_sample_moments_all(self._h, _ptr(out), _ptr(ns)))
        return out, ns


class DsmcPool(_Multi):
    """A handle whose instances come and go (``dsmc_pool_create``): continuous batching."""

    def __init__(self, max_particles: int, max_cells: int, max_instances: int,
                 max_cells_per_instance: int, *, stream=None, workspace: str = "torch",
                 **opts):
        L = load_library()
        self._lib = L
        self.limits = PoolLimits(int(max_particles), int(max_cells), int(max_instances),
                                 int(max_cells_per_instance))
        o = _options(**opts)
        ws_ptr, ws_bytes, stream = self._alloc(
            workspace,
            L.dsmc_pool_workspace_bytes(ctypes.byref(self.limits)) if workspace == "torch" else 0,
            stream)
        o.stream = int(stream) if stream is not None else None
        self._opt = o
        h = ctypes.c_void_p()
        _check(L.dsmc_pool_create(ctypes.byref(self.limits), ctypes.byref(o), ws_ptr, ws_bytes,
                                  ctypes.byref(h)))
        self._h = h

    def add(self, **instance) -> int:
        """Adds a run (keyword arguments of ``make_instance``); returns its id.  Raises
        DsmcError (status 2) when the pool has no room."""
        inst = make_instance(**instance)
        i = ctypes.c_int(-1)
        _check(self._lib.dsmc_pool_add(self._h, ctypes.byref(inst), ctypes.byref(i)))
        return i.value

    def remove(self, i: int) -> None:
        _check(self._lib.dsmc_pool_remove(self._h, int(i)))

    def serve(self, requests, *, epoch_steps: int = 32, batches: int = 16, max_active: int = 0,
              time_limit: float = 0.0):
        """Runs ``dsmc_serve`` over ``requests`` (a sequence of dicts with ``arrival``,
        ``target_se``, ``max_steps`` and the keyword arguments of ``make_instance``);
        returns one dict per request."""
        arr = (Request * len(requests))()
        for k, r in enumerate(requests):
            inst = {x: r[x] for x in r if x not in ("arrival", "target_se", "max_steps")}
            arr[k] = Request(make_instance(**inst), float(r["arrival"]), float(r["target_se"]),
                             int(r["max_steps"]))
        so = serve_options(epoch_steps=epoch_steps, batches=batches, max_active=max_active,
                           time_limit=time_limit)
        res = (RequestResult * len(requests))()
        _check(self._lib.dsmc_serve(self._h, arr, len(requests), ctypes.byref(so), res))
        return [{k: getattr(x, k) for k, _ in RequestResult._fields_} for x in res]


def serve_options(**kw) -> ServeOptions:
    so = ServeOptions()
    _check(load_library().dsmc_default_serve_options(ctypes.byref(so)))
    for k, v in kw.items():
        setattr(so, k, v)
    return so


def solve(request: dict, *, epoch_steps: int = 32, batches: int = 16, stream=None,
          **opts) -> dict:
    """One request as a plain run of its own (``dsmc_solve``) on ``stream`` (a
    cudaStream_t as an integer; None: the legacy default stream)."""
    inst = {x: request[x] for x in request if x not in ("arrival", "target_se", "max_steps")}
    r = Request(make_instance(**inst), float(request.get("arrival", 0.0)),
                float(request["target_se"]), int(request["max_steps"]))
    o = _options(**opts)
    o.stream = int(stream) if stream is not None else None
    so = serve_options(epoch_steps=epoch_steps, batches=batches)
    res = RequestResult()
    _check(load_library().dsmc_solve(ctypes.byref(r), ctypes.byref(o), ctypes.byref(so),
                                      ctypes.byref(res)))
    return {k: getattr(res, k) for k, _ in RequestResult._fields_}


def _fit_dict(f: SurrogateFit) -> dict:
    out = {}
    for k, _ in SurrogateFit._fields_:
        v = getattr(f, k)
        if isinstance(v, ctypes.Array):
            v = np.ctypeslib.as_array(v).copy()
        out[k] = v
    out["_raw"] = SurrogateFit.from_buffer_copy(f)
    return out


class Surrogate:
    """The surrogate stage (``dsmc_surrogate_*``): training samples from windows of
    moment sums, model fitting and selection, Monte Carlo bands of the corrected
    macroscopic profile."""

    def __init__(self, Kn: float, F: float, n_cells: int, ppc: int, b=None, stream=None,
                 length: float = 1.0, n_train: int = 0):
        """length < 1: runs covering the Knudsen layer [0, length] of the channel, training
        cells 1 .. n_train - 1 (``dsmc_surrogate_create_region``)."""
        L = load_library()
        self._lib = L
        self.n_cells = int(n_cells)
        bb = None if b is None else np.ascontiguousarray(b, np.float64)
        h = ctypes.c_void_p()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = None
        sp = int(stream) if stream else None
        if length == 1.0:
            _check(L.dsmc_surrogate_create(float(Kn), float(F), self.n_cells, int(ppc), _ptr(bb),
                                           sp, ctypes.byref(h)))
        else:
            _check(L.dsmc_surrogate_create_region(float(Kn), float(F), self.n_cells, int(ppc),
                                                  float(length), int(n_train), _ptr(bb), sp,
                                                  ctypes.byref(h)))
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.dsmc_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self) -> None:
        _check(self._lib.dsmc_surrogate_reset(self._h))

    def add_window(self, acc, n_steps: int) -> None:
        a = np.ascontiguousarray(acc, np.float64) if isinstance(acc, np.ndarray) else acc
        _check(self._lib.dsmc_surrogate_add_window(self._h, _ptr(a), int(n_steps)))

    def add_run(self, run, i: int = 0) -> None:
        """One sample from what run (Dsmc, DsmcBatch or DsmcPool) instance i has sampled
        since its last reset; resets it."""
        _check(self._lib.dsmc_surrogate_add_run(self._h, run._h, int(i)))

    def train(self) -> dict:
        f = SurrogateFit()
        _check(self._lib.dsmc_surrogate_train(self._h, ctypes.byref(f)))
        return _fit_dict(f)

    def profile(self, n_cfd: int, z, fit: Optional[dict] = None):
        zz = np.ascontiguousarray(z, np.float64)
        assert zz.ndim == 2 and zz.shape[1] == 4
        mean = np.empty(int(n_cfd), np.float64)
        sd = np.empty(int(n_cfd), np.float64)
        fp = ctypes.byref(fit["_raw"]) if fit is not None else None
        _check(self._lib.dsmc_surrogate_profile(self._h, fp, int(n_cfd), _ptr(zz), zz.shape[0],
                                                _ptr(mean), _ptr(sd)))
        return mean, sd


def mms_hybrid(Kn: float, F: float, *, omega: float = 0.5, dy: float = 0.005, ppc: int = 50,
               buffer: int = 5, iterations: int = 5, steps: int = 2000, window: int = 100,
               warmup: int = 1000, n_cfd: int = 200, seed: int = 0, group_size: int = 256,
               z=None, stream=None) -> dict:
    """The MMS hybrid (``dsmc_mms_run``): returns the final CFD profile, its Monte Carlo
    standard deviation (when z, n_trials x 4 standard normals, is given), the interface
    history and the last fit."""
    L = load_library()
    p = MmsParams()
    _check(L.dsmc_default_mms_params(ctypes.byref(p)))
    p.gas.omega = float(omega)
    p.Kn, p.body_force, p.dy, p.ppc, p.buffer = float(Kn), float(F), float(dy), int(ppc), int(buffer)
    p.iterations, p.steps, p.window, p.warmup = int(iterations), int(steps), int(window), int(warmup)
    p.n_cfd, p.seed, p.group_size = int(n_cfd), int(seed) & 0xFFFFFFFFFFFFFFFF, int(group_size)
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except Exception:
            stream = None
    prof = np.empty(int(n_cfd), np.float64)
    zz = None if z is None else np.ascontiguousarray(z, np.float64)
    sd = None if z is None else np.empty(int(n_cfd), np.float64)
    r = MmsResult()
    _check(L.dsmc_mms_run(ctypes.byref(p), int(stream) if stream else None, _ptr(prof),
                          _ptr(zz), 0 if zz is None else zz.shape[0], _ptr(sd), ctypes.byref(r)))
    k = r.iterations_done
    return {"profile": prof, "band_sd": sd, "n_train": r.n_train, "n_sub": r.n_sub,
            "L_d": r.L_d, "b": tuple(r.b), "samples": r.samples,
            "interface": [(r.u_interface[i], r.p_interface[i]) for i in range(k)],
            "fit": _fit_dict(r.fit)}


def _default_stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except Exception:
            stream = None
    return int(stream) if stream else None


class GaussianProcess:
    """GP regression on the device (``dsmc_gp_*``): the GP variant of the surrogate stage
    (not the paper's method).  X: (n, 2) inputs on the unit square; Y: (n, m) outputs; grid:
    sequence of (l1, l2, s2)."""

    def __init__(self, X, Y, grid, stream=None):
        L = load_library()
        self._lib = L
        X = np.ascontiguousarray(X, np.float64)
        Y = np.ascontiguousarray(Y, np.float64)
        if Y.ndim == 1:
            Y = Y[:, None].copy()
        g = np.ascontiguousarray(np.asarray(grid, np.float64).reshape(-1, 3))
        self.m = Y.shape[1]
        self.lml = np.empty(len(g), np.float64)
        best = ctypes.c_int()
        h = ctypes.c_void_p()
        _check(L.dsmc_gp_fit(_ptr(X), _ptr(Y), X.shape[0], self.m, _ptr(g), len(g),
                             _default_stream(stream), ctypes.byref(h), _ptr(self.lml),
                             ctypes.byref(best)))
        self._h = h
        self.best = best.value
        v = [ctypes.c_double() for _ in range(3)]
        _check(L.dsmc_gp_hyper(h, *[ctypes.byref(x) for x in v]))
        self.hyper = tuple(x.value for x in v)

    def predict(self, Xs):
        Xs = np.ascontiguousarray(Xs, np.float64).reshape(-1, 2)
        out = np.empty((Xs.shape[0], self.m), np.float64)
        _check(self._lib.dsmc_gp_predict(self._h, _ptr(Xs), Xs.shape[0], _ptr(out)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dsmc_gp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cfd_faces(Kn: float, F: float, n: int, sigma_p, S_faces, stream=None):
    """``dsmc_cfd_faces``: Eq. 8 on n cells with the stress correction at the faces;
    sigma_p None means no slip."""
    S = np.ascontiguousarray(S_faces, np.float64)
    u = np.empty(int(n), np.float64)
    _check(load_library().dsmc_cfd_faces(float(Kn), float(F), int(n), 0 if sigma_p is None else 1,
                                         0.0 if sigma_p is None else float(sigma_p), _ptr(S),
                                         _ptr(u), _default_stream(stream)))
    return u


def surrogate_correction(fit: dict, n: int, stream=None):
    """S at the n + 1 faces of an n-cell grid for a fit's selected model."""
    S = np.empty(int(n) + 1, np.float64)
    _check(load_library().dsmc_surrogate_correction(ctypes.byref(fit["_raw"]), int(n), _ptr(S),
                                                    _default_stream(stream)))
    return S


def surrogate_exponents(Kn: float):
    b = np.empty(3, np.float64)
    _check(load_library().dsmc_surrogate_exponents(float(Kn), _ptr(b)))
    return tuple(float(x) for x in b)


FIELD_NAMES = ("n", "ux", "uy", "uz", "T", "Pxy", "qx", "qy", "qz")
NFIELD = len(FIELD_NAMES)


def _field_dict(out: np.ndarray) -> dict:
    return {k: out[:, i].copy() for i, k in enumerate(FIELD_NAMES)}


def fields(acc, n_samples: int, ppc: int) -> dict:
    """Cell fields from raw sums (``dsmc_cell_fields``): relative density n, velocity
    (v0), temperature (T0), shear stress P_xy (P0) and heat flux (P0 v0), one array per
    name of ``FIELD_NAMES``."""
    a = np.ascontiguousarray(acc, np.float64)
    out = np.empty((a.shape[0], NFIELD), np.float64)
    _check(load_library().dsmc_cell_fields(_ptr(a), int(n_samples), int(ppc), a.shape[0],
                                           _ptr(out)))
    return _field_dict(out)

