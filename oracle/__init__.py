"""CPU oracle for the DSMC hot path: build and ctypes binding.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library and its binding) never imports, links or runs anything here, and this
package never imports the product path.

The oracle itself is ``dsmc_oracle.c``: a plain single-threaded C implementation of
the DSMC step (collide, sample, move with the body force and diffuse walls, stable
counting sort into cells) written from the paper's problem statement (Sec. 2.1,
Eqs. 1-8, Sec. 3) and Bird's DSMC method, which the paper cites for its micro model.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NMOM = 13

# binary32 arithmetic rounded once per operation: no contraction, no fast-math.
CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared", "-fvisibility=hidden", "-Wall"]


def build(force: bool = False) -> str:
    """Compile ``dsmc_oracle.c`` into ``_build/liboracle.so`` (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            c = ctypes
            u32p = c.POINTER(c.c_uint32)
            fp = c.POINTER(c.c_float)
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_philox4x32_10.restype = None
            L.or_u01.argtypes = [c.c_uint32]
            L.or_u01.restype = c.c_float
            L.or_ln.argtypes = [c.c_float]
            L.or_ln.restype = c.c_float
            L.or_exp.argtypes = [c.c_float]
            L.or_exp.restype = c.c_float
            L.or_pow.argtypes = [c.c_float, c.c_float]
            L.or_pow.restype = c.c_float
            L.or_normal_pair.argtypes = [c.c_uint32, c.c_uint32, fp, fp]
            L.or_normal_pair.restype = c.c_int
            L.or_nsigma.argtypes = [c.c_double, c.c_double]
            L.or_nsigma.restype = c.c_double
            L.or_cell_of.argtypes = [c.c_float, c.c_int]
            L.or_cell_of.restype = c.c_int
            L.or_stable_cell_sort.argtypes = [c.c_void_p, c.c_int, c.c_int, c.c_void_p, c.c_void_p]
            L.or_stable_cell_sort.restype = None
            L.or_move_particle.argtypes = [fp, fp, fp, fp, c.c_float, c.c_float,
                                           c.c_uint64, c.c_uint32, c.c_uint32]
            L.or_move_particle.restype = c.c_int
            L.or_move_particle_open.argtypes = [fp, fp, fp, fp, c.c_float, c.c_float,
                                                c.c_uint64, c.c_uint32, c.c_uint32, c.c_float,
                                                c.c_float]
            L.or_move_particle_open.restype = c.c_int
            L.or_set_open_top.argtypes = [c.c_void_p, c.c_double, c.c_double]
            L.or_set_open_top.restype = None
            L.or_pair_choice.argtypes = [c.c_uint32, c.c_int, c.POINTER(c.c_uint32),
                                         c.POINTER(c.c_uint32)]
            L.or_pair_choice.restype = None
            L.or_sincos_turn.argtypes = [c.c_float, fp, fp]
            L.or_sincos_turn.restype = None
            L.or_scatter_pair.argtypes = [fp, fp, c.c_uint64, c.c_uint32, c.c_uint32,
                                          c.c_uint32, c.c_uint32]
            L.or_scatter_pair.restype = c.c_int
            L.or_accept_threshold.argtypes = [c.c_void_p, c.c_float, c.c_float]
            L.or_accept_threshold.restype = c.c_float
            L.or_group_count.argtypes = [c.c_int, c.c_int]
            L.or_group_count.restype = c.c_int
            L.or_create.argtypes = [c.c_double, c.c_double, c.c_double, c.c_int, c.c_int,
                                    c.c_uint64, c.c_int, c.c_double, c.c_double,
                                    c.c_longlong, c.c_int]
            L.or_create.restype = c.c_void_p
            L.or_destroy.argtypes = [c.c_void_p]
            L.or_destroy.restype = None
            L.or_step.argtypes = [c.c_void_p, c.c_int]
            L.or_step.restype = c.c_int
            L.or_n_particles.argtypes = [c.c_void_p]
            L.or_n_particles.restype = c.c_int
            L.or_step_count.argtypes = [c.c_void_p]
            L.or_step_count.restype = c.c_longlong
            L.or_error.argtypes = [c.c_void_p]
            L.or_error.restype = c.c_int
            L.or_params.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p]
            L.or_params.restype = None
            L.or_get_state.argtypes = [c.c_void_p] + [c.c_void_p] * 4
            L.or_get_state.restype = None
            L.or_get_cells.argtypes = [c.c_void_p] + [c.c_void_p] * 4
            L.or_get_cells.restype = None
            L.or_get_moments.argtypes = [c.c_void_p, c.c_void_p]
            L.or_get_moments.restype = c.c_longlong
            L.or_reset_samples.argtypes = [c.c_void_p]
            L.or_reset_samples.restype = None
            L.or_get_abs_moments.argtypes = [c.c_void_p, c.c_void_p]
            L.or_get_abs_moments.restype = None
            L.or_ln_array.argtypes = [c.c_void_p, c.c_void_p, c.c_longlong]
            L.or_ln_array.restype = None
            L.or_exp_array.argtypes = [c.c_void_p, c.c_void_p, c.c_longlong]
            L.or_exp_array.restype = None
            L.or_init_velocities.argtypes = [c.c_uint64, c.c_longlong, c.c_void_p]
            L.or_init_velocities.restype = c.c_int
            L.or_emission_speeds.argtypes = [c.c_uint64, c.c_longlong, c.c_void_p]
            L.or_emission_speeds.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def ln32(x: float) -> float:
    return lib().or_ln(float(x))


def exp32(x: float) -> float:
    return lib().or_exp(float(x))


def ln32_array(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(x)
    lib().or_ln_array(_ptr(x), _ptr(out), x.size)
    return out


def exp32_array(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(x)
    lib().or_exp_array(_ptr(x), _ptr(out), x.size)
    return out


def init_velocities(seed: int, n: int) -> np.ndarray:
    out = np.empty((n, 3), np.float32)
    ok = lib().or_init_velocities(int(seed), int(n), _ptr(out))
    if not ok:
        raise RuntimeError("normal attempts ran out")
    return out


def emission_speeds(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    lib().or_emission_speeds(int(seed), int(n), _ptr(out))
    return out


def u01(x: int) -> float:
    return lib().or_u01(int(x) & 0xffffffff)


def nsigma(omega: float, Kn: float) -> float:
    return lib().or_nsigma(float(omega), float(Kn))


def group_count(nc: int, G: int) -> int:
    return lib().or_group_count(int(nc), int(G))


def stable_cell_sort(cell: np.ndarray, n_cells: int):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    perm = np.empty(len(cell), dtype=np.int32)
    off = np.empty(n_cells + 1, dtype=np.int32)
    lib().or_stable_cell_sort(_ptr(cell), len(cell), n_cells, _ptr(perm), _ptr(off))
    return perm, off


def move_particle(y, vx, vy, vz, dt, F, seed, step, slot):
    a = [ctypes.c_float(v) for v in (y, vx, vy, vz)]
    ok = lib().or_move_particle(*[ctypes.byref(v) for v in a], float(dt), float(F),
                                int(seed), int(step) & 0xffffffff, int(slot))
    return tuple(v.value for v in a), bool(ok)


def move_particle_open(y, vx, vy, vz, dt, F, seed, step, slot, u_top, p_top):
    """One flight with the open Chapman-Enskog boundary at y = 1; returns the new
    (y, vx, vy, vz) and the error bits."""
    a = [ctypes.c_float(y), ctypes.c_float(vx), ctypes.c_float(vy), ctypes.c_float(vz)]
    err = lib().or_move_particle_open(*[ctypes.byref(v) for v in a], float(dt), float(F),
                                      int(seed), int(step) & 0xffffffff, int(slot),
                                      float(u_top), float(p_top))
    return tuple(v.value for v in a), int(err)


def pair_choice(w0, ng):
    """The candidate pair (i, j), i != j, from one 32-bit word."""
    i = ctypes.c_uint32()
    j = ctypes.c_uint32()
    lib().or_pair_choice(int(w0) & 0xFFFFFFFF, int(ng), ctypes.byref(i), ctypes.byref(j))
    return i.value, j.value


def sincos_turn(v):
    """(sin 2 pi v, cos 2 pi v) in binary32 by the oracle's own polynomial."""
    sn = ctypes.c_float()
    cs = ctypes.c_float()
    lib().or_sincos_turn(float(v), ctypes.byref(sn), ctypes.byref(cs))
    return np.float32(sn.value), np.float32(cs.value)


def scatter_pair(vi, vj, seed, k, cell, step, group):
    a = (ctypes.c_float * 3)(*vi)
    b = (ctypes.c_float * 3)(*vj)
    ok = lib().or_scatter_pair(a, b, int(seed), int(k), int(cell), int(step), int(group))
    return np.array(list(a), np.float32), np.array(list(b), np.float32), bool(ok)


class OracleSim:
    """One oracle DSMC run.  Arguments as in ``or_create`` (see dsmc_oracle.c)."""

    def __init__(self, omega=0.5, Kn=1.0, F=0.0, n_cells=100, ppc=200, seed=0, G=256,
                 dt_factor=0.2, dt=0.0, sample_start=0, collisions=True):
        self.n_cells = int(n_cells)
        self.h = lib().or_create(float(omega), float(Kn), float(F), int(n_cells), int(ppc),
                                 int(seed), int(G), float(dt_factor), float(dt),
                                 int(sample_start), 1 if collisions else 0)
        if not self.h:
            raise ValueError("oracle: invalid arguments")
        self.N = lib().or_n_particles(self.h)

    def close(self):
        if self.h:
            lib().or_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_open_top(self, u: float, P: float) -> None:
        """The boundary at y = 1 becomes an open Chapman-Enskog reservoir (bulk velocity
        u, shear stress P) from the next step on."""
        lib().or_set_open_top(self.h, float(u), float(P))

    def step(self, n=1) -> int:
        return lib().or_step(self.h, int(n))

    @property
    def step_count(self) -> int:
        return lib().or_step_count(self.h)

    @property
    def error(self) -> int:
        return lib().or_error(self.h)

    def params(self):
        f = np.zeros(8, np.float32)
        d = np.zeros(2, np.float64)
        lib().or_params(self.h, _ptr(f), _ptr(d))
        return {"dt": f[0], "F": f[1], "coef": f[2], "cvhs": f[3], "vexp": f[4],
                "smax0": f[5], "vinv": f[6], "lncv": f[7], "nsig": d[0], "dt_d": d[1]}

    def state(self):
        arrs = [np.empty(self.N, np.float32) for _ in range(4)]
        lib().or_get_state(self.h, *[_ptr(a) for a in arrs])
        return tuple(arrs)

    def cells(self):
        off = np.empty(self.n_cells + 1, np.int32)
        smax = np.empty(self.n_cells, np.float32)
        nc = np.empty(self.n_cells, np.uint64)
        na = np.empty(self.n_cells, np.uint64)
        lib().or_get_cells(self.h, _ptr(off), _ptr(smax), _ptr(nc), _ptr(na))
        return off, smax, nc, na

    def moments(self):
        out = np.empty((self.n_cells, NMOM), np.float64)
        n = lib().or_get_moments(self.h, _ptr(out))
        return out, int(n)

    def abs_moments(self):
        """Sums of |product| per cell and moment, for error bounds of other summation
        orders of the same products."""
        out = np.empty((self.n_cells, NMOM), np.float64)
        lib().or_get_abs_moments(self.h, _ptr(out))
        return out

    def reset_samples(self):
        lib().or_reset_samples(self.h)

    def accept_threshold(self, u: float, smax: float) -> float:
        return lib().or_accept_threshold(self.h, float(u), float(smax))


def fields(acc: np.ndarray, n_samples: int, ppc: int) -> dict:
    """Cell fields from the raw moment sums of ``OracleSim.moments`` (plain numpy).

    Units as in Eq. 6 of the paper: density relative to the initial one, velocity in
    v0, temperature in T0, shear stress P_xy in P0 = n0 k T0 (rho / P0 = 2 / v0^2),
    heat flux in P0 v0.
    """
    a = np.asarray(acc, np.float64)
    N = a[:, 0]
    with np.errstate(invalid="ignore", divide="ignore"):
        nhat = N / (n_samples * ppc)
        u = a[:, 1:4] / N[:, None]
        vxx, vyy, vzz = a[:, 4] / N, a[:, 5] / N, a[:, 6] / N
        vxy, vxz, vyz = a[:, 7] / N, a[:, 8] / N, a[:, 9] / N
        vv = vxx + vyy + vzz
        uu = (u ** 2).sum(axis=1)
        T = (2.0 / 3.0) * (vv - uu)
        Pxy = 2.0 * nhat * (vxy - u[:, 0] * u[:, 1])
        M = np.stack([np.stack([vxx, vxy, vxz], 1), np.stack([vxy, vyy, vyz], 1),
                      np.stack([vxz, vyz, vzz], 1)], 1)  # <v_i v_j>
        q = np.empty_like(u)
        for i in range(3):
            q[:, i] = nhat * (a[:, 10 + i] / N - 2.0 * (M[:, i, :] * u).sum(axis=1)
                              - u[:, i] * vv + 2.0 * u[:, i] * uu)
    return {"n": nhat, "ux": u[:, 0], "uy": u[:, 1], "uz": u[:, 2], "T": T, "Pxy": Pxy,
            "qx": q[:, 0], "qy": q[:, 1]}
