"""ctypes wrapper of the compiled FP64 CPU baseline (oracle/sem_cpu.c).

TEST INFRASTRUCTURE ONLY: loaded by tests/ and by the cpu_baseline / --impl reference legs
of bench.py, never by the product. It takes a numpy oracle Model's geometry and material
(oracle/sem_oracle.py) and runs the time step of Sec. I, II-B and V-C as plain C loops in
float64, single-threaded or with OpenMP over the elements of one colour at a time (Sec.
IV-C); ``tests/test_oracle_cpu.py`` pins it to the numpy oracle."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sem_cpu.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsemcpu.so")
_lib = None
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the baseline with gcc (-O3, OpenMP) if the source is newer than the library."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + ".tmp"
    r = subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp, "-lm"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("building the CPU baseline failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.sem_cpu_color.restype = ctypes.c_int
        _lib.sem_cpu_max_threads.restype = ctypes.c_int
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_P)


class CpuBaseline:
    """The time step of one oracle Model as compiled loops; ``threads`` OpenMP threads."""

    def __init__(self, model, threads: int = 1):
        self.m = model
        n, nspec = model.ngll, model.nspec
        np_ = n ** 3
        self.threads = int(threads)
        self.ibool = np.ascontiguousarray(model.ibool.reshape(nspec, np_), dtype=np.int32)
        self.h = np.ascontiguousarray(model.basis.hprime, dtype=np.float64)
        self.w = np.ascontiguousarray(model.basis.w, dtype=np.float64)
        self.G = np.ascontiguousarray(model.dxi_dx.reshape(nspec, 3, 3, np_))
        self.J = np.ascontiguousarray(model.jac.reshape(nspec, np_))
        self.kappa = np.ascontiguousarray(model.kappa.reshape(nspec, np_))
        self.mu = np.ascontiguousarray(model.mu.reshape(nspec, np_))
        self.minv = np.ascontiguousarray(1.0 / model.mass)
        self.order = np.empty(nspec, dtype=np.int32)
        off = np.empty(65, dtype=np.int32)
        nc = lib().sem_cpu_color(nspec, n, model.nglob, _ptr(self.ibool), _ptr(self.order), _ptr(off), 64)
        if nc < 0:
            raise RuntimeError("colouring needs more than 64 colours")
        self.ncolors = nc
        self.color_off = off[:nc + 1].copy()

    def forces(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        f = np.empty_like(u)
        m = self.m
        lib().sem_cpu_forces(m.nspec, m.ngll, m.nglob, _ptr(self.ibool), _ptr(self.h), _ptr(self.w), _ptr(self.G),
                             _ptr(self.J), _ptr(self.kappa), _ptr(self.mu), _ptr(self.order), _ptr(self.color_off),
                             self.ncolors, _ptr(u), _ptr(f), self.threads)
        return f

    def run(self, dt, nsteps, u=None, v=None, a=None, src_node=-1, src_force=(0.0, 0.0, 0.0), f0=10.0, t0=0.12):
        """nsteps Newmark steps from (u, v, a) (zero when None); returns (u, v, a)."""
        m = self.m
        z = lambda x: np.zeros((m.nglob, 3)) if x is None else np.array(x, dtype=np.float64)  # noqa: E731
        u, v, a = z(u), z(v), z(a)
        f = np.empty_like(u)
        sf = np.ascontiguousarray(src_force, dtype=np.float64).reshape(3)
        lib().sem_cpu_run(m.nspec, m.ngll, m.nglob, _ptr(self.ibool), _ptr(self.h), _ptr(self.w), _ptr(self.G),
                          _ptr(self.J), _ptr(self.kappa), _ptr(self.mu), _ptr(self.minv), _ptr(self.order),
                          _ptr(self.color_off), self.ncolors, int(nsteps), ctypes.c_double(dt), int(src_node),
                          _ptr(sf), ctypes.c_double(f0), ctypes.c_double(t0), _ptr(u), _ptr(v), _ptr(a), _ptr(f),
                          self.threads)
        return u, v, a


def max_threads() -> int:
    return int(lib().sem_cpu_max_threads())
