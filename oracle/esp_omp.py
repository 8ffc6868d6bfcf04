"""ctypes wrapper of oracle/esp_omp.c, the plain FP64 OpenMP ESP step (test and benchmark
infrastructure: the CPU baseline on all host cores).  ``build()`` compiles it with gcc."""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import lattice
from .pswf import prolate

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "esp_omp.c")
LIB = os.path.join(HERE, "libesp_omp.so")


def build() -> str:
    cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", LIB + ".tmp", SRC, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"gcc failed:\n{' '.join(cmd)}\n{res.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        lib = ctypes.CDLL(LIB)
        d, i64, ci = ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int
        lib.esp_omp_step.restype = ci
        lib.esp_omp_step.argtypes = [i64, d, d, d, ctypes.POINTER(ci), ci, ctypes.c_double,
                                     ctypes.c_double, ci, d, d, ctypes.c_double, ctypes.c_double,
                                     d, d, d, ci]
        _lib = lib
    return _lib


def esp_omp(pos, q, h, M, P, c, rc, forces=True, threads=0):
    """U_F, W_F and (optionally) forces of the ESP long-range step; threads = 0: all."""
    lib = _load()
    h = lattice.check_cell(h)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    p = prolate(c)
    coef = np.ascontiguousarray(p.coef, dtype=np.float64)
    dcoef = np.zeros_like(coef)
    dcoef[:len(p.dcoef)] = p.dcoef
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    hh = np.ascontiguousarray(h, dtype=np.float64)
    Mc = (ctypes.c_int * 3)(*[int(m) for m in M])
    e = ctypes.c_double()
    W = np.zeros(9)
    F = np.zeros((len(q), 3)) if forces else None
    rc_ = lib.esp_omp_step(len(q), dp(pos), dp(q), dp(hh), Mc, int(P), float(c), float(rc),
                           len(coef), dp(coef), dp(dcoef), float(p.lam0), float(p.C0),
                           ctypes.byref(e), dp(W), dp(F) if forces else None, int(threads))
    if rc_ != 0:
        raise RuntimeError(f"esp_omp_step failed ({rc_})")
    return {"energy": e.value, "virial": W.reshape(3, 3), "forces": F}
