"""OpenMP timing build of the FP64 oracle -- BENCHMARK CPU BASELINE ONLY.

``timing_omp.cpp`` compiles the oracle's source unchanged together with
OpenMP versions of the render and its adjoint (the projection, pixel and
per-Gaussian loops spread over the host cores; per-Gaussian sums by atomic
additions).  It exists to time the oracle on all host cores for the CPU
baseline of ``bench.py``; the parity tests use the single-threaded oracle.
Only ``tests/`` and ``bench.py``'s CPU-baseline leg may import this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import _cams, _f64, _p, _params, settings_array

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "timing_omp.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle_omp.so with g++ -fopenmp (the oracle's source included)."""
    deps = [_SRC, os.path.join(_HERE, "airgs_oracle.cpp")]
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(map(os.path.getmtime, deps)):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-o", _LIB_PATH + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.orc_omp_threads.restype = ctypes.c_int
        lib.orc_omp_render.argtypes = [ctypes.c_int64, ctypes.c_int] + [P] * 5 + [ctypes.c_int, P, P] + [P] * 6
        lib.orc_omp_render_backward.argtypes = [ctypes.c_int64, ctypes.c_int] + [P] * 5 + [ctypes.c_int, P, P] + \
            [P] * 6
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the build uses (OMP_NUM_THREADS, else the host's cores)."""
    return int(_load().orc_omp_threads())


def render(g: dict, cams, **settings):
    """rgb [3,H,W], T [H,W], n_contrib [H,W] per view, usage frequency and the
    evaluated pair count, as oracle.render computes them."""
    lib = _load()
    means, ls, qs, ol, sh = _params(g)
    N = means.shape[0]
    sizes = [(int(c["height"]), int(c["width"])) for c in cams]
    tot = sum(h * w for h, w in sizes)
    rgb, T, nc = np.zeros(3 * tot), np.zeros(tot), np.zeros(tot, np.int32)
    w, cnt, pairs = np.zeros(N), np.zeros(N, np.int64), np.zeros(1, np.int64)
    rc = lib.orc_omp_render(N, int(g["sh_degree"]), _p(means), _p(ls), _p(qs), _p(ol), _p(sh), len(cams),
                            _p(_cams(cams)), _p(settings_array(**settings)), _p(rgb), _p(T), _p(nc), _p(w), _p(cnt),
                            _p(pairs))
    if rc != 0:
        raise ValueError("bad sh degree")
    out = dict(rgb=[], T=[], n_contrib=[], importance_w=w, importance_cnt=cnt, pairs=int(pairs[0]))
    off = 0
    for h, wd in sizes:
        hw = h * wd
        out["rgb"].append(rgb[3 * off:3 * (off + hw)].reshape(3, h, wd))
        out["T"].append(T[off:off + hw].reshape(h, wd))
        out["n_contrib"].append(nc[off:off + hw].reshape(h, wd))
        off += hw
    return out


def render_backward(g: dict, cams, dL_drgb, **settings):
    """Gradients of sum(dL_drgb * rgb) w.r.t. the raw parameters, as
    oracle.render_backward computes them (up to the order of additions)."""
    lib = _load()
    means, ls, qs, ol, sh = _params(g)
    N = means.shape[0]
    K = sh.shape[1]
    flat = _f64(np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in dL_drgb]))
    gm, gl, gq, go, gs = np.zeros((N, 3)), np.zeros((N, 3)), np.zeros((N, 4)), np.zeros(N), np.zeros((N, K, 3))
    rc = lib.orc_omp_render_backward(N, int(g["sh_degree"]), _p(means), _p(ls), _p(qs), _p(ol), _p(sh), len(cams),
                                     _p(_cams(cams)), _p(settings_array(**settings)), _p(flat), _p(gm), _p(gl),
                                     _p(gq), _p(go), _p(gs))
    if rc != 0:
        raise ValueError("bad sh degree")
    return dict(means=gm, log_scales=gl, quats=gq, opacity_logit=go, sh=gs)
