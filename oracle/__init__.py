"""FP64 CPU oracle for the Spring-Ising Algorithm (arXiv 2305.07187).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library (``paper_2305_07187_gb300``) never imports, links or calls it,
and the two share no code: this package holds a plain C restatement of the
paper's equations (``si_oracle.c``, compiled with gcc, no fast-math, no FMA
contraction) and thin ctypes marshalling.

Functions follow the paper's equations:
  run               Eq. 8 (order 0, kick-drift) or Eq. 5 (order 1), walls Eq. 6
  energy            Eq. 1, pair sum over i < j
  cut               MAX-CUT value with weights w = -J
  relaxed_energy    Eq. 1 with sigma -> q (continuous relaxation)
  hamiltonian       Eq. 3 / Eq. 7
  bruteforce        exhaustive minimum of Eq. 1 (n <= 24)
  grad              reverse-mode gradient of the relaxed final energy
  fd_grad           FP64 central finite differences of the same objective
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "si_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsi_oracle.so")
_lock = threading.Lock()
_lib = None

SQRT2 = math.sqrt(2.0)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over replicas, strict FP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            D = ctypes.c_double
            I = ctypes.c_int
            P = ctypes.c_void_p
            lib.or_run.argtypes = [I, I, I, P, P, P, P, D, D, D, D, D, I, I, P, P]
            lib.or_run.restype = I
            lib.or_sign.argtypes = [I, P, P]
            lib.or_energy.argtypes = [I, I, P, P, P, P]
            lib.or_cut.argtypes = [I, I, P, P, P]
            lib.or_relaxed_energy.argtypes = [I, I, P, P, P, P]
            lib.or_hamiltonian.argtypes = [I, I, P, P, D, D, D, D, P, P, P]
            lib.or_bruteforce.argtypes = [I, P, P, P, P]
            lib.or_bruteforce.restype = I
            lib.or_grad.argtypes = [I, I, I, P, P, P, P, D, D, D, D, D, I,
                                    P, P, P, P, P, P]
            lib.or_grad.restype = I
            lib.or_num_threads.restype = I
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().or_num_threads())


def run(J, h, zeta, dt, q, p=None, *, k=0.5, m=1.0, q0=0.0, q_max=SQRT2,
        p_max=2.0, order=0, wall_zero_p=False):
    """Run len(zeta) steps for every replica.  q, p: (R, n).  Returns (q, p)."""
    J = _f64(J)
    n = J.shape[0]
    q = np.array(q, dtype=np.float64, copy=True).reshape(-1, n)
    R = q.shape[0]
    p = np.zeros_like(q) if p is None else np.array(p, dtype=np.float64, copy=True).reshape(R, n)
    zeta = _f64(zeta).reshape(-1)
    dt = _f64(dt).reshape(-1)
    T = zeta.shape[0]
    assert dt.shape[0] == T
    hh = None if h is None else _f64(h).reshape(n)
    rc = _load().or_run(n, R, T, _ptr(J), _ptr(hh), _ptr(zeta), _ptr(dt),
                        float(k), float(m), float(q0), float(q_max), float(p_max),
                        int(order), int(bool(wall_zero_p)), _ptr(q), _ptr(p))
    if rc != 0:
        raise RuntimeError("or_run failed with code %d" % rc)
    return q, p


def sign(q):
    """sigma = sign(q) with sign(0) = +1, as int8."""
    q = _f64(q)
    s = np.empty(q.shape, dtype=np.int8)
    _load().or_sign(int(q.size), _ptr(q), _ptr(s))
    return s


def energy(J, h, sigma):
    """Eq. 1 for each row of sigma (R, n) -> float64 (R,)."""
    J = _f64(J)
    n = J.shape[0]
    s = np.ascontiguousarray(sigma, dtype=np.int8).reshape(-1, n)
    E = np.empty(s.shape[0], dtype=np.float64)
    hh = None if h is None else _f64(h).reshape(n)
    _load().or_energy(n, s.shape[0], _ptr(J), _ptr(hh), _ptr(s), _ptr(E))
    return E


def cut(J, sigma):
    """MAX-CUT value with weights w = -J for each row of sigma -> (R,)."""
    J = _f64(J)
    n = J.shape[0]
    s = np.ascontiguousarray(sigma, dtype=np.int8).reshape(-1, n)
    c = np.empty(s.shape[0], dtype=np.float64)
    _load().or_cut(n, s.shape[0], _ptr(J), _ptr(s), _ptr(c))
    return c


def relaxed_energy(J, h, q):
    J = _f64(J)
    n = J.shape[0]
    x = _f64(q).reshape(-1, n)
    E = np.empty(x.shape[0], dtype=np.float64)
    hh = None if h is None else _f64(h).reshape(n)
    _load().or_relaxed_energy(n, x.shape[0], _ptr(J), _ptr(hh), _ptr(x), _ptr(E))
    return E


def hamiltonian(J, h, q, p, *, zeta, k=0.5, m=1.0, q0=0.0):
    J = _f64(J)
    n = J.shape[0]
    x = _f64(q).reshape(-1, n)
    y = _f64(p).reshape(-1, n)
    H = np.empty(x.shape[0], dtype=np.float64)
    hh = None if h is None else _f64(h).reshape(n)
    _load().or_hamiltonian(n, x.shape[0], _ptr(J), _ptr(hh), float(zeta), float(k),
                           float(m), float(q0), _ptr(x), _ptr(y), _ptr(H))
    return H


def bruteforce(J, h=None):
    """Exhaustive ground state of Eq. 1: returns (E_min, sigma_argmin)."""
    J = _f64(J)
    n = J.shape[0]
    hh = None if h is None else _f64(h).reshape(n)
    Emin = ctypes.c_double(0.0)
    s = np.empty(n, dtype=np.int8)
    rc = _load().or_bruteforce(n, _ptr(J), _ptr(hh), ctypes.byref(Emin), _ptr(s))
    if rc != 0:
        raise ValueError("bruteforce needs 1 <= n <= 24")
    return float(Emin.value), s


def grad(J, h, zeta, dt, q, p=None, *, k=0.5, m=1.0, q0=0.0, q_max=SQRT2,
         p_max=2.0, order=0):
    """Reverse-mode gradient of sum_r relaxed_energy(q_T) w.r.t. zeta, dt, k.

    Returns (objective, g_zeta, g_dt, g_k)."""
    J = _f64(J)
    n = J.shape[0]
    q = _f64(q).reshape(-1, n)
    R = q.shape[0]
    p = None if p is None else _f64(p).reshape(R, n)
    zeta = _f64(zeta).reshape(-1)
    dt = _f64(dt).reshape(-1)
    T = zeta.shape[0]
    gz = np.empty(T, dtype=np.float64)
    gd = np.empty(T, dtype=np.float64)
    gk = ctypes.c_double(0.0)
    obj = ctypes.c_double(0.0)
    hh = None if h is None else _f64(h).reshape(n)
    rc = _load().or_grad(n, R, T, _ptr(J), _ptr(hh), _ptr(zeta), _ptr(dt),
                         float(k), float(m), float(q0), float(q_max), float(p_max),
                         int(order), _ptr(q), _ptr(p), _ptr(gz), _ptr(gd),
                         ctypes.byref(gk), ctypes.byref(obj))
    if rc != 0:
        raise RuntimeError("or_grad failed with code %d" % rc)
    return float(obj.value), gz, gd, float(gk.value)


def objective(J, h, zeta, dt, q, p=None, **kw):
    """sum_r relaxed_energy(q_T): the quantity that ``grad`` differentiates."""
    qT, _ = run(J, h, zeta, dt, q, p, **kw)
    return float(relaxed_energy(J, h, qT).sum())


def fd_grad(J, h, zeta, dt, q, p=None, *, eps=1e-6, which=("zeta", "dt", "k"),
            k=0.5, **kw):
    """FP64 central finite differences of ``objective``.

    Returns dict name -> array (zeta, dt) or float (k)."""
    zeta = _f64(zeta).reshape(-1).copy()
    dt = _f64(dt).reshape(-1).copy()
    out = {}
    if "zeta" in which:
        g = np.empty_like(zeta)
        for t in range(zeta.size):
            zp = zeta.copy(); zp[t] += eps
            zm = zeta.copy(); zm[t] -= eps
            g[t] = (objective(J, h, zp, dt, q, p, k=k, **kw)
                    - objective(J, h, zm, dt, q, p, k=k, **kw)) / (2 * eps)
        out["zeta"] = g
    if "dt" in which:
        g = np.empty_like(dt)
        for t in range(dt.size):
            dp_ = dt.copy(); dp_[t] += eps
            dm_ = dt.copy(); dm_[t] -= eps
            g[t] = (objective(J, h, zeta, dp_, q, p, k=k, **kw)
                    - objective(J, h, zeta, dm_, q, p, k=k, **kw)) / (2 * eps)
        out["dt"] = g
    if "k" in which:
        out["k"] = (objective(J, h, zeta, dt, q, p, k=k + eps, **kw)
                    - objective(J, h, zeta, dt, q, p, k=k - eps, **kw)) / (2 * eps)
    return out
