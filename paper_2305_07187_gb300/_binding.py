"""ctypes binding of libspring_ising.so (include/spring_ising.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  There is no CPU fallback -- if the library is missing the
import fails loudly.  Arrays may be NumPy (host) or torch tensors (host or
CUDA); CUDA tensors are passed by data_ptr() and the context's stream is the
caller's current torch stream unless another is given.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspring_ising.so")

SI_OK = 0
SI_ERR_INVALID_ARG = 1
SI_ERR_CUDA = 2
SI_ERR_OOM = 3
SI_ERR_TIMEOUT = 4
SI_ERR_UNSUPPORTED = 5
SI_ERR_NOT_SYMMETRIC = 6
STATUS_NAMES = {0: "SI_OK", 1: "SI_ERR_INVALID_ARG", 2: "SI_ERR_CUDA", 3: "SI_ERR_OOM",
                4: "SI_ERR_TIMEOUT", 5: "SI_ERR_UNSUPPORTED", 6: "SI_ERR_NOT_SYMMETRIC"}

SI_PREC_FP32 = 0
SI_PREC_FP64 = 1
SI_PREC_J_FP8_Q_BF16 = 2
SI_PREC_J_BF16_Q_BF16 = 3
PREC = {"fp32": 0, "fp64": 1, "j_fp8_q_bf16": 2, "j_bf16_q_bf16": 3}

EXPORTS = ("si_default_params", "si_create", "si_set_params", "si_run", "si_get_state", "si_energy", "si_grad",
           "si_enable_timing", "si_last_kernel_time", "si_synchronize", "si_describe", "si_last_launch_count",
           "si_last_error", "si_destroy", "si_run_noalloc", "si_hamiltonian", "si_create_group", "si_run_group",
           "si_group_energy", "si_group_enable_timing", "si_group_last_kernel_time",
           "si_group_describe", "si_group_last_launch_count", "si_destroy_group")


class SiParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("replicas", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("k", ctypes.c_float), ("m", ctypes.c_float), ("q0", ctypes.c_float),
                ("q_max", ctypes.c_float), ("p_max", ctypes.c_float),
                ("prec", ctypes.c_int32), ("update_order", ctypes.c_int32),
                ("wall_zero_p", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("fused_readout", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class SpringIsingError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libspring_ising.so not built (run __graft_entry__.build() "
                          "or python -m paper_2305_07187_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I32 = ctypes.c_int32
    lib.si_default_params.argtypes = [ctypes.POINTER(SiParams)]
    lib.si_default_params.restype = None
    lib.si_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(SiParams), P, P, P]
    lib.si_create.restype = ctypes.c_int
    lib.si_set_params.argtypes = [P, ctypes.POINTER(SiParams)]
    lib.si_set_params.restype = ctypes.c_int
    lib.si_run.argtypes = [P, P, P, P, P, P, P, P]
    lib.si_run_watch.argtypes = [P, P, P, P, P, I32, ctypes.c_int64, P, P, P, P, P]
    lib.si_run_watch.restype = ctypes.c_int
    lib.si_run.restype = ctypes.c_int
    lib.si_get_state.argtypes = [P, P, P]
    lib.si_get_state.restype = ctypes.c_int
    lib.si_energy.argtypes = [P, P, I32, P, P, P]
    lib.si_energy.restype = ctypes.c_int
    lib.si_grad.argtypes = [P, P, P, P, P, P, P, P, P]
    lib.si_grad.restype = ctypes.c_int
    lib.si_hamiltonian.argtypes = [P, P, P, I32, ctypes.c_double, P]
    lib.si_hamiltonian.restype = ctypes.c_int
    lib.si_enable_timing.argtypes = [P, I32]
    lib.si_enable_timing.restype = ctypes.c_int
    lib.si_last_kernel_time.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.si_last_kernel_time.restype = ctypes.c_int
    lib.si_synchronize.argtypes = [P]
    lib.si_synchronize.restype = ctypes.c_int
    lib.si_run_noalloc.argtypes = [ctypes.POINTER(SiParams), P, P, P, P, P, P, P, P]
    lib.si_run_noalloc.restype = ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.si_create_group.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(SiParams), PP, PP, P]
    lib.si_create_group.restype = ctypes.c_int
    lib.si_run_group.argtypes = [P, P, P, PP, PP, PP, PP, PP]
    lib.si_run_group.restype = ctypes.c_int
    lib.si_group_energy.argtypes = [P, I32, P, I32, P, P, P]
    lib.si_group_energy.restype = ctypes.c_int
    lib.si_group_enable_timing.argtypes = [P, I32]
    lib.si_group_enable_timing.restype = ctypes.c_int
    lib.si_group_last_kernel_time.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.si_group_last_kernel_time.restype = ctypes.c_int
    lib.si_group_describe.argtypes = [P, ctypes.c_char_p, I32]
    lib.si_group_describe.restype = ctypes.c_int
    lib.si_group_last_launch_count.argtypes = [P]
    lib.si_group_last_launch_count.restype = I32
    lib.si_destroy_group.argtypes = [P]
    lib.si_destroy_group.restype = None
    lib.si_describe.argtypes = [P, ctypes.c_char_p, I32]
    lib.si_describe.restype = ctypes.c_int
    lib.si_last_launch_count.argtypes = [P]
    lib.si_last_launch_count.restype = I32
    lib.si_last_error.argtypes = []
    lib.si_last_error.restype = ctypes.c_char_p
    lib.si_destroy.argtypes = [P]
    lib.si_destroy.restype = None
    _lib = lib
    return lib


def _check(status):
    if status != SI_OK:
        msg = load().si_last_error()
        raise SpringIsingError(status, msg.decode() if msg else "")


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class _Arg:
    """Pointer to an array argument; keeps converted copies alive."""

    def __init__(self, x, dtype, size=None, writable=False):
        self.obj = None
        self.ptr = None
        if x is None:
            return
        if _is_torch(x):
            import torch
            tdt = {np.float32: torch.float32, np.int8: torch.int8, np.int32: torch.int32,
                   np.float64: torch.float64}[dtype]
            if x.dtype != tdt or not x.is_contiguous():
                if writable:
                    raise TypeError("output tensor must be contiguous %s" % tdt)
                x = x.to(tdt).contiguous()
            if size is not None and x.numel() != size:
                raise ValueError("expected %d elements, got %d" % (size, x.numel()))
            self.obj = x
            self.ptr = ctypes.c_void_p(x.data_ptr())
        else:
            if writable:
                if not (isinstance(x, np.ndarray) and x.dtype == dtype and x.flags.c_contiguous):
                    raise TypeError("output array must be C-contiguous %s" % np.dtype(dtype))
                a = x
            else:
                a = np.ascontiguousarray(x, dtype=dtype)
            if size is not None and a.size != size:
                raise ValueError("expected %d elements, got %d" % (size, a.size))
            self.obj = a
            self.ptr = a.ctypes.data_as(ctypes.c_void_p)


def default_params(**kw) -> SiParams:
    p = SiParams()
    load().si_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        setattr(p, k, v)
    return p


def _stream_handle(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


class Context:
    """One Ising instance on the GPU (wraps si_ctx)."""

    def __init__(self, J, h=None, *, n=None, replicas=1, steps=0, prec="fp32", stream=None,
                 **params):
        lib = load()
        if n is None:
            n = int(J.shape[0])
        self.n, self.replicas, self.steps = int(n), int(replicas), int(steps)
        self.params = default_params(n=self.n, replicas=self.replicas, steps=self.steps,
                                     prec=prec, **params)
        self._J = _Arg(J, np.float32, self.n * self.n)
        self._h = _Arg(h, np.float32, self.n)
        self._stream = _stream_handle(stream)
        ctx = ctypes.c_void_p()
        _check(lib.si_create(ctypes.byref(ctx), ctypes.byref(self.params), self._J.ptr,
                             self._h.ptr, self._stream))
        self._J = self._h = None
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            load().si_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(256)
        _check(load().si_describe(self.ctx, buf, 256))
        return buf.value.decode()

    def enable_timing(self, on=True):
        _check(load().si_enable_timing(self.ctx, 1 if on else 0))

    def set_params(self, **params):
        """si_set_params: change integrator fields (k, m, q0, q_max, p_max,
        update_order, wall_zero_p, ckpt_every) of this context in place."""
        p = SiParams()
        ctypes.memmove(ctypes.byref(p), ctypes.byref(self.params), ctypes.sizeof(SiParams))
        for key, v in params.items():
            setattr(p, key, v)
        _check(load().si_set_params(self.ctx, ctypes.byref(p)))
        self.params = p

    def synchronize(self):
        """si_synchronize: wait for this context's work; raises a pending
        device error of an earlier call that returned early."""
        _check(load().si_synchronize(self.ctx))

    def last_kernel_ms(self) -> float:
        v = ctypes.c_float(0.0)
        _check(load().si_last_kernel_time(self.ctx, ctypes.byref(v)))
        return float(v.value)

    def last_launch_count(self) -> int:
        return int(load().si_last_launch_count(self.ctx))

    def run_into(self, zeta, dt, q_init, p_init=None, q_out=None, p_out=None, spins_out=None):
        """si_run with caller-provided outputs (numpy or torch, host or device).
        q_init None (with p_init None) continues from the context's state."""
        nR = self.n * self.replicas
        z = _Arg(zeta, np.float32, self.steps)
        d = _Arg(dt, np.float32, self.steps)
        qi = _Arg(q_init, np.float32, nR)
        pi = _Arg(p_init, np.float32, nR)
        qo = _Arg(q_out, np.float32, nR, writable=True)
        po = _Arg(p_out, np.float32, nR, writable=True)
        so = _Arg(spins_out, np.int8, nR, writable=True)
        _check(load().si_run(self.ctx, z.ptr, d.ptr, qi.ptr, pi.ptr, qo.ptr, po.ptr, so.ptr))

    def run_watch_into(self, zeta, dt, q_init, every, target_energy, p_init=None, q_out=None, p_out=None,
                       spins_out=None, energy_out=None):
        """si_run_watch: run until the first readout (every `every` steps)
        at which some replica's energy is <= target_energy; returns the
        number of steps made."""
        nR = self.n * self.replicas
        z = _Arg(zeta, np.float32, self.steps)
        d = _Arg(dt, np.float32, self.steps)
        qi = _Arg(q_init, np.float32, nR)
        pi = _Arg(p_init, np.float32, nR)
        qo = _Arg(q_out, np.float32, nR, writable=True)
        po = _Arg(p_out, np.float32, nR, writable=True)
        so = _Arg(spins_out, np.int8, nR, writable=True)
        eo = _Arg(energy_out, np.int32, self.replicas, writable=True)
        done = ctypes.c_int32(0)
        _check(load().si_run_watch(self.ctx, z.ptr, d.ptr, qi.ptr, pi.ptr, int(every), int(target_energy),
                                   qo.ptr, po.ptr, so.ptr, ctypes.c_void_p(ctypes.addressof(done)), eo.ptr))
        return int(done.value)

    def run_watch(self, zeta, dt, q_init, every, target_energy, p_init=None):
        """Host convenience: returns (steps_done, q, p, spins, energies)."""
        R, n = self.replicas, self.n
        q = np.empty((R, n), np.float32)
        p = np.empty((R, n), np.float32)
        s = np.empty((R, n), np.int8)
        e = np.empty(R, np.int32)
        done = self.run_watch_into(zeta, dt, q_init, every, target_energy, p_init, q, p, s, e)
        return done, q, p, s, e

    def run(self, zeta, dt, q_init, p_init=None):
        """Host convenience: returns (q, p, spins) as NumPy arrays."""
        R, n = self.replicas, self.n
        q = np.empty((R, n), np.float32)
        p = np.empty((R, n), np.float32)
        s = np.empty((R, n), np.int8)
        self.run_into(zeta, dt, q_init, p_init, q, p, s)
        return q, p, s

    def get_state(self):
        """si_get_state: the last run's (q, p) at working precision, as float64."""
        q = np.empty((self.replicas, self.n), np.float64)
        p = np.empty((self.replicas, self.n), np.float64)
        _check(load().si_get_state(self.ctx, q.ctypes.data_as(ctypes.c_void_p),
                                   p.ctypes.data_as(ctypes.c_void_p)))
        return q, p

    def energy_into(self, spins, R, energy_out=None, cut_out=None, energy_f=None):
        sp = _Arg(spins, np.int8, R * self.n)
        eo = _Arg(energy_out, np.int32, R, writable=True)
        co = _Arg(cut_out, np.int32, R, writable=True)
        fo = _Arg(energy_f, np.float64, R, writable=True)
        _check(load().si_energy(self.ctx, sp.ptr, int(R), eo.ptr, co.ptr, fo.ptr))

    def energy(self, spins, exact=True):
        """Host convenience: returns (energy_int32 or None, cut or None, energy_f).
        spins=None reads the spins of the last run() on this context."""
        if spins is None:
            s, R = None, self.replicas
        else:
            s = spins if _is_torch(spins) else np.ascontiguousarray(spins, dtype=np.int8)
            R = int(s.numel() // self.n) if _is_torch(s) else s.size // self.n
        e = np.empty(R, np.int32) if exact else None
        c = np.empty(R, np.int32) if exact else None
        f = np.empty(R, np.float64)
        self.energy_into(s, R, e, c, f)
        return e, c, f

    def hamiltonian(self, q, p, zeta, out=None):
        """si_hamiltonian: FP64 H per replica for the state (q, p) at coupling
        coefficient zeta.  q, p: NumPy or CUDA tensors of R*n floats; returns
        a NumPy float64 array, or fills `out` (NumPy or CUDA float64)."""
        R = (int(q.numel()) if _is_torch(q) else np.asarray(q).size) // self.n
        qa = _Arg(q, np.float32, R * self.n)
        pa = _Arg(p, np.float32, R * self.n)
        res = np.empty(R, np.float64) if out is None else out
        oa = _Arg(res, np.float64, R, writable=True)
        _check(load().si_hamiltonian(self.ctx, qa.ptr, pa.ptr, R, float(zeta), oa.ptr))
        return res

    def grad_into(self, zeta, dt, q_init, p_init=None, g_zeta=None, g_dt=None, g_k=None, objective=None):
        """si_grad into caller buffers (NumPy or CUDA tensors; any output may be None)."""
        nR = self.n * self.replicas
        a = [_Arg(zeta, np.float32, self.steps), _Arg(dt, np.float32, self.steps),
             _Arg(q_init, np.float32, nR), _Arg(p_init, np.float32, nR),
             _Arg(g_zeta, np.float32, self.steps, writable=True), _Arg(g_dt, np.float32, self.steps, writable=True),
             _Arg(g_k, np.float32, 1, writable=True), _Arg(objective, np.float32, 1, writable=True)]
        _check(load().si_grad(self.ctx, *[x.ptr for x in a]))

    def grad(self, zeta, dt, q_init, p_init=None):
        """si_grad: returns (objective, g_zeta, g_dt, g_k) as NumPy/float."""
        nR = self.n * self.replicas
        gz = np.empty(max(self.steps, 1), np.float32)
        gd = np.empty(max(self.steps, 1), np.float32)
        gk = np.empty(1, np.float32)
        ob = np.empty(1, np.float32)
        z = _Arg(zeta, np.float32, self.steps)
        d = _Arg(dt, np.float32, self.steps)
        qi = _Arg(q_init, np.float32, nR)
        pi = _Arg(p_init, np.float32, nR)
        _check(load().si_grad(self.ctx, z.ptr, d.ptr, qi.ptr, pi.ptr,
                              gz.ctypes.data_as(ctypes.c_void_p), gd.ctypes.data_as(ctypes.c_void_p),
                              gk.ctypes.data_as(ctypes.c_void_p), ob.ctypes.data_as(ctypes.c_void_p)))
        return float(ob[0]), gz[:self.steps], gd[:self.steps], float(gk[0])


SQRT2_F32 = float(np.float32(math.sqrt(2.0)))
NOALLOC_MAX_N = 16384


def run_noalloc(J, h, zeta, dt, q, p, spins_out=None, stream=None, **params):
    """si_run_noalloc: one replica, FP32, no device allocation by the library.

    All arrays must be CUDA tensors; q and p (shape [n]) are updated in place."""
    n = int(q.numel())
    prm = default_params(n=n, replicas=1, steps=int(zeta.numel()), **params)
    args = [_Arg(J, np.float32, n * n), _Arg(h, np.float32, n), _Arg(zeta, np.float32),
            _Arg(dt, np.float32), _Arg(q, np.float32, n, writable=True),
            _Arg(p, np.float32, n, writable=True), _Arg(spins_out, np.int8, n, writable=True)]
    _check(load().si_run_noalloc(ctypes.byref(prm), *[a.ptr for a in args], _stream_handle(stream)))


def _ptr_array(args):
    arr = (ctypes.c_void_p * len(args))()
    for k, a in enumerate(args):
        arr[k] = a.ptr.value if (a is not None and a.ptr is not None) else None
    return arr


class Group:
    """Grouped batch of independent instances (wraps si_group)."""

    def __init__(self, Js, hs=None, *, replicas, steps, precs="j_bf16_q_bf16", stream=None, **params):
        lib = load()
        count = len(Js)
        if isinstance(precs, str):
            precs = [precs] * count
        if isinstance(replicas, int):
            replicas = [replicas] * count
        self.count, self.steps = count, int(steps)
        self.ns = [int(J.shape[0]) for J in Js]
        self.Rs = [int(r) for r in replicas]
        prm = (SiParams * count)()
        for k in range(count):
            p = default_params(n=self.ns[k], replicas=self.Rs[k], steps=self.steps, prec=precs[k], **params)
            prm[k] = p
        Jargs = [_Arg(J, np.float32, self.ns[k] ** 2) for k, J in enumerate(Js)]
        hargs = None if hs is None else [_Arg(h, np.float32, self.ns[k]) if h is not None else None
                                         for k, h in enumerate(hs)]
        self._stream = _stream_handle(stream)
        g = ctypes.c_void_p()
        _check(lib.si_create_group(ctypes.byref(g), count, prm, _ptr_array(Jargs),
                                   None if hargs is None else _ptr_array(hargs), self._stream))
        self.g = g

    def close(self):
        if getattr(self, "g", None):
            load().si_destroy_group(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def describe(self):
        buf = ctypes.create_string_buffer(512)
        _check(load().si_group_describe(self.g, buf, 512))
        return buf.value.decode()

    def enable_timing(self, on=True):
        _check(load().si_group_enable_timing(self.g, 1 if on else 0))

    def last_kernel_ms(self):
        v = ctypes.c_float(0.0)
        _check(load().si_group_last_kernel_time(self.g, ctypes.byref(v)))
        return float(v.value)

    def last_launch_count(self):
        return int(load().si_group_last_launch_count(self.g))

    def run_into(self, zeta, dt, q_inits, p_inits=None, q_outs=None, p_outs=None, spins_outs=None):
        c = self.count
        sz = [self.ns[k] * self.Rs[k] for k in range(c)]
        z = _Arg(zeta, np.float32, self.steps)
        d = _Arg(dt, np.float32, self.steps)
        qi = [_Arg(q_inits[k], np.float32, sz[k]) for k in range(c)]
        pi = None if p_inits is None else [_Arg(p_inits[k], np.float32, sz[k]) for k in range(c)]
        qo = None if q_outs is None else [_Arg(q_outs[k], np.float32, sz[k], writable=True) for k in range(c)]
        po = None if p_outs is None else [_Arg(p_outs[k], np.float32, sz[k], writable=True) for k in range(c)]
        so = None if spins_outs is None else [_Arg(spins_outs[k], np.int8, sz[k], writable=True) for k in range(c)]
        arr = lambda xs: None if xs is None else _ptr_array(xs)
        _check(load().si_run_group(self.g, z.ptr, d.ptr, arr(qi), arr(pi), arr(qo), arr(po), arr(so)))

    def run(self, zeta, dt, q_inits, p_inits=None):
        qs = [np.empty((R, n), np.float32) for n, R in zip(self.ns, self.Rs)]
        ps = [np.empty((R, n), np.float32) for n, R in zip(self.ns, self.Rs)]
        ss = [np.empty((R, n), np.int8) for n, R in zip(self.ns, self.Rs)]
        self.run_into(zeta, dt, q_inits, p_inits, qs, ps, ss)
        return qs, ps, ss

    def energy(self, index, spins, exact=True):
        """si_group_energy for member `index`; spins may be NumPy or a torch tensor."""
        n = self.ns[index]
        s = spins if _is_torch(spins) else np.ascontiguousarray(spins, dtype=np.int8)
        R = (int(s.numel()) if _is_torch(s) else s.size) // n
        e = np.empty(R, np.int32) if exact else None
        cc = np.empty(R, np.int32) if exact else None
        f = np.empty(R, np.float64)
        sa = _Arg(s, np.int8, R * n)
        ea, ca, fa = _Arg(e, np.int32, R, True), _Arg(cc, np.int32, R, True), _Arg(f, np.float64, R, True)
        _check(load().si_group_energy(self.g, int(index), sa.ptr, R, ea.ptr, ca.ptr, fa.ptr))
        return e, cc, f
