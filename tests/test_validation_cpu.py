"""Host-side validation at the C ABI, checked without a GPU: every call
returns a status and a message instead of aborting, si_create rejects bad
parameters before it touches a device, the calls reject missing handles and
arrays, and without a GPU the product path fails with an error status (there
is no CPU fallback).  Also the binding's marshalling of array arguments."""
import ctypes

import numpy as np
import pytest

from paper_2305_07187_gb300 import _binding as b

P = ctypes.c_void_p


def _create_status(**kw):
    lib = b.load()
    prm = b.default_params(n=8, replicas=2, steps=3)
    for k, v in kw.items():
        if k == "reserved":
            prm.reserved[0] = v
        else:
            setattr(prm, k, v)
    J = np.zeros((8, 8), np.float32)
    ctx = P()
    st = lib.si_create(ctypes.byref(ctx), ctypes.byref(prm), J.ctypes.data_as(P), None, None)
    return st, lib.si_last_error().decode(), ctx


@pytest.mark.parametrize("field,value,words", [
    ("n", 0, "n >= 1"),
    ("replicas", 0, "replicas >= 1"),
    ("steps", -1, "steps >= 0"),
    ("prec", 9, "precision"),
    ("update_order", 2, "update_order"),
    ("m", 0.0, "positive finite m"),
    ("q_max", -1.0, "q_max"),
    ("p_max", float("nan"), "p_max"),
    ("k", float("inf"), "finite k"),
    ("q0", float("nan"), "q0"),
    ("ckpt_every", -1, "ckpt_every"),
    ("tile_n", -64, "tile_n"),
    ("fused_readout", 2, "fused_readout"),
    ("reserved", 1, "reserved"),
])
def test_create_rejects_bad_parameters_before_any_device_work(field, value, words):
    st, msg, ctx = _create_status(**{field: value})
    assert st == b.SI_ERR_INVALID_ARG, (field, st, msg)
    assert words in msg
    assert not ctx.value


def test_create_rejects_a_coupling_matrix_beyond_the_index_range():
    st, msg, _ = _create_status(n=200000)
    assert st == b.SI_ERR_UNSUPPORTED and "too large" in msg


def test_create_needs_its_output_handle_and_J():
    lib = b.load()
    prm = b.default_params(n=8, replicas=1, steps=1)
    J = np.zeros((8, 8), np.float32)
    assert lib.si_create(None, ctypes.byref(prm), J.ctypes.data_as(P), None, None) == b.SI_ERR_INVALID_ARG
    ctx = P()
    assert lib.si_create(ctypes.byref(ctx), ctypes.byref(prm), None, None, None) == b.SI_ERR_INVALID_ARG
    assert lib.si_create(ctypes.byref(ctx), None, J.ctypes.data_as(P), None, None) == b.SI_ERR_INVALID_ARG


def test_calls_without_a_context_return_invalid_arg():
    lib = b.load()
    z = np.zeros(4, np.float32)
    zp = z.ctypes.data_as(P)
    assert lib.si_run(None, zp, zp, zp, None, None, None, None) == b.SI_ERR_INVALID_ARG
    assert lib.si_run_watch(None, zp, zp, zp, None, 10, 0, None, None, None, None, None) == b.SI_ERR_INVALID_ARG
    assert lib.si_energy(None, None, 1, None, None, None) == b.SI_ERR_INVALID_ARG
    assert lib.si_grad(None, zp, zp, zp, None, None, None, None, None) == b.SI_ERR_INVALID_ARG
    assert lib.si_get_state(None, None, None) == b.SI_ERR_INVALID_ARG
    assert lib.si_last_error().decode() != ""
    lib.si_destroy(None)          # a no-op, not a crash
    lib.si_destroy_group(None)


def test_noalloc_rejects_bad_sizes_before_any_device_work():
    lib = b.load()
    buf = np.zeros(4, np.float32)
    bp = buf.ctypes.data_as(P)
    prm = b.default_params(n=b.NOALLOC_MAX_N + 1, replicas=1, steps=1)
    assert lib.si_run_noalloc(ctypes.byref(prm), bp, None, bp, bp, bp, bp, None, None) == b.SI_ERR_INVALID_ARG
    assert "SI_NOALLOC_MAX_N" in lib.si_last_error().decode()
    prm = b.default_params(n=8, replicas=2, steps=1)
    assert lib.si_run_noalloc(ctypes.byref(prm), bp, None, bp, bp, bp, bp, None, None) == b.SI_ERR_INVALID_ARG
    assert lib.si_run_noalloc(None, bp, None, bp, bp, bp, bp, None, None) == b.SI_ERR_INVALID_ARG


def test_no_cpu_fallback_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    J = np.zeros((8, 8), np.float32)
    with pytest.raises(b.SpringIsingError) as ei:
        b.Context(J, replicas=2, steps=3, prec="fp32")
    assert ei.value.status != b.SI_OK


def test_array_arguments_are_checked_and_kept_alive():
    out = np.zeros(6, np.float32)
    assert b._Arg(out, np.float32, 6, writable=True).ptr.value == out.ctypes.data
    with pytest.raises(ValueError):
        b._Arg(out, np.float32, 5, writable=True)
    with pytest.raises(TypeError):
        b._Arg(np.zeros(6, np.float64), np.float32, 6, writable=True)
    with pytest.raises(TypeError):
        b._Arg(np.zeros((6, 2), np.float32)[:, 0], np.float32, 6, writable=True)
    # inputs of another type or layout are converted into a copy the argument keeps
    a = b._Arg(np.arange(6, dtype=np.float64), np.float32, 6)
    assert a.obj.dtype == np.float32 and a.obj.flags.c_contiguous
    assert a.ptr.value == a.obj.ctypes.data
    assert b._Arg(None, np.float32, 6).ptr is None
    torch = pytest.importorskip("torch")
    t = torch.arange(6, dtype=torch.float32)
    assert b._Arg(t, np.float32, 6).ptr.value == t.data_ptr()
    with pytest.raises(TypeError):
        b._Arg(torch.zeros(6, dtype=torch.float64), np.float32, 6, writable=True)
