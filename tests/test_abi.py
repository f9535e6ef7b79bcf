"""The C-ABI library builds, loads and exports every entry point that
include/gbla.h declares (no compute call: this runs without a GPU)."""
import os
import re

import pytest

from paper_1602_06097_gb300 import _build, gbla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gbla.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbla_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for name in ["gbla_reduce", "gbla_reduce_ex", "gbla_free", "gbla_strerror", "gbla_modmatmul"]:
        assert name in syms


def test_library_builds_and_exports_every_symbol():
    path = _build.build()
    assert os.path.exists(path)
    lib = gbla.load()
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} declared in gbla.h but not exported"
    assert set(gbla.EXPORTS) <= set(declared_symbols())


def test_binding_covers_every_entry_point():
    """The Python binding lists and declares every entry point of gbla.h."""
    lib = gbla.load()
    assert set(declared_symbols()) <= set(gbla.EXPORTS)
    for name in gbla.EXPORTS:
        assert getattr(lib, name).argtypes is not None, f"{name} has no declared argument types"


def test_strerror_and_version():
    lib = gbla.load()
    assert lib.gbla_version() >= 100
    assert gbla.strerror(0) == "ok"
    assert "invalid" in gbla.strerror(1)
    assert gbla.strerror(999) == "unknown error"


def test_invalid_prime_rejected_on_host():
    """Argument checks happen on the host before any device work."""
    import numpy as np
    with pytest.raises(gbla.GblaError) as e:
        gbla.reduce(np.array([0, 1]), np.array([0]), np.array([1]), (1, 1), 65535)
    assert e.value.code == 1


def _csr_in(m, n, nnz, rp=None, col=None, val=None):
    return gbla.CsrIn(m, n, nnz, rp, col, val)


@pytest.mark.parametrize("case", ["p not prime", "p too large", "p one", "negative rows", "entries without arrays",
                                  "rows without pointers", "bad product variant"])
def test_reduce_arguments_rejected_on_host(case):
    """The boundary's argument checks run on the host, before any device call:
    each bad argument gives GBLA_E_INVAL and a zeroed result."""
    import ctypes
    lib = gbla.load()
    import numpy as np
    rp = np.array([0, 1], np.int64)
    p, cin, variant = 65521, _csr_in(1, 1, 1, rp.ctypes.data, rp.ctypes.data, rp.ctypes.data), 0
    if case == "p not prime":
        p = 65535
    elif case == "p too large":
        p = 65537
    elif case == "p one":
        p = 1
    elif case == "negative rows":
        cin = _csr_in(-1, 1, 0)
    elif case == "entries without arrays":
        cin = _csr_in(1, 1, 1, rp.ctypes.data, None, None)
    elif case == "rows without pointers":
        cin = _csr_in(3, 1, 0, None, None, None)
    else:
        variant = 7
    out = gbla.CsrOut()
    out.nnz = 99
    rank = ctypes.c_int64(5)
    opt = gbla.Options(0, variant, 0, 0)
    rc = lib.gbla_reduce_ex(ctypes.byref(cin), p, ctypes.byref(opt), None, ctypes.byref(out), ctypes.byref(rank), None)
    assert rc == 1
    assert out.nnz == 0 and not out.row_ptr


def test_batch_and_server_arguments_rejected_on_host():
    import ctypes
    lib = gbla.load()
    assert lib.gbla_reduce_batch(-1, None, None, None, 0, None, None, None) == 1
    assert lib.gbla_reduce_batch(0, None, None, None, 0, None, None, None) == 0
    assert lib.gbla_server_create(0, 1, None) == 1
    assert lib.gbla_server_cancel(None, 1) == 1


def _format2_rc(buf):
    import ctypes
    lib = gbla.load()
    out = gbla.CsrOut()
    p = ctypes.c_uint32(0)
    return lib.gbla_decode_format2(buf, len(buf), None, ctypes.byref(out), ctypes.byref(p)), out


def test_format2_header_checks_on_host():
    """The decoder checks the file's fixed fields and section sizes on the host;
    a well-formed file then reaches the device check (GBLA_E_UNSUPPORTED on a
    machine without an sm_103a GPU)."""
    import struct
    from test_formats import hand_format2
    good = hand_format2(1, 251, "B", [5, 6, 7, 9, 3, 250])
    bad = [good[:10], good[:-1], good + b"\0",
           good[:12] + struct.pack("<Q", 1 << 16) + good[20:],          # p = 2^16
           good[:12] + struct.pack("<Q", 1) + good[20:],                # p = 1
           good[:52] + struct.pack("<Q", 1 << 40) + good[60:]]          # k far past the file
    for buf in bad:
        rc, out = _format2_rc(buf)
        assert rc == 1 and out.nnz == 0 and not out.row_ptr
    rc, _ = _format2_rc(good)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        assert rc == 6


def test_noalloc_binding_checks_its_tensors_before_the_library():
    """pivots_noalloc hands raw pointers to a library that writes ncols int64
    values through ``out``: wrong types, lengths, layouts and host tensors
    are rejected in Python (no GPU needed)."""
    torch = pytest.importorskip("torch")
    rp = torch.tensor([0, 1, 2], dtype=torch.int64)
    col = torch.tensor([0, 1], dtype=torch.int32)
    val = torch.tensor([1, 1], dtype=torch.int16)
    out = torch.empty(3, dtype=torch.int64)
    bad = [
        dict(out=torch.empty(2, dtype=torch.int64)),                 # shorter than ncols
        dict(out=torch.empty(3, dtype=torch.int32)),                 # wrong dtype
        dict(out=torch.empty(6, dtype=torch.int64)[::2]),            # not contiguous
        dict(row_ptr=torch.tensor([0, 2], dtype=torch.int64)),       # m + 1 entries expected
        dict(col=torch.tensor([0, 1], dtype=torch.int64)),           # int32 columns expected
        dict(val=torch.tensor([1, 1], dtype=torch.int32)),           # 16-bit values expected
        dict(val=torch.tensor([1], dtype=torch.int16)),              # col and val differ
        dict(row_ptr=[0, 1, 2]),                                     # not a tensor
        dict(),                                                      # host tensors
    ]
    for change in bad:
        args = dict(row_ptr=rp, col=col, val=val, out=out)
        args.update(change)
        with pytest.raises(ValueError):
            gbla.pivots_noalloc(args["row_ptr"], args["col"], args["val"], (2, 3), 7, args["out"])
