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
