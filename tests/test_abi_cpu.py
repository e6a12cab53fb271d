"""CPU checks of the boundary: the library builds, exports every symbol the header
declares, and rejects invalid arguments before touching the GPU."""
import os
import re

import numpy as np
import pytest

import paper_1909_02894_gb300 as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    D.build()
    return D.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "dirac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dirac_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(built):
    declared = header_functions()
    assert declared, "no functions found in include/dirac.h"
    for name in declared:
        assert hasattr(built, name), f"{name} declared in dirac.h but not exported"
    assert set(D.ABI_SYMBOLS) <= set(declared)


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(D, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(D, "_lib", None)
    with pytest.raises(ImportError):
        D.lib()


@pytest.mark.parametrize("kw,status", [
    (dict(nx=24, ny=32), D.DIRAC_EINVAL),            # not a power of two
    (dict(nx=8, ny=32), D.DIRAC_EINVAL),             # below 16
    (dict(nx=32, ny=8192), D.DIRAC_EINVAL),          # above 4096
    (dict(ax=0.0), D.DIRAC_EINVAL),
    (dict(c=-1.0), D.DIRAC_EINVAL),
    (dict(mass=float("nan")), D.DIRAC_EINVAL),
    (dict(pml_wx=16), D.DIRAC_EINVAL),               # width >= N/2
    (dict(pml_wx=4, pml_type=7), D.DIRAC_EINVAL),
    (dict(pml_wx=4, theta=0.3), D.DIRAC_EUNSUPPORTED),  # complex layer in complex64
    (dict(precision=5), D.DIRAC_EINVAL),
    (dict(conn=9), D.DIRAC_EINVAL),
    (dict(g11=-np.ones((32, 32))), D.DIRAC_EINVAL),  # non-positive metric
])
def test_create_validates_before_any_device_work(built, kw, status):
    args = dict(nx=32, ny=32, ax=1.0, ay=1.0)
    args.update(kw)
    nx, ny, ax, ay = args.pop("nx"), args.pop("ny"), args.pop("ax"), args.pop("ay")
    with pytest.raises(D.DiracError) as e:
        D.dirac_create(nx, ny, ax, ay, **args)
    assert e.value.status == status
    assert D.dirac_last_error(None)


def test_null_context_calls_are_rejected(built):
    L = built
    assert L.dirac_step(None, 1, 0.1) == D.DIRAC_EINVAL
    assert L.dirac_set_state(None, None, 0) == D.DIRAC_EINVAL
    assert L.dirac_get_state(None, None, 0) == D.DIRAC_EINVAL
    assert L.dirac_synchronize(None) == D.DIRAC_EINVAL
    assert L.dirac_launch_count(None) == 0
    L.dirac_destroy(None)  # NULL-safe
