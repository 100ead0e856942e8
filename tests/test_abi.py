"""The C-ABI library loads and exports every entry point include/*.h
declares; host-side argument validation (no device work)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(al_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def _lib():
    from paper_2609_39443_b300 import al
    return al.lib()


def test_header_declares_the_core_entry_points():
    names = _declared()
    for n in ("al_create_grid", "al_load_beams", "al_sample_drag_spread", "al_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = _lib()
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_argument_errors_are_reported_before_any_device_work():
    from paper_2609_39443_b300 import al
    L = _lib()
    h = C.c_void_p()
    assert L.al_create_grid(None, C.byref(h)) == al.AL_ERR_ARG
    bad = [dict(nx=0), dict(dx=0.0), dict(dx=float("nan")), dict(precision=7), dict(has_alpha=1, rho1=0.0)]
    for kw in bad:
        base = dict(nx=4, ny=4, nz=4, dx=0.1, precision=al.AL_FP32, has_alpha=0, rho1=1000.0, rho2=1.2,
                    rho_const=1000.0)
        base.update(kw)
        d = al.GridDesc(base["nx"], base["ny"], base["nz"], base["dx"], (C.c_double * 3)(0, 0, 0),
                        base["precision"], base["has_alpha"], base["rho1"], base["rho2"], base["rho_const"])
        assert L.al_create_grid(C.byref(d), C.byref(h)) == al.AL_ERR_ARG, kw
    assert L.al_load_beams(None, None) == al.AL_ERR_ARG
    assert L.al_sample_drag_spread(None, None, None, None) == al.AL_ERR_ARG
    assert L.al_destroy(None) == al.AL_ERR_ARG
    assert L.al_error_string(al.AL_ERR_ARG) == b"invalid argument"


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2609_39443_b300 import al
    monkeypatch.setattr(al, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(al, "_lib", None)
    with pytest.raises(al.ALError):
        al.lib()
