"""CPU checks of the boundary: the library builds, loads without a GPU, and exports
every entry point that include/serial_emd.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2106_15319_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "serial_emd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(serial_emd_\w+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("serial_emd_plan", "serial_emd_decompose", "serial_emd_submit", "serial_emd_poll",
              "serial_emd_destroy", "serial_emd_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_declared()) == set(capi.SIGNATURES)


def test_params_struct_layout_and_defaults():
    p = capi.serial_emd_default_params()
    assert ctypes.sizeof(capi.semd_params) == 80
    assert (p.max_imfs, p.fixed_sifts, p.mirror_knots, p.transition_len) == (10, 10, 2, -1)
    assert (p.s_number, p.spline_end) == (4, capi.SPLINE_NATURAL)
    assert p.sd_threshold == pytest.approx(0.2)


def test_plan_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = capi.serial_emd_default_params(rows=4, cols=64)
    with pytest.raises(capi.SemdError) as ei:
        capi.serial_emd_plan(p, 1, 0)
    assert ei.value.status == capi.SEMD_ECUDA


def test_invalid_params_rejected_before_device_use():
    bad = [dict(max_imfs=0), dict(max_imfs=33), dict(fixed_sifts=0), dict(mirror_knots=3),
           dict(order=5), dict(precision=7), dict(transition_len=-2), dict(stop=3),
           dict(stop=capi.STOP_SNUMBER, s_number=0),
           dict(stop=capi.STOP_SNUMBER, max_sifts=0), dict(spline_end=2)]
    for kw in bad:
        p = capi.serial_emd_default_params(rows=4, cols=64, **kw)
        with pytest.raises(capi.SemdError) as ei:
            capi.serial_emd_plan(p, 1, 0)
        assert ei.value.status == capi.SEMD_EINVAL, kw
    p = capi.serial_emd_default_params(rows=4, cols=8, transition_len=9)
    with pytest.raises(capi.SemdError) as ei:
        capi.serial_emd_plan(p, 1, 0)
    assert ei.value.status == capi.SEMD_EINVAL


def test_server_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = capi.serial_emd_default_params(rows=4, cols=64)
    with pytest.raises(capi.SemdError) as ei:
        capi.serial_emd_server_create(p, 1 << 20, 2)
    assert ei.value.status == capi.SEMD_ECUDA
    with pytest.raises(capi.SemdError) as ei:
        capi.serial_emd_server_create(p, 0, 2)
    assert ei.value.status == capi.SEMD_EINVAL
