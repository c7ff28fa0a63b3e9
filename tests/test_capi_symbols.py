"""CPU checks of the boundary: the library builds, loads without a GPU, and exports
every entry point that include/serial_emd.h declares (no compute calls here)."""
import ctypes
import math
import os
import re

import numpy as np
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


def _documented_valid(kw) -> bool:
    """The parameter rules that include/serial_emd.h documents, restated in Python."""
    if kw["rows"] < 1 or kw["cols"] < 1:
        return False
    if kw["order"] not in (capi.ORDER_ROWS, capi.ORDER_COLS):
        return False
    if not 1 <= kw["max_imfs"] <= 32:
        return False
    stop = kw["stop"]
    if stop == capi.STOP_FIXED:
        if not 1 <= kw["fixed_sifts"] <= 1000:
            return False
    elif stop == capi.STOP_SD:
        if not (1 <= kw["max_sifts"] <= 1000 and kw["sd_threshold"] >= 0):
            return False
    elif stop == capi.STOP_SNUMBER:
        if not (1 <= kw["max_sifts"] <= 1000 and 1 <= kw["s_number"] <= 1000):
            return False
    else:
        return False
    if kw["boundary"] == capi.BOUNDARY_MIRROR:
        if kw["mirror_knots"] not in (1, 2):
            return False
    elif kw["boundary"] != capi.BOUNDARY_ENDPOINTS:
        return False
    if kw["precision"] not in (capi.FP64, capi.FP32_MIXED):
        return False
    if kw["spline_end"] not in (capi.SPLINE_NATURAL, capi.SPLINE_NOT_A_KNOT):
        return False
    if kw["ensemble_trials"] > 1 and not kw["noise_rel_std"] >= 0:
        return False
    if kw["transition_len"] < -1:
        return False
    rows_axis = kw["order"] == capi.ORDER_ROWS
    M, N = (kw["cols"], kw["rows"]) if rows_axis else (kw["rows"], kw["cols"])
    D = int(math.floor(0.2 * M + 0.5)) if kw["transition_len"] < 0 else kw["transition_len"]
    if N == 1:
        D = 0
    if D > M:
        return False
    return M * N + D * N - D < (1 << 30)


def test_random_params_follow_the_documented_rules():
    """Seeded random parameter sets, each field drawn from valid values, edges and invalid
    values: serial_emd_plan rejects exactly the sets that break a documented rule with
    EINVAL, before any device use. Without a GPU the valid sets end in ECUDA; on a GPU machine
    only the invalid sets are tried (a valid one would allocate)."""
    import torch
    gpu = torch.cuda.is_available()
    g = np.random.default_rng(90210)

    def pick(good, bad=()):
        # mostly values that the rules allow (edges included), sometimes ones they reject
        pool = good if not bad or g.uniform() < 0.93 else bad
        return pool[int(g.integers(len(pool)))]

    n_valid = n_invalid = 0
    for _ in range(3000):
        kw = dict(
            rows=pick([1, 2, 3, 64, 1000, 40000, 1 << 20], [0, -5]),
            cols=pick([1, 2, 5, 64, 1000, 40000, 1 << 20], [0, -1]),
            order=pick([capi.ORDER_ROWS, capi.ORDER_COLS], [2, -1]),
            transition_len=pick([-1, 0, 1, 3, 64, 999, 1000, 50000], [-2, -7]),
            max_imfs=pick([1, 10, 32], [0, 33]),
            stop=pick([capi.STOP_FIXED, capi.STOP_SD, capi.STOP_SNUMBER], [3, -1]),
            fixed_sifts=pick([1, 10, 1000], [0, 1001]),
            max_sifts=pick([1, 50, 1000], [0, 1001]),
            sd_threshold=pick([0.0, 0.2, 5.0], [-0.1, float("nan")]),
            boundary=pick([capi.BOUNDARY_MIRROR, capi.BOUNDARY_ENDPOINTS], [2]),
            mirror_knots=pick([1, 2], [0, 3]),
            precision=pick([capi.FP64, capi.FP32_MIXED], [2]),
            ensemble_trials=pick([-3, 0, 1, 2, 100]),  # <= 1 is EMD
            noise_rel_std=pick([0.0, 0.2], [-1.0, float("nan")]),
            s_number=pick([1, 4, 1000], [0, 1001]),
            spline_end=pick([capi.SPLINE_NATURAL, capi.SPLINE_NOT_A_KNOT], [2]))
        valid = _documented_valid(kw)
        if valid and gpu:
            continue
        p = capi.serial_emd_default_params(**kw)
        with pytest.raises(capi.SemdError) as ei:
            capi.serial_emd_plan(p, 1, 0)
        want = capi.SEMD_ECUDA if valid else capi.SEMD_EINVAL
        assert ei.value.status == want, (kw, ei.value)
        n_valid += valid
        n_invalid += not valid
    assert n_invalid > 500 and (gpu or n_valid > 300), (n_valid, n_invalid)
