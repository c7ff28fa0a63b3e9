"""The allocation-free sift (serial_emd_sift_noalloc) against the plan-based one.

Some callers cannot reserve device memory at the point where they sift: plug-ins
inside a framework whose caching allocator owns the device memory, real-time paths
that forbid allocation after start-up, code under a hard device-memory cap. For them
the library keeps the scratch of one sift in a static device array. This test calls that entry point through the C ABI
twice in a row, on different inputs and lengths, and checks each result against
serial_emd_sift on the same input and against the FP64 oracle's single sift (O.sift),
within the tolerance of the other single-sift parity test (1e-12 relative in FP64, 2e-5
in FP32), with natural and with not-a-knot spline ends. It also checks that a length
past the array's limit is refused with a clear error. The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2106_15319_gb300 import capi, synth  # noqa: E402
from paper_2106_15319_gb300.serial_emd import Plan, make_params  # noqa: E402

NP = {capi.FP64: np.float64, capi.FP32_MIXED: np.float32}
TOL = {capi.FP64: 1e-12, capi.FP32_MIXED: 2e-5}
MAX_L = 65536


def _signal(L, seed):
    g = synth.rng(seed)
    t = np.arange(L)
    return np.sin(t / 5.0) + 0.3 * g.standard_normal(L) + 0.5 * np.sin(t / 97.0)


@pytest.mark.parametrize("end", [capi.SPLINE_NATURAL, capi.SPLINE_NOT_A_KNOT])
@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_noalloc_sift_matches_plan_sift_twice(prec, end):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()
    params = make_params(1, MAX_L, precision=prec, spline_end=end)
    plan = Plan(params)
    ob = O.BOUNDARY_MIRROR + (O.SPLINE_NOT_A_KNOT if end == capi.SPLINE_NOT_A_KNOT else 0)
    try:
        for L, seed in ((MAX_L, 11), (3001, 12)):
            hx = _signal(L, seed).astype(NP[prec])
            h = torch.from_numpy(hx).cuda()
            ref, rnum, rden = plan.sift(h)
            out = torch.full_like(h, float("nan"))
            num, den = capi.serial_emd_sift_noalloc(params, h, out)
            torch.cuda.synchronize()
            got, want = out.double().cpu().numpy(), ref.double().cpu().numpy()
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert err <= TOL[prec], (L, err)
            assert abs(num - rnum) <= TOL[prec] * 10 * rnum, (num, rnum)
            assert abs(den - rden) <= TOL[prec] * 10 * rden, (den, rden)
            # and directly against the oracle's single sift of the same stored input
            o_out, o_num, o_den = O.sift(hx.astype(np.float64), boundary=ob, mirror_knots=2)
            err = np.linalg.norm(got - o_out) / np.linalg.norm(o_out)
            assert err <= TOL[prec], (L, "oracle", err)
            assert abs(num - o_num) <= TOL[prec] * 10 * o_num, (num, o_num)
            assert abs(den - o_den) <= TOL[prec] * 10 * o_den, (den, o_den)
    finally:
        plan.close()


def test_noalloc_sift_rejects_unknown_spline_end():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    params = make_params(1, 8, precision=capi.FP32_MIXED)
    params.spline_end = 2
    h = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(capi.SemdError) as ei:
        capi.serial_emd_sift_noalloc(params, h, torch.empty_like(h))
    assert ei.value.status == capi.SEMD_EINVAL
    assert "spline_end" in str(ei.value)


def test_noalloc_sift_rejects_lengths_past_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    params = make_params(1, 8, precision=capi.FP32_MIXED)
    h = torch.zeros(MAX_L + 1, dtype=torch.float32, device="cuda")
    out = torch.empty_like(h)
    with pytest.raises(capi.SemdError) as ei:
        capi.serial_emd_sift_noalloc(params, h, out)
    assert ei.value.status == capi.SEMD_EINVAL
    assert "65536" in str(ei.value)
