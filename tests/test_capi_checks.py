"""CPU checks of the binding's argument checks: buffers that the C ABI would read or write
out of bounds, or read as the wrong element type, are refused with SEMD_EINVAL before any
library call (the library is replaced by a stub that fails the test if it is reached)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2106_15319_gb300 import capi  # noqa: E402


class FakeCuda:
    """Stands in for a CUDA tensor on a machine without one (no data is touched)."""

    def __init__(self, n, dtype, contiguous=True, shape=None):
        self.is_cuda = True
        self.device = torch.device("cuda", 0)
        self.dtype = dtype
        self._n = n
        self._c = contiguous
        self.shape = shape or (n,)

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        raise AssertionError("data pointer taken before the checks refused the call")


@pytest.fixture
def no_library(monkeypatch):
    def boom(*a, **k):
        raise AssertionError("the library was called")
    monkeypatch.setattr(capi, "load", boom)


def _refused(fn, *args, msg=None):
    with pytest.raises(capi.SemdError) as ei:
        fn(*args)
    assert ei.value.status == capi.SEMD_EINVAL
    if msg:
        assert msg in str(ei.value)


def test_noalloc_sift_refuses_mismatched_buffers(no_library):
    f32, f64 = torch.float32, torch.float64
    p64 = capi.semd_params(precision=capi.FP64)
    p32 = capi.semd_params(precision=capi.FP32_MIXED)
    # float32 data with an FP64 precision: the kernels would read 8 bytes per element
    _refused(capi.serial_emd_sift_noalloc, p64, FakeCuda(100, f32), FakeCuda(100, f64),
             msg="dtype")
    _refused(capi.serial_emd_sift_noalloc, p32, FakeCuda(100, f32), FakeCuda(100, f64),
             msg="dtype")
    # an output shorter than the input
    _refused(capi.serial_emd_sift_noalloc, p32, FakeCuda(100, f32), FakeCuda(99, f32),
             msg="elements")
    # non-contiguous, host tensors, unknown precision
    _refused(capi.serial_emd_sift_noalloc, p32, FakeCuda(100, f32, contiguous=False),
             FakeCuda(100, f32), msg="contiguous")
    _refused(capi.serial_emd_sift_noalloc, p32, torch.zeros(100), FakeCuda(100, f32),
             msg="CUDA")
    _refused(capi.serial_emd_sift_noalloc, capi.semd_params(precision=7), FakeCuda(100, f32),
             FakeCuda(100, f32))


def test_plan_calls_refuse_mismatched_buffers(no_library):
    f32, f64 = torch.float32, torch.float64
    plan = 0x1234  # a handle the binding knows the parameters of
    capi._PLAN_PARAMS[plan] = capi.semd_params(rows=4, cols=64, max_imfs=10,
                                               precision=capi.FP32_MIXED, transition_len=0,
                                               order=capi.ORDER_ROWS, ensemble_trials=1)
    try:
        _refused(capi.serial_emd_sift, plan, FakeCuda(256, f64), FakeCuda(256, f64),
                 msg="dtype")
        _refused(capi.serial_emd_sift, plan, FakeCuda(256, f32), FakeCuda(255, f32))
        _refused(capi.serial_emd_extrema, plan, FakeCuda(256, f32), FakeCuda(100, torch.int32),
                 FakeCuda(129, torch.int32), msg="tmax")
        _refused(capi.serial_emd_extrema, plan, FakeCuda(256, f32), FakeCuda(129, torch.int64),
                 FakeCuda(129, torch.int32))
        x = FakeCuda(256, f32, shape=(4, 64))
        _refused(capi.serial_emd_decompose, plan, x, None, FakeCuda(10 * 256 - 1, f32),
                 FakeCuda(256, f64), msg="imfs")
        _refused(capi.serial_emd_decompose, plan, x, None, FakeCuda(10 * 256, f32),
                 FakeCuda(256, f32), msg="residue")
        _refused(capi.serial_emd_decompose, plan, FakeCuda(256, f64, shape=(4, 64)), None,
                 FakeCuda(10 * 256, f32), None, msg="dtype")
        _refused(capi.serial_emd_decompose_batch, plan,
                 [(x, FakeCuda(2559, f32), None)], msg="imfs")
    finally:
        capi._PLAN_PARAMS.pop(plan, None)


def test_packed_batch_layout_and_refusals(no_library):
    """A packed batch: input i at the sum of the earlier inputs' sizes, its K IMFs at K
    times that offset, its residue at that offset (8-byte elements); buffers shorter than
    the batch, or shapes with a zero size, are refused before any library call."""
    f32, f64 = torch.float32, torch.float64
    plan = 0x4321
    capi._PLAN_PARAMS[plan] = capi.semd_params(rows=64, cols=64, max_imfs=3,
                                               precision=capi.FP32_MIXED, transition_len=0,
                                               order=capi.ORDER_ROWS, ensemble_trials=1)
    try:
        shapes = [(2, 3), (1, 5), (7, 1)]
        a = capi._packed_instance_array(plan, 1000, shapes, 50000, 90000)  # raw pointers
        assert list(a["x"]) == [1000, 1000 + 6 * 4, 1000 + 11 * 4]
        assert list(a["rows"]) == [2, 1, 7] and list(a["cols"]) == [3, 5, 1]
        assert list(a["imfs"]) == [50000, 50000 + 3 * 6 * 4, 50000 + 3 * 11 * 4]
        assert list(a["res"]) == [90000, 90000 + 6 * 8, 90000 + 11 * 8]
        assert list(capi._packed_instance_array(plan, 1000, shapes, 50000, None)["res"]) == \
            [0, 0, 0]
        total = 18
        _refused(capi.serial_emd_decompose_packed, plan, FakeCuda(total - 1, f32), shapes,
                 FakeCuda(3 * total, f32), None, msg="x")
        _refused(capi.serial_emd_decompose_packed, plan, FakeCuda(total, f32), shapes,
                 FakeCuda(3 * total - 1, f32), None, msg="imfs")
        _refused(capi.serial_emd_decompose_packed, plan, FakeCuda(total, f32), shapes,
                 FakeCuda(3 * total, f32), FakeCuda(total, f32), msg="residue")
        _refused(capi.serial_emd_decompose_packed, plan, FakeCuda(total, f64), shapes,
                 FakeCuda(3 * total, f32), None, msg="dtype")
        _refused(capi.serial_emd_decompose_packed, plan, FakeCuda(total, f32), [(2, 0)],
                 FakeCuda(3 * total, f32), None, msg="shapes")
    finally:
        capi._PLAN_PARAMS.pop(plan, None)
