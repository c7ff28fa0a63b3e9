"""ctypes binding of the FP64 Serial-EMD oracle (``serial_emd_oracle.c``).

Test infrastructure only: the test suite, the smoke check and the CPU-baseline leg
of the benchmark use it. The CUDA library never imports or links anything here.

Each wrapper names the paper passage its C function follows (Zhang et al.,
arXiv 2106.15319): serialization Sec. 3.2, de-serialization Sec. 3.3, EMD Sec. 2.1
(Eq. 1, Steps 1-5), EEMD and CEEMDAN Sec. 2.2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "serial_emd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

STOP_FIXED, STOP_SD, STOP_SNUMBER = 0, 1, 2
BOUNDARY_MIRROR, BOUNDARY_ENDPOINTS = 0, 1
SPLINE_NOT_A_KNOT = 16  # added to a boundary code: not-a-knot spline ends (Reading 6b)

_dp = ctypes.POINTER(ctypes.c_double)
_ip32 = ctypes.POINTER(ctypes.c_int32)
_ip64 = ctypes.POINTER(ctypes.c_int64)
_ipint = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc. -ffp-contract=off keeps x86 and Arm results equal."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_serial_length.restype = _i64
            L.oracle_serial_length.argtypes = [_i64, _i64, _i64]
            L.oracle_serialize.argtypes = [_dp, _i64, _i64, _i64, _dp]
            L.oracle_deserialize.argtypes = [_dp, _i64, _i64, _i64, _i64, _dp]
            L.oracle_extrema.argtypes = [_dp, _i64, _ip32, _ip64, _ip32, _ip64]
            L.oracle_spline_second_derivs.argtypes = [_dp, _dp, _i64, _dp]
            L.oracle_spline_second_derivs_nak.argtypes = [_dp, _dp, _i64, _dp]
            L.oracle_envelope.argtypes = [_dp, _i64, _ip32, _i64, ctypes.c_int, ctypes.c_int,
                                          _dp]
            L.oracle_sift.restype = ctypes.c_int
            L.oracle_sift.argtypes = [_dp, _i64, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            L.oracle_emd.restype = ctypes.c_int
            L.oracle_emd.argtypes = [_dp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     _dp, _dp, _ipint, ctypes.c_int]
            L.oracle_zero_crossings.restype = _i64
            L.oracle_zero_crossings.argtypes = [_dp, _i64]
            L.oracle_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32),
                                               ctypes.POINTER(ctypes.c_uint32),
                                               ctypes.POINTER(ctypes.c_uint32)]
            L.oracle_white_noise.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _i64,
                                             _dp]
            L.oracle_std.restype = ctypes.c_double
            L.oracle_std.argtypes = [_dp, _i64]
            L.oracle_eemd.restype = ctypes.c_int
            L.oracle_eemd.argtypes = [_dp, _i64, _dp, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                      ctypes.c_int]
            L.oracle_serial_emd.restype = ctypes.c_int
            L.oracle_serial_emd.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, _dp, _dp, _dp, _ipint, ctypes.c_int]
            L.oracle_ceemdan.restype = ctypes.c_int
            L.oracle_ceemdan.argtypes = [_dp, _i64, _dp, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _dp, _dp, ctypes.c_int]
            L.oracle_serial_ceemdan.restype = ctypes.c_int
            L.oracle_serial_ceemdan.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                                ctypes.c_int]
            _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def serial_length(M: int, N: int, D: int) -> int:
    """Sec. 3.2: L = MN + DN - D."""
    return int(lib().oracle_serial_length(M, N, D))


def serialize(X, D: int) -> np.ndarray:
    """Sec. 3.2. X is (N, M): N signals of length M (row i = the paper's column x_i)."""
    X = _f64(X)
    N, M = X.shape
    x = np.empty(serial_length(M, N, D), np.float64)
    lib().oracle_serialize(_d(X), M, N, D, _d(x))
    return x


def deserialize(R, M: int, N: int, D: int) -> np.ndarray:
    """Sec. 3.3. R is (K, L); returns (K, N, M)."""
    R = _f64(np.atleast_2d(R))
    K = R.shape[0]
    out = np.empty((K, N, M), np.float64)
    lib().oracle_deserialize(_d(R), K, M, N, D, _d(out))
    return out


def extrema(h):
    """Sec. 2.1 Step 1 (extremum rule of the oracle header). Returns (t_max, t_min)."""
    h = _f64(h)
    L = h.size
    a = np.empty(max(L, 1), np.int32)
    b = np.empty(max(L, 1), np.int32)
    na, nb = ctypes.c_int64(), ctypes.c_int64()
    lib().oracle_extrema(_d(h), L, a.ctypes.data_as(_ip32), ctypes.byref(na),
                         b.ctypes.data_as(_ip32), ctypes.byref(nb))
    return a[:na.value].copy(), b[:nb.value].copy()


def spline_second_derivs(s, v, not_a_knot: bool = False) -> np.ndarray:
    """Cubic spline second derivatives (Thomas algorithm): natural ends, or not-a-knot
    ends (Reading 6b)."""
    s, v = _f64(s), _f64(v)
    out = np.empty(s.size, np.float64)
    fn = lib().oracle_spline_second_derivs_nak if not_a_knot else \
        lib().oracle_spline_second_derivs
    fn(_d(s), _d(v), s.size, _d(out))
    return out


def envelope(h, t, boundary: int = BOUNDARY_MIRROR, mirror_knots: int = 2) -> np.ndarray:
    """Sec. 2.1 Step 2: the spline envelope through the knots t of h, at every sample."""
    h = _f64(h)
    t = np.ascontiguousarray(np.asarray(t, np.int32))
    out = np.empty(h.size, np.float64)
    lib().oracle_envelope(_d(h), h.size, t.ctypes.data_as(_ip32), t.size, boundary,
                          mirror_knots, _d(out))
    return out


def sift(h, boundary: int = BOUNDARY_MIRROR, mirror_knots: int = 2):
    """Sec. 2.1 Steps 1-4: returns (h - m, sum (h - h')^2, sum h^2) or None."""
    h = _f64(h)
    out = np.empty(h.size, np.float64)
    num, den = ctypes.c_double(), ctypes.c_double()
    rc = lib().oracle_sift(_d(h), h.size, boundary, mirror_knots, _d(out), ctypes.byref(num),
                           ctypes.byref(den))
    if rc != 0:
        return None
    return out, num.value, den.value


def emd(x, K: int, stop: int = STOP_FIXED, fixed_sifts: int = 10, sd_threshold: float = 0.2,
        max_sifts: int = 50, boundary: int = BOUNDARY_MIRROR, mirror_knots: int = 2,
        store_f32: bool = False, s_number: int = 4):
    """Sec. 2.1: returns (imfs (K, L) zero-filled, residue (L,), n_imfs, sifts per IMF).

    store_f32 rounds the sifted signal to single precision where the FP32 form stores it.
    Under the S-number rule (stop = STOP_SNUMBER) s_number is S.
    """
    if stop == STOP_SNUMBER:
        fixed_sifts = s_number
    x = _f64(x)
    L = x.size
    imfs = np.empty((K, L), np.float64)
    res = np.empty(L, np.float64)
    sifts = np.zeros(K, np.int32)
    n = lib().oracle_emd(_d(x), L, K, stop, fixed_sifts, sd_threshold, max_sifts, boundary,
                         mirror_knots, _d(imfs), _d(res),
                         sifts.ctypes.data_as(_ipint), int(store_f32))
    return imfs, res, int(n), sifts


def std(x) -> float:
    x = _f64(x)
    return float(lib().oracle_std(_d(x), x.size))


def eemd(x, w, beta: float, K: int, stop: int = STOP_FIXED, fixed_sifts: int = 10,
         sd_threshold: float = 0.2, max_sifts: int = 50, boundary: int = BOUNDARY_MIRROR,
         mirror_knots: int = 2, store_f32: bool = False):
    """Sec. 2.2: w is (trials, L). Returns (mean imfs (K, L), mean residue, max n_imfs)."""
    x, w = _f64(x), _f64(w)
    trials, L = w.shape
    assert L == x.size
    imfs = np.empty((K, L), np.float64)
    res = np.empty(L, np.float64)
    n = lib().oracle_eemd(_d(x), L, _d(w), trials, beta, K, stop, fixed_sifts, sd_threshold,
                          max_sifts, boundary, mirror_knots, _d(imfs), _d(res), int(store_f32))
    return imfs, res, int(n)


def serial_emd(X, D: int, K: int, stop: int = STOP_FIXED, fixed_sifts: int = 10,
               sd_threshold: float = 0.2, max_sifts: int = 50, boundary: int = BOUNDARY_MIRROR,
               mirror_knots: int = 2, trials: int = 1, noise_rel_std: float = 0.0, w=None,
               store_f32: bool = False, s_number: int = 4):
    """Sec. 3: serialize, EMD/EEMD, de-serialize. X is (N, M).

    Returns (imfs (K, N, M), residue (N, M), n_imfs, sifts per IMF (EMD only)).
    Under the S-number rule (stop = STOP_SNUMBER) s_number is S.
    """
    if stop == STOP_SNUMBER:
        fixed_sifts = s_number
    X = _f64(X)
    N, M = X.shape
    L = serial_length(M, N, D)
    imfs = np.empty((K, N, M), np.float64)
    res = np.empty((N, M), np.float64)
    sifts = np.zeros(K, np.int32)
    if trials > 1:
        w = _f64(w)
        assert w.shape == (trials, L)
        wp = _d(w)
    else:
        wp = None
    n = lib().oracle_serial_emd(_d(X), M, N, D, K, stop, fixed_sifts, sd_threshold, max_sifts,
                                boundary, mirror_knots, trials, noise_rel_std, wp, _d(imfs),
                                _d(res), sifts.ctypes.data_as(_ipint), int(store_f32))
    return imfs, res, int(n), sifts


def ceemdan(x, w, noise_rel_std: float, K: int, stop: int = STOP_FIXED, fixed_sifts: int = 10,
            sd_threshold: float = 0.2, max_sifts: int = 50, boundary: int = BOUNDARY_MIRROR,
            mirror_knots: int = 2, store_f32: bool = False, s_number: int = 4):
    """Sec. 2.2 CEEMDAN (Steps 1-4; Reading 12 of the C source): w is (trials, L).

    Returns (modes (K, L), residue (L), number of modes)."""
    if stop == STOP_SNUMBER:
        fixed_sifts = s_number
    x, w = _f64(x), _f64(w)
    trials, L = w.shape
    assert L == x.size
    modes = np.empty((K, L), np.float64)
    res = np.empty(L, np.float64)
    n = lib().oracle_ceemdan(_d(x), L, _d(w), trials, noise_rel_std, K, stop, fixed_sifts,
                             sd_threshold, max_sifts, boundary, mirror_knots, _d(modes),
                             _d(res), int(store_f32))
    return modes, res, int(n)


def serial_ceemdan(X, D: int, K: int, w, noise_rel_std: float, stop: int = STOP_FIXED,
                   fixed_sifts: int = 10, sd_threshold: float = 0.2, max_sifts: int = 50,
                   boundary: int = BOUNDARY_MIRROR, mirror_knots: int = 2,
                   store_f32: bool = False, s_number: int = 4):
    """Sec. 3 with CEEMDAN as the decomposition: serialize, CEEMDAN, de-serialize.
    X is (N, M), w is (trials, L). Returns (modes (K, N, M), residue (N, M), count)."""
    if stop == STOP_SNUMBER:
        fixed_sifts = s_number
    X, w = _f64(X), _f64(w)
    N, M = X.shape
    L = serial_length(M, N, D)
    trials = w.shape[0]
    assert w.shape == (trials, L)
    modes = np.empty((K, N, M), np.float64)
    res = np.empty((N, M), np.float64)
    n = lib().oracle_serial_ceemdan(_d(X), M, N, D, K, stop, fixed_sifts, sd_threshold,
                                    max_sifts, boundary, mirror_knots, trials, noise_rel_std,
                                    _d(w), _d(modes), _d(res), int(store_f32))
    return modes, res, int(n)


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al., SC 2011) of 4 counter and 2 key words."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def white_noise(seed: int, trials: int, L: int, first: int = 0) -> np.ndarray:
    """Reading 11b: the white noise the library draws itself for EEMD, realizations
    first .. first + trials - 1, (trials, L)."""
    w = np.empty((trials, L), np.float64)
    lib().oracle_white_noise(ctypes.c_uint64(seed), first, trials, L, _d(w))
    return w


def zero_crossings(h) -> int:
    """Reading 8b: pairs (k, k+1) of h with exactly one negative sample."""
    h = _f64(h)
    return int(lib().oracle_zero_crossings(_d(h), h.size))
