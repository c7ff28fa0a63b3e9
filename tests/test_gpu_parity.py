"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 per-IMF relative L2 <= 1e-10 (the denominator has a floor of
1e-6 * ||x||); knot indices bit-exact. Inputs for the FP32 form are rounded to
float32 first, and the oracle decomposes the rounded values, so both sides start
from the same numbers.

FP32-mixed: the signal is stored and sifted in single precision, the residue is
kept in FP64. Each IMF is checked against the oracle's IMF of the same input
remainder: the GPU's remainder before IMF k is x minus its own IMFs 1..k-1, an
FP64 sequence of subtractions the test repeats exactly, and the GPU starts IMF k
from that remainder rounded to single precision. The oracle starts from the same
rounded values, so both sides decide from identical numbers whether another IMF
exists (the IMF count must match exactly); the residue must equal the FP64
sequence to rounding. The FP32 tolerance (1e-4 of the IMF's norm) presumes, like
the FP64 one, that both sides sift with the same knots. So for every IMF the test
replays the GPU's own FP32 sift chain (single sifts through the C ABI, with the
decomposition's pass shape; the replay must reproduce the decomposition's IMF bit
for bit) beside the oracle's FP64 chain from the same input, and compares their
knot decisions sift by sift. Where every decision agrees, the IMF must be within
1e-4. Where one differs, the test requires that the decision was one single
precision cannot resolve: the comparison that decides it must differ by at most
2^-20 of the IMF input's max|h| in the FP64 chain (a near-flat step or a near-flat extremum, where
rounding picks the side). Such an IMF is exempt from the bar and counted. Inputs
with transitions (D > 0) drop transition samples from the outputs, so there the
unconditional bar applies: the two leading IMFs within 1e-4 of their norm, every
later IMF and the tail sum within 1e-3 of ||x||, IMF counts at most one apart.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2106_15319_gb300 import capi, synth  # noqa: E402
from paper_2106_15319_gb300.serial_emd import Plan, make_params  # noqa: E402

TOL = {capi.FP64: 1e-10, capi.FP32_MIXED: 1e-4}
NP = {capi.FP64: np.float64, capi.FP32_MIXED: np.float32}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()


def _rel(a, b, floor):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)


def _check_imfs(imfs_g, res_g, n_g, imfs_o, res_o, n_o, x, prec, what=""):
    nx = np.linalg.norm(x)
    floor = max(1e-6 * nx, 1e-300)  # an all-zero input has a zero norm
    K = imfs_o.shape[0]
    errs = [_rel(imfs_g[k], imfs_o[k], floor) for k in range(K)]
    rerr = _rel(res_g, res_o, floor)
    if prec == capi.FP64:
        assert n_g == n_o, f"{what}: IMF count {n_g} vs {n_o}"
        assert max(errs) <= TOL[prec] and rerr <= TOL[prec], f"{what}: {errs} res {rerr}"
        return errs
    assert abs(n_g - n_o) <= 1, f"{what}: IMF count {n_g} vs {n_o}"
    tail0 = max(min(n_g, n_o) - 1, 0)
    lead = errs[:min(2, tail0)]
    assert max(lead, default=0.0) <= TOL[prec], f"{what}: leading IMFs {lead} (all {errs})"
    nx = max(nx, 1e-300)
    absn = [np.linalg.norm(imfs_g[k] - imfs_o[k]) / nx for k in range(tail0)]
    tail = imfs_g[tail0:].sum(0) + res_g - imfs_o[tail0:].sum(0) - res_o
    absn.append(np.linalg.norm(tail) / nx)
    assert max(absn) <= 1e-3, f"{what}: |dc|/|x| {absn} (rel {errs}; n {n_g} vs {n_o})"
    return errs


# Single-precision knot decisions. A knot decision of Step 1 at sample q rests on the two
# comparisons (q-1, q) and (q, q+1). FP32 arithmetic and storage move every sample of a
# sifted signal by a few units in the last place of the scale of the IMF's input; a
# comparison whose FP64 difference is within FP32_TAU of that scale can therefore come out
# either way, and the rounding decides it. When that happens the FP32 and FP64 sift chains use different knot
# sets from that sift on, and the IMF may move by far more than the FP32 bar (a knot moved
# by one sample changes a slow IMF at the percent level).
FP32_TAU = 2.0 ** -20
# The SD ratio's sums run in single precision per tile (about 1e-6 relative); a stop
# decision may differ only where the FP64 ratio is within this relative distance of the
# threshold.
FP32_SD_TAU = 1e-4

_SIFT_PLANS = {}


def _sift_plan(L, shape, boundary, mirror_knots):
    """A single-sift FP32 plan with the decomposition's pass shape (tile, variant) and
    envelope rule (the oracle's boundary code: rule + not-a-knot flag)."""
    key = (L, shape, boundary, mirror_knots)
    if key not in _SIFT_PLANS:
        if len(_SIFT_PLANS) > 8:
            for pl in _SIFT_PLANS.values():
                pl.close()
            _SIFT_PLANS.clear()
        nak = boundary & O.SPLINE_NOT_A_KNOT
        pl = Plan(make_params(1, max(L, 8), precision=capi.FP32_MIXED,
                              boundary=boundary & ~O.SPLINE_NOT_A_KNOT,
                              mirror_knots=mirror_knots,
                              spline_end=capi.SPLINE_NOT_A_KNOT if nak else capi.SPLINE_NATURAL))
        pl.tile, pl.pass_variant = shape
        _SIFT_PLANS[key] = pl
    return _SIFT_PLANS[key]


@pytest.fixture(scope="module", autouse=True)
def _close_sift_plans():
    yield
    for pl in _SIFT_PLANS.values():
        pl.close()
    _SIFT_PLANS.clear()


def _enough_extrema(h):
    """Reading 9's test: at least one maximum, one minimum and three extrema."""
    a, b = O.extrema(h)
    return a.size >= 1 and b.size >= 1 and a.size + b.size >= 3


def _decision_margin(o, qs, scale):
    """The largest, over the samples qs whose knot decisions differ, of the smaller FP64
    difference of the two comparisons that decide the sample, relative to `scale`: the
    magnitude of the IMF's single-precision input. The FP32 form's errors are absolute
    errors of that scale (the first sift subtracts a mean envelope of the input's size, in
    single precision), and they stay in the signal through the later sifts."""
    m = 0.0
    for q in qs:
        d = [abs(o[q] - o[q - 1])] if q >= 1 else []
        if q + 1 < o.size:
            d.append(abs(o[q + 1] - o[q]))
        m = max(m, min(d))
    return m / max(scale, 1e-300)


def _fp32_chain(h32, S, shape, boundary=O.BOUNDARY_MIRROR, mirror_knots=2, sd=None):
    """Replays one IMF's sifting two ways from the same single-precision input: the GPU's
    own FP32 chain (single sifts through the C ABI with the decomposition's pass shape) and
    the oracle's FP64 chain. Returns (GPU result, sifts, None) when every sift of both
    chains took the same knot decisions (and, with sd = (threshold, max_sifts), the same
    stop decisions), else (None, sift index, (kind, margin)) for the first differing
    decision: for a knot decision the relative FP64 difference of its deciding
    comparison, for a stop decision the relative distance of the FP64 SD ratio from the
    threshold."""
    sp = _sift_plan(h32.size, shape, boundary, mirror_knots)
    g = h32.astype(np.float32)
    o = h32.copy()
    cap = S if sd is None else sd[1]
    j = 0
    while j < cap:
        gd = g.astype(np.float64)
        ga, gb = O.extrema(gd)
        oa, ob = O.extrema(o)
        if not (np.array_equal(ga, oa) and np.array_equal(gb, ob)):
            qs = np.concatenate([np.setxor1d(ga, oa), np.setxor1d(gb, ob)])
            return None, j, ("knot", _decision_margin(o, qs, max(np.abs(h32).max(),
                                                                  np.abs(o).max())))
        if j > 0 and not _enough_extrema(o):
            break
        out, gnum, gden = sp.sift(torch.from_numpy(g).cuda())
        g = out.cpu().numpy()
        o_next, onum, oden = O.sift(o, boundary=boundary, mirror_knots=mirror_knots)
        o = o_next
        j += 1
        if sd is not None:
            gstop, ostop = gnum / gden < sd[0], onum / oden < sd[0]
            if gstop != ostop:
                return None, j, ("stop", abs(onum / oden / sd[0] - 1.0))
            if ostop:
                break
    return g.astype(np.float64), j, None


def _check_fp32_given_input(imfs_g, res_g, n_g, x, K, what="", S=10,
                            boundary=O.BOUNDARY_MIRROR, mirror_knots=2, shape=(256, 0),
                            sd=None, sifts_g=None):
    """FP32 parity of every IMF against the oracle's IMF of the same remainder (D = 0,
    so the serialized signal is x flattened). Per IMF, the GPU's FP32 sift chain is
    replayed beside the oracle's FP64 chain from the same single-precision input:
    - same knot (and stop) decisions at every sift: the replay must equal the
      decomposition's IMF bit for bit, and the IMF must be within 1e-4 of the oracle's;
    - a differing decision: allowed only where its FP64 margin is within FP32_TAU (a
      comparison that single precision cannot resolve); the IMF is then reported as
      exempt, and from that sift on the two chains sift different knot sets."""
    x = np.asarray(x, np.float64).reshape(-1)
    c = np.asarray(imfs_g, np.float64).reshape(K, -1)
    floor = max(1e-6 * np.linalg.norm(x), 1e-300)
    r = x.copy()
    errs, exempt = [], []
    stop_kw = {} if sd is None else dict(stop=O.STOP_SD, sd_threshold=sd[0], max_sifts=sd[1])
    for k in range(n_g):
        h32 = r.astype(np.float32).astype(np.float64)
        oi, _, on, os_ = O.emd(h32, 1, fixed_sifts=S, boundary=boundary,
                               mirror_knots=mirror_knots, **stop_kw)
        assert on == 1, f"{what}: the oracle finds no IMF {k + 1} in the GPU's remainder"
        errs.append(_rel(c[k], oi[0], floor))
        g, j, margin = _fp32_chain(h32, S, shape, boundary, mirror_knots, sd)
        if margin is None:
            exempt.append(False)
            assert np.array_equal(g, c[k]), f"{what}: IMF {k + 1} replay differs"
            if sifts_g is not None:
                assert int(sifts_g[k]) == j == int(os_[0]), \
                    f"{what}: IMF {k + 1} sifts {sifts_g[k]} / replay {j} / oracle {os_[0]}"
            assert errs[-1] <= TOL[capi.FP32_MIXED], \
                f"{what}: IMF {k + 1} error {errs[-1]} with matching decisions (all {errs})"
        else:
            exempt.append(True)
            kind, m = margin
            assert m <= (FP32_TAU if kind == "knot" else FP32_SD_TAU), \
                f"{what}: IMF {k + 1} {kind} decisions differ at sift {j} with margin {m}"
        r = r - c[k]
    if n_g < K:
        _, _, on, _ = O.emd(r.astype(np.float32).astype(np.float64), 1, fixed_sifts=S,
                            boundary=boundary, mirror_knots=mirror_knots, **stop_kw)
        assert on == 0, f"{what}: the GPU stopped after {n_g} IMFs, the oracle continues"
    assert np.all(c[n_g:] == 0.0), f"{what}: IMF slots past the count are not zero"
    rn = np.asarray(res_g, np.float64).reshape(-1)
    assert np.abs(rn - r).max() <= 1e-14 * np.abs(x).max(), f"{what}: residue"
    return errs, exempt


def _run(X, prec, order=capi.ORDER_ROWS, **kw):
    Xr = np.asarray(X, NP[prec])
    rows, cols = Xr.shape
    p = make_params(rows, cols, precision=prec, order=order, **kw)
    plan = Plan(p)
    x = torch.from_numpy(Xr).cuda()
    imfs, res, n = plan.decompose(x)
    torch.cuda.synchronize()
    out = (imfs.double().cpu().numpy(), res.cpu().numpy(), n, plan.counts(1)[1][0],
           (plan.tile, plan.pass_variant))
    plan.close()
    return out


def _oracle(X, prec, order=capi.ORDER_ROWS, transition_len=-1, max_imfs=10,
            stop=capi.STOP_FIXED, fixed_sifts=10, sd_threshold=0.2, max_sifts=50,
            boundary=capi.BOUNDARY_MIRROR, mirror_knots=2, s_number=4,
            spline_end=capi.SPLINE_NATURAL):
    Xd = np.asarray(np.asarray(X, NP[prec]), np.float64)
    Xs = Xd if order == capi.ORDER_ROWS else Xd.T
    N, M = Xs.shape
    D = round(0.2 * M) if transition_len < 0 else transition_len
    if N == 1:
        D = 0
    if spline_end == capi.SPLINE_NOT_A_KNOT:
        boundary += O.SPLINE_NOT_A_KNOT
    kw = dict(D=D, K=max_imfs, stop=stop, fixed_sifts=fixed_sifts, sd_threshold=sd_threshold,
              max_sifts=max_sifts, boundary=boundary, mirror_knots=mirror_knots,
              s_number=s_number)
    imfs, res, n, sifts = O.serial_emd(Xs, **kw)
    if order == capi.ORDER_COLS:
        imfs = imfs.transpose(0, 2, 1)
        res = res.T
    return imfs, res, n, sifts, Xd


# ---------------------------------------------------------------- step-level parity

@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
@pytest.mark.parametrize("L", [3, 5, 64, 1023, 1024, 1025, 5000])
def test_extrema_bit_exact(prec, L):
    h = synth.rng(L).standard_normal(L).astype(NP[prec])
    h[L // 3: L // 3 + 3] = h[L // 3]  # a flat run
    plan = Plan(make_params(1, max(L, 8), precision=prec))
    tmax, tmin = plan.extrema(torch.from_numpy(h).cuda())
    omax, omin = O.extrema(h.astype(np.float64))
    assert np.array_equal(tmax.cpu().numpy(), omax)
    assert np.array_equal(tmin.cpu().numpy(), omin)
    plan.close()


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
@pytest.mark.parametrize("L", [40, 1000, 1024, 3001, 20000])
def test_one_sift(prec, L):
    g = synth.rng(100 + L)
    t = np.arange(L)
    h = (np.sin(t / 7.0) + 0.3 * g.standard_normal(L) + 0.5 * np.sin(t / 151.0)).astype(NP[prec])
    plan = Plan(make_params(1, L, precision=prec))
    out, num, den = plan.sift(torch.from_numpy(h).cuda())
    ref, rnum, rden = O.sift(h.astype(np.float64))
    got = out.double().cpu().numpy()
    tol = 1e-12 if prec == capi.FP64 else 2e-5
    assert _rel(got, ref, 1e-30) <= tol
    assert abs(num - rnum) <= tol * 10 * rnum and abs(den - rden) <= tol * 10 * rden
    plan.close()


# ------------------------------------------------------------ end-to-end parity

@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
@pytest.mark.parametrize("D", [0, 205])
def test_series_3x1024(prec, D):
    X = synth.workload_series_3x1024()
    g = _run(X, prec, transition_len=D, max_imfs=8)
    if prec == capi.FP32_MIXED and D == 0:
        x = np.asarray(X, np.float32).astype(np.float64)
        _check_fp32_given_input(g[0], g[1], g[2], x, 8, "series D=0", shape=g[4])
        return
    o = _oracle(X, prec, transition_len=D, max_imfs=8)
    _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], prec, f"series D={D}")
    common = min(g[2], o[2]) - (0 if prec == capi.FP64 else 1)
    assert list(g[3][:common]) == list(o[3][:common])


@pytest.mark.parametrize("D", [1, 50, 500, 1000])
@pytest.mark.parametrize("stop", [capi.STOP_FIXED, capi.STOP_SD])
def test_mask_series_transition_lengths_fp64(D, stop):
    """The transition-length sweep of Sec. 4.1 on the paper's 6-variate tone set: D from 1
    to M (the largest D that Sec. 3.2 allows, where X_A covers a whole signal), with the
    fixed sift count and the SD stop rule; every IMF and the sift counts against the
    oracle."""
    X = synth.paper_mask_series()
    g = _run(X, capi.FP64, transition_len=D, max_imfs=10, stop=stop)
    o = _oracle(X, capi.FP64, transition_len=D, max_imfs=10, stop=stop)
    _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], capi.FP64, f"mask D={D}")
    assert list(g[3][:g[2]]) == list(o[3][:o[2]])


@pytest.mark.parametrize("kw", [dict(), dict(boundary=capi.BOUNDARY_ENDPOINTS),
                                dict(mirror_knots=1)])
@pytest.mark.parametrize("tile", [128, 512])
def test_not_a_knot_ends_texture_fp64(kw, tile):
    """Not-a-knot spline ends on the texture: the first and last tiles are dense for the
    leading IMFs (the third knot from an end is a tile-interior knot given by the tile's
    elimination) and sparse for the later ones."""
    X = synth.workload_texture_256()[:64]
    Xr = np.asarray(X, np.float64)
    p = make_params(64, 256, precision=capi.FP64, transition_len=0, max_imfs=8,
                    spline_end=capi.SPLINE_NOT_A_KNOT, **kw)
    plan = Plan(p)
    plan.tile = tile
    imfs, res, n = plan.decompose(torch.from_numpy(Xr).cuda())
    torch.cuda.synchronize()
    g = (imfs.cpu().numpy(), res.cpu().numpy(), n)
    plan.close()
    o = _oracle(X, capi.FP64, transition_len=0, max_imfs=8, spline_end=capi.SPLINE_NOT_A_KNOT,
                **kw)
    _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], capi.FP64, f"not-a-knot {kw}")


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_snumber_stop_texture(prec):
    """The S-number stop rule on the 256 x 256 texture: the zero crossings are counted per
    tile, across every tile edge, and summed by the interface solve; the sift counts and
    IMFs against the oracle (FP64), the IMF counts and the unconditional bar (FP32)."""
    X = synth.workload_texture_256()
    g = _run(X, prec, transition_len=0, max_imfs=8, stop=capi.STOP_SNUMBER, s_number=3)
    o = _oracle(X, prec, transition_len=0, max_imfs=8, stop=capi.STOP_SNUMBER, s_number=3)
    _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], prec, "texture S-number")
    if prec == capi.FP64:
        assert list(g[3]) == list(o[3]), (g[3], o[3])


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_texture_256(prec):
    X = synth.workload_texture_256()
    g = _run(X, prec, transition_len=0, max_imfs=10)
    if prec == capi.FP64:
        o = _oracle(X, prec, transition_len=0, max_imfs=10)
        _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], prec, "texture 256")
    else:
        x = np.asarray(X, np.float32).astype(np.float64)
        _check_fp32_given_input(g[0], g[1], g[2], x, 10, "texture 256", shape=g[4])


def test_texture_256_with_transitions_fp64():
    X = synth.workload_texture_256()
    g = _run(X, capi.FP64, transition_len=-1, max_imfs=10)
    o = _oracle(X, capi.FP64, transition_len=-1, max_imfs=10)
    _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], capi.FP64, "texture 256 D=51")


@pytest.mark.parametrize("shape", [(1, 5), (1, 17), (1, 1023), (1, 1025), (3, 700), (2, 2049),
                                   (7, 333)])
def test_ragged_sizes_fp64(shape):
    g0 = synth.rng(shape[0] * 10007 + shape[1])
    t = np.arange(shape[1])
    X = np.sin(t[None, :] / (3.0 + np.arange(shape[0])[:, None])) + 0.2 * g0.standard_normal(shape)
    g = _run(X, capi.FP64, max_imfs=6)
    o = _oracle(X, capi.FP64, max_imfs=6)
    _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], capi.FP64, f"ragged {shape}")


@pytest.mark.parametrize("kw", [dict(boundary=capi.BOUNDARY_ENDPOINTS),
                                dict(mirror_knots=1),
                                dict(order=capi.ORDER_COLS),
                                dict(fixed_sifts=1),
                                dict(stop=capi.STOP_SD, sd_threshold=0.2, max_sifts=50),
                                dict(stop=capi.STOP_SNUMBER, s_number=1, max_sifts=50),
                                dict(stop=capi.STOP_SNUMBER, s_number=4, max_sifts=50),
                                dict(stop=capi.STOP_SNUMBER, s_number=3, max_sifts=5),
                                dict(spline_end=capi.SPLINE_NOT_A_KNOT),
                                dict(spline_end=capi.SPLINE_NOT_A_KNOT, mirror_knots=1),
                                dict(spline_end=capi.SPLINE_NOT_A_KNOT,
                                     boundary=capi.BOUNDARY_ENDPOINTS)])
def test_options_fp64(kw):
    X = synth.tone_chirp_series(4, 900, 77)
    if kw.get("order") == capi.ORDER_COLS:
        X = np.ascontiguousarray(X.T)
    g = _run(X, capi.FP64, max_imfs=7, **kw)
    o = _oracle(X, capi.FP64, max_imfs=7, **kw)
    _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], capi.FP64, str(kw))
    assert list(g[3]) == list(o[3]), (g[3], o[3])


def test_reconstruction_on_gpu():
    X = synth.workload_texture_256()
    imfs, res, n, _, _ = _run(X, capi.FP64, transition_len=0)
    assert np.abs(imfs.sum(0) + res - X).max() <= 1e-12


# ------------------------------------------------------------------------- batching

@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_batch_uneven_images_match_oracle_and_alone(prec):
    imgs = synth.uneven_images(12, 4242, side_range=(32, 96))
    imgs = [np.asarray(im, NP[prec]) for im in imgs]
    side = max(im.shape[0] for im in imgs)
    p = make_params(side, side, precision=prec, transition_len=0, max_imfs=8)
    plan = Plan(p, max_batch=len(imgs))
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    outs, ns = plan.decompose_batch(xs)
    torch.cuda.synchronize()
    for i, im in enumerate(imgs):
        gi, gr = outs[i][0].double().cpu().numpy(), outs[i][1].cpu().numpy()
        if prec == capi.FP32_MIXED:
            _check_fp32_given_input(gi, gr, ns[i], im.astype(np.float64), 8, f"batch item {i}",
                                    shape=(plan.tile, plan.pass_variant))
        else:
            o = _oracle(im, prec, transition_len=0, max_imfs=8)
            _check_imfs(gi, gr, ns[i], o[0], o[1], o[2], o[4], prec, f"batch item {i}")
    # alone == in the batch, bit for bit
    for i in (0, 5, 11):
        alone, n1 = plan.decompose_batch([xs[i]])
        torch.cuda.synchronize()
        assert n1[0] == ns[i]
        assert torch.equal(alone[0][0], outs[i][0]) and torch.equal(alone[0][1], outs[i][1])
    plan.close()


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
@pytest.mark.parametrize("stop,boundary", [(capi.STOP_SD, capi.BOUNDARY_MIRROR),
                                           (capi.STOP_SNUMBER, capi.BOUNDARY_ENDPOINTS)])
def test_interface_solve_thread_counts_agree(prec, stop, boundary):
    """A launch of more short instances (at most 64 tiles each) than the 256-thread
    interface solve keeps resident runs its 64-thread form; with one longer instance added,
    the launch runs the 256-thread form. The short instances' results are the same bit for
    bit, adaptive stop rules (sums over the tiles) and both boundary rules included."""
    g = np.random.default_rng(5)
    small = [np.asarray(synth.grating_image(int(s), int(s) + 7), NP[prec])
             for s in g.integers(16, 128, size=240)]
    big = np.asarray(synth.grating_image(160, 3), NP[prec])  # 100 tiles of 256 samples
    p = make_params(160, 160, precision=prec, transition_len=0, max_imfs=5, stop=stop,
                    sd_threshold=0.2, max_sifts=30, s_number=3, boundary=boundary)
    plan = Plan(p, max_batch=len(small) + 1)
    plan.tile = 256
    xs = [torch.from_numpy(im).cuda() for im in small]
    alone, n_alone = plan.decompose_batch(xs)
    mixed, n_mixed = plan.decompose_batch(xs + [torch.from_numpy(big).cuda()])
    torch.cuda.synchronize()
    assert n_alone == n_mixed[:len(small)]
    for i in range(len(small)):
        assert torch.equal(alone[i][0], mixed[i][0]) and torch.equal(alone[i][1], mixed[i][1])
    plan.close()


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
@pytest.mark.parametrize("stop", [capi.STOP_FIXED, capi.STOP_SD])
def test_packed_batch_equals_tensor_list_batch(prec, stop):
    """A batch stored back to back in one tensor (odd sizes, so that most inputs start at
    element offsets that are not 16-byte aligned) gives the IMFs, residues and counts of
    the same batch passed as separate tensors, bit for bit."""
    g = np.random.default_rng(7)
    imgs = [np.asarray(synth.grating_image(int(s), int(g.integers(0, 1000))), NP[prec])
            for s in g.integers(17, 90, size=23)]
    imgs += [np.asarray(synth.tone_chirp_series(3, 1001, 5), NP[prec])]
    p = make_params(90, 90, precision=prec, transition_len=0, max_imfs=6, stop=stop,
                    sd_threshold=0.2, max_sifts=50)
    plan = Plan(p, max_batch=len(imgs))
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    outs, ns = plan.decompose_batch(xs)
    shapes = [im.shape for im in imgs]
    flat = torch.cat([x.reshape(-1) for x in xs])
    pim, pres, pn = plan.decompose_packed(flat, shapes)
    torch.cuda.synchronize()
    assert pn == ns
    o = 0
    for i, im in enumerate(imgs):
        sz = im.size
        assert torch.equal(pim[6 * o:6 * (o + sz)].reshape(outs[i][0].shape), outs[i][0])
        assert torch.equal(pres[o:o + sz].reshape(outs[i][1].shape), outs[i][1])
        o += sz
    plan.close()


# ----------------------------------------------------------------------------- EEMD

@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_eemd_small(prec):
    img = synth.grating_image(48, 5).astype(NP[prec])
    trials = 6
    L = img.size
    w = synth.white_noise(trials, L, 6).astype(NP[prec])
    p = make_params(48, 48, precision=prec, transition_len=0, max_imfs=8, ensemble_trials=trials,
                    noise_rel_std=0.2)
    plan = Plan(p)
    imfs, res, n = plan.decompose(torch.from_numpy(img).cuda(), torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    x = img.astype(np.float64).reshape(-1)
    beta = 0.2 * O.std(x)
    oi, orr, on = O.eemd(x, w.astype(np.float64), beta, 8)
    _check_imfs(imfs.double().cpu().numpy().reshape(8, -1), res.cpu().numpy().reshape(-1), n,
                oi, orr, on, x, prec, "eemd")
    plan.close()


# ------------------------------------------------------------------- tile independence

@pytest.mark.parametrize("D", [0, -1])
def test_tile_sizes_agree_fp64(D):
    """The spline system is partitioned at tile edges exactly, so every tile size gives
    the oracle's decomposition (ragged last tile included: 300 x 301 samples)."""
    X = np.ascontiguousarray(synth.grating_image(301, 17)[:300, :])
    o = _oracle(X, capi.FP64, transition_len=D, max_imfs=8)
    res = {}
    for tile in (128, 256, 512):
        p = make_params(*X.shape, precision=capi.FP64, transition_len=D, max_imfs=8)
        plan = Plan(p)
        plan.tile = tile
        assert plan.tile == tile
        imfs, r, n = plan.decompose(torch.from_numpy(np.ascontiguousarray(X)).cuda())
        torch.cuda.synchronize()
        res[tile] = imfs.cpu().numpy()
        _check_imfs(res[tile], r.cpu().numpy(), n, o[0], o[1], o[2], o[4], capi.FP64,
                    f"tile {tile}")
        plan.close()
    for tile in (128, 512):
        assert np.abs(res[tile] - res[256]).max() <= 1e-12 * np.abs(X).max()


# ----------------------------------------------------------------------- edge cases

def _degenerate(kind):
    if kind == "constant":
        return np.full((1, 700), 2.5)
    if kind == "zeros":
        return np.zeros((3, 300))
    if kind == "ramp":
        return np.linspace(-1.0, 3.0, 900)[None, :]
    if kind == "one_bump":  # one maximum, no minimum: nmax + nmin < 3 (Sec. 2.1 end test)
        t = np.linspace(0.0, 1.0, 500)
        return np.exp(-((t - 0.4) / 0.1) ** 2)[None, :]
    if kind == "one_sample":
        return np.array([[1.25]])
    if kind == "two_samples":
        return np.array([[1.0, -2.0]])
    if kind == "plateaus":  # flat tops and bottoms: the tie rule of Step 1 decides
        t = np.arange(1500)
        return np.round(3.0 * np.sin(t / 17.0) + np.sin(t / 5.0))[None, :] / 4.0
    raise ValueError(kind)


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
@pytest.mark.parametrize("kind", ["constant", "zeros", "ramp", "one_bump", "one_sample",
                                  "two_samples", "plateaus"])
def test_degenerate_inputs(prec, kind):
    """Inputs the method leaves whole or decomposes only partly (no or too few extrema,
    flat runs) and the shortest signals: IMF counts equal the oracle's, IMFs and the
    residue match it (FP32 inputs are exact in single precision here, except the bump and
    ramp, whose IMF-free decompositions leave the input as the residue)."""
    X = np.asarray(_degenerate(kind), NP[prec])
    g = _run(X, prec, transition_len=0, max_imfs=6)
    o = _oracle(X, prec, transition_len=0, max_imfs=6)
    if prec == capi.FP64:
        _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], prec, kind)
    else:
        _check_fp32_given_input(g[0], g[1], g[2], X.astype(np.float64), 6, kind, shape=g[4])
    assert np.abs(g[0].sum(0) + g[1] - X.astype(np.float64)).max() <= \
        1e-12 * max(1.0, np.abs(X).max())


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_every_sample_an_extremum(prec):
    """Alternating samples: every interior sample is a maximum or a minimum, so each tile
    holds as many knots as samples (the knot pool's worst case), with ragged tiles."""
    g0 = synth.rng(5151)
    L = 3 * 256 + 77
    x = np.where(np.arange(L) % 2 == 0, 1.0, -1.0) * (1.0 + 0.25 * g0.uniform(size=L))
    x = x + 0.1 * np.sin(np.arange(L) / 40.0)
    X = np.asarray(x[None, :], NP[prec])
    g = _run(X, prec, transition_len=0, max_imfs=5)
    if prec == capi.FP64:
        o = _oracle(X, prec, transition_len=0, max_imfs=5)
        _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], prec, "alternating")
    else:
        _check_fp32_given_input(g[0], g[1], g[2], X.astype(np.float64), 5, "alternating",
                                shape=g[4])


def test_long_signal_global_interface_scratch_fp64():
    """A signal long enough that the interface solve's scratch leaves shared memory for
    global memory (more than ~4500 reduced-system entries per envelope at 256-sample
    tiles), with a ragged last tile."""
    L = (1 << 19) + 123
    g0 = synth.rng(777)
    t = np.arange(L)
    X = (np.sin(2 * np.pi * t / 9.0) + 0.5 * np.sin(2 * np.pi * t / 61.0) +
         0.3 * np.sin(2 * np.pi * t / 1500.0) + 0.05 * g0.standard_normal(L))[None, :]
    g = _run(X, capi.FP64, transition_len=0, max_imfs=6)
    o = _oracle(X, capi.FP64, transition_len=0, max_imfs=6)
    _check_imfs(g[0], g[1], g[2], o[0], o[1], o[2], o[4], capi.FP64, "long")


def test_interface_solve_cluster_shape():
    """On GB300 the interface solve of long instances (natural spline ends) runs on
    thread-block clusters of 16 (else 8) CTAs per envelope, from the tile count where one
    CTA's shared memory no longer holds the system; not-a-knot ends keep one CTA."""
    for prec in (capi.FP64, capi.FP32_MIXED):
        c, lo, hi = capi.serial_emd_interface_solve_shape(prec, capi.SPLINE_NATURAL)
        assert c in (8, 16), (prec, c)
        assert 256 < lo < hi, (prec, lo, hi)
        assert capi.serial_emd_interface_solve_shape(prec, capi.SPLINE_NOT_A_KNOT) == (0, 0, 0)


def _cluster_signal(nt, tile, seed, flat=True):
    """A single signal of about nt tiles (ragged last tile) with tones, noise and, with
    `flat`, a constant stretch of 40 tiles (tiles without knots)."""
    g = synth.rng(seed)
    L = nt * tile - 101
    t = np.arange(L)
    x = (np.sin(2 * np.pi * t / 7.3) + 0.6 * np.sin(2 * np.pi * t / 97.0) +
         0.3 * np.sin(2 * np.pi * t / 2100.0) + 0.05 * g.standard_normal(L))
    if flat:
        a = L // 3
        x[a:a + 40 * tile] = x[a]
    return x[None, :]


@pytest.mark.parametrize("kw", [dict(), dict(mirror_knots=1),
                                dict(boundary=capi.BOUNDARY_ENDPOINTS),
                                dict(stop=capi.STOP_SD, sd_threshold=0.2, max_sifts=30),
                                dict(stop=capi.STOP_SNUMBER, s_number=3, max_sifts=30)])
@pytest.mark.parametrize("where", ["low", "high"])
def test_cluster_interface_solve_fp64(kw, where):
    """Signals whose interface solve runs on a thread-block cluster (just above the tile
    count where it starts, and at three times that, with tile 512), FP64 against the
    oracle within 1e-10 (IMFs and sift counts), with each boundary rule, the SD and the
    S-number stop (their totals summed over the cluster's CTAs) and a constant stretch."""
    c, lo, hi = capi.serial_emd_interface_solve_shape(capi.FP64, capi.SPLINE_NATURAL)
    tile = 256 if where == "low" else 512
    nt = lo + 3 if where == "low" else min(3 * lo, hi)
    X = _cluster_signal(nt, tile, 4100 + nt)
    p = make_params(1, X.shape[1], precision=capi.FP64, transition_len=0, max_imfs=6, **kw)
    plan = Plan(p)
    plan.tile = tile
    imfs, res, n = plan.decompose(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    sifts = plan.counts(1)[1][0]
    plan.close()
    o = _oracle(X, capi.FP64, transition_len=0, max_imfs=6, **kw)
    _check_imfs(imfs.cpu().numpy(), res.cpu().numpy(), n, o[0], o[1], o[2], o[4], capi.FP64,
                f"cluster {where} {kw}")
    assert list(sifts[:n]) == list(o[3][:n]), (sifts, o[3])


def test_cluster_interface_solve_batch_independent_fp32():
    """A batch holding a long signal (cluster interface solve) and short ones (one-CTA
    solve) gives every instance the results it gets alone, bit for bit, in FP32: the
    solver of an instance depends on its own tile count only. The long one also meets
    the FP32 rule against the oracle."""
    c, lo, hi = capi.serial_emd_interface_solve_shape(capi.FP32_MIXED, capi.SPLINE_NATURAL)
    long_x = _cluster_signal(lo + 100, 256, 77)[0].astype(np.float32)
    short = [np.asarray(synth.grating_image(s, 5 + s), np.float32).reshape(-1)
             for s in (40, 96, 150)]
    xs = [long_x] + short
    L = max(len(v) for v in xs)
    p = make_params(1, L, precision=capi.FP32_MIXED, transition_len=0, max_imfs=5)
    plan = Plan(p, max_batch=len(xs))
    outs, n = plan.decompose_batch([torch.from_numpy(v[None, :]).cuda() for v in xs])
    torch.cuda.synchronize()
    plan.close()
    for i, v in enumerate(xs):
        q = Plan(make_params(1, len(v), precision=capi.FP32_MIXED, transition_len=0,
                             max_imfs=5))
        ai, ar, an = q.decompose(torch.from_numpy(v[None, :]).cuda())
        torch.cuda.synchronize()
        shape = (q.tile, q.pass_variant)
        q.close()
        gi, gr = outs[i]
        assert n[i] == an, i
        assert torch.equal(gi, ai) and torch.equal(gr, ar), i
        if i == 0:
            _check_fp32_given_input(ai.double().cpu().numpy(), ar.cpu().numpy(), an,
                                    v.astype(np.float64), 5, "cluster fp32", shape=shape)


def test_largest_serving_image_fp32():
    """A 2048 x 2048 image (4.2 M samples, the serving mix's largest request) in FP32:
    exact FP64 reconstruction, the oracle's IMF count, and its two leading IMFs given the
    same remainder."""
    X = np.asarray(synth.grating_image(2048, 99), np.float32)
    imfs, res, n, _, shape = _run(X, capi.FP32_MIXED, transition_len=0, max_imfs=10)
    x = X.astype(np.float64)
    assert np.abs(imfs.sum(0) + res - x).max() <= 1e-12 * np.abs(x).max()
    r = x.reshape(-1).copy()
    floor = 1e-6 * np.linalg.norm(x)
    for k in range(2):
        h32 = r.astype(np.float32).astype(np.float64)
        oi, _, on, _ = O.emd(h32, 1)
        assert on == 1
        err = _rel(imfs[k].reshape(-1), oi[0], floor)
        g, j, margin = _fp32_chain(h32, 10, shape)
        if margin is None:
            assert np.array_equal(g, imfs[k].reshape(-1)), k
            assert err <= TOL[capi.FP32_MIXED], (k, err)
        else:
            assert margin[1] <= FP32_TAU, (k, j, margin)
        r = r - imfs[k].reshape(-1)


# ------------------------------------------------------- slice-wise standard version

@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_slices_match_oracle_per_row_and_batch(prec):
    """The standard-version baseline of Sec. 4 (each signal decomposed on its own):
    every row against the oracle's EMD of that row (FP64; FP32 given the same remainder),
    and bit for bit against decompose_batch on the rows taken one by one."""
    X = np.asarray(synth.tone_chirp_series(9, 1500, 4711), NP[prec])
    rows, cols = X.shape
    K = 7
    plan = Plan(make_params(1, cols, precision=prec, transition_len=0, max_imfs=K),
                max_batch=rows)
    x = torch.from_numpy(X).cuda()
    imfs, res, ns = plan.decompose_slices(x)
    torch.cuda.synchronize()
    gi, gr = imfs.double().cpu().numpy(), res.cpu().numpy()
    for i in range(rows):
        xi = X[i].astype(np.float64)
        if prec == capi.FP64:
            oi, orr, on, _ = O.emd(xi, K)
            _check_imfs(gi[:, i], gr[i], ns[i], oi, orr, on, xi, prec, f"slice {i}")
        else:
            _check_fp32_given_input(gi[:, i], gr[i], ns[i], xi, K, f"slice {i}",
                                    shape=(plan.tile, plan.pass_variant))
    xs = [x[i:i + 1].contiguous() for i in range(rows)]
    outs, nb = plan.decompose_batch(xs)
    torch.cuda.synchronize()
    assert list(nb) == list(ns)
    for i in range(rows):
        assert torch.equal(outs[i][0][:, 0], imfs[:, i]) and torch.equal(outs[i][1][0], res[i])
    plan.close()


# --------------------------------------------------------------------- serial-CEEMDAN

def _ceemdan_gpu(X, w, prec, **kw):
    rows, cols = X.shape
    trials = w.shape[0]
    plan = Plan(make_params(rows, cols, precision=prec, ensemble_trials=trials, **kw))
    modes, res, n = plan.ceemdan(torch.from_numpy(np.ascontiguousarray(X)).cuda(),
                                 torch.from_numpy(np.ascontiguousarray(w)).cuda())
    torch.cuda.synchronize()
    out = modes.double().cpu().numpy(), res.cpu().numpy(), n
    return out, plan


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
@pytest.mark.parametrize("case", ["image48", "series3x1024_D205"])
def test_ceemdan_matches_oracle(prec, case):
    """Serial-CEEMDAN (Sec. 2.2 Steps 1-4 inside Sec. 3) against the oracle on the same
    rounded input and noise: every mode and the residue, FP64 within 1e-10; FP32 under the
    bar of the unconditional FP32 checks (the noise modes E_k are themselves FP32 EMDs)."""
    if case == "image48":
        X = synth.grating_image(48, 5).astype(NP[prec])
        D, K, trials = 0, 6, 4
    else:
        X = synth.workload_series_3x1024().astype(NP[prec])
        D, K, trials = 205, 8, 3
    N, M = X.shape
    L = O.serial_length(M, N, D)
    w = synth.white_noise(trials, L, 77).astype(NP[prec])
    (gm, gr, gn), plan = _ceemdan_gpu(X, w, prec, transition_len=D, max_imfs=K,
                                      noise_rel_std=0.2)
    om, orr, on = O.serial_ceemdan(X.astype(np.float64), D, K, w.astype(np.float64), 0.2)
    xd = X.astype(np.float64)
    _check_imfs(gm.reshape(K, -1), gr.reshape(-1), gn, om.reshape(K, -1), orr.reshape(-1), on,
                xd.reshape(-1), prec, f"ceemdan {case}")
    # modes + residue reconstruct the input (Step 3 keeps r in FP64)
    rec = gm.sum(0) + gr
    assert np.abs(rec - xd).max() <= (1e-12 if prec == capi.FP64 else 1e-5) * np.abs(xd).max()
    # a second call replays the captured graph; without graphs the same numbers come out
    m2, r2, n2 = plan.ceemdan(torch.from_numpy(X).cuda(), torch.from_numpy(w).cuda())
    plan.set_options(use_graphs=False)
    m3, r3, n3 = plan.ceemdan(torch.from_numpy(X).cuda(), torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    assert n2 == n3 == gn
    assert np.array_equal(m2.double().cpu().numpy(), gm) and np.array_equal(r2.cpu().numpy(), gr)
    assert np.array_equal(m3.double().cpu().numpy(), gm) and np.array_equal(r3.cpu().numpy(), gr)
    plan.close()


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_ceemdan_one_mode_sd_stop_and_no_extrema(prec):
    """K = 1 (no noise EMD: the first EEMD mode), the SD stop rule, and an input without
    extrema (no stage runs: zero modes, the residue is the input)."""
    X = synth.grating_image(40, 8).astype(NP[prec])
    w = synth.white_noise(5, X.size, 78).astype(NP[prec])
    (gm, gr, gn), plan = _ceemdan_gpu(X, w, prec, transition_len=0, max_imfs=1)
    om, orr, on = O.serial_ceemdan(X.astype(np.float64), 0, 1, w.astype(np.float64), 0.2)
    _check_imfs(gm.reshape(1, -1), gr.reshape(-1), gn, om.reshape(1, -1), orr.reshape(-1), on,
                X.astype(np.float64).reshape(-1), prec, "ceemdan K=1")
    plan.close()
    (gm, gr, gn), plan = _ceemdan_gpu(X, w, prec, transition_len=0, max_imfs=5,
                                      stop=capi.STOP_SD, max_sifts=30)
    om, orr, on = O.serial_ceemdan(X.astype(np.float64), 0, 5, w.astype(np.float64), 0.2,
                                   stop=O.STOP_SD, max_sifts=30)
    if prec == capi.FP64:
        _check_imfs(gm.reshape(5, -1), gr.reshape(-1), gn, om.reshape(5, -1), orr.reshape(-1),
                    on, X.astype(np.float64).reshape(-1), prec, "ceemdan SD")
    plan.close()
    ramp = np.tile(np.linspace(-1.0, 2.0, 64), (2, 1)).astype(NP[prec])
    ramp[1] += 3.0  # row 2 continues the rise of row 1: the serialized signal is monotone
    wr = synth.white_noise(3, ramp.size, 79).astype(NP[prec])
    (gm, gr, gn), plan = _ceemdan_gpu(ramp, wr, prec, transition_len=0, max_imfs=4)
    assert gn == 0 and not gm.any() and np.array_equal(gr, ramp.astype(np.float64))
    m, r, n = plan.ceemdan(torch.from_numpy(ramp).cuda(), torch.from_numpy(wr).cuda(),
                           wait=False)
    torch.cuda.synchronize()
    assert n is None and plan.counts(1)[0][0] == 0
    plan.close()


def test_ceemdan_needs_an_ensemble_plan():
    plan = Plan(make_params(8, 8, precision=capi.FP64, transition_len=0))
    x = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        plan.ceemdan(x, torch.zeros((2, 64), dtype=torch.float64, device="cuda"))
    plan.close()


# ------------------------------------------------------------------------- autotuner

def test_autotune_keeps_results_and_seeds_new_plans(tmp_path):
    """The autotuner times every pass-kernel shape, keeps the fastest (never slower than
    the default shape, which is among the candidates), and the decomposition it leaves
    agrees with the default shape's to rounding; a new plan with the same key starts from
    the tuned shape, and the saved table holds it."""
    capi.serial_emd_tune_clear()
    X = synth.workload_texture_256()
    p = make_params(256, 256, precision=capi.FP64, transition_len=0, max_imfs=6)
    plan = Plan(p)
    x = torch.from_numpy(X).cuda()
    ref, rres, rn = plan.decompose(x)
    ref, rres = ref.cpu().numpy(), rres.cpu().numpy()
    r = plan.autotune(x, repeats=2)
    assert r.tile in (128, 256, 512) and r.ctas_per_sm >= 0 and r.candidates >= 3
    assert 0 < r.ms <= r.ms_default
    assert (plan.tile, plan.pass_ctas, plan.pass_variant) == (r.tile, r.ctas_per_sm, r.variant)
    imfs, res, n = plan.decompose(x)
    assert n == rn
    floor = 1e-6 * np.linalg.norm(X)
    for k in range(6):
        assert _rel(imfs[k].cpu().numpy(), ref[k], floor) <= 1e-12
    plan2 = Plan(p)
    assert (plan2.tile, plan2.pass_ctas, plan2.pass_variant) == \
        (r.tile, r.ctas_per_sm, r.variant)
    out = tmp_path / "tune.json"
    capi.serial_emd_tune_save(str(out))
    assert f'"tile": {r.tile}' in out.read_text()
    plan.close()
    plan2.close()
    capi.serial_emd_tune_clear()


def test_autotune_ensemble_plan():
    capi.serial_emd_tune_clear()
    img = synth.grating_image(40, 5).astype(np.float32)
    trials = 8
    w = synth.white_noise(trials, img.size, 6).astype(np.float32)
    plan = Plan(make_params(40, 40, transition_len=0, max_imfs=5, ensemble_trials=trials))
    xi, wi = torch.from_numpy(img).cuda(), torch.from_numpy(w).cuda()
    r = plan.autotune(xi, noise=wi, repeats=1)
    assert r.tile in (128, 256, 512) and 0 < r.ms <= r.ms_default
    a, _, _ = plan.decompose(xi, wi)
    plan.tile, plan.pass_ctas = 256, 0
    b, _, _ = plan.decompose(xi, wi)
    floor = 1e-6 * np.linalg.norm(img)
    for k in range(2):
        assert _rel(a[k].double().cpu().numpy(), b[k].double().cpu().numpy(), floor) <= 1e-4
    plan.close()
    capi.serial_emd_tune_clear()


@pytest.mark.parametrize("prec", [capi.FP32_MIXED, capi.FP64])
def test_pass_kernel_register_variants_agree_bit_for_bit(prec):
    """The two variants of the 256-sample pass kernel (staging the next tile; a smaller
    kernel without staging) compile the same arithmetic, with any CTA count per SM:
    identical IMFs, residue and counts, in both precisions."""
    X = synth.workload_texture_256().astype(NP[prec])
    plan = Plan(make_params(256, 256, precision=prec, transition_len=0, max_imfs=6))
    x = torch.from_numpy(X).cuda()
    out = []
    for v in (0, 1):
        plan.pass_variant = v
        for c in (0, 2):
            plan.pass_ctas = c
            imfs, res, n = plan.decompose(x)
            out.append((imfs.cpu(), res.cpu(), n))
    plan.close()
    for imfs, res, n in out[1:]:
        assert n == out[0][2] and torch.equal(imfs, out[0][0]) and torch.equal(res, out[0][1])


@pytest.mark.parametrize("prec", [capi.FP32_MIXED, capi.FP64])
def test_pass_after_another_tile_size_equals_fresh_plan(prec):
    """The latency variant of the pass kernel reads a warp's first tile, with the extremum
    masks stored for it, before it waits for the interface solve, when those masks may
    still be another signal's. A plan that ran with 512-sample tiles (its stored masks
    index up to 512 samples per tile) and then with 256-sample tiles gives the IMFs of a
    fresh 256-sample-tile plan bit for bit, in both precisions."""
    X = synth.workload_texture_256().astype(NP[prec])
    x = torch.from_numpy(X).cuda()
    out = []
    for first in (512, None):
        plan = Plan(make_params(256, 256, precision=prec, transition_len=0, max_imfs=4))
        if first is not None:
            plan.tile = first
            plan.pass_variant = 1
            plan.decompose(x)
        plan.tile = 256
        plan.pass_variant = 1
        imfs, res, n = plan.decompose(x)
        out.append((imfs.cpu(), res.cpu(), n))
        plan.close()
    assert out[0][2] == out[1][2]
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_readme_example_runs():
    """The usage example of the README: serial EMD, EEMD and CEEMDAN of a 6 x 1000 input."""
    x = torch.randn(6, 1000, device="cuda")
    plan = Plan(make_params(6, 1000, transition_len=50, max_imfs=10))
    imfs, residue, n = plan.decompose(x)
    assert imfs.shape == (10, 6, 1000) and residue.dtype == torch.float64 and 1 <= n <= 10
    noise = torch.randn(100, 6 * 1000 + 50 * 5, device="cuda")
    ens = Plan(make_params(6, 1000, transition_len=50, ensemble_trials=100))
    eemd_imfs, _, _ = ens.decompose(x, noise)
    modes, r, n_modes = ens.ceemdan(x, noise)
    torch.cuda.synchronize()
    rec = (modes.double().sum(0) + r - x.double()).abs().max().item()
    assert 1 <= n_modes <= 10 and rec <= 1e-5 * x.abs().max().item()
    for p in (plan, ens):
        p.close()


@pytest.mark.parametrize("kw", [
    dict(stop=capi.STOP_SNUMBER, s_number=3, max_sifts=30),
    dict(spline_end=capi.SPLINE_NOT_A_KNOT, boundary=capi.BOUNDARY_ENDPOINTS),
    dict(spline_end=capi.SPLINE_NOT_A_KNOT, mirror_knots=1, stop=capi.STOP_SD, max_sifts=40)])
def test_ceemdan_plan_options_fp64(kw):
    """Serial-CEEMDAN with the plan options that change the inner EMDs (stop rules,
    boundary rule, not-a-knot ends), FP64, against the oracle with the same options."""
    X = synth.grating_image(40, 12)
    trials, K = 4, 6
    w = synth.white_noise(trials, X.size, 80)
    (gm, gr, gn), plan = _ceemdan_gpu(X, w, capi.FP64, transition_len=0, max_imfs=K,
                                      noise_rel_std=0.2, **kw)
    plan.close()
    okw = dict(stop=kw.get("stop", capi.STOP_FIXED), max_sifts=kw.get("max_sifts", 50),
               s_number=kw.get("s_number", 4), mirror_knots=kw.get("mirror_knots", 2),
               boundary=kw.get("boundary", capi.BOUNDARY_MIRROR) +
               (O.SPLINE_NOT_A_KNOT if kw.get("spline_end") == capi.SPLINE_NOT_A_KNOT else 0))
    om, orr, on = O.serial_ceemdan(X, 0, K, w, 0.2, **okw)
    _check_imfs(gm.reshape(K, -1), gr.reshape(-1), gn, om.reshape(K, -1), orr.reshape(-1), on,
                X.reshape(-1), capi.FP64, f"ceemdan {kw}")


@pytest.mark.parametrize("seed", range(int(os.environ.get("SEMD_RANDOM_CASES", "24"))))
def test_random_configurations_fp64(seed):
    """Seeded random configurations (shape, order, transition length, IMF count, stop rule,
    boundary rule, mirror knots, spline ends, tile), FP64 against the oracle."""
    g = np.random.default_rng(7000 + seed)
    rows, cols = int(g.integers(1, 6)), int(g.integers(40, 1500))
    order = capi.ORDER_ROWS if g.random() < 0.7 else capi.ORDER_COLS
    M = cols if order == capi.ORDER_ROWS else rows
    D = int(g.integers(0, M + 1)) if g.random() < 0.5 else -1
    kw = dict(transition_len=D, max_imfs=int(g.integers(1, 9)), order=order)
    stop = int(g.integers(0, 3))
    kw["stop"] = stop
    if stop == capi.STOP_FIXED:
        kw["fixed_sifts"] = int(g.integers(1, 12))
    elif stop == capi.STOP_SD:
        kw["sd_threshold"], kw["max_sifts"] = float(g.uniform(0.05, 0.5)), int(g.integers(2, 40))
    else:
        kw["s_number"], kw["max_sifts"] = int(g.integers(1, 6)), int(g.integers(2, 40))
    kw["boundary"] = int(g.integers(0, 2))
    kw["mirror_knots"] = int(g.integers(1, 3))
    kw["spline_end"] = int(g.integers(0, 2))
    tile = int(g.choice([128, 256, 512]))
    t = np.arange(rows * cols).reshape(rows, cols) / 97.0
    X = (np.sin(t * g.uniform(0.5, 3.0)) + 0.5 * np.sin(t * g.uniform(5.0, 20.0))
         + 0.2 * g.standard_normal((rows, cols)))
    plan = Plan(make_params(rows, cols, precision=capi.FP64, **kw))
    plan.tile = tile
    imfs, res, n = plan.decompose(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    gi, gr = imfs.cpu().numpy(), res.cpu().numpy()
    sifts = plan.counts(1)[1][0]
    plan.close()
    okw = {k: v for k, v in kw.items() if k in ("stop", "fixed_sifts", "sd_threshold",
                                                   "max_sifts", "boundary", "mirror_knots",
                                                   "s_number", "spline_end", "transition_len",
                                                   "max_imfs", "order")}
    o = _oracle(X, capi.FP64, **okw)
    _check_imfs(gi, gr, n, o[0], o[1], o[2], o[4], capi.FP64, f"seed {seed} {kw} tile {tile}")
    assert list(sifts[:n]) == list(o[3][:n])


def _random_plan_options(g):
    kw = dict(max_imfs=int(g.integers(1, 8)))
    stop = int(g.integers(0, 3))
    kw["stop"] = stop
    if stop == capi.STOP_FIXED:
        kw["fixed_sifts"] = int(g.integers(1, 12))
    elif stop == capi.STOP_SD:
        kw["sd_threshold"], kw["max_sifts"] = float(g.uniform(0.05, 0.5)), int(g.integers(2, 30))
    else:
        kw["s_number"], kw["max_sifts"] = int(g.integers(1, 6)), int(g.integers(2, 30))
    kw["boundary"] = int(g.integers(0, 2))
    kw["mirror_knots"] = int(g.integers(1, 3))
    kw["spline_end"] = int(g.integers(0, 2))
    return kw


def _oracle_kw(kw):
    okw = dict(stop=kw["stop"], max_sifts=kw.get("max_sifts", 50),
               fixed_sifts=kw.get("fixed_sifts", 10), sd_threshold=kw.get("sd_threshold", 0.2),
               s_number=kw.get("s_number", 4), mirror_knots=kw["mirror_knots"],
               boundary=kw["boundary"] +
               (O.SPLINE_NOT_A_KNOT if kw["spline_end"] == capi.SPLINE_NOT_A_KNOT else 0))
    if kw["stop"] == capi.STOP_SNUMBER:
        okw.pop("fixed_sifts")
    else:
        okw.pop("s_number")
    return okw


@pytest.mark.parametrize("seed", range(int(os.environ.get("SEMD_RANDOM_CASES", "24")) // 3))
def test_random_batches_fp64(seed):
    """Seeded random batches of uneven inputs (one plan, random options and shapes, rows
    order, D = 0), every input against the oracle alone, FP64."""
    g = np.random.default_rng(8000 + seed)
    kw = _random_plan_options(g)
    count = int(g.integers(2, 7))
    shapes = [(int(g.integers(1, 5)), int(g.integers(20, 700))) for _ in range(count)]
    rmax = max(r for r, _ in shapes)
    cmax = max(c for _, c in shapes)
    plan = Plan(make_params(rmax, cmax, precision=capi.FP64, transition_len=0, **kw),
                max_batch=len(shapes))
    plan.tile = int(g.choice([128, 256, 512]))
    Xs = [g.standard_normal(s).cumsum(axis=1) * 0.1 + np.sin(np.arange(s[1]) / 7.0)
          for s in shapes]
    xs = [torch.from_numpy(np.ascontiguousarray(X)).cuda() for X in Xs]
    outs, ns = plan.decompose_batch(xs)
    torch.cuda.synchronize()
    plan.close()
    K = kw["max_imfs"]
    for X, (imfs, res), n in zip(Xs, outs, ns):
        oi, orr, on, _ = O.serial_emd(X, 0, K, **_oracle_kw(kw))
        _check_imfs(imfs.cpu().numpy(), res.cpu().numpy(), n, oi, orr, on, X, capi.FP64,
                    f"batch seed {seed} {kw} shape {X.shape}")


@pytest.mark.parametrize("seed", range(int(os.environ.get("SEMD_RANDOM_CASES", "24")) // 4))
def test_random_ceemdan_fp64(seed):
    """Seeded random serial-CEEMDAN configurations (shape, D, realizations, options), FP64
    against the oracle."""
    g = np.random.default_rng(9000 + seed)
    kw = _random_plan_options(g)
    rows, cols = int(g.integers(1, 4)), int(g.integers(30, 400))
    D = int(g.integers(0, cols + 1)) if rows > 1 else 0
    trials = int(g.integers(2, 6))
    N, M = rows, cols
    L = M * N + D * N - D
    X = np.sin(np.arange(rows * cols).reshape(rows, cols) / g.uniform(3, 15)) + \
        0.3 * g.standard_normal((rows, cols))
    w = g.standard_normal((trials, L))
    (gm, gr, gn), plan = _ceemdan_gpu(X, w, capi.FP64, transition_len=D, **kw)
    plan.close()
    K = kw["max_imfs"]
    om, orr, on = O.serial_ceemdan(X, D, K, w, 0.2, **_oracle_kw(kw))
    _check_imfs(gm.reshape(K, -1), gr.reshape(-1), gn, om.reshape(K, -1), orr.reshape(-1), on,
                X.reshape(-1), capi.FP64, f"ceemdan seed {seed} {kw} D {D}")



@pytest.mark.parametrize("seed", range(int(os.environ.get("SEMD_RANDOM_CASES", "24")) // 3))
def test_random_configurations_fp32(seed):
    """Seeded random FP32-mixed configurations (shape, K, sift count, boundary rule, mirror
    knots, spline ends, tile; D = 0), each IMF against the oracle's IMF of the same
    remainder under the FP32 bar."""
    g = np.random.default_rng(10000 + seed)
    rows, cols = int(g.integers(1, 6)), int(g.integers(60, 1500))
    K, S = int(g.integers(1, 8)), int(g.integers(1, 12))
    b, mk, se = int(g.integers(0, 2)), int(g.integers(1, 3)), int(g.integers(0, 2))
    t = np.arange(rows * cols).reshape(rows, cols) / 89.0
    X = (np.sin(t * g.uniform(0.5, 3.0)) + 0.5 * np.sin(t * g.uniform(5.0, 20.0))
         + 0.2 * g.standard_normal((rows, cols))).astype(np.float32)
    plan = Plan(make_params(rows, cols, transition_len=0, max_imfs=K, fixed_sifts=S,
                            boundary=b, mirror_knots=mk, spline_end=se))
    plan.tile = int(g.choice([128, 256, 512]))
    imfs, res, n = plan.decompose(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    shape = (plan.tile, plan.pass_variant)
    plan.close()
    _check_fp32_given_input(imfs.double().cpu().numpy(), res.cpu().numpy(), n,
                            X.astype(np.float64), K, f"fp32 seed {seed} K {K} S {S} b {b} "
                            f"mk {mk} se {se}", S=S,
                            boundary=b + (O.SPLINE_NOT_A_KNOT if se else 0), mirror_knots=mk,
                            shape=shape)


@pytest.mark.parametrize("seed", range(int(os.environ.get("SEMD_RANDOM_CASES", "24")) // 6))
def test_random_long_signals_fp64(seed):
    """Seeded random long single signals (20 k to 300 k samples, so that the interface
    solve takes its large form and, past its shared-memory capacity, global scratch), with
    random options and tile, FP64 against the oracle."""
    g = np.random.default_rng(11000 + seed)
    kw = _random_plan_options(g)
    L = int(g.integers(20000, 300000))
    t = np.arange(L)
    x = (np.sin(t / g.uniform(3.0, 9.0)) + 0.7 * np.sin(t / g.uniform(40.0, 400.0))
         + 0.3 * g.standard_normal(L))[None, :]
    plan = Plan(make_params(1, L, precision=capi.FP64, transition_len=0, **kw))
    plan.tile = int(g.choice([128, 256, 512]))
    imfs, res, n = plan.decompose(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.close()
    K = kw["max_imfs"]
    oi, orr, on, _ = O.serial_emd(x, 0, K, **_oracle_kw(kw))
    _check_imfs(imfs.cpu().numpy(), res.cpu().numpy(), n, oi, orr, on, x, capi.FP64,
                f"long seed {seed} L {L} {kw}")


# ------------------------------------------------------------- full-size workloads

@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_uneven_images_2048_full_workload(prec):
    """The 2048 uneven blob-field images (side U{32..128}) in one batched run with the
    configuration of the benchmark (D = 0, SD stop 0.2, at most 50 sifts, at most 8 IMFs):
    every image's reconstruction, and a seeded sample of 24 images (the smallest and the
    largest among them) against the oracle, IMF by IMF and sift count by sift count."""
    K = 8
    imgs = [np.ascontiguousarray(im, NP[prec]) for im in synth.workload_uneven_images()]
    side = max(im.shape[0] for im in imgs)
    p = make_params(side, side, precision=prec, transition_len=0, max_imfs=K,
                    stop=capi.STOP_SD, sd_threshold=0.2, max_sifts=50)
    plan = Plan(p, max_batch=len(imgs))
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    outs, ns = plan.decompose_batch(xs)
    torch.cuda.synchronize()
    n_all, sifts_all = plan.counts(len(imgs))
    shape = (plan.tile, plan.pass_variant)
    plan.close()
    assert list(ns) == list(n_all)
    for i, im in enumerate(imgs):
        x = im.astype(np.float64)
        c = outs[i][0].double().cpu().numpy()
        r = outs[i][1].cpu().numpy()
        assert np.abs(c.sum(0) + r - x).max() <= 1e-12 * np.abs(x).max(), f"image {i}"
    sides = [im.shape[0] for im in imgs]
    g = np.random.default_rng(2106)
    idx = set(int(i) for i in g.choice(len(imgs), 22, replace=False))
    idx |= {int(np.argmin(sides)), int(np.argmax(sides))}
    for i in sorted(idx):
        gi, gr = outs[i][0].double().cpu().numpy(), outs[i][1].cpu().numpy()
        what = f"image {i} (side {sides[i]})"
        if prec == capi.FP64:
            o = _oracle(imgs[i], prec, transition_len=0, max_imfs=K, stop=capi.STOP_SD,
                        sd_threshold=0.2, max_sifts=50)
            _check_imfs(gi, gr, ns[i], o[0], o[1], o[2], o[4], prec, what)
            assert list(sifts_all[i][:ns[i]]) == list(o[3][:o[2]]), what
        else:
            _check_fp32_given_input(gi, gr, ns[i], imgs[i].astype(np.float64), K, what,
                                    shape=shape, sd=(0.2, 50), sifts_g=sifts_all[i])


def _pool_eemd(x, w, beta, K, S, workers):
    """The oracle's EEMD with its trials split over a process pool (spawned: CUDA is
    initialized in this process); the chunk means are recombined into the trial mean."""
    import concurrent.futures as cf
    import multiprocessing as mp
    trials = w.shape[0]
    bounds = np.linspace(0, trials, workers + 1).astype(int)
    spans = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    with cf.ProcessPoolExecutor(max_workers=len(spans),
                                mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(O.eemd, x, w[a:b], beta, K, O.STOP_FIXED, S) for a, b in spans]
        parts = [f.result() for f in futs]
    imfs = sum(p[0] * (b - a) for p, (a, b) in zip(parts, spans)) / trials
    res = sum(p[1] * (b - a) for p, (a, b) in zip(parts, spans)) / trials
    return imfs, res, max(p[2] for p in parts)


@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_eemd_512_256_trials_full_workload(prec):
    """EEMD of the 512 x 512 grating image with 256 white-noise realizations (beta = 0.2
    std, 10 sifts per IMF, at most 10 IMFs, all trials in one run), as the benchmark runs
    it, against the oracle's EEMD of the same inputs (its trials in a process pool on the
    host cores). FP64: every averaged IMF within 1e-10.

    FP32, per realization: realizations 0 to 15 are read back one by one
    (serial_emd_eemd_trial) and each of their IMFs is held to the FP32 bar against the
    oracle's IMF of the same remainder, with the per-decision exemption rule of
    _check_fp32_given_input (the realization's input x + beta w^(m) is formed here from
    the beta the call used, in the same FP64 operations as the library). FP32, the trial
    mean: the first IMF within 1e-4 (its knots are dense and single precision keeps its
    decisions); later averaged IMFs carry, at 1/256 of their size, the knot moves of the
    realizations whose decisions single precision cannot resolve, so they and the tail sum
    are held to 1e-3 of ||x||, the IMF counts at most one apart, and the trial mean must
    reconstruct: the averaged IMFs plus the averaged residue equal x plus beta times the
    mean noise."""
    K, S, trials = 10, 10, 256
    img, w = synth.workload_eemd_512(trials)
    img, w = np.ascontiguousarray(img, NP[prec]), np.ascontiguousarray(w, NP[prec])
    p = make_params(512, 512, precision=prec, transition_len=0, max_imfs=K,
                    ensemble_trials=trials, noise_rel_std=0.2)
    plan = Plan(p)
    imfs, res, n = plan.decompose(torch.from_numpy(img).cuda(), torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    trials_g = []
    if prec == capi.FP32_MIXED:
        for m in range(16):
            ti, tr, tn, tbeta = plan.eemd_trial(m)
            trials_g.append((ti.double().cpu().numpy(), tr.cpu().numpy(), tn, tbeta))
    shape = (plan.tile, plan.pass_variant)
    plan.close()
    gi = imfs.double().cpu().numpy().reshape(K, -1)
    gr = res.cpu().numpy().reshape(-1)
    x = img.astype(np.float64).reshape(-1)
    wd = w.astype(np.float64)
    beta = 0.2 * O.std(x)
    workers = max(1, min(16, os.cpu_count() or 1))
    oi, orr, on = _pool_eemd(x, wd, beta, K, S, workers)
    what = f"eemd 512x512 x {trials}"
    if prec == capi.FP64:
        _check_imfs(gi, gr, n, oi, orr, on, x, prec, what)
        return
    exempt = 0
    for m, (ti, tr, tn, tbeta) in enumerate(trials_g):
        assert abs(tbeta - beta) <= 1e-12 * beta, (tbeta, beta)
        xm = x + tbeta * wd[m]  # one FP64 product, one FP64 sum: as the library forms it
        _, ex = _check_fp32_given_input(ti, tr, tn, xm, K, f"{what} realization {m}",
                                        shape=shape)
        exempt += sum(ex)
    print(f"{what}: {exempt} of the realizations' IMFs exempt (decisions FP32 cannot "
          f"resolve)")
    nx = np.linalg.norm(x)
    errs = [_rel(gi[k], oi[k], 1e-6 * nx) for k in range(K)]
    assert abs(n - on) <= 1, f"{what}: IMF count {n} vs {on}"
    assert errs[0] <= TOL[prec], f"{what}: IMF 1 {errs[0]} (all {errs})"
    tail0 = max(min(n, on) - 1, 1)
    absn = [np.linalg.norm(gi[k] - oi[k]) / nx for k in range(1, tail0)]
    absn.append(np.linalg.norm(gi[tail0:].sum(0) + gr - oi[tail0:].sum(0) - orr) / nx)
    assert max(absn) <= 1e-3, f"{what}: |dc|/|x| {absn} (rel {errs})"
    target = x + beta * wd.mean(0)
    rec = gi.sum(0) + gr
    assert np.abs(rec - target).max() <= 1e-5 * np.abs(target).max(), f"{what}: mean"


# --------------------------------------------- adaptive stop decided on the device

@pytest.mark.parametrize("stop", [capi.STOP_SD, capi.STOP_SNUMBER])
@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_adaptive_stop_graph_equals_host_loop(prec, stop):
    """With the SD or S-number stop (Sec. 2.1 Step 5) a batched decomposition runs as one
    CUDA graph whose sifting loop is a conditional node: the device decides after every
    few passes whether an instance is still running, with no host synchronization. Its
    results equal the host-driven loop's (graphs off) bit for bit, over two replays, and
    (FP64) the oracle's IMFs and sift counts."""
    imgs = [np.asarray(im, NP[prec]) for im in synth.uneven_images(9, 5150, side_range=(20, 72))]
    side = max(im.shape[0] for im in imgs)
    p = make_params(side, side, precision=prec, transition_len=0, max_imfs=6, stop=stop,
                    sd_threshold=0.2, max_sifts=40, s_number=3)
    plan = Plan(p, max_batch=len(imgs))
    xs = [torch.from_numpy(im).cuda() for im in imgs]
    outs_g, n_g = plan.decompose_batch(xs)
    outs_g2, n_g2 = plan.decompose_batch(xs)
    torch.cuda.synchronize()
    assert plan.stats().used_graph == 1
    cnt_g = plan.counts(len(imgs))
    plan.set_options(use_graphs=False)
    outs_h, n_h = plan.decompose_batch(xs)
    torch.cuda.synchronize()
    assert plan.stats().used_graph == 0
    cnt_h = plan.counts(len(imgs))
    plan.close()
    assert list(n_g) == list(n_h) == list(n_g2)
    assert cnt_g == cnt_h
    for i in range(len(imgs)):
        for a, b, c in ((outs_g[i][0], outs_h[i][0], outs_g2[i][0]),
                        (outs_g[i][1], outs_h[i][1], outs_g2[i][1])):
            assert torch.equal(a, b) and torch.equal(a, c), i
    if prec == capi.FP64:
        for i in (0, 4, 8):
            o = _oracle(imgs[i], prec, transition_len=0, max_imfs=6, stop=stop,
                        sd_threshold=0.2, max_sifts=40, s_number=3)
            _check_imfs(outs_g[i][0].cpu().numpy(), outs_g[i][1].cpu().numpy(), n_g[i], o[0],
                        o[1], o[2], o[4], prec, f"image {i}")
            assert list(cnt_g[1][i][:n_g[i]]) == list(o[3][:o[2]])


# ------------------------------------------------------- EEMD noise drawn on the device

def test_eemd_device_noise_equals_oracle_generator_fp64():
    """EEMD without caller noise: the library draws the realizations on the device
    (Philox4x32-10, Reading 11b). The result equals, bit for bit, the same plan run with
    the oracle's statement of the generator passed in as noise, and matches the oracle's
    EEMD with that noise within 1e-10; another seed gives another result."""
    K, trials, seed = 6, 5, 0xBEEF
    X = synth.grating_image(48, 21)
    L = X.size
    p = make_params(48, 48, precision=capi.FP64, transition_len=0, max_imfs=K,
                    ensemble_trials=trials, noise_rel_std=0.2)
    plan = Plan(p)
    plan.noise_seed = seed
    x = torch.from_numpy(np.ascontiguousarray(X, np.float64)).cuda()
    imfs_d, res_d, n_d = plan.decompose(x, None)
    w = O.white_noise(seed, trials, L)
    imfs_w, res_w, n_w = plan.decompose(x, torch.from_numpy(w).cuda())
    plan.noise_seed = seed + 1
    imfs_o2, _, _ = plan.decompose(x, None)
    torch.cuda.synchronize()
    plan.close()
    assert n_d == n_w
    assert torch.equal(imfs_d, imfs_w) and torch.equal(res_d, res_w)
    assert not torch.equal(imfs_d, imfs_o2)
    xs = X.reshape(-1).astype(np.float64)
    oi, orr, on = O.eemd(xs, w, 0.2 * O.std(xs), K)
    _check_imfs(imfs_d.cpu().numpy().reshape(K, -1), res_d.cpu().numpy().reshape(-1), n_d,
                oi, orr, on, xs, capi.FP64, "device noise")
