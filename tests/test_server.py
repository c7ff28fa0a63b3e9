"""Continuous-batching server (serial_emd_server_create / _submit / _poll).

Requests of different shapes are admitted as slots and the memory budget allow, while
others are mid-decomposition; each result must be bit-identical to decomposing the same
input alone with a plan (FP64 and FP32), and FP64 results must match the oracle.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2106_15319_gb300 import capi, synth  # noqa: E402
from paper_2106_15319_gb300.serial_emd import Plan, Server, make_params  # noqa: E402

NP = {capi.FP64: np.float64, capi.FP32_MIXED: np.float32}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    capi.load()


def _mix(seed):
    """Series and images of different shapes; one column-ordered."""
    g = synth.rng(seed)
    items = []
    for k in range(5):
        ch, n = int(g.integers(2, 6)), int(g.integers(700, 3000))
        items.append((synth.tone_chirp_series(ch, n, seed + k), capi.ORDER_ROWS))
    for k in range(4):
        side = int(g.integers(32, 90))
        items.append((synth.grating_image(side, seed + 10 + k), capi.ORDER_ROWS))
    items.append((np.ascontiguousarray(synth.tone_chirp_series(3, 900, seed + 20).T),
                  capi.ORDER_COLS))
    return items


def _wait(server, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = server.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "server did not finish in time"
        time.sleep(0.002)
    return out


OPTIONS = {"default": {},
           "snumber_notaknot_endpoints": dict(stop=capi.STOP_SNUMBER, s_number=3, max_sifts=30,
                                              spline_end=capi.SPLINE_NOT_A_KNOT,
                                              boundary=capi.BOUNDARY_ENDPOINTS)}


@pytest.mark.parametrize("opt", list(OPTIONS))
@pytest.mark.parametrize("prec", [capi.FP64, capi.FP32_MIXED])
def test_server_results_equal_alone(prec, opt):
    kw = OPTIONS[opt]
    items = _mix(31)
    K = 8
    base = make_params(64, 4096, precision=prec, transition_len=-1, max_imfs=K, **kw)
    # a small budget and 3 slots: requests must queue and join while others run
    server = Server(base, 24 << 20, 3)
    xs = [torch.from_numpy(np.asarray(X, NP[prec])).cuda() for X, _ in items]
    subs = []
    for i, ((X, order), x) in enumerate(zip(items, xs)):
        subs.append((server.submit(x, order=order), order))
        if i == 4:
            time.sleep(0.01)  # the second half arrives while the first is on the GPU
    res = _wait(server, [s[0][0] for s in subs])
    server.close()
    for (X, order), x, ((t, imfs, r), _) in zip(items, xs, subs):
        out = res[t]
        assert out.status == capi.SEMD_OK
        p = make_params(*X.shape, precision=prec, transition_len=-1, max_imfs=K, order=order,
                        **kw)
        plan = Plan(p)
        ai, ar, an = plan.decompose(x)
        torch.cuda.synchronize()
        plan.close()
        assert out.n_imfs == an
        assert torch.equal(imfs, ai) and torch.equal(r, ar), (X.shape, order)
        assert out.queue_ms >= 0.0 and out.run_ms > 0.0
        assert out.sifts >= (10 * an if not kw else an)
    # FP64 against the oracle, for two of the requests
    if prec == capi.FP64 and not kw:
        for j in (0, 6):
            X, order = items[j]
            Xs = X if order == capi.ORDER_ROWS else X.T
            D = round(0.2 * Xs.shape[1]) if Xs.shape[0] > 1 else 0
            oi, orr, on, _ = O.serial_emd(np.asarray(Xs, np.float64), D, K)
            g = subs[j][0][1].cpu().numpy()
            assert res[subs[j][0][0]].n_imfs == on
            for k in range(K):
                den = max(np.linalg.norm(oi[k]), 1e-6 * np.linalg.norm(Xs))
                assert np.linalg.norm(g[k] - oi[k]) / den <= 1e-10


def test_server_rejects_and_reports():
    base = make_params(16, 1024, precision=capi.FP32_MIXED, max_imfs=4)
    server = Server(base, 8 << 20, 2)
    too_long = torch.zeros((32, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(capi.SemdError) as ei:
        server.submit(too_long)
    assert ei.value.status == capi.SEMD_EBUDGET
    with pytest.raises(capi.SemdError) as ei:
        server.submit(torch.zeros((4, 64), dtype=torch.float32, device="cuda"), order=7)
    assert ei.value.status == capi.SEMD_EINVAL
    with pytest.raises(capi.SemdError) as ei:
        server.poll(123456)
    assert ei.value.status == capi.SEMD_EINVAL
    x = torch.from_numpy(synth.tone_chirp_series(2, 500, 3).astype(np.float32)).cuda()
    t, imfs, r = server.submit(x)
    out = _wait(server, [t])[t]
    assert out.status == capi.SEMD_OK and out.n_imfs >= 1
    with pytest.raises(capi.SemdError):
        server.poll(t)  # a result is returned once
    server.close()


def test_server_destroy_while_busy_leaves_gpu_usable():
    base = make_params(8, 4096, precision=capi.FP32_MIXED, max_imfs=6)
    server = Server(base, 16 << 20, 2)
    xs = [torch.from_numpy(synth.tone_chirp_series(4, 3000, s).astype(np.float32)).cuda()
          for s in range(8)]
    keep = [server.submit(x) for x in xs]
    server.close()  # cancels what is queued or running
    del keep
    X = synth.workload_series_3x1024().astype(np.float32)
    plan = Plan(make_params(3, 1024, precision=capi.FP32_MIXED, transition_len=0, max_imfs=8))
    _, _, n = plan.decompose(torch.from_numpy(X).cuda())
    plan.close()
    assert n >= 3


def test_server_large_request_lane_results_equal_alone():
    """A request of at least 2^21 serialized samples runs in the server's second lane
    (its own worker and stream, 512-sample pass tiles) while small requests keep arriving;
    every result equals the same input decomposed alone with the same tile (FP32 results
    depend on the tile, which decides where the spline system is partitioned)."""
    base = make_params(1600, 1600, precision=capi.FP32_MIXED, transition_len=0, max_imfs=6)
    server = Server(base, 2 << 30, 8)
    big = synth.grating_image(1500, 4)  # 2.25 M samples
    items = [(big, capi.ORDER_ROWS)] + _mix(52)
    xs = [torch.from_numpy(np.asarray(X, np.float32)).cuda() for X, _ in items]
    subs = [server.submit(x, order=o) for x, (_, o) in zip(xs, items)]
    res = _wait(server, [s[0] for s in subs])
    server.close()
    for (X, order), x, (t, imfs, r) in zip(items, xs, subs):
        assert res[t].status == capi.SEMD_OK
        plan = Plan(make_params(*X.shape, precision=capi.FP32_MIXED, transition_len=0,
                                max_imfs=6, order=order))
        if X.size >= 1 << 21:
            plan.tile = 512
        ai, ar, an = plan.decompose(x)
        torch.cuda.synchronize()
        plan.close()
        assert res[t].n_imfs == an
        assert torch.equal(imfs, ai) and torch.equal(r, ar), X.shape


def test_server_mixed_interface_solvers_results_equal_alone():
    """A small-lane request long enough for the cluster interface solve (a 700 x 700
    image: 1914 tiles) beside short ones: every launch of the lane then runs both
    interface-solve kernels, each on its own instances; every result equals the same
    input decomposed alone, bit for bit."""
    c, lo, hi = capi.serial_emd_interface_solve_shape(capi.FP32_MIXED, capi.SPLINE_NATURAL)
    base = make_params(1000, 1000, precision=capi.FP32_MIXED, transition_len=0, max_imfs=5)
    server = Server(base, 1 << 30, 8)
    big = synth.grating_image(700, 8)
    assert c == 0 or (700 * 700 + 255) // 256 >= lo
    items = [(big, capi.ORDER_ROWS)] + _mix(61)
    xs = [torch.from_numpy(np.asarray(X, np.float32)).cuda() for X, _ in items]
    subs = [server.submit(x, order=o) for x, (_, o) in zip(xs, items)]
    res = _wait(server, [s[0] for s in subs])
    server.close()
    for (X, order), x, (t, imfs, r) in zip(items, xs, subs):
        assert res[t].status == capi.SEMD_OK
        plan = Plan(make_params(*X.shape, precision=capi.FP32_MIXED, transition_len=0,
                                max_imfs=5, order=order))
        ai, ar, an = plan.decompose(x)
        torch.cuda.synchronize()
        plan.close()
        assert res[t].n_imfs == an
        assert torch.equal(imfs, ai) and torch.equal(r, ar), X.shape


# ------------------------------------------------------- failures made on the host

def test_server_allocation_failure_is_reported():
    """A budget no GPU can hold: creation fails with SEMD_ENOMEM and a message, nothing is
    left behind, and a server of a sensible size works afterwards."""
    base = make_params(16, 1024, precision=capi.FP32_MIXED, max_imfs=4)
    with pytest.raises(capi.SemdError) as ei:
        Server(base, 1 << 52, 4)
    assert ei.value.status == capi.SEMD_ENOMEM
    assert "server set-up" in capi.serial_emd_server_last_error(None)
    server = Server(base, 8 << 20, 2)
    x = torch.from_numpy(synth.tone_chirp_series(2, 700, 5).astype(np.float32)).cuda()
    t, _, _ = server.submit(x)
    assert _wait(server, [t])[t].status == capi.SEMD_OK
    server.close()


def test_server_poisoned_requests_do_not_disturb_others():
    """Requests whose samples are NaN or infinite (all of them, or a few) run to the end
    beside ordinary ones; the ordinary results stay bit-identical to decomposing alone."""
    base = make_params(64, 4096, precision=capi.FP32_MIXED, transition_len=-1, max_imfs=6)
    server = Server(base, 64 << 20, 6)
    items = _mix(61)
    bad = [np.full((3, 800), np.nan, np.float32), synth.tone_chirp_series(2, 900, 9)]
    bad[1] = bad[1].astype(np.float32)
    bad[1][0, 100:110] = np.inf
    bad[1][1, 400] = np.nan
    xs = [torch.from_numpy(np.asarray(X, np.float32)).cuda() for X, _ in items]
    xb = [torch.from_numpy(b).cuda() for b in bad]
    subs = []
    for k, (x, (_, o)) in enumerate(zip(xs, items)):
        subs.append(server.submit(x, order=o))
        if k == 2:
            tb = [server.submit(b) for b in xb]
    res = _wait(server, [s[0] for s in subs] + [t[0] for t in tb])
    server.close()
    for t, _, _ in tb:
        assert res[t].status == capi.SEMD_OK
    assert res[tb[0][0]].n_imfs == 0  # no sample of an all-NaN signal is an extremum
    for (X, order), x, (t, imfs, r) in zip(items, xs, subs):
        plan = Plan(make_params(*X.shape, precision=capi.FP32_MIXED, transition_len=-1,
                                max_imfs=6, order=order))
        ai, ar, an = plan.decompose(x)
        torch.cuda.synchronize()
        plan.close()
        assert res[t].status == capi.SEMD_OK and res[t].n_imfs == an
        assert torch.equal(imfs, ai) and torch.equal(r, ar), X.shape


def test_server_wait_time_limit():
    """serial_emd_wait with a time limit far below the request's run time returns
    SEMD_ETIMEOUT (None here) and leaves the request pending; a later wait gets it."""
    base = make_params(1024, 1024, precision=capi.FP32_MIXED, transition_len=0, max_imfs=10)
    server = Server(base, 1 << 30, 2)
    x = torch.from_numpy(synth.grating_image(1024, 77).astype(np.float32)).cuda()
    t, _, _ = server.submit(x)
    assert server.wait(t, 0.001) is None
    r = server.wait(t, 60000.0)
    assert r is not None and r.status == capi.SEMD_OK and r.n_imfs >= 1
    with pytest.raises(capi.SemdError):
        server.wait(t, 1.0)  # returned once
    with pytest.raises(capi.SemdError):
        server.wait(t + 1000, -1.0)
    server.close()
