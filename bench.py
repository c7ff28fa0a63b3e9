#!/usr/bin/env python
"""Benchmark of the GB300 Serial-EMD hot path.

One step = one full Serial-EMD decomposition (serialize, all sifting passes of all
IMFs, de-serialize) of the workload's synthetic input, resident in HBM. The metric
is serialized samples sifted per second (sum over instances of L x sifts, divided
by the device time of the step). Default workload: the 256 x 256 texture image
(gratings of period 4, 16 and 64 px plus noise), row-serialized without
transitions (L = 65536), 10 sifts per IMF, at most 10 IMFs, mirror boundary; the
FP32-mixed form gives `value`, the plain FP64 form is timed beside it, and the
batched FP32 form is also measured on the EEMD workload (512 x 512 image, 256
noise realizations in one batched run). The CPU oracle is timed on a bounded
sample of the same workload on the host cores (`cpu_baseline`), and
`--impl reference` times only the oracle.

N > 1 (torchrun): every rank runs its own replica of the workload (the method has
no cross-instance exchange), timing is max over ranks, `value` sums all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "serialized samples sifted/s: batched FP32 vs plain FP64 on GB300; p99 request latency"
UNIT = "samples*sifts/s"
L2_FLUSH_BYTES = 512 << 20
EEMD_NOISE_SEED = 20210629 + 4  # seed of the white noise the library draws for the EEMD leg
# DRAM bytes (read + write) of one k_pass launch of the default workload (pass launch 6 of a
# decomposition: an IMF-1 sift) per (tile, variant), from an ncu capture of that launch with
# the dram__bytes counters (cold caches, as ncu replays). Emptied whenever the pass kernel
# changes, until the changed kernel is captured again; an empty entry is reported as null.
PASS_TRAFFIC_TEXTURE = {(128, 0): 583168, (128, 1): 583680, (256, 0): 467456,
                        (256, 1): 465920, (512, 0): 412672, (512, 1): 412160}
# FP64-pipe lane operations (sm__inst_executed_pipe_fp64 x 32) of one k_pass<double> launch
# of the default workload, per (tile, variant), from an ncu capture of that launch; emptied
# whenever the pass kernel changes.
PASS_FP64_OPS_TEXTURE = {(128, 0): 173952 * 32, (128, 1): 173952 * 32, (256, 0): 134356 * 32,
                         (256, 1): 134356 * 32, (512, 0): 86475 * 32, (512, 1): 86475 * 32}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- workloads

def workload_inputs(name: str, trials: int = 256):
    from paper_2106_15319_gb300 import synth
    if name == "texture256":
        return {"X": synth.workload_texture_256(), "K": 10, "S": 10, "D": 0, "trials": 1,
                "desc": "256x256 texture (gratings 4/16/64 px + N(0,0.05^2)), row-serialized, "
                        "D=0, L=65536, 10 sifts/IMF, <=10 IMFs, mirror boundary"}
    if name == "eemd512":
        img = synth.workload_eemd_512(1)[0]
        return {"X": img, "W": None, "seed": EEMD_NOISE_SEED, "K": 10, "S": 10, "D": 0,
                "trials": trials,
                "desc": f"EEMD of a 512x512 grating image (L=262144), {trials} white-noise "
                        "realizations drawn on the device (Philox4x32-10, uniform, unit "
                        "variance; beta = 0.2 std), one batched run, 10 sifts/IMF, <=10 IMFs"}
    if name == "ceemdan_mask":
        X = synth.paper_mask_series()
        L = 6 * 1000 + 50 * 6 - 50
        return {"X": X, "W": synth.white_noise(100, L, 9001), "K": 10, "S": 10, "D": 50,
                "trials": 100, "method": "ceemdan",
                "desc": "serial-CEEMDAN of the 6-variate tone set (6 x 1000, D=50, L=6250), "
                        "100 noise realizations (beta_k = 0.2 std(r_k)), 10 sifts/mode, "
                        "<=10 modes"}
    if name in ("image1024", "image2048"):
        side = 1024 if name == "image1024" else 2048
        return {"X": synth.grating_image(side, 99), "K": 10, "S": 10, "D": 0, "trials": 1,
                "desc": f"{side}x{side} grating image (the serving mix's largest requests), "
                        f"row-serialized, D=0, L={side * side}, 10 sifts/IMF, <=10 IMFs"}
    if name == "series3x1024":
        return {"X": synth.workload_series_3x1024(), "K": 8, "S": 10, "D": 0, "trials": 1,
                "desc": "3-channel series x 1024 samples (tones + chirp + noise), D=0, L=3072, "
                        "10 sifts/IMF, <=8 IMFs"}
    raise SystemExit(f"unknown workload {name}")


def _flush_l2(buf):
    buf.add_(1)


def _call(plan, wl, x, noise, imfs, res, stream):
    """One decomposition of the workload through the public API (enqueued, no wait)."""
    if wl.get("method") == "ceemdan":
        plan.ceemdan(x, noise, imfs, res, stream=stream, wait=False)
    else:
        plan.decompose(x, noise, imfs, res, stream=stream, wait=False)


def run_ours(wl, precision, steps, warmup, device, flush, tile=0, tune=False, variant=None):
    import torch
    from paper_2106_15319_gb300 import capi
    from paper_2106_15319_gb300.serial_emd import Plan, make_params
    dt = np.float64 if precision == capi.FP64 else np.float32
    X = np.ascontiguousarray(wl["X"], dt)
    rows, cols = X.shape
    p = make_params(rows, cols, precision=precision, transition_len=wl["D"], max_imfs=wl["K"],
                    fixed_sifts=wl["S"], ensemble_trials=wl["trials"])
    plan = Plan(p)
    if tile:
        plan.tile = tile
    if variant is not None:
        plan.pass_variant = variant
    x = torch.from_numpy(X).to(device)
    noise = torch.from_numpy(np.ascontiguousarray(wl["W"], dt)).to(device) \
        if wl["trials"] > 1 and wl["W"] is not None else None
    if wl.get("seed") is not None:
        plan.noise_seed = wl["seed"]
    imfs, res = plan.outputs(rows, cols, device=device)
    stream = torch.cuda.Stream(device)
    shape = None
    if tune and not tile and variant is None:  # setup, before the warm-up: the autotuner
        # picks the pass shape
        r = plan.autotune(x, noise, outs=[(imfs, res)], repeats=3, stream=stream)
        shape = {"tile": r.tile, "ctas_per_sm": r.ctas_per_sm, "variant": r.variant,
                 "tuned_ms": r.ms,
                 "default_shape_ms": r.ms_default, "candidates": r.candidates}
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            _call(plan, wl, x, noise, imfs, res, stream)
        stream.synchronize()
        times = []
        for _ in range(steps):
            if flush is not None:
                _flush_l2(flush)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _call(plan, wl, x, noise, imfs, res, stream)
            b.record(stream)
            times.append((a, b))
        stream.synchronize()
    ms = [a.elapsed_time(b) for a, b in times]
    st = plan.stats()
    out = {"ms": ms, "sample_sifts": st.sample_sifts, "launches": st.kernel_launches,
           "graph": st.used_graph, "plan": plan, "x": x, "noise": noise, "imfs": imfs, "res": res,
           "stream": stream, "wl": wl,
           "shape": shape or {"tile": plan.tile, "ctas_per_sm": plan.pass_ctas,
                              "variant": plan.pass_variant}}
    return out


def profile_pass(run, steps, flush):
    """Replays the steps with events around every pass and reduce launch (no graph)."""
    import torch
    plan, stream = run["plan"], run["stream"]
    plan.set_options(use_graphs=False, profile=True)
    tot = {"pass_ms": 0.0, "pass_n": 0, "reduce_ms": 0.0, "reduce_n": 0, "bytes": 0}
    with torch.cuda.stream(stream):
        for _ in range(steps):
            if flush is not None:
                _flush_l2(flush)
            _call(plan, run["wl"], run["x"], run["noise"], run["imfs"], run["res"], stream)
            stream.synchronize()
            st = plan.stats()
            tot["pass_ms"] += st.pass_ms
            tot["pass_n"] += st.pass_launches
            tot["reduce_ms"] += st.reduce_ms
            tot["reduce_n"] += st.reduce_launches
            tot["bytes"] += st.pass_bytes
    plan.set_options(use_graphs=True, profile=False)
    return tot


def decompose_once(args, wl, device):
    """One decomposition of the workload with no warm-up and without CUDA graphs, so that
    every kernel is a separate launch in a fixed order (for ncu captures of one launch):
    precision from --forms (its first entry), pass shape from --tile / --pass-variant."""
    import torch
    from paper_2106_15319_gb300 import capi
    from paper_2106_15319_gb300.serial_emd import Plan, make_params
    prec = capi.FP64 if args.forms.split(",")[0] == "fp64" else capi.FP32_MIXED
    dt = np.float64 if prec == capi.FP64 else np.float32
    X = np.ascontiguousarray(wl["X"], dt)
    rows, cols = X.shape
    plan = Plan(make_params(rows, cols, precision=prec, transition_len=wl["D"],
                            max_imfs=wl["K"], fixed_sifts=wl["S"],
                            ensemble_trials=wl["trials"]))
    if args.tile:
        plan.tile = args.tile
    if args.pass_variant is not None:
        plan.pass_variant = args.pass_variant
    if wl.get("seed") is not None:
        plan.noise_seed = wl["seed"]
    noise = torch.from_numpy(np.ascontiguousarray(wl["W"], dt)).to(device) \
        if wl["trials"] > 1 and wl["W"] is not None else None
    plan.set_options(use_graphs=False, profile=False)
    _, _, n = plan.decompose(torch.from_numpy(X).to(device), noise)
    torch.cuda.synchronize()
    out = {"imfs": n, "tile": plan.tile, "variant": plan.pass_variant}
    plan.close()
    return out


def e2e_ours(wl, precision, steps, warmup, device):
    """Same metric through the public API with host buffers (H2D of the input, D2H of IMFs
    and residue inside the timed region)."""
    import torch
    from paper_2106_15319_gb300 import capi
    from paper_2106_15319_gb300.serial_emd import Plan, make_params
    dt = np.float64 if precision == capi.FP64 else np.float32
    X = np.ascontiguousarray(wl["X"], dt)
    rows, cols = X.shape
    p = make_params(rows, cols, precision=precision, transition_len=wl["D"], max_imfs=wl["K"],
                    fixed_sifts=wl["S"], ensemble_trials=wl["trials"])
    plan = Plan(p)
    hx = torch.from_numpy(X).pin_memory()
    hn = torch.from_numpy(np.ascontiguousarray(wl["W"], dt)).pin_memory() \
        if wl["trials"] > 1 and wl["W"] is not None else None
    if wl.get("seed") is not None:
        plan.noise_seed = wl["seed"]
    x = torch.empty_like(hx, device=device)
    noise = torch.empty_like(hn, device=device) if hn is not None else None
    imfs, res = plan.outputs(rows, cols, device=device)
    h_imfs = torch.empty(imfs.shape, dtype=imfs.dtype).pin_memory()
    h_res = torch.empty(res.shape, dtype=res.dtype).pin_memory()
    stream = torch.cuda.Stream(device)
    bi = hx.numel() * hx.element_size() + (hn.numel() * hn.element_size() if hn is not None else 0)
    bo = h_imfs.numel() * h_imfs.element_size() + h_res.numel() * h_res.element_size()

    def step():
        x.copy_(hx, non_blocking=True)
        if noise is not None:
            noise.copy_(hn, non_blocking=True)
        _call(plan, wl, x, noise, imfs, res, stream)
        h_imfs.copy_(imfs, non_blocking=True)
        h_res.copy_(res, non_blocking=True)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        stream.synchronize()
    ms = a.elapsed_time(b) / steps
    ss = plan.stats().sample_sifts
    plan.close()
    return ms, ss, bi, bo


def fp32_imf_errors(wl, run):
    """Per-IMF relative L2 of the FP32 result against the FP64 oracle (untimed)."""
    from oracle import oracle as O
    X = np.asarray(np.asarray(wl["X"], np.float32), np.float64)
    oi, orr, on, _ = O.serial_emd(X, wl["D"], wl["K"], fixed_sifts=wl["S"])
    g = run["imfs"].double().cpu().numpy()
    floor = 1e-6 * np.linalg.norm(X)
    return [float(np.linalg.norm(g[k] - oi[k]) / max(np.linalg.norm(oi[k]), floor))
            for k in range(wl["K"])]


FP32_TAU = 2.0 ** -20  # knot decisions whose FP64 margin is below this (of max|h|) are ties


def _fp32_replay(h32, S, shape, sift_plans):
    """One IMF's sifting replayed two ways from the same single-precision input: the GPU's
    FP32 chain (single sifts through the C ABI with the decomposition's pass shape) and the
    oracle's FP64 chain. Returns (decisions agree at every sift, margin of the first
    differing knot decision relative to max|h|, or None)."""
    import torch
    from oracle import oracle as O
    from paper_2106_15319_gb300 import capi
    from paper_2106_15319_gb300.serial_emd import Plan, make_params
    key = (h32.size, shape)
    if key not in sift_plans:
        sp = Plan(make_params(1, max(h32.size, 8), precision=capi.FP32_MIXED))
        sp.tile, sp.pass_variant = shape
        sift_plans[key] = sp
    sp = sift_plans[key]
    g, o = h32.astype(np.float32), h32.copy()
    for j in range(S):
        ga, gb = O.extrema(g.astype(np.float64))
        oa, ob = O.extrema(o)
        if not (np.array_equal(ga, oa) and np.array_equal(gb, ob)):
            m = 0.0
            for q in np.concatenate([np.setxor1d(ga, oa), np.setxor1d(gb, ob)]):
                d = [abs(o[q] - o[q - 1])] if q >= 1 else []
                if q + 1 < o.size:
                    d.append(abs(o[q + 1] - o[q]))
                m = max(m, min(d))
            return False, m / max(np.abs(h32).max(), np.abs(o).max(), 1e-300)
        if j > 0 and (oa.size < 1 or ob.size < 1 or oa.size + ob.size < 3):
            break
        g = sp.sift(torch.from_numpy(g).to("cuda"))[0].cpu().numpy()
        o = O.sift(o)[0]
    return True, None


def fp32_imf_errors_given_input(x, imfs, K, S, shape, sift_plans=None):
    """Per-IMF relative L2 of an FP32 result against the oracle's IMF of the same input
    remainder (x minus the GPU's earlier IMFs, rounded to single precision), untimed, and
    per IMF whether its sifting took the FP64 chain's knot decisions at every sift (else the
    FP64 margin of the first differing decision: a tie single precision cannot resolve)."""
    from oracle import oracle as O
    own = sift_plans is None
    sift_plans = {} if own else sift_plans
    x = np.asarray(x, np.float64).reshape(-1)
    g = np.asarray(imfs, np.float64).reshape(K, -1)
    floor = 1e-6 * np.linalg.norm(x)
    r, errs, exempt, margins = x.copy(), [], [], []
    for k in range(K):
        if not np.any(g[k]):
            break
        h32 = r.astype(np.float32).astype(np.float64)
        oi, _, on, _ = O.emd(h32, 1, fixed_sifts=S)
        if on < 1:
            break
        errs.append(float(np.linalg.norm(g[k] - oi[0]) / max(np.linalg.norm(oi[0]), floor)))
        same, margin = _fp32_replay(h32, S, shape, sift_plans)
        exempt.append(not same)
        margins.append(margin)
        r = r - g[k]
    if own:
        for sp in sift_plans.values():
            sp.close()
    return {"rel_l2": errs, "exempt": exempt, "exempt_margin": margins,
            "max_rel_l2_not_exempt": max([e for e, x_ in zip(errs, exempt) if not x_],
                                         default=None),
            "n_exempt": int(sum(exempt)), "n_imfs": len(errs)}


def _trial_noise(wl, m, L):
    """Realization m of the EEMD leg's noise: the caller's array, or the library's
    generator (Philox4x32-10, stated by the oracle)."""
    from oracle import oracle as O
    if wl["W"] is not None:
        return np.asarray(wl["W"][m], np.float64)
    return O.white_noise(wl["seed"], 1, L, first=m)[0]


def _oracle_trial(args):
    """One EEMD trial through the oracle (a process-pool task): its sample-sifts."""
    x, w, beta, K, S = args
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    if isinstance(w, tuple):  # (seed, realization): drawn here by the generator
        w = O.white_noise(w[0], 1, x.size, first=w[1])[0]
    _, _, _, sifts = O.emd(x + beta * w, K, fixed_sifts=S)
    return int(np.sum(sifts)) * x.size


def _cpu_model() -> str:
    """The host CPU, for the oracle timings: /proc/cpuinfo's model name, else (Arm) its
    implementer and part numbers, else the machine type."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if fields.get("model name"):
        return fields["model name"]
    part = fields.get("CPU part")
    if part:
        names = {"0xd4f": "Neoverse V2"}
        return (f"{platform.machine()} {names.get(part, 'CPU part ' + part)} "
                f"(implementer {fields.get('CPU implementer', '?')})")
    return platform.machine()


def cpu_pool_eemd(wl, budget_s: float = 10.0):
    """The oracle on every host core: EEMD trials (independent EMDs) in a process pool
    (spawned, as CUDA is already initialized in this process), as many whole trials as
    about budget_s allows."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from oracle import oracle as O
    X = np.asarray(wl["X"], np.float64)
    x = O.serialize(X, wl["D"])
    beta = 0.2 * O.std(x)
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_trial, [(x[:4096], _trial_noise(wl, m, x.size)[:4096], beta,
                                     wl["K"], wl["S"]) for m in range(cores)]))  # warm up
        t0 = time.perf_counter()
        done, ss, m = 0, 0, 0
        while time.perf_counter() - t0 < budget_s and m < wl["trials"]:
            batch = range(m, min(m + cores, wl["trials"]))
            ss += sum(ex.map(_oracle_trial, [(x, wl["W"][j] if wl["W"] is not None
                                              else (wl["seed"], j), beta, wl["K"], wl["S"])
                                             for j in batch]))
            done += len(batch)
            m += len(batch)
        el = time.perf_counter() - t0
    return {"value": ss / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "sample": f"{done} of {wl['trials']} EEMD trials, FP64, one process per core"}


def _oracle_instance(args):
    """One independent instance of a batched workload through the oracle (also a
    process-pool task): its sample-sifts. args = (X (N, M), D, K, stop, fixed sifts)."""
    X, D, K, stop, S = args
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    _, _, _, sifts = O.serial_emd(X, D, K, stop=stop, fixed_sifts=S, sd_threshold=0.2,
                                  max_sifts=50)
    return int(np.sum(sifts)) * O.serial_length(X.shape[1], X.shape[0], D)


def _oracle_group(tasks):
    """Consecutive instances through the oracle in one process-pool task (fewer round
    trips for short instances): their sample-sifts."""
    return sum(_oracle_instance(a) for a in tasks)


def cpu_instances(tasks, what: str, budget_s: float = 10.0, group: int = 1):
    """The oracle on the independent instances of a batched workload (tasks: arguments of
    _oracle_instance in the workload's order), single-threaded in this process and then
    in a process pool with one process per host core (spawned, as CUDA is already
    initialized here), each over the leading instances that about budget_s allows; the
    pool hands out `group` consecutive instances at a time. Returns (single thread, all
    cores)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    t0 = time.perf_counter()
    done, ss = 0, 0
    while done < len(tasks) and (time.perf_counter() - t0 < budget_s or done == 0):
        ss += _oracle_instance(tasks[done])
        done += 1
    el = time.perf_counter() - t0
    one = {"value": ss / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "cpu_model": _cpu_model(),
           "sample": f"the first {done} of {len(tasks)} {what}, FP64, single thread"}
    cores = os.cpu_count() or 1
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        # start-up on the smallest instances
        list(ex.map(_oracle_instance, sorted(tasks, key=lambda a: a[0].size)[:cores]))
        # one group per process at a time; a process that finishes takes the next group
        # while the budget lasts, and the time runs until the last one finishes
        groups = [tasks[i:i + group] for i in range(0, len(tasks), group)]
        t0 = time.perf_counter()
        done, ss, nxt, run = 0, 0, 0, {}
        while nxt < len(groups) and len(run) < cores:
            run[ex.submit(_oracle_group, groups[nxt])] = len(groups[nxt])
            nxt += 1
        while run:
            fin, _ = cf.wait(set(run), return_when=cf.FIRST_COMPLETED)
            for f in fin:
                ss += f.result()
                done += run.pop(f)
            while (nxt < len(groups) and len(run) < cores
                   and time.perf_counter() - t0 < budget_s):
                run[ex.submit(_oracle_group, groups[nxt])] = len(groups[nxt])
                nxt += 1
        el = time.perf_counter() - t0
    take = "the next one" if group == 1 else f"the next {group}"
    return one, {"value": ss / el, "unit": UNIT, "cores": cores, "kind": "oracle",
                 "cpu_model": _cpu_model(),
                 "sample": f"the first {done} of {len(tasks)} {what}, FP64, one process "
                           f"per core, each taking {take} when it finishes"}


def cpu_baseline(wl, budget_s: float = 12.0, ss_per_step: int = 0):
    """The oracle as it stands, single-threaded, on a bounded sample of the workload."""
    from oracle import oracle as O
    X = np.asarray(wl["X"], np.float64)
    if wl.get("method") == "ceemdan":
        # whole CEEMDAN calls; the work per call is counted as the GPU counts it
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < budget_s or done == 0:
            O.serial_ceemdan(X, wl["D"], wl["K"], wl["W"], 0.2, fixed_sifts=wl["S"])
            done += 1
        el = time.perf_counter() - t0
        return {"value": ss_per_step * done / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                "cpu_model": _cpu_model(),
                "sample": f"{done} full serial-CEEMDAN calls of the workload, FP64, single "
                          "thread (samples*sifts per call as counted by the GPU run)",
                "ms_per_call": el / done * 1e3}
    if wl["trials"] > 1:
        x = O.serialize(X, wl["D"])
        beta = 0.2 * O.std(x)
        t0 = time.perf_counter()
        done, ss = 0, 0
        while time.perf_counter() - t0 < budget_s and done < wl["trials"]:
            _, _, n, sifts = O.emd(x + beta * _trial_noise(wl, done, x.size), wl["K"],
                                   fixed_sifts=wl["S"])
            ss += int(np.sum(sifts)) * x.size
            done += 1
        el = time.perf_counter() - t0
        return {"value": ss / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                "cpu_model": _cpu_model(),
                "sample": f"{done} of {wl['trials']} EEMD trials, FP64, single thread"}
    t0 = time.perf_counter()
    done, ss = 0, 0
    while time.perf_counter() - t0 < budget_s or done == 0:
        _, _, n, sifts = O.serial_emd(X, wl["D"], wl["K"], fixed_sifts=wl["S"])
        ss += int(np.sum(sifts)) * O.serial_length(X.shape[1], X.shape[0], wl["D"])
        done += 1
    el = time.perf_counter() - t0
    return {"value": ss / el, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": _cpu_model(),
            "sample": f"{done} full decompositions of the workload, FP64, single thread"}


# ----------------------------------------------------------------------------- arms

def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def max_over_ranks(v: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time (every rank calls it, in the same order)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, work_per_rank: float, ms_max: float) -> float:
    """Weak scaling, one replica per rank: the units all ranks processed over the slowest
    rank's time."""
    return world * work_per_rank / (ms_max * 1e-3)


def barrier(world, cuda: bool = True):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if cuda:
        torch.cuda.synchronize()


def arm_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload_inputs(args.workload, args.trials)
    if wl.get("method") == "ceemdan":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the EMD "
                          "workloads; serial-CEEMDAN is timed beside the GPU run "
                          "(cpu_baseline of --workload ceemdan_mask)"}), flush=True)
        return
    from oracle import oracle as O
    X = np.asarray(wl["X"], np.float64)
    # a step is a bounded sample of the workload (whole decompositions, or whole EEMD
    # trials) of about per_step_budget seconds
    per_step_budget = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    vals, step_ms = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(wl, budget_s=per_step_budget)
        if i >= args.warmup:
            vals.append(cb["value"])
            step_ms.append((time.perf_counter() - t0) * 1e3)
    v = statistics.mean(vals)
    cb["value"] = v
    cb["sample"] += " per step"
    L = O.serial_length(X.shape[1], X.shape[0], wl["D"])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(step_ms),
            "ms_per_decomposition": L * wl["S"] * wl["K"] / v * 1e3 * max(1, wl["trials"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["desc"], "L": L},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def arm_ours(args):
    import torch
    from paper_2106_15319_gb300 import capi
    world, rank, local = dist_setup(args)
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    capi.load()
    wl = workload_inputs(args.workload, args.trials)
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    peak, peak_kind = _peaks()
    if args.only_leg == "once":  # one decomposition of the workload, graphs off (profiling)
        print(json.dumps({"only_leg": "once", "result": decompose_once(args, wl, device)}),
              flush=True)
        return
    if args.only_leg:  # one extra leg alone (for profiling it), no headline line
        legs = {"batched": lambda: batched_eemd(args, device, flush, peak, peak_kind, world),
                "images": lambda: batched_images(args, device, flush, peak, peak_kind, world),
                "slices": lambda: standard_slices(args, device, flush, world),
                "ceemdan": lambda: ceemdan_legs(args, device, flush, world),
                "dsweep": lambda: d_sweep(args, device, world),
                "serving": lambda: serving(args, device),
                "large": lambda: large_images_leg(args, device, flush, world)}
        out = legs[args.only_leg]()
        if rank == 0:
            print(json.dumps({"only_leg": args.only_leg, "result": out}), flush=True)
        return

    barrier(world)
    with ClockSampler(local) as clk:
        r32 = run_ours(wl, capi.FP32_MIXED, args.steps, args.warmup, device, flush, args.tile,
                       tune=not args.no_tune, variant=args.pass_variant)
    barrier(world)
    ms32 = statistics.mean(r32["ms"])
    ms32_max = max_over_ranks(ms32, world)
    value = whole_job_rate(world, r32["sample_sifts"], ms32_max)

    fp64_roof = None
    if "fp64" in args.forms:
        r64 = run_ours(wl, capi.FP64, args.steps, args.warmup, device, flush, args.tile,
                       tune=not args.no_tune)
        ms64 = max_over_ranks(statistics.mean(r64["ms"]), world)
        v64 = world * r64["sample_sifts"] / (ms64 * 1e-3)
        r64_shape = r64["shape"]
        # the plain FP64 form is bound by GB300's narrow FP64 pipe: its pass kernel's FP64
        # instructions per launch (ncu) against the measured FP64 FMA rate
        prof64 = profile_pass(r64, 1, flush)
        avg64 = prof64["pass_ms"] / max(1, prof64["pass_n"])
        t64 = r64["plan"].launch_times(0)
        l6 = t64[5] if len(t64) > 5 else avg64  # pass launch 6, the one ncu counted
        peak64 = capi.serial_emd_fma_rate(capi.FP64, 4096) / 2.0  # FMA lane-ops, G/s
        ops = PASS_FP64_OPS_TEXTURE.get((r64_shape["tile"], r64_shape["variant"])) \
            if args.workload == "texture256" else None
        fp64_roof = {"bound": "alu", "kernel": "k_pass<double>", "unit": "G FP64 ops/s",
                     "peak": peak64, "peak_source": "measured: serial_emd_fma_rate (FP64 "
                     "FMA chains; 1 op = 1 lane FMA)", "avg_launch_us": avg64 * 1e3,
                     "launch": "pass launch 6 (an IMF-1 sift)", "launch_us": l6 * 1e3,
                     "fp64_ops_per_launch": ops,
                     "achieved": ops / (l6 * 1e-3) / 1e9 if ops else None,
                     "frac": ops / (l6 * 1e-3) / 1e9 / peak64 if ops else None}
        r64["plan"].close()
    else:
        ms64, v64, r64_shape = None, None, None

    prof = profile_pass(r32, args.steps, flush)
    pass_avg_ms = prof["pass_ms"] / max(1, prof["pass_n"])
    bytes_per_launch = prof["bytes"] / max(1, prof["pass_n"])
    achieved = bytes_per_launch / (pass_avg_ms * 1e-3) / 1e9

    if not args.no_e2e:
        e2e_ms, e2e_ss, bi, bo = e2e_ours(wl, capi.FP32_MIXED, args.steps, args.warmup, device)
        e2e_ms = max_over_ranks(e2e_ms, world)
        e2e = {"value": world * e2e_ss / (e2e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo, "ms_per_step": e2e_ms}
    else:
        e2e = None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; stands in for the paper's texture images)",
        "config": {"workload": wl["desc"], "form": "FP32-mixed (FP64 interface solve, "
                   "stop reductions and residue)", "L": int(r32["x"].numel()),
                   "sample_sifts_per_step": r32["sample_sifts"], "cuda_graph": bool(r32["graph"]),
                   "pass_shape": r32["shape"],
                   "l2": "flushed between timed steps (512 MB write); "
                         "the 65536-sample working set is L2-resident within a step",
                   "parallelism": f"replicas x{world}"},
        "plain_fp64": {"value": v64, "ms_per_step": ms64, "dtype": "f64",
                       "pass_shape": r64_shape, "roofline": fp64_roof},
        "fma_rate_gflops": {"fp64": capi.serial_emd_fma_rate(capi.FP64, 4096),
                            "fp32": capi.serial_emd_fma_rate(capi.FP32_MIXED, 4096)},
        "speedup_fp32_vs_fp64": value / v64 if v64 else None,
        "fp32_imf_rel_l2": None,
        "roofline": {"bound": "hbm", "kernel": "k_pass<float>", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind,
                     # the captures were of 256-sample tiles (64 CTAs); other tiles differ
                     "traffic": PASS_TRAFFIC_TEXTURE.get((r32["shape"]["tile"],
                                                          r32["shape"]["variant"]))
                     if args.workload == "texture256" else None,
                     "traffic_launch": "pass launch 6 (an IMF-1 sift), ncu, cold caches",
                     "avg_launch_us": pass_avg_ms * 1e3, "bytes_per_launch": bytes_per_launch,
                     "launches": prof["pass_n"], "reduce_avg_us":
                         prof["reduce_ms"] / max(1, prof["reduce_n"]) * 1e3,
                     "note": "events around every kernel launch of the sifting loop over a "
                             "replay of the timed steps (graphs off); working set L2-resident"},
        "e2e": e2e,
        "gpu_launches": int(r32["launches"]) * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0:
        if wl["trials"] == 1 and wl["D"] == 0:
            line["fp32_imf_rel_l2"] = fp32_imf_errors(wl, r32)
            sh = r32["shape"]
            line["fp32_imf_given_input"] = fp32_imf_errors_given_input(
                np.asarray(np.asarray(wl["X"], np.float32), np.float64),
                r32["imfs"].double().cpu().numpy(), wl["K"], wl["S"],
                (sh["tile"], sh["variant"]))
        if not args.no_batched:
            line["batched"] = batched_eemd(args, device, flush, peak, peak_kind, world)
            line["batched_images"] = batched_images(args, device, flush, peak, peak_kind,
                                                    world)
        if not args.no_batched:
            line["series_3x1024"] = series_leg(args, device, flush, world)
            line["large_images"] = large_images_leg(args, device, flush, world)
            line["standard_slices"] = standard_slices(args, device, flush, world)
            line["standard_slices"]["serial_over_slices_time"] = \
                line["ms_per_step"] / line["standard_slices"]["ms_per_step"]
        if not args.no_batched:
            line["ceemdan"] = ceemdan_legs(args, device, flush, world)
            line["d_sweep"] = d_sweep(args, device, world)
            line["paper_context"] = paper_context(line)
        if not args.no_serving:
            line["serving"] = serving(args, device)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, ss_per_step=r32["sample_sifts"])
        print(json.dumps(line), flush=True)
    elif not args.no_batched:  # the same collective calls as rank 0 (max over ranks)
        batched_eemd(args, device, flush, peak, peak_kind, world)
        batched_images(args, device, flush, peak, peak_kind, world)
        series_leg(args, device, flush, world)
        large_images_leg(args, device, flush, world)
        standard_slices(args, device, flush, world)
        ceemdan_legs(args, device, flush, world)
        d_sweep(args, device, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def batched_eemd(args, device, flush, peak, peak_kind, world):
    """The batched FP32 form on the EEMD workload (256 realizations in one run)."""
    from paper_2106_15319_gb300 import capi
    wl = workload_inputs("eemd512", args.trials)
    steps = max(1, min(args.steps, 5))
    r = run_ours(wl, capi.FP32_MIXED, steps, min(args.warmup, 3), device, flush,
                 tune=not args.no_tune)
    ms = max_over_ranks(statistics.mean(r["ms"]), world)
    prof = profile_pass(r, 1, flush)
    pass_avg_ms = prof["pass_ms"] / max(1, prof["pass_n"])
    bpl = prof["bytes"] / max(1, prof["pass_n"])
    ach = bpl / (pass_avg_ms * 1e-3) / 1e9
    out = {"workload": wl["desc"], "value": world * r["sample_sifts"] / (ms * 1e-3),
           "unit": UNIT, "ms_per_step": ms, "steps": steps, "dtype": "f32",
           "pass_shape": r["shape"],
           "roofline": {"bound": "hbm", "kernel": "k_pass<float>", "achieved": ach,
                        "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "peak_source": peak_kind, "avg_launch_us": pass_avg_ms * 1e3,
                        "bytes_per_launch": bpl, "launches": prof["pass_n"],
                        "reduce_avg_us": prof["reduce_ms"] / max(1, prof["reduce_n"]) * 1e3}}
    if int(os.environ.get("RANK", "0")) == 0 and not args.no_fp32_errors:
        out["fp32_realizations_given_input"] = eemd_trial_errors(wl, r, args.error_trials)
    r["plan"].close()
    if not args.no_e2e:
        e2e_ms, e2e_ss, bi, bo = e2e_ours(wl, capi.FP32_MIXED, steps, min(args.warmup, 3),
                                          device)
        e2e_ms = max_over_ranks(e2e_ms, world)
        out["e2e"] = {"value": world * e2e_ss / (e2e_ms * 1e-3), "unit": UNIT,
                      "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                      "ms_per_step": e2e_ms,
                      "note": "host buffers: the image in, the averaged IMFs and residue out; "
                              "the noise is drawn on the device"}
    if not args.no_cpu_baseline and int(os.environ.get("RANK", "0")) == 0:
        out["cpu_baseline"] = cpu_baseline(wl, 10.0)
        out["cpu_baseline_all_cores"] = cpu_pool_eemd(wl)
    return out


def eemd_trial_errors(wl, r, ntrials):
    """Per-IMF FP32 error of EEMD realizations 0..ntrials-1 (each read back from the
    plan after the timed run), against the oracle's IMF of the same remainder, with the
    knot-decision replay of fp32_imf_errors_given_input; untimed."""
    from oracle import oracle as O
    plan = r["plan"]
    K, S = wl["K"], wl["S"]
    x = O.serialize(np.asarray(np.asarray(wl["X"], np.float32), np.float64), wl["D"])
    sh = r["shape"]
    shape = (sh["tile"], sh["variant"])
    sift_plans, per = {}, []
    for m in range(ntrials):
        imfs, _, n, beta = plan.eemd_trial(m)
        wm = _trial_noise(wl, m, x.size)
        if wl["W"] is not None:  # the caller's noise is stored in the plan's precision
            wm = np.asarray(np.asarray(wm, np.float32), np.float64)
        xm = x + beta * wm
        per.append(fp32_imf_errors_given_input(xm, imfs.double().cpu().numpy(), K, S, shape,
                                               sift_plans))
    for sp in sift_plans.values():
        sp.close()
    ok = [e for d in per for e, x_ in zip(d["rel_l2"], d["exempt"]) if not x_]
    return {"realizations": ntrials, "per_realization": per,
            "max_rel_l2_not_exempt": max(ok, default=None),
            "n_exempt": int(sum(d["n_exempt"] for d in per)),
            "n_imfs": int(sum(d["n_imfs"] for d in per))}


def batched_images(args, device, flush, peak, peak_kind, world):
    """The batched uneven-images workload: 2048 blob-field images (side U{32..128}),
    row-serialized (D = 0), FP32-mixed, SD stop 0.2 (at most 50 sifts), <= 8 IMFs, every
    instance in each pass launch, the sifting loop decided on the device. The images are
    stored back to back in one tensor (the packed batch call); the same batch passed as
    2048 separate tensors is timed beside it (its host-side buffer checks are in the
    timed region too)."""
    import torch
    from paper_2106_15319_gb300 import capi, synth
    from paper_2106_15319_gb300.serial_emd import Plan, make_params
    imgs = synth.workload_uneven_images(args.images)
    side = max(im.shape[0] for im in imgs)
    p = make_params(side, side, precision=capi.FP32_MIXED, transition_len=0, max_imfs=8,
                    stop=capi.STOP_SD, sd_threshold=0.2, max_sifts=50)
    plan = Plan(p, max_batch=len(imgs))
    xs = [torch.from_numpy(np.ascontiguousarray(im, np.float32)).to(device) for im in imgs]
    outs = [plan.outputs(*x.shape, device=device) for x in xs]
    shapes = [tuple(im.shape) for im in imgs]
    flat = torch.cat([x.reshape(-1) for x in xs])
    samples = int(flat.numel())
    pimfs = torch.empty(8 * samples, dtype=torch.float32, device=device)
    pres = torch.empty(samples, dtype=torch.float64, device=device)
    stream = torch.cuda.Stream(device)
    steps = max(1, min(args.steps, 5))

    def run_packed():
        plan.decompose_packed(flat, shapes, pimfs, pres, stream=stream, wait=False)

    def run_list():
        plan.decompose_batch(xs, outs, stream=stream, wait=False)

    def timed(call):
        with torch.cuda.stream(stream):
            for _ in range(min(args.warmup, 3)):
                call()
            stream.synchronize()
            ms = []
            for _ in range(steps):
                _flush_l2(flush)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                call()
                b.record(stream)
                stream.synchronize()
                ms.append(a.elapsed_time(b))
        return statistics.mean(ms)

    ms_list = max_over_ranks(timed(run_list), world)
    ms_step = max_over_ranks(timed(run_packed), world)
    st = plan.stats()
    plan.set_options(use_graphs=True, profile=True)
    with torch.cuda.stream(stream):
        _flush_l2(flush)
        run_packed()
        stream.synchronize()
    pr = plan.stats()
    pass_avg_ms = pr.pass_ms / max(1, pr.pass_launches)
    bpl = pr.pass_bytes / max(1, pr.pass_launches)
    ach = bpl / (pass_avg_ms * 1e-3) / 1e9
    n_imfs, sifts = plan.counts(len(xs))
    plan.close()
    cpu = {}
    if not args.no_cpu_baseline and int(os.environ.get("RANK", "0")) == 0:
        from oracle import oracle as O
        tasks = [(np.asarray(im, np.float32).astype(np.float64), 0, 8, O.STOP_SD, 10)
                 for im in imgs]
        one, allc = cpu_instances(tasks, "images (SD stop 0.2, <= 8 IMFs)", group=8)
        cpu = {"cpu_baseline": one, "cpu_baseline_all_cores": allc}
    return {"workload": f"{len(xs)} uneven blob-field images, side U{{32..128}} "
                        f"({samples} samples), row-serialized D=0, SD stop 0.2 (max 50 "
                        "sifts), <=8 IMFs, all instances in every pass launch, stored back "
                        "to back in one tensor",
            "value": world * st.sample_sifts / (ms_step * 1e-3), "unit": UNIT,
            "ms_per_step": ms_step, "steps": steps, "dtype": "f32",
            "ms_per_step_tensor_list": ms_list,
            "sifts_per_imf_mean": float(np.sum(sifts)) / max(1, int(np.sum(n_imfs))),
            "roofline": {"bound": "hbm", "kernel": "k_pass<float>", "achieved": ach,
                         "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "peak_source": peak_kind, "avg_launch_us": pass_avg_ms * 1e3,
                         "bytes_per_launch": bpl, "launches": pr.pass_launches,
                         "reduce_avg_us": pr.reduce_ms / max(1, pr.reduce_launches) * 1e3},
            **cpu}


def serving(args, device):
    """The serving mix: Poisson arrivals of requests, half tone+chirp series (2..16
    channels x 1k..64k samples), half grating images (side 32..1024 px, plus a 2 % tail
    of 2048^2 images), transitions D = round(0.2 M), FP32-mixed, 10 sifts/IMF, <= 10
    IMFs, one server with a 40 GB device budget and 64 slots. One set of requests is drawn
    (arrival gaps at rate 1, scaled by 1/rate for each rate); each rate's requests are
    submitted at their arrival times, and "saturation" submits them all at once. Latency
    is the server's submit -> outputs-written time (queue + run)."""
    import time as _t
    import torch
    from paper_2106_15319_gb300 import capi, synth
    from paper_2106_15319_gb300.serial_emd import Server, make_params, serialized_length
    base = make_params(2048, 2048, precision=capi.FP32_MIXED, transition_len=-1, max_imfs=10,
                       fixed_sifts=10)
    out = {"workload": "serving mix: Poisson arrivals; 50% series 2..16 ch x 1k..64k, 50% "
                       "images 32..1024 px (+2% 2048^2), D=round(0.2 M), FP32-mixed, 10 "
                       "sifts/IMF, <=10 IMFs, 40 GB budget, 64 slots",
           "latency": "submit -> outputs written, measured by the server", "rates": []}
    nreq = args.serve_requests
    mix = synth.serving_mix(nreq, 20210629 + 5, 1.0)
    xs = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device) for _, _, a in mix]
    server = Server(base, 40 << 30, 64)
    outs = [server.outputs(*x.shape, device=device) for x in xs]
    torch.cuda.synchronize()
    sizes = [serialized_length(*x.shape) for x in xs]
    try:
        for rate in list(args.serve_rates) + [float("inf")]:
            # slow rates: a bounded prefix of the requests, so that the leg ends in minutes
            n = nreq if rate >= 100 else min(nreq, int(args.serve_slow_seconds * rate))
            arr = [0.0 if rate == float("inf") else mix[k][0] / rate for k in range(n)]
            pend, res = {}, {}
            t0 = _t.perf_counter()
            i = 0
            while i < n or pend:
                now = _t.perf_counter() - t0
                while i < n and arr[i] <= now:
                    t, _, _ = server.submit(xs[i], outs[i][0], outs[i][1])
                    pend[t] = i
                    i += 1
                for t in list(pend):
                    r = server.poll(t)
                    if r is not None:
                        res[pend.pop(t)] = (r, _t.perf_counter() - t0)
                if i < n and not pend:
                    _t.sleep(max(0.0, min(arr[i] - now, 0.002)))
                elif pend:
                    _t.sleep(0.0002)
            wall = max(v[1] for v in res.values()) - arr[0]
            lat = np.array([r.queue_ms + r.run_ms for r, _ in res.values()])
            lat_small = np.array([r.queue_ms + r.run_ms for k, (r, _) in res.items()
                                  if sizes[k] < (1 << 21)])
            lat_big = np.array([r.queue_ms + r.run_ms for k, (r, _) in res.items()
                                if sizes[k] >= (1 << 21)])
            ss = sum(r.sifts * sizes[k] for k, (r, _) in res.items())
            ok = all(r.status == capi.SEMD_OK for r, _ in res.values())
            out["rates"].append({
                "rate_hz": "saturation" if rate == float("inf") else rate, "requests": n,
                "all_ok": bool(ok),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()),
                "small_requests": {"count": int(lat_small.size),
                                   "p50_ms": float(np.percentile(lat_small, 50)),
                                   "p99_ms": float(np.percentile(lat_small, 99))}
                if lat_small.size else None,
                "large_requests": {"count": int(lat_big.size),
                                   "p50_ms": float(np.percentile(lat_big, 50)),
                                   "max_ms": float(lat_big.max())} if lat_big.size else None,
                "served_per_s": n / wall, "samples_sifts_per_s": ss / wall,
                "samples": int(sum(sizes[:n]))})
    finally:
        server.close()
    del xs, outs
    if not args.no_cpu_baseline and int(os.environ.get("RANK", "0")) == 0:
        # the requests in arrival order, each decomposed alone (D = round(0.2 M), one
        # signal: D = 0), as the server decomposes them
        from oracle import oracle as O
        tasks = []
        for _, _, a in mix:
            X = np.asarray(a, np.float32).astype(np.float64)
            X = X.reshape(1, -1) if X.ndim == 1 else X
            D = 0 if X.shape[0] == 1 else int(round(0.2 * X.shape[1]))
            tasks.append((X, D, 10, O.STOP_FIXED, 10))
        out["cpu_baseline"], out["cpu_baseline_all_cores"] = cpu_instances(
            tasks, "requests of the mix, in arrival order")
    return out


def series_leg(args, device, flush, world):
    """The 3-channel series (3 x 1024 samples, tones + chirp + noise, D = 0, L = 3072, 10
    sifts per IMF, at most 8 IMFs), plain FP64 and FP32-mixed, one decomposition per step,
    beside the oracle on one host core."""
    from paper_2106_15319_gb300 import capi
    wl = workload_inputs("series3x1024")
    out = {"workload": wl["desc"]}
    for tag, prec in (("fp64", capi.FP64), ("fp32", capi.FP32_MIXED)):
        r = run_ours(wl, prec, max(1, min(args.steps, 10)), min(args.warmup, 3), device, flush,
                     tune=not args.no_tune)
        ms = max_over_ranks(statistics.mean(r["ms"]), world)
        out[tag] = {"ms_per_step": ms, "value": world * r["sample_sifts"] / (ms * 1e-3),
                    "unit": UNIT, "pass_shape": r["shape"], "cuda_graph": bool(r["graph"])}
        r["plan"].close()
    if not args.no_cpu_baseline and int(os.environ.get("RANK", "0")) == 0:
        out["cpu_baseline"] = cpu_baseline(wl, budget_s=3.0)
    return out


def large_images_leg(args, device, flush, world):
    """Single long instances, whose interface solve runs on a thread-block cluster: the
    1024 x 1024 and 2048 x 2048 grating images in FP32-mixed (10 sifts per IMF, at most 10
    IMFs), one decomposition per step (graph replay), and the per-launch device time of
    the pass and interface-solve kernels from one profiled decomposition."""
    from paper_2106_15319_gb300 import capi
    out = {"shape": dict(zip(("cluster_ctas", "min_tiles", "max_tiles"),
                             capi.serial_emd_interface_solve_shape(capi.FP32_MIXED)))}
    for name in ("image1024", "image2048"):
        wl = workload_inputs(name)
        r = run_ours(wl, capi.FP32_MIXED, max(1, min(args.steps, 5)), min(args.warmup, 3),
                     device, flush, tune=False)
        ms = max_over_ranks(statistics.mean(r["ms"]), world)
        prof = profile_pass(r, 1, flush)
        out[name] = {"workload": wl["desc"], "ms_per_step": ms,
                     "value": world * r["sample_sifts"] / (ms * 1e-3), "unit": UNIT,
                     "pass_shape": r["shape"], "cuda_graph": bool(r["graph"]),
                     "pass_avg_us": 1e3 * prof["pass_ms"] / max(1, prof["pass_n"]),
                     "interface_solve_avg_us": 1e3 * prof["reduce_ms"] / max(1, prof["reduce_n"])}
        r["plan"].close()
    return out


def standard_slices(args, device, flush, world):
    """The paper's standard-version baseline (Sec. 4) on the default workload: the 256
    rows of the 256 x 256 texture decomposed one by one (no serialization), all rows in
    one batched run, against the serial form of the same input."""
    import torch
    from paper_2106_15319_gb300 import capi
    from paper_2106_15319_gb300.serial_emd import Plan, make_params
    wl = workload_inputs("texture256")
    X = np.ascontiguousarray(wl["X"], np.float32)
    rows, cols = X.shape
    plan = Plan(make_params(1, cols, precision=capi.FP32_MIXED, transition_len=0,
                            max_imfs=wl["K"], fixed_sifts=wl["S"]), max_batch=rows)
    x = torch.from_numpy(X).to(device)
    imfs, res = plan.outputs(rows, cols, device=device)
    stream = torch.cuda.Stream(device)
    steps = max(1, min(args.steps, 10))
    with torch.cuda.stream(stream):
        for _ in range(min(args.warmup, 3)):
            plan.decompose_slices(x, imfs, res, stream=stream, wait=False)
        stream.synchronize()
        ms = []
        for _ in range(steps):
            _flush_l2(flush)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.decompose_slices(x, imfs, res, stream=stream, wait=False)
            b.record(stream)
            stream.synchronize()
            ms.append(a.elapsed_time(b))
    st = plan.stats()
    n, _ = plan.counts(rows)
    plan.close()
    m = max_over_ranks(statistics.mean(ms), world)
    return {"workload": f"{rows} rows of the 256x256 texture, each decomposed alone "
                        f"(1 x {cols} signals, no transitions), one batched run, "
                        f"{wl['S']} sifts/IMF, <={wl['K']} IMFs",
            "value": world * st.sample_sifts / (m * 1e-3), "unit": UNIT, "ms_per_step": m,
            "steps": steps, "dtype": "f32", "imfs_per_row_mean": float(np.mean(n))}


def ceemdan_legs(args, device, flush, world):
    """Serial-CEEMDAN (Sec. 2.2 Steps 1-4 inside Sec. 3) on stand-ins for the two inputs the
    paper times it on: its 6-variate tone set (6 x 1000 samples, D = 50) and a 101 x 101
    texture image (D = 20), with 100 noise realizations, noise_rel_std 0.2, 10 sifts per
    mode, at most 10 modes. One step = one full CEEMDAN call (EMD of the noise
    realizations, then every stage). The paper's CPU times are context only."""
    import torch
    from paper_2106_15319_gb300 import capi, synth
    from paper_2106_15319_gb300.serial_emd import Plan, make_params
    trials = 100
    # (name, input, D, the paper's serial-CEEMDAN and serial-EEMD CPU times in ms)
    cases = [("mask6x1000_D50", synth.paper_mask_series(), 50, 1154.97, 397.92),
             ("texture101_D20", synth.grating_image(101, 2106), 20, 20580.0, 6410.0)]
    out = {}
    steps = max(1, min(args.steps, 5))
    for name, X0, D, paper_ms, paper_eemd_ms in cases:
        rows, cols = X0.shape
        N, M = rows, cols
        L = M * N + D * N - D
        for prec, np_t in ((capi.FP32_MIXED, np.float32), (capi.FP64, np.float64)):
            X = np.ascontiguousarray(X0, np_t)
            w = synth.white_noise(trials, L, 9001).astype(np_t)
            plan = Plan(make_params(rows, cols, precision=prec, transition_len=D, max_imfs=10,
                                    ensemble_trials=trials, noise_rel_std=0.2))
            x = torch.from_numpy(X).to(device)
            wt = torch.from_numpy(w).to(device)
            modes, res = plan.outputs(rows, cols, device=device)
            stream = torch.cuda.Stream(device)
            if not args.no_tune:  # setup: the pass shape of the ensemble's sifting
                plan.autotune(x, wt, outs=[(modes, res)], repeats=2, stream=stream)
            def timed(call):
                ms = []
                with torch.cuda.stream(stream):
                    for _ in range(min(args.warmup, 3)):
                        call()
                    stream.synchronize()
                    for _ in range(steps):
                        _flush_l2(flush)
                        a = torch.cuda.Event(enable_timing=True)
                        b = torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        call()
                        b.record(stream)
                        stream.synchronize()
                        ms.append(a.elapsed_time(b))
                return max_over_ranks(statistics.mean(ms), world)

            # serial-EEMD of the same input and noise (the paper times both)
            eemd_ms = timed(lambda: plan.decompose(x, wt, modes, res, stream=stream, wait=False))
            m = timed(lambda: plan.ceemdan(x, wt, modes, res, stream=stream, wait=False))
            st = plan.stats()
            n = plan.counts(1)[0][0]
            shape = {"tile": plan.tile, "ctas_per_sm": plan.pass_ctas,
                     "variant": plan.pass_variant}
            plan.close()
            key = f"{name}_{'fp32' if prec == capi.FP32_MIXED else 'fp64'}"
            out[key] = {"ms_per_step": m, "value": world * st.sample_sifts / (m * 1e-3),
                        "unit": UNIT, "modes": int(n), "L": L, "trials": trials,
                        "launches_per_step": int(st.kernel_launches),
                        "cuda_graph": bool(st.used_graph),
                        "pass_shape": shape,
                        "paper_cpu_ms_context": paper_ms,
                        "eemd_ms_per_step": eemd_ms,
                        "paper_eemd_cpu_ms_context": paper_eemd_ms}
    return out


def paper_context(line):
    """The paper's own timings (Sec. 4; one i7-6700HQ laptop CPU, language and precision
    not stated) beside this run's GPU times of the same method on stand-in inputs. Context,
    not a target."""
    out = {"hardware": "paper: Intel i7-6700HQ laptop CPU (Sec. 4); here: one GB300",
           "rows": []}
    ds = {r["D"]: r for r in line.get("d_sweep", {}).get("rows", [])}
    ce = line.get("ceemdan", {})
    if 50 in ds:
        out["rows"].append({"what": "serial-EMD, 6-variate tone set, D=50", "paper_ms": 10.96,
                            "ours_ms_fp32": ds[50]["emd_fixed10_ms"]})
    if "mask6x1000_D50_fp32" in ce:
        c32, c64 = ce["mask6x1000_D50_fp32"], ce.get("mask6x1000_D50_fp64", {})
        out["rows"].append({"what": "serial-EEMD, 6-variate tone set, D=50, 100 realizations",
                            "paper_ms": 397.92, "ours_ms_fp32": c32["eemd_ms_per_step"],
                            "ours_ms_fp64": c64.get("eemd_ms_per_step")})
        out["rows"].append({"what": "serial-CEEMDAN, 6-variate tone set, D=50, "
                                    "100 realizations", "paper_ms": 1154.97,
                            "ours_ms_fp32": c32["ms_per_step"],
                            "ours_ms_fp64": c64.get("ms_per_step")})
    if "texture101_D20_fp32" in ce:
        c32, c64 = ce["texture101_D20_fp32"], ce.get("texture101_D20_fp64", {})
        out["rows"].append({"what": "serial-EEMD, 101x101 texture (ATI stand-in), D=20",
                            "paper_ms": 6410.0, "ours_ms_fp32": c32["eemd_ms_per_step"],
                            "ours_ms_fp64": c64.get("eemd_ms_per_step")})
        out["rows"].append({"what": "serial-CEEMDAN, 101x101 texture (ATI stand-in), D=20",
                            "paper_ms": 20580.0, "ours_ms_fp32": c32["ms_per_step"],
                            "ours_ms_fp64": c64.get("ms_per_step")})
    return out


def _tone_similarity(imfs, tones, mask):
    """IMF quality on the 6-variate tone set: for IMF k (k = 1, 2) and each variate, the
    normalized correlation of the IMF with the k-th highest tone the mask puts into that
    variate (the component an ideal decomposition would return), averaged over variates."""
    out = []
    for k in range(2):
        cs = []
        for v in range(mask.shape[1]):
            present = [j for j in range(mask.shape[0]) if mask[j, v]]
            if k >= len(present):
                continue
            c, ref = imfs[k, v], tones[present[k]]
            den = np.linalg.norm(c) * np.linalg.norm(ref)
            cs.append(float(np.dot(c, ref) / den) if den > 0 else 0.0)
        out.append(float(np.mean(cs)))
    return out


def d_sweep(args, device, world):
    """Transition length D (Sec. 3.2) from 1 to 500 (half a variate) on the paper's
    6-variate tone set (6 x 1000), as in Sec. 4.1: device time of serial EMD (fixed 10
    sifts and SD stop 0.2), serial EEMD and serial CEEMDAN (100 realizations, fixed 10
    sifts), FP32-mixed, and the IMF-tone correlation of IMF 1 and 2 for both EMD stops."""
    import torch
    from paper_2106_15319_gb300 import capi, synth
    from paper_2106_15319_gb300.serial_emd import Plan, make_params
    tones, mask = synth.paper_mask_components()
    X = np.ascontiguousarray(synth.paper_mask_series(), np.float32)
    rows, cols = X.shape
    x = torch.from_numpy(X).to(device)
    trials = 100
    stream = torch.cuda.Stream(device)

    def timed(fn, steps):
        with torch.cuda.stream(stream):
            for _ in range(2):
                fn()
            stream.synchronize()
            ms = []
            for _ in range(steps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                stream.synchronize()
                ms.append(a.elapsed_time(b))
        return max_over_ranks(statistics.mean(ms), world)

    rows_out = []
    for D in (1, 10, 20, 50, 100, 200, 500):
        L = cols * rows + D * rows - D
        rec = {"D": D, "L": L}
        for tag, kw in (("emd_fixed10", {}), ("emd_sd0.2", {"stop": capi.STOP_SD})):
            plan = Plan(make_params(rows, cols, transition_len=D, max_imfs=10, **kw))
            imfs, res = plan.outputs(rows, cols, device=device)
            rec[tag + "_ms"] = timed(lambda: plan.decompose(x, None, imfs, res, stream=stream,
                                                            wait=False), 5)
            n, sifts = plan.counts(1)
            rec[tag + "_imfs"] = int(n[0])
            rec[tag + "_sifts"] = int(sum(sifts[0]))
            rec[tag + "_tone_corr"] = _tone_similarity(imfs.double().cpu().numpy(), tones, mask)
            plan.close()
        w = torch.from_numpy(synth.white_noise(trials, L, 9002).astype(np.float32)).to(device)
        plan = Plan(make_params(rows, cols, transition_len=D, max_imfs=10,
                                ensemble_trials=trials, noise_rel_std=0.2))
        imfs, res = plan.outputs(rows, cols, device=device)
        rec["eemd_ms"] = timed(lambda: plan.decompose(x, w, imfs, res, stream=stream,
                                                      wait=False), 3)
        rec["ceemdan_ms"] = timed(lambda: plan.ceemdan(x, w, imfs, res, stream=stream,
                                                       wait=False), 3)
        plan.close()
        rows_out.append(rec)
    return {"workload": "6-variate tone set (32/16/8/2 Hz by the pickup mask), 6 x 1000, "
                        f"FP32-mixed, <= 10 IMFs; EEMD/CEEMDAN {trials} realizations",
            "rows": rows_out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="texture256",
                    choices=["texture256", "eemd512", "series3x1024", "ceemdan_mask",
                             "image1024", "image2048"])
    ap.add_argument("--trials", type=int, default=256, help="EEMD realizations (eemd512)")
    ap.add_argument("--forms", default="fp32,fp64", help="comma list of fp32, fp64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="pass-kernel tile (0: the plan's)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--images", type=int, default=2048, help="batched uneven images")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-rates", type=float, nargs="+",
                    default=[10.0, 30.0, 100.0, 300.0, 1000.0])
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-slow-seconds", type=float, default=30.0,
                    help="rates below 100/s submit at most this many seconds of arrivals")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default pass shape (no autotuning before the warm-up)")
    ap.add_argument("--only-leg", default=None,
                    choices=["batched", "images", "slices", "ceemdan", "dsweep", "serving",
                             "large", "once"],
                    help="run one extra leg alone and print its result (for profiling); "
                         "once: one decomposition of --workload, graphs off, no warm-up")
    ap.add_argument("--no-fp32-errors", action="store_true",
                    help="skip the untimed FP32 per-IMF error report of the EEMD leg")
    ap.add_argument("--error-trials", type=int, default=4,
                    help="EEMD realizations whose FP32 IMFs are checked against the oracle")
    ap.add_argument("--pass-variant", type=int, default=None, choices=[0, 1],
                    help="register budget of the FP32 pass kernel (no autotuning)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        arm_reference(args)
    else:
        arm_ours(args)


if __name__ == "__main__":
    main()
