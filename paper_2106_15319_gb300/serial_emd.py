"""Python front end of the GB300 Serial-EMD library.

`Plan` owns a C-ABI plan (device workspaces reserved once); `decompose` is the
one-call convenience form. Tensors are torch CUDA tensors; every computation runs
in libserial_emd.so.
"""
from __future__ import annotations

import torch

from . import capi

_DTYPE = {capi.FP64: torch.float64, capi.FP32_MIXED: torch.float32}


def make_params(rows: int, cols: int, *, order: int = capi.ORDER_ROWS, transition_len: int = -1,
                max_imfs: int = 10, stop: int = capi.STOP_FIXED, fixed_sifts: int = 10,
                sd_threshold: float = 0.2, max_sifts: int = 50,
                boundary: int = capi.BOUNDARY_MIRROR, mirror_knots: int = 2,
                precision: int = capi.FP32_MIXED, ensemble_trials: int = 1,
                noise_rel_std: float = 0.2, s_number: int = 4,
                spline_end: int = capi.SPLINE_NATURAL) -> capi.semd_params:
    return capi.serial_emd_default_params(
        rows=rows, cols=cols, order=order, transition_len=transition_len, max_imfs=max_imfs,
        stop=stop, fixed_sifts=fixed_sifts, sd_threshold=sd_threshold, max_sifts=max_sifts,
        boundary=boundary, mirror_knots=mirror_knots, precision=precision,
        ensemble_trials=ensemble_trials, noise_rel_std=noise_rel_std, s_number=s_number,
        spline_end=spline_end)


def serialized_length(rows: int, cols: int, order: int = capi.ORDER_ROWS,
                      transition_len: int = -1) -> int:
    M, N = (cols, rows) if order == capi.ORDER_ROWS else (rows, cols)
    D = round(0.2 * M) if transition_len < 0 else transition_len
    if N == 1:
        D = 0
    return M * N + D * N - D


class Plan:
    def __init__(self, params: capi.semd_params, max_batch: int = 1, mem_budget: int = 0):
        self.params = params
        self.handle = capi.serial_emd_plan(params, max_batch, mem_budget)
        self.dtype = _DTYPE[params.precision]
        self.max_batch = max_batch

    @property
    def nbytes(self) -> int:
        return capi.serial_emd_plan_bytes(self.handle)

    def close(self):
        if self.handle:
            capi.serial_emd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, rows: int, cols: int, device="cuda"):
        imfs = torch.empty((self.params.max_imfs, rows, cols), dtype=self.dtype, device=device)
        res = torch.empty((rows, cols), dtype=torch.float64, device=device)
        return imfs, res

    def decompose(self, x: torch.Tensor, noise: torch.Tensor | None = None, imfs=None,
                  residue=None, stream=None, wait: bool = True):
        assert x.is_cuda and x.dtype == self.dtype and x.is_contiguous()
        if imfs is None:
            imfs, residue = self.outputs(*x.shape, device=x.device)
        n = capi.serial_emd_decompose(self.handle, x, noise, imfs, residue, stream, wait)
        return imfs, residue, n

    def ceemdan(self, x: torch.Tensor, noise: torch.Tensor, modes=None, residue=None,
                stream=None, wait: bool = True):
        """Serial-CEEMDAN of x with the noise realizations (trials, L) (an ensemble plan).
        Returns (modes (K, rows, cols), residue, mode count or None when not waiting)."""
        assert x.is_cuda and x.dtype == self.dtype and x.is_contiguous()
        assert noise.is_cuda and noise.dtype == self.dtype and noise.is_contiguous()
        if modes is None:
            modes, residue = self.outputs(*x.shape, device=x.device)
        n = capi.serial_emd_ceemdan(self.handle, x, noise, modes, residue, stream, wait)
        return modes, residue, n

    def decompose_batch(self, xs, outs=None, stream=None, wait: bool = True):
        if outs is None:
            outs = [self.outputs(*x.shape, device=x.device) for x in xs]
        items = [(x, o[0], o[1]) for x, o in zip(xs, outs)]
        n = capi.serial_emd_decompose_batch(self.handle, items, stream, wait)
        return outs, n

    def decompose_packed(self, x: torch.Tensor, shapes, imfs=None, residue=None, stream=None,
                         wait: bool = True):
        """decompose_batch of inputs stored back to back in one flat tensor x (input i,
        shapes[i] = (rows, cols), at the sum of the earlier inputs' sizes); imfs holds each
        input's K IMFs back to back (K * rows * cols elements each), residue each input's
        residue. Returns (imfs, residue, IMF count per input, or None without wait)."""
        import numpy as np
        total = int(np.prod(np.asarray(shapes, dtype=np.int64).reshape(-1, 2), axis=1).sum())
        if imfs is None:
            imfs = torch.empty(self.params.max_imfs * total, dtype=self.dtype, device=x.device)
            residue = torch.empty(total, dtype=torch.float64, device=x.device)
        n = capi.serial_emd_decompose_packed(self.handle, x, shapes, imfs, residue, stream, wait)
        return imfs, residue, n

    def decompose_slices(self, x: torch.Tensor, imfs=None, residue=None, stream=None,
                         wait: bool = True):
        """Slice-wise standard EMD: every row of x decomposed on its own (the plan must hold
        one row, with max_batch >= rows). Returns (imfs, residue, n per row)."""
        assert x.is_cuda and x.dtype == self.dtype and x.is_contiguous() and x.dim() == 2
        if imfs is None:
            imfs, residue = self.outputs(*x.shape, device=x.device)
        n = capi.serial_emd_decompose_slices(self.handle, x, imfs, residue, stream, wait)
        return imfs, residue, n

    @property
    def tile(self) -> int:
        return capi.serial_emd_plan_get_tile(self.handle)

    @tile.setter
    def tile(self, value: int):
        capi.serial_emd_plan_set_tile(self.handle, value)

    @property
    def pass_ctas(self) -> int:
        return capi.serial_emd_plan_get_pass_ctas(self.handle)

    @pass_ctas.setter
    def pass_ctas(self, value: int):
        capi.serial_emd_plan_set_pass_ctas(self.handle, value)

    @property
    def pass_variant(self) -> int:
        return capi.serial_emd_plan_get_pass_variant(self.handle)

    @pass_variant.setter
    def pass_variant(self, value: int):
        capi.serial_emd_plan_set_pass_variant(self.handle, value)

    def autotune(self, xs, noise: torch.Tensor | None = None, outs=None, repeats: int = 3,
                 stream=None):
        """Picks the fastest pass-kernel shape for these inputs (one tensor or a list, as
        decompose_batch takes them). Returns the tuning result."""
        if isinstance(xs, torch.Tensor):
            xs = [xs]
        if outs is None:
            outs = [self.outputs(*x.shape, device=x.device) for x in xs]
        items = [(x, o[0], o[1]) for x, o in zip(xs, outs)]
        return capi.serial_emd_plan_autotune(self.handle, items, noise, repeats, stream)

    def set_options(self, use_graphs: bool = True, profile: bool = False):
        capi.serial_emd_plan_set_options(self.handle, use_graphs, profile)

    def stats(self) -> capi.semd_stats:
        return capi.serial_emd_plan_stats(self.handle)

    def counts(self, count: int = 1):
        return capi.serial_emd_plan_counts(self.handle, count, self.params.max_imfs)

    @property
    def noise_seed(self) -> int:
        return getattr(self, "_seed", 0)

    @noise_seed.setter
    def noise_seed(self, value: int):
        capi.serial_emd_plan_set_noise_seed(self.handle, value)
        self._seed = value

    def eemd_trial(self, trial: int, stream=None):
        """Realization `trial` of the last EEMD call: (imfs (K, rows, cols), residue,
        its IMF count, beta of the call)."""
        imfs, res = self.outputs(self.params.rows, self.params.cols)
        n, beta = capi.serial_emd_eemd_trial(self.handle, trial, imfs, res, stream)
        return imfs, res, n, beta

    def launch_times(self, kind: int = 0):
        """Per-launch device times (ms) of the last profiled call (kind 0: passes, 1:
        interface solves)."""
        return capi.serial_emd_plan_launch_times(self.handle, kind)

    def extrema(self, h: torch.Tensor, stream=None):
        L = h.numel()
        tmax = torch.empty(L // 2 + 1, dtype=torch.int32, device=h.device)
        tmin = torch.empty(L // 2 + 1, dtype=torch.int32, device=h.device)
        a, b = capi.serial_emd_extrema(self.handle, h, tmax, tmin, stream)
        return tmax[:a], tmin[:b]

    def sift(self, h: torch.Tensor, stream=None):
        out = torch.empty_like(h)
        num, den = capi.serial_emd_sift(self.handle, h, out, stream)
        return out, num, den


def decompose(x: torch.Tensor, noise: torch.Tensor | None = None, **kw):
    """One-shot Serial-EMD of a 2D CUDA tensor (rows, cols). Returns (imfs, residue, n)."""
    prec = capi.FP64 if x.dtype == torch.float64 else capi.FP32_MIXED
    kw.setdefault("precision", prec)
    p = make_params(x.shape[0], x.shape[1], **kw)
    plan = Plan(p)
    try:
        return plan.decompose(x.contiguous(), noise)
    finally:
        plan.close()


class Server:
    """Continuous-batching server (serial_emd_server_*): requests of different shapes are
    admitted as slots and the memory budget allow, and sifted together."""

    def __init__(self, params: capi.semd_params, mem_budget: int, max_inflight: int):
        self.params = params
        self.handle = capi.serial_emd_server_create(params, mem_budget, max_inflight)
        self.dtype = _DTYPE[params.precision]

    def outputs(self, rows: int, cols: int, device="cuda"):
        imfs = torch.empty((self.params.max_imfs, rows, cols), dtype=self.dtype, device=device)
        res = torch.empty((rows, cols), dtype=torch.float64, device=device)
        return imfs, res

    def submit(self, x: torch.Tensor, imfs=None, residue=None, order: int = capi.ORDER_ROWS):
        """Queues x (rows, cols); returns (ticket, imfs, residue). The tensors must stay
        alive until poll() returns the ticket's result."""
        assert x.is_cuda and x.dtype == self.dtype and x.is_contiguous()
        if imfs is None:
            imfs, residue = self.outputs(*x.shape, device=x.device)
        t = capi.serial_emd_submit(self.handle, x, imfs, residue, order)
        return t, imfs, residue

    def wait(self, ticket: int, timeout_ms: float):
        """The request's result, or None if it did not finish within timeout_ms."""
        return capi.serial_emd_wait(self.handle, ticket, timeout_ms)

    def poll(self, ticket: int):
        return capi.serial_emd_poll(self.handle, ticket)

    def close(self):
        if self.handle:
            capi.serial_emd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
