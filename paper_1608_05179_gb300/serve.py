"""Binding of the library's serving loop (damas_serve_*): continuous batching of
independent requests, each one array, one grid and several frequency bins.
Argument marshalling only; the loop itself runs in libdamas.so."""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

import numpy as np

from . import _lib
from .damas import Context, DamasError, EPS_KEEP_FRAC, FORM_E, PRED_LINEAR


@dataclass
class Request:
    mics: np.ndarray          # (M, 3)
    grid: object              # nx, ny, x0, y0, dx, dy, z
    freqs: np.ndarray         # (F,)
    C: np.ndarray             # (F, M, M) complex
    iters: int
    levels: int = 3           # 0 = full grid
    predictor: int = PRED_LINEAR
    eps_mode: int = EPS_KEEP_FRAC
    eps: float = 0.1
    c: float = 343.0


@dataclass
class Result:
    x: np.ndarray             # (F, S) power maps
    total_power: np.ndarray   # (F,)
    S_sub: np.ndarray         # (F,)
    t_submit: float
    t_admit: float
    t_done: float
    t_solve: float = 0.0      # stage-2 admission (matrices and solve)
    hbm_bytes: int = 0        # device memory charged against the budget
    sm_units: int = 0         # half-SM units charged to its solve

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class Server:
    """damas_serve_start/submit/poll/release/stop on a context."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int = 0, max_inflight: int = 8, sm_slots: int = 0,
                 rows_per_cta: int = 0):
        self.ctx = ctx
        cfg = _lib.damas_serve_cfg(int(hbm_budget_bytes), int(max_inflight), int(sm_slots), int(rows_per_cta))
        ctx.check(ctx.lib.damas_serve_start(ctx.handle, ctypes.byref(cfg)))
        self._keep = {}

    def submit(self, r: Request) -> int:
        mics = np.ascontiguousarray(r.mics, dtype=np.float64)
        freqs = np.ascontiguousarray(r.freqs, dtype=np.float64)
        C = np.empty(r.C.shape + (2,), np.float32)
        C[..., 0] = np.real(r.C)
        C[..., 1] = np.imag(r.C)
        g = r.grid
        w = _lib.damas_wavelet_cfg(int(r.levels), int(r.predictor), int(r.eps_mode), float(r.eps))
        req = _lib.damas_request(mics.shape[0], mics.ctypes.data, g.nx, g.ny, g.x0, g.y0, g.dx, g.dy, g.z, float(r.c),
                                 FORM_E, len(freqs), freqs.ctypes.data, C.ctypes.data, w, int(r.iters))
        t = ctypes.c_uint64()
        self.ctx.check(self.ctx.lib.damas_serve_submit(self.ctx.handle, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """None while in flight, else the Result (copied out; the ticket is then released)."""
        res = _lib.damas_result()
        self.ctx.check(self.ctx.lib.damas_serve_poll(self.ctx.handle, ctypes.c_uint64(ticket), ctypes.byref(res)))
        if res.status == _lib.DAMAS_EBUSY:
            return None
        if res.status != 0:
            raise DamasError(res.status, f"request {ticket} failed")
        F, S = res.n_bins, res.S
        out = Result(np.ctypeslib.as_array(res.x, shape=(F * S,)).reshape(F, S).copy(),
                     np.ctypeslib.as_array(res.total_power, shape=(F,)).copy(),
                     np.ctypeslib.as_array(res.S_sub, shape=(F,)).copy(), res.t_submit, res.t_admit, res.t_done,
                     res.t_solve, int(res.hbm_bytes), int(res.sm_units))
        self.ctx.check(self.ctx.lib.damas_serve_release(self.ctx.handle, ctypes.c_uint64(ticket)))
        return out

    def wait(self, ticket: int, timeout: float = 120.0) -> Result:
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"request {ticket}")
            time.sleep(2e-4)

    def stop(self):
        self.ctx.check(self.ctx.lib.damas_serve_stop(self.ctx.handle))
