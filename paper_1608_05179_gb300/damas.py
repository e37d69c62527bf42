"""Python binding of libdamas.so: the C-ABI entry points under the same names.

Each function marshals torch tensors (device memory) into the C call and
checks the status; every computation runs in the library's CUDA kernels.
PyTorch provides device memory and streams only.  There is no CPU path: the
functions raise when the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import (BF16, EPS_ABS, EPS_KEEP_FRAC, EPS_REL_MAX, F32, FORM_E, FORM_P, INIT_STATE, INIT_X,  # noqa: F401
                   INIT_ZERO, PRED_HAAR, PRED_LINEAR)


class DamasError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_lib.ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor required")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor required")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A library context on one CUDA device (damas_create / damas_destroy)."""

    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = _lib.load()
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.damas_create(ctypes.byref(h), device)
        if rc != 0:
            raise DamasError(rc, "damas_create failed")
        self.handle = h

    def check(self, rc: int):
        if rc != 0:
            raise DamasError(rc, self.lib.damas_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.damas_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Geometry:
    """Array and scan grid (§2): microphone positions on the device plus grid parameters."""
    mic_xyz: torch.Tensor  # (M, 3) float64 on the device
    nx: int
    ny: int
    x0: float
    y0: float
    dx: float
    dy: float
    z: float
    c: float = 343.0
    formulation: int = FORM_E
    diag_removal: int = 0      # 1: the CSM diagonal is removed (§2)

    @property
    def M(self):
        return int(self.mic_xyz.shape[0])

    @property
    def S(self):
        return self.nx * self.ny

    def cstruct(self) -> _lib.damas_geom:
        return _lib.damas_geom(self.M, self.mic_xyz.data_ptr(), self.nx, self.ny, self.x0, self.y0, self.dx, self.dy,
                               self.z, self.c, self.formulation, int(self.diag_removal))

    @staticmethod
    def from_scene(mics: np.ndarray, grid, c: float, formulation: int = FORM_E, device="cuda",
                   diag_removal: int = 0) -> "Geometry":
        m = torch.as_tensor(np.ascontiguousarray(mics, dtype=np.float64), device=device)
        return Geometry(m, grid.nx, grid.ny, grid.x0, grid.y0, grid.dx, grid.dy, grid.z, c, formulation,
                        int(diag_removal))


def damas_set_option(ctx: Context, option: int, value: int):
    """Context option: _lib.OPT_BUILD_TIMEOUT_MS (bound on the build kernels'
    device waits), _lib.OPT_TEST_HOLD_BUILD (test hook of those waits) or
    _lib.OPT_HBM_BUDGET_BYTES (cap on the context's device memory; 0 = none)."""
    ctx.check(ctx.lib.damas_set_option(ctx.handle, int(option), int(value)))


def damas_check(ctx: Context, stream=None):
    """Synchronise the stream; raise DamasError(DAMAS_ETIMEDOUT) when a build
    kernel of the context gave up a bounded wait since the last check."""
    ctx.check(ctx.lib.damas_check(ctx.handle, _stream(stream)))


def damas_lda(S: int) -> int:
    return _lib.load().damas_lda(int(S))


def damas_state_floats(S: int) -> int:
    """Length of the solver state of an S-unknown system (System.state)."""
    return _lib.load().damas_state_floats(int(S))


def damas_build_psf(ctx: Context, geom: Geometry, freq: float, idx: torch.Tensor | None = None, S_sub: int | None = None,
                    a_dtype: int = F32, A: torch.Tensor | None = None, gnorm2: torch.Tensor | None = None,
                    stream=None):
    """PSF matrix A (S_sub x lda) of the selected points; returns (A, gnorm2)."""
    S_sub = geom.S if idx is None and S_sub is None else (S_sub if S_sub is not None else int(idx.numel()))
    lda = damas_lda(S_sub)
    dt = torch.float32 if a_dtype == F32 else torch.bfloat16
    if A is None:
        A = torch.empty((S_sub, lda), dtype=dt, device=geom.mic_xyz.device)
    if gnorm2 is None:
        gnorm2 = torch.empty(S_sub, dtype=torch.float32, device=geom.mic_xyz.device)
    g = geom.cstruct()
    ctx.check(ctx.lib.damas_build_psf(ctx.handle, ctypes.byref(g), float(freq), _ptr(idx), int(S_sub), int(a_dtype),
                                      _ptr(A), int(A.shape[1]), _ptr(gnorm2), _stream(stream)))
    return A, gnorm2


def damas_build_psf_f32_bf16(ctx: Context, geom: Geometry, freq: float, idx: torch.Tensor | None = None,
                             S_sub: int | None = None, A: torch.Tensor | None = None,
                             A_bf16: torch.Tensor | None = None, gnorm2: torch.Tensor | None = None, stream=None):
    """The PSF matrix in FP32 and in BF16 from one build; returns (A, A_bf16, gnorm2)."""
    S_sub = geom.S if idx is None and S_sub is None else (S_sub if S_sub is not None else int(idx.numel()))
    lda = damas_lda(S_sub)
    dev = geom.mic_xyz.device
    if A is None:
        A = torch.empty((S_sub, lda), dtype=torch.float32, device=dev)
    if A_bf16 is None:
        A_bf16 = torch.empty((S_sub, lda), dtype=torch.bfloat16, device=dev)
    if gnorm2 is None:
        gnorm2 = torch.empty(S_sub, dtype=torch.float32, device=dev)
    g = geom.cstruct()
    ctx.check(ctx.lib.damas_build_psf_f32_bf16(ctx.handle, ctypes.byref(g), float(freq), _ptr(idx), int(S_sub),
                                               _ptr(A), _ptr(A_bf16), int(A.shape[1]), _ptr(gnorm2),
                                               _stream(stream)))
    return A, A_bf16, gnorm2


def damas_build_psf_dr(ctx: Context, geom: Geometry, freq: float, idx: torch.Tensor | None = None,
                       S_sub: int | None = None, A: torch.Tensor | None = None, gnorm2: torch.Tensor | None = None,
                       dscale: torch.Tensor | None = None, stream=None):
    """PSF without the m = m' microphone pairs (diagonal removal, §2), rescaled to a
    unit diagonal; returns (A', gnorm2, dscale = sqrt of the unscaled diagonal)."""
    S_sub = geom.S if idx is None and S_sub is None else (S_sub if S_sub is not None else int(idx.numel()))
    lda = damas_lda(S_sub)
    dev = geom.mic_xyz.device
    if A is None:
        A = torch.empty((S_sub, lda), dtype=torch.float32, device=dev)
    if gnorm2 is None:
        gnorm2 = torch.empty(S_sub, dtype=torch.float32, device=dev)
    if dscale is None:
        dscale = torch.empty(S_sub, dtype=torch.float32, device=dev)
    g = geom.cstruct()
    ctx.check(ctx.lib.damas_build_psf_dr(ctx.handle, ctypes.byref(g), float(freq), _ptr(idx), int(S_sub), _ptr(A),
                                         int(A.shape[1]), _ptr(gnorm2), _ptr(dscale), _stream(stream)))
    return A, gnorm2, dscale


def damas_divide(ctx: Context, v: torch.Tensor, div: torch.Tensor, n: int | None = None, stream=None):
    """v[:n] /= div[:n] in place (FP32 device tensors)."""
    n = int(v.numel()) if n is None else int(n)
    ctx.check(ctx.lib.damas_divide(ctx.handle, _ptr(v), _ptr(div), n, _stream(stream)))
    return v


def damas_csm(ctx: Context, p: torch.Tensor, K: int, hop: int, bins: torch.Tensor, C: torch.Tensor | None = None,
              stream=None):
    """CSM (F, M, M, 2) of the DFT bins `bins` (int32 device tensor) from the time
    series p (M, T) float32 on the device: Hann-windowed blocks of K samples every
    hop samples, averaged (Welch)."""
    M, T = int(p.shape[0]), int(p.shape[1])
    F = int(bins.numel())
    if C is None:
        C = torch.empty((F, M, M, 2), dtype=torch.float32, device=p.device)
    ctx.check(ctx.lib.damas_csm(ctx.handle, _ptr(p), M, T, int(K), int(hop), _ptr(bins), F, _ptr(C), _stream(stream)))
    return C


def das_map(ctx: Context, geom: Geometry, freq: float, C: torch.Tensor, b: torch.Tensor | None = None, stream=None):
    """DAS map of Eq. (2) on the full grid; C is (M, M, 2) float32 (re, im)."""
    if b is None:
        b = torch.empty(geom.S, dtype=torch.float32, device=C.device)
    g = geom.cstruct()
    ctx.check(ctx.lib.das_map(ctx.handle, ctypes.byref(g), float(freq), _ptr(C), _ptr(b), _stream(stream)))
    return b


def wavelet_compress_grid(ctx: Context, b: torch.Tensor, nx: int, ny: int, levels: int, predictor: int = PRED_HAAR,
                          eps_mode: int = EPS_KEEP_FRAC, eps: float = 0.1, idx: torch.Tensor | None = None,
                          S_sub: torch.Tensor | None = None, detail: torch.Tensor | None = None,
                          eps_abs: torch.Tensor | None = None, stream=None):
    """Algorithm 1.  Returns (idx capacity tensor, S_sub device tensor, detail, eps_abs)."""
    dev = b.device
    idx = torch.empty(nx * ny, dtype=torch.int32, device=dev) if idx is None else idx
    S_sub = torch.empty(1, dtype=torch.int32, device=dev) if S_sub is None else S_sub
    cfg = _lib.damas_wavelet_cfg(int(levels), int(predictor), int(eps_mode), float(eps))
    ctx.check(ctx.lib.wavelet_compress_grid(ctx.handle, _ptr(b), int(nx), int(ny), ctypes.byref(cfg), _ptr(idx),
                                            _ptr(S_sub), _ptr(detail), _ptr(eps_abs), _stream(stream)))
    return idx, S_sub, detail, eps_abs


def wavelet_compress_grid_noalloc(ctx: Context, b: torch.Tensor, nx: int, ny: int, levels: int,
                                  predictor: int = PRED_HAAR, eps_mode: int = EPS_KEEP_FRAC, eps: float = 0.1,
                                  idx: torch.Tensor | None = None, S_sub: torch.Tensor | None = None,
                                  detail: torch.Tensor | None = None, eps_abs: torch.Tensor | None = None,
                                  stream=None):
    """Algorithm 1 through the allocation-free entry point: same results as
    wavelet_compress_grid, with the library's own fixed device work array instead
    of context scratch (for callers that cannot allocate device memory when they
    run, e.g. real-time threads or plug-ins limited to memory their host gave
    them).  The output tensors passed in are used as given; pass them all to keep
    the call free of allocations on the Python side too."""
    dev = b.device
    idx = torch.empty(nx * ny, dtype=torch.int32, device=dev) if idx is None else idx
    S_sub = torch.empty(1, dtype=torch.int32, device=dev) if S_sub is None else S_sub
    cfg = _lib.damas_wavelet_cfg(int(levels), int(predictor), int(eps_mode), float(eps))
    ctx.check(ctx.lib.wavelet_compress_grid_noalloc(ctx.handle, _ptr(b), int(nx), int(ny), ctypes.byref(cfg),
                                                    _ptr(idx), _ptr(S_sub), _ptr(detail), _ptr(eps_abs),
                                                    _stream(stream)))
    return idx, S_sub, detail, eps_abs


def damas_pad_grid(ctx: Context, idx: torch.Tensor, S_sub: torch.Tensor, nx: int, ny: int, radius: int,
                   out_idx: torch.Tensor | None = None, out_S: torch.Tensor | None = None, stream=None):
    """Neighbour padding of a compressed grid (every point within Chebyshev
    distance radius of a kept point).  Returns (out_idx capacity tensor, out_S
    device tensor)."""
    dev = idx.device
    out_idx = torch.empty(nx * ny, dtype=torch.int32, device=dev) if out_idx is None else out_idx
    out_S = torch.empty(1, dtype=torch.int32, device=dev) if out_S is None else out_S
    ctx.check(ctx.lib.damas_pad_grid(ctx.handle, int(nx), int(ny), _ptr(idx), _ptr(S_sub), int(radius), _ptr(out_idx),
                                     _ptr(out_S), _stream(stream)))
    return out_idx, out_S


def damas_gather(ctx: Context, src: torch.Tensor, idx: torch.Tensor, n: int, dst: torch.Tensor | None = None,
                 stream=None):
    dst = torch.empty(n, dtype=torch.float32, device=src.device) if dst is None else dst
    ctx.check(ctx.lib.damas_gather(ctx.handle, _ptr(src), _ptr(idx), int(n), _ptr(dst), _stream(stream)))
    return dst


def damas_scatter_power(ctx: Context, x_sub: torch.Tensor, idx: torch.Tensor | None, gnorm2: torch.Tensor | None,
                        n: int, S: int, x_full: torch.Tensor | None = None, total: torch.Tensor | None = None,
                        stream=None):
    dev = x_sub.device
    x_full = torch.empty(S, dtype=torch.float32, device=dev) if x_full is None else x_full
    total = torch.empty(1, dtype=torch.float64, device=dev) if total is None else total
    ctx.check(ctx.lib.damas_scatter_power(ctx.handle, _ptr(x_sub), _ptr(idx), _ptr(gnorm2), int(n), _ptr(x_full),
                                          int(S), _ptr(total), _stream(stream)))
    return x_full, total


@dataclass
class System:
    """One A x = b system for damas_solve (device tensors)."""
    A: torch.Tensor
    b: torch.Tensor
    x: torch.Tensor
    iters: int
    S: int | None = None
    state: torch.Tensor | None = None
    init: int = INIT_ZERO
    At: torch.Tensor | None = None  # transpose of A; None when A is symmetric
    ctas: int = 0                   # team size; 0 = automatic

    def cstruct(self) -> _lib.damas_system:
        S = self.S if self.S is not None else int(self.b.numel())
        dt = F32 if self.A.dtype == torch.float32 else BF16
        return _lib.damas_system(self.A.data_ptr(), self.At.data_ptr() if self.At is not None else None, dt,
                                 int(self.A.shape[1]), S, self.b.data_ptr(), self.x.data_ptr(),
                                 self.state.data_ptr() if self.state is not None else None, int(self.init),
                                 int(self.iters), int(self.ctas))


PLACE_AUTO, PLACE_RESIDENT, PLACE_STREAM = 0, 1, 2


def damas_solve(ctx: Context, systems, ctas_per_system: int = 0, timeout_ms: int = 0,
                status: torch.Tensor | None = None, a_placement: int = PLACE_AUTO, withhold_block: int = 0,
                stats: torch.Tensor | None = None, stream=None):
    """DAMAS Gauss-Seidel sweeps (Eq. (13)-(14)) on a batch of systems in one persistent launch:
    one CTA per system (small systems, when every system of the call qualifies) or a team
    of CTAs per system; both forms give bit-identical x and state.  stats (optional int64
    device tensor of 3) is added to: blocks solved, rows that entered a chain, nonzero dx."""
    if isinstance(systems, System):
        systems = [systems]
    arr = (_lib.damas_system * len(systems))(*[s.cstruct() for s in systems])
    if stats is not None and (stats.dtype != torch.int64 or stats.numel() < 3):
        raise ValueError("stats must be an int64 tensor of 3")
    cfg = _lib.damas_solve_cfg(int(ctas_per_system), int(timeout_ms),
                               status.data_ptr() if status is not None else None, int(a_placement),
                               int(withhold_block), stats.data_ptr() if stats is not None else None)
    ctx.check(ctx.lib.damas_solve(ctx.handle, arr, len(systems), ctypes.byref(cfg), _stream(stream)))
    return systems


def damas_solve_plan(ctx: Context, S: int, a_dtype: int = F32, ctas: int = 0, a_placement: int = PLACE_AUTO,
                     lda: int | None = None):
    """The plan damas_solve would use for one system alone: (CTAs, rows per CTA, resident).
    One CTA for S >= 97 is the single-CTA form (no hand-overs between CTAs)."""
    n, r, res = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ctx.check(ctx.lib.damas_solve_plan(ctx.handle, int(S), int(damas_lda(S) if lda is None else lda), int(a_dtype),
                                       int(ctas), int(a_placement), ctypes.byref(n), ctypes.byref(r),
                                       ctypes.byref(res)))
    return n.value, r.value, bool(res.value)


def damas_handover_probe(ctx: Context, rounds: int = 100, max_pairs: int = 1 << 30, timeout_us: int = 0,
                         stream=None) -> list[float]:
    """One-way CTA-to-CTA hand-over latency in ns, one value per CTA paired with CTA 0."""
    cap = max(1, min(int(max_pairs), 4096))
    buf = (ctypes.c_double * cap)()
    n = ctypes.c_int()
    ctx.check(ctx.lib.damas_handover_probe(ctx.handle, int(rounds), cap, int(timeout_us), buf, ctypes.byref(n),
                                           _stream(stream)))
    return [buf[i] for i in range(n.value)]


def damas_chain_probe(ctx: Context, rounds: int = 100000, stream=None):
    """Row-chain latency on this device: (ns per candidate update, ns per 512-thread barrier step)."""
    out = (ctypes.c_double * 2)()
    ctx.check(ctx.lib.damas_chain_probe(ctx.handle, int(rounds), out, _stream(stream)))
    return out[0], out[1]


def solve_mixed(ctx: Context, A_bf16: torch.Tensor, A_f32: torch.Tensor, b: torch.Tensor, x: torch.Tensor,
                iters_bulk: int, iters_refine: int, At_bf16: torch.Tensor | None = None,
                At_f32: torch.Tensor | None = None, ctas: int = 0, ctas_per_system: int = 0, timeout_ms: int = 0,
                status: torch.Tensor | None = None, a_placement: int = PLACE_AUTO, stream=None):
    """Mixed-precision schedule in one C call (damas_solve_mixed): iters_bulk sweeps
    with A stored in BF16 from x = 0, then iters_refine sweeps with the FP32 A from
    the exact FP32 residual of the current x."""
    if A_bf16.dtype != torch.bfloat16 or A_f32.dtype != torch.float32 or A_bf16.shape != A_f32.shape:
        raise ValueError("A_bf16 (bfloat16) and A_f32 (float32) of one shape are required")
    S = int(b.numel())
    m = _lib.damas_mixed_system(A_bf16.data_ptr(), At_bf16.data_ptr() if At_bf16 is not None else None,
                                A_f32.data_ptr(), At_f32.data_ptr() if At_f32 is not None else None,
                                int(A_f32.shape[1]), S, b.data_ptr(), x.data_ptr(), int(iters_bulk),
                                int(iters_refine), int(ctas))
    cfg = _lib.damas_solve_cfg(int(ctas_per_system), int(timeout_ms),
                               status.data_ptr() if status is not None else None, int(a_placement), 0, None)
    ctx.check(ctx.lib.damas_solve_mixed(ctx.handle, ctypes.byref(m), 1, ctypes.byref(cfg), _stream(stream)))
    return x


# ----------------------------------------------------------------------------- one frequency bin
def solve_bin(ctx: Context, geom: Geometry, freq: float, C: torch.Tensor, iters: int, compressed: bool = True,
              levels: int = 2, predictor: int = PRED_HAAR, eps_mode: int = EPS_KEEP_FRAC, eps: float = 0.1,
              a_dtype: int = F32, pad_radius: int = 0, stream=None):
    """The method for one bin (§5): DAS map, wavelet-compressed grid (Algorithm 1),
    optionally padded with the neighbours within pad_radius of every kept point,
    PSF matrix of the kept points, Gauss-Seidel from x = 0, power map on the
    full grid.  One host synchronisation reads the compressed size."""
    b = das_map(ctx, geom, freq, C, stream=stream)
    if compressed:
        idx, S_sub_t, _, _ = wavelet_compress_grid(ctx, b, geom.nx, geom.ny, levels, predictor, eps_mode, eps,
                                                   stream=stream)
        if pad_radius:
            idx, S_sub_t = damas_pad_grid(ctx, idx, S_sub_t, geom.nx, geom.ny, pad_radius, out_idx=idx,
                                          stream=stream)
        S_sub = int(S_sub_t.item())
        idx = idx[:S_sub]
        b_sub = damas_gather(ctx, b, idx, S_sub, stream=stream)
    else:
        idx, S_sub, b_sub = None, geom.S, b
    if geom.diag_removal:
        # unit-diagonal form of the system without the CSM diagonal: b' = b / sqrt(d), x = x' / sqrt(d)
        if a_dtype != F32:
            raise ValueError("diagonal removal builds A in FP32")
        A, g2, dsc = damas_build_psf_dr(ctx, geom, freq, idx, S_sub, stream=stream)
        if not compressed:
            b_sub = b_sub.clone()
        damas_divide(ctx, b_sub, dsc, S_sub, stream=stream)
    else:
        A, g2 = damas_build_psf(ctx, geom, freq, idx, S_sub, a_dtype, stream=stream)
    x = torch.empty(S_sub, dtype=torch.float32, device=b.device)
    damas_solve(ctx, System(A, b_sub, x, iters), stream=stream)
    if geom.diag_removal:
        damas_divide(ctx, x, dsc, S_sub, stream=stream)
    x_full, total = damas_scatter_power(ctx, x, idx, g2 if geom.formulation == FORM_E else None, S_sub, geom.S,
                                        stream=stream)
    return {"b": b, "idx": idx, "S_sub": S_sub, "A": A, "gnorm2": g2, "b_sub": b_sub, "x_sub": x, "x": x_full,
            "total_power": total}


def csm_tensor(C: np.ndarray, device="cuda") -> torch.Tensor:
    """M x M complex CSM as the (M, M, 2) float32 device tensor das_map takes."""
    out = np.empty(C.shape + (2,), np.float32)
    out[..., 0] = np.real(C)
    out[..., 1] = np.imag(C)
    return torch.as_tensor(out, device=device)
