"""Band processing (§6): every frequency bin of a band through the compressed-grid
path, with all bins' Gauss-Seidel iterations in one persistent launch.

Phase 1 (per bin, no host synchronisation): DAS map and compressed grid.  The
compressed sizes S_f of all bins are then read back once.  Phase 2: restriction
of b, PSF matrix of each bin's kept points, ONE damas_solve launch over all bins
(each bin a team of CTAs sized by the plan), and the power maps.  Phase 2 can be
captured once as a CUDA graph and replayed while the S_f stay the same.  Every
step runs in the library's kernels; this module only sequences the calls.
"""
from __future__ import annotations

import heapq
import math
import time
from dataclasses import dataclass, field

import torch

from . import damas as D


@dataclass
class BandGrids:
    """Phase-1 output: maps, kept indices and sizes of every bin."""
    b: torch.Tensor        # (F, S) float32
    idx: torch.Tensor      # (F, S) int32, first S_f entries valid
    S_f_dev: torch.Tensor  # (F,) int32
    S_f: list[int] = field(default_factory=list)


def compress_band(ctx: D.Context, geom: D.Geometry, freqs, C: torch.Tensor, levels: int, predictor: int,
                  eps_mode: int, eps: float, stream=None) -> BandGrids:
    """DAS map and compressed grid of every bin (C: (F, M, M, 2) float32 on the device)."""
    F, S = len(freqs), geom.S
    dev = C.device
    g = BandGrids(torch.empty((F, S), dtype=torch.float32, device=dev),
                  torch.empty((F, S), dtype=torch.int32, device=dev),
                  torch.empty(F, dtype=torch.int32, device=dev))
    for f, fr in enumerate(freqs):
        D.das_map(ctx, geom, float(fr), C[f], b=g.b[f], stream=stream)
        D.wavelet_compress_grid(ctx, g.b[f], geom.nx, geom.ny, levels, predictor, eps_mode, eps, idx=g.idx[f],
                                S_sub=g.S_f_dev[f:f + 1], stream=stream)
    return g


def team_sizes(S_f, rows_per_cta: int, capacity: int) -> list[int]:
    """CTAs per bin: about rows_per_cta rows each, scaled down to fit the device at once."""
    P = [max(1, math.ceil(s / rows_per_cta)) for s in S_f]
    while sum(P) > capacity:
        P = [max(1, p * capacity // sum(P)) for p in P]
        if sum(P) > capacity:
            P = [max(1, p - 1) for p in P]
    return P


def team_sizes_balanced(S_f, capacity: int, r0: float) -> list[int]:
    """CTAs per bin that even out the bins' solve times.  Step-time model: a
    step of a team with R rows per CTA costs about 1 + R / r0 (a fixed part -
    the 32-row solve, the barrier, the hand-over - plus the fold of the step's
    dx into the CTA's rows), and a bin of nb blocks takes nb steps per sweep.
    Every bin starts with one CTA; each further CTA goes to the bin with the
    longest estimated time, up to one CTA per 32-row block and `capacity` CTAs
    in all.  Small bins have short chains and keep few CTAs; the largest bins,
    whose chains set the length of the launch, get the rest."""
    F = len(S_f)
    nb = [max(1, -(-int(s) // 32)) for s in S_f]
    P = [1] * F

    def cost(f):
        return nb[f] * (1.0 + S_f[f] / P[f] / r0)

    heap = [(-cost(f), f) for f in range(F) if nb[f] > 1]
    heapq.heapify(heap)
    left = capacity - F
    while left > 0 and heap:
        _, f = heapq.heappop(heap)
        P[f] += 1
        left -= 1
        if P[f] < nb[f]:
            heapq.heappush(heap, (-cost(f), f))
    return P


class BandSolver:
    """Phase 2 for a fixed set of compressed sizes: buffers, plan and (optionally) a captured graph."""

    def __init__(self, ctx: D.Context, geom: D.Geometry, freqs, S_f, iters: int, a_dtype: int = D.F32,
                 rows_per_cta: int = 1024, capacity: int | None = None, balance_r0: float | None = None):
        self.ctx, self.geom, self.freqs, self.S_f, self.iters = ctx, geom, list(freqs), list(S_f), iters
        self.a_dtype = a_dtype
        dev = geom.mic_xyz.device
        dt = torch.float32 if a_dtype == D.F32 else torch.bfloat16
        cap = capacity or torch.cuda.get_device_properties(dev).multi_processor_count
        self.ctas = (team_sizes_balanced(self.S_f, cap, balance_r0) if balance_r0
                     else team_sizes(self.S_f, rows_per_cta, cap))
        self.A = [torch.empty((s, D.damas_lda(s)), dtype=dt, device=dev) for s in self.S_f]
        self.g2 = [torch.empty(s, dtype=torch.float32, device=dev) for s in self.S_f]
        self.b_sub = [torch.empty(s, dtype=torch.float32, device=dev) for s in self.S_f]
        self.x = [torch.empty(s, dtype=torch.float32, device=dev) for s in self.S_f]
        self.x_full = torch.empty((len(self.S_f), geom.S), dtype=torch.float32, device=dev)
        self.total = torch.empty(len(self.S_f), dtype=torch.float64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.graph = None

    def systems(self):
        return [D.System(self.A[f], self.b_sub[f], self.x[f], self.iters, ctas=self.ctas[f])
                for f in range(len(self.S_f))]

    def run(self, grids: BandGrids, stream=None):
        """Restriction, PSF matrices, one solve launch for all bins, power maps."""
        for f, fr in enumerate(self.freqs):
            n = self.S_f[f]
            idx = grids.idx[f, :n]
            D.damas_gather(self.ctx, grids.b[f], idx, n, dst=self.b_sub[f], stream=stream)
            D.damas_build_psf(self.ctx, self.geom, float(fr), idx, n, self.a_dtype, A=self.A[f], gnorm2=self.g2[f],
                              stream=stream)
        D.damas_solve(self.ctx, self.systems(), status=self.status, stream=stream)
        for f in range(len(self.S_f)):
            n = self.S_f[f]
            D.damas_scatter_power(self.ctx, self.x[f], grids.idx[f, :n], self.g2[f], n, self.geom.S,
                                  x_full=self.x_full[f], total=self.total[f:f + 1], stream=stream)

    def capture(self, grids: BandGrids):
        """Record phase 2 as a CUDA graph (run once eagerly first so every scratch buffer exists)."""
        self.run(grids)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run(grids, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def check(self):
        torch.cuda.synchronize()
        st = int(self.status.item())
        if st != 0:
            raise D.DamasError(st, "band solve status")


def plan_solver(ctx, geom, freqs, S_f, iters: int, a_dtype: int, plan) -> "BandSolver":
    """BandSolver for a team plan (policy, value, capacity): ("rows", rows per CTA,
    capacity) sizes teams in proportion to S_f; ("balance", r0, capacity) evens
    out the bins' solve times (team_sizes_balanced)."""
    policy, value, cap = plan
    if policy == "rows":
        return BandSolver(ctx, geom, freqs, S_f, iters, a_dtype, rows_per_cta=int(value), capacity=cap)
    if policy == "balance":
        return BandSolver(ctx, geom, freqs, S_f, iters, a_dtype, capacity=cap, balance_r0=float(value))
    raise ValueError(f"unknown team policy {policy!r}")


def autotune_rows(ctx, geom, freqs, grids: BandGrids, iters_probe: int = 20, a_dtype: int = D.F32,
                  candidates=(256, 512, 1024, 2048), cta_per_sm=(1, 2), balance=(256, 1024, 4096)):
    """Pick the team plan for this band by timing a short solve of each
    candidate: teams in proportion to S_f at each rows-per-CTA candidate, or
    balanced solve times at each r0 in `balance`, with the device asked to hold
    one or two CTAs per SM.  Returns (plan, {plan: seconds}), plan = (policy,
    value, capacity) as plan_solver takes it."""
    sms = torch.cuda.get_device_properties(geom.mic_xyz.device).multi_processor_count
    best, timings = None, {}
    plans = [(pol, v, per_sm * sms) for per_sm in cta_per_sm
             for pol, vals in (("rows", candidates), ("balance", balance)) for v in vals]
    for plan in plans:
        bs = plan_solver(ctx, geom, freqs, grids.S_f, iters_probe, a_dtype, plan)
        bs.run(grids)
        bs.check()
        systems = bs.systems()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            D.damas_solve(ctx, systems, status=bs.status)
            bs.check()
        except D.DamasError:
            continue  # this plan does not fit the device at once
        timings[plan] = time.perf_counter() - t0
        if best is None or timings[plan] < timings[best]:
            best = plan
    return best, timings


def solve_band(ctx, geom, freqs, C, iters, levels=3, predictor=D.PRED_LINEAR, eps_mode=D.EPS_REL_MAX, eps=1e-3,
               a_dtype=D.F32, rows_per_cta=1024):
    """One band end to end; returns (grids, solver) with maps in solver.x_full and powers in solver.total."""
    grids = compress_band(ctx, geom, freqs, C, levels, predictor, eps_mode, eps)
    grids.S_f = [int(v) for v in grids.S_f_dev.cpu().tolist()]
    bs = BandSolver(ctx, geom, freqs, grids.S_f, iters, a_dtype, rows_per_cta)
    bs.run(grids)
    bs.check()
    return grids, bs
