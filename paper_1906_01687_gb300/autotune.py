"""Autotuner of the fused sampled-gradient launch shape.

For one handle, factor layout and sampling spec, times ``gcp_grad`` for a set
of candidate shapes -- lanes per draw x float4 chunks per lane (rows per
warp), threads per block, replica slabs per mode (the pre-reduction width of
the L2 accumulation), warp-level pre-reduction of same-address updates, the
fold (and Adam step) as the kernel's own tail work, the
draw layout (group walk, prefetch or staged walk) and optional
shared-memory accumulation -- with CUDA
events around back-to-back launches, and keeps the fastest through
``gcp_set_tuning``.  A shape changes only the summation order of the
gradient, never the draws.
"""
from __future__ import annotations

import statistics
from typing import Iterable, Optional

import torch

from . import gcp

COMPILED = [(1, 1), (1, 2), (1, 3), (1, 4), (2, 1), (2, 2), (4, 1), (4, 2), (8, 1), (8, 2), (16, 1), (32, 1), (32, 2)]


# modes of at most this many rows get the warp-level pre-reduction in the
# candidates that try it (short modes, where a warp step's draws share rows)
COMBINE_ROWS = 4096


def candidate_shapes(rank: int) -> list:
    """(lanes, chunks) pairs that cover ceil(rank / 4) chunks without more than
    doubling the lanes' work."""
    chunks = (rank + 3) // 4
    out = []
    for L, NC in COMPILED:
        cover = L * NC
        if cover >= chunks and (cover < 2 * chunks or cover <= 4):
            out.append((L, NC))
    return out


def candidates(rank: int) -> list:
    out = []
    for L, NC in candidate_shapes(rank):
        layouts = [dict(group_draws=0), dict(group_draws=0, warp_combine=COMBINE_ROWS)]
        if L > 1:
            layouts += [dict(group_draws=1), dict(group_draws=1, warp_combine=COMBINE_ROWS)]
        if NC == 1 and L in (2, 4):
            layouts.append(dict(prefetch=1))
        if NC == 1 and L <= 8:
            layouts.append(dict(prefetch=2))
        for layout in layouts:
            for block in (128, 256):
                for reps, target in ((0, 0), (-1, 0), (8, 128), (32, 16)):
                    out.append(dict(lanes=L, chunks=NC, block=block, max_replicas=reps, replica_target=target,
                                    **layout))
        out.append(dict(lanes=L, chunks=NC, block=256, max_replicas=0, smem_bytes=48 * 1024, smem_min_hits=10))
    return out


def with_grids(configs, n_draws: int) -> list:
    """Each candidate twice: with the automatic grid (one resident wave when
    the draws fill at least half of it) and with the grid that gives every
    warp exactly one batch of draws (no idle warps in a small launch)."""
    out = []
    for cfg in configs:
        out.append(dict(cfg))
        block = cfg.get("block", 0) or 256
        lanes = cfg.get("lanes", 0) or 1
        per_warp = 32 // lanes if cfg.get("group_draws") else 32
        warps = -(-int(n_draws) // per_warp)
        fit = max(1, -(-warps // (block // 32)))
        out.append(dict(cfg, grid_blocks=fit))
    return out


def side_stream(stream):
    """A stream other than `stream` (torch hands streams out round-robin from
    a small pool, so a new one can be `stream` itself)."""
    for _ in range(64):
        s = torch.cuda.Stream(device=stream.device)
        if s.cuda_stream != stream.cuda_stream:
            return s
    raise RuntimeError("no CUDA stream other than the working stream")


def time_graph(call, spec, launches, stream, cap=None) -> float:
    """Device time (s) per call of `launches` back-to-back calls captured in a
    CUDA graph: the calls overlap as they do in a captured epoch."""
    with torch.cuda.stream(stream):
        call(spec, stream)  # allocate any workspace outside the capture
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    cap = cap if cap is not None else side_stream(stream)
    with torch.cuda.graph(g, stream=cap):
        for i in range(launches):
            s = gcp.Sampling(spec.kind, spec.p, spec.q, spec.seed, (1 << 62) + i, spec.problem, spec.oversample)
            call(s, cap)
    with torch.cuda.stream(stream):
        g.replay()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            g.replay()
        b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) * 1e-3 / (3 * launches)


def time_grad(h, F, loss, spec, launches=20, stream=None, call=None, graph=False, cap=None) -> float:
    """Median device time (s) of one gcp_grad call (or of call(spec, stream))
    for the current tuning; with graph, the time per call of a captured
    sequence of calls."""
    stream = stream or torch.cuda.current_stream()
    if call is None:
        G = F.like()

        def call(s, st):
            gcp.gcp_grad(h, F, loss, G, S=s, stream=st)
    if graph:
        return time_graph(call, spec, launches, stream, cap)
    with torch.cuda.stream(stream):
        call(spec, stream)  # allocate any workspace outside the timing
        stream.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(launches)]
        torch.cuda._sleep(50_000_000)
        for i, (a, b) in enumerate(evs):
            s = gcp.Sampling(spec.kind, spec.p, spec.q, spec.seed, (1 << 62) + i, spec.problem, spec.oversample)
            a.record(stream)
            call(s, stream)
            b.record(stream)
    stream.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in evs) * 1e-3


def autotune(h, F, loss, spec, configs: Optional[Iterable[dict]] = None, launches=20, stream=None,
             log=None, call=None, graph=False) -> dict:
    """Times every candidate (gcp_grad, or call(spec, stream) when given, e.g.
    a whole GCP-Adam iteration; with graph, as a captured sequence of calls),
    sets the fastest on the handle, returns it with its time."""
    best, best_t = None, float("inf")
    results = []
    stream = stream or torch.cuda.current_stream()
    cap = side_stream(stream) if graph else None
    seen = set()
    for cfg in configs if configs is not None else candidates(F.rank):
        try:
            gcp.gcp_set_tuning(h, **cfg)
        except gcp.GcpError:
            continue
        # candidates that come out as the same launch (e.g. a warp-level
        # pre-reduction with no mode short enough for it) are timed once
        launch = gcp.gcp_get_launch(h, F, spec.count())
        key = (tuple(sorted((k, tuple(v) if isinstance(v, list) else v) for k, v in launch.items())),
               cfg.get("tail_work", 0), cfg.get("zero_pass", 0))
        if key in seen:
            continue
        seen.add(key)
        t = time_grad(h, F, loss, spec, launches, stream, call, graph, cap)
        results.append((t, cfg))
        if log:
            log(dict(seconds=t, **cfg))
        if t < best_t:
            best, best_t = cfg, t
    # the fastest shape once more with its fold (and Adam step) as the kernel's tail work
    if best is not None and not best.get("tail_work"):
        cfg = dict(best, tail_work=1)
        gcp.gcp_set_tuning(h, **cfg)
        t = time_grad(h, F, loss, spec, launches, stream, call, graph, cap)
        results.append((t, cfg))
        if log:
            log(dict(seconds=t, **cfg))
        if t < best_t:
            best, best_t = cfg, t
    gcp.gcp_set_tuning(h, **best)
    return dict(best=best, seconds=best_t, tried=len(results))
