"""Autotuner of the batch executor's launch configuration.

The batch executor (bp_batch_*) deals scenarios of uneven sizes over concurrent
streams and can replay each stream's launches from CUDA graphs.  How many streams pay
off depends on the mix of sizes (small scenarios want many streams to fill the GPU,
large ones contend for it), so the tuner measures: for each candidate (streams, graph)
it builds the batch on a sample of the scenarios, runs warm-up steps, times a few
steps with CUDA events on the batch's fork/join stream, and returns the fastest
candidate with the whole table.  The scenarios' results do not depend on the choice
(each scenario runs the same kernels in the same order).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import bp

DEFAULT_CANDIDATES: Tuple[Tuple[int, bool], ...] = ((8, True), (16, True), (32, True), (64, True), (128, True),
                                                    (32, False))


def tune_batch(scenarios: Sequence[tuple], z, candidates: Sequence[Tuple[int, bool]] = DEFAULT_CANDIDATES,
               steps: int = 3, warmup: int = 2, sample: int = None, stream=None) -> Dict:
    """scenarios: the (geom, params, P, S_max, S0, seed) tuples of bp.Batch; z: a torch CUDA
    float32 tensor (steps x z_floats) of the full batch's observations (scenario order;
    a prefix of scenarios uses a prefix of each row); sample: tune on the first `sample`
    scenarios (all if None).  Returns {"best": (streams, graph), "ms": {...}, "sample": n}."""
    import torch
    sc = list(scenarios)[:sample] if sample else list(scenarios)
    st = stream or torch.cuda.Stream()
    table: List[Tuple[Tuple[int, bool], float]] = []
    for n_streams, graph in candidates:
        b = bp.Batch(sc, n_streams=n_streams, shared_workspace=True, use_graph=graph, stream=st)
        try:
            nz = b.z_floats()
            for i in range(warmup):
                with torch.cuda.stream(st):
                    b.step(z[i % z.shape[0], :nz])
            st.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            with torch.cuda.stream(st):
                ev[0].record(st)
                for i in range(steps):
                    b.step(z[(warmup + i) % z.shape[0], :nz])
                    ev[i + 1].record(st)
            st.synchronize()
            ms = float(np.mean([ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]))
        finally:
            b.close()
        table.append(((int(n_streams), bool(graph)), ms))
    best = min(table, key=lambda t: t[1])[0]
    return {"best": best, "ms": {f"{s} streams, graph {g}": ms for (s, g), ms in table}, "sample": len(sc)}
