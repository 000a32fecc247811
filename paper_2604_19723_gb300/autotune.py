"""Autotuners: the batch executor's launch configuration, and the kernels' own tile shapes.

The batch executor (bp_batch_*) deals scenarios of uneven sizes over concurrent
streams and can replay each stream's launches from CUDA graphs.  How many streams pay
off depends on the mix of sizes (small scenarios want many streams to fill the GPU,
large ones contend for it), so the tuner measures: for each candidate (streams, graph)
it builds the batch on a sample of the scenarios, runs warm-up steps, times a few
steps with CUDA events on the batch's fork/join stream, and returns the fastest
candidate with the whole table.  The scenarios' results do not depend on the choice
(each scenario runs the same kernels in the same order).

The tile tuner (tune_tiles, tune_batch_tiles) picks, per filter or per shape class of a
batch, the kernels' tile shapes (bp_set_tiles): the PF likelihood's column bucket S~,
its blocks per SM and staged frequency chunk (the Nz tile), tensor-core or CUDA-core
kernel, and the message table's particle chunk.  Each candidate is timed on the same
predicted state with the library's own per-stage CUDA events (the PF-likelihood and
message-table stages), the median of a few updates.  Results depend on the tiles only
through FP32 rounding.
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


BUCKETS = (8, 16, 24, 32, 48, 64)


def basis_stride(S_max: int) -> int:
    """Column stride of a filter's basis buffers (the largest usable bucket)."""
    return 8 if S_max <= 8 else 16 if S_max <= 16 else 32 if S_max <= 32 else 64


def tensor_core_large(geom) -> bool:
    """The arrays whose tensor-core pass-1 rounds lie within one frequency (My Mz a
    multiple of 16, at least 32); their kernel forms the steering elements as (hi, lo)
    pairs in pass 2."""
    nm = geom.My * geom.Mz
    return nm >= 32 and nm % 16 == 0


def tensor_core_smem(geom, width: int) -> int:
    """Dynamic shared memory of the tensor-core PF likelihood (one 128-particle tile per
    block; width = basis columns incl. r0): the operand region of either pass, barriers,
    r0 per element, 1/lambda and y~0, the factors (frequency factors kept up to 16, and
    never for the large arrays), and for the large arrays the low parts of a_z and the
    (hi, lo) cis table."""
    large = tensor_core_large(geom)
    region = max(2 * 128 * 32 + 2 * (2 * width) * 32, 2 * 128 * 32 + 2 * 2 * 64 * 32)
    nfac = (geom.Nf if geom.Nf <= 16 and not large else 0) + geom.My + geom.Mz
    pairs = geom.Mz * 128 * 8 + 16 + 256 * 16 if large else 0
    return region * 4 + 32 + geom.Nf * geom.My * geom.Mz * 16 + 2 * width * 8 + nfac * 128 * 8 + pairs


def tensor_core_shape(geom, S_max: int) -> bool:
    """Whether the tensor-core PF likelihood applies to this shape: Mz even and either
    64 basis columns with 2 My Mz in {8, 16, 32} (a pass-1 round is whole frequencies) or
    64 or 32 columns with My Mz a multiple of 16, at least 32 (a round is part of one
    frequency); its shared memory within 227 KB.  It runs at the basis stride's width."""
    width, nm = basis_stride(S_max), geom.My * geom.Mz
    if geom.Mz % 2:
        return False
    whole = width == 64 and 2 * nm in (8, 16, 32)
    part = width in (32, 64) and tensor_core_large(geom)
    return (whole or part) and tensor_core_smem(geom, width) <= 227 * 1024


def kappa_candidates(S: int, S_max: int, geom) -> List[Dict[str, int]]:
    """Tile candidates of the PF likelihood: the two smallest buckets that hold S (within
    the basis stride), two blocks per SM where the bucket allows it (<= 32), half the
    staged frequency chunk, and the tensor-core kernel on or off where the shape allows."""
    top = basis_stride(S_max)
    bks = [b for b in BUCKETS if S <= b <= top][:2]
    out = []
    for b in bks:
        if b == top and tensor_core_shape(geom, S_max):
            out.append(dict(kappa_sc=b, kappa_tc=1, kappa_blocks=0, kappa_fch=0))
        if b == 64 and tensor_core_shape(geom, S_max):
            out.append(dict(kappa_sc=64, kappa_tc=-1, kappa_blocks=0, kappa_fch=0))
            continue
        for mb in ((1, 2) if b in (24, 32) else (0,)):
            out.append(dict(kappa_sc=b, kappa_tc=-1, kappa_blocks=mb, kappa_fch=0))
        if geom.Nf >= 4:
            out.append(dict(kappa_sc=b, kappa_tc=-1, kappa_blocks=0, kappa_fch=(geom.Nf + 3) // 4))
    return out


def table_candidates() -> List[Dict[str, int]]:
    return [dict(table_chunk=c) for c in (32, 64, 128)]


def _time_stage(f, gp, z, stage: str, reps: int) -> float:
    import torch
    ms = []
    for r in range(reps + 1):
        f.set_predicted(gp["n"], gp["S"], gp["x"], gp["phi"], gp["eta"], gp["w_beta"], gp["w_alpha"], gp["w_xi"],
                        gp["zeta"], S_legacy=gp["S_legacy"])
        f.update(z)
        torch.cuda.synchronize()
        if r > 0:                       # the first run of a configuration warms it up
            ms.append(f.profile()[stage])
    return float(np.median(ms))


def tune_tiles(f, z, reps: int = 3, kappa: Sequence[Dict[str, int]] = None,
               table: Sequence[Dict[str, int]] = None) -> Dict:
    """Measure tile candidates on filter f (its current belief state, observation z: a
    torch CUDA complex64 (J, Nz) tensor) and leave the fastest set on f.  The filter's
    state is restored to its prediction before every timed update, so that every
    candidate sees the same work; afterwards f holds the last timed update's result.
    Returns {"best": tiles, "kappa_ms": {...}, "table_ms": {...}}."""
    f.set_profiling(True)
    f.predict()
    gp = f.get_predicted()
    S = int(gp["S"])
    kappa = list(kappa) if kappa is not None else kappa_candidates(S, f.S_max, f.geom)
    table = list(table) if table is not None else table_candidates()
    best = {k: 0 for k in ("kappa_sc", "kappa_blocks", "kappa_fch", "kappa_tc", "table_chunk", "table_split")}
    k_ms, t_ms = {}, {}
    for cand in kappa:
        f.set_tiles(**{**best, **cand})
        k_ms[_key(cand)] = _time_stage(f, gp, z, "kappa", reps)
    if k_ms:
        best.update(_parse(min(k_ms, key=k_ms.get)))
    for cand in table:
        f.set_tiles(**{**best, **cand})
        t_ms[_key(cand)] = _time_stage(f, gp, z, "table", reps)
    if t_ms:
        best.update(_parse(min(t_ms, key=t_ms.get)))
    f.set_tiles(**best)
    return {"best": best, "kappa_ms": k_ms, "table_ms": t_ms}


def _key(d: Dict[str, int]) -> str:
    return ",".join(f"{k}={v}" for k, v in sorted(d.items()))


def _parse(key: str) -> Dict[str, int]:
    return {k: int(v) for k, v in (kv.split("=") for kv in key.split(","))}


def shape_class(geom, P: int, S: int, S_max: int) -> Tuple:
    """Scenarios that share their tile choice: the PF-likelihood bucket of S, the basis
    stride, the tensor-core eligibility, the array size and the frequency count in
    ranges of 16."""
    b = next(x for x in BUCKETS if x >= S)
    return (b, basis_stride(S_max), tensor_core_shape(geom, S_max), geom.My * geom.Mz, (geom.Nf + 15) // 16)


def tune_batch_tiles(batch, scenarios: Sequence[tuple], z_row, reps: int = 2, max_classes: int = None) -> Dict:
    """Tile tuning of a Batch: per shape class, the scenario of median P is rebuilt as a
    single filter from the batch member's current state and tuned (tune_tiles); the
    choice goes to every scenario of the class (Batch.set_tiles).  scenarios: the
    (geom, params, P, S_max, S0, seed) tuples of the batch; z_row: one step's
    concatenated observations (torch CUDA float32).  Returns the classes and choices."""
    import torch
    from . import bp
    classes: Dict[Tuple, List[int]] = {}
    for i, (g, prm, P, S_max, S0, seed) in enumerate(scenarios):
        st = batch.member(i).get_state()
        classes.setdefault(shape_class(g, P, st.S, S_max), []).append(i)
    keys = sorted(classes, key=lambda k: -sum(scenarios[i][2] for i in classes[k]))
    if max_classes is not None:
        keys = keys[:max_classes]
    out = {}
    for k in keys:
        members = classes[k]
        rep = sorted(members, key=lambda i: scenarios[i][2])[len(members) // 2]
        g, prm, P, S_max, S0, seed = scenarios[rep]
        f = bp.Filter(g, prm, P=P, S_max=S_max, seed=seed)
        try:
            f.set_state(batch.member(rep).get_state())
            o = batch.z_offset(rep)
            nz = 2 * g.J * g.Nz
            zc = torch.view_as_complex(z_row[o:o + nz].reshape(g.J, g.Nz, 2).contiguous())
            res = tune_tiles(f, zc, reps=reps)
        finally:
            f.close()
        for i in members:
            batch.set_tiles(i, **res["best"])
        out[str(k)] = {"scenarios": len(members), "members": members, "tuned_on": rep, **res}
    return out
