"""Per-block run records of a channel as JSON lines.

Each record covers one block of LB steps (by default one FD interval,
dt_FD steps): the step count, the FP64 diagnostics of the state at the end
of the block (mass, lattice Frank energy, max |u|, |n| extrema, non-finite
sites, tube centroids) and the block's throughput from CUDA events on the
channel's stream.

Usage:
    from paper_2503_06610_gb300 import inputs, nh, runlog
    ch = nh.Channel(params); ch.set_fields(n0); ch.set_tubes(centres)
    records = runlog.run(ch, n_blocks=100, path="run.jsonl")
"""
from __future__ import annotations

import json


def run(channel, n_blocks: int, path: str | None = None, block: int | None = None) -> list:
    """Advance `channel` by n_blocks blocks of `block` LB steps (default dt_FD)
    and return (and, with `path`, append as JSON lines) one record per block."""
    import torch
    block = int(block or channel.params["dt_fd"])
    records = []
    out = open(path, "a") if path else None
    try:
        for _ in range(n_blocks):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(channel.stream)
            channel.step(block)
            e1.record(channel.stream)
            d = channel.diagnostics(allow_unstable=True)
            ms = e0.elapsed_time(e1)
            rec = {
                "step": int(d["step"]), "lb_steps": block,
                "mlups": channel.N * block / (ms * 1e-3) / 1e6 if ms > 0 else None,
                "mass": d["mass"], "energy": d["energy"], "max_u": d["max_u"],
                "min_norm": d["min_norm"], "max_norm": d["max_norm"], "nonfinite": int(d["nonfinite"]),
                "centroids": [list(map(float, c)) for c in d["centroids"]],
            }
            records.append(rec)
            if out:
                out.write(json.dumps(rec) + "\n")
                out.flush()
    finally:
        if out:
            out.close()
    return records
