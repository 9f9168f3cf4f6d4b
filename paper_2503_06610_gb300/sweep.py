"""Precision x dt_FD sweep of the hybrid step (the experiment of Secs. III.A-III.B).

For one workload (by default the 96x96x32 single skyrmion tube in Poiseuille
flow, g_x in {1e-6, 1e-5}; also the Table I regime of Sec. III.A and the
256x256x64 multi-tube channel) every combination of arithmetic / population store
(FP64, FP32 plain, FP32 shifted, FP16 and BF16 shifted) and dt_FD is run on the
GPU through the C ABI; each run reports

* MLUPS of the timed run (LB + FD + force, CUDA events),
* the errors of u and n against the reference run - FP64, shifted, dt_FD = 1
  as in the paper, or the smallest dt_FD that is stable for the workload
  (``--ref-dt``) - as relative L2 and as the paper's epsilon (Sec. III.A) and
  its per-component form (Sec. III.B),
* the tube centroids and their largest distance from the reference centroids.

Usage:  python -m paper_2503_06610_gb300.sweep [--steps 5000] [--gx 1e-5] [--out sweep.json]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs
from . import nh

SETTINGS = [
    ("fp64", "f64", True),
    ("fp32", "f32", False),
    ("fp32", "f32", True),
    ("fp32", "f16s", True),
    ("fp32", "bf16s", True),
]


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def eps(u, uref):
    return float(np.sum(np.linalg.norm(u - uref, axis=0)) / np.sum(np.linalg.norm(uref, axis=0)))


def eps_component(u, uref, a):
    return float(np.sum(np.abs(u[a] - uref[a])) / np.sum(np.abs(uref[a])))


def run_one(params, n0, centres, precision, storage, shifted, steps):
    import torch
    ch = nh.Channel(dict(params, precision=precision, storage=storage, shifted=shifted))
    ch.set_fields(n0)
    ch.set_tubes(centres)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ch.stream)
    ch.step(steps)
    e1.record(ch.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n, u, rho = ch.get_fields()
    d = ch.diagnostics(allow_unstable=True)
    ch.close()
    return {"mlups": ch.N * steps / (ms * 1e-3) / 1e6, "n": n, "u": u, "centroid": d["centroids"].tolist(),
            "max_u": float(np.nanmax(np.abs(u))) if np.isfinite(u).any() else float("nan"),
            "nonfinite": d["nonfinite"], "energy": d["energy"]}


def sweep(steps=5000, gx=1e-5, dts=(1, 2, 4, 8, 16), settings=SETTINGS, nx=96, ny=96, nz=32, radius=12.0,
          regime="skyrmion", ref_dt=1, split=0.3, paper_order=None):
    if regime == "table1":
        base, n0 = inputs.table1_regime(nx=nx, ny=ny, nz=nz, dt_fd=1, split=split,
                                        paper_order=True if paper_order is None else paper_order)
        radius = 7.0
        centres = [(nx / 2, ny / 2)]
    elif regime == "multitube":
        base, n0, centres = inputs.multi_tube_channel(dt_fd=1, nx=nx, ny=ny, nz=nz)
        radius = 20.0
        if paper_order is not None:
            base = dict(base, paper_order=paper_order)
    else:
        base, n0 = inputs.skyrmion_channel(gx=gx, dt_fd=1, nx=nx, ny=ny, nz=nz, radius=radius)
        if paper_order is not None:
            base = dict(base, paper_order=paper_order)
        centres = [(nx / 2, ny / 2)]
    ref = run_one(dict(base, dt_fd=ref_dt), n0, centres, "fp64", "f64", True, steps)
    rows = []
    for dt in dts:
        for precision, storage, shifted in settings:
            if (precision, storage, shifted, dt) == ("fp64", "f64", True, ref_dt):
                r = ref
            else:
                r = run_one(dict(base, dt_fd=dt), n0, centres, precision, storage, shifted, steps)
            dx = (np.array(r["centroid"]) - np.array(ref["centroid"]) + 0.5 * np.array([nx, ny])) % np.array(
                [nx, ny]) - 0.5 * np.array([nx, ny])
            shift = np.hypot(dx[:, 0], dx[:, 1])
            rows.append({
                "dt_fd": dt, "precision": precision, "storage": storage, "shifted": shifted,
                "mlups": r["mlups"], "rel_l2_u": rel_l2(r["u"], ref["u"]), "rel_l2_n": rel_l2(r["n"], ref["n"]),
                "eps_u": eps(r["u"], ref["u"]), "eps_ux": eps_component(r["u"], ref["u"], 0),
                "eps_uy": eps_component(r["u"], ref["u"], 1), "eps_uz": eps_component(r["u"], ref["u"], 2),
                "centroid": r["centroid"], "centroid_shift": float(np.max(shift)), "nonfinite": r["nonfinite"],
                "max_u": r["max_u"], "max_u_ref": ref["max_u"],
            })
    name = {"table1": "Table I regime", "multitube": "multi-tube channel"}.get(regime, "skyrmion channel") + \
        f" {nx}x{ny}x{nz}, R={radius}, q0={base['q0']:.4f}, gx={base['g'][0]}, K={base['K']:.3g}" + \
        (", loop order of Sec. II.D" if base.get("paper_order") else ", fused loop order")
    return {"workload": name,
            "steps": steps, "reference": f"fp64 shifted dt_FD={ref_dt}", "reference_centroid": ref["centroid"],
            "tau": base["tau"], "alpha4p": base["alpha4p"], "reference_nonfinite": ref["nonfinite"],
            "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--gx", type=float, nargs="+", default=[1e-6, 1e-5])
    ap.add_argument("--dts", type=int, nargs="+", default=[1, 2, 4, 8, 16])
    ap.add_argument("--out", default=None)
    ap.add_argument("--regime", default="skyrmion", choices=["skyrmion", "table1", "multitube"])
    ap.add_argument("--settings", nargs="+", default=None,
                    help="precision/storage/s|p triples, e.g. fp32/f16s/s (default: all five)")
    ap.add_argument("--size", type=int, nargs=3, default=None, help="nx ny nz")
    ap.add_argument("--ref-dt", type=int, default=1, help="dt_FD of the FP64 reference run")
    ap.add_argument("--split", type=float, default=0.3, help="table1: share of alpha4 carried by the FD force")
    ap.add_argument("--order", choices=["default", "paper", "fused"], default="default",
                    help="loop order: paper = Sec. II.D as printed (the table1 default), fused = the collision keeps "
                         "the force of the previous interval (the skyrmion default)")
    args = ap.parse_args()
    results = []
    size = args.size or {"table1": (64, 64, 16), "multitube": (256, 256, 64)}.get(args.regime, (96, 96, 32))
    gxs = {"table1": [2e-9], "multitube": [1e-5]}.get(args.regime, args.gx)
    settings = SETTINGS
    if args.settings:
        settings = [(a, b, c == "s") for a, b, c in (t.split("/") for t in args.settings)]
    for gx in gxs:
        t0 = time.time()
        res = sweep(steps=args.steps, gx=gx, dts=tuple(args.dts), nx=size[0], ny=size[1], nz=size[2], settings=settings,
                    regime=args.regime, split=args.split, ref_dt=args.ref_dt,
                    paper_order={"default": None, "paper": True, "fused": False}[args.order])
        res["wall_s"] = time.time() - t0
        results.append(res)
        for r in res["rows"]:
            print(f"gx={gx:g} dt={r['dt_fd']:3d} {r['precision']}/{r['storage']}/{'s' if r['shifted'] else 'p'}: "
                  f"{r['mlups']:9.1f} MLUPS  eps_u {r['eps_u']:.3e}  relL2 n {r['rel_l2_n']:.3e}  "
                  f"centroid shift {r['centroid_shift']:.3e}  max|u| {r['max_u']:.3e}  nonfinite {r['nonfinite']}")
    if args.out:
        with open(args.out, "w") as f:
            json.dump(results, f, indent=1)


if __name__ == "__main__":
    main()
