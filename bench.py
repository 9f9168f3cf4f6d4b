"""Throughput benchmark of the hybrid LB + FD nematohydrodynamics step on GB300.

Workload: the 256x256x64 multi-tube channel (8 skyrmion tubes of radius 20,
q0 = 2 pi/64, g_x = 1e-5, K = 0.005), FP32 arithmetic with shifted FP32
populations, dt_FD = 16.  One bench step is one hybrid block: dt_FD fused LB
collide-and-stream launches, one FD predictor-corrector + stress + force update
and one FP64 diagnostics reduction (mass, Frank energy, tube centroids).
Metric: MLUPS = sites x LB steps / s (FD, force and diagnostics time included).

The populations (2 x 319 MB) are larger than L2, so no L2 flush is needed
between steps.  Per-kernel times come from CUDA events on the launching stream
inside the timed region.  With --gpus N (torchrun) every rank runs its own
replica of the workload (independent channels, no data-path collective):
weak scaling, value = sum over ranks.

--impl reference times the FP64 CPU oracle on the host's CPU cores on the same
workload (one LB step per bench step plus the FD update every dt_FD steps).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_SITE_LB = {"f32": 164, "f64": 328, "f16s": 88, "bf16s": 88}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16s", "bf16s"])
    ap.add_argument("--dt-fd", type=int, default=16)
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--small", action="store_true", help="64x64x32 case (profiling only)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-channel sweep")
    ap.add_argument("--batch-blocks", type=int, default=20, help="dt_FD blocks timed in the batched sweep")
    ap.add_argument("--lb-sweep", action="store_true",
                    help="also time every LB launch shape the workload admits (lb_sweep_us in the JSON line)")
    ap.add_argument("--no-diag-fold", action="store_true",
                    help="diagnostics read the populations, u and rho themselves (nh_set_diag_fold 0)")
    return ap.parse_args()


def workload(args):
    from paper_2503_06610_gb300 import inputs
    if args.small:
        params, n0, centres = inputs.multi_tube_channel(dt_fd=args.dt_fd, nx=64, ny=64, nz=32, tubes=2, radius=10)
        name = f"multi-tube channel 64x64x32, 2 tubes R=10, dt_FD={args.dt_fd}"
    else:
        params, n0, centres = inputs.multi_tube_channel(dt_fd=args.dt_fd)
        name = f"multi-tube channel 256x256x64, 8 tubes R=20, q0=2pi/64, gx=1e-5, dt_FD={args.dt_fd}"
    return params, n0, centres, name


def ncu_traffic():
    """DRAM read+write bytes per LB launch from the committed ncu summary, or
    None when csrc/lb.cu changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "lb_kernel_multitube_256x256x64_fp32.md")
    src = os.path.join(ROOT, "paper_2503_06610_gb300", "csrc", "lb.cu")
    try:
        vals = {}
        for line in open(path):
            line = line.strip()
            if line.startswith("traffic_bytes_per_launch:") or line.startswith("lb_source_sha256_16:"):
                k, v = line.split(":", 1)
                vals[k] = v.strip()
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != vals.get("lb_source_sha256_16"):
            return None
        return int(vals["traffic_bytes_per_launch"])
    except Exception:
        return None


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons, one line every 50 ms, started
    before the warm-up so that it samples from the first timed step on.  The
    lines carry nvidia-smi's timestamp; stop() reports the samples taken between
    region_start() and region_end() (host wall clock), or, when none fell inside
    (a region shorter than the interval), the sample nearest to the region."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index, interval_ms=50):
        self.gpu = self.smi_id(gpu_index)
        self.interval_ms = interval_ms
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)

    def region_start(self):
        self.t0 = time.time()

    def region_end(self):
        self.t1 = time.time()

    @staticmethod
    def smi_id(local):
        """nvidia-smi's -i argument for CUDA device `local` of this process: its
        UUID, else its CUDA_VISIBLE_DEVICES entry, else the index -- the first
        that nvidia-smi accepts (the index alone when nvidia-smi is missing)."""
        cands = []
        try:
            import torch
            u = str(torch.cuda.get_device_properties(local).uuid)
            cands.append(u if u.startswith("GPU-") else "GPU-" + u)
        except Exception:
            pass
        ids = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
        if local < len(ids):
            cands.append(ids[local])
        cands.append(str(local))
        for c in cands:
            try:
                r = subprocess.run(["nvidia-smi", "-i", c, "--query-gpu=index", "--format=csv,noheader"],
                                   capture_output=True, timeout=20)
            except Exception:
                break  # no nvidia-smi
            if r.returncode == 0 and r.stdout.strip():
                return c
        return str(local)

    @staticmethod
    def _stamp(text):
        """nvidia-smi's local-time stamp 'YYYY/MM/DD HH:MM:SS.mmm' in seconds since the epoch."""
        try:
            whole, _, frac = text.partition(".")
            return time.mktime(time.strptime(whole, "%Y/%m/%d %H:%M:%S")) + (float("0." + frac) if frac else 0.0)
        except ValueError:
            return None

    def parse(self, lines):
        samples = []  # (time or None, sm MHz, max sm MHz, reasons)
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm, smax = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            reasons = {nm for nm, v in zip(self.REASONS, parts[6:10]) if v.lower() in ("active", "1")}
            samples.append((self._stamp(parts[0]), sm, smax, reasons))
        inside, use = [], samples
        stamped = [x for x in samples if x[0] is not None]
        if self.t0 is not None and self.t1 is not None and stamped:
            inside = [x for x in stamped if self.t0 <= x[0] <= self.t1]
            # a region shorter than the interval: the sample nearest to it
            use = inside or [min(stamped, key=lambda x: max(self.t0 - x[0], x[0] - self.t1))]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median([x[1] for x in use])), "sm_max_mhz": float(max(x[2] for x in use)),
                "reasons": sorted(set().union(*[x[3] for x in use])), "samples": len(use),
                "samples_in_region": len(inside)}

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return self.parse(lines)


# ------------------------------------------------------------------ CPU oracle baseline

def cpu_oracle_mlups(params, n0, sample_lb_steps):
    """Time the FP64 oracle (as it stands) for `sample_lb_steps` LB steps with the
    FD update every dt_FD steps; returns (MLUPS, threads, seconds)."""
    import oracle
    oracle.build()
    p = oracle.OracleParams.from_dict(params)
    sim = oracle.OracleSim(p, n0)
    t0 = time.perf_counter()
    sim.step(sample_lb_steps)
    dt = time.perf_counter() - t0
    return p.N * sample_lb_steps / dt / 1e6, oracle.num_threads(), dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    params, n0, centres, name = workload(args)
    import oracle
    oracle.build()
    p = oracle.OracleParams.from_dict(params)
    sim = oracle.OracleSim(p, n0)
    for _ in range(args.warmup):
        sim.step(1)
    t0 = time.perf_counter()
    sim.step(args.steps)
    el = time.perf_counter() - t0
    mlups = p.N * args.steps / el / 1e6
    out = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "precision": "fp64 CPU oracle", "step": "1 LB step (+ FD every dt_FD)"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{args.steps} LB steps of the full workload after {args.warmup} warm-up steps"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ multi-rank reduction

def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time: all ranks time the same replica workload, so
    the job's throughput is set by the maximum."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(world, sites_per_rank, lb_steps, ms_max):
    """Whole-job MLUPS: every rank updates sites_per_rank sites lb_steps times
    (weak scaling, independent replicas) within ms_max milliseconds."""
    return world * sites_per_rank * lb_steps / (ms_max * 1e-3) / 1e6


# ------------------------------------------------------------------ GPU arm

def batched_sweep(nh, torch, store, blocks):
    """64 channels (L in {32,48,64,96}, Lz in {16,24,32}, one tube each, FP32
    shifted, dt_FD = 16): one batched launch per pass vs a per-channel loop."""
    from paper_2503_06610_gb300 import inputs
    sweep = inputs.batched_sweep(64, seed=0, dt_fd=16)
    chans = []
    for params, n0, centre in sweep:
        ch = nh.Channel(dict(params, precision="fp32", storage=store, shifted=True))
        ch.set_fields(n0)
        chans.append(ch)
    sites = sum(c.N for c in chans)
    dt = sweep[0][0]["dt_fd"]
    variant = nh.batch_autotune(chans)
    nh.batch_step(chans, dt)
    for c in chans:
        c.step(dt)
    torch.cuda.synchronize()
    st = chans[0].stream
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    launches0 = chans[0].launch_count()
    e[0].record(st)
    nh.batch_step(chans, dt * blocks)
    e[1].record(st)
    torch.cuda.synchronize()
    batch_launches = chans[0].launch_count() - launches0
    e[2].record(st)
    for _ in range(blocks):
        for c in chans:
            c.step(dt)
    e[3].record(st)
    torch.cuda.synchronize()
    t_b = e[0].elapsed_time(e[1]) * 1e-3
    t_s = e[2].elapsed_time(e[3]) * 1e-3
    for c in chans:
        c.close()
    return {"channels": len(chans), "sites": sites, "lb_steps": dt * blocks, "lb_variant": variant,
            "batched_mlups": sites * dt * blocks / t_b / 1e6, "sequential_mlups": sites * dt * blocks / t_s / 1e6,
            "speedup": t_s / t_b, "batched_launches": batch_launches}


def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2503_06610_gb300 import nh
    nh.load_library()

    params, n0, centres, name = workload(args)
    dt = params["dt_fd"]
    store = args.storage

    # CPU baseline first (rank 0, N=1 only), before heavy GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        mlups, threads, secs = cpu_oracle_mlups(params, n0, dt)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": f"{dt} LB steps + 1 FD update of the full workload in FP64 ({secs:.1f} s)"}

    ch = nh.Channel(dict(params, precision="fp32", storage=store, shifted=True))
    if args.no_diag_fold:
        ch.set_diag_fold(False)
    ch.set_fields(n0)
    ch.set_tubes(centres)
    stream = ch.stream

    def block():
        ch.step(dt)
        ch.diagnostics_enqueue()

    clocks = ClockSampler(local)
    clocks.start()  # sampling from before the autotuner and the warm-up on
    lb_variant = ch.autotune()
    for _ in range(args.warmup):
        block()
    ch.diagnostics_read()
    torch.cuda.synchronize()

    ch.set_timing(2)  # events around the LB launches only (the roofline kernel)
    ch.timing()  # reset counters
    launches0 = ch.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks.region_start()
    e0.record(stream)
    for _ in range(args.steps):
        block()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.region_end()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = ch.launch_count() - launches0
    kt = ch.timing()
    diag = ch.diagnostics_read()
    ch.set_timing(False)
    ch.timing()

    # same loop without per-kernel events (whole dt_FD blocks replayed from CUDA graphs)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    g0.record(stream)
    for _ in range(args.steps):
        block()
    g1.record(stream)
    torch.cuda.synchronize()
    ch.diagnostics_read()
    value_graphs = ch.N * dt * args.steps / (g0.elapsed_time(g1) * 1e-3) / 1e6


    ms_max = max_over_ranks(ms, dist, device="cuda")
    N = ch.N
    value = aggregate_mlups(world, N, dt * args.steps, ms_max)

    lb_n, lb_ms = kt["lb"]
    lb_avg_s = lb_ms / max(lb_n, 1) * 1e-3
    bytes_per_launch = BYTES_PER_SITE_LB[store] * N
    achieved = bytes_per_launch / lb_avg_s / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        peak, peak_src = 6800.0, "fallback"
    traffic = ncu_traffic() if (store == "f32" and not args.small and dt == 16) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "lb_kernel (fused collide+stream)", "peak_source": peak_src,
                "lb_variant": lb_variant,
                "bytes_per_launch": bytes_per_launch, "avg_launch_us": lb_avg_s * 1e6,
                "share_of_kernel_time": None}

    # FP64 comparison on the same workload: throughput, and the error of this
    # store against FP64 after a fixed 2000 LB steps from the same start (the
    # trajectories of this strongly driven channel separate over longer runs)
    compare = None
    if not args.no_compare and rank == 0:
        steps_done = 2000
        c32 = nh.Channel(dict(params, precision="fp32", storage=store, shifted=True))
        c32.set_lb_variant(lb_variant)
        c32.set_fields(n0)
        c32.step(steps_done)
        n32, u32, _ = c32.get_fields()
        c32.close()
        c64 = nh.Channel(dict(params, precision="fp64", storage="f64", shifted=True))
        c64.set_fields(n0)
        pre = steps_done - 4 * dt
        c64.step(pre)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(c64.stream)
        c64.step(4 * dt)
        f1.record(c64.stream)
        torch.cuda.synchronize()
        fp64_mlups = N * 4 * dt / (f0.elapsed_time(f1) * 1e-3) / 1e6
        n64, u64, _ = c64.get_fields()
        rel = lambda a, b: float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
        eps = float(np.sum(np.linalg.norm(u32 - u64, axis=0)) / np.sum(np.linalg.norm(u64, axis=0)))
        compare = {"fp64_mlups": fp64_mlups, "speedup_fp32s_vs_fp64": value / world / fp64_mlups,
                   "lb_steps_compared": steps_done, "rel_l2_u_vs_fp64": rel(u32, u64),
                   "rel_l2_n_vs_fp64": rel(n32, n64), "eps_u_vs_fp64": eps}
        c64.close()

    # per-class breakdown (events around every kernel class), untimed, after the
    # FP32 fields above were compared with the FP64 run
    breakdown_steps = min(args.steps, 20)
    ch.set_timing(1)
    ch.timing()
    for _ in range(breakdown_steps):
        block()
    kt_all = ch.timing()
    ch.diagnostics_read()
    ch.set_timing(0)
    ch.timing()
    total_kernel_ms = sum(v[1] for v in kt_all.values())
    roofline["share_of_kernel_time"] = kt_all["lb"][1] / total_kernel_ms if total_kernel_ms else None

    # end to end through the C ABI with host buffers: per call the initial
    # director goes up from pinned host memory, then `blocks` bench steps run,
    # each ending with a host read of its diagnostics (nh_diagnostics), and the
    # final n, u, rho come back to pinned host memory; every copy sits inside
    # the timed region, and the bytes are reported per bench step (a call's
    # field copies spread over its bench steps) and per call
    e2e = None
    if rank == 0:
        blocks, reps = 10, 3
        pin_n = torch.from_numpy(np.ascontiguousarray(n0)).pin_memory()
        out_n = torch.empty((3, N), dtype=torch.float64).pin_memory()
        out_u = torch.empty((3, N), dtype=torch.float64).pin_memory()
        out_r = torch.empty((N,), dtype=torch.float64).pin_memory()
        host = lambda t: t.numpy()
        ce = nh.Channel(dict(params, precision="fp32", storage=store, shifted=True))
        ce.set_lb_variant(lb_variant)  # the launch shape the autotuner chose above
        ce.set_tubes(centres)

        def call():
            nh.nh_set_fields(ce.ctx, host(pin_n))
            for _ in range(blocks):
                ce.step(dt)
                ce.diagnostics()
            nh.nh_get_fields(ce.ctx, host(out_n), host(out_u), host(out_r))

        call()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            call()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        diag_bytes = 8 * (6 + 5 * len(centres))
        h2d_call, d2h_call = 3 * N * 8, 7 * N * 8 + blocks * diag_bytes
        e2e = {"value": N * dt * blocks * reps / el / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": int(h2d_call // blocks), "d2h_bytes_per_step": int(d2h_call // blocks),
               "h2d_bytes_per_call": int(h2d_call), "d2h_bytes_per_call": int(d2h_call),
               "bench_steps_per_call": blocks, "lb_steps_per_call": dt * blocks,
               "api": "nh_set_fields(host) + bench steps of nh_step + nh_diagnostics(host) + nh_get_fields(host)"}
        ce.close()

    # every LB launch shape on the same workload (nh_set_lb_variant), CUDA events around the LB launches
    lb_sweep = None
    if rank == 0 and args.lb_sweep:
        lb_sweep = {}
        cs = nh.Channel(dict(params, precision="fp32", storage=store, shifted=True))
        cs.set_fields(n0)
        cs.step(4 * dt)
        for v in range(7):
            try:
                cs.set_lb_variant(v)
            except nh.NHError:
                continue  # this shape does not fit the workload
            cs.step(2 * dt)
            torch.cuda.synchronize()
            cs.set_timing(2)
            cs.timing()
            cs.step(20 * dt)
            n_l, ms_l = cs.timing()["lb"]
            cs.set_timing(0)
            cs.timing()
            lb_sweep[str(v)] = 1000.0 * ms_l / max(n_l, 1)
        cs.close()

    # batched sweep: 64 independent channels of uneven size in one launch per pass
    batched = None
    if rank == 0 and not args.no_batch:
        batched = batched_sweep(nh, torch, store, args.batch_blocks)

    if rank == 0:
        out = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": name, "storage": f"{store} shifted populations", "sites": N,
                       "lb_steps_per_step": dt, "l2": "inputs larger than L2 (populations 2x%.0f MB)"
                       % (19 * N * (2 if store != 'f32' else 4) / 1e6), "parallelism": f"replicas x{world}",
                       "diagnostics": "every bench step, " + ("reading f, u, rho" if args.no_diag_fold or store not in
                                                              ("f32", "f64") else "sums of f, u, rho folded into the "
                                                              "LB launch that writes u, rho")},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": int(launches),
            "value_graphs_no_kernel_events": value_graphs,
            "kernel_ms": {k: {"launches": v[0], "ms": v[1]} for k, v in kt.items()},
            "kernel_ms_breakdown": {"steps": breakdown_steps,
                                    **{k: {"launches": v[0], "ms": v[1]} for k, v in kt_all.items()}},
            "fp64_compare": compare,
            "batched_sweep": batched,
            "lb_sweep_us": lb_sweep,
            "diagnostics": {"mass_minus_N": diag["mass"] - N, "energy": diag["energy"], "max_u": diag["max_u"],
                            "centroids": diag["centroids"].tolist()[:8], "nonfinite": diag["nonfinite"]},
        }
        print(json.dumps(out), flush=True)
    ch.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
