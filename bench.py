#!/usr/bin/env python3
"""Benchmark of CG-SENSE on the cine workload (one JSON line on rank 0).

Workload (one "step"): a CG-SENSE reconstruction of a 256x256 cine series,
20 frames, 12 coils, acceleration 4 (64 of 256 phase-encode lines per frame,
16 of them centre lines, a fresh line pattern per frame), 30 CG iterations
per frame from x0 = 0: the adjoint E^H y, then 30 x (E^H E p, CG scalars,
fused x/r update), all in libsense.so.  Inputs are seeded synthetic
phantoms, coil maps and masks; k-space is E x plus complex Gaussian noise.

Metric: E^H E applications per second (one application = one normal-operator
product for one frame).  `value` times the steps with inputs resident in
HBM; `e2e` times the same call with the inputs copied from pinned host
memory and the image copied back inside the timed region.  L2 is flushed
(a 512 MiB write) before every timed step.

With --gpus N under torchrun, each rank runs an independent replica of the
workload on its own GPU (the problems do not exchange data; weak scaling);
the step time is the maximum over ranks.  ``--impl reference`` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

class Workload:
    """A CG-SENSE workload: n x n images, `frames` sharing `coils` maps,
    acceleration `accel` with `centre` fully sampled centre lines, `iters` CG
    iterations per frame; `make` draws its seeded inputs (synth)."""

    def __init__(self, name, n, frames, coils, accel, centre, iters, make, desc):
        self.name, self.n, self.frames, self.coils = name, n, frames, coils
        self.accel, self.centre, self.iters, self.make, self.desc = accel, centre, iters, make, desc
        self.lines = int(round(n / accel))


def _cine(frames):
    from paper_1807_11830_gb300 import synth
    return synth.cine_256(frames=frames)


def _slices(frames):
    from paper_1807_11830_gb300 import synth
    return synth.slices_320(frames=frames)


WORKLOADS = {
    "cine": Workload("cine", 256, 20, 12, 4, 16, 30, _cine,
                     "cine 256x256, 20 frames, 12 coils, R=4 (64 lines, 16 centre), 30 CG-SENSE iterations"),
    "slices320": Workload("slices320", 320, 16, 32, 3, 24, 50, _slices,
                          "slices 320x320, 16 slices, 32 coils, R=3 (107 lines, 24 centre), "
                          "50 CG-SENSE iterations"),
}
CINE = WORKLOADS["cine"]
FRAMES, COILS, N, ACCEL, CENTRE, ITERS = CINE.frames, CINE.coils, CINE.n, CINE.accel, CINE.centre, CINE.iters
WORKLOAD = CINE.desc
STORAGE_NAMES = {"c64": "complex64", "bf16": "bfloat16 pairs (S and y); FP32 transforms, coil sums and CG "
                                              "vectors; FP64 CG inner products"}
METRIC = "E^H·E applications/s"
UNIT = "applications/s"
FLUSH_BYTES = 512 << 20
# ncu DRAM traffic of k_cg_persistent on this workload, bytes per CG iteration,
# keyed by (kernel variant, CG mode), one launch of 30 iterations each: the
# lane-major 8·4·8 variant (53.0 MB read + 120.0 MB written) and the
# lane-major 16·16 variant (49.5 MB read + 93.6 MB written)
CINE_TRAFFIC_PER_ITER = {(1, "persistent"): (52.997888e6 + 119.976192e6) / 30,
                         (2, "persistent"): (49.472512e6 + 93.554176e6) / 30}
# ncu DRAM traffic (read + write) of one k_cg_persistent launch of a mix size class, bytes per CG
# iteration (empty until captured)
MIX_TRAFFIC_PER_ITER = {}
PAPER_WORKLOAD = ("paper reconstruction: 16 frames x 160x160, 8 coils, fully sampled; "
                  "2D inverse FFT + root-sum-of-squares (Sec. IV-B)")
PAPER_METRIC, PAPER_UNIT = "reconstructions/s", "reconstructions/s"
# OpenCLIPER's own time for this workload on a GTX 970 (Table II: clFFT 1.361 ms + RSS 0.252 ms): context
PAPER_GTX970_MS = 1.361 + 0.252
# ncu DRAM traffic per launch of the paper workload's kernels (read + write, mean over the launches of one
# launch list of `bench.py --workload paper --steps 20 --warmup 3 --no-cpu-baseline`: k_rows_bulk<160,+1>
# 26.23 MB read; k_adj_col_tma<160,c64,rss> 26.25 MB read; their writes leave L2 after the launch)
PAPER_TRAFFIC = {"rows_inv": 26.234243e6, "adj_col": 26.246184e6}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-iters", type=int, default=20)
    ap.add_argument("--workload", default="cine", choices=("cine", "slices320", "mix", "serve", "paper"),
                    help="cine: the headline line; slices320: the 320x320, 32-coil, 50-iteration precision-study "
                         "shape; mix: 512-instance uneven batch vs the plain loop; "
                         "serve: Poisson request streams through the serving queue vs serial plain solves; "
                         "paper: the paper's timed FFT + RSS reconstruction (and the Eq. 1 combine)")
    ap.add_argument("--storage", default="c64", choices=("c64", "bf16"),
                    help="storage of S and y for the cine and slices320 workloads")
    ap.add_argument("--accuracy-iters", type=int, default=0,
                    help="CG iterations of the accuracy sample against the FP64 oracle (0: the workload's own "
                         "count for cine, 4 for slices320)")
    ap.add_argument("--mix-count", type=int, default=512)
    ap.add_argument("--serve-rates", default="50,200,800")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-pool", type=int, default=256,
                    help="serving: distinct request instances drawn from the uneven-batch distribution")
    ap.add_argument("--serve-log-dir", default="",
                    help="serving: keep each rate's per-request queue log (JSON lines) in this directory")
    ap.add_argument("--serve-queue-only", action="store_true",
                    help="serving: skip the serial baseline (for tuning the queue)")
    ap.add_argument("--serve-admit-waves", default="0",
                    help="serving: the queue's admit_waves (0 = its default, negative = no saturation limit); "
                         "a comma list runs the queue once per value")
    ap.add_argument("--serve-live-work", type=int, default=0,
                    help="serving: the queue's max_live_work (frames x coils x ny x nx live at once; 0 = default)")
    ap.add_argument("--cg-mode", default="auto", choices=("auto", "graph", "persistent"),
                    help="CG iteration scheme; 'auto' times both briefly and keeps the faster")
    ap.add_argument("--lam", type=float, default=0.0,
                    help="Tikhonov weight of the cine workload's CG, (E^H E + lam I) x = E^H y")
    ap.add_argument("--lam-t", type=float, default=0.0,
                    help="temporal weight of the cine workload: one CG over the 20 frames, "
                         "(E^H E + lam I + lam_t L) x = E^H y with L the cyclic second difference")
    ap.add_argument("--centred", action="store_true",
                    help="centred k-space convention (DC at n/2) for the cine and paper workloads")
    ap.add_argument("--normal-variant", default="auto",
                    help="normal-operator kernel variant, or 'auto' for the library's autotuner")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank timings (a list of floats) over all
    ranks of the default process group; identity for one rank."""
    import torch

    if world <= 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def instance_cost(spec):
    """Relative cost of one instance of the uneven batch: frames x coils x
    transform work of an n x n image (n^2 log2 n)."""
    n = spec["n"]
    return spec["frames"] * spec["coils"] * n * n * np.log2(n)


def shard_instances(specs, world, rank):
    """Longest-processing-time-first assignment of instances to ranks: the
    instances never exchange data, so each rank solves its own share."""
    order = sorted(range(len(specs)), key=lambda i: -instance_cost(specs[i]))
    load = [0.0] * world
    owner = [0] * len(specs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += instance_cost(specs[i])
    return [i for i in range(len(specs)) if owner[i] == rank]


def base_config(world, centred=False, wl=CINE, storage="c64"):
    return {
        "workload": wl.desc + (", centred k-space" if centred else "") + (", BF16 storage" if storage == "bf16" else ""),
        "ny": wl.n, "nx": wl.n, "frames": wl.frames,
        "coils": wl.coils, "lines": wl.lines, "centre_lines": wl.centre, "cg_iterations": wl.iters,
        "storage": STORAGE_NAMES[storage],
        "kspace": "centred (DC at n/2)" if centred else "uncentred (DC at 0)",
        "l2": "flushed before every timed step (512 MiB device write)",
        "parallelism": "replicas x%d (independent problems, no collective)" % world,
    }


# ---------------------------------------------------------------------------
# CPU side: the FP64 oracle on a bounded sample (reference arm / cpu_baseline)
# ---------------------------------------------------------------------------
_ORACLE_INPUTS = {}


def oracle_inputs(centred=False, wl=CINE):
    """k-space of the whole workload made once by the oracle's E (untimed)."""
    key = (wl.name, centred)
    if key not in _ORACLE_INPUTS:
        import oracle
        from paper_1807_11830_gb300 import synth

        p = wl.make(wl.frames)
        lines = synth.centred_lines(p.lines, wl.n) if centred else p.lines
        S = p.S.astype(np.complex64).astype(np.complex128)
        y = oracle.forward(p.x_true.astype(np.complex64), S, lines, centred=centred) + p.noise
        _ORACLE_INPUTS[key] = dict(y=y, S=S, lines=lines, centred=centred)
    return _ORACLE_INPUTS[key]


def oracle_sample(frames, iters, seed_offset=0, centred=False, lam=0.0, lam_t=0.0, wl=CINE, y=None, S=None):
    """Time oracle CG-SENSE on `frames` frames of the workload for `iters`
    iterations (on the given k-space and maps if passed, e.g. BF16-rounded
    ones).  Returns (applications/s, wall seconds, threads, images, frame indices)."""
    import oracle

    d = oracle_inputs(centred, wl)
    sel = [(i + seed_offset) % wl.frames for i in range(frames)]
    yy = (d["y"] if y is None else y)[sel]
    SS = d["S"] if S is None else S
    lines = d["lines"][sel]
    t0 = time.perf_counter()
    x = oracle.cg(yy, SS, lines, iters, centred=d["centred"], lam=lam, lam_t=lam_t)[0]
    wall = time.perf_counter() - t0
    return frames * iters / wall, wall, min(oracle.threads(), frames), x, sel


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    if args.workload == "paper":
        return run_reference_paper(args)
    import oracle

    wl = WORKLOADS.get(args.workload, CINE)
    threads = oracle.threads()
    frames = max(1, min(wl.frames, threads))
    iters = 2 if wl.n <= 256 else 1
    for _ in range(args.warmup):
        oracle_sample(frames, 1, centred=args.centred, wl=wl)
    walls = []
    apps = 0
    for k in range(args.steps):
        _, wall, _, _, _ = oracle_sample(frames, iters, seed_offset=k, centred=args.centred, wl=wl)
        walls.append(wall)
        apps += frames * iters
    total = sum(walls)
    value = apps / total
    sample = "%d of %d frames x %d CG iterations per step (full %dx%d, %d coils, R=%d)" % (
        frames, wl.frames, iters, wl.n, wl.n, wl.coils, wl.accel)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": base_config(1, args.centred, wl, args.storage),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(threads, frames), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [v.strip() for v in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [s for t, s in self.samples if t0 <= t <= t1]
        window = "timed region"
        if len(rows) < 2:  # short timed region: widen to the loaded period around it
            rows = [s for t, s in self.samples if t0 - 2.0 <= t <= t1 + 0.5]
            window = "timed region +- load around it"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        sm, smax, pw = [], [], []
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
                pw.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(rows),
                "window": window}


# ---------------------------------------------------------------------------
# GPU side
# ---------------------------------------------------------------------------
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def cg_accuracy(plan, y, S, lines, x_ref, sel, iters, wl, args, requant_sample):
    """Relative L2 error of this plan's CG images (frames `sel`, `iters`
    iterations) against the FP64 oracle's on the same k-space and maps.  For
    BF16 storage the oracle also runs on the BF16-rounded inputs, which
    separates the storage error from the arithmetic error."""
    import torch

    import oracle
    from paper_1807_11830_gb300 import sense

    F, ny, nx = wl.frames, wl.n, wl.n
    x = torch.empty((F, ny, nx), dtype=torch.complex64, device=y.device)
    it = torch.zeros(F, dtype=torch.int32, device=y.device)
    sense.sense_cg_solve(plan, y, S, lines, iters, 0.0, x, it)
    sense.sense_plan_check(plan)
    xg = x.cpu().numpy()[sel].astype(np.complex128)

    def rel(a, b):
        return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

    out = {"cg_iterations": iters, "frames": len(sel), "metric": "relative L2 over the sampled frames",
           "vs_fp64_oracle": rel(xg, x_ref)}
    if requant_sample is not None:
        d = oracle_inputs(args.centred, wl)
        _, _, _, x_q, _ = requant_sample(len(sel), iters, centred=args.centred, lam=args.lam, lam_t=args.lam_t,
                                         wl=wl, y=oracle.quantize_c64_bf16(d["y"]),
                                         S=oracle.quantize_c64_bf16(d["S"]))
        out["vs_fp64_oracle_on_bf16_inputs"] = rel(xg, x_q)
        out["note"] = ("vs_fp64_oracle: storage + arithmetic error (exact inputs); "
                       "vs_fp64_oracle_on_bf16_inputs: arithmetic error alone")
    return out


_FP32_PEAK = {}


def fp32_peak(device, sm_max_mhz):
    """(TFLOP/s, source) of the FP32 ALU roofline: the library's FMA-chain
    microbenchmark on this GPU (measured once per process)."""
    from paper_1807_11830_gb300 import sense

    if device not in _FP32_PEAK:
        try:
            _FP32_PEAK[device] = (sense.sense_fp32_peak(device),
                                  "measured: sense_fp32_peak FMA-chain microbenchmark on this GPU")
        except Exception as exc:  # report the derived figure and say so
            _FP32_PEAK[device] = (152 * 128 * 2 * sm_max_mhz * 1e6 / 1e12,
                                  "derived (measurement failed: %s): 152 SMs x 128 lanes x 2 flop x %.0f MHz"
                                  % (exc, sm_max_mhz))
    return _FP32_PEAK[device]


def time_operators(plan, x_img, y, S, lines, flush, stream, dev, sbytes=8, reps=20, only=None):
    """E (sense_forward), E^H (sense_adjoint) and E^H E (sense_normal) on the
    workload's configuration, each call timed alone with CUDA events on
    `stream` after 3 warm-up calls, L2 flushed before each.  Applications =
    frames.  Algorithmic bytes per call: the operator's inputs and outputs once
    (S once for all frames; `sbytes` per stored complex value of S and y); the
    two-pass intermediate is not counted.  `hbm_frac_s_per_frame` counts S
    once per frame instead (the per-frame minimum of the forward operator);
    `hbm_frac_two_pass` adds, for E and E^H, the write and re-read of the
    compacted [F][C][L][nx] complex64 intermediate (16·F·C·L·nx bytes) that
    the two-launch form moves between its row and column passes."""
    import torch

    from paper_1807_11830_gb300 import sense

    F, ny, nx = x_img.shape
    C, L = S.shape[0], lines.shape[1]
    img = ny * nx
    y_out = torch.empty_like(y)
    x_out = torch.empty_like(x_img)
    calls = {
        "forward": (lambda: sense.sense_forward(plan, x_img, S, lines, y_out, stream=stream),
                    8 * F * img + sbytes * (C * img + F * C * L * nx), sbytes * (F - 1) * C * img, 16 * F * C * L * nx),
        "adjoint": (lambda: sense.sense_adjoint(plan, y, S, lines, x_out, stream=stream),
                    sbytes * (F * C * L * nx + C * img) + 8 * F * img, sbytes * (F - 1) * C * img, 16 * F * C * L * nx),
        "normal": (lambda: sense.sense_normal(plan, x_img, S, lines, x_out, stream=stream),
                   sbytes * C * img + 16 * F * img, sbytes * (F - 1) * C * img, 0),
    }
    hbm_gbs, _, _ = peaks()
    out = {}
    for name, (call, nbytes, s_extra, inter) in calls.items():
        if only and name not in only:
            continue
        for _ in range(3):
            call()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in ev:
            flush.fill_(3)
            e0.record(stream)
            call()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        sense.sense_plan_check(plan)
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / reps
        gbs = nbytes / (ms / 1e3) / 1e9
        out[name] = {"applications_per_s": F / (ms / 1e3), "ms": ms, "algorithmic_mb": nbytes / 1e6,
                     "achieved_gbs": gbs, "hbm_frac": gbs / hbm_gbs,
                     "hbm_frac_s_per_frame": (nbytes + s_extra) / (ms / 1e3) / 1e9 / hbm_gbs}
        if inter:
            out[name]["hbm_frac_two_pass"] = (nbytes + s_extra + inter) / (ms / 1e3) / 1e9 / hbm_gbs
    return out


def run_ours(args):
    import torch

    from paper_1807_11830_gb300 import build as sense_build
    from paper_1807_11830_gb300 import sense, synth

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if not os.path.exists(sense.LIB_PATH):
        sense_build.build()
    sense.load_library()

    wl = WORKLOADS[args.workload]
    FRAMES, COILS, N, ITERS = wl.frames, wl.coils, wl.n, wl.iters
    bf16 = args.storage == "bf16"
    store = sense.STORE_BF16 if bf16 else sense.STORE_C64
    sbytes = 4 if bf16 else 8  # bytes per stored complex value of S and y

    # ---- inputs (seeded; k-space made on the device by the library's E) ----
    p = wl.make(FRAMES)
    L = p.lines.shape[1]
    x_true = torch.from_numpy(p.x_true.astype(np.complex64)).to(dev)
    S = torch.from_numpy(p.S.astype(np.complex64)).to(dev)
    lines_np = synth.centred_lines(p.lines, N) if args.centred else p.lines
    lines = torch.from_numpy(lines_np).to(dev)
    y = torch.empty((FRAMES, COILS, L, N), dtype=torch.complex64, device=dev)
    mk = sense.Plan(N, N, COILS, FRAMES, L, device=local_rank, centred=args.centred)
    sense.sense_forward(mk, x_true, S, lines, y)
    y += torch.from_numpy(p.noise.astype(np.complex64)).to(dev)
    torch.cuda.synchronize(dev)
    mk.close()
    if bf16:  # S and y stored as bfloat16 pairs, rounded by the library's RNE conversion
        S, y = sense.to_bf16_pairs(S), sense.to_bf16_pairs(y)
        torch.cuda.synchronize(dev)
    plan = sense.Plan(N, N, COILS, FRAMES, L, store, device=local_rank, centred=args.centred)
    if args.lam:
        sense.sense_plan_set_lambda(plan, args.lam)
    if args.lam_t:
        sense.sense_plan_set_temporal(plan, args.lam_t)
    if args.normal_variant == "auto":
        variant, tune_ms = sense.sense_plan_autotune(plan, S, lines)
    else:
        variant, tune_ms = int(args.normal_variant), {}
        sense.sense_plan_set_variant(plan, variant)
    x = torch.empty((FRAMES, N, N), dtype=torch.complex64, device=dev)
    iters = torch.zeros(FRAMES, dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        sense.sense_cg_solve(plan, y, S, lines, ITERS, 0.0, x, iters, stream=stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()

    modes = {"graph": sense.CG_MODE_GRAPH, "persistent": sense.CG_MODE_PERSISTENT}
    mode_ms = {}
    if args.cg_mode == "auto":
        for name, m in modes.items():
            sense.sense_plan_set_cg_mode(plan, m)
            for _ in range(3):
                step()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            mode_ms[name] = e0.elapsed_time(e1) / 5
        cg_mode = min(mode_ms, key=mode_ms.get)
    else:
        cg_mode = args.cg_mode
    sense.sense_plan_set_cg_mode(plan, modes[cg_mode])
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    sense.sense_plan_check(plan)
    if int(iters.min()) != ITERS:
        raise RuntimeError("CG did not run %d iterations per frame" % ITERS)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)

    # ---- device-resident timed region ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    t_wall0 = time.time()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    barrier()
    t_wall1 = time.time()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)

    # ---- end to end through the host-buffer C-ABI call: pinned host inputs in, image out ----
    # (sense_cg_solve_host copies y, S and lines to the device, solves, copies x back and
    # synchronises the stream, all inside the timed region)
    y_h = y.cpu().pin_memory()
    S_h = S.cpu().pin_memory()
    lines_h = lines.cpu().pin_memory()
    x_h = torch.empty(x.shape, dtype=x.dtype).pin_memory()

    def e2e_step():
        sense.sense_cg_solve_host(plan, y_h, S_h, lines_h, ITERS, 0.0, x_h, stream=stream)

    for _ in range(3):
        e2e_step()
    e_starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        e_starts[k].record(stream)
        e2e_step()
        e_ends[k].record(stream)
    barrier()
    clocks.stop()
    e2e_ms = sum(s.elapsed_time(e) for s, e in zip(e_starts, e_ends))
    h2d = sum(t.numel() * t.element_size() for t in (y, S, lines))
    d2h = x.numel() * x.element_size()

    # ---- kernel roofline: the same step with the plan's event timers on ----
    timed_steps = 5
    sense.sense_plan_set_timing(plan, True)
    for _ in range(timed_steps):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(dev)
    phase = {}
    for name in sense.PHASES:
        ms, n = sense.sense_plan_phase_time(plan, name)
        if n:
            phase[name] = {"ms_per_launch": ms / n, "launches": n, "ms_total": ms}
    sense.sense_plan_set_timing(plan, False)

    # ---- the operators on their own (steps A, B, C outside CG), same plan and inputs ----
    operators = time_operators(plan, x_true, y, S, lines, flush, stream, dev, sbytes) if rank == 0 else None
    if operators is not None:  # the same calls with the two-launch forms, for comparison
        for mode, key in ((2, "fused_single_launch"), (0, "per_tile_column_kernels")):
            sense.sense_plan_set_column_pass(plan, mode)
            reg = time_operators(plan, x_true, y, S, lines, flush, stream, dev, sbytes, only=("forward", "adjoint"))
            operators[key] = {k: {"ms": v["ms"], "hbm_frac": v["hbm_frac"]} for k, v in reg.items()}
        sense.sense_plan_set_column_pass(plan, 1)

    # max over ranks
    total_ms, e2e_ms = max_over_ranks([total_ms, e2e_ms], world, dev)

    apps_per_step = FRAMES * ITERS
    value = apps_per_step * world * args.steps / (total_ms / 1e3)
    e2e_value = apps_per_step * world * args.steps / (e2e_ms / 1e3)

    if rank == 0:
        hbm_gbs, sm_max_mhz, peak_src = peaks()
        img = N * N
        # dominant kernel: the CG iteration.  Algorithmic work per CG iteration (all 20 frames):
        #   flops = C * F * (2 * Nx * 5 Ny log2 Ny + 14 Ny Nx)   (5 n log2 n per length-n transform)
        #   bytes = 8 * img * (C + 10 F): S once for the plan's frames; per frame the normal
        #           product with its p-update prologue moves 4 image vectors (r, p_prev read;
        #           p, q written) and the fused x/r update 6 (x, p, q, r read; x, r written)
        cgn = phase.get("cg_normal", {})
        dur_s = cgn.get("ms_per_launch", float("nan")) / 1e3
        kernel_name = "k_normal (CG mode)"
        if cg_mode == "persistent":
            # one launch runs every iteration: normal products and updates, all frames
            pers = phase.get("cg_persistent", {})
            dur_s = pers.get("ms_per_launch", float("nan")) / 1e3 / ITERS
            kernel_name = "k_cg_persistent (per CG iteration: normal product + update, %d frames)" % FRAMES
        flops = COILS * FRAMES * (2 * N * 5 * N * np.log2(N) + 14 * img)
        bytes_ = img * (sbytes * COILS + 80 * FRAMES)
        bytes_s_per_frame = img * FRAMES * (sbytes * COILS + 80)
        alu_peak_tflops, alu_peak_src = fp32_peak(local_rank, sm_max_mhz)
        achieved_tflops = flops / dur_s / 1e12
        # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one ncu
        # capture of this launch configuration, per CG iteration; null for any
        # other configuration
        traffic = CINE_TRAFFIC_PER_ITER.get((variant, cg_mode)) if (wl is CINE and not bf16) else None
        roofline = {
            "kernel": kernel_name, "bound": "alu", "achieved": achieved_tflops, "peak": alu_peak_tflops,
            "unit": "TFLOP/s", "frac": achieved_tflops / alu_peak_tflops, "traffic": traffic,
            "peak_source": alu_peak_src,
            "algorithmic_gflop_per_launch": flops / 1e9, "algorithmic_mb_per_launch": bytes_ / 1e6,
            "hbm_achieved_gbs": bytes_ / dur_s / 1e9, "hbm_peak_gbs": hbm_gbs,
            "hbm_frac": bytes_ / dur_s / 1e9 / hbm_gbs,
            "hbm_frac_s_per_frame": bytes_s_per_frame / dur_s / 1e9 / hbm_gbs,
            "hbm_peak_source": "%s copy bandwidth (MEASURED_PEAKS.json)" % peak_src,
            "duration_us": dur_s * 1e6,
        }
        cpu = None
        accuracy = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            frames = max(1, min(FRAMES, oracle.threads()))
            acc_iters = args.accuracy_iters or (ITERS if N <= 256 else 4)
            # the oracle on the same inputs: the timed sample doubles as the accuracy check of this
            # run's images (the GPU solves again for acc_iters iterations when that differs)
            v, wall, cores, x_ref, sel = oracle_sample(frames, acc_iters, centred=args.centred, lam=args.lam,
                                                       lam_t=args.lam_t, wl=wl)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d of %d frames x %d CG iterations (full %dx%d, %d coils, R=%d, FP64), %.1f s"
                             % (frames, FRAMES, acc_iters, N, N, COILS, wl.accel, wall)}
            accuracy = cg_accuracy(plan, y, S, lines, x_ref, sel, acc_iters, wl, args, oracle_sample if bf16 else None)
        # our kernels per step, counted by the plan's launch timers in the timing pass
        launches_per_step = sum(v["launches"] for v in phase.values()) / timed_steps
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 storage / f32 math / f64 dots" if bf16 else "f32", "data": "synthetic",
            "config": dict(base_config(world, args.centred, wl, args.storage),
                           **({"tikhonov_lambda": args.lam} if args.lam else {}),
                           **({"temporal_lambda": args.lam_t} if args.lam_t else {})),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": e2e_ms / args.steps,
                    "path": "sense_cg_solve_host: pinned host buffers through the C ABI (copies in the timed region)"},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "accuracy": accuracy,
            "clocks": clocks.summary(t_wall0, t_wall1),
            "kernels_us": {k: round(v["ms_per_launch"] * 1e3, 2) for k, v in phase.items()},
            "operators": operators,
            "normal_variant": variant,
            "cg_mode": cg_mode,
            "cg_mode_ms": {k: round(v, 4) for k, v in mode_ms.items()},
            "autotune_us": {str(k): round(v * 1e3, 2) for k, v in tune_ms.items()},
            "step_ms_p50": statistics.median(step_ms), "step_ms_min": min(step_ms),
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    plan.close()
    return 0


# ---------------------------------------------------------------------------
# uneven batching: 512 seeded instances, one persistent launch per size class
# ---------------------------------------------------------------------------
def mix_inputs(args, dev):
    """Seeded mix: shapes from synth.draw_mix; maps from the coil model,
    cached per (n, coils); lines per instance; k-space seeded complex
    Gaussian on the device (the CG cost does not depend on the values)."""
    import torch

    from paper_1807_11830_gb300 import sense, synth

    specs = synth.draw_mix(args.mix_count)
    smaps = {}
    gen = torch.Generator(device=dev)
    gen.manual_seed(1810)
    inst = []
    for k, sp in enumerate(specs):
        n, C, F, L = sp["n"], sp["coils"], sp["frames"], sp["lines"]
        if (n, C) not in smaps:
            smaps[(n, C)] = torch.from_numpy(synth.sensitivities(C, n, n).astype(np.complex64)).to(dev)
        lines = synth.mask_lines(n, L, sp["centre"], F, synth.rng_for(20000 + k))
        y = torch.randn((F, C, L, n), dtype=torch.complex64, device=dev, generator=gen) * 1e-2
        inst.append(dict(spec=sp, S=smaps[(n, C)], lines=torch.from_numpy(lines).to(dev), y=y,
                         x=torch.empty((F, n, n), dtype=torch.complex64, device=dev)))
    return specs, inst


def run_mix(args):
    import torch

    from paper_1807_11830_gb300 import sense

    rank, local_rank, world = dist_env()
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    sense.load_library()
    ITER = 20
    t0 = time.time()
    specs, inst = mix_inputs(args, dev)
    if world > 1:  # independent instances: each rank solves its longest-first share
        mine = shard_instances(specs, world, rank)
        specs, inst = [specs[i] for i in mine], [inst[i] for i in mine]
    shapes = [dict(ny=sp["n"], nx=sp["n"], coils=sp["coils"], frames=sp["frames"], lines=sp["lines"])
              for sp in specs]
    batch = sense.Batch(shapes)
    items = [dict(y=d["y"], S=d["S"], lines=d["lines"], x_out=d["x"]) for d in inst]
    sense.sense_batch_autotune(batch, items)
    setup_s = time.time() - t0
    frames = sum(sp["frames"] for sp in specs)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 1)):
        sense.sense_batch_cg_solve(batch, items, ITER)
    torch.cuda.synchronize(dev)
    ms = []
    for k in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sense.sense_batch_cg_solve(batch, items, ITER)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    sense.sense_batch_check(batch)
    batch_ms = statistics.median(ms)
    ws = batch.workspace_bytes
    batch.close()
    # per size class: a batch of that class's instances alone (one persistent launch per solve plus
    # the instances' CG starts), timed the same way; its algorithmic bytes and flops per CG iteration
    hbm_gbs, _, peak_src = peaks()
    fp32_tflops, fp32_src = fp32_peak(local_rank, 2070.0)
    classes = {}
    for n in sorted({sp["n"] for sp in specs}):
        sel = [k for k, sp in enumerate(specs) if sp["n"] == n]
        cb = sense.Batch([shapes[k] for k in sel])
        citems = [items[k] for k in sel]
        sense.sense_batch_autotune(cb, citems)
        sense.sense_batch_cg_solve(cb, citems, ITER)
        torch.cuda.synchronize(dev)
        cms = []
        for _ in range(max(1, min(args.steps, 3))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sense.sense_batch_cg_solve(cb, citems, ITER)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            cms.append(e0.elapsed_time(e1))
        sense.sense_batch_check(cb)
        cb.close()
        c_ms = statistics.median(cms)
        img = n * n
        nbytes = sum(8 * img * (specs[k]["coils"] + 10 * specs[k]["frames"]) for k in sel) * ITER
        flops = sum(specs[k]["coils"] * specs[k]["frames"] for k in sel) * (2 * n * 5 * n * np.log2(n) + 14 * img) * ITER
        classes[str(n)] = {"instances": len(sel), "frames": sum(specs[k]["frames"] for k in sel), "ms": c_ms,
                           "algorithmic_gb": nbytes / 1e9, "achieved_gbs": nbytes / (c_ms / 1e3) / 1e9,
                           "hbm_frac": nbytes / (c_ms / 1e3) / 1e9 / hbm_gbs,
                           "achieved_tflops": flops / (c_ms / 1e3) / 1e12,
                           "fp32_frac": flops / (c_ms / 1e3) / 1e12 / fp32_tflops}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    d = classes[dom]
    roofline = {"kernel": "k_cg_persistent, size class %s (%d instances, %d frames, %d CG iterations in one launch)"
                          % (dom, d["instances"], d["frames"], ITER),
                "bound": "alu", "achieved": d["achieved_tflops"], "peak": fp32_tflops, "unit": "TFLOP/s",
                "frac": d["fp32_frac"], "traffic": MIX_TRAFFIC_PER_ITER.get(dom), "peak_source": fp32_src,
                "hbm_achieved_gbs": d["achieved_gbs"], "hbm_peak_gbs": hbm_gbs, "hbm_frac": d["hbm_frac"],
                "hbm_peak_source": "%s copy bandwidth (MEASURED_PEAKS.json)" % peak_src,
                "algorithmic_bytes": "8 n^2 (C + 10 F) per instance and CG iteration (S once; 4 image vectors for "
                                     "the normal product and its p update, 6 for the x/r update per frame)",
                "duration_us_per_iteration": d["ms"] * 1e3 / ITER}
    # plain per-instance loop: the same kernels, per-iteration launches, no graphs, one instance at a time
    plans = []
    for d, sp in zip(inst, specs):
        pl = sense.Plan(sp["n"], sp["n"], sp["coils"], sp["frames"], sp["lines"])
        sense.sense_plan_set_cg_mode(pl, sense.CG_MODE_DIRECT)
        plans.append(pl)
    for pl, d in zip(plans, inst):  # warm-up (kernel attributes, caches)
        sense.sense_cg_solve(pl, d["y"], d["S"], d["lines"], 1, 0.0, d["x"])
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for pl, d in zip(plans, inst):
        sense.sense_cg_solve(pl, d["y"], d["S"], d["lines"], ITER, 0.0, d["x"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = e0.elapsed_time(e1)
    for pl in plans:
        pl.close()
    batch_ms, plain_ms = max_over_ranks([batch_ms, plain_ms], world, dev)
    if world > 1:
        tot = torch.tensor([frames], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tot)
        frames = int(tot.item())
        torch.distributed.destroy_process_group()
        if rank != 0:
            return 0
    apps = frames * ITER
    line = {
        "metric": METRIC, "value": apps / (batch_ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": batch_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "uneven batch: %d instances (n in {128,192,256,384}, coils 8..32, frames 1..30, "
                               "R in {2,3,4,6}), %d CG iterations" % (len(specs), ITER),
                   "frames": frames, "size_classes": len(set(sp["n"] for sp in specs)),
                   "l2": "working set far larger than L2"},
        "plain_loop": {"value": apps / (plain_ms / 1e3), "unit": UNIT, "ms_per_step": plain_ms,
                       "kind": "same kernels, per-iteration launches, one instance at a time"},
        "speedup_vs_plain": plain_ms / batch_ms,
        "workspace_gb": ws / 1e9, "setup_s": setup_s,
        "roofline": roofline, "size_classes": classes,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# serving: Poisson request streams through the queue
# ---------------------------------------------------------------------------
# page-locked staging the serving queue reserves up front: the inputs of the whole stream (under
# overload every request's inputs are staged at once), at most 64 GiB
SERVE_STAGING_CAP = 64 << 30


def serve_pool(count, dev):
    """`count` request instances drawn from the uneven-batch distribution (n,
    coils, frames, acceleration), each its own phantom series, lines and
    noise; maps per (n, coils); k-space = E x + noise made by the library's E.
    Host copies (the queue and the serial loop both take host buffers)."""
    import torch

    from paper_1807_11830_gb300 import sense, synth

    specs = synth.draw_mix(count, seed=1811)
    maps = {}
    pool = []
    for k, sp in enumerate(specs):
        p = synth.mix_instance(sp, 30000 + k)
        F, n = p.x_true.shape[0], p.x_true.shape[1]
        C, L = p.S.shape[0], p.lines.shape[1]
        if (n, C) not in maps:
            maps[(n, C)] = p.S.astype(np.complex64)
        S = maps[(n, C)]
        plan = sense.Plan(n, n, C, F, L)
        S_d = torch.from_numpy(S).to(dev)
        l_d = torch.from_numpy(p.lines).to(dev)
        y_d = torch.empty((F, C, L, n), dtype=torch.complex64, device=dev)
        sense.sense_forward(plan, torch.from_numpy(p.x_true.astype(np.complex64)).to(dev), S_d, l_d, y_d)
        y_d += torch.from_numpy(p.noise.astype(np.complex64)).to(dev)
        pool.append(dict(shape=dict(ny=n, nx=n, coils=C, frames=F, lines=L), y=y_d.cpu().numpy(), S=S,
                         lines=np.ascontiguousarray(p.lines, np.int32), frames=F, n=n, spec=sp))
        plan.close()
    return pool


def run_serve(args):
    import tempfile

    import torch

    from paper_1807_11830_gb300 import sense, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sense.load_library()
    MAXIT, TOL = 100, 1e-4
    t_setup = time.time()
    pool = serve_pool(args.serve_pool, dev)
    # serial plain solver: a plan per pool instance in direct mode (per-iteration launches, no graphs,
    # one request at a time), its kernel variant autotuned for that mode, inputs and image through the
    # host-buffer C-ABI call; plans and their device buffers made before any stream (untimed)
    plans = []
    for e in pool:
        sh = e["shape"]
        pl = sense.Plan(sh["ny"], sh["nx"], sh["coils"], sh["frames"], sh["lines"])
        sense.sense_plan_set_cg_mode(pl, sense.CG_MODE_DIRECT)
        sense.sense_plan_autotune(pl, torch.from_numpy(e["S"]).to(dev), torch.from_numpy(e["lines"]).to(dev))
        plans.append(pl)
    host = []
    for e, pl in zip(pool, plans):
        F, n = e["frames"], e["n"]
        h = dict(y=torch.from_numpy(e["y"]), S=torch.from_numpy(e["S"]), lines=torch.from_numpy(e["lines"]),
                 x=torch.empty((F, n, n), dtype=torch.complex64), it=torch.zeros(F, dtype=torch.int32),
                 res=torch.zeros(F, dtype=torch.float64))
        sense.sense_cg_solve_host(pl, h["y"], h["S"], h["lines"], 1, 0.0, h["x"])  # device buffers, warm-up
        host.append(h)
    # kernel variant per size class for the queue: autotuned in persistent mode once, before any
    # stream (as a deployment would load it from a cache), on a loaded class -- 30 frames of 16
    # coils at R = 4 -- since under load each class launch carries the frames of many requests
    class_variant = {}
    for n in sorted({e["n"] for e in pool}):
        F_t, C_t, L_t = 30, 16, n // 4
        tp = sense.Plan(n, n, C_t, F_t, L_t)
        sense.sense_plan_set_cg_mode(tp, sense.CG_MODE_PERSISTENT)
        lines_t = synth.mask_lines(n, L_t, synth.centre_for(n), F_t, synth.rng_for(4242 + n))
        S_t = synth.sensitivities(C_t, n, n).astype(np.complex64)
        class_variant[n], _ = sense.sense_plan_autotune(tp, torch.from_numpy(S_t).to(dev),
                                                        torch.from_numpy(np.ascontiguousarray(lines_t, np.int32)).to(dev))
        tp.close()
    setup_s = time.time() - t_setup

    def pct(v, p):
        return float(np.percentile(v, p)) if len(v) else None

    def converged(iters, resid):
        return bool(np.all((resid <= TOL) | (iters >= MAXIT)))

    results = {}
    wave_list = [float(w) for w in str(args.serve_admit_waves).split(",")]
    for rate, waves in [(float(r), w) for r in args.serve_rates.split(",") for w in wave_list]:
        count = args.serve_requests
        arrivals = synth.poisson_arrivals(rate, count, seed=int(rate) + 1811)
        picks = synth.rng_for(int(rate) + 7).integers(0, len(pool), size=count)
        # ---- the queue: latency from each request's arrival time to its retirement (queue log) ----
        log_path = tempfile.mktemp(prefix="sense_queue_", suffix=".jsonl")
        os.environ["SENSE_QUEUE_LOG"] = log_path
        staging = min(SERVE_STAGING_CAP, int(sum(pool[pk]["y"].nbytes + pool[pk]["S"].nbytes + pool[pk]["lines"].nbytes
                                                 + 8 * pool[pk]["frames"] * pool[pk]["n"] ** 2 for pk in picks)))
        try:
            q = sense.Queue(device=0, staging_reserve_bytes=staging, max_live_work=args.serve_live_work,
                            admit_waves=waves)
        except sense.SenseError:  # not that much page-locked memory: let the arena grow on demand
            staging = 4 << 30
            q = sense.Queue(device=0, staging_reserve_bytes=staging, max_live_work=args.serve_live_work,
                            admit_waves=waves)
        os.environ.pop("SENSE_QUEUE_LOG", None)
        for n, v in class_variant.items():
            q.set_variant(n, n, v)
        t0 = time.perf_counter()
        ids, sub_t, late = [], [], 0.0
        for a, pk in zip(arrivals, picks):
            now = time.perf_counter() - t0
            if a > now:
                time.sleep(a - now)
            else:
                late = max(late, now - a)
            e = pool[pk]
            sub_t.append(time.perf_counter() - t0)
            ids.append(q.submit(e["shape"], e["y"], e["S"], e["lines"], MAXIT, TOL))
        q_ok = True
        for rid, pk in zip(ids, picks):
            F = pool[pk]["frames"]
            it, rs = np.zeros(F, np.int32), np.zeros(F, np.float64)
            q.wait(rid, iters=it, resid=rs)
            q_ok = q_ok and converged(it, rs)
        wall = time.perf_counter() - t0
        st = q.stats()
        q.close()
        done_ms, submit_ms = {}, {}
        with open(log_path) as fh:
            for line in fh:
                d = json.loads(line)
                done_ms[d["id"]] = d["done_ms"]
                submit_ms[d["id"]] = d["submit_ms"]
        if args.serve_log_dir:  # keep the queue's per-request log
            os.makedirs(args.serve_log_dir, exist_ok=True)
            os.replace(log_path, os.path.join(args.serve_log_dir, "queue_%dhz_w%g.jsonl" % (int(rate), waves)))
        else:
            os.remove(log_path)
        # the queue log's clock (ms since its creation) against ours: each submit call's start is
        # stamped by both, so their median difference maps retirement times onto arrival times
        offset = float(np.median([submit_ms[rid] - 1e3 * t for rid, t in zip(ids, sub_t)]))
        q_lat = [done_ms[rid] - offset - 1e3 * a for rid, a in zip(ids, arrivals)]
        # ---- serial plain solves, live: one request at a time in arrival order ----
        s_lat, s_ok = [], True
        t0 = time.perf_counter()
        for a, pk in zip(arrivals, picks if not args.serve_queue_only else []):
            now = time.perf_counter() - t0
            if a > now:
                time.sleep(a - now)
            h = host[pk]
            sense.sense_cg_solve_host(plans[pk], h["y"], h["S"], h["lines"], MAXIT, TOL, h["x"], h["it"], h["res"])
            s_lat.append((time.perf_counter() - t0 - a) * 1e3)
            s_ok = s_ok and converged(h["it"].numpy(), h["res"].numpy())
        s_wall = time.perf_counter() - t0
        frames = int(sum(pool[pk]["frames"] for pk in picks))
        results[str(int(rate)) if len(wave_list) == 1 else "%d@%g" % (int(rate), waves)] = {
            "p50_ms": pct(q_lat, 50), "p99_ms": pct(q_lat, 99), "mean_ms": float(np.mean(q_lat)),
            "solves_per_s": count / wall, "ticks": st["ticks"],
            "latency_from_submit_p50_p99_ms": [st["p50_ms"], st["p99_ms"]],
            "submit_lag_max_ms": 1e3 * late,
            "every_request_converged_or_at_100_iterations": q_ok,
            "serial_plain": {"p50_ms": pct(s_lat, 50), "p99_ms": pct(s_lat, 99),
                             "mean_ms": float(np.mean(s_lat)) if s_lat else None,
                             "solves_per_s": count / s_wall if s_lat else None,
                             "every_request_converged_or_at_100_iterations": s_ok,
                             "kind": "live: one request at a time in arrival order through sense_cg_solve_host "
                                     "(host buffers in and out), plain per-iteration launches, a prepared plan per "
                                     "instance"},
            "requests": count, "frames": frames,
        }
    line = {
        "metric": "served recon latency p50/p99 (ms) and solves/s", "value": list(results.values())[-1]["solves_per_s"],
        "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals, %d requests per rate, each a draw from a pool of %d "
                               "instances sampled from the uneven-batch distribution (n in {128,192,256,384}, "
                               "coils 8..32, frames 1..30, R in {2,3,4,6}); CG to a relative residual of 1e-4 or "
                               "100 iterations" % (args.serve_requests, len(pool)),
                   "latency": "from each request's Poisson arrival time to its result being ready in host memory",
                   "queue_variants": {str(n): v for n, v in sorted(class_variant.items())},
                   "admit_waves": args.serve_admit_waves if args.serve_admit_waves != "0" else "default (12)",
                   "max_live_work": args.serve_live_work or "no limit",
                   "staging": "page-locked host staging for every input of the stream (at most %d GiB) reserved "
                              "at queue creation, before the stream starts" % (SERVE_STAGING_CAP >> 30),
                   "setup_s": setup_s},
        "rates": results,
    }
    print(json.dumps(line))
    for pl in plans:
        pl.close()
    return 0


# ---------------------------------------------------------------------------
# the paper's timed workload: fully sampled 2D inverse FFT + RSS (and Eq. 1)
# ---------------------------------------------------------------------------
_PAPER_ORACLE = {}


def paper_oracle_inputs(centred=False):
    """k-space of the paper workload made once by the oracle's E (untimed)."""
    if not _PAPER_ORACLE:
        import oracle
        from paper_1807_11830_gb300 import synth

        p = synth.paper_160()
        S = p.S.astype(np.complex64).astype(np.complex128)
        y = oracle.forward(p.x_true.astype(np.complex64), S, p.lines, centred=centred) + p.noise
        _PAPER_ORACLE.update(y=y, lines=p.lines, n=p.x_true.shape[1], centred=centred)
    return _PAPER_ORACLE


def paper_oracle_sample(min_seconds, centred=False):
    """Oracle FFT + RSS reconstructions of the whole workload, repeated for at
    least `min_seconds`.  Returns (reconstructions/s, wall, count, threads)."""
    import oracle

    d = paper_oracle_inputs(centred)
    count, t0 = 0, time.perf_counter()
    while True:
        oracle.rss(d["y"], d["lines"], d["n"], centred=d["centred"])
        count += 1
        wall = time.perf_counter() - t0
        if wall >= min_seconds:
            return count / wall, wall, count, min(oracle.threads(), d["y"].shape[0])


def run_reference_paper(args):
    for _ in range(args.warmup):
        paper_oracle_sample(0.0, args.centred)
    walls, count = [], 0
    for _ in range(args.steps):
        _, wall, c, threads = paper_oracle_sample(0.0, args.centred)
        walls.append(wall)
        count += c
    value = count / sum(walls)
    line = {
        "metric": PAPER_METRIC, "value": value, "unit": PAPER_UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": PAPER_WORKLOAD + (", centred k-space" if args.centred else ""), "ny": 160, "nx": 160,
                   "frames": 16, "coils": 8},
        "cpu_baseline": {"value": value, "unit": PAPER_UNIT, "cores": threads, "kind": "oracle",
                         "sample": "one whole reconstruction (16 frames x 8 coils) per step"},
        "e2e": {"value": value, "unit": PAPER_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_paper(args):
    import torch

    from paper_1807_11830_gb300 import build as sense_build
    from paper_1807_11830_gb300 import sense, synth

    rank, local_rank, world = dist_env()
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if not os.path.exists(sense.LIB_PATH):
        sense_build.build()
    sense.load_library()

    p = synth.paper_160()
    F, C, n = p.x_true.shape[0], p.S.shape[0], p.x_true.shape[1]
    plan = sense.Plan(n, n, C, F, n, device=local_rank, centred=args.centred)
    x_true = torch.from_numpy(p.x_true.astype(np.complex64)).to(dev)
    S = torch.from_numpy(p.S.astype(np.complex64)).to(dev)
    lines = torch.from_numpy(p.lines).to(dev)
    y = torch.empty((F, C, n, n), dtype=torch.complex64, device=dev)
    sense.sense_forward(plan, x_true, S, lines, y)
    y += torch.from_numpy(p.noise.astype(np.complex64)).to(dev)
    out = torch.empty((F, n, n), dtype=torch.float32, device=dev)
    combined = torch.empty((F, n, n), dtype=torch.complex64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        sense.sense_rss(plan, y, lines, out, stream=stream)

    def step_eq1():
        sense.sense_adjoint(plan, y, S, lines, combined, stream=stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
        step_eq1()
    torch.cuda.synchronize(dev)
    sense.sense_plan_check(plan)

    def timed(fn):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            starts[k].record(stream)
            fn()
            ends[k].record(stream)
        barrier()
        return [a.elapsed_time(b) for a, b in zip(starts, ends)]

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.3)
    t_wall0 = time.time()
    step_ms = timed(step)
    t_wall1 = time.time()
    eq1_ms = timed(step_eq1)

    # end to end: pinned k-space in, RSS image out, inside the timed region
    y_h = y.cpu().pin_memory()
    lines_h = lines.cpu().pin_memory()
    out_h = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    y_d = torch.empty_like(y)
    lines_d = torch.empty_like(lines)

    def e2e_step():
        y_d.copy_(y_h, non_blocking=True)
        lines_d.copy_(lines_h, non_blocking=True)
        sense.sense_rss(plan, y_d, lines_d, out, stream=stream)
        out_h.copy_(out, non_blocking=True)

    for _ in range(3):
        e2e_step()
    e2e_list = timed(e2e_step)
    clocks.stop()

    # per-kernel times with the plan's event timers
    sense.sense_plan_set_timing(plan, True)
    for _ in range(5):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(dev)
    phase = {}
    launches_per_step = 0.0
    for name in sense.PHASES:
        ms, cnt = sense.sense_plan_phase_time(plan, name)
        if cnt:
            phase[name] = ms / cnt
            launches_per_step += cnt / 5.0
    sense.sense_plan_set_timing(plan, False)
    sense.sense_plan_check(plan)

    total_ms, eq1_total, e2e_total = max_over_ranks([sum(step_ms), sum(eq1_ms), sum(e2e_list)], world, dev)
    value = world * args.steps / (total_ms / 1e3)
    if rank == 0:
        hbm_gbs, _, peak_src = peaks()
        cimg = 8.0 * F * C * n * n  # one pass over the complex k-space (or its row-transformed copy)
        kernel_bytes = {"rows_inv": 2 * cimg, "adj_col": cimg + 4.0 * F * n * n,
                        "adj_fused": cimg + 4.0 * F * n * n}  # one launch: read y, write the image
        dom = max(kernel_bytes, key=lambda k: phase.get(k, 0.0))
        dur_s = phase[dom] / 1e3
        achieved = kernel_bytes[dom] / dur_s / 1e9
        roofline = {
            "kernel": {"rows_inv": "k_rows_bulk<160,+1> (inverse x-transforms of every k-space row)",
                       "adj_col": "k_adj_col_tma<160,c64,rss> (inverse y-transforms, |.|^2 summed over coils, "
                                  "sqrt)",
                       "adj_fused": "k_adjoint_fused<160,c64,rss> (both passes in one launch: inverse x- and "
                                    "y-transforms, |.|^2 summed over coils, sqrt)"}[dom],
            "bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
            "traffic": PAPER_TRAFFIC.get(dom), "peak_source": "%s hbm_gbs (copy)" % peak_src,
            "algorithmic_mb_per_launch": kernel_bytes[dom] / 1e6, "duration_us": dur_s * 1e6,
            "whole_op_minimum_mb": (cimg + 4.0 * F * n * n) / 1e6,
        }
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            v, wall, cnt, threads = paper_oracle_sample(10.0, args.centred)
            cpu = {"value": v, "unit": PAPER_UNIT, "cores": threads, "kind": "oracle",
                   "sample": "%d whole reconstructions (16 frames x 8 coils, FP64), %.1f s" % (cnt, wall)}
        paper_value = 1e3 / PAPER_GTX970_MS
        line = {
            "metric": PAPER_METRIC, "value": value, "unit": PAPER_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / paper_value, "dtype": "f32", "data": "synthetic",
            "config": {"workload": PAPER_WORKLOAD + (", centred k-space" if args.centred else ""), "ny": n, "nx": n,
                       "frames": F, "coils": C, "kspace": "centred (DC at n/2)" if args.centred else "uncentred (DC at 0)",
                       "l2": "flushed before every timed step (512 MiB device write)",
                       "parallelism": "replicas x%d (independent problems, no collective)" % world},
            "baseline_context": "OpenCLIPER on a GTX 970, clFFT 1.361 ms + RSS 0.252 ms (Table II): "
                                "another machine, context only",
            "e2e": {"value": world * args.steps / (e2e_total / 1e3), "unit": PAPER_UNIT,
                    "h2d_bytes_per_step": int(y.numel() * 8 + lines.numel() * 4),
                    "d2h_bytes_per_step": int(out.numel() * 4), "ms_per_step": e2e_total / args.steps},
            "eq1_combine": {"value": world * args.steps / (eq1_total / 1e3), "unit": PAPER_UNIT,
                            "ms_per_step": eq1_total / args.steps,
                            "kind": "sense_adjoint with every line sampled: sum_c conj(S_c) F^-1(Y_c)"},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks.summary(t_wall0, t_wall1),
            "kernels_us": {k: round(v * 1e3, 2) for k, v in phase.items()},
            "step_ms_p50": statistics.median(step_ms), "step_ms_min": min(step_ms),
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    plan.close()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mix":
        return run_mix(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "paper":
        return run_paper(args)
    return run_ours(args)  # cine, slices320


if __name__ == "__main__":
    sys.exit(main())
