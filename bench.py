#!/usr/bin/env python
"""Grid-point updates per second of the explicit FD wave step on GB300.

Workload: the smooth-random acoustic model, 512^3 physical points, h = 10 m,
40-point sponge on every face (592^3 computational points), Ricker 10 Hz
source at the centre, 256 x 256 receivers at 20 m depth, dt at CFL 0.4.
A bench step advances one time step at EACH space order 2/4/8/12/16 (five
solvers, the order sweep), i.e. the whole hot path five times: stencil
update with fused sponge, source injection, receiver interpolation.

Outputs one JSON line (rank 0). `value` is whole-job Gpts/s (computational
points x orders x steps / time, all ranks); the roofline entry is the
stencil kernel's algorithmic bytes (16 B per point: read u_n, u_{n-1}, c;
write u_{n+1}) over its CUDA-event time, against the measured HBM copy
bandwidth. `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ORDERS = (2, 4, 8, 12, 16)
BYTES_PER_POINT = 16          # acoustic l + s = 4 fields x 4 B (Section "Operational intensity")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="fdwave", choices=["fdwave", "reference"])
    p.add_argument("--n", type=int, default=512, help="physical grid points per axis")
    p.add_argument("--nb", type=int, default=40)
    p.add_argument("--orders", default=",".join(map(str, ORDERS)))
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--tile", type=int, default=-1, help="2.5D kernel tile configuration (-1 default)")
    p.add_argument("--zchunks", type=int, default=0, help="CTAs along z (0 default)")
    p.add_argument("--no-tti", action="store_true")
    p.add_argument("--no-fwi", action="store_true")
    p.add_argument("--no-storage", action="store_true")
    p.add_argument("--fwi-n", type=int, default=256)
    p.add_argument("--fwi-nt", type=int, default=2000)
    p.add_argument("--fwi-shots-side", type=int, default=4)
    p.add_argument("--tti-n", type=int, default=384, help="physical TTI grid points per axis")
    p.add_argument("--no-closure", action="store_true")
    p.add_argument("--closure-n", type=int, default=256, help="coarse physical points per axis (evaluation)")
    p.add_argument("--closure-train-n", type=int, default=96, help="coarse points per axis (training models)")
    p.add_argument("--closure-models", type=int, default=64)
    p.add_argument("--closure-patches", type=int, default=2000, help="patches kept per training model")
    p.add_argument("--closure-iters", type=int, default=8000)
    p.add_argument("--closure-eval", type=int, default=16, help="held-out models at full size")
    p.add_argument("--no-config1", action="store_true")
    p.add_argument("--details", default="bench_details.json",
                   help="file that receives every section of the run (the printed line is the summary)")
    p.add_argument("--profile-closure-step", type=int, default=0, metavar="N",
                   help="only run 40 plain and 2 closure steps on an N^3 coarse grid (+20 sponge), "
                        "random network: the case the closure kernel is profiled on")
    p.add_argument("--profile-closure-variant", type=int, default=0, choices=[0, 1, 2],
                   help="inference kernels of --profile-closure-step: 0 tcgen05, 1 FP32, 2 mma.sync")
    return p.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def launches_per_step(nrec):
    """Kernels of one forward step: the stencil, then the source injection
    and the receiver interpolation -- one block for both up to 256
    receivers (or the injection alone without receivers), two kernels
    above."""
    return 3 if nrec > 256 else 2


def kernel_source_sha(root=ROOT):
    """Hash of the acoustic stencil kernel's source (template + dispatch + PTX
    helpers), comments and white space removed: any change of the code
    changes it, an edit of a comment does not."""
    h = hashlib.sha256()
    for f in ("acoustic.cu", "acoustic_kernel.cuh", "ptx.cuh"):
        with open(os.path.join(root, "paper_1608_03984_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


TRAFFIC_SUMMARY = "acoustic_tma_dram_336.md"


def ncu_traffic_per_point(root=ROOT):
    """{order: DRAM bytes per point} of the stencil kernel from the committed
    ncu summary of the small case (336^3, one solver, one order per
    capture), if its kernel-source hash matches the source. The bench
    scales it to a full launch by the points of the workload."""
    path = os.path.join(root, "profiles", TRAFFIC_SUMMARY)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_sha=([0-9a-f]+)", text)
    if not m or m.group(1) != kernel_source_sha(root):
        return None
    out = {}
    for o, v in re.findall(r"TRAFFIC_BYTES_PER_POINT order=(\d+) ([0-9.]+)", text):
        out[int(o)] = float(v)
    return out or None


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, device="cpu"):
    """Largest value over the ranks of the default process group (the
    slowest rank's time); the value itself without a group (one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_rank, world, ms):
    """Gpts/s of the whole job: every rank's points over the slowest rank's
    time (weak scaling: each rank runs its own replica of the workload)."""
    return points_per_rank * world / (ms / 1e3) / 1e9


def workload(args, order, nt):
    from paper_1608_03984_gb300 import synth
    return synth.random_acoustic(n=args.n, nb=args.nb, order=order, nt=nt, nrec_side=256)


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(vp, h, nb, order, dt, planes=16):
    """A slab of `planes` computational z planes of the workload (full x/y
    extent) with a smooth random state: the bounded sample the oracle steps."""
    import numpy as np
    from oracle import oracle as O
    from paper_1608_03984_gb300 import synth
    k0 = vp.shape[0] // 2
    slab = vp[k0:k0 + planes]
    s = O.Setup(slab, h, nb, order, dt, gamma_vmax=float(vp.max()))
    # keep the sponge in x/y only: the slab is an interior piece along z
    s.c = s.c[nb:nb + planes]
    s.gz = np.zeros(planes)
    s.shape = s.c.shape
    u = synth.random_wavefield(s.shape, 3, scale=1e-3).astype(np.float64)
    um = synth.random_wavefield(s.shape, 4, scale=1e-3).astype(np.float64)
    return s, u, um


def time_oracle(samples, steps, max_seconds=None):
    from oracle import oracle as O
    pts = 0
    t0 = time.perf_counter()
    for it in range(steps):
        for s, u, um in samples:
            up = O.acoustic_step(s, u, um)
            pts += up.size
        if max_seconds and time.perf_counter() - t0 > max_seconds:
            break
    return pts, time.perf_counter() - t0


def cpu_threads():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args, orders):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    from paper_1608_03984_gb300 import synth
    base = workload(args, orders[0], 4)
    samples = []
    for o in orders:
        dt = base.dt
        samples.append(oracle_sample(base.vp, base.h, base.nb, o, dt))
    time_oracle(samples, args.warmup)
    pts, sec = time_oracle(samples, args.steps)
    gpts = pts / sec / 1e9
    nz, ny, nx = base.n_comp
    sample_desc = ("%d x %d x %d slab (16 z planes, full x/y incl. sponge) of the 592^3 grid per order,"
                   " orders %s, FP64 oracle" % (16, ny, nx, "/".join(map(str, orders))))
    line = {
        "impl": "reference", "metric": "Gpts/s per timestep", "value": gpts, "unit": "Gpts/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, orders, base),
        "e2e": {"value": gpts, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cpu_baseline": {"value": gpts, "unit": "Gpts/s", "cores": cpu_threads(), "kind": "oracle",
                         "sample": sample_desc},
    }
    print(json.dumps(line), flush=True)


def config_dict(args, orders, w):
    nz, ny, nx = w.n_comp
    return {"workload": "random_acoustic %d^3 + %d-point sponge (%dx%dx%d computational), h=10 m, "
                        "orders %s (one step of each per bench step), Ricker 10 Hz, 256x256 receivers"
                        % (args.n, args.nb, nz, ny, nx, "/".join(map(str, orders))),
            "grid": [nz, ny, nx], "orders": list(orders), "equation": "acoustic",
            "l2": "inputs larger than L2 (each field %.0f MB)" % (nz * ny * nx * 4 / 1e6),
            "global_batch": len(orders), "parallelism": "replicas" if args.gpus > 1 else "single"}


def run_fdwave(args, orders):
    import numpy as np
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1608_03984_gb300 import fdwave, opmodel

    nt = args.warmup + args.steps + 2
    base = workload(args, orders[0], nt)
    points = base.points
    stream = torch.cuda.current_stream()
    solvers = []
    for o in orders:
        s = fdwave.Solver(base.n, base.h, base.nb, o, stream=stream)
        s.set_model(base.vp).set_dt(base.dt).set_sources(base.src_xyz, base.wavelet)
        s.set_receivers(base.rec_xyz, nt)
        s.set_tile_config(args.tile)
        s.set_zchunks(args.zchunks)
        solvers.append(s)

    for s in solvers:
        s.step(args.warmup)
    for s in solvers:
        s.check()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    for s in solvers:
        s.profile_begin(args.steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for s in solvers:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    kern = [s.profile_end() for s in solvers]
    tiles = {o: s.tile_config for o, s in zip(orders, solvers)}
    zchs = {o: s.zchunks for o, s in zip(orders, solvers)}
    for s in solvers:
        s.check()
    ms = max_over_ranks(ms, device="cuda")
    value = whole_job_rate(points * len(orders) * args.steps, world, ms)
    hbm, peak_src = peaks()
    per_order = {}
    sum_bytes, sum_kms = 0.0, 0.0
    for o, (kms, nl) in zip(orders, kern):
        k = o + 1
        avg = kms / max(nl, 1)
        achieved = BYTES_PER_POINT * points / (avg / 1e3) / 1e9
        gpts_k = points / (avg / 1e3) / 1e9
        per_order[str(o)] = {
            "kernel_ms": avg, "kernel_gpts": gpts_k, "tile": tiles[o], "zchunks": zchs[o],
            "achieved_gbs": achieved,
            "frac_of_measured_hbm": achieved / hbm,
            "I_alg_paper": opmodel.oi("acoustic", k),
            "paper_model_gflops": gpts_k * opmodel.flops_per_point("acoustic", k),
            "roofline_gpts_paper_model": hbm / BYTES_PER_POINT,
        }
        sum_bytes += BYTES_PER_POINT * points * nl
        sum_kms += kms
    achieved = sum_bytes / (sum_kms / 1e3) / 1e9
    tpp = ncu_traffic_per_point()
    traffic = None
    if tpp is not None and all(o in tpp for o in orders):
        # mean DRAM bytes per launch over the orders of the sweep: bytes per
        # point measured on the 336^3 case, times the points of one launch
        traffic = sum(tpp[o] for o in orders) / len(orders) * points
        for o in orders:
            per_order[str(o)]["ncu_dram_bytes_per_point"] = tpp[o]
    roof = {"kernel": "acoustic_tma_kernel (orders %s)" % "/".join(map(str, orders)),
            "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_source": peak_src, "traffic": traffic,
            "algorithmic_bytes_per_launch": BYTES_PER_POINT * points}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, orders, base, stream)
    for s in solvers:
        s.close()
    tti = None
    if not args.no_tti:
        tti = run_tti(args, stream, steps=min(args.steps, 30), warmup=3)
    storage = None
    if not args.no_storage:
        storage = run_storage(args, base, stream,
                              {o: per_order[str(o)]["kernel_ms"] for o in orders},
                              steps=min(args.steps, 30), warmup=3)
    fwi_res = None
    if not args.no_fwi and world == 1:
        fwi_res = run_fwi(args)

    closure_res = None
    if not args.no_closure and world == 1:
        closure_res = run_closure(args)

    cfg1 = None
    if not args.no_config1:
        cfg1 = run_config1(stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        samples = [oracle_sample(base.vp, base.h, base.nb, o, base.dt) for o in orders]
        time_oracle(samples, 1)
        pts, sec = time_oracle(samples, 10 ** 6, max_seconds=args.cpu_seconds)
        nz, ny, nx = base.n_comp
        cpu = {"value": pts / sec / 1e9, "unit": "Gpts/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": "16 x %d x %d slab of the %dx%dx%d grid per order (orders %s), FP64 oracle, "
                         "%.1f s" % (ny, nx, nz, ny, nx, "/".join(map(str, orders)), sec)}

    # the paper's model restated for this GPU (measured HBM bandwidth; FP32
    # peak from 152 SMs x 128 FMA lanes x 2 FLOP x the measured SM clock)
    sm_ghz = (clk.get("sm_mhz") or 2070.0) / 1e3
    paper = opmodel.restate(hbm, opmodel.fp32_peak_gflops(clock_ghz=sm_ghz))
    for o, v in paper["table_cost"].items():
        if o in per_order:  # measured time for the Table tab:stab problem at this order
            v["measured_runtime_s"] = v["N"] * v["nt"] / (per_order[o]["kernel_gpts"] * 1e9)

    if rank == 0:
        full = {
            "metric": "Gpts/s per timestep", "value": value, "unit": "Gpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_dict(args, orders, base),
            "roofline": roof, "per_order": per_order, "e2e": e2e, "cpu_baseline": cpu, "tti": tti,
            "fwi": fwi_res, "storage": storage, "closure": closure_res, "config1": cfg1,
            "paper_model_gb300": paper, "clocks": clk,
            "gpu_launches": launches_per_step(base.rec_xyz.shape[0]) * len(orders) * args.steps,
        }
        line = headline(full, args.details)
        try:
            with open(args.details, "w") as f:
                json.dump(full, f, indent=1)
        except OSError as e:
            line["details"] = "not written: %s" % e
        # the summary line is the last line of the run
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


TTI_FIELD_BYTES = 11  # TTI kernel: read p, r, p-, r-, c, e, d, nx, ny; write p+, r+


def run_tti(args, stream, steps, warmup):
    """The TTI workload: 384^3 + 40-point sponge (464^3), h = 12.5 m, smooth
    random eps/delta/theta/phi, orders 8 and 12, FP32 / BF16 / FP16 storage
    (FP32 arithmetic). Kernel time from CUDA events around each launch."""
    import torch
    from paper_1608_03984_gb300 import fdwave, opmodel, synth
    hbm, _ = peaks()
    w = synth.random_tti(n=args.tti_n, nb=args.nb, order=8, nt=steps + warmup + 2, nrec_side=128)
    out = {"workload": "random_tti %d^3 + %d-point sponge (%d^3), h=12.5 m, orders 8/12"
                       % (args.tti_n, args.nb, w.n_comp[0]),
           "algorithmic_bytes_per_point": {"f32": 4 * TTI_FIELD_BYTES, "bf16": 2 * TTI_FIELD_BYTES,
                                           "f16": 2 * TTI_FIELD_BYTES},
           "paper_model_bytes_per_point": 60}
    for order in (8, 12):
        for st in ("f32", "bf16", "f16"):
            s = fdwave.Solver(w.n, w.h, w.nb, order, equation="tti", storage=st, stream=stream)
            s.set_model(w.vp, w.eps, w.delta, w.theta, w.phi).set_dt(w.dt)
            s.set_sources(w.src_xyz, w.wavelet).set_receivers(w.rec_xyz, w.nt)
            s.step(warmup)
            torch.cuda.synchronize()
            s.profile_begin(steps)
            s.step(steps)
            ms, n = s.profile_end()
            s.check()
            s.close()
            avg = ms / max(n, 1)
            gpts = w.points / (avg / 1e3) / 1e9
            bpp = (4 if st == "f32" else 2) * TTI_FIELD_BYTES
            # the paper's model of this kernel (Table 1, Eq. eqn_oi and
            # Eq. perf-limits: 15 fields in the storage's word, F(k) FLOP per
            # point) with the measured HBM bandwidth and the FP32 peak at the
            # maximum SM clock: the roof the paper would predict
            k = order + 1
            word = 4 if st == "f32" else 2
            model_roof = opmodel.roofline(opmodel.oi("tti", k, word), hbm, opmodel.fp32_peak_gflops()) / \
                opmodel.flops_per_point("tti", k)
            out.setdefault(str(order), {})[st] = {
                "kernel_ms": avg, "gpts": gpts, "achieved_gbs": gpts * bpp,
                "frac_of_measured_hbm": gpts * bpp / hbm,
                "paper_model_roof_gpts": model_roof, "frac_of_paper_model_roof": gpts / model_roof}
    return out


def storage_errors():
    """Relative L2 errors against the FP64 oracle of FP32 / BF16 / FP16
    storage on reduced problems (acoustic 48^3 + 10 sponge, order 8, 150
    steps; TTI 64^3 + 8 sponge, order 8, 150 steps), per field."""
    import numpy as np
    from oracle import oracle as O
    from paper_1608_03984_gb300 import fdwave, synth

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))

    out = {"acoustic": {}, "tti": {}}
    w = synth.two_layer(n=48, nb=10, order=8, nt=150, nrec=16)
    ref = O.acoustic_forward(O.Setup(w.vp, w.h, w.nb, w.order, w.dt), w.src_xyz, w.wavelet,
                             w.nt, w.rec_xyz)
    for st in ("f32", "bf16", "f16"):
        s = fdwave.Solver(w.n, w.h, w.nb, w.order, storage=st)
        s.set_model(w.vp).set_dt(w.dt).set_sources(w.src_xyz, w.wavelet)
        s.set_receivers(w.rec_xyz, w.nt).step(w.nt)
        out["acoustic"][st] = {"traces": rel(s.traces(), ref["traces"]),
                               "u": rel(s.wavefield(0, 0), ref["u"])}
        s.close()
    t = synth.random_tti(n=64, nb=8, order=8, nt=150, nrec_side=8)
    ref = O.tti_forward(O.Setup(t.vp, t.h, t.nb, t.order, t.dt, eps=t.eps, delta=t.delta,
                                theta=t.theta, phi=t.phi), t.src_xyz, t.wavelet, t.nt, t.rec_xyz)
    for st in ("f32", "bf16", "f16"):
        s = fdwave.Solver(t.n, t.h, t.nb, t.order, equation="tti", storage=st)
        s.set_model(t.vp, t.eps, t.delta, t.theta, t.phi).set_dt(t.dt)
        s.set_sources(t.src_xyz, t.wavelet).set_receivers(t.rec_xyz, t.nt).step(t.nt)
        out["tti"][st] = {"traces": rel(s.traces(), ref["traces"]), "p": rel(s.wavefield(0, 0), ref["p"]),
                          "r": rel(s.wavefield(1, 0), ref["r"])}
        s.close()
    out["problems"] = ("acoustic two-layer 48^3 + 10 sponge, order 8, 150 steps; "
                       "TTI random 64^3 + 8 sponge, order 8, 150 steps; relative L2 vs FP64 oracle")
    return out


def run_storage(args, base, stream, fp32_kernel_ms, steps, warmup):
    """16-bit storage (BF16 / FP16, FP32 arithmetic) of the acoustic step on
    the 592^3 workload at every order of the sweep: kernel time and speedup
    over FP32 (8 B per point instead of 16)."""
    import torch
    from paper_1608_03984_gb300 import fdwave
    hbm, _ = peaks()
    out = {}
    for o in sorted(fp32_kernel_ms):
        if o not in fp32_kernel_ms:
            continue
        for st in ("bf16", "f16"):
            s = fdwave.Solver(base.n, base.h, base.nb, o, storage=st, stream=stream)
            s.set_model(base.vp).set_dt(base.dt).set_sources(base.src_xyz, base.wavelet)
            s.set_receivers(base.rec_xyz, steps + warmup + 2)
            s.step(warmup)
            torch.cuda.synchronize()
            s.profile_begin(steps)
            s.step(steps)
            ms, n = s.profile_end()
            s.check()
            s.close()
            avg = ms / max(n, 1)
            gpts = base.points / (avg / 1e3) / 1e9
            out.setdefault(str(o), {})[st] = {
                "kernel_ms": avg, "gpts": gpts, "speedup_vs_f32": fp32_kernel_ms[o] / avg,
                "achieved_gbs": gpts * 8, "frac_of_measured_hbm": gpts * 8 / hbm}
    out["errors_vs_fp64_oracle"] = storage_errors()
    return out


def run_fwi(args):
    """FWI gradient wall time: 256^3 + 40-point sponge (336^3), h = 15 m,
    order 8, 2000 steps, 4 x 4 shots, 128 x 128 receivers, 20 checkpoints
    per shot: observed data from the true model (untimed), then the misfit
    and its velocity gradient for all shots from the starting model (timed:
    forward runs, checkpoint replays, adjoint runs, gradient reductions)."""
    import torch
    from paper_1608_03984_gb300 import fwi, synth
    w = synth.fwi(n=args.fwi_n, nt=args.fwi_nt, shots_side=args.fwi_shots_side)
    vref = 1.1 * float(max(w.v_true.max(), w.v_start.max()))
    sv = fwi.Survey(w.n, w.h, w.nb, w.order, w.dt, w.nt, w.src_xyz, w.wavelet, w.rec_xyz,
                    checkpoints=w.checkpoints, sponge_vref=vref)
    with torch.no_grad():
        d_obs = fwi.fwi_traces(torch.from_numpy(w.v_true).cuda(), sv)
    v0 = torch.from_numpy(w.v_start).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, g = fwi.misfit_and_gradient(v0, sv, d_obs)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    nz, ny, nx = (k + 2 * w.nb for k in w.n)
    pts = nz * ny * nx
    nshot = sv.nshot
    # stencil steps per shot: forward + replay + adjoint
    return {"workload": "fwi %d^3 + %d-point sponge (%d^3), h=15 m, order 8, %d steps, %d shots, "
                        "%d receivers, %d checkpoints/shot" % (w.n[0], w.nb, nz, w.nt, nshot,
                                                                w.rec_xyz.shape[0], w.checkpoints),
            "gradient_s": sec, "per_shot_s": sec / nshot, "shots": nshot, "misfit": float(J),
            "stencil_steps": 3 * w.nt * nshot,
            "gpts_equiv": 3 * w.nt * nshot * pts / sec / 1e9,
            "gradient_finite": bool(torch.isfinite(g).all())}


EVERIES = (1, 2, 4, 8, 16)  # closure on every e-th step (correction times e)


def operating_point(field_err_1, ms, sub, val=None):
    """Largest k of `sub` (every-k results) whose mean field error is within
    5% of the every-step closure's (field_err_1); k = 1 if none. With `val`
    ({"closure": e1, "every": {k: e}, "label": ...}: mean field errors on
    separate validation models) k is chosen on those, and the evaluation
    models' error and speed-up at that k are reported."""
    if val is None:
        ref, cand = field_err_1, {k: sub[k]["error_vs_fine"]["field"] for k in sub}
    else:
        ref, cand = val["closure"], val["every"]
    k_best = 1
    for k in sorted(cand, key=int):
        if cand[k] <= 1.05 * ref and int(k) > k_best and str(int(k)) in sub:
            k_best = int(k)
    if k_best == 1:
        best = {"every": 1, "field_error": field_err_1, "speedup_vs_fine": ms["fine"] / ms["closure"]}
    else:
        r = sub[str(k_best)]
        best = {"every": k_best, "field_error": r["error_vs_fine"]["field"], "speedup_vs_fine": r["speedup_vs_fine"]}
    best["selected_on"] = "evaluation models" if val is None else val["label"]
    return best


def run_closure(args):
    """The learned closure: fine order 16 at h = 10 m vs coarse order 4 at
    h = 20 m (coarse point i = fine point 2i, dt_c = 2 dt_f), 10 Hz Ricker
    at the centre. Trained (library kernels) on restricted fine runs of
    64 random models of the same spacing and statistics at a smaller size
    (the network is local: 7^3 receptive field), evaluated on 16 held-out
    models at full size: relative L2 error against the restricted fine run
    with and without the closure, and device time of each run (CUDA
    events)."""
    import numpy as np
    import torch
    from paper_1608_03984_gb300 import closure as C, fdwave
    tr = C.Pairing(n_c=args.closure_train_n, nb_c=8, src_sigma=1.5)
    nt_tr = tr.steps_to_cross(0.45)
    t0 = time.perf_counter()
    gen = torch.Generator(device="cuda").manual_seed(11)
    bank = C.PatchBank()
    for seed in range(5000, 5000 + args.closure_models):
        x, t = C.samples(tr, seed, nt_tr, stride=2)
        bank.add(C.PatchSampler(x, t, P=12, nb=tr.nb_c), args.closure_patches, gen)
        del x, t
    bank.freeze()
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net = fdwave.Closure()
    losses = C.train(net, [bank], iters=args.closure_iters, batch=32, lr=3e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    held = C.PatchSampler(*C.samples(tr, 6000, nt_tr, stride=2), P=12, nb=tr.nb_c)
    unexpl = {"train": C.unexplained(net, bank), "held_out": C.unexplained(net, held)}
    del bank, held
    torch.cuda.empty_cache()
    pr = C.Pairing(n_c=args.closure_n, nb_c=20, src_sigma=1.5)
    nt = pr.steps_to_cross(0.45)
    evals = []
    for seed in range(5064, 5064 + args.closure_eval):
        evals.append(C.evaluate(pr, net, seed, nt, timing=True, everies=EVERIES))
    # the operating point's k is chosen on two further models (seeds after
    # the evaluation ones), not on the models whose errors are reported
    vseeds = (5064 + args.closure_eval, 5065 + args.closure_eval)
    vals = [C.evaluate(pr, net, seed, nt, everies=EVERIES) for seed in vseeds]
    net.close()
    val = {"closure": float(np.mean([r["closure"]["field"] for r in vals])),
           "every": {str(e): float(np.mean([r["closure_every%d" % e]["field"] for r in vals]))
                     for e in EVERIES[1:]},
           "label": "validation models %d, %d" % vseeds}
    ms = {k: float(np.mean([r["ms"][k] for r in evals])) for k in evals[0]["ms"]}
    # the closure on every e-th step with the correction times e: 1/e of the
    # network's cost per unit of time
    sub = {}
    for e in EVERIES[1:]:
        key = "closure_every%d" % e
        sub[str(e)] = {
            "error_vs_fine": {k: float(np.mean([r[key][k] for r in evals])) for k in ("field", "traces")},
            "models_improved": {k: int(sum(r[key][k] < r["coarse"][k] for r in evals)) for k in ("field", "traces")},
            "median_error_ratio": {k: float(np.median([r[key][k] / r["coarse"][k] for r in evals]))
                                   for k in ("field", "traces")},
            "traces_400m": float(np.mean([r[key]["traces_by_depth"][20] for r in evals])),
            "ms": ms[key], "speedup_vs_fine": ms["fine"] / ms[key]}
    err = {m: {k: float(np.mean([r[m][k] for r in evals])) for k in ("field", "traces")}
           for m in ("coarse", "closure")}
    better = {k: int(sum(r["closure"][k] < r["coarse"][k] for r in evals)) for k in ("field", "traces")}
    # per-model error ratios (closure / coarse): the median is not moved by one bad model
    ratio = {k: float(np.median([r["closure"][k] / r["coarse"][k] for r in evals])) for k in ("field", "traces")}
    depths = sorted(evals[0]["coarse"]["traces_by_depth"])
    by_depth = {str(dep): {m: float(np.mean([r[m]["traces_by_depth"][dep] for r in evals]))
                           for m in ("coarse", "closure")} for dep in depths}
    for dep in depths:
        by_depth[str(dep)]["median_ratio"] = float(np.median(
            [r["closure"]["traces_by_depth"][dep] / r["coarse"]["traces_by_depth"][dep] for r in evals]))
        by_depth[str(dep)]["models_improved"] = int(sum(
            r["closure"]["traces_by_depth"][dep] < r["coarse"]["traces_by_depth"][dep] for r in evals))
    k1 = pr.source_steps()
    return {"workload": "fine %d^3 + %d-pt sponge h=%g order %d, %d steps; coarse %d^3 + %d-pt sponge "
                        "h=%g order %d, %d steps (closure after step %d); %d held-out models; trained "
                        "on %d models of %d^3 coarse points (%d patches each)" % (
                            pr.n_f, pr.nb_f, pr.h_f, pr.order_f, 2 * nt, pr.n_c, pr.nb_c, pr.h_c,
                            pr.order_c, nt, k1, args.closure_eval, args.closure_models, tr.n_c,
                            args.closure_patches),
            "error_vs_fine": err, "models_improved": better, "median_error_ratio": ratio,
            "traces_by_depth_m": {str(int(d) * int(pr.h_c)): v for d, v in by_depth.items()}, "ms": ms,
            "speedup_vs_fine": {"coarse": ms["fine"] / ms["coarse"], "closure": ms["fine"] / ms["closure"]},
            "closure_ms_per_step": (ms["closure"] - ms["coarse"] * k1 / nt) / (nt - k1),
            "coarse_ms_per_step": ms["coarse"] / nt,
            "inference": "tcgen05.mma kind::f16 (M = 128 points, N = 48 / 32, K = 16; FP16 operands, FP32 "
                         "accumulators in tensor memory)",
            "one_step_unexplained": unexpl, "train_loss_first_last": [losses[0], losses[-1]],
            "data_s": t1 - t0, "train_s": t2 - t1, "iters": args.closure_iters,
            "every_k_steps": sub,
            # the largest k whose mean field error stays within 5% of the
            # every-step closure's on the validation models: the speed-up and
            # the evaluation models' error at that k
            "operating_point": operating_point(err["closure"]["field"], ms, sub, val),
            "validation": val,
            "per_model": [{k: v for k, v in r.items() if k != "ms"} for r in evals]}


HEADLINE_MAX_BYTES = 4096  # the summary line stays short enough to be read whole


def _r(x, nd=4):
    """Round to nd significant digits (None stays None)."""
    if x is None:
        return None
    return float("%.*g" % (nd, x))


def headline(full, details_path):
    """The printed JSON line: the headline metric with its roofline, e2e,
    CPU baseline and clocks, plus one short summary per further section; the
    sections themselves go to the details file."""
    keep = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "cpu_baseline",
            "clocks", "gpu_launches")
    line = {k: full.get(k) for k in keep}
    if line["e2e"]:
        line["e2e"] = {k: v for k, v in line["e2e"].items() if k != "note"}
    line["per_order"] = {o: {"kernel_ms": _r(v["kernel_ms"]), "gpts": _r(v["kernel_gpts"]),
                             "frac_of_measured_hbm": _r(v["frac_of_measured_hbm"])}
                         for o, v in (full.get("per_order") or {}).items()}
    summ = {}
    tti = full.get("tti")
    if tti:
        summ["tti"] = {o: {st: {"gpts": _r(v["gpts"]), "frac": _r(v["frac_of_measured_hbm"]),
                                "frac_model": _r(v.get("frac_of_paper_model_roof"), 3)}
                           for st, v in tti[o].items()} for o in tti if o.isdigit()}
    st = full.get("storage")
    if st:
        summ["storage_speedup_vs_f32"] = {o: {k: _r(v["speedup_vs_f32"]) for k, v in st[o].items()}
                                          for o in st if o.isdigit()}
        er = st.get("errors_vs_fp64_oracle") or {}
        summ["storage_error_vs_fp64"] = {eq: {sto: {f: _r(x, 3) for f, x in v.items()} for sto, v in er[eq].items()}
                                         for eq in ("acoustic", "tti") if eq in er}
    fw = full.get("fwi")
    if fw:
        summ["fwi"] = {"gradient_s": _r(fw["gradient_s"]), "per_shot_s": _r(fw["per_shot_s"]),
                       "shots": fw["shots"]}
    cl = full.get("closure")
    if cl:
        summ["closure"] = {
            "field_error_vs_fine": {m: _r(v["field"]) for m, v in cl["error_vs_fine"].items()},
            "speedup_vs_fine_every_step": _r(cl["speedup_vs_fine"]["closure"]),
            "operating_point": {k: (_r(v) if not isinstance(v, str) else v)
                                for k, v in cl["operating_point"].items()}}
    c1 = full.get("config1")
    if c1:
        summ["config1"] = {"gpts": _r(c1["gpts"]), "ms_per_run": _r(c1["ms_per_run"])}
    line["sections"] = summ
    line["details"] = os.path.basename(details_path)
    return line


def run_config1(stream, reps=5):
    """The two-layer 64^3 workload (+ 10-point sponge = 84^3, order 4, 200
    steps, 32 receivers) through the CUDA-graph time loop: launch-bound, so
    this is the per-step overhead figure. Gpts/s over the 200-step run
    (CUDA events, mean of `reps` runs after one warm-up run)."""
    import torch
    from paper_1608_03984_gb300 import fdwave, synth
    w = synth.two_layer()
    s = fdwave.Solver(w.n, w.h, w.nb, w.order, stream=stream)
    s.set_model(w.vp).set_dt(w.dt).set_sources(w.src_xyz, w.wavelet).set_receivers(w.rec_xyz, w.nt)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    times = []
    for rep in range(reps + 1):
        s.reset()
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(w.nt)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep:
            times.append(e0.elapsed_time(e1))
    s.check()
    s.close()
    ms = sum(times) / len(times)
    nz, ny, nx = (k + 2 * w.nb for k in w.n)
    return {"workload": "two_layer %d^3 + %d-point sponge (%d^3), order %d, %d steps, %d receivers"
                        % (w.n[0], w.nb, nz, w.order, w.nt, w.rec_xyz.shape[0]),
            "ms_per_run": ms, "us_per_step": 1e3 * ms / w.nt,
            "gpts": nz * ny * nx * w.nt / (ms / 1e3) / 1e9}


def run_e2e(args, orders, base, stream):
    """The same sweep through the public API from pinned host buffers: per
    order, upload the model, sources, receivers, run the steps, read the
    traces back. Host<->device copies are inside the timed region."""
    import torch
    from paper_1608_03984_gb300 import fdwave
    vp_h = torch.from_numpy(base.vp).pin_memory()
    w_h = torch.from_numpy(base.wavelet).pin_memory()
    nsteps = args.steps
    total = 0.0
    h2d = d2h = 0
    tr = torch.empty((nsteps + 1, base.rec_xyz.shape[0]), dtype=torch.float64).pin_memory()
    for o in orders:
        s = fdwave.Solver(base.n, base.h, base.nb, o, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_model(vp_h).set_dt(base.dt).set_sources(base.src_xyz, w_h)
        s.set_receivers(base.rec_xyz, nsteps)
        s.step(nsteps)
        s.traces(out=tr)  # into pinned host memory
        total += time.perf_counter() - t0
        h2d += vp_h.numel() * 4 + w_h.numel() * 4 + base.src_xyz.nbytes + base.rec_xyz.nbytes
        d2h += tr.numel() * tr.element_size()
        s.close()
    world, _, _ = dist_setup()
    total = max_over_ranks(total, device="cuda")  # the slowest rank's wall clock
    pts = base.points * len(orders) * nsteps
    return {"value": whole_job_rate(pts, world, total * 1e3), "unit": "Gpts/s",
            "h2d_bytes_per_step": h2d // nsteps,
            "d2h_bytes_per_step": d2h // nsteps,
            "note": "per order: model/sources/receivers uploaded from pinned host memory, "
                    "%d steps, traces read back; wall clock" % nsteps}


def profile_closure_step(n, variant=0):
    """A small, fixed closure case for kernel profiling (not a measurement)."""
    import torch
    from paper_1608_03984_gb300 import closure as C, fdwave
    torch.cuda.set_device(0)
    pr = C.Pairing(n_c=n, nb_c=20, src_sigma=1.5)
    v_f, v_c, src = C.model(pr, 5064)
    cs = C.coarse_solver(pr, v_c, src, 100)
    net = fdwave.Closure()
    net.set_variant(variant)
    net.set_params(C.init_params(0, last_scale=0.3))
    cs.step(40)
    cs.step_closure(net, 2)
    torch.cuda.synchronize()
    net.close()
    cs.close()
    print("closure step case done")


def main():
    args = parse()
    if args.profile_closure_step:
        profile_closure_step(args.profile_closure_step, args.profile_closure_variant)
        return
    orders = tuple(int(x) for x in args.orders.split(","))
    if args.impl == "reference":
        run_reference(args, orders)
    else:
        run_fdwave(args, orders)


if __name__ == "__main__":
    main()
