"""Benchmark: GF(2)[x] products on GB300 through the C ABI.

Default workload: one product of two seeded uniform-random 2^24-bit
polynomials per step (the 2^24 x 2^24 configuration); ``--config 1`` / ``3``
select 2^16 x 2^16 and 2^30 x 2^30.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gf2x|reference]

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the stream the library launches on; before every timed step a 256 MiB
buffer (larger than the 129 MB L2) is written, outside the events, to flush
L2.  Barrier + synchronize on both sides, max over ranks.  Per-stage times
come from the library's own event pairs (gf2x_profile_*), recorded inside the
same timed region.  ``e2e`` repeats the metric through gf2x_mul_host with
pinned host operands (host<->device copies inside the timed region).

Multi-GPU: the path is one product per GPU with no exchange between GPUs, so
N ranks run N independent replicas (weak scaling); there is no collective on
the data path, only the barrier and the max-time reduction.

``--impl reference`` times the CPU oracle (portable C Karatsuba, OpenMP) on
the host cores for the same workload and metric.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

CONFIGS = {
    1: dict(na=1 << 16, nb=1 << 16, name="single product 2^16 x 2^16 bits, uniform random"),
    2: dict(na=1 << 24, nb=1 << 24, name="single product 2^24 x 2^24 bits, uniform random"),
    3: dict(na=1 << 30, nb=1 << 30, name="single product 2^30 x 2^30 bits, uniform random"),
}
METRIC = "operand Gbit/s (na+nb bits per product / time)"
UNIT = "Gbit/s"
L2_FLUSH_BYTES = 256 << 20

# Measured peaks (MEASURED_PEAKS.json is written on the GPU machine; these are its values).
HBM_PEAK_GBS_FALLBACK = 6784.5
SM_MAX_MHZ_FALLBACK = 2070.0
NUM_SMS = 152

# GF(2^64)-product roofline: one butterfly = one product (+2 XORs).  The
# fastest product form measured here (16 four-bit windows of a per-twiddle
# table in shared memory, 16 x 8 B = 128 B per product) is bound by the
# shared-memory port, 128 B per SM-clock: at most 1 product per SM per clock.
PRODUCTS_PER_SM_CLOCK = 1.0
BOTTOM_LAYERS = 11            # low layers done by the fused bottom kernel

# ncu dram bytes per launch of the dominant kernel, from profiles/ (None when
# the kernel changed since the capture).
TRAFFIC_BYTES_PER_LAUNCH = None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_PEAK_GBS_FALLBACK)), float(d.get("sm_max_mhz", SM_MAX_MHZ_FALLBACK)), "measured"
    except Exception:
        return HBM_PEAK_GBS_FALLBACK, SM_MAX_MHZ_FALLBACK, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
            self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ distributed
def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def dist_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------- CPU oracle
def oracle_sample(na: int, nb: int, budget_s: float = 20.0, max_products: int = 4):
    """Time the CPU oracle on whole products of the workload until ~budget_s."""
    from oracle import clmul as O
    O.build()
    done, t0 = 0, time.perf_counter()
    elapsed = 0.0
    while done < max_products:
        a = synth.operand(synth.config_seed(50, 2 * done), na)
        b = synth.operand(synth.config_seed(50, 2 * done + 1), nb)
        t = time.perf_counter()
        O.mul(a, na, b, nb)
        elapsed += time.perf_counter() - t
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return done, elapsed, O.num_threads()


def scaled_oracle_workload(na, nb):
    """The oracle finishes 2^24 x 2^24 in seconds; at 2^30 it cannot, so it is
    timed on 2^24 x 2^24 products and reported per operand bit."""
    if na * nb > (1 << 48):
        return 1 << 24, 1 << 24
    return na, nb


def run_reference(args, world, rank):
    if rank != 0:
        return
    cfg = CONFIGS[args.config]
    na, nb = scaled_oracle_workload(cfg["na"], cfg["nb"])
    from oracle import clmul as O
    O.build()
    for i in range(args.warmup):
        a = synth.operand(synth.config_seed(51, 2 * i), na)
        b = synth.operand(synth.config_seed(51, 2 * i + 1), nb)
        O.mul(a, na, b, nb)
    times = []
    for i in range(args.steps):
        a = synth.operand(synth.config_seed(52, 2 * i), na)
        b = synth.operand(synth.config_seed(52, 2 * i + 1), nb)
        t = time.perf_counter()
        O.mul(a, na, b, nb)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = (na + nb) * args.steps / total / 1e9
    sample = (f"{args.steps} whole products of {na}x{nb} bits" +
              ("" if (na, nb) == (cfg["na"], cfg["nb"]) else f" (the {cfg['na']}x{cfg['nb']} workload scaled per operand bit)"))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": cfg["name"], "na_bits": cfg["na"], "nb_bits": cfg["nb"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def stage_work(stage, na, nb, n, products, square=False):
    """Algorithmic work of one stage over `products` products: (amount, kind).

    kind "mul": GF(2^64) products (one per butterfly); kind "hbm": bytes."""
    l = n.bit_length() - 1 - 6
    n_p = 1 << l
    bt = min(BOTTOM_LAYERS, l)
    fw = 1 if square else 2
    la = max(64, 1 << max(0, (na - 1).bit_length()))
    lb = max(64, 1 << max(0, (nb - 1).bit_length()))
    if stage == "butterfly":       # top layers of the forward transforms
        return products * fw * (l - bt) * (n_p // 2), "mul"
    if stage == "ibutterfly":      # top layers of the inverse
        return products * (l - bt) * (n_p // 2), "mul"
    if stage == "bottom_fused":    # low layers: forward x fw, pointwise, inverse
        return products * ((fw + 1) * bt * (n_p // 2) + n_p), "mul"
    if stage == "pointwise":
        return products * n_p, "mul"
    if stage == "basis_cvt":       # read + write each operand's L bits once
        return products * 2 * (la + (0 if square else lb)) // 8, "hbm"
    if stage == "ibasis_cvt":
        return products * 2 * n // 8, "hbm"
    if stage == "encode":          # read n bits, write n_p words, per operand
        return products * fw * 2 * n // 8, "hbm"
    if stage == "decode":
        return products * 2 * n // 8, "hbm"
    if stage == "load":
        return products * ((na + 7) // 8 + n // 8 + (0 if square else (nb + 7) // 8 + n // 8)), "hbm"
    if stage == "store":
        nc = na + nb - 1
        return products * 2 * ((nc + 63) // 64) * 8, "hbm"
    return 0, "hbm"


def run_gpu(args, world, rank, local):
    import torch
    from paper_1803_11301_gb300 import Context, build as lib_build
    lib_build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = CONFIGS[args.config]
    na, nb = cfg["na"], cfg["nb"]
    nc = na + nb - 1
    ctx = Context(local)
    stream = torch.cuda.current_stream(dev)
    seed = synth.config_seed(args.config, 1000 + 17 * rank)
    a_h = synth.operand(seed, na)
    b_h = synth.operand(seed + 1, nb)
    a = torch.from_numpy(a_h.view(np.int64)).to(dev)
    b = torch.from_numpy(b_h.view(np.int64)).to(dev)
    c = torch.empty((nc + 63) // 64, dtype=torch.int64, device=dev)
    from paper_1803_11301_gb300 import workspace_bytes, host_workspace_bytes
    ws = torch.empty(max(workspace_bytes(na, nb), host_workspace_bytes(na, nb)), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step():
        ctx.mul(a, na, b, nb, out=c, workspace=ws, stream=stream)

    # profiling on from the first warm-up step: the library captures its CUDA
    # graph (with the stage event nodes) on the second call with these buffers
    ctx.profile_enable(True)
    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ctx.profile_enable(True)                     # reset stage times and launch counts
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    dist_barrier(world)
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.fill_(k)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
        prof = ctx.profile_read()                # waits for this step; outside the events
    torch.cuda.synchronize(dev)
    dist_barrier(world)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    clk = clocks.stop()
    ms_steps = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = dist_max(sum(ms_steps), world)
    value = world * (na + nb) * args.steps / (total_ms / 1e3) / 1e9
    launches = sum(v[1] for v in prof.values())

    # end to end: host operands through gf2x_mul_host (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        a_pin = torch.from_numpy(a_h.view(np.int64)).pin_memory()
        b_pin = torch.from_numpy(b_h.view(np.int64)).pin_memory()
        c_pin = torch.empty((nc + 63) // 64, dtype=torch.int64).pin_memory()
        an, bn, cn = (t.numpy().view(np.uint64) for t in (a_pin, b_pin, c_pin))
        for _ in range(max(1, args.warmup)):
            ctx.mul_host(an, na, bn, nb, out=cn, workspace=ws, stream=stream)
        e2e_times = []
        dist_barrier(world)
        for k in range(args.steps):
            flush.fill_(k)
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            ctx.mul_host(an, na, bn, nb, out=cn, workspace=ws, stream=stream)   # synchronous
            e2e_times.append(time.perf_counter() - t)
        e2e_total = dist_max(sum(e2e_times), world)
        h2d = ((na + 63) // 64 + (nb + 63) // 64) * 8
        d2h = ((nc + 63) // 64) * 8
        e2e = {"value": world * (na + nb) * args.steps / e2e_total / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_total / args.steps}
        if not np.array_equal(cn, c.cpu().numpy().view(np.uint64)):
            raise RuntimeError("e2e product differs from the device-resident product")

    # roofline of the dominant stage
    hbm_peak, sm_max_mhz, peak_src = load_peaks()
    n = 1 << max(6, (nc - 1).bit_length())
    stages = {}
    for name, (ms, nl) in prof.items():
        work, kind = stage_work(name, na, nb, n, args.steps)
        stages[name] = {"ms": ms / args.steps, "launches_per_step": nl / args.steps, "bound": kind,
                        "work_per_step": work / args.steps}
    dom = max(stages, key=lambda k: stages[k]["ms"])
    d = stages[dom]
    if d["bound"] == "mul":
        achieved = d["work_per_step"] / (d["ms"] / 1e3) / 1e9
        peak = NUM_SMS * PRODUCTS_PER_SM_CLOCK * sm_max_mhz * 1e6 / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gmul/s", "frac": achieved / peak,
                "peak_source": (f"derived: {NUM_SMS} SMs x {sm_max_mhz:.0f} MHz x {PRODUCTS_PER_SM_CLOCK:g} GF(2^64) "
                                "product per SM-clock (shared-memory port bound of the table product)"),
                "traffic": TRAFFIC_BYTES_PER_LAUNCH, "kernel_stage": dom,
                "avg_launch_us": 1e3 * d["ms"] / max(d["launches_per_step"], 1)}
    else:
        achieved = d["work_per_step"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": f"{peak_src} copy bandwidth", "traffic": TRAFFIC_BYTES_PER_LAUNCH, "kernel_stage": dom,
                "avg_launch_us": 1e3 * d["ms"] / max(d["launches_per_step"], 1)}

    compulsory = ((na + 63) // 64 + (nb + 63) // 64 + (nc + 63) // 64) * 8
    ms_per_step = total_ms / args.steps
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "us_per_product": 1e3 * ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": cfg["name"], "na_bits": na, "nb_bits": nb, "transform_bits": n,
                       "l2": "flushed before every timed step (256 MiB write)",
                       "parallelism": f"{world} independent replica(s)"},
            "hbm_compulsory": {"bytes_per_product": compulsory,
                               "frac": compulsory / (ms_per_step / 1e3) / 1e9 / hbm_peak},
            "roofline": roof, "stages_ms": {k: round(v["ms"], 4) for k, v in stages.items()},
            "gpu_launches": int(launches), "clocks": clk, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ona, onb = scaled_oracle_workload(na, nb)
        done, el, cores = oracle_sample(ona, onb)
        line["cpu_baseline"] = {"value": (ona + onb) * done / el / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{done} whole {ona}x{onb}-bit products, portable C Karatsuba, OpenMP"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_stage(args):
    """One stage of Alg. 5 on its own, through its C-ABI entry point (for profiling)."""
    import torch
    from paper_1803_11301_gb300 import Context, build as lib_build
    lib_build.build()
    ctx = Context(0)
    n = 64 << args.log2_points
    x = torch.from_numpy(synth.splitmix64(7, n // 64).view(np.int64)).cuda()
    y = torch.empty_like(x)
    fns = {
        "butterfly": lambda: ctx.butterfly(x, n),
        "ibutterfly": lambda: ctx.ibutterfly(x, n),
        "basis_cvt": lambda: ctx.basis_cvt(x, n),
        "ibasis_cvt": lambda: ctx.ibasis_cvt(x, n),
        "encode": lambda: ctx.encode(x, n, out=y),
        "decode": lambda: ctx.decode(x, n, out=y),
        "pointwise": lambda: ctx.pointwise(x, x, out=y),
    }
    fn = fns[args.stage]
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    for _ in range(args.steps):
        fn()
    prof = ctx.profile_read()
    ms, launches = prof[args.stage]
    print(json.dumps({"stage": args.stage, "points": n // 64, "transform_bits": n, "steps": args.steps,
                      "ms_per_call": ms / args.steps, "launches_per_call": launches / args.steps}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gf2x", choices=["gf2x", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=sorted(CONFIGS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stage", default=None,
                    choices=["butterfly", "ibutterfly", "basis_cvt", "ibasis_cvt", "encode", "decode", "pointwise"],
                    help="time one stage alone through its entry point (profiling aid)")
    ap.add_argument("--log2-points", type=int, default=24, help="n_p = 2^this GF(2^64) points for --stage")
    args = ap.parse_args()
    if args.stage:
        run_stage(args)
        return
    if args.warmup < 3 and args.impl == "gf2x":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    world, rank, local = dist_setup(args.gpus)
    run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
