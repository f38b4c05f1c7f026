"""Benchmark: GF(2)[x] products on GB300 through the C ABI.

Default workload: one product of two seeded uniform-random 2^30-bit
polynomials per step (the 2^30 x 2^30 configuration, the largest single
product of the workload list); ``--config 1`` / ``2`` select 2^16 x 2^16 and
2^24 x 2^24.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gf2x|reference]

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the stream the library launches on; before every timed step a 256 MiB
buffer (larger than the 129 MB L2) is written, outside the events, to flush
L2.  Barrier + synchronize on both sides, max over ranks.  ``value`` comes
from a plain timed region; a second timed region of K steps, identical but
with the library's per-stage event pairs (gf2x_profile_*) in its CUDA graph,
gives the stage times, the launch count and the roofline of the dominant
kernel (its cost is reported as ``profiled_ms_per_step``).  ``e2e`` repeats the metric through gf2x_mul_host with
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
    4: dict(name="4096 independent products, operand lengths log-uniform in [2^10, 2^20] bits, a and b drawn "
                 "independently, uniform random bits, one gf2x_mul_batch call per step"),
    5: dict(name="serving: Poisson arrivals of products, operand lengths log-uniform in [2^12, 2^26] bits, "
                 "5% with one operand of exactly 2^28 bits, continuous batching over 3 streams"),
    6: dict(na=1 << 24, nb=1 << 24, name="reused operand: 2^24 x 2^24-bit products a_k * b with one fixed b, "
                                        "b's transform computed once (gf2x_forward_transform) outside the timing"),
    7: dict(na=1 << 24, nb=1 << 24, field=128,
            name="single product 2^24 x 2^24 bits, uniform random, GF(2^128) points (gf2x_mul_m128)"),
    8: dict(na=1 << 30, nb=1 << 30, field=128,
            name="single product 2^30 x 2^30 bits, uniform random, GF(2^128) points (gf2x_mul_m128)"),
}
METRIC = "operand Gbit/s (na+nb bits per product / time)"
UNIT = "Gbit/s"
L2_FLUSH_BYTES = 256 << 20

# Peaks measured on GB300 (the copy bandwidth and SM clock of MEASURED_PEAKS.json; used when it is absent).
HBM_PEAK_GBS_FALLBACK = 6784.5
SM_MAX_MHZ_FALLBACK = 2070.0
NUM_SMS = 152

# GF(2^64)-product roofline: one butterfly = one product (+2 XORs).  The
# fastest product form measured here (16 four-bit windows of a per-twiddle
# table in shared memory, 16 x 8 B = 128 B per product) is bound by the
# shared-memory port, 128 B per SM-clock: at most 1 product per SM per clock.
PRODUCTS_PER_SM_CLOCK = 1.0
BOTTOM_LAYERS = 11            # default low layers of the fused bottom kernel (the library reports its choice)
# GF(2^128) points: the table product reads 32 windows x 16 B = 512 B of
# shared memory, so at most 1/4 product per SM per clock; up to 10 bottom layers.
PRODUCTS_PER_SM_CLOCK_128 = 0.25
BOTTOM_LAYERS_128 = 10

# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of a stage's
# kernel, keyed by (stage, na, nb, field bits, bottom layers), from one ncu
# capture of the same workload (the summaries under profiles/ give the
# commands).  Each entry carries the digest of the kernel's sources at capture
# time (comments and blank space stripped, see source_digest): when the
# sources have changed since, the line reports traffic null and says so.
KERNEL_SOURCES = {64: ["paper_1803_11301_gb300/csrc/bfly.cu", "paper_1803_11301_gb300/csrc/bfly_dev.cuh",
                       "paper_1803_11301_gb300/csrc/gf2x_tables.cuh", "paper_1803_11301_gb300/csrc/gf2x_common.cuh"],
                  128: ["paper_1803_11301_gb300/csrc/m128.cu", "paper_1803_11301_gb300/csrc/gf2x_common.cuh"]}
TRAFFIC_BYTES_PER_LAUNCH = {     # (stage, na, nb, field bits, bottom layers): (bytes, source digest)
    ("bottom_fused", 1 << 24, 1 << 24, 64, 11): (8482048 + 768, "8b7f8352c7915a71"),
    ("bottom_fused", 1 << 24, 1 << 24, 128, 9): (8484096 + 0, "07457971a17da7e1"),
    ("bottom_fused", 1 << 30, 1 << 30, 64, 11): (537438208 + 224828928, "8b7f8352c7915a71"),
    ("bottom_fused", 1 << 30, 1 << 30, 128, 10): (539217408 + 224975360, "07457971a17da7e1"),
}


def source_digest(field: int) -> str:
    """Digest of the dominant kernel's sources, comments and blank space removed."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[field]:
        with open(os.path.join(ROOT, rel)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(re.sub(r"\s+", "", text).encode())
    return h.hexdigest()[:16]


def traffic_entry(key, field: int):
    """(bytes per launch or None, note) for the roofline's traffic field."""
    ent = TRAFFIC_BYTES_PER_LAUNCH.get(key)
    if ent is None:
        return None, "no ncu capture of this kernel at this workload"
    nbytes, digest = ent
    if digest != source_digest(field):
        return None, "stale: the kernel's sources changed since the ncu capture"
    return nbytes, "ncu dram__bytes_read.sum + dram__bytes_write.sum, one capture of this workload"


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
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="gf2x_clocks_", suffix=".csv")
            os.close(fd)
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
# Multi-GPU: replicas only.  Each rank multiplies its own operands (its own
# seed); the only cross-rank calls are a barrier around the timed region and
# the max-reduction of the timed seconds.  backend="gloo" / device="cpu" run
# the same code on CPU processes (tests); the bench uses NCCL on the GPUs.
def dist_setup(n_gpus, backend: str = "nccl"):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def dist_max(x: float, world: int, device: str = "cuda") -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(config: int, rank: int) -> int:
    """Operand seed of a rank: every replica multiplies different operands."""
    return synth.config_seed(config, 1000 + 17 * rank)


def whole_job_value(units_per_rank: float, seconds_max: float, world: int, scale: float = 1e9) -> float:
    """Weak-scaling throughput: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / seconds_max / scale


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


def single_config(args):
    """The configuration of a single-product run, with --log2-bits applied."""
    cfg = dict(CONFIGS[args.config])
    if args.log2_bits is not None and "na" in cfg:
        k = args.log2_bits
        cfg["na"] = cfg["nb"] = 1 << k
        cfg["name"] = f"single product 2^{k} x 2^{k} bits, uniform random" + (
            ", GF(2^128) points (gf2x_mul_m128)" if cfg.get("field") == 128 else "")
    return cfg


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.config == 4:
        return run_reference_batch(args)
    if args.config == 5:
        print(json.dumps({"impl": "reference", "unavailable": "the serving mix has 2^28-bit operands, minutes per "
                          "product for the CPU oracle; the reference arm covers configs 1-4 and 6"}), flush=True)
        return
    cfg = single_config(args)
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


def run_reference_batch(args):
    """The oracle on the batched mix: each step multiplies a bounded sample (256 of the products)."""
    from oracle import clmul as O
    O.build()
    lens = synth.loguniform_lengths(synth.config_seed(4, 100), 2 * args.batch, 10.0, 20.0).reshape(args.batch, 2)
    sample = 256
    def one_step(offset):
        t = 0.0
        for k in range(sample):
            na, nb = int(lens[(offset + k) % args.batch, 0]), int(lens[(offset + k) % args.batch, 1])
            a = synth.operand(synth.config_seed(4, 10000 + 2 * k), na)
            b = synth.operand(synth.config_seed(4, 10001 + 2 * k), nb)
            t0 = time.perf_counter()
            O.mul(a, na, b, nb)
            t += time.perf_counter() - t0
        return t
    for w in range(args.warmup):
        one_step(w * sample)
    total = sum(one_step(s * sample) for s in range(args.steps))
    value = sample * args.steps / total
    line = {"impl": "reference", "metric": "products/s (batched, uneven lengths)", "value": value, "unit": "products/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": CONFIGS[4]["name"], "products": args.batch},
            "cpu_baseline": {"value": value, "unit": "products/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{sample} products of the mix per step"},
            "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def stage_work(stage, na, nb, n, products, field=64, bottom_layers=None):
    """Algorithmic work of one stage over `products` products: (amount, kind).

    kind "mul": GF(2^m) products (one per butterfly); kind "hbm": bytes.
    bottom_layers: Butterfly layers done by the fused low-layer kernel (the
    library's choice, gf2x_bottom_layers); the rest are top passes."""
    l = n.bit_length() - 1 - (7 if field == 128 else 6)
    n_p = 1 << l
    if bottom_layers is None:
        bottom_layers = BOTTOM_LAYERS_128 if field == 128 else BOTTOM_LAYERS
    bt = min(bottom_layers, l)
    fw = 2                         # two forward transforms
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
        return products * 2 * (la + lb) // 8, "hbm"
    if stage == "ibasis_cvt":
        return products * 2 * n // 8, "hbm"
    if stage == "encode":          # read n bits, write n_p words, per operand
        return products * fw * 2 * n // 8, "hbm"
    if stage == "decode":
        return products * 2 * n // 8, "hbm"
    if stage == "load":
        return products * ((na + 7) // 8 + (nb + 7) // 8 + n // 8), "hbm"
    if stage == "store":
        nc = na + nb - 1
        return products * 2 * ((nc + 63) // 64) * 8, "hbm"
    return 0, "hbm"


def whole_product_alu(n, field, ms_per_step, mul_peak):
    """The whole product against the product-rate roofline: Alg. 5 needs
    1.5 l n_p + n_p field products (three transforms of l layers, n_p/2
    butterflies each, and the pointwise step)."""
    l = n.bit_length() - 1 - (7 if field == 128 else 6)
    n_p = 1 << l
    products = 3 * l * (n_p // 2) + n_p
    achieved = products / (ms_per_step / 1e3) / 1e9
    return {"products": products, "achieved": achieved, "peak": mul_peak, "unit": "Gmul/s",
            "frac": achieved / mul_peak}


def run_gpu(args, world, rank, local):
    import torch
    from paper_1803_11301_gb300 import Context, build as lib_build
    lib_build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = single_config(args)
    na, nb = cfg["na"], cfg["nb"]
    field = cfg.get("field", 64)
    nc = na + nb - 1
    ctx = Context(local)
    stream = torch.cuda.current_stream(dev)
    seed = replica_seed(args.config, rank)
    a_h = synth.operand(seed, na)
    b_h = synth.operand(seed + 1, nb)
    a = torch.from_numpy(a_h.view(np.int64)).to(dev)
    b = torch.from_numpy(b_h.view(np.int64)).to(dev)
    c = torch.empty((nc + 63) // 64, dtype=torch.int64, device=dev)
    from paper_1803_11301_gb300 import workspace_bytes, host_workspace_bytes, m128_workspace_bytes
    ws_bytes = m128_workspace_bytes(na, nb) if field == 128 else max(workspace_bytes(na, nb),
                                                                      host_workspace_bytes(na, nb))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    mul = ctx.mul_m128 if field == 128 else ctx.mul

    def step():
        mul(a, na, b, nb, out=c, workspace=ws, stream=stream)

    # Two timed regions of K steps each, both with warm-up, L2 flush and CUDA
    # events on the launching stream: (1) plain, for `value`; (2) with the
    # library's per-stage event nodes in its CUDA graph, for the stage times,
    # the launch count and the roofline of the dominant kernel.
    def timed(profiled):
        ctx.profile_enable(profiled)
        for _ in range(args.warmup):
            flush.fill_(1)
            step()
        torch.cuda.synchronize(dev)
        if profiled:
            ctx.profile_enable(True)             # reset stage times and launch counts
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        dist_barrier(world)
        torch.cuda.synchronize(dev)
        prof = None
        if not profiled:
            torch.cuda.profiler.start()          # `ncu --profile-from-start off` sees this region only
        for k in range(args.steps):
            flush.fill_(k)
            starts[k].record(stream)
            step()
            ends[k].record(stream)
            if profiled:
                prof = ctx.profile_read()        # waits for this step; outside the events
        torch.cuda.synchronize(dev)
        if not profiled:
            torch.cuda.profiler.stop()
        dist_barrier(world)
        if profiled:
            prof = ctx.profile_read()
            ctx.profile_enable(False)
        ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        return dist_max(sum(ms), world), prof

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    total_ms, _ = timed(False)
    prof_total_ms, prof = timed(True)
    clk = clocks.stop()
    value = whole_job_value((na + nb) * args.steps, total_ms / 1e3, world)
    launches = sum(v[1] for v in prof.values())

    # end to end: host operands through gf2x_mul_host (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        a_pin = torch.from_numpy(a_h.view(np.int64)).pin_memory()
        b_pin = torch.from_numpy(b_h.view(np.int64)).pin_memory()
        c_pin = torch.empty((nc + 63) // 64, dtype=torch.int64).pin_memory()
        an, bn, cn = (t.numpy().view(np.uint64) for t in (a_pin, b_pin, c_pin))

        def host_step():
            if field == 128:
                # pinned host operands copied in, gf2x_mul_m128, product copied out, on one stream
                with torch.cuda.stream(stream):
                    a.copy_(a_pin, non_blocking=True)
                    b.copy_(b_pin, non_blocking=True)
                    ctx.mul_m128(a, na, b, nb, out=c, workspace=ws, stream=stream)
                    c_pin.copy_(c, non_blocking=True)
                stream.synchronize()
            else:
                ctx.mul_host(an, na, bn, nb, out=cn, workspace=ws, stream=stream)   # synchronous

        for _ in range(max(1, args.warmup)):
            host_step()
        e2e_times = []
        dist_barrier(world)
        for k in range(args.steps):
            flush.fill_(k)
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            host_step()
            e2e_times.append(time.perf_counter() - t)
        e2e_total = dist_max(sum(e2e_times), world)
        h2d = ((na + 63) // 64 + (nb + 63) // 64) * 8
        d2h = ((nc + 63) // 64) * 8
        e2e = {"value": whole_job_value((na + nb) * args.steps, e2e_total, world), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_total / args.steps}
        if not np.array_equal(cn, c.cpu().numpy().view(np.uint64)):
            raise RuntimeError("e2e product differs from the device-resident product")

    # roofline of the dominant stage
    hbm_peak, sm_max_mhz, peak_src = load_peaks()
    n = 1 << max(7 if field == 128 else 6, (nc - 1).bit_length())
    bottom_layers = ctx.bottom_layers(na, nb, field)
    stages = {}
    for name, (ms, nl) in prof.items():
        work, kind = stage_work(name, na, nb, n, args.steps, field, bottom_layers)
        stages[name] = {"ms": ms / args.steps, "launches_per_step": nl / args.steps, "bound": kind,
                        "work_per_step": work / args.steps}
    dom = max(stages, key=lambda k: stages[k]["ms"])
    d = stages[dom]
    traffic, traffic_note = traffic_entry((dom, na, nb, field, bottom_layers), field)
    per_clock = PRODUCTS_PER_SM_CLOCK_128 if field == 128 else PRODUCTS_PER_SM_CLOCK
    mul_peak = NUM_SMS * per_clock * sm_max_mhz * 1e6 / 1e9
    if d["bound"] == "mul":
        achieved = d["work_per_step"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": mul_peak, "unit": "Gmul/s", "frac": achieved / mul_peak,
                "peak_source": (f"derived: {NUM_SMS} SMs x {sm_max_mhz:.0f} MHz x {per_clock:g} GF(2^{field}) "
                                "product per SM-clock (shared-memory port bound of the table product, "
                                "bench.py --stage field_mul)"),
                "traffic": traffic, "traffic_note": traffic_note, "kernel_stage": dom,
                "avg_launch_us": 1e3 * d["ms"] / max(d["launches_per_step"], 1)}
    else:
        achieved = d["work_per_step"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": f"{peak_src} copy bandwidth", "traffic": traffic, "traffic_note": traffic_note,
                "kernel_stage": dom,
                "avg_launch_us": 1e3 * d["ms"] / max(d["launches_per_step"], 1)}

    compulsory = ((na + 63) // 64 + (nb + 63) // 64 + (nc + 63) // 64) * 8
    ms_per_step = total_ms / args.steps
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "us_per_product": 1e3 * ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": cfg["name"], "na_bits": na, "nb_bits": nb, "transform_bits": n, "field_bits": field,
                       "bottom_layers": bottom_layers,
                       "l2": "flushed before every timed step (256 MiB write)",
                       "parallelism": f"{world} independent replica(s)"},
            "hbm_compulsory": {"bytes_per_product": compulsory,
                               "frac": compulsory / (ms_per_step / 1e3) / 1e9 / hbm_peak,
                               "peak_gbs": hbm_peak, "peak_source": f"{peak_src} copy bandwidth"},
            "alu_whole_product": whole_product_alu(n, field, ms_per_step, mul_peak),
            "roofline": roof, "stages_ms": {k: round(v["ms"], 4) for k, v in stages.items()},
            "profiled_ms_per_step": prof_total_ms / args.steps,
            "gpu_launches": int(launches), "clocks": clk, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ona, onb = scaled_oracle_workload(na, nb)
        done, el, cores = oracle_sample(ona, onb)
        line["cpu_baseline"] = {"value": (ona + onb) * done / el / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{done} whole {ona}x{onb}-bit products, portable C Karatsuba, OpenMP"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_field_mul(args):
    """The GF(2^64) product forms (gf2x_bench_field_mul), each timed on the same
    chains of products by a fixed element; the measurement behind the
    product-rate peak of the roofline (the four-bit-window table form)."""
    import torch
    from paper_1803_11301_gb300 import Context, build as lib_build
    lib_build.build()
    ctx = Context(0)
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    rows = []
    for v in range(len(Context.FIELD_VARIANTS)):
        steps = args.field_steps if Context.FIELD_VARIANTS[v] != "bitslice" else max(1, args.field_steps // 8)
        best = None
        for _ in range(3):
            r = ctx.bench_field_mul(v, steps)
            r["steps"] = steps
            if best is None or r["ms"] < best["ms"]:
                best = r
        rows.append(best)
    clk = clocks.stop()
    mhz = clk.get("sm_mhz") or SM_MAX_MHZ_FALLBACK
    ref = {}                                     # variant 0's checksum per chain length
    for r in rows:
        if r["steps"] not in ref:
            ref[r["steps"]] = ctx.bench_field_mul(0, r["steps"])["checksum"]
        r["gmul_s"] = r["products"] / (r["ms"] / 1e3) / 1e9
        r["mul_per_sm_clock"] = r["gmul_s"] * 1e9 / (NUM_SMS * mhz * 1e6)
        r["checksum_matches_variant0"] = r["checksum"] == ref[r["steps"]]
    torch.cuda.synchronize()
    print(json.dumps({"stage": "field_mul", "what": "dependent chains x <- c x, 4 per thread, 8 blocks of 256 "
                      "threads per SM; products / CUDA-event time of one launch (best of 3)",
                      "variants": rows, "clocks": clk}), flush=True)
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


def make_jobs(ctx, count, lo, hi, seed, dev):
    import torch
    lens = synth.loguniform_lengths(synth.config_seed(4, seed), 2 * count, lo, hi).reshape(count, 2)
    jobs, hosts = [], []
    for k in range(count):
        na, nb = int(lens[k, 0]), int(lens[k, 1])
        a = synth.operand(synth.config_seed(4, 10000 + 2 * k), na)
        b = synth.operand(synth.config_seed(4, 10001 + 2 * k), nb)
        c = torch.empty((na + nb - 1 + 63) // 64, dtype=torch.int64, device=dev)
        jobs.append((torch.from_numpy(a.view(np.int64)).to(dev), na, torch.from_numpy(b.view(np.int64)).to(dev), nb, c))
        hosts.append((a, b))
    return jobs, hosts


def run_batch(args, world, rank, local):
    """Batched products/s (one gf2x_mul_batch per step) vs one gf2x_mul call per product."""
    import torch
    from paper_1803_11301_gb300 import Context, build as lib_build, workspace_bytes
    lib_build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = Context(local)
    stream = torch.cuda.current_stream(dev)
    count = args.batch
    jobs, hosts = make_jobs(ctx, count, 10.0, 20.0, 100 + rank, dev)
    ws = torch.empty(ctx.batch_workspace_bytes(jobs), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    prepared = ctx.prepare_batch(jobs)       # argument marshalling once, outside the timed region
    from paper_1803_11301_gb300 import KNOB_BATCH_PERSISTENT

    def timed_batch(mode):
        """K batch calls: one persistent launch each (mode 1), one launch per kernel and size class (0),
        or the library's choice (None: the tuner times both on the first call)."""
        ctx.tune_pin(KNOB_BATCH_PERSISTENT, -1 if mode is None else mode)
        ctx.profile_enable(True)
        for _ in range(args.warmup):
            flush.fill_(1)
            ctx.mul_batch(prepared, workspace=ws, stream=stream)
        torch.cuda.synchronize(dev)
        ctx.profile_enable(True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        dist_barrier(world)
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.fill_(k)
            starts[k].record(stream)
            ctx.mul_batch(prepared, workspace=ws, stream=stream)
            ends[k].record(stream)
            ctx.profile_read()
        torch.cuda.synchronize(dev)
        dist_barrier(world)
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        ctx.tune_pin(KNOB_BATCH_PERSISTENT, -1)
        return dist_max(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world), prof

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    class_ms, class_prof = timed_batch(0)
    pers_ms, pers_prof = timed_batch(1)
    total_ms, prof = timed_batch(None)
    clk = clocks.stop()
    value = world * count * args.steps / (total_ms / 1e3)
    class_value = world * count * args.steps / (class_ms / 1e3)
    pers_value = world * count * args.steps / (pers_ms / 1e3)
    chose = "persistent" if prof.get("persistent_batch", (0, 0))[1] else "class launches"
    # one gf2x_mul per product (sequential calls on the same stream), one pass after one warm-up pass
    wsp = torch.empty(max(workspace_bytes(j[1], j[3]) for j in jobs), dtype=torch.uint8, device=dev)
    for j in jobs:
        ctx.mul(j[0], j[1], j[2], j[3], out=j[4], workspace=wsp, stream=stream)
    torch.cuda.synchronize(dev)
    flush.fill_(3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for j in jobs:
        ctx.mul(j[0], j[1], j[2], j[3], out=j[4], workspace=wsp, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = dist_max(e0.elapsed_time(e1), world)
    plain = world * count / (plain_ms / 1e3)
    # end to end: the operands of all jobs packed in one pinned host buffer (16-byte aligned
    # slots), one host-to-device copy, the batch on views into the device copy, one
    # device-to-host copy of all results packed the same way, all inside the timed region
    def slots(sizes):
        offs, o = [], 0
        for w in sizes:
            offs.append(o)
            o += (w + 1) // 2 * 2
        return offs, max(o, 2)
    in_words = [(a.size, b.size) for a, b in hosts]
    in_offs, in_total = slots([x for ab in in_words for x in ab])
    out_offs, out_total = slots([j[4].numel() for j in jobs])
    host_in = torch.zeros(in_total, dtype=torch.int64).pin_memory()
    hin = host_in.numpy().view(np.uint64)
    for k, (a, b) in enumerate(hosts):
        hin[in_offs[2 * k]:in_offs[2 * k] + a.size] = a
        hin[in_offs[2 * k + 1]:in_offs[2 * k + 1] + b.size] = b
    host_out = torch.empty(out_total, dtype=torch.int64).pin_memory()
    dev_in = torch.empty(in_total, dtype=torch.int64, device=dev)
    dev_out = torch.empty(out_total, dtype=torch.int64, device=dev)
    e2e_jobs = []
    for k, j in enumerate(jobs):
        wa, wb = in_words[k]
        e2e_jobs.append((dev_in[in_offs[2 * k]:in_offs[2 * k] + wa], j[1], dev_in[in_offs[2 * k + 1]:in_offs[2 * k + 1] + wb],
                         j[3], dev_out[out_offs[k]:out_offs[k] + j[4].numel()]))
    prepared_e2e = ctx.prepare_batch(e2e_jobs)

    def e2e_step():
        with torch.cuda.stream(stream):
            dev_in.copy_(host_in, non_blocking=True)
            ctx.mul_batch(prepared_e2e, workspace=ws, stream=stream)
            host_out.copy_(dev_out, non_blocking=True)
        stream.synchronize()
    e2e_step()
    e2e_step()
    hout = host_out.numpy().view(np.uint64)
    for k in (0, count // 2, count - 1):                  # the packed results equal the per-job ones
        if not np.array_equal(hout[out_offs[k]:out_offs[k] + jobs[k][4].numel()], jobs[k][4].cpu().numpy().view(np.uint64)):
            raise RuntimeError("e2e batch result differs from the device-resident batch")
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = dist_max(time.perf_counter() - t0, world)
    h2d = in_total * 8                                 # the packed buffers copied each step
    d2h = out_total * 8
    launches = sum(v[1] for v in prof.values())
    line = {"metric": "products/s (batched, uneven lengths)", "value": value, "unit": "products/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": CONFIGS[4]["name"], "products": count,
                       "l2": "flushed before every timed step (256 MiB write)"},
            "batch_mode": f"the library's choice, timed on the first call: {chose}",
            "persistent": {"value": pers_value, "unit": "products/s", "ms_per_step": pers_ms / args.steps,
                           "gpu_launches": int(sum(v[1] for v in pers_prof.values()) / args.steps),
                           "how": "one persistent launch per batch (device work queue), graph replay"},
            "class_launches": {"value": class_value, "unit": "products/s", "ms_per_step": class_ms / args.steps,
                               "stages_ms": {k: round(v[0] / args.steps, 4) for k, v in class_prof.items()},
                               "gpu_launches": int(sum(v[1] for v in class_prof.values()) / args.steps),
                               "how": "the same call with one launch per kernel and size class, graph replay"},
            "plain": {"value": plain, "unit": "products/s", "how": "one gf2x_mul call per product, same stream"},
            "batched_over_plain": value / plain,
            "operand_gbits": world * sum(j[1] + j[3] for j in jobs) * args.steps / (total_ms / 1e3) / 1e9,
            "stages_ms": {k: round(v[0] / args.steps, 4) for k, v in prof.items()},
            "gpu_launches": int(launches), "clocks": clk,
            "e2e": {"value": world * count * args.steps / e2e_s, "unit": "products/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def serving_requests(count, seed):
    """(na, nb) per request: log-uniform 2^12..2^26, 5% with one operand of exactly 2^28 bits."""
    lens = synth.loguniform_lengths(synth.config_seed(5, seed), 2 * count, 12.0, 26.0).reshape(count, 2)
    u = synth.uniform01(synth.config_seed(5, seed + 1), 2 * count).reshape(count, 2)
    out = []
    for k in range(count):
        na, nb = int(lens[k, 0]), int(lens[k, 1])
        if u[k, 0] < 0.05:
            if u[k, 1] < 0.5:
                na = 1 << 28
            else:
                nb = 1 << 28
        out.append((na, nb))
    return out


def run_reuse(args, world, rank, local):
    """Products with one fixed operand whose transform is computed once, vs gf2x_mul."""
    import torch
    from paper_1803_11301_gb300 import Context, build as lib_build, transform_bits, workspace_bytes
    lib_build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = CONFIGS[6]
    na, nb = cfg["na"], cfg["nb"]
    ctx = Context(local)
    stream = torch.cuda.current_stream(dev)
    n = transform_bits(na, nb)
    b = torch.from_numpy(synth.operand(synth.config_seed(6, 1), nb).view(np.int64)).to(dev)
    a_list = [torch.from_numpy(synth.operand(synth.config_seed(6, 100 + k), na).view(np.int64)).to(dev)
              for k in range(4)]
    c = torch.empty((na + nb - 1 + 63) // 64, dtype=torch.int64, device=dev)
    ws = torch.empty(workspace_bytes(na, nb), dtype=torch.uint8, device=dev)
    bhat = ctx.forward_transform(b, nb, n, workspace=ws, stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def timed(fn):
        for k in range(args.warmup):
            flush.fill_(1)
            fn(a_list[k % len(a_list)])
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        dist_barrier(world)
        torch.cuda.synchronize(dev)
        for k in range(args.steps):
            flush.fill_(k)
            starts[k].record(stream)
            fn(a_list[k % len(a_list)])
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
        dist_barrier(world)
        return dist_max(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), world)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    reuse_ms = timed(lambda a: ctx.mul_transformed(a, na, bhat, nb, out=c, workspace=ws, stream=stream))
    plain_ms = timed(lambda a: ctx.mul(a, na, b, nb, out=c, workspace=ws, stream=stream))
    clk = clocks.stop()
    want = ctx.mul(a_list[0], na, b, nb, workspace=ws, stream=stream)
    got = ctx.mul_transformed(a_list[0], na, bhat, nb, workspace=ws, stream=stream)
    if not torch.equal(want, got):
        raise RuntimeError("product with the reused transform differs from gf2x_mul")
    value = world * (na + nb) * args.steps / (reuse_ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": reuse_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": cfg["name"], "na_bits": na, "nb_bits": nb, "transform_bits": n,
                       "l2": "flushed before every timed step (256 MiB write)"},
            "plain": {"value": world * (na + nb) * args.steps / (plain_ms / 1e3) / 1e9, "unit": UNIT,
                      "ms_per_step": plain_ms / args.steps, "how": "gf2x_mul with both operands"},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_serving(args, world, rank, local):
    """Continuous batching under Poisson arrivals at several loads, against one
    gf2x_mul per request on the same arrival stream, and end to end with host
    operands (copies in and out inside each request's latency)."""
    import torch
    from paper_1803_11301_gb300 import Context, build as lib_build, workspace_bytes
    from paper_1803_11301_gb300.serving import Server, Request, percentile
    lib_build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = Context(local)
    count = args.requests
    sizes = serving_requests(count, 7 + rank)
    # operand pools (device, and page-locked host copies for the e2e leg); a
    # request uses a prefix of a pool entry
    small_h = [synth.operand(synth.config_seed(5, 100 + k), 1 << 26) for k in range(8)]
    big_h = [synth.operand(synth.config_seed(5, 200 + k), 1 << 28) for k in range(2)]
    small = [torch.from_numpy(w.view(np.int64)).to(dev) for w in small_h]
    big = [torch.from_numpy(w.view(np.int64)).to(dev) for w in big_h]
    small_p = [torch.from_numpy(w.view(np.int64)).pin_memory() for w in small_h]
    big_p = [torch.from_numpy(w.view(np.int64)).pin_memory() for w in big_h]

    def pool_of(bits, host):
        if bits > (1 << 26):
            return (big_p if host else big), 1000
        return (small_p if host else small), 0

    def operand(bits, k, host=False):
        pool, base = pool_of(bits, host)
        t = pool[k % len(pool)]
        return t[: (bits + 63) // 64], base + k % len(pool)

    rng_reuse = synth.uniform01(synth.config_seed(5, 77), count)

    def make(k, host=False):
        na, nb = sizes[k]
        a, _ = operand(na, 3 * k, host)
        if args.reuse_frac > 0 and rng_reuse[k] < args.reuse_frac:
            b, key = operand(nb, 0, host)             # one recurring b per pool and length
        else:
            b, key = operand(nb, 3 * k + 1, host)
        return Request(a, na, b, nb, tag=k, host=host, b_key=(key, nb) if args.reuse_frac > 0 else None)

    def drop_output(r):                 # latencies only: a served product is released at once
        r.out = None

    def server():
        return Server(ctx, streams=3, reuse_after=2 if args.reuse_frac > 0 else 0, on_done=drop_output)

    srv = server()
    for k in range(min(count, 400)):                        # warm-up
        srv.submit(make(k))
    srv.drain()
    for k in range(min(count, 400)):                        # warm-up of the one-call path
        r = make(k)
        ctx.mul(r.a, r.na, r.b, r.nb)
    torch.cuda.synchronize(dev)
    ctx.tune_freeze(True)       # launch shapes measured in the warm-up; no request waits on a measurement
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # saturated: everything queued at once
    srv = server()
    t0 = time.perf_counter()
    for k in range(count):
        srv.submit(make(k))
    srv.drain()
    sat = count / (time.perf_counter() - t0)
    del srv
    gaps01 = -np.log(1.0 - synth.uniform01(synth.config_seed(5, 55), count))

    def replay(arrivals, submit_fn, poll_fn, done_fn):
        start = time.perf_counter()
        k = 0
        while k < count or not done_fn():
            now = time.perf_counter() - start
            while k < count and arrivals[k] <= now:
                submit_fn(k, start + arrivals[k])
                k += 1
            poll_fn()
        return time.perf_counter() - start

    def served_at(load, host=False):
        arrivals = np.cumsum(gaps01 / (load * sat))
        s2 = server()
        reqs = []

        def s_submit(k, t):
            r = make(k, host)
            r.arrival = t
            reqs.append(r)
            s2.submit(r)
        wall = replay(arrivals, s_submit, s2.poll, lambda: not s2.pending and not s2.inflight)
        lat = [1e3 * (r.done - r.arrival) for r in reqs if r.state == "done"]
        return {"load": load, "arrival_rate_per_s": load * sat, "products_per_s": count / wall,
                "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99), "batches": s2._next_batch,
                "rejected": len(s2.rejected), "reused": sum(1 for r in reqs if r.reused)}

    loads = {str(x): served_at(x) for x in (0.5, 0.8, 1.0)}
    headline = loads["0.8"]
    from paper_1803_11301_gb300 import KNOB_BATCH_PERSISTENT
    modes = {}
    for name, m in (("persistent", 1), ("class_launches", 0)):     # the server's batches pinned to one way
        ctx.tune_pin(KNOB_BATCH_PERSISTENT, m)
        modes[name] = served_at(0.8)
    ctx.tune_pin(KNOB_BATCH_PERSISTENT, -1)
    # one gf2x_mul per request, in arrival order on one stream, at 0.8 x saturated
    stream = torch.cuda.current_stream(dev)
    wsp = torch.empty(max(workspace_bytes(na, nb) for na, nb in sizes), dtype=torch.uint8, device=dev)
    plain_pending = []
    plain_lat = []

    def p_submit(k, t):
        na, nb = sizes[k]
        out = torch.empty((na + nb - 1 + 63) // 64, dtype=torch.int64, device=dev)
        r = make(k)
        ctx.mul(r.a, na, r.b, nb, out=out, workspace=wsp, stream=stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        plain_pending.append((t, ev, out))

    def p_poll():
        now = time.perf_counter()
        while plain_pending and plain_pending[0][1].query():
            t, _, _ = plain_pending.pop(0)
            plain_lat.append(1e3 * (now - t))
    pwall = replay(np.cumsum(gaps01 / (0.8 * sat)), p_submit, p_poll, lambda: not plain_pending)
    plain = {"products_per_s": count / pwall, "p50_ms": percentile(plain_lat, 50), "p99_ms": percentile(plain_lat, 99)}
    # end to end: page-locked host operands, copies to and from the device inside the latency,
    # at 0.8 x its own saturated rate
    s3 = server()
    t0 = time.perf_counter()
    for k in range(count):
        s3.submit(make(k, host=True))
    s3.drain()
    sat_e2e = count / (time.perf_counter() - t0)
    del s3

    def served_host(load):
        arrivals = np.cumsum(gaps01 / (load * sat_e2e))
        s4 = server()
        reqs = []

        def s_submit(k, t):
            r = make(k, True)
            r.arrival = t
            reqs.append(r)
            s4.submit(r)
        wall = replay(arrivals, s_submit, s4.poll, lambda: not s4.pending and not s4.inflight)
        lat = [1e3 * (r.done - r.arrival) for r in reqs if r.state == "done"]
        return {"load": load, "products_per_s": count / wall, "p50_ms": percentile(lat, 50),
                "p99_ms": percentile(lat, 99), "saturated_products_per_s": sat_e2e}
    e2e_run = served_host(0.8)
    clk = clocks.stop()
    h2d = sum(8 * ((na + 63) // 64 + (nb + 63) // 64) for na, nb in sizes) / count
    d2h = sum(8 * ((na + nb - 1 + 63) // 64) for na, nb in sizes) / count
    line = {"metric": "products/s under Poisson load (continuous batching)", "value": headline["products_per_s"],
            "unit": "products/s", "n_gpus": world, "steps": count, "warmup": min(count, 400),
            "ms_per_step": 1e3 / headline["products_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": CONFIGS[5]["name"], "requests": count, "load": 0.8,
                       "saturated_products_per_s": sat, "reuse_frac": args.reuse_frac},
            "served": headline, "loads": loads, "batch_modes_at_0.8": modes, "plain_one_call_per_request": plain,
            "e2e": {"value": e2e_run["products_per_s"], "unit": "products/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "p50_ms": e2e_run["p50_ms"], "p99_ms": e2e_run["p99_ms"],
                    "load": 0.8, "saturated_products_per_s": sat_e2e,
                    "how": "page-locked host operands; the server copies them in and the product out on the "
                           "batch's stream, inside each request's latency; bytes per request"},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gf2x", choices=["gf2x", "reference"])
    ap.add_argument("--config", type=int, default=3, choices=sorted(CONFIGS))
    ap.add_argument("--batch", type=int, default=4096, help="products per batch for --config 4")
    ap.add_argument("--requests", type=int, default=20000, help="requests for --config 5")
    ap.add_argument("--reuse-frac", type=float, default=0.0,
                    help="--config 5: share of requests whose b recurs (resident transforms); 0 keeps the workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stage", default=None,
                    choices=["butterfly", "ibutterfly", "basis_cvt", "ibasis_cvt", "encode", "decode", "pointwise",
                             "field_mul"],
                    help="time one stage alone through its entry point (profiling aid); field_mul: every "
                         "GF(2^64) product form")
    ap.add_argument("--field-steps", type=int, default=2000, help="chain steps per thread for --stage field_mul")
    ap.add_argument("--log2-points", type=int, default=24, help="n_p = 2^this GF(2^64) points for --stage")
    ap.add_argument("--log2-bits", type=int, default=None,
                    help="operands of 2^this bits for the single-product configs (1-3, 7, 8): the length sweep")
    args = ap.parse_args()
    if args.stage == "field_mul":
        run_field_mul(args)
        return
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
    if args.config == 4:
        run_batch(args, world, rank, local)
    elif args.config == 5:
        run_serving(args, world, rank, local)
    elif args.config == 6:
        run_reuse(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
