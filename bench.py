"""Benchmark: simulated paths/s of the Schroedinger-Feynman path sum on the
7x8 grid, depth 1+40+1 (28+28-qubit halves, 35 cut CZs), fidelity f = 0.5%
(FRACTION selection, seed 7), 1M random 56-bit bitstrings.

A step is one 128-path prefix subtree of the selection (the unit a single
process of the paper ran, 28 prefix bits + 7 suffix bits), taken in the
selection's sorted order, through the C ABI with every input resident in HBM.
`e2e` repeats the measurement through the host-buffer call (bitstrings copied
in, amplitudes copied out inside the timed region).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank takes every N-th prefix (weak scaling, no collective
in the data path); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "7x8_d40"   # the headline workload; --workload picks a profiling case
FIDELITY = 0.005
SEED = 7
METRIC = "simulated paths/s at 7x8 depth 1+40+1"
UNIT = "paths/s"


def config_dict(n_bits, extra=None, workload=WORKLOAD):
    if workload == "5x10_d16":
        d = {"workload": "5x10 grid, depth 1+16+1 (v2 one-qubit rule), cut 25+25 qubits, f = 0.5% "
                         "(FRACTION, seed 7), random bitstrings; step = one 128-path prefix subtree "
                         "(the profiling case: 256 MB half-states, above the 129 MB L2)",
             "grid": "5x10", "depth": "1+16+1", "fidelity": FIDELITY, "bitstrings": n_bits,
             "paths_per_step": 128}
    else:
        d = {"workload": "7x8 grid, depth 1+40+1 (v2 one-qubit rule), cut cols 0-3 | 4-7 (28+28 qubits), "
                         "35 cut CZs, f = 0.5% (FRACTION, 28 prefix bits, seed 7), 1M random bitstrings; "
                         "step = one 128-path prefix subtree",
             "grid": "7x8", "depth": "1+40+1", "fidelity": FIDELITY, "bitstrings": n_bits,
             "paths_per_step": 128,
             "l2": "no flush: every pass streams 2 GiB half-states, far larger than the 129 MB L2"}
    if extra:
        d.update(extra)
    return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxes.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return None
        return {"sm_mhz": float(np.median(sms)), "sm_max_mhz": max(maxes), "samples": len(sms),
                "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources the pass kernels are built from."""
    h = hashlib.sha256()
    for f in ("kernels.cu", "pass_common.cuh", "dev_types.h", "jit.cpp"):
        with open(os.path.join(ROOT, "paper_1807_10749_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(alg_bytes_per_launch):
    """DRAM bytes per pass launch: the DRAM-to-algorithmic byte ratio of the
    committed ncu capture (a smaller case of the same kernel) times this
    workload's algorithmic bytes per launch, if the capture was taken on the
    current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_7x8_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        if d.get("pass_sources_sha256_16") != kernel_source_hash():
            return None
        return float(d["dram_bytes_per_algorithmic_byte"]) * alg_bytes_per_launch
    except Exception:
        return None


def oracle_path_sample(text, mask, bits, fraction, prefix_index=0):
    """The FP64 oracle as it stands (oracle_sf) on a bounded sample of one
    selected 7x8 path: both 28-qubit halves evolved from |0> through the first
    `fraction` of their gate lists, then the 1024-bitstring product sum. Its
    dense evolution sweeps the whole half state once per gate, so the time of
    a full path is the sample's time times the gate-count ratio. Returns
    (seconds of the sample, that ratio, the prefix used)."""
    from oracle import circuit as ocirc
    from oracle import paths as opaths
    from oracle import sim
    sim.build()
    setup = sim.SFSetup(ocirc.parse(text), mask)
    pre, _, _ = opaths.fraction_prefixes(setup.x_bits, FIDELITY, SEED)
    prefix = int(pre[prefix_index % len(pre)])
    full = len(setup.opsA[0]) + len(setup.opsB[0])

    def cut(ops):
        g = max(1, int(round(len(ops[0]) * fraction)))
        return (ops[0][:g], ops[1][:g], ops[2][:g], ops[3][:g], ops[4][:32 * g])
    setup.opsA, setup.opsB = cut(setup.opsA), cut(setup.opsB)
    part = len(setup.opsA[0]) + len(setup.opsB[0])
    ids = np.array([prefix << (setup.x_bits - 28)], dtype=np.uint64)
    t0 = time.perf_counter()
    sim.sf_amplitudes(setup, ids, bits[:1024])
    return time.perf_counter() - t0, full / part, prefix


def cpu_baseline_sample(text, mask, bits_all):
    """The oracle's paths/s from a bounded sample (a quarter of one path)."""
    from oracle import sim
    dt, ratio, prefix = oracle_path_sample(text, mask, bits_all, 0.25)
    return {"value": 1.0 / (dt * ratio), "unit": UNIT, "cores": sim.threads(), "kind": "oracle",
            "sample": f"1 path (prefix {prefix}, suffix 0) of the 7x8 workload: the first quarter of both "
                      f"28-qubit halves' gates in FP64 from |0> and the 1024-bitstring sum, {dt:.1f} s; "
                      f"scaled by the gate-count ratio {ratio:.2f} to a whole path",
            "seconds": dt}


def amplitude_rates(paths_per_s, n_bits, n_selected):
    """Amplitude throughput beside paths/s: path-amplitude contributions per
    second (every path adds one term to each requested amplitude), and
    finished amplitudes per second of the whole request, extrapolated from
    the timed prefixes to all n_selected paths at the same rate."""
    return {"path_amplitudes_per_s": paths_per_s * n_bits,
            "request_amplitudes_per_s": n_bits * paths_per_s / n_selected,
            "request_seconds": n_selected / paths_per_s,
            "note": "request figures extrapolated from the timed 128-path prefixes to the whole selection"}


def rank_prefixes(first_ids, world, rank, n_steps):
    """First path id of each 128-path prefix this rank processes: every
    world-th prefix of the sorted selection (the ranks' sets are disjoint)."""
    n_pre = len(first_ids) // 128
    return [int(first_ids[128 * ((world * s + rank) % n_pre)]) for s in range(n_steps)]


def max_over_ranks(value, device=None):
    """Largest value over all ranks (the job time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def serving_window(sfsim, inputs, n_req=24, seed=42, max_paths=1 << 17, load=0.8, jit=1):
    """Serving mix (time-boxed): requests drawn like the 2000-request stream -
    grids uniform over 4x5, 5x5, 5x6, 6x6, 6x7, depth 1+d+1 with d uniform in
    16..32, f log-uniform in [0.01, 1], 1e3..1e6 bitstrings log-uniform -
    keeping the first n_req whose selected path count is <= max_paths (the
    full stream is hours of work). Each request first runs alone, one after
    the other (the plain form); then all are submitted to the server with
    Poisson arrivals at `load` times the plain capacity. Returns latency
    percentiles, aggregate paths/s both ways, and whether every served result
    equals the request run alone."""
    rng = np.random.default_rng(seed)
    grids = [(4, 5), (5, 5), (5, 6), (6, 6), (6, 7)]
    reqs = []
    while len(reqs) < n_req:
        R, C = grids[rng.integers(len(grids))]
        d = int(rng.integers(16, 33))
        f = float(np.exp(rng.uniform(np.log(0.01), 0.0)))
        na = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        text = inputs.google_circuit(R, C, d, 1 + len(reqs)).text()
        plan = sfsim.Plan(text)
        sel = sfsim.selection("fraction", fidelity=f, seed=7 + len(reqs))
        npaths, _ = sfsim.sf_selection_size(plan.handle, sel)
        plan.close()
        if npaths > max_paths:
            continue
        plan = sfsim.Plan(text, jit=jit)   # kernels compiled here, before any timing
        bits = inputs.random_bitstrings(R * C, na, 2000 + len(reqs))
        reqs.append((plan, bits, sel, npaths))
    alone, t_alone = [], []
    for plan, bits, sel, _ in reqs:
        t0 = time.perf_counter()
        alone.append(plan.amplitudes(bits, sel)[0])
        t_alone.append(time.perf_counter() - t0)
    paths = sum(r[3] for r in reqs)
    t_seq = sum(t_alone)
    rate = load * len(reqs) / t_seq
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    srv = sfsim.sf_server_create(0, 4)
    tickets = []
    t0 = time.perf_counter()
    for (plan, bits, sel, _), ta in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append(sfsim.sf_server_submit(srv, plan.handle, bits, sel))
    lat, same = [], True
    for t, (plan, bits, sel, _), a in zip(tickets, reqs, alone):
        while True:  # the server's own submit-to-done time, read before the wait releases it
            try:
                lat.append(sfsim.sf_server_times(srv, t)[1])
                break
            except sfsim.SFError as e:
                if e.code != sfsim.SF_ETIMEOUT:
                    raise
                time.sleep(0.001)
        got = sfsim.sf_server_wait(srv, t, len(bits))
        same = same and bool(np.array_equal(got, a))
    makespan = time.perf_counter() - t0
    # closed loop: every request submitted at once (server capacity)
    t1 = time.perf_counter()
    tk = [sfsim.sf_server_submit(srv, plan.handle, bits, sel) for plan, bits, sel, _ in reqs]
    for t, (plan, bits, sel, _) in zip(tk, reqs):
        sfsim.sf_server_wait(srv, t, len(bits))
    saturated = time.perf_counter() - t1
    sfsim.sf_server_destroy(srv)
    for plan, _, _, _ in reqs:
        plan.close()
    return {"requests": len(reqs), "paths": int(paths), "offered_load": load,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                  "plain_paths_per_s": paths / t_seq, "served_paths_per_s": paths / makespan,
                  "served_identical_to_alone": same, "makespan_s": makespan, "plain_total_s": t_seq,
            "saturated_paths_per_s": paths / saturated,
            "window": f"first {n_req} requests of the seeded mix with <= {max_paths} paths",
            "pass_kernels": "specialised" if jit else "generic"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores, same metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1807_10749_gb300 import inputs
    w = inputs.WORKLOADS[WORKLOAD]
    text = inputs.workload_circuit(WORKLOAD).text()
    bits = inputs.random_bitstrings(56, 1024, w["bitstring_seed"])
    from oracle import sim
    sim.build()
    times = []
    for step in range(args.warmup + args.steps):
        dt, ratio, _ = oracle_path_sample(text, w["side_b_mask"], bits, 0.125, step)
        if step >= args.warmup:
            times.append(dt * ratio)   # the seconds of one whole path
    total = sum(times)
    value = len(times) / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": config_dict(1024, {"reference": "FP64 CPU oracle (oracle/core.c, OpenMP)",
                                         "step": "one selected path x 1024 bitstrings, timed on the first "
                                                 "eighth of its gates and scaled by the gate-count ratio"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": sim.threads(), "kind": "oracle",
                             "sample": "per step one selected path (the step's prefix) of the 7x8 workload: the "
                                       "first eighth of both 28-qubit halves' gates in FP64 from |0> and the "
                                       "1024-bitstring sum, scaled by the gate-count ratio to a whole path"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--bitstrings", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--exec-mode", default="batched", choices=["batched", "plain"])
    ap.add_argument("--workload", default=WORKLOAD, choices=["7x8_d40", "5x10_d16"])
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--fuse-bits", type=int, default=0)
    ap.add_argument("--run-bits", type=int, default=0)
    ap.add_argument("--split-last", type=int, default=0, choices=[0, 1],
                    help="1: run the level before the folded last level as its own segment")
    ap.add_argument("--fp32x2", type=int, default=0, choices=[0, 1],
                    help="1: packed FP32x2 arithmetic in the specialised kernels' Google-gate stages")
    ap.add_argument("--dense-finals", type=int, default=0, choices=[0, 1],
                    help="1: the final programs write whole final states (no compact blocks)")
    ap.add_argument("--jit", type=int, default=1, choices=[0, 1],
                    help="1: per-pass specialised kernels compiled at plan time; 0: the generic pass kernel")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1807_10749_gb300 import build as sfbuild
    if rank == 0 or world == 1:
        sfbuild.build()
    if world > 1:
        dist.barrier()
    from paper_1807_10749_gb300 import inputs, sfsim

    w = inputs.WORKLOADS[args.workload]
    text = inputs.workload_circuit(args.workload).text()
    nq = w["rows"] * w["cols"]
    bits = inputs.random_bitstrings(nq, args.bitstrings, w["bitstring_seed"])
    mode = sfsim.SF_EXEC_PLAIN if args.exec_mode == "plain" else sfsim.SF_EXEC_BATCHED
    t_plan = time.perf_counter()
    plan = sfsim.Plan(text, side_b_mask=w["side_b_mask"], exec_mode=mode, tile_bits=args.tile_bits,
                      fuse_bits=args.fuse_bits, run_bits=args.run_bits, jit=args.jit,
                      split_last=args.split_last, fp32x2=args.fp32x2, dense_finals=args.dense_finals)
    t_plan = time.perf_counter() - t_plan
    fsel = sfsim.selection("fraction", fidelity=FIDELITY, seed=SEED)
    n_sel, f_actual = sfsim.sf_selection_size(plan.handle, fsel)
    n_steps_total = args.warmup + args.steps
    # this rank's prefixes: every world-th 128-path subtree of the sorted selection
    first_ids = sfsim.sf_selection_ids(plan.handle, fsel, cap=128 * world * (n_steps_total + 2))
    prefixes = rank_prefixes(first_ids, world, rank, n_steps_total + 1)
    sels = [sfsim.selection("range", first=p, count=128) for p in prefixes]

    d_bits = torch.from_numpy(bits.view(np.int64)).to(f"cuda:{dev}")
    d_out = torch.zeros((len(bits), 2), dtype=torch.float64, device=f"cuda:{dev}")
    ws_bytes = max(sfsim.sf_workspace_size(plan.handle, len(bits), s) for s in sels[:2])
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()

    def step(i):
        sfsim.sf_amplitudes_device(plan.handle, d_bits, sels[i], d_out, ws, stream=stream, accumulate=True)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    sfsim.sf_plan_profile(plan.handle, True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.warmup, n_steps_total):
        step(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    pass_n, pass_s, pass_b = sfsim.sf_plan_profile_read(plan.handle, 0)
    gat_n, gat_s, gat_b = sfsim.sf_plan_profile_read(plan.handle, 1)
    oth_n, _, _ = sfsim.sf_plan_profile_read(plan.handle, 2)
    sfsim.sf_plan_profile(plan.handle, False)
    t_max = max_over_ranks(elapsed, f"cuda:{dev}")
    paths_total = 128 * args.steps * world
    value = paths_total / t_max

    # end to end through the host-buffer call: every step copies the
    # bitstrings from pinned host memory to the device and the amplitudes back
    e2e_steps = max(2, min(args.steps, 6))
    pin_bits = torch.from_numpy(bits.view(np.int64)).pin_memory().numpy().view(np.uint64)
    pin_out = torch.empty(2 * len(bits), dtype=torch.float64).pin_memory().numpy()
    sfsim.sf_amplitudes_into(plan.handle, pin_bits, sels[0], pin_out)  # warm the host-form workspace
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t1 = time.perf_counter()
    for i in range(e2e_steps):
        sfsim.sf_amplitudes_into(plan.handle, pin_bits, sels[(args.warmup + i) % len(sels)], pin_out)
    e2e_wall = max_over_ranks(time.perf_counter() - t1, f"cuda:{dev}")
    e2e_value = 128 * e2e_steps * world / e2e_wall

    plain = None
    if world == 1 and not args.no_plain and args.exec_mode == "batched":
        # the plain form: the same kernels, one path at a time from the prefix
        # checkpoint (no shared levels below it, no folded last level)
        pplan = sfsim.Plan(text, side_b_mask=w["side_b_mask"], exec_mode=sfsim.SF_EXEC_PLAIN,
                           tile_bits=args.tile_bits, fuse_bits=args.fuse_bits, run_bits=args.run_bits,
                           jit=args.jit)
        pws = torch.empty(sfsim.sf_workspace_size(pplan.handle, len(bits), sels[0]), dtype=torch.uint8,
                          device=f"cuda:{dev}")
        sub = [sfsim.selection("range", first=int(prefixes[args.warmup]), count=16)]
        sfsim.sf_amplitudes_device(pplan.handle, d_bits, sub[0], d_out, pws, stream=stream, accumulate=True)
        torch.cuda.synchronize()
        sub2 = sfsim.selection("range", first=int(prefixes[args.warmup]) + 16, count=32)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sfsim.sf_amplitudes_device(pplan.handle, d_bits, sub2, d_out, pws, stream=stream, accumulate=True)
        e1.record(stream)
        torch.cuda.synchronize()
        plain = {"value": 32 / (e0.elapsed_time(e1) / 1e3), "unit": UNIT,
                 "sample": "32 paths of the first timed prefix, each evolved alone from the resident "
                           "prefix checkpoint (no shared levels below it, no folded last level)"}
        del pws
        pplan.close()
    serving = None
    if world == 1 and not args.no_serve and args.workload == WORKLOAD:
        serving = serving_window(sfsim, inputs, jit=args.jit)

    if rank == 0:
        peak, peak_kind = measured_peaks()
        achieved = (pass_b / pass_s) / 1e9 if pass_s > 0 else None
        traffic = ncu_traffic(pass_b / max(1, pass_n))
        cpu = None
        if world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
            cpu = cpu_baseline_sample(text, w["side_b_mask"], bits)
        line = {
            "metric": METRIC if args.workload == WORKLOAD else f"simulated paths/s ({args.workload})",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": config_dict(len(bits), workload=args.workload, extra={
                "exec_mode": args.exec_mode, "f_actual": f_actual,
                "tile_bits": args.tile_bits or "per segment (12 or 13)", "fuse_bits": args.fuse_bits or 5,
                "run_bits": args.run_bits or "per segment (3 or 4)",
                "pass_kernels": "specialised" if args.jit else "generic",
                "split_last": args.split_last, "fp32x2": args.fp32x2,
                "finals": ("dense (whole final states written)" if args.dense_finals else
                           "compact where the planner allows (only the 2^g-amplitude blocks of "
                           "requested bitstrings written)"),
                "plan_seconds": t_plan,
                "paths_selected": n_sel, "parallelism": f"paths x{world}", "wall_s": wall}),
            "roofline": {"kernel": ("sf_pass_spec (per-pass specialised fused tile pass)" if args.jit
                                    else "pass_kernel (generic fused tile pass)"), "bound": "hbm",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": pass_b / max(1, pass_n),
                         "avg_launch_ms": 1e3 * pass_s / max(1, pass_n),
                         "share_of_step": pass_s / t_max if t_max > 0 else None},
            "kernels": {"pass": {"launches": pass_n, "seconds": pass_s, "bytes": pass_b},
                        "gather": {"launches": gat_n, "seconds": gat_s, "bytes": gat_b},
                        "other": {"launches": oth_n}},
            "gpu_launches": pass_n + gat_n + oth_n,
            "amplitudes": amplitude_rates(value, len(bits), n_sel),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * len(bits),
                    "d2h_bytes_per_step": 16 * len(bits), "steps": e2e_steps,
                    "host_buffers": "pinned (sf_amplitudes with host pointers)"},
            "clocks": clocks,
            "plain_form": plain,
            "batched_over_plain": (value / plain["value"]) if plain else None,
            "serving": serving,
            "cpu_baseline": ({k: v for k, v in cpu.items() if k != "seconds"} if cpu else None),
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
