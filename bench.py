"""Benchmark: simulated paths/s of the Schroedinger-Feynman path sum on the
7x8 grid, depth 1+40+1 (28+28-qubit halves, 35 cut CZs), fidelity f = 0.5%
(FRACTION selection, seed 7), 1M random 56-bit bitstrings.

A step is one 128-path prefix subtree of the selection (the unit a single
process of the paper ran, 28 prefix bits + 7 suffix bits), taken in the
selection's sorted order, through the C ABI with every input resident in HBM.
`e2e` repeats the measurement through the host-buffer call (bitstrings copied
in, amplitudes copied out inside the timed region).

Beside the headline the line carries: the accuracy of the benchmark's own
configuration against stored FP64 oracle values, the other workloads (4x4,
5x6 autotuned, 6x7 at two fidelities and its Haar variant) each with its
pass-kernel roofline and an oracle baseline, the runtime model of Eq. t_tot
fitted on this GPU, and a serving window of the seeded request mix.

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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "7x8_d40"   # the headline workload; --workload picks a profiling case
FIDELITY = 0.005
SEED = 7
METRIC = "simulated paths/s at 7x8 depth 1+40+1"
UNIT = "paths/s"
GOLDEN_7X8 = os.path.join(ROOT, "tests", "golden", "oracle_7x8_d40_paths.npz")


def config_dict(n_bits, extra=None, workload=WORKLOAD):
    if workload in ("5x10_d16", "5x10_d14"):
        d = {"workload": f"5x10 grid, depth 1+{workload[-2:]}+1 (v2 one-qubit rule), cut 25+25 qubits, f = 0.5% "
                         "(FRACTION, seed 7), random bitstrings; step = one 128-path prefix subtree "
                         "(a profiling case: 256 MB half-states, above the 129 MB L2"
                         + ("; its last level folds into the gather)" if workload == "5x10_d14" else ")"),
             "grid": "5x10", "depth": f"1+{workload[-2:]}+1", "fidelity": FIDELITY, "bitstrings": n_bits,
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
    """DRAM bytes per pass launch from the committed ncu capture of this
    kernel (a smaller case of it, see profiles/): there the reads equal the
    algorithmic reads and the writes fall short by the part still in L2 when
    the kernel ends, a tail of fixed size per launch; so traffic =
    algorithmic bytes - that tail. None unless the capture was taken on the
    current kernel sources."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_7x8_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        if d.get("pass_sources_sha256_16") != kernel_source_hash():
            return None
        return max(0.0, alg_bytes_per_launch - float(d["l2_write_tail_bytes_per_launch"]))
    except Exception:
        return None


def oracle_path_sample(text, mask, bits, fraction, prefix_index=0):
    """The FP64 oracle as it stands (oracle_sf) on a bounded sample of one
    selected 7x8 path: both 28-qubit halves evolved from |0> through the first
    `fraction` of their gate lists, then the product sum over `bits`. Its
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
    sim.sf_amplitudes(setup, ids, bits)
    return time.perf_counter() - t0, full / part, prefix


def cpu_baseline_sample(text, mask, bits_all):
    """The oracle's paths/s from a bounded sample (a quarter of one path,
    all 1M bitstrings)."""
    from oracle import sim
    dt, ratio, prefix = oracle_path_sample(text, mask, bits_all, 0.25)
    return {"value": 1.0 / (dt * ratio), "unit": UNIT, "cores": sim.threads(), "kind": "oracle",
            "sample": f"1 path (prefix {prefix}, suffix 0) of the 7x8 workload: the first quarter of both "
                      f"28-qubit halves' gates in FP64 from |0> and the sum over all {len(bits_all)} bitstrings, "
                      f"{dt:.1f} s measured; scaled by the gate-count ratio {ratio:.2f} to a whole path",
            "sample_seconds": dt, "extrapolated": True}


def amplitude_rates(paths_per_s, n_bits, n_selected):
    """Amplitude throughput beside paths/s: path-amplitude contributions per
    second (every path adds one term to each requested amplitude), and
    finished amplitudes per second of the whole request, extrapolated from
    the timed prefixes to all n_selected paths at the same rate."""
    sec = n_selected / paths_per_s
    return {"path_amplitudes_per_s": paths_per_s * n_bits,
            "request_amplitudes_per_s": n_bits * paths_per_s / n_selected,
            "request_seconds": sec,
            "gpu_hours_per_1M_amplitudes": sec / 3600.0 * 1e6 / n_bits,
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


# ------------------------------------------------------------ helpers
def _device_run(sfsim, plan, d_bits, sel, d_out, ws, stream, reps=1):
    """CUDA-event seconds per call of `reps` back-to-back device calls (after
    one untimed call) and the pass kernel's profile over them."""
    import torch
    sfsim.sf_amplitudes_device(plan.handle, d_bits, sel, d_out, ws, stream=stream)
    torch.cuda.synchronize()
    sfsim.sf_plan_profile(plan.handle, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        sfsim.sf_amplitudes_device(plan.handle, d_bits, sel, d_out, ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sfsim.sf_plan_status(plan.handle, stream)
    prof = sfsim.sf_plan_profile_read(plan.handle, 0)
    sfsim.sf_plan_profile(plan.handle, False)
    return e0.elapsed_time(e1) / 1e3 / reps, prof


def _roofline(prof, reps, peak):
    n, s, b = prof
    ach = b / s / 1e9 if s > 0 else None
    return {"kernel": "sf_pass_spec", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak if ach else None, "launches_per_call": n / max(1, reps),
            "avg_launch_ms": 1e3 * s / max(1, n), "seconds_per_call": s / max(1, reps)}


def _oracle_paths_per_s(text, mask, ids, bits, decomposition="schmidt"):
    from oracle import circuit as ocirc
    from oracle import sim
    sim.build()
    setup = sim.SFSetup(ocirc.parse(text), mask, decomposition)
    t0 = time.perf_counter()
    sim.sf_amplitudes(setup, np.asarray(ids, dtype=np.uint64), bits)
    dt = time.perf_counter() - t0
    return len(ids) / dt, dt, sim.threads()


# --------------------------------------------------- other workloads
def other_configs(sfsim, inputs, peak, stream):
    """The smaller workloads of the benchmark suite, each once warm and then
    timed through the device call (inputs resident), with the pass kernel's
    roofline, amplitude rates and the FP64 oracle timed on a bounded sample
    of the same workload on the host cores."""
    import torch
    out = {}

    def run(name, text, mask, bits, sel, opts, oracle_ids, extra, f_scale=None):
        plan = sfsim.Plan(text, side_b_mask=mask, **opts)
        n_sel, fa = sfsim.sf_selection_size(plan.handle, sel)
        d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
        d_out = torch.zeros((len(bits), 2), dtype=torch.float64, device="cuda")
        ws = torch.empty(sfsim.sf_workspace_size(plan.handle, len(bits), sel), dtype=torch.uint8, device="cuda")
        reps = 3 if n_sel * len(bits) < 5e10 else 1
        sec, prof = _device_run(sfsim, plan, d_bits, sel, d_out, ws, stream, reps)
        plan.close()
        del ws
        ops, odt, cores = _oracle_paths_per_s(text, mask, oracle_ids, bits)
        line = {"paths_selected": int(n_sel), "f_actual": fa, "bitstrings": len(bits), "seconds": sec,
                "paths_per_s": n_sel / sec, "path_amplitudes_per_s": n_sel * len(bits) / sec,
                "amplitudes_per_s": len(bits) / sec, "roofline": _roofline(prof, reps, peak),
                "cpu_baseline": {"value": ops, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{len(oracle_ids)} selected paths x {len(bits)} bitstrings, "
                                           f"{odt:.2f} s measured"},
                "gpu_over_oracle": (n_sel / sec) / ops}
        if f_scale:
            line["f1_seconds_extrapolated"] = sec * f_scale
        line.update(extra)
        out[name] = line

    w = inputs.WORKLOADS["4x4_d10"]
    text = inputs.workload_circuit("4x4_d10").text()
    bits = inputs.random_bitstrings(16, w["n_bitstrings"], w["bitstring_seed"])
    run("4x4_d10", text, w["side_b_mask"], bits, sfsim.selection("fraction", fidelity=1.0), {},
        np.arange(16), {"workload": "4x4, 1+10+1, rows 0-1 | 2-3, all 16 paths, 1024 bitstrings"})

    w = inputs.WORKLOADS["5x6_d24"]
    text = inputs.workload_circuit("5x6_d24").text()
    bits = inputs.random_bitstrings(30, w["n_bitstrings"], w["bitstring_seed"])
    sel = sfsim.selection("fraction", fidelity=1.0)
    c = sfsim.sf_circuit_parse(text)
    base = sfsim.sf_plan_opts_default(side_b_mask=w["side_b_mask"])
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    t_tune = time.perf_counter()
    best, t_best, t_base = sfsim.sf_plan_autotune(c, base, sel, 1 << 12, d_bits)
    t_tune = time.perf_counter() - t_tune
    sfsim.sf_circuit_destroy(c)
    tuned = {k: getattr(best, k) for k in ("tile_bits", "fuse_bits", "run_bits", "batch_paths")}
    run("5x6_d24", text, w["side_b_mask"], bits, sel, tuned, np.arange(64) * 512,
        {"workload": "5x6, 1+24+1, cols 0-2 | 3-5, all 2^15 paths, 100k bitstrings, autotuned",
         "autotune": {"chosen": tuned, "sample_seconds": t_best, "base_sample_seconds": t_base,
                      "search_seconds": t_tune,
                      "sample": "first 4096 paths, timed per candidate (pass shape, k in 2..5, paths per launch)"}})

    w = inputs.WORKLOADS["6x7_d26"]
    text = inputs.workload_circuit("6x7_d26").text()
    bits = inputs.random_bitstrings(42, w["n_bitstrings"], w["bitstring_seed"])
    for f in (0.01, 0.1):
        run(f"6x7_d26_f{f:g}", text, w["side_b_mask"], bits, sfsim.selection("fraction", fidelity=f, seed=SEED),
            {}, [1 << 20, (1 << 20) + 1],
            {"workload": f"6x7, 1+26+1, rows 0-2 | 3-5, f = {f:g} (FRACTION, seed 7), 1M bitstrings"},
            f_scale=1.0 / f)
    text_h = inputs.workload_circuit("6x7_d26", haar=True).text()
    run("6x7_d26_haar", text_h, w["side_b_mask"], bits, sfsim.selection("range", first=1 << 40, count=4096),
        {}, [1 << 40, (1 << 40) + 1],
        {"workload": "6x7, 1+26+1, every CZ a seeded Haar U(4) (4-way operator-Schmidt branching, 2^50 paths); "
                     "a 4096-path subtree, 1M bitstrings"})
    return out


# ------------------------------------------------------ runtime model
def calibrate_runtime_model(sfsim, inputs, stream, extra=()):
    """Eq. t_tot's constants fitted on this GPU from measured requests, device
    timing, best of three each: 4 small circuits (halves of 10-18 qubits, in
    L2) x 3 fidelities x 2 bitstring counts, the 6x7 workload (21-qubit
    halves) and the 5x10 profiling workload (25-qubit halves) at two
    fidelities and bitstring counts each, plus `extra` measured points
    (terms, seconds) - a 7x8 headline step. Every timed call starts without
    resident nodes, as the model's features assume: a repeated call on one
    workspace would find its upper levels already computed."""
    import torch
    T, S = [list(t) for t, _ in extra], [s for _, s in extra]
    cases = [(inputs.google_circuit(R, C, D, 3).text(),
              (inputs.column_cut_mask if cut[0] == "col" else inputs.row_cut_mask)(R, C, cut[1]), R * C,
              (1 / 16, 1 / 4, 1.0), (10_000, 200_000))
             for (R, C, D, cut) in [(5, 6, 24, ("col", 3)), (4, 5, 24, ("col", 2)), (6, 6, 20, ("col", 3)),
                                    (5, 5, 28, ("row", 2))]]
    for name, fs, nas in (("6x7_d26", (1 / 1024, 1 / 256), (100_000, 1_000_000)),
                          ("5x10_d16", (1 / 8, 1 / 2), (100_000, 1_000_000))):
        wl = inputs.WORKLOADS[name]
        cases.append((inputs.workload_circuit(name).text(), wl["side_b_mask"], wl["rows"] * wl["cols"], fs, nas))
    for text, mask, nq, fs, nas in cases:
        plan = sfsim.Plan(text, side_b_mask=mask)
        for f in fs:
            for n_a in nas:
                bits = inputs.random_bitstrings(nq, n_a, 11)
                sel = sfsim.selection("fraction", fidelity=f, seed=3)
                d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
                d_out = torch.zeros((n_a, 2), dtype=torch.float64, device="cuda")
                ws = torch.empty(sfsim.sf_workspace_size(plan.handle, n_a, sel), dtype=torch.uint8, device="cuda")
                best = 1e30
                for _ in range(3):
                    sfsim.sf_plan_drop_resident(plan.handle)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    sfsim.sf_amplitudes_device(plan.handle, d_bits, sel, d_out, ws, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1) / 1e3)
                S.append(best)
                T.append(sfsim.sf_plan_cost_terms(plan.handle, sel, n_a))
        plan.close()
        del ws
    T, S = np.array(T), np.array(S)
    coeffs = sfsim.sf_cost_fit(T, S)
    pred = np.array([sfsim.sf_cost_predict(t, coeffs) for t in T])
    rel = np.abs(pred - S) / S
    return coeffs, {"C0_s": coeffs[0], "C1_s": coeffs[1], "C1C2_s": coeffs[2],
                    "C2": coeffs[2] / coeffs[1] if coeffs[1] > 0 else None, "C3_s": coeffs[3],
                    "requests": len(S), "median_rel_err": float(np.median(rel)), "max_rel_err": float(rel.max()),
                    "headline_points_rel_err": [float(x) for x in rel[:len(extra)]],
                    "form": "T = C0 + C1 f 2^x_p (q1 2^q1 + q2 2^q2)(d_p + C2 2^x_b d_b) + C3 P n_a (Eq. t_tot, "
                            "plus a fixed cost per request C0)"}


# ------------------------------------------------------------ serving
def serving_window(sfsim, inputs, coeffs, n_req=200, seed=42, load=0.8, max_pred_s=1.0):
    """Serving mix: the first n_req requests of the seeded stream - grid
    uniform over 4x5, 5x5, 5x6, 6x6, 6x7, depth 1+d+1 with d uniform in
    16..32 (circuit seed 1, so requests on one grid and depth share a
    circuit), f log-uniform in [0.01, 1], 1e3..1e6 bitstrings log-uniform.
    The runtime model predicts each request's time; the window holds those
    predicted at most max_pred_s (the rest, listed with their predicted
    total, would take hours). Every windowed request runs alone, one after
    another (one request at a time); then all are submitted to the server
    with Poisson arrivals at `load` times that sequential capacity, and once
    more all at once (saturated). Results must equal the alone runs bit for
    bit."""
    rng = np.random.default_rng(seed)
    grids = [(4, 5), (5, 5), (5, 6), (6, 6), (6, 7)]
    stream = []
    for i in range(n_req):
        R, C = grids[rng.integers(len(grids))]
        d = int(rng.integers(16, 33))
        f = float(np.exp(rng.uniform(np.log(0.01), 0.0)))
        na = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        stream.append((R, C, d, f, na, i))
    probe = {}
    win, excluded, excl_pred = [], 0, 0.0
    for (R, C, d, f, na, i) in stream:
        key = (R, C, d)
        if key not in probe:
            probe[key] = sfsim.Plan(inputs.google_circuit(R, C, d, 1).text(), jit=0)
        sel = sfsim.selection("fraction", fidelity=f, seed=7 + i)
        pred = sfsim.sf_cost_predict(sfsim.sf_plan_cost_terms(probe[key].handle, sel, na), coeffs)
        if pred > max_pred_s:
            excluded += 1
            excl_pred += pred
            continue
        win.append((key, sel, na, i, pred))
    for p in probe.values():
        p.close()
    plans = {}
    t_plan = time.perf_counter()
    for key, _, _, _, _ in win:
        if key not in plans:   # kernels compiled here, before any timing
            R, C, d = key
            plans[key] = sfsim.Plan(inputs.google_circuit(R, C, d, 1).text())
    t_plan = time.perf_counter() - t_plan
    reqs = []
    for key, sel, na, i, pred in win:
        R, C, d = key
        n_sel, _ = sfsim.sf_selection_size(plans[key].handle, sel)
        reqs.append((plans[key], inputs.random_bitstrings(R * C, na, 2000 + i), sel, n_sel, pred))
    # one request at a time through the device call, with device buffers
    # allocated once for the largest request; bitstrings in and amplitudes
    # out inside each request's time, as the server does
    import torch
    nmax = max(len(r[1]) for r in reqs)
    ws = torch.empty(max(sfsim.sf_workspace_size(p.handle, len(b), s) for p, b, s, _, _ in reqs),
                     dtype=torch.uint8, device="cuda")
    d_bits = torch.empty(nmax, dtype=torch.int64, device="cuda")
    d_out = torch.empty((nmax, 2), dtype=torch.float64, device="cuda")

    def alone_call(plan, bits, sel):
        n = len(bits)
        d_bits[:n].copy_(torch.from_numpy(bits.view(np.int64)))
        sfsim.sf_amplitudes_device(plan.handle, d_bits[:n], sel, d_out[:n], ws)
        o = d_out[:n].cpu().numpy()
        return o[:, 0] + 1j * o[:, 1]
    for plan, bits, sel, _, _ in reqs[:4]:
        alone_call(plan, bits, sel)   # warm up
    alone, t_alone = [], []
    for plan, bits, sel, _, _ in reqs:
        t0 = time.perf_counter()
        alone.append(alone_call(plan, bits, sel))
        t_alone.append(time.perf_counter() - t0)
    del ws, d_bits, d_out
    paths = sum(r[3] for r in reqs)
    t_seq = sum(t_alone)
    rate = load * len(reqs) / t_seq
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    srv = sfsim.sf_server_create(0, 4)
    tickets = []
    t0 = time.perf_counter()
    for (plan, bits, sel, _, _), ta in zip(reqs, arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append(sfsim.sf_server_submit(srv, plan.handle, bits, sel))
    lat, same = [], True
    for t, (plan, bits, sel, _, _), a in zip(tickets, reqs, alone):
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
    b_load = sfsim.sf_server_stats(srv)
    sfsim.sf_server_destroy(srv)
    srv = sfsim.sf_server_create(0, 4)
    t1 = time.perf_counter()
    tk = [sfsim.sf_server_submit(srv, plan.handle, bits, sel) for plan, bits, sel, _, _ in reqs]
    for t, (plan, bits, sel, _, _), a in zip(tk, reqs, alone):
        same = same and bool(np.array_equal(sfsim.sf_server_wait(srv, t, len(bits)), a))
    saturated = time.perf_counter() - t1
    b_sat = sfsim.sf_server_stats(srv)
    sfsim.sf_server_destroy(srv)
    for plan in plans.values():
        plan.close()
    pred_win = sum(r[4] for r in reqs)
    return {"requests": len(reqs), "stream": n_req, "circuits": len(plans), "paths": int(paths),
            "offered_load": load,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "one_at_a_time_paths_per_s": paths / t_seq, "served_paths_per_s": paths / makespan,
            "saturated_paths_per_s": paths / saturated,
            "saturated_over_one_at_a_time": t_seq / saturated,
            "served_identical_to_alone": same, "makespan_s": makespan, "one_at_a_time_s": t_seq,
            "batches": {"at_load": {"batches": b_load[0], "requests": b_load[1], "largest": b_load[2]},
                        "saturated": {"batches": b_sat[0], "requests": b_sat[1], "largest": b_sat[2]}},
            "plan_seconds": t_plan,
            "window": f"the first {n_req} requests of the seeded mix, those the runtime model predicts at "
                      f"<= {max_pred_s:g} s ({len(reqs)} requests, {pred_win:.1f} s predicted)",
            "excluded": {"requests": excluded, "predicted_seconds": excl_pred,
                         "note": "the rest of the first requests, extrapolated by the runtime model fitted on "
                                 "this GPU"},
            "note": "at offered load rho < 1 the served rate equals the arrival rate (<= rho x capacity); "
                    "capacity is the saturated rate"}


def accuracy_7x8(sfsim, plan, bits):
    """The benchmark plan (its kernels, 1M bitstrings, compact finals) on the
    paths whose FP64 oracle amplitudes are stored: one whole 16-leaf group of
    the folded last level and 8 paths of other groups of the first prefix."""
    if not os.path.exists(GOLDEN_7X8):
        return None
    g = np.load(GOLDEN_7X8)
    ids, amps = g["ids"], g["amps"]
    k = amps.shape[1]
    if not np.array_equal(bits[:k], g["bits"]):
        return None
    a, _ = plan.amplitudes(bits, sfsim.selection("list", ids=ids))
    ref = amps.sum(axis=0)
    s = float(np.sqrt(np.mean(np.sum(np.abs(amps) ** 2, axis=0))))
    d = np.abs(a[:k] - ref)
    return {"paths": len(ids), "bitstrings_compared": int(k), "max_abs_err": float(d.max()),
            "max_err_over_path_scale": float(d.max() / s),
            "rms_err_over_path_scale": float(np.sqrt(np.mean(d ** 2)) / s),
            "max_err_times_2^(n/2)": float(d.max() * 2.0 ** 28),
            "bound": "3e-5 x path scale s = sqrt(mean_x sum_j |a_j(x)|^2)",
            "oracle": "stored FP64 values (tests/golden/oracle_7x8_d40_paths.npz, written from oracle/ only)"}


# ------------------------------------------------------ reference arm
def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores, same metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1807_10749_gb300 import inputs
    w = inputs.WORKLOADS[WORKLOAD]
    text = inputs.workload_circuit(WORKLOAD).text()
    bits = inputs.random_bitstrings(56, w["n_bitstrings"], w["bitstring_seed"])
    from oracle import sim
    sim.build()
    times, samples = [], []
    for step in range(args.warmup + args.steps):
        dt, ratio, _ = oracle_path_sample(text, w["side_b_mask"], bits, 0.125, step)
        if step >= args.warmup:
            times.append(dt * ratio)   # the seconds of one whole path
            samples.append(dt)
    total = sum(times)
    value = len(times) / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": config_dict(len(bits), {"reference": "FP64 CPU oracle (oracle/core.c, OpenMP)",
                                              "step": "one selected path x all 1M bitstrings, timed on the first "
                                                      "eighth of its gates and scaled by the gate-count ratio",
                                              "same_config": True}),
            "timing": {"measured_seconds_per_step": float(np.mean(samples)),
                       "extrapolated_seconds_per_path": float(np.mean(times)),
                       "measured_total_seconds": float(sum(samples)),
                       "note": "ms_per_step is the extrapolated time of a whole path; the measured seconds are "
                               "of the sampled eighth"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": sim.threads(), "kind": "oracle",
                             "sample": "per step one selected path (the step's prefix) of the 7x8 workload: the "
                                       "first eighth of both 28-qubit halves' gates in FP64 from |0> and the sum "
                                       "over all 1M bitstrings, scaled by the gate-count ratio to a whole path"},
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
    ap.add_argument("--no-suite", action="store_true", help="skip the other workloads and the runtime model")
    ap.add_argument("--exec-mode", default="batched", choices=["batched", "plain"])
    ap.add_argument("--workload", default=WORKLOAD, choices=["7x8_d40", "5x10_d16", "5x10_d14"])
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--fuse-bits", type=int, default=0)
    ap.add_argument("--run-bits", type=int, default=0)
    ap.add_argument("--split-last", type=int, default=0, choices=[0, 1],
                    help="1: run the level before the folded last level as its own segment")
    ap.add_argument("--fp32x2", type=int, default=1, choices=[0, 1],
                    help="1: packed FP32x2 arithmetic in the specialised kernels' Google-gate stages; 0: scalar")
    ap.add_argument("--dense-finals", type=int, default=0, choices=[0, 1],
                    help="1: the final programs write whole final states (no compact blocks)")
    ap.add_argument("--batch-paths", type=int, default=0,
                    help="finals (leaf groups) per block of the executor, 0: from the memory budget")
    ap.add_argument("--tile-buffers", type=int, default=0, choices=[0, 2, 3],
                    help="shared-memory tile buffers per CTA of the specialised kernels (0: per tile size)")
    ap.add_argument("--proj-side", type=int, default=0, choices=[0, 1],
                    help="0: Eq. 1's projector on half A of every cut CZ; 1: alternating halves")
    ap.add_argument("--cycle-segments", type=int, default=0, choices=[0, 1],
                    help="1: segments are the cycle ranges between branch levels (no light-cone scheduling)")
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
                      split_last=args.split_last, fp32x2=args.fp32x2, dense_finals=args.dense_finals,
                      projector_side=args.proj_side, tile_buffers=args.tile_buffers,
                      batch_paths=args.batch_paths, cycle_segments=args.cycle_segments)
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
    sfsim.sf_plan_status(plan.handle, stream)   # no kernel wait timed out
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

    # the headline step as a point of the runtime model: one 128-path range,
    # timed from the root (the timed steps reuse the previous step's upper
    # levels, which the model's features do not see)
    step_terms = sfsim.sf_plan_cost_terms(plan.handle, sels[args.warmup], len(bits))
    sfsim.sf_plan_drop_resident(plan.handle)
    ef0, ef1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ef0.record(stream)
    sfsim.sf_amplitudes_device(plan.handle, d_bits, sels[args.warmup], d_out, ws, stream=stream, accumulate=True)
    ef1.record(stream)
    torch.cuda.synchronize()
    step_fresh_s = ef0.elapsed_time(ef1) / 1e3
    accuracy = None
    if rank == 0 and args.workload == WORKLOAD and len(bits) == w["n_bitstrings"]:
        accuracy = accuracy_7x8(sfsim, plan, bits)

    plain = None
    if world == 1 and not args.no_plain and args.exec_mode == "batched":
        # the plain form: the same kernels, one path at a time from the prefix
        # checkpoint (no shared levels below it, no folded last level)
        pplan = sfsim.Plan(text, side_b_mask=w["side_b_mask"], exec_mode=sfsim.SF_EXEC_PLAIN,
                           tile_bits=args.tile_bits, fuse_bits=args.fuse_bits, run_bits=args.run_bits,
                           jit=args.jit, fp32x2=args.fp32x2)
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
    plan.close()
    del ws

    peak, peak_kind = measured_peaks()
    suite = model = serving = None
    if world == 1 and not args.no_suite and args.workload == WORKLOAD:
        coeffs, model = calibrate_runtime_model(sfsim, inputs, stream, [(step_terms, step_fresh_s)])
        # the headline request (all f = 0.5% paths, 1M bitstrings) in the model
        mplan = sfsim.Plan(text, side_b_mask=w["side_b_mask"], jit=0, hbm_budget_bytes=1 << 40)
        t7 = sfsim.sf_cost_predict(sfsim.sf_plan_cost_terms(mplan.handle, fsel, len(bits)), coeffs)
        mplan.close()
        model["headline_request_predicted_s"] = t7
        model["headline_request_measured_rate_s"] = n_sel / value
        model["cost_per_1M_amplitudes_gpu_hours_at_f_0.5%"] = (n_sel / value) / 3600.0 * 1e6 / len(bits)
        suite = other_configs(sfsim, inputs, peak, stream)
        if not args.no_serve:
            torch.cuda.empty_cache()   # the server allocates its own buffers
            serving = serving_window(sfsim, inputs, coeffs)

    if rank == 0:
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
            "accuracy_vs_oracle": accuracy,
            "plain_form": plain,
            "batched_over_plain": (value / plain["value"]) if plain else None,
            "serving": serving,
            "configs": suite,
            "runtime_model": model,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
