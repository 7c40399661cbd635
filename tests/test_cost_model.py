"""Runtime model of Section 8 (Eq. t_tot) on the GPU: calibrate C1..C3 from
measured requests, check its predictions, and the server admission policy
that uses it (shortest predicted request first)."""
import time

import numpy as np
import pytest

from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10749_gb300 import build
    build.build()


def _timed(plan, bits, sel):
    """Device seconds of one request, fresh workspace (no resident nodes)."""
    import torch
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    d_out = torch.zeros((len(bits), 2), dtype=torch.float64, device="cuda")
    ws = torch.empty(sfsim.sf_workspace_size(plan.handle, len(bits), sel), dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    sfsim.sf_amplitudes_device(plan.handle, d_bits, sel, d_out, ws)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _configs():
    """4 circuits x 3 fidelities x 2 bitstring counts, plus the 5x6 circuit
    with path-level selection (x_p = x, so d_p and x_b differ)."""
    out = []
    for (R, C, D, cut, xs) in [(5, 6, 24, ("col", 3), -1), (4, 5, 24, ("col", 2), -1),
                               (6, 6, 20, ("col", 3), -1), (5, 5, 28, ("row", 2), -1),
                               (5, 6, 24, ("col", 3), 64)]:
        mask = (inputs.column_cut_mask if cut[0] == "col" else inputs.row_cut_mask)(R, C, cut[1])
        text = inputs.google_circuit(R, C, D, 3).text()
        for f in (1 / 16, 1 / 4, 1.0):
            for n_a in (10_000, 200_000):
                out.append((text, mask, R * C, f, n_a, xs))
    return out


def test_calibrated_model_predicts_request_times():
    plans = {}
    T, S, names = [], [], []
    for text, mask, n, f, n_a, xs in _configs():
        key = (text, mask, xs)
        if key not in plans:
            plans[key] = sfsim.Plan(text, side_b_mask=mask, select_prefix_bits=xs)
        plan = plans[key]
        bits = inputs.random_bitstrings(n, n_a, 11)
        sel = sfsim.selection("fraction", fidelity=f, seed=3)
        _timed(plan, bits, sel)                      # warm-up (tables, allocator)
        S.append(min(_timed(plan, bits, sel) for _ in range(2)))
        T.append(sfsim.sf_plan_cost_terms(plan.handle, sel, n_a))
        names.append(f"{n}q{'' if xs < 0 else ' xs=x'} f={f:.3g} n_a={n_a}")
    T, S = np.array(T), np.array(S)
    coeffs = sfsim.sf_cost_fit(T, S)
    pred = np.array([sfsim.sf_cost_predict(t, coeffs) for t in T])
    rel = np.abs(pred - S) / S
    for nm, s, p_ in zip(names, S, pred):
        print(f"{nm:28s} measured {s * 1e3:9.3f} ms  predicted {p_ * 1e3:9.3f} ms")
    c0, c1, c1c2, c3 = coeffs
    print(f"C0 = {c0:.3e} s, C1 = {c1:.3e} s, C1*C2 = {c1c2:.3e} s, C3 = {c3:.3e} s per path-amplitude; "
          f"median |rel err| {np.median(rel):.3f}, max {rel.max():.3f}")
    assert np.all(coeffs >= 0) and c3 > 0 and (c1 > 0 or c1c2 > 0)
    # Eq. t_tot models a prefix/suffix split; the executor caches every tree
    # level and runs each gate at the depth of the light cone that reaches
    # it, so the fit carries a model error of its own: median 0.25-0.35 on
    # this set over repeated runs, the 5x6 prefix selections under-predicted
    assert np.median(rel) < 0.4
    for p_ in plans.values():
        p_.close()


def _times_when_done(srv, ticket, limit_s=600.0):
    t_end = time.time() + limit_s
    while True:
        try:
            return sfsim.sf_server_times(srv, ticket)
        except sfsim.SFError as e:
            if e.code != sfsim.SF_ETIMEOUT or time.time() > t_end:
                raise
            time.sleep(0.01)


def test_server_admits_shortest_predicted_first():
    """With the model set, a small request submitted after a large one is
    admitted first; without it, arrival order holds."""
    w = inputs.WORKLOADS["6x7_d26"]
    long_plan = sfsim.Plan(inputs.workload_circuit("6x7_d26").text(), side_b_mask=w["side_b_mask"])
    big = sfsim.Plan(inputs.workload_circuit("5x6_d24").text(),
                     side_b_mask=inputs.WORKLOADS["5x6_d24"]["side_b_mask"])
    small = sfsim.Plan(inputs.workload_circuit("4x4_d10").text(),
                       side_b_mask=inputs.WORKLOADS["4x4_d10"]["side_b_mask"])
    b_long = inputs.random_bitstrings(42, 2000, 1)
    b_big = inputs.random_bitstrings(30, 100_000, 2)
    b_small = inputs.random_bitstrings(16, 100, 3)
    s_long = sfsim.selection("fraction", fidelity=1.0)   # all 2^25 paths: seconds of work
    s_all = sfsim.selection("fraction", fidelity=1.0)
    order = {}
    for use_model in (False, True):
        srv = sfsim.sf_server_create(0, 1)
        try:
            if use_model:
                sfsim.sf_server_set_cost_model(srv, [1e-4, 1e-12, 1e-12, 1e-9], max_wait_s=600.0)
            t0 = sfsim.sf_server_submit(srv, long_plan.handle, b_long, s_long)
            time.sleep(0.3)      # the long request is running
            tb = sfsim.sf_server_submit(srv, big.handle, b_big, s_all)
            ts = sfsim.sf_server_submit(srv, small.handle, b_small, s_all)
            sfsim.sf_server_cancel(srv, t0)   # frees the worker with both queued
            qb = _times_when_done(srv, tb)[0]
            qs = _times_when_done(srv, ts)[0]
            with pytest.raises(sfsim.SFError):
                sfsim.sf_server_wait(srv, t0, len(b_long))
            for t, n in ((tb, len(b_big)), (ts, len(b_small))):
                sfsim.sf_server_wait(srv, t, n)
            order[use_model] = (qb, qs)
        finally:
            sfsim.sf_server_destroy(srv)
    print("queued (big, small): arrival order", order[False], "model", order[True])
    assert order[False][0] < order[False][1]     # arrival order: big first
    assert order[True][1] < order[True][0]       # model: small first
    for p_ in (long_plan, big, small):
        p_.close()
