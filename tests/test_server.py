"""Request server: continuous batching, admission by device footprint,
cancellation, and results identical alone and in a mix."""
import time

import numpy as np
import pytest

from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plans():
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10749_gb300 import build
    build.build()
    out = {}
    for name, (R, C, D, mask) in {
        "4x4": (4, 4, 12, inputs.row_cut_mask(4, 4, 2)),
        "4x5": (4, 5, 20, inputs.column_cut_mask(4, 5, 2)),
        "5x6": (5, 6, 20, inputs.column_cut_mask(5, 6, 3)),
        "6x6": (6, 6, 18, inputs.column_cut_mask(6, 6, 3)),
    }.items():
        spec = inputs.google_circuit(R, C, D, 3)
        out[name] = (sfsim.Plan(spec.text(), side_b_mask=mask), R * C)
    w = inputs.WORKLOADS["6x7_d26"]
    out["long"] = (sfsim.Plan(inputs.workload_circuit("6x7_d26").text(), side_b_mask=w["side_b_mask"]), 42)
    yield out
    for p, _ in out.values():
        p.close()


def _requests(plans, n_req, seed):
    rng = np.random.default_rng(seed)
    names = sorted(k for k in plans if k != "long")
    reqs = []
    for i in range(n_req):
        name = names[rng.integers(len(names))]
        plan, n = plans[name]
        f = float(np.exp(rng.uniform(np.log(0.02), 0.0)))
        nb = int(rng.integers(200, 5000))
        bits = inputs.random_bitstrings(n, nb, 5000 + i)
        reqs.append((plan, bits, sfsim.selection("fraction", fidelity=f, seed=11 + i)))
    return reqs


def test_results_equal_alone_and_in_the_mix(plans):
    reqs = _requests(plans, 24, 1)
    alone = [p.amplitudes(b, s)[0] for p, b, s in reqs]
    srv = sfsim.sf_server_create(0, 4)
    try:
        tickets = [sfsim.sf_server_submit(srv, p.handle, b, s) for p, b, s in reqs]
        for t, a, (p, b, s) in zip(tickets, alone, reqs):
            got = sfsim.sf_server_wait(srv, t, len(b))
            assert np.array_equal(got, a)
    finally:
        sfsim.sf_server_destroy(srv)


def test_admission_by_footprint_and_latency(plans):
    plan, n = plans["5x6"]
    bits = inputs.random_bitstrings(n, 1000, 3)
    sel = sfsim.selection("fraction", fidelity=1.0)
    ws = sfsim.sf_workspace_size(plan.handle, len(bits), sel)
    one = ws + 24 * len(bits)
    # a budget that admits one such request at a time
    srv = sfsim.sf_server_create(one + one // 2, 4)
    try:
        big = inputs.random_bitstrings(n, one // 24, 4)   # its bitstrings alone exceed the rest
        with pytest.raises(sfsim.SFError) as e:
            sfsim.sf_server_submit(srv, plan.handle, big, sel)
        assert e.value.code == sfsim.SF_ENOMEM
        ts = [sfsim.sf_server_submit(srv, plan.handle, bits, sel) for _ in range(3)]
        want = plan.amplitudes(bits, sel)[0]
        res = []
        for t in ts:
            while True:
                try:
                    res.append(sfsim.sf_server_wait(srv, t, len(bits), timeout_ms=10))
                    break
                except sfsim.SFError as err:
                    assert err.code == sfsim.SF_ETIMEOUT
        for r in res:
            assert np.array_equal(r, want)
    finally:
        sfsim.sf_server_destroy(srv)


def test_cancel_queued_and_running(plans):
    plan, n = plans["long"]   # 6x7, all 2^25 paths: minutes of work
    bits = inputs.random_bitstrings(n, 2000, 6)
    sel = sfsim.selection("fraction", fidelity=1.0)
    srv = sfsim.sf_server_create(0, 1)
    try:
        t1 = sfsim.sf_server_submit(srv, plan.handle, bits, sel)
        t2 = sfsim.sf_server_submit(srv, plan.handle, bits, sel)
        time.sleep(0.5)
        sfsim.sf_server_cancel(srv, t2)   # still queued behind t1
        sfsim.sf_server_cancel(srv, t1)   # running: stops at the next path block
        for t in (t1, t2):
            with pytest.raises(sfsim.SFError) as e:
                sfsim.sf_server_wait(srv, t, len(bits))
            assert e.value.code in (sfsim.SF_ECANCELLED,)
        # the server keeps working after cancellations
        small, _ = plans["4x4"]
        b2 = inputs.random_bitstrings(16, 100, 7)
        s2 = sfsim.selection("fraction", fidelity=1.0)
        t3 = sfsim.sf_server_submit(srv, small.handle, b2, s2)
        assert np.array_equal(sfsim.sf_server_wait(srv, t3, len(b2)), small.amplitudes(b2, s2)[0])
    finally:
        sfsim.sf_server_destroy(srv)


def test_failed_request_does_not_affect_others(plans):
    plan, n = plans["4x5"]
    bits = inputs.random_bitstrings(n, 500, 8)
    srv = sfsim.sf_server_create(0, 2)
    try:
        with pytest.raises(sfsim.SFError) as e:
            sfsim.sf_server_submit(srv, plan.handle, bits, sfsim.selection("list", ids=[3, 3]))
        assert e.value.code == sfsim.SF_EINVAL
        sel = sfsim.selection("range", first=0, count=64)
        t = sfsim.sf_server_submit(srv, plan.handle, bits, sel)
        assert np.array_equal(sfsim.sf_server_wait(srv, t, len(bits)), plan.amplitudes(bits, sel)[0])
    finally:
        sfsim.sf_server_destroy(srv)


def test_queued_requests_on_one_plan_run_as_one_batch(plans):
    """Requests that queue up on one plan while the only worker is busy run
    together as one batch (one path tree, every pass launch carrying all of
    them); each result is bit for bit the request's result alone."""
    long_plan, n_long = plans["long"]
    plan, n = plans["5x6"]
    reqs = [(inputs.random_bitstrings(n, 300 + 100 * i, 70 + i),
             sfsim.selection("fraction", fidelity=[1.0, 0.25, 0.5, 1 / 16, 1.0][i], seed=3 + i)) for i in range(5)]
    alone = [plan.amplitudes(b, s)[0] for b, s in reqs]
    srv = sfsim.sf_server_create(0, 1)
    try:
        b_long = inputs.random_bitstrings(n_long, 500, 9)
        # 2^23 paths: seconds of work, so the worker is still busy with it
        # when the five requests below have been submitted
        t0 = sfsim.sf_server_submit(srv, long_plan.handle, b_long, sfsim.selection("fraction", fidelity=1 / 4))
        time.sleep(0.2)   # the long request occupies the worker
        tickets = [sfsim.sf_server_submit(srv, plan.handle, b, s) for b, s in reqs]
        sfsim.sf_server_wait(srv, t0, len(b_long))
        for t, (b, s), a in zip(tickets, reqs, alone):
            assert np.array_equal(sfsim.sf_server_wait(srv, t, len(b)), a)
        batches, requests, largest = sfsim.sf_server_stats(srv)
        print("server batches", batches, "requests", requests, "largest", largest)
        assert requests == 6 and largest == 5 and batches == 2
    finally:
        sfsim.sf_server_destroy(srv)
