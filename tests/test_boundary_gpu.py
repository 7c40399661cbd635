"""The C ABI's reporting and output forms on the GPU: wait timeouts reported
by every form, probabilities, several requests in one batched call, the
compensated path sum, and results independent of how the finals are batched.

No test makes a kernel wait time out on the device. The flag a timed-out wait
would set is written from the host (sf_debug_set_wait_flag), or a timeout is
injected at the host-side check (sf_debug_inject_wait_timeouts); either way
the form must return SF_ECUDA and the plan must stay usable."""
import numpy as np
import pytest

from oracle import circuit as ocirc
from oracle import sim
from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu

TOL = 1e-5  # x 2^{-n/2}, the parity tolerance


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10749_gb300 import build
    build.build()
    sim.build()


@pytest.fixture(scope="module")
def c2():
    w = inputs.WORKLOADS["5x6_d24"]
    text = inputs.workload_circuit("5x6_d24").text()
    plan = sfsim.Plan(text, side_b_mask=w["side_b_mask"])
    yield plan, text, w
    plan.close()


def _dev(bits):
    import torch
    return torch.from_numpy(np.ascontiguousarray(bits).view(np.int64)).cuda()


def _host(d_out):
    import torch
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    return o[:, 0] + 1j * o[:, 1]


def _device_call(plan, bits, sel, start=None):
    import torch
    d_bits = _dev(bits)
    d_out = (torch.zeros((len(bits), 2), dtype=torch.float64, device="cuda") if start is None
             else start.clone())
    ws = torch.empty(sfsim.sf_workspace_size(plan.handle, len(bits), sel), dtype=torch.uint8, device="cuda")
    sfsim.sf_amplitudes_device(plan.handle, d_bits, sel, d_out, ws, accumulate=start is not None)
    return _host(d_out)


def test_wait_timeouts_are_reported_by_every_form(c2):
    import torch
    plan, _, w = c2
    bits = inputs.random_bitstrings(30, 3000, 21)
    sel = sfsim.selection("range", first=100, count=300)
    want = plan.amplitudes(bits, sel)[0]
    try:
        # host form: the device flag set (as a timed-out kernel would) ...
        sfsim.sf_debug_set_wait_flag(plan.handle, 1)
        with pytest.raises(sfsim.SFError) as e:
            plan.amplitudes(bits, sel)
        assert e.value.code == sfsim.SF_ECUDA and "timed out" in str(e.value)
        # ... is cleared by the report: the next call succeeds, same result
        assert np.array_equal(plan.amplitudes(bits, sel)[0], want)
        # host form, injected at the check
        sfsim.sf_debug_inject_wait_timeouts(1)
        with pytest.raises(sfsim.SFError) as e:
            sfsim.sf_probabilities(plan.handle, bits, sel)
        assert e.value.code == sfsim.SF_ECUDA
        # device form: reported by sf_plan_status, then clear
        d_bits = _dev(bits)
        d_out = torch.zeros((len(bits), 2), dtype=torch.float64, device="cuda")
        ws = torch.empty(sfsim.sf_workspace_size(plan.handle, len(bits), sel), dtype=torch.uint8, device="cuda")
        sfsim.sf_amplitudes_device(plan.handle, d_bits, sel, d_out, ws)
        sfsim.sf_debug_set_wait_flag(plan.handle, 1)
        with pytest.raises(sfsim.SFError) as e:
            sfsim.sf_plan_status(plan.handle)
        assert e.value.code == sfsim.SF_ECUDA
        sfsim.sf_plan_status(plan.handle)
        # batch form
        reqs = [(d_bits, sel, d_out, False)]
        ws2 = torch.empty(sfsim.sf_workspace_size_batch(plan.handle, reqs), dtype=torch.uint8, device="cuda")
        sfsim.sf_amplitudes_device_batch(plan.handle, reqs, ws2)
        sfsim.sf_debug_inject_wait_timeouts(1)
        with pytest.raises(sfsim.SFError) as e:
            sfsim.sf_plan_status(plan.handle)
        assert e.value.code == sfsim.SF_ECUDA
        # fixed-scratch form
        sfsim.sf_amplitudes_device_noalloc(plan.handle, d_bits, sel, d_out)
        sfsim.sf_debug_set_wait_flag(plan.handle, 1)
        with pytest.raises(sfsim.SFError) as e:
            sfsim.sf_plan_status(plan.handle)
        assert e.value.code == sfsim.SF_ECUDA
        assert np.array_equal(_host(d_out), want)   # the data itself was complete
        # server: the worker's check fails the request, the next one succeeds
        srv = sfsim.sf_server_create(0, 1)
        try:
            sfsim.sf_debug_inject_wait_timeouts(1)
            t = sfsim.sf_server_submit(srv, plan.handle, bits, sel)
            with pytest.raises(sfsim.SFError) as e:
                sfsim.sf_server_wait(srv, t, len(bits))
            assert e.value.code == sfsim.SF_ECUDA
            t = sfsim.sf_server_submit(srv, plan.handle, bits, sel)
            assert np.array_equal(sfsim.sf_server_wait(srv, t, len(bits)), want)
        finally:
            sfsim.sf_server_destroy(srv)
    finally:
        sfsim.sf_debug_inject_wait_timeouts(0)
    sfsim.sf_plan_status(plan.handle)


def test_probabilities_host_and_device(c2):
    import torch
    plan, _, _ = c2
    bits = inputs.random_bitstrings(30, 5001, 22)
    sel = sfsim.selection("fraction", fidelity=1 / 8, seed=3)
    amp, fa = plan.amplitudes(bits, sel)
    p, fa2 = sfsim.sf_probabilities(plan.handle, bits, sel)
    assert fa2 == fa and 0 < fa < 1
    assert np.array_equal(p, amp.real * amp.real + amp.imag * amp.imag)
    q, _ = sfsim.sf_probabilities(plan.handle, bits, sel, divide_by_f=True)
    assert np.array_equal(q, (amp.real * amp.real + amp.imag * amp.imag) * (1.0 / fa))
    d_amp = torch.from_numpy(np.stack([amp.real, amp.imag], 1).copy()).cuda()
    d_p = torch.empty(len(bits), dtype=torch.float64, device="cuda")
    sfsim.sf_probabilities_device(d_amp, d_p, scale=2.0)
    torch.cuda.synchronize()
    assert np.array_equal(d_p.cpu().numpy(), p * 2.0)


def test_batch_equals_each_request_alone(c2):
    """Three requests on one plan (different selections and bitstrings, one
    accumulating) in one batched call: each bit for bit as alone."""
    import torch
    plan, _, _ = c2
    cases = [(inputs.random_bitstrings(30, 4000, 31), sfsim.selection("range", first=2048, count=700), False),
             (inputs.random_bitstrings(30, 777, 32), sfsim.selection("fraction", fidelity=1 / 16, seed=9), False),
             (inputs.random_bitstrings(30, 2500, 33), sfsim.selection("list", ids=[5, 2100, 2101, 30000]), True)]
    start = torch.from_numpy(np.random.default_rng(4).normal(size=(2500, 2)) * 1e-5).cuda()
    alone = [_device_call(plan, b, s, start if acc else None) for b, s, acc in cases]
    reqs, outs = [], []
    for b, s, acc in cases:
        d_out = start.clone() if acc else torch.full((len(b), 2), 3.0, dtype=torch.float64, device="cuda")
        outs.append(d_out)
        reqs.append((_dev(b), s, d_out, acc))
    ws = torch.empty(sfsim.sf_workspace_size_batch(plan.handle, reqs), dtype=torch.uint8, device="cuda")
    sfsim.sf_amplitudes_device_batch(plan.handle, reqs, ws)
    sfsim.sf_plan_status(plan.handle)
    for got, want in zip(outs, alone):
        assert np.array_equal(_host(got), want)


def test_result_does_not_depend_on_the_batch_size(c2):
    """The path sum adds the finals in path order whatever their grouping into
    launches: a budget that forces small blocks gives the same bits."""
    plan, text, w = c2
    bits = inputs.random_bitstrings(30, 3000, 41)
    sel = sfsim.selection("fraction", fidelity=1 / 4, seed=5)
    want = plan.amplitudes(bits, sel)[0]
    node = 2 * (1 << 15) * 8
    for batch in (1, 3, 64):
        small = sfsim.Plan(text, side_b_mask=w["side_b_mask"], batch_paths=batch)
        assert np.array_equal(small.amplitudes(bits, sel)[0], want), batch
        small.close()
    tight = sfsim.Plan(text, side_b_mask=w["side_b_mask"], hbm_budget_bytes=40 * node)
    assert np.array_equal(tight.amplitudes(bits, sel)[0], want)
    tight.close()


@pytest.mark.parametrize("jit", [0, 1])
def test_compensated_path_sum(c2, jit):
    """SF_PREC_COMPENSATED: Neumaier-compensated FP64 path sum. Within the
    parity tolerance of the oracle, and of the plain FP64 sum to far below it;
    batched and alone bit for bit."""
    import torch
    _, text, w = c2
    bits = inputs.random_bitstrings(30, 20000, 51)
    sel = sfsim.selection("fraction", fidelity=1.0)
    plain = sfsim.Plan(text, side_b_mask=w["side_b_mask"], jit=jit)
    comp = sfsim.Plan(text, side_b_mask=w["side_b_mask"], jit=jit, precision=sfsim.SF_PREC_COMPENSATED)
    a = plain.amplitudes(bits, sel)[0]
    b = comp.amplitudes(bits, sel)[0]
    scale = 2.0 ** -15
    d = np.abs(a - b).max()
    print(f"compensated vs FP64 sum over 2^15 paths: max|d| = {d:.3e} = {d / scale:.2e} * 2^-n/2")
    assert d <= 1e-9 * scale
    c = ocirc.parse(text)
    ref = sim.sv_amplitudes(c, bits[:2000])
    err = np.abs(b[:2000] - ref).max()
    print(f"compensated vs oracle state vector: max|d| = {err / scale:.2e} * 2^-n/2")
    assert err <= TOL * scale
    # accumulate into an existing output, and batched with another request
    d_bits = _dev(bits)
    start = torch.from_numpy(np.random.default_rng(6).normal(size=(len(bits), 2)) * 1e-6).cuda()
    out1 = start.clone()
    ws = torch.empty(sfsim.sf_workspace_size(comp.handle, len(bits), sel), dtype=torch.uint8, device="cuda")
    sfsim.sf_amplitudes_device(comp.handle, d_bits, sel, out1, ws, accumulate=True)
    out2 = start.clone()
    other = torch.zeros((100, 2), dtype=torch.float64, device="cuda")
    reqs = [(d_bits, sel, out2, True), (d_bits[:100], sfsim.selection("range", count=5), other, False)]
    ws2 = torch.empty(sfsim.sf_workspace_size_batch(comp.handle, reqs), dtype=torch.uint8, device="cuda")
    sfsim.sf_amplitudes_device_batch(comp.handle, reqs, ws2)
    assert np.array_equal(_host(out1), _host(out2))
    st = start.cpu().numpy()
    assert np.abs(_host(out1) - (st[:, 0] + 1j * st[:, 1]) - b).max() <= 1e-12 * scale
    plain.close()
    comp.close()


def test_plans_sharing_one_workspace_never_reuse_each_others_nodes(c2):
    """A plan reuses the path-tree nodes it left in a workspace on its next
    call; when another plan ran in the same workspace in between, nothing is
    reused. Two plans (5x6 and 4x5) alternate on one workspace; each call
    equals the same call on a fresh workspace, bit for bit."""
    import torch
    plan_a, _, _ = c2
    mask_b = inputs.column_cut_mask(4, 5, 2)
    plan_b = sfsim.Plan(inputs.google_circuit(4, 5, 20, 2).text(), side_b_mask=mask_b)
    bits_a = inputs.random_bitstrings(30, 2000, 61)
    bits_b = inputs.random_bitstrings(20, 2000, 62)
    # ranges valid for both plans (the 4x5 circuit has 2^10 paths)
    sel = [sfsim.selection("range", first=256 * i, count=200) for i in range(3)]
    want_a = [_device_call(plan_a, bits_a, s) for s in sel]
    want_b = [_device_call(plan_b, bits_b, s) for s in sel]
    need = max(sfsim.sf_workspace_size(p.handle, 2000, s) for p in (plan_a, plan_b) for s in sel)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    da, db = _dev(bits_a), _dev(bits_b)
    for i, s in enumerate(sel):
        for plan, d_bits, want in ((plan_a, da, want_a), (plan_b, db, want_b)):
            d_out = torch.zeros((2000, 2), dtype=torch.float64, device="cuda")
            sfsim.sf_amplitudes_device(plan.handle, d_bits, s, d_out, ws)
            assert np.array_equal(_host(d_out), want[i])
    # the caller overwrites the workspace: after sf_plan_drop_resident the
    # plan recomputes everything
    sfsim.sf_amplitudes_device(plan_a.handle, da, sel[0], torch.zeros((2000, 2), dtype=torch.float64, device="cuda"), ws)
    ws.fill_(0x7f)
    sfsim.sf_plan_drop_resident(plan_a.handle)
    d_out = torch.zeros((2000, 2), dtype=torch.float64, device="cuda")
    sfsim.sf_amplitudes_device(plan_a.handle, da, sel[0], d_out, ws)
    assert np.array_equal(_host(d_out), want_a[0])
    plan_b.close()
