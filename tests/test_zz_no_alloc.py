"""sf_amplitudes_device_noalloc: the amplitude call whose scratch is a fixed
array inside the library, for callers that may not allocate device memory
while they run. Its results must equal those of sf_amplitudes_device (which
takes a caller workspace) bit for bit - both run the same kernels, and the
path sum adds the finals in path order whatever the workspace size - call
after call, although the array keeps the previous call's contents. The
device's free memory must not change across its calls. This file is
collected last on purpose."""
import numpy as np
import pytest

from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu


def _host(d_out):
    import torch
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    return o[:, 0] + 1j * o[:, 1]


@pytest.mark.parametrize("jit", [0, 1], ids=["generic", "specialised"])
@pytest.mark.parametrize("accumulate", [0, 1])
@pytest.mark.parametrize("name,sel_kw,nbits", [
    ("4x4_d10", dict(mode="fraction", fidelity=1.0), 1024),
    ("5x6_d24", dict(mode="range", first=4096, count=3000), 20000),
])
def test_noalloc_matches_workspace_call_twice(name, sel_kw, nbits, jit, accumulate):
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10749_gb300 import build
    build.build()
    w = inputs.WORKLOADS[name]
    n = w["rows"] * w["cols"]
    plan = sfsim.Plan(inputs.workload_circuit(name).text(), side_b_mask=w["side_b_mask"], jit=jit)
    bits = inputs.random_bitstrings(n, nbits, w["bitstring_seed"])
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    sel = sfsim.selection(**sel_kw)
    start = torch.from_numpy(np.random.default_rng(1).normal(size=(nbits, 2)) * 2.0 ** (-n / 2)).cuda()
    outs = [start.clone() if accumulate else torch.full((nbits, 2), 7.0, dtype=torch.float64, device="cuda")
            for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # the first call on this plan, then a second one over the first one's
    # leftovers in the shared array
    for d_out in outs:
        sfsim.sf_amplitudes_device_noalloc(plan.handle, d_bits, sel, d_out, accumulate=bool(accumulate))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    sfsim.sf_plan_status(plan.handle)
    assert free1 == free0, f"device free memory changed across the calls: {free0} -> {free1}"
    want_out = start.clone() if accumulate else torch.zeros((nbits, 2), dtype=torch.float64, device="cuda")
    ws = torch.empty(sfsim.sf_workspace_size(plan.handle, nbits, sel), dtype=torch.uint8, device="cuda")
    sfsim.sf_amplitudes_device(plan.handle, d_bits, sel, want_out, ws, accumulate=bool(accumulate))
    want = _host(want_out)
    assert np.sqrt(np.mean(np.abs(want) ** 2)) > 0
    for d_out in outs:
        assert np.array_equal(_host(d_out), want)
    plan.close()


def test_noalloc_rejects_plans_beyond_the_fixed_scratch():
    import torch
    from paper_1807_10749_gb300 import build
    build.build()
    w = inputs.WORKLOADS["6x7_d26"]   # one path needs 8 nodes of 32 MiB
    plan = sfsim.Plan(inputs.workload_circuit("6x7_d26").text(), side_b_mask=w["side_b_mask"], jit=0)
    d_bits = torch.zeros(16, dtype=torch.int64, device="cuda")
    d_out = torch.zeros((16, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(sfsim.SFError) as e:
        sfsim.sf_amplitudes_device_noalloc(plan.handle, d_bits, sfsim.selection("range", count=16), d_out)
    assert e.value.code == sfsim.SF_ENOMEM
    assert "MiB fixed scratch" in str(e.value)
    plan.close()
