"""sf_amplitudes_device_noalloc: the amplitude call whose scratch is a fixed
array inside the library, for callers that may not allocate device memory
while they run. Its results must equal those of sf_amplitudes_device (which
takes a caller workspace), call after call, although the array keeps the
previous call's contents. This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-5  # x 2^{-n/2}, the tolerance of the parity tests


def _device_call(plan, d_bits, sel, n):
    import torch
    d_out = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    ws = torch.empty(sfsim.sf_workspace_size(plan.handle, n, sel), dtype=torch.uint8, device="cuda")
    sfsim.sf_amplitudes_device(plan.handle, d_bits, sel, d_out, ws)
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    return o[:, 0] + 1j * o[:, 1]


def _noalloc_call(plan, d_bits, sel, n):
    import torch
    d_out = torch.full((n, 2), 7.0, dtype=torch.float64, device="cuda")  # overwritten
    sfsim.sf_amplitudes_device_noalloc(plan.handle, d_bits, sel, d_out)
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    return o[:, 0] + 1j * o[:, 1]


@pytest.mark.parametrize("name,sel_kw,nbits", [
    ("4x4_d10", dict(mode="fraction", fidelity=1.0), 1024),
    ("5x6_d24", dict(mode="range", first=4096, count=3000), 20000),
])
def test_noalloc_matches_workspace_call_twice(name, sel_kw, nbits):
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10749_gb300 import build
    build.build()
    w = inputs.WORKLOADS[name]
    n = w["rows"] * w["cols"]
    plan = sfsim.Plan(inputs.workload_circuit(name).text(), side_b_mask=w["side_b_mask"])
    bits = inputs.random_bitstrings(n, nbits, w["bitstring_seed"])
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    sel = sfsim.selection(**sel_kw)
    want = _device_call(plan, d_bits, sel, len(bits))
    scale = 2.0 ** (-n / 2)
    for _ in range(2):  # the second call starts from the first call's leftovers
        got = _noalloc_call(plan, d_bits, sel, len(bits))
        assert np.abs(got - want).max() <= ABS_TOL * scale
        assert np.sqrt(np.mean(np.abs(want) ** 2)) > 0
    plan.close()


def test_noalloc_rejects_plans_beyond_the_fixed_scratch():
    import torch
    from paper_1807_10749_gb300 import build
    build.build()
    w = inputs.WORKLOADS["6x7_d26"]   # one path needs 8 nodes of 32 MiB
    plan = sfsim.Plan(inputs.workload_circuit("6x7_d26").text(), side_b_mask=w["side_b_mask"])
    d_bits = torch.zeros(16, dtype=torch.int64, device="cuda")
    d_out = torch.zeros((16, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(sfsim.SFError) as e:
        sfsim.sf_amplitudes_device_noalloc(plan.handle, d_bits, sfsim.selection("range", count=16), d_out)
    assert e.value.code == sfsim.SF_ENOMEM
    assert "MiB fixed scratch" in str(e.value)
    plan.close()
