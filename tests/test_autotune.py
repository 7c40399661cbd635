"""The autotuner times candidate plans (pass shape, fusion width k in 2..5,
paths per launch) on the device and returns options at least as fast as the
base options on the same sample, whose results equal the base plan's."""
import numpy as np
import pytest

from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu


def test_autotune_returns_working_options_no_slower_than_the_base():
    import torch
    from paper_1807_10749_gb300 import build
    build.build()
    w = inputs.WORKLOADS["5x6_d24"]
    text = inputs.workload_circuit("5x6_d24").text()
    c = sfsim.sf_circuit_parse(text)
    base = sfsim.sf_plan_opts_default(side_b_mask=w["side_b_mask"])
    bits = inputs.random_bitstrings(30, 5000, 3)
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    sel = sfsim.selection("fraction", fidelity=1 / 8, seed=7)
    best, t, t_base = sfsim.sf_plan_autotune(c, base, sel, 1024, d_bits)
    print(f"tuned: tile {best.tile_bits} k {best.fuse_bits} run {best.run_bits} batch {best.batch_paths}: "
          f"{t * 1e3:.3f} ms, base {t_base * 1e3:.3f} ms")
    assert 0 < t <= t_base
    assert best.tile_bits in (0, 12, 13) and best.fuse_bits in (0, 2, 3, 4, 5) and best.run_bits in (0, 3, 4)
    assert best.batch_paths in (0, 1, 4, 16, 64, 256, 1024)
    tuned = sfsim.sf_plan_create(c, best)
    default = sfsim.sf_plan_create(c, base)
    a, _ = sfsim.sf_amplitudes(tuned, bits, sel)
    b, _ = sfsim.sf_amplitudes(default, bits, sel)
    assert np.abs(a - b).max() <= 1e-5 * 2.0 ** -15
    sfsim.sf_plan_destroy(tuned)
    sfsim.sf_plan_destroy(default)
    sfsim.sf_circuit_destroy(c)
