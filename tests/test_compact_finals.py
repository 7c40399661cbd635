"""Compact finals on the GPU: the last pass of each half's final program
writes only the blocks of 2^g amplitudes that hold a requested bitstring, and
the gather reads them from their slots. The stored values and the gather's
summation order are those of the dense finals, so the results must be equal
bit for bit; the dense form itself is held to the oracle by the parity tests.
Cases: duplicates and a ragged count, one bitstring, partial leaf groups of
the folded level, both kernel forms, the 7x8 workload at its bench size, and
a bitstring count at which the planner keeps dense finals."""
import numpy as np
import pytest

from oracle import circuit as ocirc
from oracle import sim
from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1807_10749_gb300 import build
    build.build()
    sim.build()


def _ws(plan, n, sel):
    return sfsim.sf_workspace_size(plan.handle, n, sel)


def _pass_bytes(plan, bits, sel):
    sfsim.sf_plan_profile(plan.handle, True)
    a, _ = plan.amplitudes(bits, sel)
    launches, _, b = sfsim.sf_plan_profile_read(plan.handle, 0)
    other = sfsim.sf_plan_profile_read(plan.handle, 2)[0]
    return a, b, launches, other


@pytest.mark.parametrize("jit", [0, 1], ids=["generic", "specialised"])
def test_6x7_compact_equals_dense(jit):
    w = inputs.WORKLOADS["6x7_d26"]
    text = inputs.workload_circuit("6x7_d26").text()
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    q = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"], dense_finals=1)
    bits = inputs.random_bitstrings(42, 3001, 21)
    bits = np.concatenate([bits, bits[:7], bits[100:101]])   # duplicates, ragged count
    for sel in (sfsim.selection("range", first=1 << 12, count=64),     # 4 whole leaf groups
                sfsim.selection("range", first=(1 << 12) + 5, count=40),  # partial groups
                sfsim.selection("fraction", fidelity=1 / 4096, seed=3)):
        for b in (bits, bits[:1]):
            assert _ws(p, len(b), sel) > _ws(q, len(b), sel), "compact finals not in use"
            a, bytes_c, la, oa = _pass_bytes(p, b, sel)
            d, bytes_d, ld, od = _pass_bytes(q, b, sel)
            assert np.abs(d).max() > 0
            assert np.array_equal(a, d), np.abs(a - d).max()
            # same pass launches; fewer bytes written; the block maps are built
            assert la == ld and bytes_c < bytes_d
            assert oa >= od + 4
    # 200k bitstrings: the blocks would fill more than a quarter of a half
    big = inputs.random_bitstrings(42, 200000, 4)
    sel = sfsim.selection("range", first=1 << 12, count=16)
    assert _ws(p, len(big), sel) == _ws(q, len(big), sel)
    a, _ = p.amplitudes(big, sel)
    d, _ = q.amplitudes(big, sel)
    assert np.array_equal(a, d)
    p.close()
    q.close()


def test_6x7_compact_matches_oracle():
    """A seeded path list (12 random paths and one whole leaf group of the
    folded level) through the compact finals against the oracle's path sum,
    on a ragged bitstring count."""
    w = inputs.WORKLOADS["6x7_d26"]
    text = inputs.workload_circuit("6x7_d26").text()
    setup = sim.SFSetup(ocirc.parse(text), w["side_b_mask"])
    bits = inputs.random_bitstrings(42, 700, 8)
    ids = inputs.random_path_list(setup.x_bits, 12, 11)
    grp = (int(ids[0]) >> 4) << 4
    ids = np.unique(np.concatenate([ids, np.arange(grp, grp + 16, dtype=np.uint64)]))
    ref = sim.sf_amplitudes(setup, ids, bits)
    p = sfsim.Plan(text, jit=1, side_b_mask=w["side_b_mask"])
    q = sfsim.Plan(text, jit=1, side_b_mask=w["side_b_mask"], dense_finals=1)
    sel = sfsim.selection("list", ids=ids)
    assert _ws(p, len(bits), sel) > _ws(q, len(bits), sel), "compact finals not in use"
    q.close()
    a, _ = p.amplitudes(bits, sel)
    err = np.abs(a - ref).max()
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert rms > 0 and err <= 1e-4 * rms and err <= 1e-5 * 2.0 ** -21, (err, rms)
    p.close()


def test_7x8_prefix_compact_equals_dense():
    """The bench's configuration (one 128-path prefix of the f = 0.5%
    selection, specialised kernels) on 100k bitstrings."""
    w = inputs.WORKLOADS["7x8_d40"]
    text = inputs.workload_circuit("7x8_d40").text()
    bits = inputs.random_bitstrings(56, 100000, w["bitstring_seed"])
    p = sfsim.Plan(text, jit=1, side_b_mask=w["side_b_mask"])
    ids = sfsim.sf_selection_ids(p.handle, sfsim.selection("fraction", fidelity=0.005, seed=7), cap=128)
    sel = sfsim.selection("range", first=int(ids[0]), count=128)
    q = sfsim.Plan(text, jit=1, side_b_mask=w["side_b_mask"], dense_finals=1)
    assert _ws(p, len(bits), sel) > _ws(q, len(bits), sel), "compact finals not in use"
    a, bytes_c, la, _ = _pass_bytes(p, bits, sel)
    p.close()
    d, bytes_d, ld, _ = _pass_bytes(q, bits, sel)
    q.close()
    assert np.array_equal(a, d)
    assert la == ld
    # 8 finals: two 2 GiB halves written each (dense) against the requested
    # blocks (compact, at most 100k x 16 amplitudes per half)
    saved = bytes_d - bytes_c
    assert 8 * 2 * (2 ** 31 - 100000 * 16 * 8) <= saved <= 8 * 2 * 2 ** 31
