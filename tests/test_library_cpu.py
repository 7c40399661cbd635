"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/sfsim.h declares, validates input, plans the
workloads, and enumerates path selections bit-exactly like the oracle."""
import os
import re

import numpy as np
import pytest

from oracle import circuit as ocirc
from oracle import paths as opaths
from oracle import sim
from paper_1807_10749_gb300 import inputs, sfsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1807_10749_gb300 import build
    build.build()


def test_library_exports_every_declared_symbol():
    with open(os.path.join(ROOT, "include", "sfsim.h")) as fh:
        declared = set(re.findall(r"SF_API\s+[\w\s\*]*?\b(sf_\w+)\s*\(", fh.read()))
    assert declared == set(sfsim.EXPORTED)
    lib = sfsim.lib()
    for name in declared:
        assert hasattr(lib, name), name


def test_parse_errors_are_reported():
    for bad in ["0 h 0\n", "grid 2 2\n0 h 9\n", "grid 2 2\n0 cz 0 0\n", "grid 2 2\n1 h 0\n1 t 0\n",
                "grid 2 2\n0 foo 1\n", "grid 2 2\n0 u1 0 1 2\n"]:
        with pytest.raises(sfsim.SFError) as e:
            sfsim.sf_circuit_parse(bad)
        assert e.value.code == sfsim.SF_EINVAL
        assert sfsim.sf_last_error()


def test_circuit_create_matches_parse():
    g = sfsim.sf_gate()
    g.cycle, g.kind, g.q0, g.q1 = 0, sfsim.SF_H, 1, -1
    c = sfsim.sf_circuit_create(2, 2, [g])
    assert sfsim.sf_circuit_info(c) == (2, 2, 1)
    sfsim.sf_circuit_destroy(c)
    with pytest.raises(sfsim.SFError):
        g.q0 = 7
        sfsim.sf_circuit_create(2, 2, [g])


@pytest.mark.parametrize("name", list(inputs.WORKLOADS))
def test_plan_matches_oracle_split(name):
    """Cut, cross-gate count and path bits agree with the oracle's split."""
    w = inputs.WORKLOADS[name]
    spec = inputs.workload_circuit(name)
    p = sfsim.Plan(spec.text(), side_b_mask=w["side_b_mask"])
    setup = sim.SFSetup(ocirc.parse(spec.text()), w["side_b_mask"])
    assert p.info["n_cross"] == setup.n_cross
    assert p.info["path_bits"] == setup.x_bits
    assert p.info["m_a"] == len(setup.posA) and p.info["m_b"] == len(setup.posB)
    st = sfsim.sf_plan_stats(p.handle)
    assert st["passes_a"] > 0 and st["passes_b"] > 0
    p.close()


def test_auto_cut_is_the_minimal_straight_cut():
    """Section 8: minimise the larger block, then the number of cross gates.
    7x8: the vertical cut between columns 3 and 4 gives 28+28 (35 xCZ)."""
    spec = inputs.google_circuit(7, 8, 40, 1)
    p = sfsim.Plan(spec.text())
    assert p.info["m_a"] == 28 and p.info["m_b"] == 28 and p.info["n_cross"] == 35
    p.close()


def test_haar_variant_branches_four_ways():
    spec = inputs.google_circuit(4, 4, 10, 1, haar=True)
    w = inputs.WORKLOADS["4x4_d10"]
    for dec in (sfsim.SF_DEC_SCHMIDT, sfsim.SF_DEC_BLOCK4):
        p = sfsim.Plan(spec.text(), side_b_mask=w["side_b_mask"], decomposition=dec)
        assert p.info["path_bits"] == 8
        p.close()


def test_selection_ids_match_oracle_bit_exactly():
    spec = inputs.google_circuit(5, 6, 24, 1)
    w = inputs.WORKLOADS["5x6_d24"]
    p = sfsim.Plan(spec.text(), side_b_mask=w["side_b_mask"])
    x = p.info["path_bits"]
    for f in (1.0, 0.25, 1 / 64, 0.001):
        sel = sfsim.selection("fraction", fidelity=f, seed=7)
        ids = sfsim.sf_selection_ids(p.handle, sel)
        want, fa = opaths.select_fraction(x, f, 7)
        assert np.array_equal(ids, np.sort(want))
        assert sfsim.sf_selection_size(p.handle, sel) == (len(want), fa)
    sel = sfsim.selection("range", first=100, count=37)
    assert np.array_equal(sfsim.sf_selection_ids(p.handle, sel), opaths.select_range(100, 37))
    lst = inputs.random_path_list(x, 50, 3)
    sel = sfsim.selection("list", ids=lst[::-1])
    assert np.array_equal(sfsim.sf_selection_ids(p.handle, sel), np.sort(lst))
    # errors: out of range, duplicates, bad fidelity
    for bad in (sfsim.selection("range", first=1 << x, count=1),
                sfsim.selection("list", ids=[1, 1]),
                sfsim.selection("fraction", fidelity=0.0)):
        with pytest.raises(sfsim.SFError) as e:
            sfsim.sf_selection_size(p.handle, bad)
        assert e.value.code == sfsim.SF_EINVAL
    p.close()


def test_feistel_matches_oracle_at_28_bits():
    """The 7x8 FRACTION selection (x_s = 28) enumerates the oracle's prefixes."""
    spec = inputs.workload_circuit("7x8_d40")
    p = sfsim.Plan(spec.text(), side_b_mask=inputs.WORKLOADS["7x8_d40"]["side_b_mask"])
    sel = sfsim.selection("fraction", fidelity=0.005, seed=7)
    n, fa = sfsim.sf_selection_size(p.handle, sel)
    assert n == 1342177 * 128 and fa == 1342177 / 2 ** 28
    ids = sfsim.sf_selection_ids(p.handle, sel, cap=128 * 64)
    pre = sorted(opaths.feistel(i, 28, 7) for i in range(1342177))[:64]
    want = np.array([(q << 7) | s for q in pre for s in range(128)], dtype=np.uint64)
    assert np.array_equal(ids, want)
    p.close()


@pytest.mark.parametrize("name,packed", [("4x4_d10", 0), ("6x7_d26", 0), ("7x8_d40", 0), ("7x8_d40", 1)])
def test_specialised_pass_kernels_compile(name, packed):
    """Every pass of the plan compiles into its own kernel (NVRTC runs
    without a GPU), scalar or with packed FP32x2 stages; a second plan of the
    same circuit reuses the binaries."""
    import time
    w = inputs.WORKLOADS[name]
    text = inputs.workload_circuit(name).text()
    try:
        p = sfsim.Plan(text, side_b_mask=w["side_b_mask"], jit=1, fp32x2=packed)
    except sfsim.SFError as e:
        if e.code == sfsim.SF_EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    p.close()
    t = time.perf_counter()
    q = sfsim.Plan(text, side_b_mask=w["side_b_mask"], jit=1, fp32x2=packed)
    assert time.perf_counter() - t < 2.0   # cached
    q.close()
    with pytest.raises(sfsim.SFError):
        sfsim.Plan(text, side_b_mask=w["side_b_mask"], jit=2)


def test_cost_terms_follow_eq_t_tot():
    """Features of the runtime model (Section 8) for the 5x6, 1+24+1 circuit,
    recomputed here from the circuit text: q1 = q2 = 15, x = 15 cross gates,
    x_p = 8 prefix bits (x_b = 7), d = 26 cycles, d_p = the cycle of the
    8th cross gate in time order."""
    w = inputs.WORKLOADS["5x6_d24"]
    text = inputs.workload_circuit("5x6_d24").text()
    c = ocirc.parse(text)
    mask = w["side_b_mask"]
    inB = lambda q: (mask >> q) & 1
    cross = sorted([g for g in c.gates if len(g.qubits) == 2 and inB(g.qubits[0]) != inB(g.qubits[1])],
                   key=lambda g: (g.cycle, min(g.qubits), max(g.qubits)))
    assert len(cross) == 15
    d = max(g.cycle for g in c.gates) + 1
    dp = cross[15 - 1 - 7].cycle       # path bit 7 <-> cross gate 7 (earliest in the MSB)
    work = 2 * 15 * 2.0 ** 15
    p = sfsim.Plan(text, side_b_mask=mask)
    n_a = 1000
    t = sfsim.sf_plan_cost_terms(p.handle, sfsim.selection("fraction", fidelity=0.25, seed=7), n_a)
    K = 64   # floor(0.25 * 2^8) prefixes of 2^7 paths
    assert np.allclose(t, [1, K * work * dp, K * work * 128 * (d - dp), K * 128 * n_a], rtol=1e-12)
    # a range inside one prefix: one prefix, 10 paths
    t = sfsim.sf_plan_cost_terms(p.handle, sfsim.selection("range", first=300, count=10), n_a)
    assert np.allclose(t, [1, work * dp, work * 128 * (d - dp), 10 * n_a], rtol=1e-12)
    # a range over a prefix boundary: two prefixes
    t = sfsim.sf_plan_cost_terms(p.handle, sfsim.selection("range", first=250, count=10), n_a)
    assert np.isclose(t[1], 2 * work * dp)
    p.close()


def test_cost_fit_recovers_coefficients():
    rng = np.random.default_rng(4)
    T = rng.uniform(0.0, 1.0, size=(12, 4)) * np.array([1, 1e9, 1e11, 1e8])
    T[:, 0] = 1.0
    a = np.array([1e-4, 2e-12, 3e-14, 5e-10])
    secs = T @ a
    got = sfsim.sf_cost_fit(T, secs)
    assert np.allclose(got, a, rtol=1e-8)
    assert abs(sfsim.sf_cost_predict(T[0], got) - secs[0]) <= 1e-9 * secs[0]
    # a coefficient that would come out negative is clipped to zero
    secs2 = 1e-4 + T[:, 1] * 2e-12 + T[:, 3] * 5e-10
    got2 = sfsim.sf_cost_fit(T, secs2)
    assert got2[2] == 0.0 and np.allclose(got2[[0, 1, 3]], [1e-4, 2e-12, 5e-10], rtol=1e-8)
    with pytest.raises(sfsim.SFError):
        sfsim.sf_cost_fit(T, -secs)


def _final_bytes(p):
    nL = sfsim.sf_plan_info(p.handle)["n_levels"]
    return sum(sfsim.sf_plan_segment_stats(p.handle, h, nL + 1)[2] for h in (0, 1))


def test_merged_last_program_moves_fewer_bytes():
    """With the last level folded into the gather, planning the level before
    it and the last segment as one program saves the node in between: at 7x8
    the merged final moves fewer bytes than the two programs together."""
    w = inputs.WORKLOADS["7x8_d40"]
    text = inputs.workload_circuit("7x8_d40").text()
    merged = sfsim.Plan(text, side_b_mask=w["side_b_mask"])
    split = sfsim.Plan(text, side_b_mask=w["side_b_mask"], split_last=1)
    nL = sfsim.sf_plan_info(split.handle)["n_levels"]
    split_bytes = _final_bytes(split) + sum(sfsim.sf_plan_segment_stats(split.handle, h, nL - 1)[2]
                                            for h in (0, 1))
    assert _final_bytes(merged) < 0.6 * split_bytes
    merged.close()
    split.close()


def test_automatic_tiles_and_runs_move_no_more_bytes_than_fixed_small_tiles():
    """Per segment the planner keeps the (tile, run) candidate of least
    estimated time, bytes over the tile size's HBM fraction (0.75 at 2^12,
    0.64 at 2^13). A 2^13 tile wins only with under 0.85x the bytes of the
    best 2^12 candidate and the runs tie on efficiency, so every segment, and
    the whole plan, moves no more bytes than with 2^12 tiles and either run
    width."""
    w = inputs.WORKLOADS["7x8_d40"]
    text = inputs.workload_circuit("7x8_d40").text()

    def total(p):
        nL = sfsim.sf_plan_info(p.handle)["n_levels"]
        t = sum(sfsim.sf_plan_segment_stats(p.handle, h, s)[2]
                for h in (0, 1) for s in list(range(nL - 1)) + [nL + 1])
        p.close()
        return t
    auto = total(sfsim.Plan(text, side_b_mask=w["side_b_mask"]))
    for rb in (3, 4):
        assert auto <= total(sfsim.Plan(text, side_b_mask=w["side_b_mask"], tile_bits=12, run_bits=rb))
