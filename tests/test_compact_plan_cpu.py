"""The planner's choice of compact finals and the workspace it sizes, on the
CPU (plans made with an explicit memory budget need no device to size their
workspace). Whole-state finals need the node slots only; compact finals add,
per half whose final pass qualifies, a part map (8 bytes per 32 parts of
2^ctl amplitudes), its chunk counts and, per final of a block, a buffer of
min(n * 2^(g - ctl), 2^(m - ctl)) parts. ctl is read off the plan's
description (the last pass's tile positions below g). A block holds as many
finals as hold 2^30 amplitudes of both halves (two at 7x8), within the
budget."""
import re

import pytest

from paper_1807_10749_gb300 import inputs, sfsim

BUDGET = 200 << 30


def _a256(b):
    return (b + 255) // 256 * 256


def _plan(name, **kw):
    w = inputs.WORKLOADS[name]
    return sfsim.Plan(inputs.workload_circuit(name).text(), side_b_mask=w["side_b_mask"],
                      hbm_budget_bytes=kw.pop("budget", BUDGET), **kw)


def _final_ctl(plan, g):
    """ctl of each half's final pass, from the plan description."""
    text = sfsim.sf_plan_describe(plan.handle)
    out = []
    for half in "AB":
        seg = text[text.index(f"half {half} segment", text.rindex(f"half {half} segment")):]
        seg = seg.split("\nhalf ")[0]
        active = [int(v) for v in re.findall(r"active \[([0-9,]+)\]", seg)[-1].split(",")]
        out.append(sum(1 for p in active if p < g))
    return out


def _compact_bytes(m, g, ctls, n, finals_per_block=1):
    extra = 0
    for ctl in ctls:
        parts = 1 << (m - ctl)
        cap = min(n << (g - ctl), parts)
        if (cap << ctl) * 4 > (1 << m):
            return 0
        nw = (parts + 31) // 32
        extra += _a256(nw * 8) + _a256(((nw + 2047) // 2048) * 4) + finals_per_block * _a256((cap << ctl) * 8)
    return extra


def test_7x8_workspace_adds_exactly_the_part_maps_and_buffers():
    p = _plan("7x8_d40")
    q = _plan("7x8_d40", dense_finals=1)
    sel = sfsim.selection("fraction", fidelity=0.005, seed=7)
    first = int(sfsim.sf_selection_ids(p.handle, sel, cap=1)[0])
    sel = sfsim.selection("range", first=first, count=128)
    g = 4
    ctls = _final_ctl(p, g)
    assert all(1 <= c <= g and g - c <= 1 for c in ctls), ctls
    B = min((1 << 30) // (2 * (1 << 28)), 128 // 16)   # finals per block: 2 of the range's 8
    for n in (1, 1000, 1_000_000):
        extra = sfsim.sf_workspace_size(p.handle, n, sel) - sfsim.sf_workspace_size(q.handle, n, sel)
        assert extra == _compact_bytes(28, g, ctls, n, B), n
        assert extra > 0
    # 5M bitstrings: the blocks would fill more than a quarter of each half
    assert _compact_bytes(28, g, ctls, 5_000_000) == 0
    assert sfsim.sf_workspace_size(p.handle, 5_000_000, sel) == sfsim.sf_workspace_size(q.handle, 5_000_000, sel)
    p.close()
    q.close()


def test_compact_finals_yield_to_the_memory_budget():
    q = _plan("7x8_d40", dense_finals=1)
    sel = sfsim.selection("range", first=0, count=16)
    dense = sfsim.sf_workspace_size(q.handle, 1000, sel)
    q.close()
    # a budget that holds the node slots but not the compact finals
    p = _plan("7x8_d40", budget=dense - 256 + 1024)
    assert sfsim.sf_workspace_size(p.handle, 1000, sel) == dense
    p.close()


def test_6x7_compact_by_bitstring_count_and_none_without_a_folded_level():
    p = _plan("6x7_d26")
    q = _plan("6x7_d26", dense_finals=1)
    sel = sfsim.selection("range", first=1 << 12, count=64)
    assert sfsim.sf_workspace_size(p.handle, 3009, sel) > sfsim.sf_workspace_size(q.handle, 3009, sel)
    assert sfsim.sf_workspace_size(p.handle, 200000, sel) == sfsim.sf_workspace_size(q.handle, 200000, sel)
    p.close()
    q.close()
    # 5x6 keeps its last level (it does not fold): finals are whole states
    p = _plan("5x6_d24")
    q = _plan("5x6_d24", dense_finals=1)
    sel = sfsim.selection("range", first=0, count=64)
    assert sfsim.sf_workspace_size(p.handle, 10, sel) == sfsim.sf_workspace_size(q.handle, 10, sel)
    p.close()
    q.close()


def test_dense_finals_option_is_validated():
    with pytest.raises(sfsim.SFError):
        _plan("4x4_d10", dense_finals=2)
