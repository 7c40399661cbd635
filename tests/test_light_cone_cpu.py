"""Light-cone scheduling of the gates (no GPU). The planner runs each gate in
the segment of the deepest branch level whose light cone holds it. Here the
cones are recomputed from the circuit text in this file's own code and
compared with the plan's description:
  * per half and segment, the non-diagonal one-qubit gates (X^1/2, Y^1/2, H)
    the plan runs there equal those whose cone depth is that segment's (the
    leading H of every qubit is absorbed into the generated root state);
  * scheduling by cycle ranges instead runs the same gates, only elsewhere.
The cone of level l on a half starts at each of its cut qubits with their
first non-diagonal gate after the level (Eq. 1's factors are diagonal) and
takes in every qubit a later gate couples to a qubit already in it."""
import re

from oracle import circuit as ocirc
from paper_1807_10749_gb300 import inputs, sfsim

ND = {"h", "x_1_2", "y_1_2"}


def _cone_segments(name):
    w = inputs.WORKLOADS[name]
    c = ocirc.parse(inputs.workload_circuit(name).text())
    mask = w["side_b_mask"]
    side = lambda q: (mask >> q) & 1
    cross = [g for g in c.gates if len(g.qubits) == 2 and side(g.qubits[0]) != side(g.qubits[1])]
    cycles = sorted({g.cycle for g in cross})
    depth = {}
    for li, lc in enumerate(cycles):
        for h in (0, 1):
            cut = {q for g in cross if g.cycle == lc for q in g.qubits if side(q) == h}
            cone = set()
            for i, g in enumerate(c.gates):
                if g.cycle < lc or g in cross or side(g.qubits[0]) != h:
                    continue
                qs = set(g.qubits)
                hit = bool(qs & cone) or (bool(qs & cut) and g.name in ND)
                if hit:
                    cone |= qs
                    depth[i] = li + 1
    # expected non-diagonal one-qubit gates per (half, segment); leading H absorbed
    seen = set()
    want = {}
    for i, g in enumerate(c.gates):
        if len(g.qubits) != 1 or g.name not in ND:
            continue
        q = g.qubits[0]
        if q not in seen and g.name == "h" and g.cycle == 0:
            seen.add(q)
            continue
        seen.add(q)
        key = ("AB"[side(q)], depth.get(i, 0))
        want[key] = want.get(key, 0) + 1
    return want


def _described(name, **kw):
    w = inputs.WORKLOADS[name]
    p = sfsim.Plan(inputs.workload_circuit(name).text(), side_b_mask=w["side_b_mask"], jit=0, **kw)
    text = sfsim.sf_plan_describe(p.handle)
    p.close()
    got = {}
    for m in re.finditer(r"half ([AB]) segment (\d+)[^\n]*\n(.*?)(?=\nhalf |\Z)", text, re.S):
        n = len(re.findall(r"(?<![A-Za-z])[XYH]\d", m.group(3)))
        if n:
            got[(m.group(1), int(m.group(2)))] = n
    return text, got


def test_5x6_segments_hold_the_gates_of_their_cones():
    text, got = _described("5x6_d24")
    assert "folded into the gather: no" in text
    assert got == _cone_segments("5x6_d24")


def test_cycle_segments_run_the_same_gates():
    for name in ("4x4_d10", "5x6_d24"):
        _, cone = _described(name)
        _, cyc = _described(name, cycle_segments=1)
        for h in "AB":
            assert sum(v for (s, _), v in cone.items() if s == h) == sum(v for (s, _), v in cyc.items() if s == h)
        assert cone != cyc or name == "4x4_d10"
