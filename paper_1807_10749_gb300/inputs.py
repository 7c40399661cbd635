"""Seeded synthetic inputs: random grid circuits, bitstrings and Haar unitaries.

This module holds no arithmetic of the simulation method. It only writes down
workloads in the text circuit format, so that the CUDA library and the FP64
oracle both read the same input. Nothing here imports the library or the oracle.

Circuit rules (Section 1 and Section 6 of arXiv:1807.10749, the "v2" benchmark
revisions):
  * cycle 0 applies H to every qubit;
  * cycles 1..D apply nearest-neighbour CZ gates in a repeating pattern of eight
    configurations, so that every grid edge carries one CZ per eight cycles and
    horizontal configurations alternate with vertical ones;
  * a qubit that was in a CZ in cycle t-1 and is not in one in cycle t receives a
    one-qubit gate in cycle t: T the first time, afterwards X^1/2, Y^1/2 or T,
    drawn uniformly from the two gates that differ from the previous one;
  * cycle D+1 applies H to every qubit.

The "v2" variant (Section 6: benchmarks revised so that no T gate follows a
CZ; Table 2's 7x8 row used them) changes the one-qubit rule:
  * the gate in a slot right after a CZ is X^1/2 or Y^1/2 (uniform the first
    time on that qubit, afterwards the one that differs from the previous);
  * a qubit that received such a gate in cycle t-1 and is idle in cycle t
    receives T in cycle t.
For 7x8, depth 1+40+1 this gives 538 X^1/2 / Y^1/2 gates, exactly Table 2's
1466 gates - 112 H - 485 CZ - 331 T, and 330 T gates (Table 2: 331). The
paper does not print the rule; this placement is our reading of it.

The eight CZ configurations (the paper names them but does not print them; the
layout below reproduces the CZ and cross-cut CZ counts of the 7x7 and 7x8 rows
of Table 2 exactly, see tests/golden/gate_counts.txt):
  H(a,b): horizontal edges (r,c)-(r,c+1) with c = a, r = b (mod 2)
  V(a,b): vertical edges   (r,c)-(r+1,c) with r = a, c = b (mod 2)
  cycle t >= 1 uses configuration (t-1) mod 8 of
      H00, V00, H11, V11, H01, V01, H10, V10.

Qubit q = r*C + c (row-major). Bit q of a bitstring is the measured value of
qubit q.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014):
    state += 0x9E3779B97F4A7C15
    z = state; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB; return z ^ (z >> 31)
One stream per (seed, purpose) starts from
    state0 = seed * 0x9E3779B97F4A7C15 + purpose * 0xD1B54A32D192ED03 (mod 2^64).

Text format, one gate per line ('#' starts a comment):
    grid R C
    <cycle> h|t|x_1_2|y_1_2|z|s <q>
    <cycle> cz|iswap <q0> <q1>
    <cycle> u1 <q> <8 reals: re,im of m00 m01 m10 m11>
    <cycle> u2 <q0> <q1> <32 reals: re,im of the 4x4 matrix, row-major,
               basis index 2*bit(q0) + bit(q1)>
Gates of one cycle act on disjoint qubits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1

PURPOSE_GATES = 1
PURPOSE_HAAR = 2
PURPOSE_BITSTRINGS = 3
PURPOSE_PATHS = 4

# Configuration order H00, V00, H11, V11, H01, V01, H10, V10 as (kind, a, b).
CZ_PATTERN = [("H", 0, 0), ("V", 0, 0), ("H", 1, 1), ("V", 1, 1),
              ("H", 0, 1), ("V", 0, 1), ("H", 1, 0), ("V", 1, 0)]


class SplitMix64:
    """SplitMix64 generator (published definition, see module docstring)."""

    def __init__(self, seed: int, purpose: int = 0):
        self.state = (seed * 0x9E3779B97F4A7C15 + purpose * 0xD1B54A32D192ED03) & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in (0, 1): the top 53 bits, offset by half an ulp."""
        return ((self.next() >> 11) + 0.5) * (1.0 / (1 << 53))


def cz_edges(rows: int, cols: int, config: int):
    """Edges (q0 < q1) of CZ configuration `config` (0..7) on an R x C grid."""
    kind, a, b = CZ_PATTERN[config % 8]
    edges = []
    if kind == "H":
        for r in range(rows):
            for c in range(cols - 1):
                if c % 2 == a and r % 2 == b:
                    edges.append((r * cols + c, r * cols + c + 1))
    else:
        for r in range(rows - 1):
            for c in range(cols):
                if r % 2 == a and c % 2 == b:
                    edges.append((r * cols + c, (r + 1) * cols + c))
    return edges


@dataclass
class Gate:
    cycle: int
    name: str
    qubits: tuple
    params: tuple = ()


@dataclass
class CircuitSpec:
    rows: int
    cols: int
    gates: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return self.rows * self.cols

    def text(self) -> str:
        lines = [f"grid {self.rows} {self.cols}"]
        for g in self.gates:
            parts = [str(g.cycle), g.name] + [str(q) for q in g.qubits]
            parts += [repr(float(p)) for p in g.params]
            lines.append(" ".join(parts))
        return "\n".join(lines) + "\n"


def haar_unitary(d: int, rng: SplitMix64) -> np.ndarray:
    """Haar-random U(d): QR of a complex Ginibre matrix, R's diagonal phases
    divided out (Mezzadri, Notices AMS 54, 2007). Normals by Box-Muller."""
    z = np.empty((d, d), dtype=np.complex128)
    for i in range(d):
        for j in range(d):
            u1, u2 = rng.uniform(), rng.uniform()
            rad = math.sqrt(-2.0 * math.log(u1))
            z[i, j] = complex(rad * math.cos(2 * math.pi * u2),
                              rad * math.sin(2 * math.pi * u2)) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def google_circuit(rows: int, cols: int, depth: int, seed: int = 1,
                   haar: bool = False, iswap: bool = False, v2: bool = False) -> CircuitSpec:
    """Random grid circuit of depth 1+depth+1 under the rules in the module
    docstring. haar=True replaces every CZ by a seeded Haar-random U(4)
    (written as a 'u2' line); iswap=True replaces every CZ by iSWAP; v2=True
    uses the revised one-qubit placement."""
    spec = CircuitSpec(rows, cols)
    n = rows * cols
    rng = SplitMix64(seed, PURPOSE_GATES)
    hrng = SplitMix64(seed, PURPOSE_HAAR)
    for q in range(n):
        spec.gates.append(Gate(0, "h", (q,)))
    last_1q = [None] * n
    prev_busy = set()
    prev_slot = set()
    for t in range(1, depth + 1):
        edges = cz_edges(rows, cols, (t - 1) % 8)
        busy = set()
        for (a, b) in edges:
            busy.add(a)
            busy.add(b)
            if haar:
                u = haar_unitary(4, hrng)
                params = []
                for i in range(4):
                    for j in range(4):
                        params += [u[i, j].real, u[i, j].imag]
                spec.gates.append(Gate(t, "u2", (a, b), tuple(params)))
            elif iswap:
                spec.gates.append(Gate(t, "iswap", (a, b)))
            else:
                spec.gates.append(Gate(t, "cz", (a, b)))
        slot = set()
        for q in range(n):
            if q in prev_busy and q not in busy:
                if v2:
                    choices = [c for c in ("x_1_2", "y_1_2") if c != last_1q[q]]
                    g = choices[rng.next() >> 63] if len(choices) == 2 else choices[0]
                elif last_1q[q] is None:
                    g = "t"
                else:
                    choices = [c for c in ("x_1_2", "y_1_2", "t") if c != last_1q[q]]
                    g = choices[rng.next() >> 63]
                last_1q[q] = g
                slot.add(q)
                spec.gates.append(Gate(t, g, (q,)))
            elif v2 and q in prev_slot and q not in busy:
                spec.gates.append(Gate(t, "t", (q,)))
        prev_busy = busy
        prev_slot = slot
    for q in range(n):
        spec.gates.append(Gate(depth + 1, "h", (q,)))
    return spec


def random_bitstrings(n_qubits: int, count: int, seed: int) -> np.ndarray:
    """`count` uniform n-bit bitstrings as uint64 (bit q = qubit q)."""
    rng = SplitMix64(seed, PURPOSE_BITSTRINGS)
    mask = (1 << n_qubits) - 1 if n_qubits < 64 else MASK64
    # vectorised SplitMix64: state_i = state0 + (i+1)*golden
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        s = np.uint64(rng.state) + i * np.uint64(0x9E3779B97F4A7C15)
        z = s
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z & np.uint64(mask)


def random_path_list(n_paths_log2: int, count: int, seed: int, digit_bits: int = 1) -> np.ndarray:
    """`count` distinct path ids drawn from [0, 2^n_paths_log2) (sorted, uint64).
    A LIST selection for parity tests; holds no method arithmetic."""
    rng = SplitMix64(seed, PURPOSE_PATHS)
    total = 1 << n_paths_log2
    count = min(count, total)
    out = set()
    while len(out) < count:
        out.add(rng.next() % total)
    return np.array(sorted(out), dtype=np.uint64)


# The workloads the benchmark and the parity tests use: grid, depth, cut
# (bit q set = qubit q in half B), bitstring count.
def column_cut_mask(rows: int, cols: int, first_b_col: int) -> int:
    m = 0
    for r in range(rows):
        for c in range(first_b_col, cols):
            m |= 1 << (r * cols + c)
    return m


def row_cut_mask(rows: int, cols: int, first_b_row: int) -> int:
    m = 0
    for r in range(first_b_row, rows):
        for c in range(cols):
            m |= 1 << (r * cols + c)
    return m


WORKLOADS = {
    # 4x4, 1+10+1, halves 2x4 (rows 0-1 | rows 2-3), all 16 paths, 1024 bitstrings
    "4x4_d10": dict(rows=4, cols=4, depth=10, side_b_mask=row_cut_mask(4, 4, 2),
                    n_bitstrings=1024, bitstring_seed=1000),
    # 5x6, 1+24+1, halves 15+15 (cols 0-2 | 3-5), all paths, 100k bitstrings
    "5x6_d24": dict(rows=5, cols=6, depth=24, side_b_mask=column_cut_mask(5, 6, 3),
                    n_bitstrings=100_000, bitstring_seed=1001),
    # 6x7, 1+26+1, halves 21+21 (rows 0-2 | 3-5), 1M bitstrings
    "6x7_d26": dict(rows=6, cols=7, depth=26, side_b_mask=row_cut_mask(6, 7, 3),
                    n_bitstrings=1_000_000, bitstring_seed=1002),
    # 7x8, 1+40+1, halves 28+28 (cols 0-3 | 4-7), f = 0.5%, 1M bitstrings;
    # v2 one-qubit rule, as in Table 2's 7x8 row
    "7x8_d40": dict(rows=7, cols=8, depth=40, side_b_mask=column_cut_mask(7, 8, 4),
                    n_bitstrings=1_000_000, bitstring_seed=1003, v2=True),
    # profiling case: the same kernels on 25+25-qubit halves (256 MiB each,
    # larger than L2) in a few GB of device memory
    "5x10_d16": dict(rows=5, cols=10, depth=16, side_b_mask=column_cut_mask(5, 10, 5),
                     n_bitstrings=100_000, bitstring_seed=1005, v2=True),
    # profiling case whose last branching level (2 cut CZs) folds into the
    # gather, so its final passes write compact blocks at 1M bitstrings
    "5x10_d14": dict(rows=5, cols=10, depth=14, side_b_mask=column_cut_mask(5, 10, 5),
                     n_bitstrings=1_000_000, bitstring_seed=1006, v2=True),
}


def workload_circuit(name: str, seed: int = 1, **kw) -> CircuitSpec:
    """The circuit of a named workload (its grid, depth and one-qubit rule)."""
    w = WORKLOADS[name]
    kw.setdefault("v2", w.get("v2", False))
    return google_circuit(w["rows"], w["cols"], w["depth"], seed, **kw)
