"""Text circuit parser for the oracle (test infrastructure only).

Reads the format written by the seeded input generator: a 'grid R C' line,
then '<cycle> <gate> <qubits...> [<reals>...]' lines. Returns the gates in
file order with their complex128 matrices (oracle.gates).
"""
from dataclasses import dataclass

import numpy as np

from . import gates


@dataclass
class OGate:
    cycle: int
    name: str
    qubits: tuple
    mat: np.ndarray  # 2x2 or 4x4 complex128


@dataclass
class OCircuit:
    rows: int
    cols: int
    gates: list

    @property
    def n(self):
        return self.rows * self.cols


def parse(text: str) -> OCircuit:
    rows = cols = None
    out = []
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "grid":
            rows, cols = int(tok[1]), int(tok[2])
            continue
        cycle, name = int(tok[0]), tok[1]
        nq = 1 if name in gates.ONE_QUBIT or name == "u1" else 2
        qubits = tuple(int(t) for t in tok[2:2 + nq])
        params = tuple(float(t) for t in tok[2 + nq:])
        out.append(OGate(cycle, name, qubits, gates.matrix(name, params)))
    if rows is None:
        raise ValueError("missing 'grid R C' line")
    return OCircuit(rows, cols, out)
