"""Brute-force dense simulation for n <= 10 (oracle; test infrastructure only).

Every gate becomes a 2^n x 2^n matrix built from Kronecker products of
one-qubit operators: a one-qubit gate G on qubit q is
    I (x) ... (x) G (x) ... (x) I     (qubit n-1 leftmost, qubit 0 rightmost),
and a two-qubit gate G on (q0, q1) is
    sum_{a,b,a',b'} G[(a b), (a' b')] |a><a'| on q0 (x) |b><b'| on q1 (x) I elsewhere.
The state is U_g ... U_1 |0...0>. This shares no code with oracle/core.c.
"""
import numpy as np

from . import gates


def _embed(ops_by_qubit, n):
    out = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        out = np.kron(out, ops_by_qubit.get(q, gates.I2))
    return out


def _ket_bra(i, j):
    m = np.zeros((2, 2), dtype=np.complex128)
    m[i, j] = 1
    return m


def full_matrix(g, n):
    if len(g.qubits) == 1:
        return _embed({g.qubits[0]: g.mat}, n)
    q0, q1 = g.qubits
    U = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            for ap in range(2):
                for bp in range(2):
                    c = g.mat[2 * a + b, 2 * ap + bp]
                    if c != 0:
                        U += c * _embed({q0: _ket_bra(a, ap), q1: _ket_bra(b, bp)}, n)
    return U


def dense_state(circ):
    n = circ.n
    if n > 10:
        raise ValueError("dense brute force is for n <= 10")
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1
    for g in circ.gates:
        psi = full_matrix(g, n) @ psi
    return psi
