"""Cross-cut gate decompositions (oracle; test infrastructure only).

A two-qubit gate U acting on (a, b), a in half A and b in half B, is written
as U = sum_k A_k (x) B_k, with U[(a b), (a' b')] = sum_k A_k[a, a'] B_k[b, b'].
Each term k is one branch of the path sum.

  projector  - Eq. 1: CZ = P0 (x) I + P1 (x) Z, projector on the A-side qubit;
               mirrored (CZ is symmetric): CZ = I (x) P0 + Z (x) P1, projector on
               the B-side qubit.
  block4     - Eq. 4way: U = P0 (x) U00 + P1 (x) U11 + |0><1| (x) U01 + |1><0| (x) U10,
               U_ij the 2x2 blocks of U indexed by the A-side bits.
  schmidt    - Section 3 / Section 7: the operator-Schmidt decomposition. The
               realigned matrix R[(a a'), (b b')] = U[(a b), (a' b')] is split by
               an SVD R = sum_k s_k u_k v_k^H; A_k = u_k as 2x2, B_k = s_k conj(v_k)
               as 2x2. Terms are kept in descending s_k, s_k < 1e-14 dropped.
               Gauge: each A_k is multiplied by the phase that makes its first
               entry (row-major) with modulus > 1e-12 real and positive, and B_k
               by the inverse phase.
"""
import numpy as np

from . import gates

SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def oriented(U, a_is_first):
    """U re-expressed with the A-side qubit as the first (high) basis bit."""
    return U if a_is_first else SWAP @ U @ SWAP


def projector_cz(on_b=False):
    if on_b:
        return [(gates.I2, gates.P0), (gates.Z, gates.P1)]
    return [(gates.P0, gates.I2), (gates.P1, gates.Z)]


def block4(U):
    U = np.asarray(U, dtype=np.complex128)
    blk = lambda i, j: U[2 * i:2 * i + 2, 2 * j:2 * j + 2]
    return [(gates.P0, blk(0, 0)), (gates.P1, blk(1, 1)),
            (gates.K01, blk(0, 1)), (gates.K10, blk(1, 0))]


def schmidt(U, tol=1e-14):
    U = np.asarray(U, dtype=np.complex128)
    R = np.empty((4, 4), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            for ap in range(2):
                for bp in range(2):
                    R[2 * a + ap, 2 * b + bp] = U[2 * a + b, 2 * ap + bp]
    u, s, vh = np.linalg.svd(R)
    terms = []
    for k in range(4):
        if s[k] < tol:
            continue
        A = u[:, k].reshape(2, 2).copy()
        B = (s[k] * vh[k, :]).reshape(2, 2).copy()
        flat = A.reshape(-1)
        for z in flat:
            if abs(z) > 1e-12:
                ph = z / abs(z)
                A = A / ph
                B = B * ph
                break
        terms.append((A, B))
    return terms


def reconstruct(terms):
    return sum(np.kron(A, B) for A, B in terms)
