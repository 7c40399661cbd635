"""Gate matrices in complex128 (oracle; test infrastructure only).

The paper names the gates (Section 1: H, CZ, X^1/2, Y^1/2, T; Section 7: iSWAP)
but does not print their matrices. Readings used here:
  H      = (1/sqrt 2) [[1, 1], [1, -1]]
  T      = diag(1, e^{i pi/4})
  X^1/2  = the principal square root of X = 1/2 [[1+i, 1-i], [1-i, 1+i]]
  Y^1/2  = the principal square root of Y = 1/2 [[1+i, -1-i], [1+i, 1+i]]
  Z = diag(1, -1), S = diag(1, i)
  CZ     = diag(1, 1, 1, -1)                                   (Eq. 1)
  iSWAP  = |00><00| + i|01><10| + i|10><01| + |11><11|          (Section 7)
Two-qubit matrices act on the basis index 2*bit(q0) + bit(q1).
"""
import numpy as np

S2 = np.sqrt(0.5)

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = S2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)
T = np.diag([1.0, np.exp(1j * np.pi / 4)]).astype(np.complex128)
S = np.diag([1.0, 1j]).astype(np.complex128)
X_HALF = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
Y_HALF = 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)
P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)
K01 = np.array([[0, 1], [0, 0]], dtype=np.complex128)   # |0><1|
K10 = np.array([[0, 0], [1, 0]], dtype=np.complex128)   # |1><0|

CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
ISWAP = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]],
                 dtype=np.complex128)

ONE_QUBIT = {"h": H, "t": T, "x_1_2": X_HALF, "y_1_2": Y_HALF, "z": Z, "s": S}
TWO_QUBIT = {"cz": CZ, "iswap": ISWAP}


def matrix(name, params=()):
    """Matrix of a named gate; 'u1'/'u2' take their entries from params."""
    if name in ONE_QUBIT:
        return ONE_QUBIT[name]
    if name in TWO_QUBIT:
        return TWO_QUBIT[name]
    if name == "u1":
        p = np.asarray(params, dtype=np.float64)
        return (p[0::2] + 1j * p[1::2]).reshape(2, 2)
    if name == "u2":
        p = np.asarray(params, dtype=np.float64)
        return (p[0::2] + 1j * p[1::2]).reshape(4, 4)
    raise ValueError(f"unknown gate {name!r}")
