"""Python side of the FP64 oracle (test infrastructure only).

Builds oracle/core.c with gcc, splits a circuit into its two halves and its
cross-cut gates, and runs the plain state-vector and path-sum simulations.
"""
import ctypes
import os
import subprocess

import numpy as np

from . import decomp, paths

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "core.c")
_LIB = os.path.join(_HERE, "_core.so")
_lib = None


def build(force=False):
    """Compile core.c (gcc, OpenMP, IEEE double: no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        _lib.oracle_sv.argtypes = [ctypes.c_int, ctypes.c_int64, P, P, P, P, ctypes.c_int64, P, P]
        _lib.oracle_sf.argtypes = ([ctypes.c_int, P, ctypes.c_int64, P, P, P, P, P] * 2 +
                                   [ctypes.c_int, ctypes.c_int64, P, ctypes.c_int64, P, P])
        _lib.oracle_threads.restype = ctypes.c_int
    return _lib


def threads():
    return lib().oracle_threads()


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mat32(m):
    out = np.zeros(32, dtype=np.float64)
    flat = np.asarray(m, dtype=np.complex128).reshape(-1)
    out[0:2 * flat.size:2] = flat.real
    out[1:2 * flat.size:2] = flat.imag
    return out


def sv_amplitudes(circ, xs):
    """Full state-vector amplitudes <x|U|0^n> (complex128) for bitstrings xs."""
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    g = circ.gates
    nq = np.array([len(x.qubits) for x in g], dtype=np.int32)
    q0 = np.array([x.qubits[0] for x in g], dtype=np.int32)
    q1 = np.array([x.qubits[1] if len(x.qubits) > 1 else -1 for x in g], dtype=np.int32)
    mats = np.concatenate([_mat32(x.mat) for x in g]) if g else np.zeros(32)
    out = np.zeros(2 * len(xs), dtype=np.float64)
    rc = lib().oracle_sv(circ.n, len(g), _p(nq), _p(q0), _p(q1), _p(mats), len(xs), _p(xs), _p(out))
    if rc != 0:
        raise RuntimeError(f"oracle_sv failed: {rc}")
    return out[0::2] + 1j * out[1::2]


class SFSetup:
    """The circuit split by a cut: per-half op lists and the cross-gate terms.

    side_b_mask: bit q set <=> qubit q is in half B. decomposition: how non-CZ
    cross gates are split ('schmidt' or 'block4'); CZ always uses Eq. 1, with
    the projector on the A-side qubit, or (projector_side='alternate') on the
    A-side qubit of the even-numbered cross gates (time order, from 0) and the
    B-side qubit of the odd-numbered ones.
    """

    def __init__(self, circ, side_b_mask, decomposition="schmidt", projector_side="a"):
        n = circ.n
        self.n = n
        self.posA = np.array([q for q in range(n) if not (side_b_mask >> q) & 1], dtype=np.int32)
        self.posB = np.array([q for q in range(n) if (side_b_mask >> q) & 1], dtype=np.int32)
        locA = {int(q): k for k, q in enumerate(self.posA)}
        locB = {int(q): k for k, q in enumerate(self.posB)}
        inB = lambda q: (side_b_mask >> q) & 1
        cross = []
        for idx, g in enumerate(circ.gates):
            if len(g.qubits) == 2 and inB(g.qubits[0]) != inB(g.qubits[1]):
                cross.append(idx)
        # time order of cross gates: (cycle, smaller qubit, larger qubit)
        cross.sort(key=lambda i: (circ.gates[i].cycle, min(circ.gates[i].qubits),
                                  max(circ.gates[i].qubits)))
        xindex = {gi: k for k, gi in enumerate(cross)}
        self.terms = []
        self.bits = []
        for k, gi in enumerate(cross):
            g = circ.gates[gi]
            a_first = not inB(g.qubits[0])
            if g.name == "cz":
                t = decomp.projector_cz(on_b=projector_side == "alternate" and k % 2 == 1)
            else:
                U = decomp.oriented(g.mat, a_first)
                t = decomp.block4(U) if decomposition == "block4" else decomp.schmidt(U)
            r = 1
            while r < len(t):
                r *= 2
            z = np.zeros((2, 2), dtype=np.complex128)
            t = list(t) + [(z, z)] * (r - len(t))
            self.terms.append(t)
            self.bits.append(r.bit_length() - 1)
        self.x_bits = sum(self.bits)
        opsA, opsB = [], []
        for idx, g in enumerate(circ.gates):
            if idx in xindex:
                k = xindex[idx]
                qa = g.qubits[0] if not inB(g.qubits[0]) else g.qubits[1]
                qb = g.qubits[1] if qa == g.qubits[0] else g.qubits[0]
                ma = np.zeros(32)
                mb = np.zeros(32)
                for d, (Af, Bf) in enumerate(self.terms[k]):
                    ma[8 * d:8 * d + 8] = _mat32(Af)[:8]
                    mb[8 * d:8 * d + 8] = _mat32(Bf)[:8]
                opsA.append((1, locA[qa], -1, k, ma))
                opsB.append((1, locB[qb], -1, k, mb))
            elif all(not inB(q) for q in g.qubits):
                opsA.append(self._local(g, locA))
            else:
                opsB.append(self._local(g, locB))
        self.opsA = self._pack(opsA)
        self.opsB = self._pack(opsB)
        self.n_cross = len(cross)

    @staticmethod
    def _local(g, loc):
        q1 = loc[g.qubits[1]] if len(g.qubits) > 1 else -1
        return (len(g.qubits), loc[g.qubits[0]], q1, -1, _mat32(g.mat))

    @staticmethod
    def _pack(ops):
        if not ops:
            z = np.zeros(0, dtype=np.int32)
            return (z, z, z, z, np.zeros(32))
        return (np.array([o[0] for o in ops], dtype=np.int32),
                np.array([o[1] for o in ops], dtype=np.int32),
                np.array([o[2] for o in ops], dtype=np.int32),
                np.array([o[3] for o in ops], dtype=np.int32),
                np.concatenate([o[4] for o in ops]))

    def path_digits(self, path_ids):
        d = np.zeros((len(path_ids), max(1, self.n_cross)), dtype=np.int32)
        for r, p in enumerate(path_ids):
            if self.n_cross:
                d[r, :self.n_cross] = paths.digits(int(p), self.bits)
        return d


def sf_amplitudes(setup, path_ids, xs):
    """Sum over the given paths of A_j[x_A] * B_j[x_B] (complex128)."""
    xs = np.ascontiguousarray(xs, dtype=np.uint64)
    dig = np.ascontiguousarray(setup.path_digits(path_ids))
    nA, a0A, a1A, xgA, mA = setup.opsA
    nB, a0B, a1B, xgB, mB = setup.opsB
    out = np.zeros(2 * len(xs), dtype=np.float64)
    rc = lib().oracle_sf(len(setup.posA), _p(setup.posA), len(nA), _p(nA), _p(a0A), _p(a1A),
                         _p(xgA), _p(mA),
                         len(setup.posB), _p(setup.posB), len(nB), _p(nB), _p(a0B), _p(a1B),
                         _p(xgB), _p(mB),
                         max(1, setup.n_cross), len(path_ids), _p(dig), len(xs), _p(xs), _p(out))
    if rc != 0:
        raise RuntimeError(f"oracle_sf failed: {rc}")
    return out[0::2] + 1j * out[1::2]
