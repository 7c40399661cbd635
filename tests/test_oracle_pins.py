"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself: an identity
the paper prints, a closed form, an independent brute-force computation, a
statistical law, or a count printed in the paper's tables.
"""
import os

import numpy as np
import pytest

from oracle import circuit, decomp, dense, gates, paths, sim
from paper_1807_10749_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def circ(rows, cols, depth, seed=1, **kw):
    return circuit.parse(inputs.google_circuit(rows, cols, depth, seed, **kw).text())


# ---------------------------------------------------------------- gate algebra
def test_gate_algebra():
    """Principal square roots and phase gates (Section 1 gate set)."""
    assert np.allclose(gates.X_HALF @ gates.X_HALF, gates.X, atol=1e-15)
    assert np.allclose(gates.Y_HALF @ gates.Y_HALF, gates.Y, atol=1e-15)
    assert np.allclose(gates.H @ gates.H, gates.I2, atol=1e-15)
    assert np.allclose(np.linalg.matrix_power(gates.T, 8), gates.I2, atol=1e-15)
    assert np.allclose(gates.T @ gates.T, gates.S, atol=1e-15)
    for m in list(gates.ONE_QUBIT.values()) + list(gates.TWO_QUBIT.values()):
        assert np.allclose(m.conj().T @ m, np.eye(len(m)), atol=1e-15)
    # principal roots: eigenvalues of X^1/2, Y^1/2 are 1 and i (not -1, -i)
    for m in (gates.X_HALF, gates.Y_HALF):
        ev = sorted(np.linalg.eigvals(m), key=lambda z: z.imag)
        assert np.allclose(ev, [1, 1j], atol=1e-14)


# -------------------------------------------------------------- decompositions
def test_eq1_projector_decomposition_of_cz():
    """Eq. 1: CZ = P0 (x) I + P1 (x) Z, exactly; and mirrored (CZ is
    symmetric), I (x) P0 + Z (x) P1, with terms that differ from Eq. 1's."""
    rec = decomp.reconstruct(decomp.projector_cz())
    assert np.array_equal(rec, gates.CZ)
    mir = decomp.projector_cz(on_b=True)
    assert np.array_equal(decomp.reconstruct(mir), gates.CZ)
    for (a, b), (c, d) in zip(decomp.projector_cz(), mir):
        assert not np.array_equal(np.kron(a, b), np.kron(c, d))


def test_alternate_projector_side_full_sum_equals_state_vector():
    """Eq. 2 under the mirrored Eq. 1 on every odd-numbered cut CZ: the sum
    over all paths is still the exact amplitude, while single paths differ
    from those of Eq. 1 on the A side (4x4, 1+10+1, all 2^16 bitstrings)."""
    w = inputs.WORKLOADS["4x4_d10"]
    c = circ(4, 4, 10)
    xs = np.arange(1 << 16, dtype=np.uint64)
    sv = sim.sv_amplitudes(c, xs)
    alt = sim.SFSetup(c, w["side_b_mask"], projector_side="alternate")
    std = sim.SFSetup(c, w["side_b_mask"])
    sf = sim.sf_amplitudes(alt, _all_paths(alt), xs)
    assert np.abs(sf - sv).max() < 1e-12 * 2 ** -8
    one = np.array([1], dtype=np.uint64)   # digit 1 on the last (odd-numbered) cut gate
    assert np.abs(sim.sf_amplitudes(alt, one, xs) - sim.sf_amplitudes(std, one, xs)).max() > 1e-4


def test_eq4way_block_decomposition():
    """Eq. 4way reconstructs any 4x4 matrix (unitary or not) exactly."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        U = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
        assert np.array_equal(decomp.reconstruct(decomp.block4(U)), U)


def test_eq_iswap1_and_iswap2():
    """Eq. iSWAP1 is the block form of iSWAP; Eq. iSWAP2 (with the printed
    doubled '+' read as one): 2 iSWAP = II + i XX + i YY + ZZ."""
    t = decomp.block4(gates.ISWAP)
    want = [(gates.P0, gates.P0), (gates.P1, gates.P1),
            (gates.K01, 1j * gates.K10), (gates.K10, 1j * gates.K01)]
    for (a, b), (wa, wb) in zip(t, want):
        assert np.array_equal(a, wa) and np.array_equal(b, wb)
    rhs = (np.kron(gates.I2, gates.I2) + 1j * np.kron(gates.X, gates.X)
           + 1j * np.kron(gates.Y, gates.Y) + np.kron(gates.Z, gates.Z))
    assert np.allclose(2 * gates.ISWAP, rhs, atol=0)


def test_schmidt_decomposition():
    """Operator-Schmidt rank is 1, 2 or 4 for unitaries (Section 7); iSWAP has
    four equal coefficients; every decomposition reconstructs its gate."""
    hr = inputs.SplitMix64(11, inputs.PURPOSE_HAAR)
    for _ in range(10):
        U = inputs.haar_unitary(4, hr)
        t = decomp.schmidt(U)
        assert len(t) == 4
        assert np.abs(decomp.reconstruct(t) - U).max() < 1e-13
        # gauge: first significant entry of each A_k real positive
        for A, _ in t:
            z = next(v for v in A.reshape(-1) if abs(v) > 1e-12)
            assert abs(z.imag) < 1e-14 and z.real > 0
    assert len(decomp.schmidt(gates.CZ)) == 2
    assert len(decomp.schmidt(np.kron(gates.H, gates.T))) == 1
    t = decomp.schmidt(gates.ISWAP)
    assert len(t) == 4
    sig = [np.linalg.norm(B) for _, B in t]   # ||A_k||_F = 1
    assert np.allclose(sig, 1.0, atol=1e-13)
    assert np.abs(decomp.reconstruct(t) - gates.ISWAP).max() < 1e-13


# --------------------------------------------------------- state-vector oracle
@pytest.mark.parametrize("rows,cols,depth", [(2, 2, 9), (2, 3, 10), (2, 4, 9), (3, 3, 8), (2, 5, 12)])
@pytest.mark.parametrize("kind", ["cz", "haar", "iswap"])
def test_sv_matches_dense_bruteforce(rows, cols, depth, kind):
    c = circ(rows, cols, depth, seed=7, haar=(kind == "haar"), iswap=(kind == "iswap"))
    psi = dense.dense_state(c)
    xs = np.arange(1 << c.n, dtype=np.uint64)
    a = sim.sv_amplitudes(c, xs)
    assert np.abs(a - psi).max() < 1e-12


def test_initial_h_closed_form():
    """The initial H layer gives amplitude 2^{-n/2} on every bitstring; adding
    only diagonal gates (CZ, T) keeps every modulus at 2^{-n/2}."""
    spec = inputs.google_circuit(4, 4, 10, seed=2)
    only_h = inputs.CircuitSpec(4, 4, [g for g in spec.gates if g.cycle == 0])
    diag = inputs.CircuitSpec(4, 4, [g for g in spec.gates if g.cycle == 0 or g.name in ("cz", "t")])
    xs = np.arange(1 << 16, dtype=np.uint64)
    a = sim.sv_amplitudes(circuit.parse(only_h.text()), xs)
    assert np.abs(a - 2.0 ** -8).max() < 1e-15
    b = sim.sv_amplitudes(circuit.parse(diag.text()), xs)
    assert np.abs(np.abs(b) - 2.0 ** -8).max() < 1e-15
    assert np.abs(b - 2.0 ** -8).max() > 1e-3  # the phases are not trivial


def test_norm_and_mean_probability():
    """Norm 1; mean probability 2^{-n} (the run logs print 2^-30, 2^-32)."""
    c = circ(4, 4, 10)
    a = sim.sv_amplitudes(c, np.arange(1 << 16, dtype=np.uint64))
    p = np.abs(a) ** 2
    assert abs(p.sum() - 1) < 1e-12
    assert abs(p.mean() * 2 ** 16 - 1) < 1e-12


def test_porter_thomas_moments():
    """Deep random circuits: E[N p] = 1 and E[(N p)^2] ~ 2 (Section 4, Fig. 4)."""
    c = circ(4, 5, 40, seed=1)
    N = 1 << c.n
    p = np.abs(sim.sv_amplitudes(c, np.arange(N, dtype=np.uint64))) ** 2
    assert abs((N * p).mean() - 1) < 1e-10
    assert abs(((N * p) ** 2).mean() - 2) < 0.05   # exponential law: E[t^2] = 2
    assert abs(((N * p) ** 3).mean() - 6) < 0.3    # E[t^3] = 3! = 6
    # the shallow 4x4 depth-10 circuit is not Porter-Thomas: only its mean holds
    c = circ(4, 4, 10)
    p = np.abs(sim.sv_amplitudes(c, np.arange(1 << 16, dtype=np.uint64))) ** 2
    assert abs((2 ** 16 * p).mean() - 1) < 1e-10


# -------------------------------------------------------- path-sum oracle (SF)
def _all_paths(setup):
    return np.arange(1 << setup.x_bits, dtype=np.uint64)


@pytest.mark.parametrize("kind,dec", [("cz", "schmidt"), ("haar", "schmidt"), ("haar", "block4"),
                                      ("iswap", "block4"), ("iswap", "schmidt")])
def test_sf_full_sum_equals_state_vector(kind, dec):
    """Eq. 2: the sum over all 2^x paths is the exact amplitude (4x4, 1+10+1,
    rows 0-1 | 2-3, all 2^16 bitstrings)."""
    w = inputs.WORKLOADS["4x4_d10"]
    c = circ(4, 4, 10, haar=(kind == "haar"), iswap=(kind == "iswap"))
    xs = np.arange(1 << 16, dtype=np.uint64)
    sv = sim.sv_amplitudes(c, xs)
    setup = sim.SFSetup(c, w["side_b_mask"], dec)
    assert setup.x_bits == (4 if kind == "cz" else 8)
    sf = sim.sf_amplitudes(setup, _all_paths(setup), xs)
    assert np.abs(sf - sv).max() < 1e-12 * 2 ** -8
    assert abs((np.abs(sf) ** 2).sum() - 1) < 1e-12


def test_sf_vertical_cut_20_qubits():
    """Full path sum vs state vector on a 4x5 grid cut 10+10 (cols 0-1 | 2-4)."""
    c = circ(4, 5, 16, seed=4)
    mask = inputs.column_cut_mask(4, 5, 2)
    xs = inputs.random_bitstrings(20, 2000, 99)
    sv = sim.sv_amplitudes(c, xs)
    setup = sim.SFSetup(c, mask)
    sf = sim.sf_amplitudes(setup, _all_paths(setup), xs)
    assert np.abs(sf - sv).max() < 1e-12 * 2 ** -10


def test_sf_without_cross_gates_is_a_product():
    """x = 0: a single path, the amplitude is A[x_A] * B[x_B]."""
    c = circ(4, 4, 2)  # cycles 1-2 use H00 and V00: no edge crosses rows 1|2
    w = inputs.WORKLOADS["4x4_d10"]
    setup = sim.SFSetup(c, w["side_b_mask"])
    assert setup.x_bits == 0
    xs = np.arange(1 << 16, dtype=np.uint64)
    assert np.abs(sim.sf_amplitudes(setup, np.zeros(1, np.uint64), xs)
                  - sim.sv_amplitudes(c, xs)).max() < 1e-15


def test_planted_mistakes_fail_the_pins():
    """A dropped term, a wrong sign or a transposed operand in the oracle's
    input makes the f = 1 pin fail (mistakes planted on the CPU)."""
    w = inputs.WORKLOADS["4x4_d10"]
    c = circ(4, 4, 10)
    xs = np.arange(1 << 16, dtype=np.uint64)
    sv = sim.sv_amplitudes(c, xs)
    setup = sim.SFSetup(c, w["side_b_mask"])
    good = sim.sf_amplitudes(setup, _all_paths(setup), xs)
    assert np.abs(good - sv).max() < 1e-14
    # Z on the B side replaced by I (dropped sign)
    nB, a0B, a1B, xgB, mB = setup.opsB
    bad = mB.copy()
    for o in np.nonzero(xgB >= 0)[0]:
        bad[32 * o + 8 + 6] = 1.0  # term 1, entry (1,1) real part: -1 -> +1
    setup.opsB = (nB, a0B, a1B, xgB, bad)
    assert np.abs(sim.sf_amplitudes(setup, _all_paths(setup), xs) - sv).max() > 1e-4
    setup.opsB = (nB, a0B, a1B, xgB, mB)
    # a dropped path
    assert np.abs(sim.sf_amplitudes(setup, _all_paths(setup)[1:], xs) - sv).max() > 1e-4
    # X^1/2 transposed (= its own transpose) is harmless, Y^1/2 transposed is not
    spec = inputs.google_circuit(4, 4, 10, 1)
    assert any(g.name == "y_1_2" for g in spec.gates)
    c2 = circuit.parse(spec.text())
    for g in c2.gates:
        if g.name == "y_1_2":
            g.mat = g.mat.T.copy()
    assert np.abs(sim.sv_amplitudes(c2, xs) - sv).max() > 1e-4


# ----------------------------------------------------------------- selection
def test_feistel_is_a_permutation():
    for w in range(0, 13):
        vals = [paths.feistel(i, w, 12345) for i in range(1 << w)]
        assert sorted(vals) == list(range(1 << w))
    assert paths.feistel(0, 28, 7) < (1 << 28)


def test_selection_modes():
    # digits: MSB = earliest gate
    assert paths.digits(0b10_1_0, [2, 1, 1]) == [2, 1, 0]
    ids, fa = paths.select_fraction(10, 1.0, 7)
    assert fa == 1.0 and np.array_equal(np.sort(ids), np.arange(1024, dtype=np.uint64))
    ids, fa = paths.select_fraction(10, 0.25, 7)
    assert fa == 0.25 and len(ids) == 256 and len(set(ids.tolist())) == 256
    # whole prefixes: each selected id's suffix (low 7 bits) runs over 0..127
    pre = sorted(set(int(i) >> 7 for i in ids))
    assert len(pre) == 2
    pre, xs, fa = paths.fraction_prefixes(35, 0.005, 7)
    assert xs == 28 and len(pre) == 1342177 and len(set(pre)) == len(pre)
    assert fa == 1342177 / 2 ** 28
    assert np.array_equal(paths.select_range(5, 3), np.array([5, 6, 7], dtype=np.uint64))


# ------------------------------------------------- approximation (Section 3)
def test_truncated_sum_norm_and_fidelity_track_f():
    """Eq. 3 / Fig. 5: keeping a fraction f of the paths gives norm ~ f and
    fidelity ~ f (4x4, 1+32+1, rows 0-1 | 2-3: 16 cut CZs; 4096 bitstrings)."""
    c = circ(4, 4, 32, seed=5)
    w = inputs.WORKLOADS["4x4_d10"]
    setup = sim.SFSetup(c, w["side_b_mask"])
    assert setup.x_bits == 16
    xs = np.arange(1 << 16, dtype=np.uint64)
    psi = sim.sv_amplitudes(c, xs)
    for f in (1 / 4, 1 / 16):
        ids, fa = paths.select_fraction(setup.x_bits, f, 7)
        a = sim.sf_amplitudes(setup, ids, xs)
        norm = (np.abs(a) ** 2).sum()
        fid = abs(np.vdot(psi, a)) ** 2 / norm
        assert norm == pytest.approx(fa, rel=0.10)
        assert fid == pytest.approx(fa, rel=0.10)


# ------------------------------------------------------ generator vs Table 2
def test_gate_counts_match_table2_and_goldens():
    with open(os.path.join(HERE, "golden", "gate_counts.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    v2rows = [r for r in rows if r[0] == "v2"]
    rows = [r for r in rows if r[0] != "v2"]
    for _, R, C, D, nxy, nt in v2rows:
        spec = inputs.google_circuit(int(R), int(C), int(D), 1, v2=True)
        assert sum(g.name in ("x_1_2", "y_1_2") for g in spec.gates) == int(nxy)
        assert sum(g.name == "t" for g in spec.gates) == int(nt)
    for R, C, D, kind, fb, ncz, nx, cyc in rows:
        R, C, D, fb = int(R), int(C), int(D), int(fb)
        mask = inputs.column_cut_mask(R, C, fb) if kind == "col" else inputs.row_cut_mask(R, C, fb)
        spec = inputs.google_circuit(R, C, D, 1)
        cz = [g for g in spec.gates if g.name == "cz"]
        x = [g for g in cz if ((mask >> g.qubits[0]) & 1) != ((mask >> g.qubits[1]) & 1)]
        assert len(cz) == int(ncz) and len(x) == int(nx)
        assert sorted(set(g.cycle for g in x)) == [int(v) for v in cyc.split(",")]


def test_v2_circuits_have_no_diagonal_only_gap_between_cut_czs():
    """Section 6: the v2 rule leaves no CZ - (diagonal gates) - CZ run on a cut
    qubit, so no path of the 7x8 workload is zero by construction; the T-first
    rule leaves six such runs there (63/64 of the paths vanish)."""
    def gaps(spec, mask):
        inB = lambda q: (mask >> q) & 1
        n = 0
        seq = {}
        for g in spec.gates:
            for q in g.qubits:
                if not inB(q):
                    seq.setdefault(q, []).append(g)
        for q, gs in seq.items():
            last, diag = False, True
            for g in gs:
                if len(g.qubits) == 2 and inB(g.qubits[0]) != inB(g.qubits[1]):
                    n += last and diag
                    last, diag = True, True
                elif g.name in ("x_1_2", "y_1_2", "h"):
                    diag = False
        return n
    w = inputs.WORKLOADS["7x8_d40"]
    assert gaps(inputs.workload_circuit("7x8_d40"), w["side_b_mask"]) == 0
    assert gaps(inputs.google_circuit(7, 8, 40, 1), w["side_b_mask"]) == 6
