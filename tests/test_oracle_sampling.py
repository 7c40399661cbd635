"""Pins of the rejection-sampling oracle (Section 4, Algorithms 1 and 2)."""
import math

import numpy as np

from oracle import circuit, sampling, sim
from paper_1807_10749_gb300 import inputs


def test_printed_constants():
    # M = ceil(ln(10^3 * 2^49)) = 41 for eps = 1e-3, n = 49
    assert sampling.basic_M(2.0 ** 49, 1e-3) == 41
    # frugal, M' = 10: eps = e^-10 * 11 = 5e-4 (printed "5 * 10^-4")
    assert abs(sampling.frugal_eps(10) - 4.994e-4) < 1e-6
    # accepting high probabilities instead of dropping them: 9e-5 (printed)
    assert abs(sampling.frugal_tv_no_drop(10) - 9.08e-5) < 1e-7


def test_closed_forms_by_quadrature():
    # e^{-M'}(1+M') = int_{M'}^inf t e^{-t} dt, numerically
    t = np.linspace(10, 80, 700001)
    assert abs(np.trapezoid(t * np.exp(-t), t) - sampling.frugal_eps(10)) < 1e-9


def test_acceptance_rule_and_rate_on_porter_thomas():
    """Exact 4x5 depth-40 probabilities (Porter-Thomas): the frugal sampler
    accepts ~1/M' of the candidates, its dropped mass is ~e^{-M'}(1+M'), and
    the accepted bitstrings follow p (heavier ones more often)."""
    c = circuit.parse(inputs.google_circuit(4, 5, 40, 1).text())
    N = 1 << c.n
    p = np.abs(sim.sv_amplitudes(c, np.arange(N, dtype=np.uint64))) ** 2
    rng = np.random.default_rng(5)
    u = rng.random(N)
    acc = sampling.accept_frugal(p, u, N, 10)
    assert abs(acc.mean() - 0.1) < 0.005            # E[min(1, Np/10)] ~ 1/10
    assert abs(sampling.dropped_mass(p, N, 10) - sampling.frugal_eps(10)) < 3e-4
    # acceptance probability is monotone in p: heavier half accepted more
    heavy = p > np.median(p)
    assert acc[heavy].mean() > 3 * acc[~heavy].mean()
    # basic sampler never accepts a dropped bitstring
    M = 12
    b = sampling.accept_basic(p, u, N, M)
    assert not np.any(b & (p > M / N))
    # a planted mistake (N p / M' replaced by p / M') accepts almost nothing
    assert (u < np.minimum(1.0, p / 10)).mean() < 1e-3


def test_validation_protocol_oracle():
    """Appendix C: the Verifier sums a fraction of the paths, reaching a state
    of fidelity f1 (its squared norm, here known over all 2^16 bitstrings);
    on k = 4096 seeded bitstrings the exact Claimant's amplitudes give
    f_e within delta of f1, while a Claimant who simulated another circuit
    gives f_e ~ 0 and fails; identical states give 1."""
    from oracle import paths, validation
    c = circuit.parse(inputs.google_circuit(4, 4, 32, 5).text())
    xs = np.arange(1 << 16, dtype=np.uint64)
    exact = sim.sv_amplitudes(c, xs)
    setup = sim.SFSetup(c, inputs.WORKLOADS["4x4_d10"]["side_b_mask"])
    ids, _ = paths.select_fraction(setup.x_bits, 1 / 4, 21)
    ver = sim.sf_amplitudes(setup, ids, xs)
    f1 = validation.fidelity_estimate(exact, ver)
    assert 0.1 < f1 < 0.4
    assert abs(f1 - np.vdot(ver, ver).real) < 1e-9   # fidelity of a path-sum = its norm here
    k = np.random.default_rng(3).choice(1 << 16, 4096, replace=False)
    assert abs(validation.fidelity_estimate(exact, exact) - 1) < 1e-12
    assert validation.protocol_passes(exact[k], ver[k], f1, 0.02)
    other = sim.sv_amplitudes(circuit.parse(inputs.google_circuit(4, 4, 32, 6).text()), xs)
    assert validation.fidelity_estimate(other[k], ver[k]) < 0.01
    assert not validation.protocol_passes(other[k], ver[k], f1, 0.02)


def test_fidelity_estimate_pins():
    """f_e = |<a|b>|^2 / (<a|a><b|b>) (Appendix C): invariant under complex
    scaling of either argument, symmetric, within [0, 1] (Cauchy-Schwarz), 0
    for orthogonal vectors, and a hand value: a = (1, i), b = (1, 1) gives
    |1 - i|^2 / (2 * 2) = 1/2."""
    from oracle import validation
    rng = np.random.default_rng(5)
    for _ in range(20):
        a = rng.normal(size=64) + 1j * rng.normal(size=64)
        b = rng.normal(size=64) + 1j * rng.normal(size=64)
        c = complex(rng.normal(), rng.normal())
        f = validation.fidelity_estimate(a, b)
        assert 0.0 <= f <= 1.0
        assert abs(validation.fidelity_estimate(b, a) - f) < 1e-12
        assert abs(validation.fidelity_estimate(c * a, b) - f) < 1e-12
        assert abs(validation.fidelity_estimate(a, c * a) - 1.0) < 1e-12
    assert validation.fidelity_estimate(np.array([1, 0]), np.array([0, 1j])) == 0.0
    assert abs(validation.fidelity_estimate(np.array([1, 1j]), np.array([1, 1])) - 0.5) < 1e-15
    re, im, na, nb = validation.overlap_sums(np.array([1, 1j]), np.array([1, 1]))
    assert (re, im, na, nb) == (1.0, -1.0, 2.0, 2.0)   # <a|b> = 1 - i
