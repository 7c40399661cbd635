"""Fidelity estimate of the validation protocol (Appendix C; oracle, test
infrastructure only): on a common set of bitstrings, the Verifier's
approximate amplitudes b and the Claimant's amplitudes a give
f_e = |<a|b>|^2 / (<a|a> <b|b>); the test passes if |f_e - f_1| <= delta."""
import numpy as np


def overlap_sums(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ip = np.vdot(a, b)
    return ip.real, ip.imag, float(np.vdot(a, a).real), float(np.vdot(b, b).real)


def fidelity_estimate(a, b):
    re, im, na, nb = overlap_sums(a, b)
    return (re * re + im * im) / (na * nb)


def protocol_passes(claimant, verifier, f1, delta):
    return abs(fidelity_estimate(claimant, verifier) - f1) <= delta
