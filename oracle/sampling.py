"""Rejection sampling from computed probabilities (Section 4; oracle, test
infrastructure only).

Algorithm 1 (basic): M = ceil(ln(N / eps)); drop bitstrings with
p(x) > M/N; accept each remaining x_j with probability p(x_j) N / M.
Algorithm 2 (frugal): a fixed M' (10 in the paper); accept each x_j with
probability min(1, p(x_j) N / M').

The uniform numbers of the accept tests are inputs (u_j in [0, 1)); a
bitstring is accepted iff u_j < p_j N / M (the same comparison in FP64 on
both sides).

Closed forms under the exponential (Porter-Thomas) law of N p:
  basic:  expected count of p(x) > M/N is N e^{-M}, so M = ln(N / eps);
  frugal: the dropped mass is int_{M'}^inf t e^{-t} dt = e^{-M'} (1 + M');
  frugal without the drop step (Algorithm 2 as printed):
          total variation 2 exp(-M' / (1 - e^{-M'})).
"""
import math

import numpy as np


def basic_M(N, eps):
    return math.ceil(math.log(N / eps))


def frugal_eps(Mp):
    return math.exp(-Mp) * (1.0 + Mp)


def frugal_tv_no_drop(Mp):
    return 2.0 * math.exp(-Mp / (1.0 - math.exp(-Mp)))


def accept_basic(p, u, N, M):
    p = np.asarray(p, dtype=np.float64)
    keep = p <= M / N
    return keep & (np.asarray(u) < p * N / M)


def accept_frugal(p, u, N, Mp):
    p = np.asarray(p, dtype=np.float64)
    return np.asarray(u) < np.minimum(1.0, p * N / Mp)


def dropped_mass(p, N, Mp):
    """sum over x with p(x) > M'/N of p(x), the empirical epsilon of the
    frugal sampler (Section 4: measured on the exact and approximate runs)."""
    p = np.asarray(p, dtype=np.float64)
    return float(p[p > Mp / N].sum())
