"""FP64 CPU oracle for the Schroedinger-Feynman path sum of arXiv:1807.10749.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg (and its reference arm) may import or run this package. The
CUDA library never calls it and shares no code with it.

What it computes, plainly and slowly, in complex128:
  * sv_amplitudes  - full state-vector (Schroedinger) simulation (Section 2),
    one dense 2x2 / 4x4 gate at a time, in circuit order;
  * dense_amplitudes - brute force: every gate as a 2^n x 2^n matrix built from
    Kronecker products (n <= 10);
  * sf_amplitudes  - the Schroedinger-Feynman path sum of Eq. 2 (and its
    truncation, Eq. 3): for every selected path, evolve the two halves from
    |0...0> independently, applying the path's term of each cross-cut gate
    (Eq. 1 for CZ; the operator-Schmidt or the four-block decomposition of
    Section 7 for other gates), then add A[x_A] * B[x_B] to each requested
    amplitude with Neumaier-compensated summation;
  * path selection (RANGE, FRACTION, LIST) per Eq. 3 and Section 3;
  * frugal rejection sampling (Section 4, Algorithm 2).

Pins (tests/test_oracle_*.py): gate algebra, exact reconstruction of every
decomposition (Eq. 1, Eq. 4way, Eq. iSWAP2), state vector vs brute force for
n <= 10, the initial-H closed form 2^{-n/2}, norm preservation, path sum at
f = 1 equal to the state vector, Porter-Thomas moments of deep circuits, and
fidelity ~ f for truncated sums.
"""
