"""Writes tests/golden/oracle_7x8_d40_paths.npz: FP64 oracle amplitudes of
single paths of the 7x8, depth 1+40+1 workload (28+28-qubit halves), one row
per path, for the first 1024 of the workload's 1M bitstrings.

Only the oracle (oracle/) computes these values; nothing from the CUDA
library is read or run. The paths are those of the first prefix of the
f = 0.5% FRACTION selection (seed 7, 28 prefix bits, 2^7 suffixes per
prefix, Section 3 / Eq. 3):
  * suffixes 0..15: one whole group of the last branching level (its four
    cut CZs, 16 leaves), which the library contracts in closed form;
  * eight suffixes scattered over the other seven groups (partial groups).
A full 7x8 path takes the oracle one to two minutes on eight cores, so the
stored values stand in for running it inside the GPU tests.

    python tests/golden/make_oracle_7x8.py [--out PATH]
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import circuit as ocirc  # noqa: E402
from oracle import paths as opaths  # noqa: E402
from oracle import sim  # noqa: E402
from paper_1807_10749_gb300 import inputs  # noqa: E402

WORKLOAD = "7x8_d40"
FIDELITY = 0.005
SEED = 7
N_BITS = 1024
SCATTERED = (19, 39, 44, 64, 89, 111, 117, 127)  # suffixes outside group 0


def path_ids(x_bits):
    pre, x_s, _ = opaths.fraction_prefixes(x_bits, FIDELITY, SEED)
    base = int(pre[0]) << (x_bits - x_s)
    return np.array([base + s for s in list(range(16)) + list(SCATTERED)], dtype=np.uint64), int(pre[0])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "oracle_7x8_d40_paths.npz"))
    args = ap.parse_args()
    w = inputs.WORKLOADS[WORKLOAD]
    text = inputs.workload_circuit(WORKLOAD).text()
    setup = sim.SFSetup(ocirc.parse(text), w["side_b_mask"])
    ids, prefix = path_ids(setup.x_bits)
    bits = inputs.random_bitstrings(56, w["n_bitstrings"], w["bitstring_seed"])[:N_BITS]
    sim.build()
    amps = np.zeros((len(ids), N_BITS), dtype=np.complex128)
    for r, j in enumerate(ids):
        t0 = time.perf_counter()
        amps[r] = sim.sf_amplitudes(setup, np.array([j], dtype=np.uint64), bits)
        print(f"path {int(j)}: {time.perf_counter() - t0:.1f} s", flush=True)
    np.savez_compressed(args.out, ids=ids, bits=bits, amps=amps, prefix=np.array(prefix),
                        note=np.array("FP64 oracle (oracle/core.c): per-path amplitudes of the 7x8 depth "
                                      "1+40+1 workload, first prefix of the f = 0.5% selection (seed 7), "
                                      "first 1024 of the 1M bitstrings (seed of the workload)"))
    print("wrote", args.out)


if __name__ == "__main__":
    main()
