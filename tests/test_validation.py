"""Validation protocol of Appendix C on the GPU path, through the C ABI:
sf_overlap_device against the oracle's overlap sums on the same amplitudes,
then the protocol itself on the 30-qubit 5x6, depth 1+24+1 circuit."""
import numpy as np
import pytest

from oracle import validation
from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available()
    from paper_1807_10749_gb300 import build
    build.build()


def _overlap(a, b):
    import torch
    da = torch.from_numpy(np.stack([a.real, a.imag], 1).copy()).cuda()
    db = torch.from_numpy(np.stack([b.real, b.imag], 1).copy()).cuda()
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    sfsim.sf_overlap_device(da, db, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n", [0, 1, 255, 257, 100003])
def test_overlap_sums_match_oracle(n):
    rng = np.random.default_rng(n + 1)
    a = rng.normal(size=n) + 1j * rng.normal(size=n)
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    out = _overlap(a, b)
    got = out[:4]
    want = np.array(validation.overlap_sums(a, b)) if n else np.zeros(4)
    # FP64 sums in another order: relative rounding ~ n * 2^-53
    assert np.all(np.abs(got - want) <= 1e-12 * (np.abs(a).sum() * np.abs(b).sum() / max(n, 1) + n))
    # the library's estimate f_e (Appendix C), 0 for empty sets
    fe = validation.fidelity_estimate(a, b) if n else 0.0
    assert abs(out[4] - fe) <= 1e-10 * max(fe, 1e-300) + 1e-15


@pytest.fixture(scope="module")
def c2():
    w = inputs.WORKLOADS["5x6_d24"]
    # path-level selection (x_s = x = 15): a random fraction f of the paths
    plan = sfsim.Plan(inputs.workload_circuit("5x6_d24").text(), side_b_mask=w["side_b_mask"],
                      select_prefix_bits=15)
    bits = inputs.random_bitstrings(30, w["n_bitstrings"], 77)   # the Verifier's seeded indices
    exact, _ = plan.amplitudes(bits, sfsim.selection("fraction", fidelity=1.0))
    yield plan, bits, exact
    plan.close()


@pytest.mark.parametrize("f", [1 / 4, 1 / 16, 1 / 64])
def test_fidelity_estimate_tracks_f_actual(c2, f):
    """The exact Claimant against a Verifier that sums a random fraction f of
    the paths (Section 3, Fig. 5; a statistical check): over three seeded
    selections the mean of f_e / f_actual is within 10% of 1 and each one
    within 25%; f_e is within 0.02 + 10% of the Verifier's own estimate
    2^n E|v|^2 (Appendix C)."""
    plan, bits, exact = c2
    ratios = []
    for seed in (5, 6, 7):
        ver, f_actual = plan.amplitudes(bits, sfsim.selection("fraction", fidelity=f, seed=seed))
        sums = _overlap(exact, ver)
        np.testing.assert_allclose(sums[:4], validation.overlap_sums(exact, ver), rtol=1e-10)
        fe = sfsim.fidelity_estimate(sums)
        f1 = 2.0 ** 30 * np.mean(np.abs(ver) ** 2)
        print(f"f = {f}, seed {seed}: f_e = {fe:.4f}, f1 = {f1:.4f}, f_actual = {f_actual:.4f}")
        assert abs(fe - f1) <= 0.02 + 0.1 * f1, (fe, f1)
        ratios.append(fe / f_actual)
    assert abs(np.mean(ratios) - 1) <= 0.1, ratios
    assert all(abs(r - 1) <= 0.25 for r in ratios), ratios


def test_protocol_pass_and_fail(c2):
    plan, bits, exact = c2
    ver, _ = plan.amplitudes(bits, sfsim.selection("fraction", fidelity=1 / 8, seed=5))
    f1 = 2.0 ** 30 * np.mean(np.abs(ver) ** 2)
    delta = 0.03
    assert validation.protocol_passes(exact, ver, f1, delta)
    assert abs(sfsim.fidelity_estimate(_overlap(exact, ver)) - f1) <= delta
    # a Claimant that simulated another circuit of the family fails
    spec = inputs.google_circuit(5, 6, 24, 1234)
    wrong = sfsim.Plan(spec.text(), side_b_mask=inputs.WORKLOADS["5x6_d24"]["side_b_mask"])
    bad, _ = wrong.amplitudes(bits, sfsim.selection("fraction", fidelity=1.0))
    fe_bad = sfsim.fidelity_estimate(_overlap(bad, ver))
    assert fe_bad < 0.01 and abs(fe_bad - f1) > delta
    wrong.close()


def test_independent_approximations_overlap_f1_times_f(c2):
    """Two independent path subsets of fidelities f1 and f: their estimated
    fidelity is f1*f on average over the seeds (Appendix C)."""
    plan, bits, exact = c2
    got, want = [], []
    for s in range(8):
        v, _ = plan.amplitudes(bits, sfsim.selection("fraction", fidelity=1 / 4, seed=100 + s))
        w, _ = plan.amplitudes(bits, sfsim.selection("fraction", fidelity=1 / 2, seed=200 + s))
        f1 = sfsim.fidelity_estimate(_overlap(exact, v))
        f = sfsim.fidelity_estimate(_overlap(exact, w))
        got.append(sfsim.fidelity_estimate(_overlap(v, w)))
        want.append(f1 * f)
    print("overlap per seed", np.round(got, 4), "f1*f", np.round(want, 4))
    assert abs(np.mean(got) - np.mean(want)) <= 0.3 * np.mean(want)
