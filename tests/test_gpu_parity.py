"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerance (the contract for complex64 halves with FP64 path accumulation):
max |amp_gpu - amp_oracle| <= 1e-5 * 2^{-n/2}. A sum over few paths is far
below 2^{-n/2} (at n = 56 one path is ~2^{-45.5}), where that bound says
nothing, so every case is also held to a relative bound:
    max |d| <= REL_TOL * s,   s = sqrt(mean_x sum_j |a_j(x)|^2),
the magnitude of a sum of paths with independent phases (the RMS of the
summed amplitude when the paths' phases are random), computed from the
oracle's per-path amplitudes a_j where the test has them, else the RMS of
the oracle's sum. Error model: each path's two halves are evolved in FP32
through G gate applications each (G ~ 300 at 6x7, ~560 at 7x8 on the
B half), every one adding a relative rounding of order 2^-24 with a random
sign, so a path's relative error is ~ sqrt(2G) 2^-24 ~ 2e-6 at 7x8; independent
errors over paths add like the paths themselves, which is what s scales.
REL_TOL = 3e-5 leaves a factor of ~15 over that estimate; the measured
values (printed per case) are recorded beside the bound in the design notes.
"""
import os

import numpy as np
import pytest

from oracle import circuit as ocirc
from oracle import paths as opaths
from oracle import sim
from paper_1807_10749_gb300 import inputs, sfsim

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-5
REL_TOL = 3e-5
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1807_10749_gb300 import build
    build.build()
    sim.build()


@pytest.fixture(params=[0, 1, 2], ids=["generic", "specialised-scalar", "specialised-packed"])
def jit(request, monkeypatch):
    """The pass-kernel forms: the generic kernel, and the per-pass specialised
    kernels compiled at plan time with scalar FP32 stages or with packed
    FP32x2 stages (the default)."""
    if request.param == 1:
        orig = sfsim.Plan.__init__

        def scalar(self, text, **kw):
            kw["fp32x2"] = 0
            orig(self, text, **kw)
        monkeypatch.setattr(sfsim.Plan, "__init__", scalar)
    return 0 if request.param == 0 else 1


def check_close(gpu, ref, n, label="", nonzero=True, path_scale=None):
    """path_scale: s of the module docstring from per-path oracle values
    (None: the RMS of the oracle's sum)."""
    err = np.abs(gpu - ref)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    s = rms if path_scale is None else path_scale
    if nonzero:
        assert rms > 0, f"{label}: the reference is identically zero (vacuous comparison)"
    bound = ABS_TOL * 2.0 ** (-n / 2)
    print(f"{label}: max|d| = {err.max():.3e} (= {err.max() / 2.0 ** (-n / 2):.2e} * 2^-n/2), "
          f"max|d|/s = {err.max() / s:.2e}, rms|d|/s = {np.sqrt(np.mean(err ** 2)) / s:.2e}, "
          f"rms|ref| = {rms:.3e}, s = {s:.3e}")
    assert err.max() <= bound, f"{label}: {err.max()} > {bound}"
    assert err.max() <= REL_TOL * s + 1e-300, f"{label}: {err.max()} > {REL_TOL} * s {s}"


def path_scale(per_path):
    """s = sqrt(mean_x sum_j |a_j(x)|^2) from per-path amplitudes (paths x bitstrings)."""
    return float(np.sqrt(np.mean(np.sum(np.abs(per_path) ** 2, axis=0))))


_REF_CACHE = {}


def oracle_sf(setup_key, setup, ids, bits):
    """The oracle's path sum, computed once per case for all kernel forms."""
    key = (setup_key, np.asarray(ids, dtype=np.uint64).tobytes(), bits.tobytes())
    if key not in _REF_CACHE:
        _REF_CACHE[key] = sim.sf_amplitudes(setup, ids, bits)
    return _REF_CACHE[key]


def oracle_per_path(setup_key, setup, ids, bits):
    """The oracle's amplitudes of each path alone (paths x bitstrings), once
    per case for all kernel forms."""
    key = ("per-path", setup_key, np.asarray(ids, dtype=np.uint64).tobytes(), bits.tobytes())
    if key not in _REF_CACHE:
        _REF_CACHE[key] = np.stack([sim.sf_amplitudes(setup, np.array([j], dtype=np.uint64), bits) for j in ids])
    return _REF_CACHE[key]


def workload(name, **kw):
    return inputs.WORKLOADS[name], inputs.workload_circuit(name, **kw).text()


# ----------------------------------------------------------------- 4x4 (C1)
def test_4x4_all_paths_equal_state_vector(jit):
    w, text = workload("4x4_d10")
    c = ocirc.parse(text)
    xs = np.arange(1 << 16, dtype=np.uint64)
    ref = sim.sv_amplitudes(c, xs)
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    amp, fa = p.amplitudes(xs, sfsim.selection("fraction", fidelity=1.0))
    assert fa == 1.0
    check_close(amp, ref, 16, "4x4 f=1 all bitstrings")
    bits = inputs.random_bitstrings(16, 1024, w["bitstring_seed"])
    amp2, _ = p.amplitudes(bits, sfsim.selection("range", first=0, count=16))
    check_close(amp2, sim.sv_amplitudes(c, bits), 16, "4x4 1024 random")
    p.close()


def test_4x4_each_path_alone_matches_oracle(jit):
    """Per-path parity: path numbering and enumeration agree exactly."""
    w, text = workload("4x4_d10")
    c = ocirc.parse(text)
    setup = sim.SFSetup(c, w["side_b_mask"])
    bits = inputs.random_bitstrings(16, 1024, w["bitstring_seed"])
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    for j in range(16):
        ref = sim.sf_amplitudes(setup, np.array([j], dtype=np.uint64), bits)
        amp, _ = p.amplitudes(bits, sfsim.selection("list", ids=[j]))
        check_close(amp, ref, 16, f"4x4 path {j}")
    p.close()


@pytest.mark.parametrize("kind,dec", [("haar", sfsim.SF_DEC_SCHMIDT), ("haar", sfsim.SF_DEC_BLOCK4),
                                      ("iswap", sfsim.SF_DEC_BLOCK4)])
def test_4x4_four_way_branching(kind, dec, jit):
    """Section 7: non-CZ cross gates branch four ways (Schmidt / Eq. 4way)."""
    w, text = workload("4x4_d10", haar=(kind == "haar"), iswap=(kind == "iswap"))
    c = ocirc.parse(text)
    xs = np.arange(1 << 16, dtype=np.uint64)
    ref = sim.sv_amplitudes(c, xs)
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"], decomposition=dec)
    amp, _ = p.amplitudes(xs, sfsim.selection("fraction", fidelity=1.0))
    check_close(amp, ref, 16, f"4x4 {kind} dec={dec}")
    # per-path parity for a few paths (tie-free decompositions)
    if kind == "haar":
        setup = sim.SFSetup(c, w["side_b_mask"], "block4" if dec == sfsim.SF_DEC_BLOCK4 else "schmidt")
        bits = inputs.random_bitstrings(16, 512, 5)
        for j in (0, 37, 255):
            r = sim.sf_amplitudes(setup, np.array([j], dtype=np.uint64), bits)
            a, _ = p.amplitudes(bits, sfsim.selection("list", ids=[j]))
            check_close(a, r, 16, f"4x4 {kind} path {j}")
    p.close()


def test_alternate_projector_side_each_path(jit):
    """Eq. 1 mirrored on the odd-numbered cut CZs (projectors, i.e. pinned
    index bits, on both halves): each of the 16 paths of 4x4 and a 6x7 path
    list (with a whole folded group) against the oracle under the same
    reading."""
    w, text = workload("4x4_d10")
    c = ocirc.parse(text)
    setup = sim.SFSetup(c, w["side_b_mask"], projector_side="alternate")
    bits = inputs.random_bitstrings(16, 1024, w["bitstring_seed"])
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"], projector_side=sfsim.SF_PROJ_ALTERNATE)
    for j in range(16):
        amp, _ = p.amplitudes(bits, sfsim.selection("list", ids=[j]))
        check_close(amp, sim.sf_amplitudes(setup, np.array([j], dtype=np.uint64), bits), 16, f"4x4 alt path {j}")
    p.close()
    w, text = workload("6x7_d26")
    c = ocirc.parse(text)
    setup = sim.SFSetup(c, w["side_b_mask"], projector_side="alternate")
    bits = inputs.random_bitstrings(42, 4096, w["bitstring_seed"])
    ids = inputs.random_path_list(setup.x_bits, 16, 12)
    grp = (int(ids[0]) >> 4) << 4
    ids = np.unique(np.concatenate([ids, np.arange(grp, grp + 16, dtype=np.uint64)]))
    per = oracle_per_path(("6x7", "alt"), setup, ids, bits)
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"], projector_side=sfsim.SF_PROJ_ALTERNATE)
    amp, _ = p.amplitudes(bits, sfsim.selection("list", ids=ids))
    check_close(amp, per.sum(axis=0), 42, f"6x7 alt {len(ids)} paths", path_scale=path_scale(per))
    p.close()


def test_tiny_halves_all_paths(jit):
    """Halves of 4 and 6 qubits: tiles smaller than one copy warp's 32 chunks."""
    for (R, C, cut) in [(2, 4, 2), (3, 4, 2)]:
        text = inputs.google_circuit(R, C, 14, 2).text()
        n = R * C
        c = ocirc.parse(text)
        xs = np.arange(1 << n, dtype=np.uint64)
        p = sfsim.Plan(text, jit=jit, side_b_mask=inputs.column_cut_mask(R, C, cut))
        amp, _ = p.amplitudes(xs, sfsim.selection("fraction", fidelity=1.0))
        check_close(amp, sim.sv_amplitudes(c, xs), n, f"{R}x{C} all paths")
        p.close()


def test_4x4_plain_equals_batched(jit):
    w, text = workload("4x4_d10")
    bits = inputs.random_bitstrings(16, 1024, w["bitstring_seed"])
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    q = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"], exec_mode=sfsim.SF_EXEC_PLAIN)
    sel = sfsim.selection("fraction", fidelity=1.0)
    a, _ = p.amplitudes(bits, sel)
    b, _ = q.amplitudes(bits, sel)
    assert np.abs(a - b).max() <= 1e-6 * 2.0 ** -8
    p.close()
    q.close()


def test_edge_cases(jit):
    w, text = workload("4x4_d10")
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    c = ocirc.parse(text)
    # empty bitstring list, empty selection
    a, _ = p.amplitudes(np.zeros(0, dtype=np.uint64), sfsim.selection("range", count=16))
    assert a.size == 0
    bits = inputs.random_bitstrings(16, 300, 9)
    a, fa = p.amplitudes(bits, sfsim.selection("range", first=3, count=0))
    assert fa == 0 and np.all(a == 0)
    # duplicates and a ragged count
    bits = np.concatenate([bits[:257], bits[:5]])
    a, _ = p.amplitudes(bits, sfsim.selection("range", count=16))
    assert np.array_equal(a[257:], a[:5])
    check_close(a, sim.sv_amplitudes(c, bits), 16, "ragged 262")
    # single bitstring, top bits above n ignored? no: bit q >= n is outside
    a1, _ = p.amplitudes(bits[:1], sfsim.selection("range", count=16))
    assert a1[0] == a[0]
    p.close()


def test_device_form_matches_host_form():
    import torch
    w, text = workload("4x4_d10")
    p = sfsim.Plan(text, side_b_mask=w["side_b_mask"])
    bits = inputs.random_bitstrings(16, 1000, 4)
    sel = sfsim.selection("fraction", fidelity=1.0)
    host, _ = p.amplitudes(bits, sel)
    d_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    d_out = torch.zeros((len(bits), 2), dtype=torch.float64, device="cuda")
    ws = torch.empty(sfsim.sf_workspace_size(p.handle, len(bits), sel), dtype=torch.uint8, device="cuda")
    sfsim.sf_amplitudes_device(p.handle, d_bits, sel, d_out, ws)
    sfsim.sf_amplitudes_device(p.handle, d_bits, sel, d_out, ws, accumulate=True)
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    dev = o[:, 0] + 1j * o[:, 1]
    assert np.abs(dev - 2 * host).max() <= 1e-12 * 2.0 ** -8
    # host form into caller-owned pinned buffers
    pin_bits = torch.from_numpy(bits.view(np.int64)).pin_memory().numpy().view(np.uint64)
    pin_out = torch.empty(2 * len(bits), dtype=torch.float64).pin_memory().numpy()
    fa = sfsim.sf_amplitudes_into(p.handle, pin_bits, sel, pin_out)
    assert fa == 1.0
    assert np.array_equal(pin_out[0::2] + 1j * pin_out[1::2], host)
    p.close()


# ---------------------------------------------------------------- 5x6 (C2)
def test_5x6_path_subsets_match_oracle(jit):
    w, text = workload("5x6_d24")
    c = ocirc.parse(text)
    setup = sim.SFSetup(c, w["side_b_mask"])
    bits = inputs.random_bitstrings(30, 20000, w["bitstring_seed"])
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    for sel, ids in [(sfsim.selection("range", first=5000, count=700), opaths.select_range(5000, 700)),
                     (sfsim.selection("fraction", fidelity=1 / 32, seed=7),
                      opaths.select_fraction(setup.x_bits, 1 / 32, 7)[0])]:
        ref = sim.sf_amplitudes(setup, ids, bits)
        amp, _ = p.amplitudes(bits, sel)
        check_close(amp, ref, 30, f"5x6 {len(ids)} paths")
    p.close()


def test_5x6_full_sum_porter_thomas(jit):
    """All 2^15 paths, 100k bitstrings: E[N p] ~ 1, E[(N p)^2] ~ 2 (Section 4)."""
    w, text = workload("5x6_d24")
    bits = inputs.random_bitstrings(30, w["n_bitstrings"], w["bitstring_seed"])
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    amp, _ = p.amplitudes(bits, sfsim.selection("fraction", fidelity=1.0))
    t = (2.0 ** 30) * np.abs(amp) ** 2
    print("5x6 PT moments", t.mean(), (t ** 2).mean())
    assert abs(t.mean() - 1) < 0.03
    assert abs((t ** 2).mean() - 2) < 0.12
    p.close()


# ---------------------------------------------------------------- 6x7 (C3)
@pytest.mark.parametrize("kind,split,cyc", [("cz", 0, 0), ("cz", 1, 0), ("haar", 0, 0), ("cz", 0, 1)])
def test_6x7_path_list_matches_oracle(kind, split, cyc, jit):
    """64 paths x 4096 bitstrings. CZ: 48 random paths and one whole group of
    the folded last level (16 leaves, contracted in closed form). Haar (every
    cut gate branches 4 ways): 32 random paths and 32 leaves of one group of
    256 (the partial-group form of the contraction). cyc = 1: segments by
    cycle ranges instead of light cones."""
    w, text = workload("6x7_d26", haar=(kind == "haar"))
    c = ocirc.parse(text)
    setup = sim.SFSetup(c, w["side_b_mask"])
    bits = inputs.random_bitstrings(42, 4096, w["bitstring_seed"])
    ids = inputs.random_path_list(setup.x_bits, 48 if kind == "cz" else 32, 11)
    grp = (int(ids[0]) >> 4) << 4 if kind == "cz" else (int(ids[0]) >> 8) << 8
    full = np.arange(grp, grp + (16 if kind == "cz" else 32), dtype=np.uint64)
    ids = np.unique(np.concatenate([ids, full]))
    per = oracle_per_path(("6x7", kind), setup, ids, bits)
    ref = per.sum(axis=0)
    # split = 0: the level before the folded last level runs inside the last
    # program; split = 1: as its own segment with the node in between
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"], split_last=split, cycle_segments=cyc)
    amp, _ = p.amplitudes(bits, sfsim.selection("list", ids=ids))
    check_close(amp, ref, 42, f"6x7 {kind} split={split} cycle_segments={cyc} {len(ids)} paths",
                path_scale=path_scale(per))
    p.close()


# ---------------------------------------------------------------- 7x8 (C4)
def test_7x8_paths_match_stored_oracle(jit):
    """Full size (28+28 qubits, 2 GiB halves) at the benchmark's density:
    the plan runs all 1M bitstrings of the workload (compact final passes,
    as in the benchmark), and the first 1024 are compared with the FP64
    oracle's per-path amplitudes stored by tests/golden/make_oracle_7x8.py:
    24 paths of the first selected prefix (f = 0.5%, seed 7) - one whole
    16-leaf group of the folded last level and 8 paths of other groups."""
    w, text = workload("7x8_d40")
    g = np.load(os.path.join(GOLDEN, "oracle_7x8_d40_paths.npz"))
    ids, amps = g["ids"], g["amps"]
    bits = inputs.random_bitstrings(56, w["n_bitstrings"], w["bitstring_seed"])
    assert np.array_equal(bits[:len(g["bits"])], g["bits"])
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    sel_all = sfsim.selection("list", ids=ids)
    assert sfsim.sf_workspace_size(p.handle, len(bits), sel_all) > \
        sfsim.sf_workspace_size(p.handle, 1024, sel_all), "compact finals not sized for 1M bitstrings"
    assert np.all(ids[:16] >> 4 == ids[0] >> 4) and ids[0] % 16 == 0
    for label, rows in [("whole 16-leaf group", slice(0, 16)), ("8 paths of other groups", slice(16, 24)),
                        ("all 24 paths", slice(0, 24))]:
        amp, _ = p.amplitudes(bits, sfsim.selection("list", ids=ids[rows]))
        per = amps[rows]
        check_close(amp[:per.shape[1]], per.sum(axis=0), 56, f"7x8 {label}", path_scale=path_scale(per))
    p.close()


def test_7x8_path_list_matches_oracle(jit):
    """A seeded path list x 1024 bitstrings against the oracle run here (v2
    circuit: every path is non-zero)."""
    w, text = workload("7x8_d40")
    c = ocirc.parse(text)
    setup = sim.SFSetup(c, w["side_b_mask"])
    bits = inputs.random_bitstrings(56, 1024, w["bitstring_seed"])
    ids = inputs.random_path_list(setup.x_bits, 2, 8)
    per = oracle_per_path(("7x8",), setup, ids, bits)
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    amp, _ = p.amplitudes(bits, sfsim.selection("list", ids=ids))
    check_close(amp, per.sum(axis=0), 56, "7x8 2 random paths", path_scale=path_scale(per))
    p.close()


def test_7x8_prefix_batched_equals_plain(jit):
    """One 128-path prefix of the f = 0.5% selection: the batched executor
    (path tree + last level folded into the gather) equals the plain
    one-path-at-a-time executor."""
    w, text = workload("7x8_d40")
    bits = inputs.random_bitstrings(56, 100000, w["bitstring_seed"])
    p = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"])
    q = sfsim.Plan(text, jit=jit, side_b_mask=w["side_b_mask"], exec_mode=sfsim.SF_EXEC_PLAIN)
    ids = sfsim.sf_selection_ids(p.handle, sfsim.selection("fraction", fidelity=0.005, seed=7), cap=128)
    sel = sfsim.selection("range", first=int(ids[0]), count=128)
    a, _ = p.amplitudes(bits, sel)
    b, _ = q.amplitudes(bits, sel)
    check_close(a, b, 56, "7x8 prefix batched vs plain")
    p.close()
    q.close()


# ----------------------------------------------- frugal sampling (Section 4)
def test_frugal_accept_matches_oracle_bit_exactly():
    """Algorithm 2's accept step on the GPU equals the oracle's decision on the
    same amplitudes (5x6, all paths, 100k candidates), and the acceptance rate
    is ~1/M' for Porter-Thomas probabilities."""
    import torch
    from oracle import sampling
    w, text = workload("5x6_d24")
    bits = inputs.random_bitstrings(30, w["n_bitstrings"], w["bitstring_seed"])
    p = sfsim.Plan(text, side_b_mask=w["side_b_mask"])
    amp, _ = p.amplitudes(bits, sfsim.selection("fraction", fidelity=1.0))
    p.close()
    rng = np.random.default_rng(2)
    u = rng.random(len(bits))
    d_amps = torch.from_numpy(np.stack([amp.real, amp.imag], 1).copy()).cuda()
    d_u = torch.from_numpy(u).cuda()
    d_acc = torch.empty(len(bits), dtype=torch.uint8, device="cuda")
    d_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    sfsim.sf_frugal_accept_device(d_amps, d_u, 30, 10.0, d_acc, d_cnt)
    torch.cuda.synchronize()
    got = d_acc.cpu().numpy().astype(bool)
    pr = (amp.real * amp.real + amp.imag * amp.imag) * 1.0
    want = sampling.accept_frugal(pr, u, 2.0 ** 30, 10.0)
    assert np.array_equal(got, want)
    assert int(d_cnt.item()) == int(want.sum())
    assert abs(want.mean() - 0.1) < 0.01
