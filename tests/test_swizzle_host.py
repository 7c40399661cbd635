"""Host check of the per-pass tile swizzle of the specialised kernels (no
GPU). Each generated pass defines swz(), the shared-memory position of tile
element e. The test reads it back from the generated source and checks, in
its own code:
  * it is a bijection of the tile that keeps 16-byte chunks (element pairs)
    whole, so the copy warps' 16-byte accesses stay valid;
  * every register stage is free of bank conflicts: an 8-byte access is
    served per half warp, so the images of a stage's four lowest thread bits
    in address bits 0..3 (16 bank pairs) must be independent; a 16-byte
    access (tile bit 0 held in registers) per quarter warp, so the images of
    its three lowest thread bits in address bits 1..3 (8 slots of 16 bytes).
"""
import os
import re

import pytest

from paper_1807_10749_gb300 import inputs, sfsim


def _rank(vs):
    vs = list(vs)
    r = 0
    for bit in range(31, -1, -1):
        piv = next((i for i in range(r, len(vs)) if (vs[i] >> bit) & 1), None)
        if piv is None:
            continue
        vs[r], vs[piv] = vs[piv], vs[r]
        for i in range(len(vs)):
            if i != r and (vs[i] >> bit) & 1:
                vs[i] ^= vs[r]
        r += 1
    return r


def _default_swz(e):
    x = e >> 4
    return e ^ (((x ^ (x >> 3) ^ (x >> 6)) & 7) << 1)


def _swizzle_of(src):
    terms = re.findall(r"__popc\(e & (\d+)u\) & 1\) << (\d)\)", src)
    if not terms:
        assert "return sf::swz(e);" in src
        return _default_swz, False
    masks = {int(sh): int(m) for m, sh in terms}
    assert sorted(masks) == [1, 2, 3]
    return (lambda e: e ^ sum((bin(e & masks[s]).count("1") & 1) << s for s in (1, 2, 3))), True


def _stage_thread_positions(src):
    """Tile bit of each thread-index bit, per stage, from the generated
    deposit expression of the stage's base address."""
    out = []
    for m in re.finditer(r"// stage \d+[^\n]*\nconst uint32_t pf = swz\((.*?)\);", src):
        pos = {}
        for t, mask, p in re.findall(r"\(\(\(tid >> (\d+)\) & 0x([0-9a-f]+)u\) << (\d+)\)", m.group(1)):
            for i in range(int(mask, 16).bit_length()):
                pos[int(t) + i] = int(p) + i
        out.append([pos[t] for t in sorted(pos)])
    return out


def _dump(tmp_path, name):
    w = inputs.WORKLOADS[name]
    d = tmp_path / name
    d.mkdir()
    os.environ["SF_JIT_DUMP"] = str(d)
    try:
        sfsim.Plan(inputs.workload_circuit(name).text(), side_b_mask=w["side_b_mask"], jit=1).close()
    except sfsim.SFError as e:
        if e.code == sfsim.SF_EUNSUPPORTED:
            pytest.skip(str(e))
        raise
    finally:
        del os.environ["SF_JIT_DUMP"]
    return [open(d / f).read() for f in sorted(os.listdir(d))]


@pytest.mark.parametrize("name", ["5x6_d24", "7x8_d40"])
def test_pass_swizzles_are_bijective_and_conflict_free(name, tmp_path):
    srcs = _dump(tmp_path, name)
    assert srcs
    n_custom = n_stages = 0
    for src in srcs:
        swz, custom = _swizzle_of(src)
        n_custom += custom
        stages = _stage_thread_positions(src)
        if not stages:
            continue
        # tile bits = register bits (R of pass_body<R, ...>) + thread bits
        R = int(re.search(r"pass_body<(\d+), ", src).group(1))
        k = R + len(stages[0])
        image = sorted(swz(e) for e in range(1 << k))
        assert image == list(range(1 << k)), "not a bijection of the tile"
        assert all(swz(e) & 1 == 0 and swz(e + 1) == swz(e) + 1 for e in range(0, 1 << k, 2)), \
            "splits a 16-byte chunk"
        for pos in stages:
            n_stages += 1
            if len(pos) < 5:
                continue
            if 0 in pos:   # 8-byte accesses, half warps: 16 bank pairs
                v = [swz(1 << p) & 15 for p in pos[:4]]
                assert _rank(v) == 4, (pos, v)
            else:          # 16-byte accesses, quarter warps: 8 slots
                v = [(swz(1 << p) >> 1) & 7 for p in pos[:3]]
                assert _rank(v) == 3, (pos, v)
    assert n_stages > 0
    if name == "7x8_d40":
        assert n_custom > 0   # the default swizzle conflicts on some of these passes
