"""Host check of the compact final store (no GPU): the device functions that
write only the requested parts of a tile are compiled with g++ against small
stand-ins for the CUDA types they use and run over every tile of a small
half, one lane after another. The part map (parts numbered tile-major: the
tile's free positions, then its active positions from ctl up; per 32 parts a
bitmap word and the count of marked parts before it) is built here, in
Python, from random requested indices. Every amplitude of a requested block
must then be found where the gather looks for it, slot(part) * 2^ctl + its
offset in the part; nothing else may be written, and no write may leave the
buffer. The gather's own index functions, compiled in too, must read every
requested amplitude's value back."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1807_10749_gb300", "csrc")

SHIM = r'''
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
struct float2 { float x, y; };
struct float4 { float x, y, z, w; };
struct uint2 { uint32_t x, y; };
inline uint2 make_uint2(uint32_t a, uint32_t b) { return {a, b}; }
#define __device__
#define __host__
#define __forceinline__ inline
inline int __popc(unsigned v) { return __builtin_popcount(v); }
inline int __ffs(unsigned v) { return __builtin_ffs((int)v); }
'''


def _gather_index_code():
    """The gather's compact-final index functions and their record."""
    h = open(os.path.join(CSRC, "sf_internal.h")).read()
    k = open(os.path.join(CSRC, "kernels.cu")).read()
    a = h.index("struct CompactMap {")
    b = h.index("struct GatherSide {")
    c = k.index("__device__ __forceinline__ uint32_t compact_part(")
    d = k.index("template <int G, bool ALL>", c)
    return h[a:b] + k[c:d]


def _extract():
    src = open(os.path.join(CSRC, "pass_common.cuh")).read()
    a = src.index("struct ItemGeo {")
    b = src.index("};", a) + 2
    c = src.index("struct CopyCtx {")
    d = src.index("};", c) + 2
    e = src.index("struct CompactWord {")
    f = src.index("\n}\n", src.index("__device__ __forceinline__ void compact_store_tile(")) + 3
    return src[a:b] + "\n" + src[c:d] + "\n" + src[e:f] + "\n" + _gather_index_code()


DRIVER = r'''
}  // namespace sf
using namespace sf;
// a swizzle other than the default one (a pass may choose its own): the
// compact store must read the tile through the one it is given
struct Swz {
  static uint32_t swz(uint32_t e) {
    return e ^ ((uint32_t)(__builtin_popcount(e & 0x2b0u) & 1) << 1) ^
           ((uint32_t)(__builtin_popcount(e & 0x150u) & 1) << 2) ^ ((uint32_t)(__builtin_popcount(e & 0x1c60u) & 1) << 3);
  }
};
// stdin: m k L g  gpos[k]  n_free freepos[n_free]  nw  (word rank)[nw]  cap
int main() {
  int m, k, L, g;
  if (scanf("%d %d %d %d", &m, &k, &L, &g) != 4) return 2;
  static PassLaunch P;
  std::memset(&P, 0, sizeof(P));
  P.pass.m = m; P.pass.k = k; P.pass.L = L;
  for (int j = 0; j < k; j++) { int v; scanf("%d", &v); P.pass.gpos[j] = (int8_t)v; }
  int nf; scanf("%d", &nf);
  P.pass.n_free = nf;
  for (int j = 0; j < nf; j++) { int v; scanf("%d", &v); P.pass.freepos[j] = (int8_t)v; }
  long nw; scanf("%ld", &nw);
  std::vector<uint32_t> map(2 * nw);
  for (long w = 0; w < nw; w++) scanf("%u %u", &map[2 * w], &map[2 * w + 1]);
  long cap; scanf("%ld", &cap);
  int tl = 0;
  while (tl < k && P.pass.gpos[tl] < g) tl++;
  P.cmap = map.data();
  P.ctl = tl;
  const long guard = 64;
  std::vector<float2> out((cap << tl) + 2 * guard, float2{-7.f, -7.f});
  P.n_nodes = 1;
  P.nodes[0].out = out.data() + guard;
  const int ntile = 1 << k, nruns = 1 << (k - L);
  std::vector<uint32_t> runoff(nruns);
  for (int r = 0; r < nruns; r++) {
    uint32_t hi = 0;
    for (int j = L; j < k; j++) hi |= (uint32_t)((r >> (j - L)) & 1) << P.pass.gpos[j];
    runoff[r] = hi;
  }
  CopyCtx cc{runoff.data(), L, ntile >> 1, (uint32_t)((1 << L) - 1)};
  std::vector<float2> buf(ntile);
  for (uint32_t t = 0; t < (1u << nf); t++) {
    ItemGeo geo;
    std::memset(&geo, 0, sizeof(geo));
    uint32_t base = 0;
    for (int i = 0; i < nf; i++) base |= ((t >> i) & 1u) << P.pass.freepos[i];
    geo.base = base;
    geo.tile = t;
    // tile element e holds the value of its global index, at Swz::swz(e)
    for (int e = 0; e < ntile; e++) {
      const uint32_t gi = base | runoff[e >> L] | ((uint32_t)e & cc.lmask);
      buf[Swz::swz((uint32_t)e)] = float2{(float)gi, 1.f};
    }
    // the store warp's order: the first round's words, then the writes
    for (int lane = 0; lane < 32; lane++) {
      const CompactWord cw = compact_word(P, geo, lane, 0);
      compact_store_tile<Swz>(P, geo, buf.data(), lane, cw);
    }
  }
  for (long i = 0; i < (long)out.size(); i++) printf("%.1f %.1f\n", out[i].x, out[i].y);
  // the gather's reads: every amplitude of each requested block, through its
  // index functions (stdin: cfree cpart csub1 nreq req[nreq])
  CompactMap cm;
  std::memset(&cm, 0, sizeof(cm));
  cm.cmap = map.data();
  cm.ckt = k - tl;
  cm.ctl = tl;
  long nreq;
  if (scanf("%u %u %u %ld", &cm.cfree, &cm.cpart, &cm.csub1, &nreq) != 4) return 3;
  const float2* fin = out.data() + guard;
  for (long r = 0; r < nreq; r++) {
    uint32_t gi;
    scanf("%u", &gi);
    const uint32_t base = gi & ~((1u << g) - 1u);
    const uint32_t p0 = compact_part(cm, base);
    const uint32_t h0 = compact_slot(cm.cmap, p0) << cm.ctl;
    const uint32_t h1 = cm.csub1 ? compact_slot(cm.cmap, p0 | cm.csub1) << cm.ctl : 0u;
    for (uint32_t o = 0; o < (1u << g); o++) {
      const float2 v = fin[compact_index(cm, h0, h1, base | o)];
      printf("G %u %.1f\n", base | o, v.x);
    }
  }
  return 0;
}
'''


def _pext(x, positions):
    return sum(((x >> p) & 1) << i for i, p in enumerate(positions))


def _parts(gi, g, tl, gpos, free):
    """Part numbers of the block holding half index gi: one per value of the
    block positions tl..g-1 (all free)."""
    kt = len(gpos) - tl
    base = gi & ~((1 << g) - 1)
    out = []
    for s in range(1 << (g - tl)):
        idx = base | (s << tl)
        out.append((_pext(idx, free) << kt) | _pext(idx, gpos[tl:]))
    return out


def _map(nparts_total, marked):
    nw = (nparts_total + 31) // 32
    words = [0] * nw
    for p in marked:
        words[p >> 5] |= 1 << (p & 31)
    ranks, run = [], 0
    for w in words:
        ranks.append(run)
        run += bin(w).count("1")
    return words, ranks, run


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("compact")
    cpp = d / "h.cpp"
    cpp.write_text(SHIM + '#include "dev_types.h"\nnamespace sf {\n' + _extract() + DRIVER)
    exe = d / "h.bin"
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, str(cpp), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[:3000]
    return str(exe)


@pytest.mark.parametrize("m,k,L,g,extra,n,seed", [
    (12, 8, 3, 4, [3, 5, 7, 9, 10], 40, 1),     # block bits 0..3 all in the tile (one part)
    (12, 8, 3, 4, [4, 6, 8, 9, 11], 40, 2),     # position 3 outside the tile (two parts)
    (14, 8, 4, 2, [5, 6, 9, 12], 300, 3),       # blocks smaller than a run
    (13, 7, 3, 3, [4, 8, 11, 12], 1, 4),        # one requested bitstring
    (8, 6, 3, 4, [5, 6, 7], 16, 5),             # 8 parts a tile: tiles share map words
    (18, 14, 3, 3, [4, 5, 6, 8, 9, 10, 11, 12, 13, 15, 17], 900, 6),  # 2048 parts: two rounds
])
def test_compact_store_writes_exactly_the_requested_parts(harness, m, k, L, g, extra, n, seed):
    gpos = list(range(L)) + sorted(p for p in extra if p >= L)
    gpos = gpos[:k]
    assert len(gpos) == k and gpos == sorted(set(gpos)) and max(gpos) < m
    free = [p for p in range(m) if p not in gpos]
    tl = sum(1 for p in gpos if p < g)
    assert gpos[:tl] == list(range(tl)) and g - tl <= 1
    rng = random.Random(seed)
    requested = [rng.randrange(1 << m) for _ in range(n)]
    marked = sorted({p for gi in requested for p in _parts(gi, g, tl, gpos, free)})
    words, ranks, total = _map(1 << (m - tl), marked)
    cap = min(n << (g - tl), 1 << (m - tl))
    assert total <= cap
    inp = [m, k, L, g, *gpos, len(free), *free, len(words)]
    inp += [v for w, r in zip(words, ranks) for v in (w, r)]
    inp.append(cap)
    kt = k - tl
    csub1 = (_pext(1 << tl, free) << kt) if g > tl else 0
    inp += [sum(1 << p for p in free), sum(1 << p for p in gpos[tl:]), csub1, len(requested), *requested]
    out = subprocess.run([harness], input=" ".join(map(str, inp)), capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.split("\n") if ln.strip()]
    greads = [ln.split()[1:] for ln in lines if ln.startswith("G ")]
    assert len(greads) == len(requested) << g
    for idx, v in greads:
        assert float(idx) == float(v), (idx, v)   # the gather finds each amplitude's own value
    vals = [tuple(map(float, ln.split())) for ln in lines if not ln.startswith("G ")]
    guard = 64
    assert len(vals) == (cap << tl) + 2 * guard
    assert all(v == (-7.0, -7.0) for v in vals[:guard] + vals[-guard:]), "write outside the buffer"
    body = vals[guard:-guard]
    slot = {p: i for i, p in enumerate(marked)}
    for gi in requested:
        base = gi & ~((1 << g) - 1)
        parts = _parts(gi, g, tl, gpos, free)
        for o in range(1 << g):
            p = parts[(o >> tl) if g > tl else 0]
            assert body[(slot[p] << tl) + (o & ((1 << tl) - 1))] == (float(base | o), 1.0), (gi, o)
    assert all(v == (-7.0, -7.0) for v in body[total << tl:]), "write beyond the marked parts"
