"""Host check of the part-map kernels of the compact finals (no GPU): the
kernel source of block_mark_kernel, block_count_kernel and block_rank_kernel
is compiled with g++ against stand-ins for the CUDA built-ins it uses. Each
block runs as 256 host threads: __syncthreads is a block barrier, and warp
shuffles exchange values through a per-warp buffer between two warp
barriers. The results are checked against plain Python:
* marks: every bitstring's part number (bits of its layout index at the free
  positions, above those at the tile positions from ctl up), and the second
  part when the block spans two;
* prefix counts: the marked parts before each map word, and the total, for
  ragged word counts (1, 5, 2047, 2048, 2049, 5000) that the GPU workloads
  (power-of-two maps) do not reach."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1807_10749_gb300", "csrc")

SHIM = r'''
#include <barrier>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>
#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
#define __launch_bounds__(x)
#define __grid_constant__
#define __shared__ static
struct Dim3 { unsigned x, y, z; };
thread_local Dim3 threadIdx;
Dim3 blockIdx, blockDim, gridDim;
std::barrier<>* g_block;
std::barrier<>* g_warp[8];
uint32_t g_xchg[8][32];
inline void __syncthreads() { g_block->arrive_and_wait(); }
inline uint32_t __shfl_down_sync(unsigned, uint32_t v, int o) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  g_xchg[w][l] = v;
  g_warp[w]->arrive_and_wait();
  const uint32_t r = l + o < 32 ? g_xchg[w][l + o] : v;
  g_warp[w]->arrive_and_wait();
  return r;
}
inline uint32_t __shfl_up_sync(unsigned, uint32_t v, int o) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  g_xchg[w][l] = v;
  g_warp[w]->arrive_and_wait();
  const uint32_t r = l >= o ? g_xchg[w][l - o] : v;
  g_warp[w]->arrive_and_wait();
  return r;
}
inline int __popc(unsigned v) { return __builtin_popcount(v); }
inline uint32_t atomicOr(uint32_t* p, uint32_t v) { return __atomic_fetch_or(p, v, __ATOMIC_RELAXED); }
'''


def _between(src, start, end_marker):
    a = src.index(start)
    return src[a:src.index(end_marker, a)]


def _extract():
    h = open(os.path.join(CSRC, "sf_internal.h")).read()
    k = open(os.path.join(CSRC, "kernels.cu")).read()
    structs = _between(h, "struct CompactMap {", "struct GatherSide {") + \
        _between(h, "struct BlockMapLaunch {", "int launch_block_maps(")
    part = _between(k, "__device__ __forceinline__ uint32_t compact_part(", "__device__ __forceinline__ uint32_t compact_slot(")
    kernels = _between(k, "__global__ void __launch_bounds__(256) block_mark_kernel(", "__global__ void zero_kernel(")
    return structs + part + kernels


DRIVER = r'''
}  // namespace sf
using namespace sf;

template <class K>
static void launch(K kernel, unsigned gx, unsigned gy, const BlockMapLaunch& P) {
  gridDim = {gx, gy, 1};
  blockDim = {256, 1, 1};
  for (unsigned by = 0; by < gy; by++)
    for (unsigned bx = 0; bx < gx; bx++) {
      blockIdx = {bx, by, 0};
      std::barrier<> blk(256);
      for (int w = 0; w < 8; w++) g_warp[w] = new std::barrier<>(32);
      g_block = &blk;
      std::vector<std::thread> th;
      for (unsigned t = 0; t < 256; t++)
        th.emplace_back([&, t] { threadIdx = {t, 0, 0}; kernel(P); });
      for (auto& x : th) x.join();
      for (int w = 0; w < 8; w++) delete g_warp[w];
    }
}

// stdin, mode 0 (marks): n bits[n] then per side: on tab[2048] cfree cpart ckt ctl csub1 nw
//        mode 1 (ranks): per side: on nw words[nw]
int main() {
  int mode;
  if (scanf("%d", &mode) != 1) return 2;
  static BlockMapLaunch P;
  std::memset(&P, 0, sizeof(P));
  std::vector<uint64_t> bits;
  std::vector<uint32_t> tab[2], map[2], sums[2];
  uint32_t count[2] = {0, 0};
  if (mode == 0) {
    long n;
    scanf("%ld", &n);
    bits.resize(n);
    for (long i = 0; i < n; i++) scanf("%lu", &bits[i]);
    P.bits = bits.data();
    P.n = n;
  }
  for (int s = 0; s < 2; s++) {
    int on;
    scanf("%d", &on);
    if (mode == 0) {
      tab[s].resize(2048);
      for (int i = 0; i < 2048; i++) scanf("%u", &tab[s][i]);
      scanf("%u %u %d %d %u", &P.c[s].cfree, &P.c[s].cpart, &P.c[s].ckt, &P.c[s].ctl, &P.c[s].csub1);
      P.tab[s] = tab[s].data();
    }
    long nw;
    scanf("%ld", &nw);
    map[s].assign(2 * nw, 0u);
    if (mode == 1)
      for (long w = 0; w < nw; w++) scanf("%u", &map[s][2 * w]);
    sums[s].assign((nw + kRankChunk - 1) / kRankChunk + 1, 0u);
    if (on) {
      P.map[s] = map[s].data();
      P.nw[s] = nw;
      P.sums[s] = sums[s].data();
      P.count[s] = &count[s];
    }
  }
  if (mode == 0) {
    launch(block_mark_kernel, 3, 1, P);
  } else {
    const long maxw = P.nw[0] > P.nw[1] ? P.nw[0] : P.nw[1];
    const unsigned gx = (unsigned)((maxw + kRankChunk - 1) / kRankChunk);
    launch(block_count_kernel, gx, 2, P);
    launch(block_rank_kernel, gx, 2, P);
  }
  for (int s = 0; s < 2; s++) {
    printf("side %d %u\n", s, count[s]);
    for (size_t w = 0; w < map[s].size() / 2; w++) printf("%u %u\n", map[s][2 * w], map[s][2 * w + 1]);
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("maps")
    cpp = d / "m.cpp"
    cpp.write_text(SHIM + '#include "dev_types.h"\nnamespace sf {\n' + _extract() + DRIVER)
    exe = d / "m.bin"
    r = subprocess.run(["g++", "-std=c++20", "-O1", "-Wno-unknown-pragmas", "-I", CSRC, str(cpp), "-o", str(exe),
                        "-pthread"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[:3000]
    return str(exe)


def _run(exe, tokens):
    out = subprocess.run([exe], input=" ".join(map(str, tokens)), capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    sides, cur = [], None
    for ln in out.stdout.split("\n"):
        if not ln.strip():
            continue
        f = ln.split()
        if f[0] == "side":
            cur = {"count": int(f[2]), "words": []}
            sides.append(cur)
        else:
            cur["words"].append((int(f[0]), int(f[1])))
    return sides


def _pext(x, positions):
    return sum(((x >> p) & 1) << i for i, p in enumerate(positions))


def _mask(positions):
    return sum(1 << p for p in positions)


def _geometry(m, g, active):
    """A final pass's geometry as the planner passes it to the kernels."""
    tl = sum(1 for p in active if p < g)
    free = [p for p in range(m) if p not in active]
    part = [p for p in active if p >= tl]
    kt = len(active) - tl
    csub1 = (_pext(1 << tl, free) << kt) if g > tl else 0
    return dict(tl=tl, free=free, part=part, kt=kt, csub1=csub1, nw=((1 << (m - tl)) + 31) // 32)


@pytest.mark.parametrize("seed", [1, 2])
def test_mark_kernel_marks_the_parts_of_every_bitstring(harness, seed):
    rng = random.Random(seed)
    nq, g = 30, 4
    qubits = list(range(nq))
    rng.shuffle(qubits)
    sides = [sorted(qubits[:15]), sorted(qubits[15:])]
    geo = [_geometry(15, g, [0, 1, 2, 5, 7, 9, 10, 12]),          # block spans two parts
           _geometry(15, g, [0, 1, 2, 3, 6, 8, 11, 13, 14])]      # one part
    tokens = [0]
    bits = [rng.getrandbits(nq) for _ in range(1500)]
    bits += bits[:20]  # duplicates
    tokens += [len(bits)] + bits
    want = []
    for s in range(2):
        # layout: the half's first g qubits take positions 0..g-1 (excluded
        # from the tables, as the folded level's qubits are), the rest take
        # positions g.. in a shuffled order
        qs = sides[s]
        pos = list(range(g, 15))
        rng.shuffle(pos)
        where = {q: p for q, p in zip(qs[g:], pos)}
        tab = []
        for b in range(8):
            for byte in range(256):
                v = 0
                for i in range(8):
                    q = 8 * b + i
                    if (byte >> i) & 1 and q in where:
                        v |= 1 << where[q]
                tab.append(v)
        G = geo[s]
        tokens += [1] + tab + [_mask(G["free"]), _mask(G["part"]), G["kt"], G["tl"], G["csub1"], G["nw"]]
        marks = set()
        for x in bits:
            ix = sum(1 << where[q] for q in where if (x >> q) & 1)
            p0 = (_pext(ix, G["free"]) << G["kt"]) | _pext(ix, G["part"])
            marks.add(p0)
            if G["csub1"]:
                marks.add(p0 | G["csub1"])
        want.append(marks)
    got = _run(harness, tokens)
    assert want[0] and want[1]
    assert geo[0]["csub1"] and not geo[1]["csub1"]
    for s in range(2):
        marked = {32 * w + j for w, (word, _) in enumerate(got[s]["words"]) for j in range(32) if (word >> j) & 1}
        assert marked == want[s]


@pytest.mark.parametrize("nw0,nw1", [(1, 5), (2047, 2048), (2049, 0), (5000, 4097), (0, 1)])
def test_rank_kernels_count_marked_parts_before_each_word(harness, nw0, nw1):
    rng = random.Random(nw0 * 7 + nw1)
    tokens = [1]
    words = []
    for nw in (nw0, nw1):
        ws = [rng.getrandbits(32) & rng.getrandbits(32) for _ in range(nw)]
        if nw > 3:
            ws[1] = 0
            ws[2] = 0xFFFFFFFF
        words.append(ws)
        tokens += [1 if nw else 0, nw] + ws
    got = _run(harness, tokens)
    for s, ws in enumerate(words):
        if not ws:
            assert got[s]["count"] == 0
            continue
        run = 0
        for w, (word, rank) in enumerate(got[s]["words"]):
            assert word == ws[w]
            assert rank == run, (s, w)
            run += bin(word).count("1")
        assert got[s]["count"] == run
