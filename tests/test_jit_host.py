"""Host check of the generated stage programs (no GPU): the scalar and the
packed FP32x2 forms of each specialised pass are compiled with g++ against
small stand-ins for the CUDA types and intrinsics they use, every stage
thread runs as a host thread (the stage barrier as a std::barrier) over the
same random tile, and the two forms must give the same tile. This covers the
packed code generation on every kind of stage the benchmark plans hold."""
import os
import re
import shutil
import subprocess

import pytest

from paper_1807_10749_gb300 import inputs, sfsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1807_10749_gb300", "csrc")

SHIM = r'''
#include <barrier>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>
struct float2 { float x, y; };
struct float4 { float x, y, z, w; };
inline float2 make_float2(float a, float b) { return {a, b}; }
inline float4 make_float4(float a, float b, float c, float d) { return {a, b, c, d}; }
#define __device__
#define __host__
#define __forceinline__ inline
inline int __popc(unsigned v) { return __builtin_popcount(v); }
inline float2 __fadd2_rn(float2 a, float2 b) { return {a.x + b.x, a.y + b.y}; }
inline float2 __fmul2_rn(float2 a, float2 b) { return {a.x * b.x, a.y * b.y}; }
inline float2 __ffma2_rn(float2 a, float2 b, float2 c) { return {std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)}; }
struct Dim3 { unsigned x; };
thread_local Dim3 threadIdx;
std::barrier<>* g_bar;
inline void compute_bar(int) { g_bar->arrive_and_wait(); }
'''


def _extract(path):
    """The stage program (the run function) of a dumped pass source as a
    struct of its own, and the number of stage threads."""
    src = open(path).read()
    name = re.search(r"struct (sf_pass_\w+)_prog \{", src).group(1)
    a = src.index(f"struct {name}_prog {{")
    b = src.index("static __device__ __forceinline__ void load_tile", a)
    m = re.search(r"__launch_bounds__\((\d+), \d+\)", src)
    return src[a:b].replace(f"{name}_prog", "sf_pass_spec_stages") + "};", int(m.group(1)) - 64


def _gate_code():
    """Gate bodies and helpers of the shared device header (up to pin_val)."""
    src = open(os.path.join(CSRC, "pass_common.cuh")).read()
    a = src.index("namespace sf {") + len("namespace sf {")
    b = src.index("__device__ __forceinline__ uint32_t pin_val(")
    c = src.index("struct ItemGeo {")
    d = src.index("};", c) + 2
    return src[a:b] + "\n" + src[c:d]


def _harness(scalar, packed, nthreads, ntile):
    return SHIM + '#include "dev_types.h"\nnamespace sf {\n' + _gate_code() + "\n" + \
        scalar.replace("sf_pass_spec_stages", "StagesScalar") + "\n" + \
        packed.replace("sf_pass_spec_stages", "StagesPacked") + r'''
}  // namespace sf
using namespace sf;
template <class S>
static void run_all(std::vector<float2>& tile, const PassLaunch& P, const ItemGeo& g, const float2* w8) {
  std::barrier<> bar(NTHREADS);
  g_bar = &bar;
  std::vector<std::thread> th;
  for (unsigned t = 0; t < NTHREADS; t++)
    th.emplace_back([&, t] { threadIdx.x = t; S::run(P, tile.data(), g, w8, NTHREADS, true); });
  for (auto& x : th) x.join();
}
int main() {
  static PassLaunch P;
  std::memset(&P, 0, sizeof(P));
  float2 w8[8];
  for (int t = 0; t < 8; t++) w8[t] = {(float)std::cos(M_PI / 4 * t), (float)std::sin(M_PI / 4 * t)};
  ItemGeo g{};
  g.base = 0x5a5a5a5au & ~((1u << 28) - 1u);
  srand(7);
  std::vector<float2> a(NTILE), b;
  for (auto& v : a) v = {(float)rand() / RAND_MAX - 0.5f, (float)rand() / RAND_MAX - 0.5f};
  b = a;
  run_all<StagesScalar>(a, P, g, w8);
  run_all<StagesPacked>(b, P, g, w8);
  double md = 0, mx = 0;
  for (size_t i = 0; i < a.size(); i++) {
    md = std::fmax(md, std::fabs(a[i].x - b[i].x) + std::fabs(a[i].y - b[i].y));
    mx = std::fmax(mx, std::fabs(a[i].x) + std::fabs(a[i].y));
  }
  std::printf("%.3e %.3e\n", md, mx);
  return 0;
}
'''.replace("NTHREADS", str(nthreads)).replace("NTILE", str(ntile))


def _compile_run(tmp_path, tag, scalar, packed, nt):
    cpp = tmp_path / f"{tag}.cpp"
    cpp.write_text(_harness(scalar, packed, nt, 1 << 13))
    exe = tmp_path / f"{tag}.bin"
    r = subprocess.run(["g++", "-std=c++20", "-O1", "-ffp-contract=off", "-I", CSRC, str(cpp), "-o", str(exe),
                        "-pthread"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[:3000]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    md, mx = map(float, out.stdout.split())
    return md, mx


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")
@pytest.mark.parametrize("name,stride", [("4x4_d10", 1), ("5x6_d24", 1), ("6x7_d26", 3), ("7x8_d40", 4)])
def test_packed_and_scalar_stage_programs_agree(name, stride, tmp_path):
    """Every stride-th pass of the plan (all three forms of a stage: packed
    butterflies, odd phases, per-thread signs and phases, post scales)."""
    w = inputs.WORKLOADS[name]
    text = inputs.workload_circuit(name).text()
    dirs = {}
    for packed in (0, 1):
        d = tmp_path / f"p{packed}"
        d.mkdir()
        os.environ["SF_JIT_DUMP"] = str(d)
        try:
            plan = sfsim.Plan(text, side_b_mask=w["side_b_mask"], jit=1, fp32x2=packed)
        except sfsim.SFError as e:
            if e.code == sfsim.SF_EUNSUPPORTED:
                pytest.skip(str(e))
            raise
        finally:
            del os.environ["SF_JIT_DUMP"]
        plan.close()
        dirs[packed] = d
    files = sorted(os.listdir(dirs[1]), key=lambda f: int(f.split("_")[1].split(".")[0]))
    assert files
    n_packed = 0
    for f in files[::stride][:12]:
        scalar, nt = _extract(os.path.join(dirs[0], f))
        packed, nt2 = _extract(os.path.join(dirs[1], f))
        assert nt == nt2
        n_packed += packed.count("(packed)")
        md, mx = _compile_run(tmp_path, f, scalar, packed, nt)
        assert mx > 0
        assert md <= 1e-5 * mx, (f, md, mx)
    assert n_packed > 0   # the check exercised packed stages


@pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")
def test_harness_catches_a_planted_mistake(tmp_path):
    """A sign flipped in one packed butterfly of a 5x6 pass must show up."""
    w = inputs.WORKLOADS["5x6_d24"]
    text = inputs.workload_circuit("5x6_d24").text()
    srcs = []
    for packed in (0, 1):
        d = tmp_path / f"p{packed}"
        d.mkdir()
        os.environ["SF_JIT_DUMP"] = str(d)
        try:
            sfsim.Plan(text, side_b_mask=w["side_b_mask"], jit=1, fp32x2=packed).close()
        finally:
            del os.environ["SF_JIT_DUMP"]
        srcs.append(_extract(os.path.join(d, "pass_2.cu")))
    (scalar, nt), (packed, _) = srcs
    assert "__fadd2_rn(a, b)" in packed
    md, mx = _compile_run(tmp_path, "planted", scalar, packed.replace("__fadd2_rn(a, b)", "__fadd2_rn(b, b)", 1), nt)
    assert md > 1e-3 * mx
