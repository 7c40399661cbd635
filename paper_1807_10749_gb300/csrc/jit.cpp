// Run-time specialised pass kernels.
//
// The generic pass kernel reads every stage, op and phase group of a pass
// from its launch record and dispatches on them per thread. A plan is fixed
// once it is made, so each of its passes can instead be compiled into a
// kernel of its own: the same warp-specialised pipeline (pass_common.cuh),
// with the stage program emitted as straight-line code. Register bits,
// shared-memory offsets, gate kinds and matrices, and the plan-static part of
// every phase group (the one-qubit phase weights and the CZs between register
// bits: the quadratic form k(idx) of Section 2, mod 8) become constants, so a
// phase costs nothing on most amplitudes. The per-thread part of a phase group
// (terms in the thread's fixed index bits, the e^{i pi k0/4} of
// DevPhaseGroup) is a scalar on the thread's whole register block; it is
// summed over the stage and applied once before the stage stores.
//
// Compilation uses NVRTC, opened with dlopen so that the library loads where
// it is absent (a plan that asks for these kernels then fails with
// SF_EUNSUPPORTED). Binaries are cached per process by source text, and loaded
// with the runtime's library API on first launch.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <thread>

#include "sf_internal.h"

namespace sf {

extern const char* const kJitDevTypes;    // text of dev_types.h
extern const char* const kJitPassCommon;  // text of pass_common.cuh

namespace {

// ------------------------------------------------------------------ NVRTC
typedef int nvrtcResult;
typedef struct _nvrtcProgram* nvrtcProgram;

struct Nvrtc {
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*log_size)(nvrtcProgram, size_t*);
  nvrtcResult (*log)(nvrtcProgram, char*);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
  nvrtcResult (*cubin)(nvrtcProgram, char*);
  nvrtcResult (*destroy)(nvrtcProgram*);
  bool ok = false;
  std::string why;
};

const Nvrtc& nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* env = std::getenv("SF_NVRTC");
    const char* names[] = {env, "libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/targets/sbsa-linux/lib/libnvrtc.so.13",
                           "/usr/local/cuda/targets/x86_64-linux/lib/libnvrtc.so.13"};
    void* h = nullptr;
    for (const char* nm : names)
      if (nm && (h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) {
      n.why = "NVRTC (libnvrtc.so.13) not found";
      return;
    }
    auto sym = [&](const char* s) { return dlsym(h, s); };
    n.create = (decltype(n.create))sym("nvrtcCreateProgram");
    n.compile = (decltype(n.compile))sym("nvrtcCompileProgram");
    n.log_size = (decltype(n.log_size))sym("nvrtcGetProgramLogSize");
    n.log = (decltype(n.log))sym("nvrtcGetProgramLog");
    n.cubin_size = (decltype(n.cubin_size))sym("nvrtcGetCUBINSize");
    n.cubin = (decltype(n.cubin))sym("nvrtcGetCUBIN");
    n.destroy = (decltype(n.destroy))sym("nvrtcDestroyProgram");
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    if (!n.ok) n.why = "NVRTC entry points missing";
  });
  return n;
}

// ------------------------------------------------------- code generation
std::string flit(float f) {
  if (!std::isfinite(f)) fail(SF_EINVAL, "internal: non-finite gate entry");
  char b[48];
  std::snprintf(b, sizeof b, "%.9ef", (double)f);
  return b;
}

std::string f2lit(const std::vector<float>& m, int i) {  // float2 at float index 2i
  return "make_float2(" + flit(m[2 * i]) + ", " + flit(m[2 * i + 1]) + ")";
}

// ---- per-pass tile swizzle -------------------------------------------------
// A tile element e lives in shared memory at e ^ (f(e) << 1), where f is a
// linear map from index bits 4 and up into three bits: bit q of f(e) is the
// parity of e & m[q]. Such a swizzle is a bijection of the tile that keeps
// 16-byte chunks (element pairs) whole, so the copy warps are unaffected;
// the default (m = bits 4,7,10 / 5,8,11 / 6,9,12) is dev_types.h's swz().
// A stage thread's accesses are one base address plus a constant per
// register slot, the lanes varying in the stage's five lowest thread bits.
// An 8-byte access of a warp is served per half warp (lanes 0-15: the
// lowest four thread bits) and is conflict-free when those lanes fall into
// 16 distinct bank pairs: the four bits' images in address bits 0..3 are
// independent. A 16-byte access (tile bit 0 in registers) is served per
// quarter warp: three bits' images in address bits 1..3. Each pass takes
// the swizzle that makes every one of its stages conflict-free, searched
// from the default in a fixed pseudo-random order (the default is kept when
// it already is).
struct TileSwz {
  uint32_t m[3];
  uint32_t operator()(uint32_t e) const {
    uint32_t r = e;
    for (int q = 0; q < 3; q++) r ^= (uint32_t)(__builtin_popcount(e & m[q]) & 1) << (1 + q);
    return r;
  }
  bool is_default() const {
    return m[0] == 0x490u && m[1] == 0x920u && m[2] == 0x1240u;
  }
};

TileSwz default_swz() { return TileSwz{{0x490u, 0x920u, 0x1240u}}; }

int gf2_rank(uint32_t* v, int n) {
  int r = 0;
  for (int bit = 31; bit >= 0 && r < n; bit--) {
    int piv = -1;
    for (int i = r; i < n; i++)
      if ((v[i] >> bit) & 1) piv = i;
    if (piv < 0) continue;
    std::swap(v[r], v[piv]);
    for (int i = 0; i < n; i++)
      if (i != r && ((v[i] >> bit) & 1)) v[i] ^= v[r];
    r++;
  }
  return r;
}

// Excess shared-memory wavefronts of the pass's stage accesses (0: none).
int swz_excess(const PassPlan& pp, const TileSwz& S) {
  const DevPass& d = pp.dev;
  const int k = d.k, R = d.R;
  int excess = 0;
  for (int s = 0; s < d.n_stages; s++) {
    const DevStage& st = pp.stages[s];
    bool wide = false;  // tile bit 0 in registers: 16-byte accesses
    for (int j = 0; j < R; j++)
      if (st.rbit[j] == 0) wide = true;
    const int nb = wide ? 3 : 4;
    if (k - R < nb) continue;
    uint32_t v[4];
    for (int t = 0; t < nb; t++) {
      const uint32_t a = S(1u << st.tpos[t]);
      v[t] = wide ? (a >> 1) & 7u : a & 15u;
    }
    excess += (1 << (nb - gf2_rank(v, nb))) - 1;
  }
  return excess;
}

TileSwz choose_swz(const PassPlan& pp) {
  TileSwz best = default_swz();
  const int k = pp.dev.k;
  if (k < 8) return best;  // tiles of the generic copy loops keep the default
  int be = swz_excess(pp, best);
  uint64_t x = 0x9e3779b97f4a7c15ull;
  for (int it = 0; it < 4096 && be > 0; it++) {
    TileSwz c{{0u, 0u, 0u}};
    for (int b = 4; b < k; b++) {
      x ^= x << 13;
      x ^= x >> 7;
      x ^= x << 17;
      const uint32_t f = (uint32_t)(x >> 61);  // three bits
      for (int q = 0; q < 3; q++)
        if ((f >> q) & 1) c.m[q] |= 1u << b;
    }
    const int e = swz_excess(pp, c);
    if (e < be) {
      be = e;
      best = c;
    }
  }
  return best;
}

// thread-index bits t -> bit positions pos[t], grouped into shifted fields
std::string deposit(const int8_t* pos, int nbits) {
  std::string e;
  int t = 0;
  while (t < nbits) {
    int len = 1;
    while (t + len < nbits && pos[t + len] == pos[t] + len) len++;
    char b[96];
    std::snprintf(b, sizeof b, "(((tid >> %d) & 0x%xu) << %d)", t, (1u << len) - 1, pos[t]);
    if (!e.empty()) e += " | ";
    e += b;
    t += len;
  }
  return e.empty() ? "0u" : e;
}

// The geometry of a work item (item_geo in pass_common.cuh) with the pass's
// free positions, active set and pin positions as constants: the tile number
// deposited into the free positions, the pin values read from the path's
// digits, and the pins' masks on tile-local bits.
void gen_geo(std::ostringstream& o, const PassPlan& pp) {
  const DevPass& d = pp.dev;
  uint32_t active = 0;
  for (int j = 0; j < d.k; j++) active |= 1u << d.gpos[j];
  o << "static __device__ __forceinline__ ItemGeo geo(const PassLaunch& P, int64_t item, int) {\n"
    << "ItemGeo g;\n"
    << "const uint32_t nn = (uint32_t)P.n_nodes, it32 = (uint32_t)item;\n"
    << "const uint32_t tid = it32 / nn;\n"
    << "g.node = (int)(it32 - tid * nn);\ng.tile = tid;\ng.path = P.nodes[g.node].path;\n"
    << "uint32_t pv = 0, lv = 0, ov = 0;\n(void)pv; (void)lv; (void)ov;\n";
  uint32_t lm = 0, om = 0;
  auto pin = [&](const DevPin& q, bool out) {
    std::string val;
    if (q.xi < 0) {
      val = std::to_string((unsigned)q.v[0]) + "u";
    } else {
      char b[160];
      std::snprintf(b, sizeof b, "((0x%xu >> (8 * digit_of(P.xshift, P.xbits, g.path, %d))) & 1u)",
                    (uint32_t)q.v[0] | (uint32_t)q.v[1] << 8 | (uint32_t)q.v[2] << 16 | (uint32_t)q.v[3] << 24, q.xi);
      val = b;
    }
    int j = -1;
    for (int t = 0; t < d.k; t++)
      if (d.gpos[t] == q.pos) j = t;
    o << "{ const uint32_t v = " << val << ";";
    if (!out) o << " pv |= v << " << (int)q.pos << ";";
    if (j >= 0) {
      o << (out ? " ov" : " lv") << " |= v << " << j << ";";
      (out ? om : lm) |= 1u << j;
    }
    o << " }\n";
  };
  for (int i = 0; i < d.n_pin_in; i++) pin(d.pin_in[i], false);
  for (int i = 0; i < d.n_pin_out; i++) pin(d.pin_out[i], true);
  o << "g.base = (" << deposit(d.freepos, d.n_free) << ") | (pv & " << (~active) << "u);\n"
    << "g.lin_m = " << lm << "u; g.lin_v = lv; g.lout_m = " << om << "u; g.lout_v = ov;\n"
    << "return g;\n}\n";
}

// The tile copies of one pass with its geometry as constants. Lane l moves
// chunks c = l + 32 j (elements 2c, 2c+1). The global offset of a chunk is
// the deposit of its tile bits into the pass's index positions, a lane part
// plus a constant per j. Its shared-memory slot swz(2c) is
// (swz(2l) ^ lo_j) | 64 j, with lo_j the swizzle's bits 1..3 for the j part:
// one base per distinct lo_j plus a constant. Runs with a pinned bit other
// than the tile's value are skipped (structural zeros).
void gen_copy(std::ostringstream& o, const PassPlan& pp, const TileSwz& S) {
  const DevPass& d = pp.dev;
  if (d.k < 6) {  // fewer chunks than lanes: the generic loops
    o << "static __device__ __forceinline__ void load_tile(const PassLaunch& P, const ItemGeo& g, uint32_t dst, "
         "int lane, const CopyCtx& cc) { GenericCopy::load_tile(P, g, dst, lane, cc); }\n"
      << "static __device__ __forceinline__ void store_tile(const PassLaunch& P, const ItemGeo& g, "
         "const float2* buf, int lane, const CopyCtx& cc) { GenericCopy::store_tile(P, g, buf, lane, cc); }\n";
    return;
  }
  const int k = d.k, L = d.L, nj = 1 << (k - 6);
  int8_t lpos[5];
  for (int t = 0; t < 5; t++) lpos[t] = d.gpos[t + 1];
  auto pin_mask = [&](const DevPin* pins, int n) {
    uint32_t m = 0;
    for (int i = 0; i < n; i++)
      for (int j = 0; j < k; j++)
        if (d.gpos[j] == pins[i].pos) m |= 1u << j;
    return m >> L;  // pinned-out runs: zeros from the load warp; pins inside a run: the stage warps
  };
  const uint32_t rm_in = pin_mask(d.pin_in, d.n_pin_in), rm_out = pin_mask(d.pin_out, d.n_pin_out);
  uint32_t G[1 << 8], lo[1 << 8], rj[1 << 8];
  uint32_t lows[8];
  int nlow = 0, lid[1 << 8];
  for (int j = 0; j < nj; j++) {
    const uint32_t e = 64u * (uint32_t)j;
    uint32_t g = 0;
    for (int b = 6; b < k; b++)
      if ((e >> b) & 1) g |= 1u << d.gpos[b];
    G[j] = g;
    lo[j] = S(e) & 0xFu;
    rj[j] = e >> L;
    int q = 0;
    while (q < nlow && lows[q] != lo[j]) q++;
    if (q == nlow) lows[nlow++] = lo[j];
    lid[j] = q;
  }
  std::string gl = deposit(lpos, 5);
  for (size_t at; (at = gl.find("tid")) != std::string::npos;) gl.replace(at, 3, "ln");
  // loads
  o << "static __device__ __forceinline__ void load_tile(const PassLaunch& P, const ItemGeo& g, uint32_t dst, "
       "int lane, const CopyCtx&) {\n"
    << "const uint32_t ln = (uint32_t)lane;\n"
    << "const float2* in = reinterpret_cast<const float2*>(P.nodes[g.node].in) + (g.base | " << gl << ");\n"
    << "const uint32_t s2 = swz(2u * ln);\n";
  for (int q = 0; q < nlow; q++) o << "const uint32_t d" << q << " = dst + 8u * (s2 ^ " << lows[q] << "u);\n";
  if (rm_in) o << "const uint32_t rl = ((2u * ln) >> " << L << ") & " << rm_in << "u, rv = g.lin_v >> " << L << ";\n";
  for (int j = 0; j < nj; j++) {
    if (rm_in) o << "if ((rl | " << (rj[j] & rm_in) << "u) == rv) ";
    o << "cp_async16(d" << lid[j] << " + " << 512u * j << "u, in + " << G[j] << "u);\n";
    if (rm_in) o << "else st_shared_zero16(d" << lid[j] << " + " << 512u * j << "u);\n";
  }
  o << "}\n";
  // stores, eight chunks in flight per lane
  o << "static __device__ __forceinline__ void store_tile(const PassLaunch& P, const ItemGeo& g, const float2* buf, "
       "int lane, const CopyCtx&) {\n"
    << "const uint32_t ln = (uint32_t)lane;\n"
    << "float2* out = reinterpret_cast<float2*>(P.nodes[g.node].out) + (g.base | " << gl << ");\n"
    << "const uint32_t s2 = swz(2u * ln);\n";
  for (int q = 0; q < nlow; q++)
    o << "const float4* b" << q << " = reinterpret_cast<const float4*>(buf + (s2 ^ " << lows[q] << "u));\n";
  if (rm_out)
    o << "const uint32_t rl = ((2u * ln) >> " << L << ") & " << rm_out << "u, rv = g.lout_v >> " << L << ";\n";
  for (int j0 = 0; j0 < nj; j0 += 8) {
    o << "{\n";
    for (int j = j0; j < std::min(nj, j0 + 8); j++)
      o << "const float4 q" << j - j0 << " = b" << lid[j] << "[" << 32u * j << "u];\n";
    for (int j = j0; j < std::min(nj, j0 + 8); j++) {
      if (rm_out) o << "if ((rl | " << (rj[j] & rm_out) << "u) == rv) ";
      o << "*reinterpret_cast<float4*>(out + " << G[j] << "u) = q" << j - j0 << ";\n";
    }
    o << "}\n";
  }
  o << "}\n";
}

// ---- packed complex stages ----------------------------------------------
// A register slot holds one complex amplitude in an FP32x2 register pair r.
// At generation time each slot carries a map M, a signed permutation of the
// pair: value (re, im) = M (r.x, r.y). Multiplying a value by i^k changes
// only M (M <- J^k M, J = [[0,-1],[1,0]]), so the Google gates' factors +-1,
// +-i and the even powers of e^{i pi/4} of the phase groups cost nothing. A
// butterfly out = c_a a + c_b b (c in {+-1, +-i}) is one packed add when the
// two terms' maps C(c_a) M_a and C(c_b) M_b have the same pattern (both
// diagonal or both anti-diagonal): r_out = r_a + D r_b, D = (C(c_a) M_a)^T
// C(c_b) M_b diagonal, with the map C(c_a) M_a; otherwise r_b is swapped first
// (two moves), which costs what the scalar form costs. Odd powers of
// e^{i pi/4}, the per-thread phase and the post scale act on the register
// pair with the map folded in; stores write the plain (re, im) layout.
struct M2 {
  int a[2][2];
};
M2 m2_id() { return M2{{{1, 0}, {0, 1}}}; }
M2 m2_mul(const M2& x, const M2& y) {
  M2 r{};
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) r.a[i][j] = x.a[i][0] * y.a[0][j] + x.a[i][1] * y.a[1][j];
  return r;
}
M2 m2_t(const M2& x) { return M2{{{x.a[0][0], x.a[1][0]}, {x.a[0][1], x.a[1][1]}}}; }  // inverse of a signed permutation
M2 m2_ipow(int k) {  // i^k as a real 2x2 matrix
  M2 J{{{0, -1}, {1, 0}}}, r = m2_id();
  for (int t = 0; t < (k & 3); t++) r = m2_mul(J, r);
  return r;
}
bool m2_anti(const M2& x) { return x.a[0][0] == 0; }
const M2 kSwap{{{0, 1}, {1, 0}}};

std::string pair_lit(int x, int y) {
  return "make_float2(" + std::string(x < 0 ? "-1.f" : "1.f") + ", " + (y < 0 ? "-1.f" : "1.f") + ")";
}

// Emit r_out = r_a + D r_b (D diagonal, entries +-1).
std::string cadd_expr(const std::string& ra, const std::string& rb, const M2& D) {
  if (D.a[0][0] == 1 && D.a[1][1] == 1) return "__fadd2_rn(" + ra + ", " + rb + ")";
  return "__ffma2_rn(" + rb + ", " + pair_lit(D.a[0][0], D.a[1][1]) + ", " + ra + ")";
}

// A packed-complex register stage (gates H, X^1/2, Y^1/2 and phase groups).
void gen_stage_cpack(std::ostringstream& o, const PassPlan& pp, const DevStage& st, int R, bool last,
                     const std::function<std::string(int)>& at, int j0) {
  const DevPass& d = pp.dev;
  const int NR = 1 << R;
  std::vector<M2> M(NR, m2_id());
  o << "float2 v[" << NR << "];\n";
  if (j0 >= 0) {
    for (int i = 0; i < NR; i++) {
      if ((i >> j0) & 1) continue;
      const int i1 = i | (1 << j0);
      o << "{ const float4 q = *reinterpret_cast<const float4*>(" << at(i) << "); v[" << i
        << "] = make_float2(q.x, q.y); v[" << i1 << "] = make_float2(q.z, q.w); }\n";
    }
  } else {
    for (int i = 0; i < NR; i++) o << "v[" << i << "] = *(" << at(i) << ");\n";
  }
  o << "int kst = 0;\n";
  bool kst = false;
  auto V = [](int i) { return "v[" + std::to_string(i) + "]"; };
  // r' = h (r + t J r): the value times e^{i pi/4} with the map M kept
  auto omega1 = [&](int i) {
    const M2 T = m2_mul(m2_t(M[i]), m2_mul(m2_ipow(1), M[i]));  // M^T J M = t J
    const int t = T.a[1][0];
    o << "{ const float2 r = " << V(i) << "; " << V(i) << " = __ffma2_rn(make_float2(r.y, r.x), make_float2("
      << (t > 0 ? "-" : "") << "0.70710678118654752f, " << (t > 0 ? "" : "-")
      << "0.70710678118654752f), __fmul2_rn(r, make_float2(0.70710678118654752f, 0.70710678118654752f))); }\n";
  };
  for (int oi = st.op_begin; oi < st.op_end; oi++) {
    const DevOp& op = pp.ops[oi];
    if (op.code == DOP_H || op.code == DOP_XH || op.code == DOP_YH) {
      // out0 = c0 a + c1 b, out1 = c2 a + c3 b as powers of i (+-1: 0 / 2, -i: 3)
      int c[4];
      if (op.code == DOP_H) c[0] = 0, c[1] = 0, c[2] = 0, c[3] = 2;
      else if (op.code == DOP_XH) c[0] = 0, c[1] = 3, c[2] = 3, c[3] = 0;
      else c[0] = 0, c[1] = 2, c[2] = 0, c[3] = 0;
      const int J = op.a;
      for (int i0 = 0; i0 < NR; i0++) {
        if ((i0 >> J) & 1) continue;
        const int i1 = i0 | (1 << J);
        const M2 Qa0 = m2_mul(m2_ipow(c[0]), M[i0]), Qb0 = m2_mul(m2_ipow(c[1]), M[i1]);
        const M2 Qa1 = m2_mul(m2_ipow(c[2]), M[i0]), Qb1 = m2_mul(m2_ipow(c[3]), M[i1]);
        const bool sw0 = m2_anti(Qa0) != m2_anti(Qb0), sw1 = m2_anti(Qa1) != m2_anti(Qb1);
        o << "{ const float2 a = " << V(i0) << ", b = " << V(i1) << ";";
        if (sw0 || sw1) o << " const float2 bs = make_float2(b.y, b.x);";
        const M2 D0 = m2_mul(m2_t(Qa0), sw0 ? m2_mul(Qb0, kSwap) : Qb0);
        const M2 D1 = m2_mul(m2_t(Qa1), sw1 ? m2_mul(Qb1, kSwap) : Qb1);
        o << " " << V(i0) << " = " << cadd_expr("a", sw0 ? "bs" : "b", D0) << "; " << V(i1) << " = "
          << cadd_expr("a", sw1 ? "bs" : "b", D1) << "; }\n";
        M[i0] = Qa0;
        M[i1] = Qa1;
      }
      continue;
    }
    if (op.code != DOP_PHASE) fail(SF_EINVAL, "internal: op without a packed complex form");
    const DevPhaseGroup& G = pp.phases[op.arg];
    for (int j = 0; j < R; j++)
      for (int l = 0; l < R; l++)
        if (((G.czq[j] >> l) & 1) != ((G.czq[l] >> j) & 1))
          fail(SF_EINVAL, "internal: asymmetric CZ partners in a phase group");
    o << "{ // phase group " << op.arg << "\n";
    for (int i = 0; i < NR; i++) {  // plan-static part
      int ku = 0;
      for (int j = 0; j < R; j++)
        if ((i >> j) & 1) {
          ku += G.wstat[j];
          for (int l = j + 1; l < R; l++)
            if (((i >> l) & 1) && ((G.czq[j] >> l) & 1)) ku += 4;
        }
      ku &= 7;
      M[i] = m2_mul(m2_ipow(ku >> 1), M[i]);
      if (ku & 1) omega1(i);
    }
    char b[160];
    auto kadd = [&](const std::string& e) {
      o << "kst += " << e << ";\n";
      kst = true;
    };
    if (G.m1) std::snprintf(b, sizeof b, "__popc(gfix & 0x%xu)", G.m1), kadd(b);
    if (G.m2) std::snprintf(b, sizeof b, "2 * __popc(gfix & 0x%xu)", G.m2), kadd(b);
    if (G.m4) std::snprintf(b, sizeof b, "4 * __popc(gfix & 0x%xu)", G.m4), kadd(b);
    for (int cc = 0; cc < G.nsh; cc++) {
      std::snprintf(b, sizeof b, "4 * __popc(gfix & (gfix >> %d) & 0x%xu)", G.sh[cc], G.shm[cc]);
      kadd(b);
    }
    std::string wr[MAX_R];
    bool sign_only[MAX_R];
    for (int j = 0; j < R; j++) {
      sign_only[j] = true;
      if (G.czf[j]) {
        std::snprintf(b, sizeof b, "4 * __popc(gfix & 0x%xu)", G.czf[j]);
        wr[j] = b;
      }
    }
    for (int si = 0; si < G.nsel; si++) {
      const auto& e = G.sel[si];
      std::string dg = e.xi >= 0 ? "digit_of(P.xshift, P.xbits, g.path, " + std::to_string(e.xi) + ")" : "0";
      std::snprintf(b, sizeof b, "(int)(0x%xu >> (8 * %s) & 0xffu)",
                    (uint32_t)e.w[0] | (uint32_t)e.w[1] << 8 | (uint32_t)e.w[2] << 16 | (uint32_t)e.w[3] << 24,
                    dg.c_str());
      if (e.reg >= 0) {
        if (!wr[e.reg].empty()) wr[e.reg] += " + ";
        wr[e.reg] += b;
        for (int dd = 0; dd < 4; dd++)
          if (e.w[dd] & 3) sign_only[e.reg] = false;
      } else {
        kadd(std::string(b) + " * (int)((gfix >> " + std::to_string(e.pos) + ") & 1u)");
      }
    }
    for (int j = 0; j < R; j++) {  // per-thread / per-path weights of register bits
      if (wr[j].empty()) continue;
      o << "{ const int w = " << wr[j] << ";\n";
      if (sign_only[j]) {
        o << "const float sg = (w & 4) ? -1.f : 1.f; const float2 sg2 = make_float2(sg, sg);\n";
        for (int i = 0; i < NR; i++)
          if ((i >> j) & 1) o << V(i) << " = __fmul2_rn(" << V(i) << ", sg2);\n";
      } else {
        // value * f = M r * f:  r' = fx r + fy (M^T J M) r
        o << "const float2 f = w8[w & 7]; const float2 fxx = make_float2(f.x, f.x), fpy = make_float2(-f.y, f.y), "
             "fny = make_float2(f.y, -f.y);\n";
        for (int i = 0; i < NR; i++) {
          if (!((i >> j) & 1)) continue;
          const M2 T = m2_mul(m2_t(M[i]), m2_mul(m2_ipow(1), M[i]));
          o << "{ const float2 r = " << V(i) << "; " << V(i) << " = __ffma2_rn(make_float2(r.y, r.x), "
            << (T.a[1][0] > 0 ? "fpy" : "fny") << ", __fmul2_rn(r, fxx)); }\n";
        }
      }
      o << "}\n";
    }
    o << "}\n";
  }
  // the stage's end: the per-thread phase e^{i pi kst/4} and the post scale,
  // with every slot's map folded in, so the registers hold (re, im)
  const bool scale = last && d.post_scale != 1.0f;
  if (kst) {
    o << "{ float2 f = w8[kst & 7];\n";
    if (scale) o << "f.x *= " << flit(d.post_scale) << "; f.y *= " << flit(d.post_scale) << ";\n";
  } else {
    o << "{\n";
  }
  for (int i = 0; i < NR; i++) {
    const M2& m = M[i];
    const bool anti = m2_anti(m);
    const int s0 = anti ? m.a[0][1] : m.a[0][0], s1 = anti ? m.a[1][0] : m.a[1][1];
    // value = (s0 c0, s1 c1), (c0, c1) = anti ? (r.y, r.x) : (r.x, r.y)
    const std::string src = anti ? "make_float2(" + V(i) + ".y, " + V(i) + ".x)" : V(i);
    const std::string sgn0 = s0 < 0 ? "-" : "", sgn1 = s1 < 0 ? "-" : "";
    if (kst) {
      // f * value: (fx c0' - fy c1', fy c0' + fx c1') with c' the signed components
      o << "{ const float2 c = " << src << "; " << V(i) << " = __ffma2_rn(make_float2(c.y, c.x), make_float2("
        << (s1 < 0 ? "" : "-") << "f.y, " << sgn0 << "f.y), __fmul2_rn(c, make_float2(" << sgn0 << "f.x, " << sgn1
        << "f.x))); }\n";
    } else if (scale) {
      o << V(i) << " = __fmul2_rn(" << src << ", make_float2(" << sgn0 << flit(d.post_scale) << ", " << sgn1
        << flit(d.post_scale) << "));\n";
    } else if (anti || s0 < 0 || s1 < 0) {
      if (s0 < 0 || s1 < 0) o << V(i) << " = __fmul2_rn(" << src << ", " << pair_lit(s0, s1) << ");\n";
      else o << V(i) << " = " << src << ";\n";
    }
  }
  o << "}\n(void)kst;\n";
  if (j0 >= 0) {
    for (int i = 0; i < NR; i++) {
      if ((i >> j0) & 1) continue;
      const int i1 = i | (1 << j0);
      o << "*reinterpret_cast<float4*>(" << at(i) << ") = make_float4(" << V(i) << ".x, " << V(i) << ".y, " << V(i1)
        << ".x, " << V(i1) << ".y);\n";
    }
  } else {
    for (int i = 0; i < NR; i++) o << "*(" << at(i) << ") = " << V(i) << ";\n";
  }
}

// One pass as a stage program: struct `name`_prog in namespace sf and an
// extern "C" kernel `name`.
std::string gen_pass(const PassPlan& pp, const std::string& name, bool pack, int nbuf) {
  const DevPass& d = pp.dev;
  const int R = d.R, k = d.k, NR = 1 << R;
  const TileSwz S = choose_swz(pp);
  std::ostringstream o;
  o << "namespace sf {\nstruct " << name << "_prog {\n";
  if (S.is_default()) {
    o << "static __device__ __forceinline__ uint32_t swz(uint32_t e) { return sf::swz(e); }\n";
  } else {
    o << "static __device__ __forceinline__ uint32_t swz(uint32_t e) {\n  return e";
    for (int q = 0; q < 3; q++) o << " ^ ((uint32_t)(__popc(e & " << S.m[q] << "u) & 1) << " << 1 + q << ")";
    o << ";\n}\n";
  }
  o
    << "static __device__ __forceinline__ void run(const PassLaunch& P, float2* sm, const ItemGeo& g, "
       "const float2* w8, int ncomp, bool active) {\n"
    << "const uint32_t tid = threadIdx.x;\n(void)P; (void)g; (void)w8;\n";
  for (int s = 0; s < d.n_stages; s++) {
    const DevStage& st = pp.stages[s];
    if (st.r != R) fail(SF_EINVAL, "internal: stage width differs from the pass");
    uint32_t C[32];
    int gr[MAX_R];
    for (int i = 0; i < NR; i++) {
      uint32_t c = 0;
      for (int j = 0; j < R; j++)
        if ((i >> j) & 1) c ^= S(1u << st.rbit[j]);
      C[i] = c;
    }
    for (int j = 0; j < R; j++) gr[j] = d.gpos[st.rbit[j]];
    // packed complex form (FP32x2): stages of H, X^1/2, Y^1/2 and phase groups
    bool packed = pack;
    for (int oi = st.op_begin; oi < st.op_end && packed; oi++) {
      const int c = pp.ops[oi].code;
      if (c != DOP_H && c != DOP_XH && c != DOP_YH && c != DOP_PHASE) packed = false;
    }
    o << "if (active) { // stage " << s << (packed ? " (packed)" : "") << "\n";
    o << "const uint32_t pf = swz(" << deposit(st.tpos, k - R) << ");\n";
    o << "const uint32_t gfix = g.base | " << deposit(st.tg, k - R) << ";\n(void)gfix;\n";
    // Addresses pf ^ C_i: the swizzle only touches bits 1..3, so with
    // pf = ph | pl and C_i = h_i | l_i split at bit 4, pf ^ C_i =
    // (ph | (pl ^ l_i)) + h_i. One base pointer per distinct low part l, and a
    // constant offset h_i per access.
    uint32_t lows[32];
    int nlow = 0;
    auto low_id = [&](uint32_t l) {
      for (int q = 0; q < nlow; q++)
        if (lows[q] == l) return q;
      lows[nlow] = l;
      return nlow++;
    };
    int lid[32];
    for (int i = 0; i < NR; i++) lid[i] = low_id(C[i] & 0xFu);
    o << "const uint32_t ph = pf & ~0xFu, pl = pf & 0xFu;\n";
    for (int q = 0; q < nlow; q++) o << "float2* const sb" << q << " = sm + (ph | (pl ^ " << lows[q] << "u));\n";
    auto at = [&](int i) { return "sb" + std::to_string(lid[i]) + " + " + std::to_string(C[i] & ~0xFu) + "u"; };
    // when tile bit 0 is a register bit, amplitudes i and i ^ (1 << j0) share
    // a 16-byte chunk (swz keeps chunks whole): move them as one float4
    int j0 = -1;
    for (int j = 0; j < R; j++)
      if (st.rbit[j] == 0) j0 = j;
    if (packed) {
      gen_stage_cpack(o, pp, st, R, s == d.n_stages - 1, at, j0);
      o << "}\ncompute_bar(ncomp);\n";
      continue;
    }
    auto RE = [&](int i) { return "v[" + std::to_string(i) + "].x"; };
    auto IM = [&](int i) { return "v[" + std::to_string(i) + "].y"; };
    o << "float2 v[" << NR << "];\n";
    if (j0 >= 0) {
      for (int i = 0; i < NR; i++) {
        if ((i >> j0) & 1) continue;
        const int i1 = i | (1 << j0);
        o << "{ const float4 q = *reinterpret_cast<const float4*>(" << at(i) << "); " << RE(i) << " = q.x; "
          << IM(i) << " = q.y; " << RE(i1) << " = q.z; " << IM(i1) << " = q.w; }\n";
      }
    } else {
      for (int i = 0; i < NR; i++) o << "v[" << i << "] = *(" << at(i) << ");\n";
    }
    bool kst = false;  // per-thread phase accumulated over the stage
    o << "int kst = 0;\n";
    for (int oi = st.op_begin; oi < st.op_end; oi++) {
      const DevOp& op = pp.ops[oi];
      switch (op.code) {
        case DOP_H:
          o << "g_h<" << R << ", " << op.a << ">(v);\n";
          break;
        case DOP_XH:
          o << "g_xh<" << R << ", " << op.a << ">(v);\n";
          break;
        case DOP_YH:
          o << "g_yh<" << R << ", " << op.a << ">(v);\n";
          break;
        case DOP_G1:
          o << "g_1<" << R << ", " << op.a << ">(v, " << f2lit(pp.mats, op.arg) << ", "
            << f2lit(pp.mats, op.arg + 1) << ", " << f2lit(pp.mats, op.arg + 2) << ", "
            << f2lit(pp.mats, op.arg + 3) << ");\n";
          break;
        case DOP_G1SEL:
          o << "{ const int dg = digit_of(P.xshift, P.xbits, g.path, " << op.xi << ");\n"
            << "const float* m = P.mats + 2 * (" << op.arg << " + 4 * dg);\n"
            << "g_1<" << R << ", " << op.a
            << ">(v, make_float2(m[0], m[1]), make_float2(m[2], m[3]), make_float2(m[4], m[5]), "
               "make_float2(m[6], m[7])); }\n";
          break;
        case DOP_G2:
          o << "g_2<" << R << ", " << op.a << ", " << op.b << ">(v, P.mats + " << 2 * op.arg << ");\n";
          break;
        case DOP_DMUL: {
          int jr = -1;
          for (int j = 0; j < R; j++)
            if (gr[j] == op.a) jr = j;
          if (jr >= 0) {
            o << "g_dmul<" << R << ", " << jr << ">(v, " << f2lit(pp.mats, op.arg) << ", "
              << f2lit(pp.mats, op.arg + 1) << ");\n";
          } else {
            o << "{ const float2 f = ((gfix >> " << op.a << ") & 1u) ? " << f2lit(pp.mats, op.arg + 1) << " : "
              << f2lit(pp.mats, op.arg) << ";\n#pragma unroll\nfor (int i = 0; i < " << NR
              << "; i++) v[i] = cmul(f, v[i]); }\n";
          }
          break;
        }
        case DOP_PHASE: {
          const DevPhaseGroup& G = pp.phases[op.arg];
          // plan-static part: weights and CZs among register bits
          for (int j = 0; j < R; j++)
            for (int l = 0; l < R; l++)
              if (((G.czq[j] >> l) & 1) != ((G.czq[l] >> j) & 1))
                fail(SF_EINVAL, "internal: asymmetric CZ partners in a phase group");
          o << "{ // phase group " << op.arg << "\n";
          for (int i = 0; i < NR; i++) {
            int ku = 0;
            for (int j = 0; j < R; j++)
              if ((i >> j) & 1) {
                ku += G.wstat[j];
                for (int l = j + 1; l < R; l++)
                  if (((i >> l) & 1) && ((G.czq[j] >> l) & 1)) ku += 4;
              }
            ku &= 7;
            if (ku)
              o << "{ const float2 a = omega_mul<" << ku << ">(make_float2(" << RE(i) << ", " << IM(i) << ")); "
                << RE(i) << " = a.x; " << IM(i) << " = a.y; }\n";
          }
          // per-thread scalar part (fixed index bits), summed over the stage
          auto kadd = [&](const std::string& e) {
            o << "kst += " << e << ";\n";
            kst = true;
          };
          char b[160];
          if (G.m1) {
            std::snprintf(b, sizeof b, "__popc(gfix & 0x%xu)", G.m1);
            kadd(b);
          }
          if (G.m2) {
            std::snprintf(b, sizeof b, "2 * __popc(gfix & 0x%xu)", G.m2);
            kadd(b);
          }
          if (G.m4) {
            std::snprintf(b, sizeof b, "4 * __popc(gfix & 0x%xu)", G.m4);
            kadd(b);
          }
          for (int c = 0; c < G.nsh; c++) {
            std::snprintf(b, sizeof b, "4 * __popc(gfix & (gfix >> %d) & 0x%xu)", G.sh[c], G.shm[c]);
            kadd(b);
          }
          // per-thread / per-path weights of register bits
          std::string wr[MAX_R];
          bool sign_only[MAX_R];
          for (int j = 0; j < R; j++) {
            sign_only[j] = true;
            if (G.czf[j]) {
              std::snprintf(b, sizeof b, "4 * __popc(gfix & 0x%xu)", G.czf[j]);
              wr[j] = b;
            }
          }
          for (int si = 0; si < G.nsel; si++) {
            const auto& e = G.sel[si];
            std::string dg = e.xi >= 0 ? "digit_of(P.xshift, P.xbits, g.path, " + std::to_string(e.xi) + ")" : "0";
            std::snprintf(b, sizeof b, "(int)(0x%xu >> (8 * %s) & 0xffu)",
                          (uint32_t)e.w[0] | (uint32_t)e.w[1] << 8 | (uint32_t)e.w[2] << 16 | (uint32_t)e.w[3] << 24,
                          dg.c_str());
            if (e.reg >= 0) {
              if (!wr[e.reg].empty()) wr[e.reg] += " + ";
              wr[e.reg] += b;
              for (int dd = 0; dd < 4; dd++)
                if (e.w[dd] & 3) sign_only[e.reg] = false;
            } else {
              kadd(std::string(b) + " * (int)((gfix >> " + std::to_string(e.pos) + ") & 1u)");
            }
          }
          for (int j = 0; j < R; j++) {
            if (wr[j].empty()) continue;
            o << "{ const int w = " << wr[j] << ";\n";
            if (sign_only[j]) {
              o << "const float sg = (w & 4) ? -1.f : 1.f;\n";
              for (int i = 0; i < NR; i++)
                if ((i >> j) & 1) o << RE(i) << " *= sg; " << IM(i) << " *= sg;\n";
            } else {
              o << "const float2 f = w8[w & 7];\n";
              for (int i = 0; i < NR; i++)
                if ((i >> j) & 1)
                  o << "{ const float2 a = cmul(make_float2(" << RE(i) << ", " << IM(i) << "), f); " << RE(i)
                    << " = a.x; " << IM(i) << " = a.y; }\n";
            }
            o << "}\n";
          }
          o << "}\n";
          break;
        }
        default:
          fail(SF_EINVAL, "internal: op code without a specialised form");
      }
    }
    const bool last = s == d.n_stages - 1;
    const bool scale = last && d.post_scale != 1.0f;
    if (kst) {
      o << "{ float2 f = w8[kst & 7];\n";
      if (scale) o << "f.x *= " << flit(d.post_scale) << "; f.y *= " << flit(d.post_scale) << ";\n";
      o << "#pragma unroll\nfor (int i = 0; i < " << NR << "; i++) v[i] = cmul(v[i], f); }\n";
    } else if (scale) {
      o << "#pragma unroll\nfor (int i = 0; i < " << NR << "; i++) { v[i].x *= " << flit(d.post_scale)
        << "; v[i].y *= " << flit(d.post_scale) << "; }\n";
    }
    o << "(void)kst;\n";
    if (j0 >= 0) {
      for (int i = 0; i < NR; i++) {
        if ((i >> j0) & 1) continue;
        const int i1 = i | (1 << j0);
        o << "*reinterpret_cast<float4*>(" << at(i) << ") = make_float4(" << RE(i) << ", " << IM(i) << ", " << RE(i1)
          << ", " << IM(i1) << ");\n";
      }
    } else {
      for (int i = 0; i < NR; i++) o << "*(" << at(i) << ") = v[" << i << "];\n";
    }
    o << "}\ncompute_bar(ncomp);\n";
  }
  o << "}\n";
  gen_geo(o, pp);
  gen_copy(o, pp, S);
  o << "};\n}  // namespace sf\n";
  const int threads = (((1 << (k - R)) + 31) / 32) * 32 + 64;  // stage warps + the two copy warps
  // tiles of up to 2^12 amplitudes leave shared memory for two CTAs per SM
  // with three buffers, three CTAs with two: ask for the registers to allow it
  const int min_blocks = k > 12 ? 1 : (nbuf == 2 ? 3 : 2);
  o << "extern \"C\" __global__ void __launch_bounds__(" << threads << ", " << min_blocks << ") " << name
    << "(const __grid_constant__ sf::PassLaunch P) {\n  sf::pass_body<" << R << ", sf::" << name << "_prog, "
    << nbuf << ">(P);\n}\n";
  return o.str();
}

std::string layout_asserts() {
  std::ostringstream o;
  auto sz = [&](const char* t, size_t n) {
    o << "static_assert(sizeof(sf::" << t << ") == " << n << ", \"layout of " << t << "\");\n";
  };
  sz("PassLaunch", sizeof(PassLaunch));
  sz("DevPass", sizeof(DevPass));
  sz("DevStage", sizeof(DevStage));
  sz("DevOp", sizeof(DevOp));
  sz("DevPhaseGroup", sizeof(DevPhaseGroup));
  sz("PassNode", sizeof(PassNode));
  return o.str();
}

// -------------------------------------------------------- compiled cache
struct Entry {
  std::string name;  // the kernel's name
  int nbuf = 3;      // tile buffers
  std::string src;
  std::string cubin;
  std::string err;
  bool compiled = false;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  size_t smem_set = 0;
  int per_sm = 0;
};

std::mutex g_mu;
std::map<std::string, std::unique_ptr<Entry>>& cache() {
  static std::map<std::string, std::unique_ptr<Entry>> c;
  return c;
}

// Kernel names: the last pass of a final program (the one that writes the
// gather's input, compact or whole) is sf_pass_final, every other pass
// sf_pass_spec, so profiles can tell them apart.
const char* kKernelName = "sf_pass_spec";
const char* kFinalKernelName = "sf_pass_final";

void compile_entry(Entry* e) {
  const Nvrtc& n = nvrtc();
  const std::string full = "#include \"dev_types.h\"\n#include \"pass_common.cuh\"\n" + layout_asserts() + e->src;
  const char* hdrs[] = {kJitDevTypes, kJitPassCommon};
  const char* hnames[] = {"dev_types.h", "pass_common.cuh"};
  nvrtcProgram prog = nullptr;
  if (n.create(&prog, full.c_str(), "sf_pass_spec.cu", 2, hdrs, hnames) != 0) {
    e->err = "nvrtcCreateProgram failed";
    e->compiled = true;
    return;
  }
  const bool verbose = std::getenv("SF_JIT_VERBOSE") != nullptr;
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "-DNDEBUG", "--ptxas-options=-v"};
  const nvrtcResult rc = n.compile(prog, verbose ? 5 : 4, opts);
  if (verbose && rc == 0) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    std::fprintf(stderr, "%s\n", log.c_str());
  }
  if (rc != 0) {
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) n.log(prog, &log[0]);
    e->err = "NVRTC compile failed: " + log.substr(0, 2000);
  } else {
    size_t cs = 0;
    n.cubin_size(prog, &cs);
    e->cubin.assign(cs, '\0');
    n.cubin(prog, &e->cubin[0]);
  }
  n.destroy(&prog);
  e->compiled = true;
}

}  // namespace

// Tile buffers of a pass's kernel: sf_plan_opts.tile_buffers, where 0 = two
// buffers for tiles of 2^12 amplitudes or fewer (three CTAs per SM) and three
// above.
int tile_buffers(const Plan& p, const PassPlan& pp) {
  if (p.opts.tile_buffers == 2 || p.opts.tile_buffers == 3) return p.opts.tile_buffers;
  return pp.dev.k <= 12 ? 2 : 3;
}

// Compile (or find in the cache) a specialised kernel for every pass of the
// plan; passes get jit_id indexes into p.jit_entries.
void jit_prepare(Plan& p) {
  const Nvrtc& n = nvrtc();
  if (!n.ok) fail(SF_EUNSUPPORTED, "run-time specialised kernels need NVRTC: " + n.why);
  std::vector<PassPlan*> all;
  std::vector<bool> fin;
  const size_t nL = p.levels.size();
  for (HalfPlan* h : {&p.A, &p.B}) {
    // the final program: the merged or deferred last segment, else the last
    SegmentPlan* last = p.merged_last ? &h->last_merged : (p.deferred ? &h->last_deferred : &h->seg[nL]);
    auto add = [&](SegmentPlan& s) {
      for (size_t i = 0; i < s.passes.size(); i++) {
        all.push_back(&s.passes[i]);
        fin.push_back(&s == last && i + 1 == s.passes.size());
      }
    };
    for (auto& s : h->seg) add(s);
    add(h->last_deferred);
    add(h->last_merged);
  }
  std::vector<Entry*> todo;
  p.jit_entries.clear();
  const char* dump = std::getenv("SF_JIT_DUMP");  // directory for the generated sources
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t ai = 0; ai < all.size(); ai++) {
      PassPlan* pp = all[ai];
      const char* kname = fin[ai] ? kFinalKernelName : kKernelName;
      const int nbuf = tile_buffers(p, *pp);
      std::string src = gen_pass(*pp, kname, p.opts.fp32x2 != 0, nbuf);
      if (dump) {
        const std::string fn = std::string(dump) + "/pass_" + std::to_string(p.jit_entries.size()) + ".cu";
        if (FILE* f = std::fopen(fn.c_str(), "w")) {
          std::fputs(src.c_str(), f);
          std::fclose(f);
        }
      }
      auto& slot = cache()[src];
      if (!slot) {
        slot = std::make_unique<Entry>();
        slot->name = kname;
        slot->nbuf = nbuf;
        slot->src = src;
        todo.push_back(slot.get());
      }
      pp->jit_id = (int)p.jit_entries.size();
      p.jit_entries.push_back(slot.get());
    }
  }
  // compile the new ones in parallel (NVRTC programs are independent)
  unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (const char* e = std::getenv("SF_JIT_THREADS")) hw = std::max(1, std::atoi(e));
  std::vector<std::thread> th;
  std::mutex qmu;
  size_t next = 0;
  for (unsigned t = 0; t < std::min<size_t>(hw, todo.size()); t++)
    th.emplace_back([&] {
      while (true) {
        size_t i;
        {
          std::lock_guard<std::mutex> lk(qmu);
          if (next >= todo.size()) return;
          i = next++;
        }
        compile_entry(todo[i]);
      }
    });
  for (auto& t : th) t.join();
  for (void* v : p.jit_entries) {
    Entry* e = static_cast<Entry*>(v);
    if (!e->err.empty()) fail(SF_EINVAL, "internal: specialised pass kernel: " + e->err);
  }
}

std::string jit_source(const PassPlan& pp) { return gen_pass(pp, kKernelName, true, 3); }

namespace {

// Threads and dynamic shared memory of a pass launch (the generic kernel's
// shape): stage warps + the two copy warps; three tile buffers, the run
// offsets and the nine mbarriers.
void pass_shape(const DevPass& d, int nbuf, int* threads, size_t* smem) {
  const int nact = 1 << (d.k - d.R);
  *threads = ((nact + 31) / 32) * 32 + 64;
  const int nruns = 1 << (d.k - d.L);
  *smem = (size_t)nbuf * ((size_t)8 << d.k) + 4 * (size_t)((nruns + 1) & ~1) + 3 * (size_t)nbuf * 8;
}

// Load the entry's library and kernel (caller holds g_mu), give it the
// shared memory of a launch of this shape and compute its occupancy; the
// attribute call loads the kernel into the current device's context.
void ready_entry(Entry* e, int threads, size_t smem) {
  if (!e->kern) {
    cudaError_t rc = cudaLibraryLoadData(&e->lib, e->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (rc != cudaSuccess) fail(SF_ECUDA, std::string("cudaLibraryLoadData: ") + cudaGetErrorString(rc));
    rc = cudaLibraryGetKernel(&e->kern, e->lib, e->name.c_str());
    if (rc != cudaSuccess) fail(SF_ECUDA, std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(rc));
  }
  if (smem > e->smem_set) {
    cudaError_t rc =
        cudaFuncSetAttribute((const void*)e->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (rc != cudaSuccess) fail(SF_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(rc));
    e->smem_set = smem;
    e->per_sm = 0;
  }
  if (!e->per_sm) {
    int v = 0;
    cudaError_t rc = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, (const void*)e->kern, threads, smem);
    if (rc != cudaSuccess) fail(SF_ECUDA, std::string("cudaOccupancy: ") + cudaGetErrorString(rc));
    e->per_sm = v > 0 ? v : 1;
  }
}

}  // namespace

void jit_load(Plan& p) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (HalfPlan* h : {&p.A, &p.B}) {
    std::vector<const PassPlan*> all;
    for (auto& s : h->seg)
      for (auto& pp : s.passes) all.push_back(&pp);
    for (auto& pp : h->last_deferred.passes) all.push_back(&pp);
    for (auto& pp : h->last_merged.passes) all.push_back(&pp);
    for (const PassPlan* pp : all) {
      if (pp->jit_id < 0) continue;
      int threads;
      size_t smem;
      Entry* e = static_cast<Entry*>(p.jit_entries[pp->jit_id]);
      pass_shape(pp->dev, e->nbuf, &threads, &smem);
      ready_entry(e, threads, smem);
    }
  }
}

// Launch a pass with its specialised kernel; same launch shape as the
// generic kernel.
void launch_pass_jit(const PassLaunch& L, int tiles, void* entry, void* stream) {
  Entry* e = static_cast<Entry*>(entry);
  int threads;
  size_t smem;
  pass_shape(L.pass, e->nbuf, &threads, &smem);
  int nb;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    ready_entry(e, threads, smem);  // a no-op once jit_load ran on this device
    nb = e->per_sm;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t items = (int64_t)tiles * L.n_nodes;
  const int64_t grid = std::min<int64_t>(items, (int64_t)sms * nb);
  if (grid < 1) return;
  // programmatic dependent launch: the kernel waits (griddepcontrol.wait)
  // for the previous work of the stream before it touches global memory
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<PassLaunch*>(&L)};
  cudaError_t rc = cudaLaunchKernelExC(&cfg, (const void*)e->kern, args);
  if (rc != cudaSuccess) fail(SF_ECUDA, std::string("specialised pass kernel launch: ") + cudaGetErrorString(rc));
}

}  // namespace sf
