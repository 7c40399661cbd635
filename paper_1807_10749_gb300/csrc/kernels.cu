// Device kernels of the Schroedinger-Feynman path sum (arXiv:1807.10749).
//
//  pass_kernel   - one fused pass over a half-state: each CTA owns a tile of
//                  2^k amplitudes (the low L index bits plus k-L chosen higher
//                  bits), stages it in shared memory, and runs a sequence of
//                  register stages; a stage gives every thread 2^R amplitudes
//                  whose R "register bits" vary, applies the stage's gates in
//                  registers, and writes them back. Gates: the Google gates in
//                  their multiplication-free integer form (Section 2: only the
//                  T gates need floating-point multiplications), general 2x2
//                  and 4x4 matrices, per-path cross-gate factors (Eq. 1 and
//                  Section 7), and groups of diagonal gates applied as one
//                  mod-8 power of e^{i pi/4} computed from bitmasks (Section 2:
//                  parity / popcount and mod-8 arithmetic). Projections are
//                  never executed: the zero half of a projected qubit is not
//                  read or written (Section 2: zero-block skipping).
//  gather_kernel - for each requested bitstring x, the product of the two
//                  halves' amplitudes at (x_A, x_B) summed over a batch of
//                  paths (Eq. 2), with the last branch level contracted in
//                  closed form when the planner deferred it; FP64 accumulation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "sf_internal.h"
#include "pass_common.cuh"

namespace sf {

namespace {

template <int R>
__device__ __forceinline__ void dispatch_1q(int code, int a, float2* v) {
#define SF_CASE(J)                                    \
  case J:                                             \
    if constexpr (J < R) {                            \
      if (code == DOP_H) g_h<R, J>(v);                \
      else if (code == DOP_XH) g_xh<R, J>(v);         \
      else g_yh<R, J>(v);                             \
    }                                                 \
    break;
  switch (a) { SF_CASE(0) SF_CASE(1) SF_CASE(2) SF_CASE(3) SF_CASE(4) }
#undef SF_CASE
}

template <int R>
__device__ __forceinline__ void dispatch_g1(int a, float2* v, float2 m0, float2 m1, float2 m2, float2 m3) {
#define SF_CASE(J) \
  case J:          \
    if constexpr (J < R) g_1<R, J>(v, m0, m1, m2, m3); \
    break;
  switch (a) { SF_CASE(0) SF_CASE(1) SF_CASE(2) SF_CASE(3) SF_CASE(4) }
#undef SF_CASE
}

template <int R>
__device__ __forceinline__ void dispatch_dmul(int a, float2* v, float2 f0, float2 f1) {
#define SF_CASE(J) \
  case J:          \
    if constexpr (J < R) g_dmul<R, J>(v, f0, f1); \
    break;
  switch (a) { SF_CASE(0) SF_CASE(1) SF_CASE(2) SF_CASE(3) SF_CASE(4) }
#undef SF_CASE
}

template <int R>
__device__ __forceinline__ void dispatch_g2(int a, int b, float2* v, const float* m) {
#define SF_C2(A, B)                                                          \
  case (A * 8 + B):                                                          \
    if constexpr (A < R && B < R && A != B) g_2<R, A, B>(v, m); \
    break;
#define SF_ROW(A) SF_C2(A, 0) SF_C2(A, 1) SF_C2(A, 2) SF_C2(A, 3) SF_C2(A, 4)
  switch (a * 8 + b) { SF_ROW(0) SF_ROW(1) SF_ROW(2) SF_ROW(3) SF_ROW(4) }
#undef SF_ROW
#undef SF_C2
}

// Phase group on a register block: the quadratic form of DevPhaseGroup,
// evaluated in Gray-code order (one update per amplitude), then a multiply by
// e^{i pi k/4} from a table in shared memory.
template <int R>
__device__ __forceinline__ void apply_phase(const DevPhaseGroup& g, float2* v, uint32_t gfix,
                                            const uint8_t* xshift, const uint8_t* xbits, uint64_t path,
                                            const float2* w8) {
  int k0 = __popc(gfix & g.m1) + 2 * __popc(gfix & g.m2) + 4 * __popc(gfix & g.m4);
  for (int c = 0; c < g.nsh; c++) k0 += 4 * __popc(gfix & (gfix >> g.sh[c]) & g.shm[c]);
  int w[R];
#pragma unroll
  for (int j = 0; j < R; j++) w[j] = (int)g.wstat[j] + 4 * __popc(gfix & g.czf[j]);
  for (int s = 0; s < g.nsel; s++) {
    const int d = g.sel[s].xi >= 0 ? digit_of(xshift, xbits, path, g.sel[s].xi) : 0;
    const int ws = g.sel[s].w[d];
    const int r = g.sel[s].reg;
    if (r >= 0) {
#pragma unroll
      for (int j = 0; j < R; j++)
        if (j == r) w[j] += ws;
    } else {
      k0 += ws * (int)((gfix >> g.sel[s].pos) & 1u);
    }
  }
  int kk = k0;
  v[0] = cmul(v[0], w8[kk & 7]);
#pragma unroll
  for (int i = 1; i < (1 << R); i++) {
    const int gi = i ^ (i >> 1);
    const int prev = (i - 1) ^ ((i - 1) >> 1);
    const int j = cctz(gi ^ prev);  // flipped bit (compile time)
    const int rest = gi & ~(1 << j);
    const int delta = w[j] + 4 * __popc((uint32_t)g.czq[j] & (uint32_t)rest);
    if (gi & (1 << j)) kk += delta;
    else kk -= delta;
    v[gi] = cmul(v[gi], w8[kk & 7]);
  }
}

}  // namespace

template <int R, bool GEN>
__device__ __forceinline__ void run_stages(const PassLaunch& P, float2* sm, const ItemGeo& g, const float2* w8,
                                           int ncomp, bool active) {
  const float post_scale = P.pass.post_scale;
  const DevPass& d = P.pass;
  const int k = d.k;
  for (int s = 0; s < d.n_stages; s++) {
    if (active) {  // idle threads skip to the same barrier instruction
      const DevStage& st = P.stages[s];
      uint32_t poff[R];
      int gr[R];
#pragma unroll
      for (int j = 0; j < R; j++) {
        poff[j] = swz(1u << st.rbit[j]);
        gr[j] = d.gpos[st.rbit[j]];
      }
      uint32_t lfix = 0, gfix = g.base;
      for (int t = 0; t < k - R; t++) {
        const uint32_t b = (threadIdx.x >> t) & 1u;
        lfix |= b << st.tpos[t];
        gfix |= b << st.tg[t];
      }
      const uint32_t pfix = swz(lfix);
      float2 v[1 << R];
      {
        uint32_t addr = pfix;
        v[0] = sm[addr];
#pragma unroll
        for (int i = 1; i < (1 << R); i++) {
          const int gi = i ^ (i >> 1), prev = (i - 1) ^ ((i - 1) >> 1);
          addr ^= poff[cctz(gi ^ prev)];
          v[gi] = sm[addr];
        }
      }
      for (int o = st.op_begin; o < st.op_end; o++) {
        const DevOp& op = P.ops[o];
        switch (op.code) {
          case DOP_H:
          case DOP_XH:
          case DOP_YH:
            dispatch_1q<R>(op.code, op.a, v);
            break;
          case DOP_PHASE:
            apply_phase<R>(P.phases[op.arg], v, gfix, P.xshift, P.xbits, g.path, w8);
            break;
          default:
            if constexpr (GEN) {
              switch (op.code) {
              case DOP_G1: {
                const float* m = P.mats + 2 * op.arg;
                dispatch_g1<R>(op.a, v, make_float2(m[0], m[1]), make_float2(m[2], m[3]),
                               make_float2(m[4], m[5]), make_float2(m[6], m[7]));
                break;
              }
              case DOP_G1SEL: {
                const int dg = digit_of(P.xshift, P.xbits, g.path, op.xi);
                const float* m = P.mats + 2 * (op.arg + 4 * dg);
                dispatch_g1<R>(op.a, v, make_float2(m[0], m[1]), make_float2(m[2], m[3]),
                               make_float2(m[4], m[5]), make_float2(m[6], m[7]));
                break;
              }
              case DOP_G2:
                dispatch_g2<R>(op.a, op.b, v, P.mats + 2 * op.arg);
                break;
              case DOP_DMUL: {
                const float* m = P.mats + 2 * op.arg;
                const float2 f0 = make_float2(m[0], m[1]), f1 = make_float2(m[2], m[3]);
                int jr = -1;
#pragma unroll
                for (int j = 0; j < R; j++)
                  if (gr[j] == op.a) jr = j;
                if (jr >= 0) {
                  dispatch_dmul<R>(jr, v, f0, f1);
                } else {
                  const float2 f = ((gfix >> op.a) & 1u) ? f1 : f0;
#pragma unroll
                  for (int i = 0; i < (1 << R); i++) v[i] = cmul(f, v[i]);
                }
                break;
              }
              default:
                  break;
              }
            }
            break;
        }
      }
      const float sc = (s == d.n_stages - 1) ? post_scale : 1.0f;
      {
        uint32_t addr = pfix;
        sm[addr] = make_float2(v[0].x * sc, v[0].y * sc);
#pragma unroll
        for (int i = 1; i < (1 << R); i++) {
          const int gi = i ^ (i >> 1), prev = (i - 1) ^ ((i - 1) >> 1);
          addr ^= poff[cctz(gi ^ prev)];
          sm[addr] = make_float2(v[gi].x * sc, v[gi].y * sc);
        }
      }
    }
    compute_bar(ncomp);
  }
}

// The generic stage program: reads the pass's stages, ops and phase groups
// from the launch record and dispatches on them.
template <int R, bool GEN>
struct GenericProg : GenericCopy {
  static __device__ __forceinline__ void run(const PassLaunch& P, float2* sm, const ItemGeo& g, const float2* w8,
                                             int ncomp, bool active) {
    run_stages<R, GEN>(P, sm, g, w8, ncomp, active);
  }
};

// Up to 2^(13-R) stage threads + the two copy warps: 320 at R = 5, 576 below.
template <int R, bool GEN>
__global__ void __launch_bounds__(R >= 5 ? 320 : 576, 1) pass_kernel(const __grid_constant__ PassLaunch P) {
  pass_body<R, GenericProg<R, GEN>>(P);
}

// ------------------------------------------------------------------ gather
// s + x with the rounding error of the addition added to c (Neumaier's
// variant of compensated summation, Numer. Math. 1974): IEEE round-to-nearest
// additions only, no contraction.
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  const double t = __dadd_rn(s, x);
  const double e = fabs(s) >= fabs(x) ? __dadd_rn(__dsub_rn(s, t), x) : __dadd_rn(__dsub_rn(x, t), s);
  c = __dadd_rn(c, e);
  s = t;
}

// Compact finals (CompactMap): part number of a layout index, and the slot
// of a part (marked parts below it; every requested bitstring's parts are
// marked).
__device__ __forceinline__ uint32_t compact_part(const CompactMap& c, uint32_t j) {
  return (pext32(j, c.cfree) << c.ckt) | pext32(j, c.cpart);
}
__device__ __forceinline__ uint32_t compact_slot(const uint32_t* cmap, uint32_t p) {
  const uint2 w = reinterpret_cast<const uint2*>(cmap)[p >> 5];
  return w.y + (uint32_t)__popc(w.x & ((1u << (p & 31)) - 1u));
}
// Index of amplitude j (layout index) of a final; h0 / h1: slot * 2^ctl of
// the block's first / second part.
__device__ __forceinline__ uint32_t compact_index(const CompactMap& c, uint32_t h0, uint32_t h1, uint32_t j) {
  if (!c.cmap) return j;
  const uint32_t h = (c.csub1 && ((j >> c.ctl) & 1u)) ? h1 : h0;
  return h | (j & ((1u << c.ctl) - 1u));
}

// ALL: every final of the launch sums all leaves of its folded group (the
// closed-form contraction only; fewer registers).
template <int G, bool ALL>
__global__ void __launch_bounds__(256, 2) gather_kernel(const __grid_constant__ GatherLaunch P) {
  __shared__ uint32_t tA[8 * 256], tB[8 * 256];
  // the folded level's 2x2 contraction matrices K_t[y, z] = sum_d MA_{t,d}[xa, y]
  // MB_{t,d}[xb, z] for every deferred gate t and bit pair (xa, xb): formed once
  // per CTA, not per bitstring
  __shared__ float2 Ks[G > 0 ? G : 1][4][2][2];
  for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) {
    tA[i] = P.tabA[i];
    tB[i] = P.tabB[i];
  }
  const int NY = 1 << G;
  const int tb = P.nterm_bits;
  const int nt = 1 << tb;
  if (G > 0 && threadIdx.x < G * 16) {
    const int t = threadIdx.x >> 4, ab = (threadIdx.x >> 2) & 3, y = (threadIdx.x >> 1) & 1, z = threadIdx.x & 1;
    const int xa_ = ab >> 1, xb_ = ab & 1;
    float2 acc = make_float2(0.f, 0.f);
    for (int dd = 0; dd < nt; dd++) {
      const float* ma = P.ma[t][dd];
      const float* mb = P.mb[t][dd];
      float2 a = make_float2(ma[2 * (2 * xa_ + y)], ma[2 * (2 * xa_ + y) + 1]);
      float2 b = make_float2(mb[2 * (2 * xb_ + z)], mb[2 * (2 * xb_ + z) + 1]);
      acc = cadd(acc, cmul(a, b));
    }
    Ks[t][ab][y][z] = acc;
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t x = P.bits[i];
    uint32_t ia = 0, ib = 0;
#pragma unroll
    for (int b = 0; b < 8; b++) {
      const uint32_t byte = (uint32_t)(x >> (8 * b)) & 255u;
      ia |= tA[b * 256 + byte];
      ib |= tB[b * 256 + byte];
    }
    int xa[G > 0 ? G : 1], xb[G > 0 ? G : 1];
#pragma unroll
    for (int t = 0; t < G; t++) {
      xa[t] = (int)((x >> P.A.dq[t]) & 1u);
      xb[t] = (int)((x >> P.B.dq[t]) & 1u);
    }
    // compact finals: slots of the parts of the bitstring's blocks (ia, ib
    // are zero at the block positions 0..G-1)
    uint32_t ha0 = 0, ha1 = 0, hb0 = 0, hb1 = 0;
    if (P.A.c.cmap) {
      const uint32_t p0 = compact_part(P.A.c, ia);
      ha0 = compact_slot(P.A.c.cmap, p0) << P.A.c.ctl;
      if (P.A.c.csub1) ha1 = compact_slot(P.A.c.cmap, p0 | P.A.c.csub1) << P.A.c.ctl;
    }
    if (P.B.c.cmap) {
      const uint32_t p0 = compact_part(P.B.c, ib);
      hb0 = compact_slot(P.B.c.cmap, p0) << P.B.c.ctl;
      if (P.B.c.csub1) hb1 = compact_slot(P.B.c.cmap, p0 | P.B.c.csub1) << P.B.c.ctl;
    }
    // Each final's contribution is added to the running FP64 sum in the
    // order of the finals, starting from the accumulator itself, so the
    // result does not depend on how finals are grouped into launches.
    double sr = P.acc[2 * i], si = P.acc[2 * i + 1];
    double cr = 0.0, ci = 0.0;  // compensation (P.comp != null)
    for (int f = 0; f < P.n_finals; f++) {
      const GatherFinal& F = P.finals[f];
      uint32_t pam = 0, pav = 0, pbm = 0, pbv = 0;
      for (int p = 0; p < P.A.npin; p++) {
        pam |= 1u << P.A.pin[p].pos;
        if (pin_val(P.A.pin[p], P.xshift, P.xbits, F.path)) pav |= 1u << P.A.pin[p].pos;
      }
      for (int p = 0; p < P.B.npin; p++) {
        pbm |= 1u << P.B.pin[p].pos;
        if (pin_val(P.B.pin[p], P.xshift, P.xbits, F.path)) pbv |= 1u << P.B.pin[p].pos;
      }
      const float2* WA = reinterpret_cast<const float2*>(F.wa);
      const float2* WB = reinterpret_cast<const float2*>(F.wb);
      auto load_a = [&](int y) {
        uint32_t ja = ia;
#pragma unroll
        for (int t = 0; t < G; t++) ja |= (uint32_t)((y >> t) & 1) << P.A.dpos[t];
        return ((ja & pam) == pav) ? WA[compact_index(P.A.c, ha0, ha1, ja)] : make_float2(0.f, 0.f);
      };
      float2 wb[1 << G];
#pragma unroll
      for (int y = 0; y < NY; y++) {
        uint32_t jb = ib;
#pragma unroll
        for (int t = 0; t < G; t++) jb |= (uint32_t)((y >> t) & 1) << P.B.dpos[t];
        wb[y] = ((jb & pbm) == pbv) ? WB[compact_index(P.B.c, hb0, hb1, jb)] : make_float2(0.f, 0.f);
      }
      float2 c = make_float2(0.f, 0.f);
      if constexpr (ALL && G > 0) {
        // every leaf of the group: contract wb (in place) with K_t[y, z] =
        // sum_d MA_{t,d}[xa_t, y] MB_{t,d}[xb_t, z], then dot with wa read
        // one amplitude at a time
#pragma unroll
        for (int t = 0; t < G; t++) {
          const float2(&K)[2][2] = Ks[t][2 * xa[t] + xb[t]];
#pragma unroll
          for (int y = 0; y < NY; y++) {
            if (y & (1 << t)) continue;
            const float2 t0 = wb[y], t1 = wb[y | (1 << t)];
            wb[y] = cadd(cmul(K[0][0], t0), cmul(K[0][1], t1));
            wb[y | (1 << t)] = cadd(cmul(K[1][0], t0), cmul(K[1][1], t1));
          }
        }
#pragma unroll
        for (int y = 0; y < NY; y++) c = cadd(c, cmul(load_a(y), wb[y]));
      } else {
      float2 wa[1 << G];
#pragma unroll
      for (int y = 0; y < NY; y++) wa[y] = load_a(y);
      if (G == 0) {
        c = cmul(wa[0], wb[0]);
      } else if (ALL || F.all_leaves) {
        // sum over every leaf: contract wb (in place) with K_t[y, z] = sum_d
        // MA_{t,d}[xa_t, y] MB_{t,d}[xb_t, z]
#pragma unroll
        for (int t = 0; t < G; t++) {
          const float2(&K)[2][2] = Ks[t][2 * xa[t] + xb[t]];
#pragma unroll
          for (int y = 0; y < NY; y++) {
            if (y & (1 << t)) continue;
            const float2 t0 = wb[y], t1 = wb[y | (1 << t)];
            wb[y] = cadd(cmul(K[0][0], t0), cmul(K[0][1], t1));
            wb[y | (1 << t)] = cadd(cmul(K[1][0], t0), cmul(K[1][1], t1));
          }
        }
#pragma unroll
        for (int y = 0; y < NY; y++) c = cadd(c, cmul(wa[y], wb[y]));
      } else if constexpr (!ALL) {
        const int nleaf = 1 << (G * tb);
        for (int b = 0; b < nleaf; b++) {
          if (!((F.leafmask[b >> 6] >> (b & 63)) & 1ull)) continue;
          float2 av = make_float2(0.f, 0.f), bv = make_float2(0.f, 0.f);
#pragma unroll
          for (int y = 0; y < NY; y++) {
            float2 ca = make_float2(1.f, 0.f), cb = make_float2(1.f, 0.f);
#pragma unroll
            for (int t = 0; t < G; t++) {
              const int dd = (b >> ((G - 1 - t) * tb)) & (nt - 1);
              const int yt = (y >> t) & 1;
              const float* ma = P.ma[t][dd];
              const float* mb = P.mb[t][dd];
              ca = cmul(ca, make_float2(ma[2 * (2 * xa[t] + yt)], ma[2 * (2 * xa[t] + yt) + 1]));
              cb = cmul(cb, make_float2(mb[2 * (2 * xb[t] + yt)], mb[2 * (2 * xb[t] + yt) + 1]));
            }
            av = cadd(av, cmul(ca, wa[y]));
            bv = cadd(bv, cmul(cb, wb[y]));
          }
          c = cadd(c, cmul(av, bv));
        }
      }
      }
      const double tr = (double)c.x * F.sre - (double)c.y * F.sim;
      const double ti = (double)c.x * F.sim + (double)c.y * F.sre;
      if (P.comp) {
        neumaier_add(sr, cr, tr);
        neumaier_add(si, ci, ti);
      } else {
        sr += tr;
        si += ti;
      }
    }
    P.acc[2 * i] = sr;
    P.acc[2 * i + 1] = si;
    if (P.comp) {
      P.comp[2 * i] += cr;
      P.comp[2 * i + 1] += ci;
    }
  }
}

// Accept step of frugal rejection sampling (Section 4, Algorithm 2), in the
// operation order documented in sfsim.h, without contraction.
__global__ void frugal_accept_kernel(const double* amps, const double* u, int64_t n, double N, double mp,
                                     double scale, uint8_t* acc, unsigned long long* count) {
  unsigned long long mine = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double re = amps[2 * i], im = amps[2 * i + 1];
    const double p = __dmul_rn(__dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im)), scale);
    const double t = __ddiv_rn(__dmul_rn(p, N), mp);
    const bool a = u[i] < fmin(1.0, t);
    acc[i] = a ? 1 : 0;
    mine += a ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

// ------------------------------------------------------ compact final maps
// Mark, per half, the parts of every requested bitstring's block.
__global__ void __launch_bounds__(256) block_mark_kernel(const __grid_constant__ BlockMapLaunch P) {
  __shared__ uint32_t tab[2][8 * 256];
  for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) {
    tab[0][i] = P.map[0] ? P.tab[0][i] : 0u;
    tab[1][i] = P.map[1] ? P.tab[1][i] : 0u;
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t x = P.bits[i];
    uint32_t ix0 = 0, ix1 = 0;
#pragma unroll
    for (int b = 0; b < 8; b++) {
      const uint32_t byte = (uint32_t)(x >> (8 * b)) & 255u;
      ix0 |= tab[0][b * 256 + byte];
      ix1 |= tab[1][b * 256 + byte];
    }
#pragma unroll
    for (int side = 0; side < 2; side++) {
      if (!P.map[side]) continue;
      const uint32_t p0 = compact_part(P.c[side], side ? ix1 : ix0);
      atomicOr(&P.map[side][2 * (p0 >> 5)], 1u << (p0 & 31));
      if (P.c[side].csub1) {
        const uint32_t p1 = p0 | P.c[side].csub1;
        atomicOr(&P.map[side][2 * (p1 >> 5)], 1u << (p1 & 31));
      }
    }
  }
}

// Prefix counts of the marked parts: chunks of kRankChunk map words per
// block of 256 threads (8 consecutive words a thread); pass 1 counts each
// chunk, pass 2 adds the chunks before it and scans within the chunk.
constexpr int kRankPer = 8;
constexpr int kRankChunk = 256 * kRankPer;

__device__ __forceinline__ uint32_t block_sum256(uint32_t v, uint32_t* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t t = 0;
  for (int q = 0; q < 8; q++) t += red[q];
  return t;
}

__global__ void __launch_bounds__(256) block_count_kernel(const __grid_constant__ BlockMapLaunch P) {
  const int side = blockIdx.y;
  const int64_t nw = P.nw[side];
  const int64_t w0 = (int64_t)blockIdx.x * kRankChunk;
  if (!P.map[side] || w0 >= nw) return;  // uniform over the block
  __shared__ uint32_t red[8];
  uint32_t c = 0;
#pragma unroll
  for (int j = 0; j < kRankPer; j++) {
    const int64_t w = w0 + (int64_t)threadIdx.x * kRankPer + j;
    if (w < nw) c += (uint32_t)__popc(P.map[side][2 * w]);
  }
  c = block_sum256(c, red);
  if (threadIdx.x == 0) P.sums[side][blockIdx.x] = c;
}

__global__ void __launch_bounds__(256) block_rank_kernel(const __grid_constant__ BlockMapLaunch P) {
  const int side = blockIdx.y;
  const int64_t nw = P.nw[side];
  const int64_t w0 = (int64_t)blockIdx.x * kRankChunk;
  if (!P.map[side] || w0 >= nw) return;  // uniform over the block
  __shared__ uint32_t red[8], wsum[8];
  uint32_t before = 0;
  for (int c = threadIdx.x; c < (int)blockIdx.x; c += blockDim.x) before += P.sums[side][c];
  before = block_sum256(before, red);
  uint32_t cnt[kRankPer], mine = 0;
#pragma unroll
  for (int j = 0; j < kRankPer; j++) {
    const int64_t w = w0 + (int64_t)threadIdx.x * kRankPer + j;
    cnt[j] = w < nw ? (uint32_t)__popc(P.map[side][2 * w]) : 0u;
    mine += cnt[j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t run = before + inc - mine;
  for (int q = 0; q < warp; q++) run += wsum[q];
#pragma unroll
  for (int j = 0; j < kRankPer; j++) {
    const int64_t w = w0 + (int64_t)threadIdx.x * kRankPer + j;
    if (w < nw) P.map[side][2 * w + 1] = run;
    run += cnt[j];
  }
  if (P.count[side] && w0 + kRankChunk >= nw && threadIdx.x == blockDim.x - 1) *P.count[side] = run;
}

__global__ void zero_kernel(double* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

// out += comp (the compensation terms of a compensated path sum).
__global__ void fold_kernel(double* out, const double* comp, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __dadd_rn(out[i], comp[i]);
}

// Probabilities |a|^2 * scale (Section 3: p(x) = |<x|psi>|^2; scale = 1 or
// 1 / f_actual), in exactly this operation order without contraction.
__global__ void prob_kernel(const double* amps, int64_t n, double scale, double* probs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double re = amps[2 * i], im = amps[2 * i + 1];
    probs[i] = __dmul_rn(__dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im)), scale);
  }
}

// ------------------------------------------------------------- launchers
static void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(SF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static int num_sms() {
  static int n = 0;  // one device per process is assumed for the SM count
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int R, bool GEN>
static void launch_pass_r(const PassLaunch& L, int tiles, int tile_k, cudaStream_t s) {
  const int nact = 1 << (tile_k - R);
  const int threads = ((nact + 31) / 32) * 32 + 64;  // compute warps + load and store warps
  const int nruns = 1 << (tile_k - L.pass.L);
  const size_t smem = 3 * ((size_t)8 << tile_k) + 4 * (size_t)((nruns + 1) & ~1) + 9 * 8;
  // The dynamic shared-memory limit is a property of the kernel function, so
  // it only ever grows; occupancy is cached per tile size.
  static std::mutex mu;
  static size_t smem_set = 0;
  static int per_sm[MAX_K + 1] = {0};
  int nb;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (smem > smem_set) {
      check(cudaFuncSetAttribute(pass_kernel<R, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "cudaFuncSetAttribute");
      smem_set = smem;
    }
    if (!per_sm[tile_k]) {
      int v = 0;
      check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, pass_kernel<R, GEN>, threads, smem),
            "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      per_sm[tile_k] = v > 0 ? v : 1;
    }
    nb = per_sm[tile_k];
  }
  const int64_t items = (int64_t)tiles * L.n_nodes;
  int64_t grid = std::min<int64_t>(items, (int64_t)num_sms() * nb);
  if (grid < 1) return;
  pass_kernel<R, GEN><<<(int)grid, threads, smem, s>>>(L);
  check(cudaGetLastError(), "pass_kernel launch");
}

void launch_pass(const PassLaunch& L, int tiles, int fuse_bits, int tile_bits, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const int k = L.pass.k;
  const int R = L.pass.R;
  if (k - R > 9 || k > 13 || R < 1) fail(SF_EINVAL, "internal: bad tile shape");
  (void)fuse_bits;
  (void)tile_bits;
  bool gen = false;  // does the pass need the general-gate variant?
  for (int i = 0; i < L.pass.n_stages; i++)
    for (int o = L.stages[i].op_begin; o < L.stages[i].op_end; o++) {
      const int c = L.ops[o].code;
      if (c == DOP_G1 || c == DOP_G1SEL || c == DOP_G2 || c == DOP_DMUL || c == DOP_DMULSEL) gen = true;
    }
#define SF_R(RR)                                                   \
  case RR:                                                         \
    if (gen) launch_pass_r<RR, true>(L, tiles, k, s);              \
    else launch_pass_r<RR, false>(L, tiles, k, s);                 \
    break;
  switch (R) {
    SF_R(1) SF_R(2) SF_R(3) SF_R(4) SF_R(5)
    default: fail(SF_EINVAL, "internal: bad register bits");
  }
#undef SF_R
}

void launch_gather(const GatherLaunch& L, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (L.n <= 0) return;
  const int threads = 256;
  int64_t blocks = (L.n + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  bool all = true;
  for (int f = 0; f < L.n_finals; f++) all = all && L.finals[f].all_leaves;
#define SF_G(GG)                                                                   \
  case GG:                                                                         \
    if (all) gather_kernel<GG, true><<<(int)blocks, threads, 0, s>>>(L);           \
    else gather_kernel<GG, false><<<(int)blocks, threads, 0, s>>>(L);              \
    break;
  switch (L.g) {
    SF_G(0) SF_G(1) SF_G(2) SF_G(3) SF_G(4)
    default: fail(SF_EINVAL, "internal: too many deferred gates");
  }
#undef SF_G
  check(cudaGetLastError(), "gather_kernel launch");
}

int launch_block_maps(const BlockMapLaunch& L0, const std::vector<std::pair<const uint64_t*, int64_t>>& sets,
                      void* stream) {
  BlockMapLaunch L = L0;
  cudaStream_t s = (cudaStream_t)stream;
  int launches = 0;
  int64_t maxw = 0;
  for (int side = 0; side < 2; side++)
    if (L.map[side]) {
      if (L.nw[side] < 1 || !L.sums[side]) fail(SF_EINVAL, "internal: block map without words");
      launch_zero(reinterpret_cast<double*>(L.map[side]), L.nw[side], stream);
      launches++;
      maxw = std::max(maxw, L.nw[side]);
    }
  if (maxw == 0) return launches;
  for (auto& set : sets) {
    if (set.second <= 0) continue;
    L.bits = set.first;
    L.n = set.second;
    const int64_t blocks = std::min<int64_t>((L.n + 255) / 256, (int64_t)num_sms() * 8);
    block_mark_kernel<<<(int)blocks, 256, 0, s>>>(L);
    check(cudaGetLastError(), "block_mark_kernel launch");
    launches++;
  }
  const dim3 grid((unsigned)((maxw + kRankChunk - 1) / kRankChunk), 2);
  block_count_kernel<<<grid, 256, 0, s>>>(L);
  check(cudaGetLastError(), "block_count_kernel launch");
  block_rank_kernel<<<grid, 256, 0, s>>>(L);
  check(cudaGetLastError(), "block_rank_kernel launch");
  return launches + 2;
}

void launch_zero(double* p, int64_t n, void* stream) {
  if (n <= 0) return;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  zero_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(p, n);
  check(cudaGetLastError(), "zero_kernel launch");
}

void launch_frugal(const double* amps, const double* u, int64_t n, double N, double mp, double scale,
                   uint8_t* acc, int64_t* count, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  check(cudaMemsetAsync(count, 0, sizeof(int64_t), s), "cudaMemsetAsync");
  if (n <= 0) return;
  int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
  frugal_accept_kernel<<<(int)blocks, 256, 0, s>>>(amps, u, n, N, mp, scale, acc,
                                                    reinterpret_cast<unsigned long long*>(count));
  check(cudaGetLastError(), "frugal_accept_kernel launch");
}

// Overlap sums for the validation protocol (Appendix C): one block-level FP64
// reduction per block, then atomics into the 4 outputs.
__global__ void overlap_kernel(const double* a, const double* b, int64_t n, double* out) {
  double r = 0, im = 0, na = 0, nb = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ar = a[2 * i], ai = a[2 * i + 1], br = b[2 * i], bi = b[2 * i + 1];
    r += ar * br + ai * bi;
    im += ar * bi - ai * br;
    na += ar * ar + ai * ai;
    nb += br * br + bi * bi;
  }
  __shared__ double red[4][32];
  for (int o = 16; o > 0; o >>= 1) {
    r += __shfl_down_sync(0xffffffffu, r, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
    na += __shfl_down_sync(0xffffffffu, na, o);
    nb += __shfl_down_sync(0xffffffffu, nb, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = r;
    red[1][w] = im;
    red[2][w] = na;
    red[3][w] = nb;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += red[threadIdx.x][q];
    atomicAdd(&out[threadIdx.x], t);
  }
}

// f_e = |<a|b>|^2 / (<a|a> <b|b>) from the four sums (Appendix C); 0 when
// either norm is zero.
__global__ void overlap_finish_kernel(double* out) {
  const double den = out[2] * out[3];
  out[4] = den > 0.0 ? (out[0] * out[0] + out[1] * out[1]) / den : 0.0;
}

void launch_overlap(const double* a, const double* b, int64_t n, double* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  check(cudaMemsetAsync(out, 0, 5 * sizeof(double), s), "cudaMemsetAsync");
  if (n > 0) {
    int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 4);
    overlap_kernel<<<(int)blocks, 256, 0, s>>>(a, b, n, out);
    check(cudaGetLastError(), "overlap_kernel launch");
  }
  overlap_finish_kernel<<<1, 1, 0, s>>>(out);
  check(cudaGetLastError(), "overlap_finish_kernel launch");
}

void launch_fold(double* out, const double* comp, int64_t n, void* stream) {
  if (n <= 0) return;
  int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  fold_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(out, comp, n);
  check(cudaGetLastError(), "fold_kernel launch");
}

void launch_prob(const double* amps, int64_t n, double scale, double* probs, void* stream) {
  if (n <= 0) return;
  int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
  prob_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(amps, n, scale, probs);
  check(cudaGetLastError(), "prob_kernel launch");
}

// Load every kernel of this library into the current device's context now
// (CUDA loads modules lazily, on a kernel's first launch or query), so that
// later calls - the fixed-scratch call in particular - load no code and
// allocate no device memory for it.
void preload_kernels() {
  cudaFuncAttributes a;
  const void* ks[] = {
      (const void*)pass_kernel<1, false>, (const void*)pass_kernel<2, false>, (const void*)pass_kernel<3, false>,
      (const void*)pass_kernel<4, false>, (const void*)pass_kernel<5, false>, (const void*)pass_kernel<1, true>,
      (const void*)pass_kernel<2, true>,  (const void*)pass_kernel<3, true>,  (const void*)pass_kernel<4, true>,
      (const void*)pass_kernel<5, true>,  (const void*)gather_kernel<0, false>, (const void*)gather_kernel<1, false>,
      (const void*)gather_kernel<2, false>, (const void*)gather_kernel<3, false>, (const void*)gather_kernel<4, false>,
      (const void*)gather_kernel<0, true>, (const void*)gather_kernel<1, true>,  (const void*)gather_kernel<2, true>,
      (const void*)gather_kernel<3, true>, (const void*)gather_kernel<4, true>,
      (const void*)frugal_accept_kernel,  (const void*)block_mark_kernel,     (const void*)block_count_kernel,
      (const void*)block_rank_kernel,     (const void*)zero_kernel,           (const void*)fold_kernel,
      (const void*)prob_kernel,           (const void*)overlap_kernel,        (const void*)overlap_finish_kernel};
  for (const void* k : ks) check(cudaFuncGetAttributes(&a, k), "cudaFuncGetAttributes (preload)");
  (void)num_sms();
}

}  // namespace sf
