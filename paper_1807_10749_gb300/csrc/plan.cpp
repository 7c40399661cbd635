// Planner: cut, cross-gate decompositions, path-tree levels, per-half op
// lists, and the fused pass / register-stage programs the kernels run.
//
// Paper correspondence:
//   cut selection ........... Section 8 (one straight cut, minimise the larger
//                             block, then the number of cross gates)
//   cross-gate terms ........ Eq. 1 (CZ), Eq. 4way and the operator-Schmidt
//                             decomposition (Sections 3 and 7)
//   path tree levels ........ Section 2 (prefix/suffix split with checkpoints)
//   zero-block skipping ..... Section 2 (projections leave blocks of zeros)
//   gate clustering, bitmask
//   diagonal passes, slices . Section 2 (clusters by kind; parity/popcount and
//                             mod-8 arithmetic for diagonal gates; cache-sized
//                             slices)
#include <algorithm>
#include <array>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>
#include <set>

#include "sf_internal.h"

namespace sf {

namespace {

const double kS2 = std::sqrt(0.5);

bool near(cd a, cd b, double tol = 1e-14) { return std::abs(a - b) <= tol; }

// e^{i pi w / 4} for w in 0..7
cd omega(int w) {
  static const double r = std::sqrt(0.5);
  static const cd t[8] = {cd(1, 0), cd(r, r), cd(0, 1), cd(-r, r),
                          cd(-1, 0), cd(-r, -r), cd(0, -1), cd(r, -r)};
  return t[((w % 8) + 8) % 8];
}

// If z is a power of e^{i pi/4} return its exponent, else -1.
int omega_exp(cd z) {
  for (int w = 0; w < 8; w++)
    if (near(z, omega(w), 1e-15)) return w;
  return -1;
}

void mul2(const cd* a, const cd* b, cd* out) {  // out = a * b (2x2)
  cd r[4];
  r[0] = a[0] * b[0] + a[1] * b[2];
  r[1] = a[0] * b[1] + a[1] * b[3];
  r[2] = a[2] * b[0] + a[3] * b[2];
  r[3] = a[2] * b[1] + a[3] * b[3];
  for (int i = 0; i < 4; i++) out[i] = r[i];
}

// ----------------------------------------------------------- cut selection
uint64_t auto_cut(const Circuit& c) {
  uint64_t best = 0;
  long best_big = 1 << 30, best_x = 1 << 30;
  auto consider = [&](uint64_t mask) {
    int nb = __builtin_popcountll(mask);
    int big = std::max(nb, c.n - nb);
    long x = 0;
    for (auto& g : c.gates)
      if (g.nq() == 2 && (((mask >> g.q0) ^ (mask >> g.q1)) & 1)) x++;
    if (big < best_big || (big == best_big && x < best_x)) {
      best = mask;
      best_big = big;
      best_x = x;
    }
  };
  for (int cc = 1; cc < c.cols; cc++) {
    uint64_t m = 0;
    for (int r = 0; r < c.rows; r++)
      for (int k = cc; k < c.cols; k++) m |= 1ull << (r * c.cols + k);
    consider(m);
  }
  for (int rr = 1; rr < c.rows; rr++) {
    uint64_t m = 0;
    for (int r = rr; r < c.rows; r++)
      for (int k = 0; k < c.cols; k++) m |= 1ull << (r * c.cols + k);
    consider(m);
  }
  if (!best) fail(SF_EINVAL, "no straight cut exists for a 1-qubit grid");
  return best;
}

// ---------------------------------------------------------- decompositions
// proj_on_b: for CZ, Eq. 1 with the halves' roles exchanged (CZ is
// symmetric): CZ = I (x) P0 + Z (x) P1, the projector on the half-B qubit.
void decompose(const Gate& g, bool q0_on_a, int decomposition, bool proj_on_b, CrossGate& x) {
  const cd I(0, 1);
  cd U[16];
  for (int i = 0; i < 16; i++) U[i] = g.m[i];
  if (!q0_on_a) {  // SWAP U SWAP: A-side qubit becomes the high basis bit
    const int sw[4] = {0, 2, 1, 3};
    cd V[16];
    for (int r = 0; r < 4; r++)
      for (int c = 0; c < 4; c++) V[4 * r + c] = U[4 * sw[r] + sw[c]];
    for (int i = 0; i < 16; i++) U[i] = V[i];
  }
  std::vector<std::pair<std::array<cd, 4>, std::array<cd, 4>>> terms;
  if (g.kind == SF_CZ && !proj_on_b) {
    // Eq. 1: CZ = P0 (x) I + P1 (x) Z
    terms.push_back({{1, 0, 0, 0}, {1, 0, 0, 1}});
    terms.push_back({{0, 0, 0, 1}, {1, 0, 0, -1}});
  } else if (g.kind == SF_CZ) {
    // Eq. 1 mirrored: CZ = I (x) P0 + Z (x) P1
    terms.push_back({{1, 0, 0, 1}, {1, 0, 0, 0}});
    terms.push_back({{1, 0, 0, -1}, {0, 0, 0, 1}});
  } else if (decomposition == SF_DEC_BLOCK4) {
    // Eq. 4way: P0 (x) U00 + P1 (x) U11 + |0><1| (x) U01 + |1><0| (x) U10
    auto blk = [&](int i, int j) {
      return std::array<cd, 4>{U[4 * (2 * i) + 2 * j], U[4 * (2 * i) + 2 * j + 1],
                               U[4 * (2 * i + 1) + 2 * j], U[4 * (2 * i + 1) + 2 * j + 1]};
    };
    terms.push_back({{1, 0, 0, 0}, blk(0, 0)});
    terms.push_back({{0, 0, 0, 1}, blk(1, 1)});
    terms.push_back({{0, 1, 0, 0}, blk(0, 1)});
    terms.push_back({{0, 0, 1, 0}, blk(1, 0)});
  } else {
    // operator-Schmidt: R[(a a'), (b b')] = U[(a b), (a' b')] = sum_k s_k u_k v_k^H
    cd R[16], Us[16], V[16];
    double s[4];
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int ap = 0; ap < 2; ap++)
          for (int bp = 0; bp < 2; bp++) R[4 * (2 * a + ap) + (2 * b + bp)] = U[4 * (2 * a + b) + (2 * ap + bp)];
    svd4(R, Us, s, V);
    for (int k = 0; k < 4; k++) {
      if (s[k] < 1e-14) continue;
      std::array<cd, 4> A, B;
      for (int i = 0; i < 4; i++) {
        A[i] = Us[4 * i + k];
        B[i] = s[k] * std::conj(V[4 * i + k]);
      }
      for (int i = 0; i < 4; i++)
        if (std::abs(A[i]) > 1e-12) {
          cd ph = A[i] / std::abs(A[i]);
          for (auto& v : A) v /= ph;
          for (auto& v : B) v *= ph;
          break;
        }
      terms.push_back({A, B});
    }
  }
  int r = 1;
  while (r < (int)terms.size()) r *= 2;
  while ((int)terms.size() < r) terms.push_back({{0, 0, 0, 0}, {0, 0, 0, 0}});
  x.nterm = r;
  x.bits = 0;
  while ((1 << x.bits) < r) x.bits++;
  for (int d = 0; d < r; d++)
    for (int i = 0; i < 4; i++) {
      x.fa[d][i] = terms[d].first[i];
      x.fb[d][i] = terms[d].second[i];
    }
  (void)I;
}

// Classify a per-digit factor set into a half op (PROJ / XPHASE / XSEL).
HOp cross_op(int pos, int xi, int nterm, const cd f[4][4]) {
  HOp o;
  o.p0 = pos;
  o.xi = xi;
  o.nterm = nterm;
  bool proj = true, phase = true;
  for (int d = 0; d < nterm; d++) {
    const cd* m = f[d];
    bool is_p0 = near(m[0], 1) && near(m[1], 0) && near(m[2], 0) && near(m[3], 0);
    bool is_p1 = near(m[0], 0) && near(m[1], 0) && near(m[2], 0) && near(m[3], 1);
    if (is_p0) o.pv[d] = 0;
    else if (is_p1) o.pv[d] = 1;
    else proj = false;
    bool dg = near(m[1], 0) && near(m[2], 0) && near(m[0], 1) && omega_exp(m[3]) >= 0;
    if (dg) o.tw[d] = omega_exp(m[3]);
    else phase = false;
    for (int i = 0; i < 4; i++) o.tm[d][i] = m[i];
  }
  o.kind = proj ? H_PROJ : (phase ? H_XPHASE : H_XSEL);
  return o;
}

// Half op of a local gate (positions already mapped).
HOp local_op(const Gate& g, int p0, int p1, cd& global) {
  HOp o;
  o.p0 = p0;
  o.p1 = p1;
  const cd* m = g.m;
  if (g.nq() == 2) {
    if (g.kind == SF_CZ) {
      o.kind = H_CZ;
    } else {
      o.kind = H_G2;
      for (int i = 0; i < 16; i++) o.m[i] = m[i];
    }
    return o;
  }
  for (int i = 0; i < 4; i++) o.m[i] = m[i];
  if (g.kind == SF_H || g.kind == SF_X_HALF || g.kind == SF_Y_HALF) {
    o.kind = H_G1;
    o.fast = g.kind == SF_H ? DOP_H : (g.kind == SF_X_HALF ? DOP_XH : DOP_YH);
    o.scale_e = 1;  // H = M_H / sqrt2; X^1/2, Y^1/2 = e^{i pi/4} M / sqrt2
    return o;
  }
  bool diag = near(m[1], 0, 0) && near(m[2], 0, 0);
  if (diag) {
    // diag(a, b) = a * diag(1, b/a); a power of e^{i pi/4} ratio -> mod-8 phase
    if (std::abs(m[0]) > 0) {
      cd ratio = m[3] / m[0];
      int w = omega_exp(ratio);
      if (w >= 0 && std::abs(std::abs(m[0]) - 1.0) < 1e-15) {
        o.kind = H_PHASE1;
        o.w = w;
        global *= m[0];
        return o;
      }
    }
    o.kind = H_DMUL;
    o.m[0] = m[0];
    o.m[1] = m[3];
    return o;
  }
  o.kind = H_G1;
  return o;
}

uint64_t op_posmask(const HOp& o) {
  uint64_t b = 1ull << o.p0;
  if (o.p1 >= 0) b |= 1ull << o.p1;
  return b;
}

// ------------------------------------------------------- program emission
struct Emitter {
  PassPlan& pp;
  explicit Emitter(PassPlan& p) : pp(p) {}
  int add_mats(const cd* m, int count) {  // returns float2 index
    int at = (int)pp.mats.size() / 2;
    for (int i = 0; i < count; i++) {
      pp.mats.push_back((float)m[i].real());
      pp.mats.push_back((float)m[i].imag());
    }
    return at;
  }
};

// Collected diagonal gates of one phase group before it is laid out for
// its stage.
struct GroupAcc {
  int w[32] = {0};
  std::vector<std::pair<int, int>> cz;  // (a < b), repeated pairs cancel
  struct Sel {
    int pos, xi;
    int w[4];
  };
  std::vector<Sel> sel;
};

// Lay a collected group out for a stage whose register bit j sits at global
// position gr[j]. Returns false if it needs more shift classes than fit.
bool finish_group(const GroupAcc& acc, const int* gr, int R, DevPhaseGroup& g) {
  std::memset(&g, 0, sizeof(g));
  uint32_t rmask = 0;
  for (int j = 0; j < R; j++) rmask |= 1u << gr[j];
  for (int p = 0; p < 32; p++) {
    int w = ((acc.w[p] % 8) + 8) % 8;
    if ((rmask >> p) & 1u) {
      for (int j = 0; j < R && j < MAX_R; j++)
        if (gr[j] == p) g.wstat[j] = (uint8_t)w;
      continue;
    }
    if (w & 1) g.m1 |= 1u << p;
    if (w & 2) g.m2 |= 1u << p;
    if (w & 4) g.m4 |= 1u << p;
  }
  auto reg = [&](int p) {
    for (int j = 0; j < R; j++)
      if (gr[j] == p) return j;
    return -1;
  };
  for (auto& pr : acc.cz) {
    const int a = pr.first, b = pr.second;
    const int ja = reg(a), jb = reg(b);
    if (ja >= 0 && jb >= 0) {
      g.czq[ja] |= (uint8_t)(1u << jb);
      g.czq[jb] |= (uint8_t)(1u << ja);
    } else if (ja >= 0) {
      g.czf[ja] |= 1u << b;
    } else if (jb >= 0) {
      g.czf[jb] |= 1u << a;
    } else {
      const int sh = b - a;
      int c = 0;
      while (c < g.nsh && g.sh[c] != sh) c++;
      if (c == g.nsh) {
        if (g.nsh >= MAX_SHIFTS) return false;
        g.sh[g.nsh++] = (uint8_t)sh;
      }
      g.shm[c] |= 1u << a;
    }
  }
  if ((int)acc.sel.size() > MAX_SEL_PER_GROUP) return false;
  g.nsel = (int)acc.sel.size();
  for (size_t i = 0; i < acc.sel.size(); i++) {
    g.sel[i].pos = (int8_t)acc.sel[i].pos;
    g.sel[i].xi = (int8_t)acc.sel[i].xi;
    g.sel[i].reg = (int8_t)reg(acc.sel[i].pos);
    for (int d = 0; d < 4; d++) g.sel[i].w[d] = (uint8_t)acc.sel[i].w[d];
  }
  return true;
}

// Order a stage's ops with as few phase groups as possible. Diagonal ops
// commute with each other and with every op on other qubits, so each may sit
// anywhere between the last earlier and the first later non-diagonal op that
// shares a qubit with it; a greedy point cover of those intervals (by right
// end) picks the fewest slots, and all diagonal ops of a slot form one group.
std::vector<const HOp*> merge_diagonals(const std::vector<const HOp*>& ops) {
  std::vector<const HOp*> nd;
  std::vector<int> nd_idx;
  for (size_t i = 0; i < ops.size(); i++)
    if (!ops[i]->diag()) {
      nd.push_back(ops[i]);
      nd_idx.push_back((int)i);
    }
  const int N = (int)nd.size();
  struct Iv {
    int lo, hi;
    const HOp* op;
  };
  std::vector<Iv> iv;
  for (size_t i = 0; i < ops.size(); i++) {
    if (!ops[i]->diag()) continue;
    const uint64_t b = op_posmask(*ops[i]);
    int lo = 0, hi = N;
    for (int j = 0; j < N; j++) {
      if (!(op_posmask(*nd[j]) & b)) continue;
      if (nd_idx[j] < (int)i) lo = j + 1;
      else {
        hi = j;
        break;
      }
    }
    iv.push_back({lo, hi, ops[i]});
  }
  std::vector<int> slot_of(iv.size(), -1);
  std::vector<size_t> order(iv.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return iv[a].hi < iv[b].hi; });
  int chosen = -1;
  for (size_t t : order) {
    if (chosen >= iv[t].lo && chosen <= iv[t].hi) {
      slot_of[t] = chosen;
      continue;
    }
    chosen = iv[t].hi;
    slot_of[t] = chosen;
  }
  std::vector<const HOp*> out;
  for (int sl = 0; sl <= N; sl++) {
    for (size_t t = 0; t < iv.size(); t++)  // diagonal ops of this slot, original order
      if (slot_of[t] == sl) out.push_back(iv[t].op);
    if (sl < N) out.push_back(nd[sl]);
  }
  return out;
}

bool emit_stage_ops(const std::vector<const HOp*>& ops_in, const DevStage& st, const int* local_of,
                    const int8_t* gpos, PassPlan& pp) {
  const std::vector<const HOp*> ops = merge_diagonals(ops_in);
  Emitter em(pp);
  auto reg_of = [&](int pos) {
    int lb = local_of[pos];
    for (int j = 0; j < st.r; j++)
      if (st.rbit[j] == lb) return j;
    return -1;
  };
  int gr[MAX_R];
  for (int j = 0; j < st.r; j++) gr[j] = gpos[st.rbit[j]];
  int cur_group = -1;
  GroupAcc acc;
  bool ok = true;
  auto close_group = [&]() {
    if (cur_group < 0) return;
    if (!finish_group(acc, gr, st.r, pp.phases[cur_group])) ok = false;
    acc = GroupAcc();
    cur_group = -1;
  };
  auto open_group = [&]() {
    if (cur_group >= 0) return true;
    if ((int)pp.phases.size() >= MAX_PHASE_GROUPS) return false;
    DevPhaseGroup g;
    std::memset(&g, 0, sizeof(g));
    pp.phases.push_back(g);
    cur_group = (int)pp.phases.size() - 1;
    DevOp d{DOP_PHASE, 0, 0, -1, cur_group};
    pp.ops.push_back(d);
    return true;
  };
  for (const HOp* o : ops) {
    if (o->kind == H_CZ || o->kind == H_PHASE1 || o->kind == H_XPHASE) {
      if (!open_group()) return false;
      if (o->kind == H_PHASE1) {
        acc.w[o->p0] += o->w;
      } else if (o->kind == H_CZ) {
        const int a = std::min(o->p0, o->p1), b = std::max(o->p0, o->p1);
        auto it = std::find(acc.cz.begin(), acc.cz.end(), std::make_pair(a, b));
        if (it != acc.cz.end()) acc.cz.erase(it);  // CZ^2 = I
        else acc.cz.push_back({a, b});
      } else {
        if ((int)acc.sel.size() >= MAX_SEL_PER_GROUP) {
          close_group();
          if (!open_group()) return false;
        }
        GroupAcc::Sel sl;
        sl.pos = o->p0;
        sl.xi = o->xi;
        for (int d = 0; d < 4; d++) sl.w[d] = d < o->nterm ? o->tw[d] : 0;
        acc.sel.push_back(sl);
      }
      continue;
    }
    close_group();
    DevOp d{0, 0, 0, -1, 0};
    switch (o->kind) {
      case H_G1:
        d.a = reg_of(o->p0);
        if (o->fast) {
          d.code = o->fast;
        } else {
          d.code = DOP_G1;
          d.arg = em.add_mats(o->m, 4);
        }
        break;
      case H_XSEL: {
        d.code = DOP_G1SEL;
        d.a = reg_of(o->p0);
        d.xi = o->xi;
        cd buf[16];
        for (int t = 0; t < 4; t++)
          for (int i = 0; i < 4; i++) buf[4 * t + i] = t < o->nterm ? o->tm[t][i] : cd(0);
        d.arg = em.add_mats(buf, 16);
        break;
      }
      case H_G2:
        d.code = DOP_G2;
        d.a = reg_of(o->p0);
        d.b = reg_of(o->p1);
        d.arg = em.add_mats(o->m, 16);
        break;
      case H_DMUL:
        d.code = DOP_DMUL;
        d.a = o->p0;
        d.arg = em.add_mats(o->m, 2);
        break;
      default:
        fail(SF_EINVAL, "internal: unexpected op kind in stage");
    }
    if ((d.code == DOP_G1 || d.code == DOP_G1SEL || d.code == DOP_G2 || d.code <= DOP_YH) && d.a < 0)
      fail(SF_EINVAL, "internal: op bit not in register block");
    if (d.code == DOP_G2 && d.b < 0) fail(SF_EINVAL, "internal: op bit not in register block");
    pp.ops.push_back(d);
  }
  close_group();
  return ok && (int)pp.mats.size() <= 2 * MAX_MATS && (int)pp.ops.size() <= MAX_OPS;
}

DevPin to_dev(const Pin& p) {
  DevPin d;
  d.pos = (int8_t)p.pos;
  d.xi = (int8_t)p.xi;
  for (int i = 0; i < 4; i++) d.v[i] = (uint8_t)p.v[i];
  return d;
}

// Plan one segment of one half into passes. ops are consumed in order.
void plan_segment(int m, const std::vector<HOp>& seg_ops, std::vector<Pin> pins, bool gen_input,
                  int tile_bits, int fuse_bits, int run_bits, SegmentPlan& out) {
  std::vector<const HOp*> rem;
  for (auto& o : seg_ops) {
    if (o.kind == H_PROJ) {
      Pin p;
      p.pos = o.p0;
      p.xi = o.xi;
      for (int d = 0; d < 4; d++) p.v[d] = o.pv[d];
      pins.push_back(p);
    } else {
      rem.push_back(&o);
    }
  }
  const int k = std::min(tile_bits, m);
  const int L = std::max(1, std::min(run_bits, k));
  // register bits: at most the fusion width, at least enough that a tile
  // needs no more than 512 threads, and leave >= 2^min(5,k-1) threads per tile
  int R = std::max(1, std::min(fuse_bits, k - std::min(5, k - 1)));
  R = std::min(MAX_R, std::max(R, k - 9));
  int res = 0;
  cd sigma = 1.0;
  bool first = true;
  out.passes.clear();
  out.n_stages = 0;
  const uint64_t low = (L >= 64) ? ~0ull : ((1ull << L) - 1);
  // Ops that run in one pass whose active set is S: in order, an op runs if
  // no earlier op on its bits was held back and its non-diagonal bits are in S.
  auto take_fixed = [&](const std::vector<const HOp*>& ops, uint64_t S, int cap,
                        std::vector<const HOp*>* taken, std::vector<const HOp*>* rest) {
    uint64_t blocked = 0;
    int n = 0;
    for (const HOp* o : ops) {
      const uint64_t b = op_posmask(*o);
      if (n >= cap || (b & blocked) || (!o->diag() && (b & ~S))) {
        blocked |= b;
        if (rest) rest->push_back(o);
        continue;
      }
      n++;
      if (taken) taken->push_back(o);
    }
    return n;
  };
  // First-come active set: bits join as the ops that need them are reached.
  auto greedy_S = [&](const std::vector<const HOp*>& ops) {
    uint64_t S = low, blocked = 0;
    for (const HOp* o : ops) {
      const uint64_t b = op_posmask(*o);
      if (b & blocked) {
        blocked |= b;
        continue;
      }
      if (o->diag()) continue;
      const uint64_t need = b & ~S;
      if (__builtin_popcountll(S | need) <= k) S |= need;
      else blocked |= b;
    }
    return S;
  };
  auto greedy_passes = [&](std::vector<const HOp*> ops) {
    int n = 0;
    while (!ops.empty() && n < 64) {
      std::vector<const HOp*> rest;
      take_fixed(ops, greedy_S(ops), MAX_OPS, nullptr, &rest);
      if (rest.size() == ops.size()) return 1000;  // no progress (cannot happen)
      ops.swap(rest);
      n++;
    }
    return n;
  };
  // Active set for the next pass: the first-come set, or one built from an
  // ordering of the bits the remaining non-diagonal ops need, whichever
  // leaves the fewest passes for the rest of the segment.
  auto choose_S = [&](const std::vector<const HOp*>& ops) {
    std::vector<uint64_t> cands;
    cands.push_back(greedy_S(ops));
    std::vector<int> first(m, 1 << 30), last(m, -1), cnt(m, 0);
    for (size_t i = 0; i < ops.size(); i++) {
      if (ops[i]->diag()) continue;
      for (int p : {ops[i]->p0, ops[i]->p1}) {
        if (p < 0 || ((low >> p) & 1)) continue;
        first[p] = std::min(first[p], (int)i);
        last[p] = std::max(last[p], (int)i);
        cnt[p]++;
      }
    }
    std::vector<int> bits;
    for (int p = 0; p < m; p++)
      if (cnt[p]) bits.push_back(p);
    auto from_order = [&](const std::vector<int>& order) {
      uint64_t S = low;
      for (int p : order)
        if (__builtin_popcountll(S) < k) S |= 1ull << p;
      return S;
    };
    std::vector<int> o = bits;
    std::sort(o.begin(), o.end(), [&](int a, int b) { return first[a] < first[b]; });
    cands.push_back(from_order(o));
    std::sort(o.begin(), o.end(), [&](int a, int b) { return last[a] < last[b]; });
    cands.push_back(from_order(o));
    std::sort(o.begin(), o.end(), [&](int a, int b) { return cnt[a] > cnt[b] || (cnt[a] == cnt[b] && first[a] < first[b]); });
    cands.push_back(from_order(o));
    std::sort(o.begin(), o.end());
    cands.push_back(from_order(o));
    std::reverse(o.begin(), o.end());
    cands.push_back(from_order(o));
    uint64_t rng = 0x9E3779B97F4A7C15ull ^ (uint64_t)ops.size();
    for (int t = 0; t < 24; t++) {
      std::vector<int> r = bits;
      for (size_t i = r.size(); i > 1; i--) {
        rng ^= rng << 13;
        rng ^= rng >> 7;
        rng ^= rng << 17;
        std::swap(r[i - 1], r[rng % i]);
      }
      cands.push_back(from_order(r));
    }
    uint64_t best = cands[0];
    int best_passes = 1 << 30, best_taken = -1;
    for (uint64_t S : cands) {
      std::vector<const HOp*> rest;
      const int n = take_fixed(ops, S, MAX_OPS, nullptr, &rest);
      if (n == 0 && !ops.empty()) continue;
      const int passes = 1 + greedy_passes(rest);
      if (passes < best_passes || (passes == best_passes && n > best_taken)) {
        best = S;
        best_passes = passes;
        best_taken = n;
      }
    }
    return best;
  };
  while (first || !rem.empty()) {
    int cap = MAX_OPS;
    PassPlan pp;
    std::vector<const HOp*> taken, deferred;
    const uint64_t S_choice = rem.empty() ? low : choose_S(rem);
    while (true) {
      pp = PassPlan();
      taken.clear();
      deferred.clear();
      uint64_t S = S_choice;
      take_fixed(rem, S, cap, &taken, &deferred);
      // pins removed by this pass: positions with a non-diagonal op
      uint64_t nd = 0;
      for (const HOp* o : taken)
        if (!o->diag()) nd |= op_posmask(*o);
      uint64_t pinned = 0;
      for (auto& p : pins) pinned |= 1ull << p.pos;
      // fill the active set with the lowest unpinned positions
      for (int p = 0; p < m && __builtin_popcountll(S) < k; p++)
        if (!((S >> p) & 1) && !((pinned >> p) & 1)) S |= 1ull << p;
      for (int p = 0; p < m && __builtin_popcountll(S) < k; p++)
        if (!((S >> p) & 1)) S |= 1ull << p;
      DevPass& dp = pp.dev;
      std::memset(&dp, 0, sizeof(dp));
      dp.m = m;
      dp.k = k;
      dp.L = L;
      dp.R = R;
      int local_of[64];
      for (int p = 0; p < 64; p++) local_of[p] = -1;
      int j = 0;
      for (int p = 0; p < m; p++)
        if ((S >> p) & 1) {
          dp.gpos[j] = (int8_t)p;
          local_of[p] = j++;
        }
      dp.n_free = 0;
      for (int p = 0; p < m; p++)
        if (!((S >> p) & 1) && !((pinned >> p) & 1)) dp.freepos[dp.n_free++] = (int8_t)p;
      if ((int)pins.size() > MAX_PINS) fail(SF_EUNSUPPORTED, "too many pending projections");
      dp.n_pin_in = (int)pins.size();
      for (size_t i = 0; i < pins.size(); i++) dp.pin_in[i] = to_dev(pins[i]);
      std::vector<Pin> pout;
      for (auto& p : pins)
        if (!((nd >> p.pos) & 1)) pout.push_back(p);
      dp.n_pin_out = (int)pout.size();
      for (size_t i = 0; i < pout.size(); i++) dp.pin_out[i] = to_dev(pout[i]);
      dp.gen_input = (first && gen_input) ? 1 : 0;
      // scale bookkeeping (exact powers of two applied in the pass)
      int e = 0, nxy = 0;
      for (const HOp* o : taken)
        if (o->kind == H_G1 && o->fast) {
          e += o->scale_e;
          if (o->fast != DOP_H) nxy++;
        }
      int t = res + e;
      int shift = t / 2;
      dp.post_scale = std::ldexp(1.0f, -shift);
      // register stages
      std::vector<const HOp*> srem = taken;
      bool ok = true;
      while (!srem.empty()) {
        uint64_t Sreg = 0, sblocked = 0;
        std::vector<const HOp*> st_ops, st_def;
        for (const HOp* o : srem) {
          uint64_t b = op_posmask(*o);
          if (b & sblocked) {
            sblocked |= b;
            st_def.push_back(o);
            continue;
          }
          if (o->diag()) {
            st_ops.push_back(o);
            continue;
          }
          uint64_t lb = 1ull << local_of[o->p0];
          if (o->p1 >= 0) lb |= 1ull << local_of[o->p1];
          uint64_t need = lb & ~Sreg;
          if (__builtin_popcountll(Sreg | need) <= R) {
            Sreg |= need;
            st_ops.push_back(o);
          } else {
            sblocked |= b;
            st_def.push_back(o);
          }
        }
        for (int lb = k - 1; lb >= 0 && __builtin_popcountll(Sreg) < R; lb--)
          if (!((Sreg >> lb) & 1)) Sreg |= 1ull << lb;
        DevStage st;
        std::memset(&st, 0, sizeof(st));
        st.r = R;
        int q = 0;
        for (int lb = 0; lb < k; lb++)
          if ((Sreg >> lb) & 1) st.rbit[q++] = (int8_t)lb;
        {
          int t = 0;
          for (int lb = 0; lb < k; lb++)
            if (!((Sreg >> lb) & 1)) {
              st.tpos[t] = (int8_t)lb;
              st.tg[t] = dp.gpos[lb];
              t++;
            }
          if (t > 9) fail(SF_EINVAL, "internal: more than 512 threads per tile");
        }
        st.op_begin = (int)pp.ops.size();
        if (!emit_stage_ops(st_ops, st, local_of, dp.gpos, pp)) {
          ok = false;
          break;
        }
        st.op_end = (int)pp.ops.size();
        pp.stages.push_back(st);
        if ((int)pp.stages.size() > MAX_STAGES) {
          ok = false;
          break;
        }
        srem = st_def;
      }
      if (ok) {
        res = t - 2 * shift;
        sigma *= std::pow(2.0, -0.5 * e) / std::ldexp(1.0, -shift) * std::polar(1.0, M_PI / 4 * (nxy % 8));
        break;
      }
      if (cap <= 1) fail(SF_EUNSUPPORTED, "a single gate exceeds the pass program limits");
      cap = std::max(1, (int)taken.size() / 2);
    }
    pp.dev.n_stages = (int)pp.stages.size();
    out.n_stages += pp.dev.n_stages;
    out.passes.push_back(std::move(pp));
    rem = deferred;
    // pins after this pass
    uint64_t nd = 0;
    for (const HOp* o : taken)
      if (!o->diag()) nd |= op_posmask(*o);
    std::vector<Pin> np;
    for (auto& p : pins)
      if (!((nd >> p.pos) & 1)) np.push_back(p);
    pins = np;
    first = false;
  }
  // the residual sqrt2 factor stays in sigma; stored values carry it
  out.pins_out = pins;
  out.scale = sigma;
  (void)res;
}

}  // namespace

// A gate whose matrix is diagonal commutes with the diagonal branch
// operators (Eq. 1's projectors and Z factors).
bool gate_diag(const Gate& g) {
  const int d = g.nq() == 2 ? 4 : 2;
  for (int r = 0; r < d; r++)
    for (int q = 0; q < d; q++)
      if (r != q && !near(g.m[r * d + q], 0, 0)) return false;
  return true;
}

// Light cones of the branch levels. At level l each cut gate is replaced,
// on each half, by one of its term factors on the cut qubit: a projector or
// Z for Eq. 1, general 2x2 factors for the Schmidt and four-block forms. A
// later gate of that half commutes with the factors unless it is causally
// after them: the cone of level l starts at each cut qubit, with its first
// non-diagonal gate after the level (at the level itself when the factors
// are not diagonal), and takes in every qubit that a later gate couples to a
// qubit already in it. A gate in no cone of a deeper level than l can run
// before that level's branching, in the node every child of it shares. The
// result: per gate, the deepest level (1-based) whose cone holds it, 0 for
// none; cross gates are not scheduled this way.
template <class InB>
std::vector<int> cone_depths(const Circuit& c, const Plan& P, const InB& inB) {
  std::vector<int> depth(c.gates.size(), 0);
  std::vector<char> is_cross(c.gates.size(), 0);
  for (const auto& x : P.cross) is_cross[x.gate_index] = 1;
  for (size_t l = 0; l < P.levels.size(); l++) {
    const Level& L = P.levels[l];
    for (int side = 0; side < 2; side++) {
      std::vector<char> in(c.n, 0), cut(c.n, 0);
      for (int i = 0; i < L.n_cross; i++) {
        const CrossGate& x = P.cross[L.first_cross + i];
        const int q = side ? x.qb : x.qa;
        cut[q] = 1;
        for (int t = 0; t < x.nterm; t++) {
          const cd* f = side ? x.fb[t] : x.fa[t];
          if (!near(f[1], 0, 0) || !near(f[2], 0, 0)) in[q] = 1;
        }
      }
      for (size_t i = 0; i < c.gates.size(); i++) {
        const Gate& g = c.gates[i];
        if (g.cycle < L.cycle || is_cross[i] || (int)inB(g.q0) != side) continue;
        bool hit = in[g.q0] || (g.nq() == 2 && in[g.q1]);
        if (!hit && (cut[g.q0] || (g.nq() == 2 && cut[g.q1])) && !gate_diag(g)) hit = true;
        if (!hit) continue;
        in[g.q0] = 1;
        if (g.nq() == 2) in[g.q1] = 1;
        depth[i] = std::max(depth[i], (int)l + 1);
      }
    }
  }
  return depth;
}

// ------------------------------------------------------------ plan create
// Plan a segment. With an automatic tile size (tile_bits option 0) the
// candidates are 2^12 and 2^13 amplitudes, with an automatic run width
// (run_bits option 0) widths 4 and 3; the program with the least estimated
// time wins: algorithmic bytes divided by the fraction of HBM bandwidth the
// pass kernel reaches at that tile size on GB300 (2^12: two CTAs per SM,
// ~0.75; 2^13: one CTA per SM, ~0.64; measured on the 7x8 workload). Ties go
// to the wider runs (longer contiguous copies).
void plan_segment_auto(int m, const std::vector<HOp>& ops, const std::vector<Pin>& pins, bool first, const Plan& P,
                       bool auto_tiles, bool auto_runs, SegmentPlan& out) {
  std::vector<int> tiles = auto_tiles ? std::vector<int>{12, 13} : std::vector<int>{P.tile_bits};
  std::vector<int> runs = auto_runs ? std::vector<int>{4, 3} : std::vector<int>{P.run_bits};
  SegmentPlan best;
  double best_t = -1;
  for (int tb : tiles)
    for (int rb : runs) {
      SegmentPlan cand;
      plan_segment(m, ops, pins, first, tb, P.fuse_bits, rb, cand);
      const double eff = std::min(tb, m) >= 13 ? 0.64 : 0.75;
      const double t = segment_bytes(cand) / eff;
      if (best_t < 0 || t < best_t * (1 - 1e-9)) {
        best = std::move(cand);
        best_t = t;
      }
    }
  out = std::move(best);
}

Plan* plan_create(const Circuit& c, const sf_plan_opts& o) {
  Plan* P = new Plan();
  try {
    P->opts = o;
    P->circ = c;
    const int n = c.n;
    uint64_t all = (n == 64) ? ~0ull : ((1ull << n) - 1);
    uint64_t bm = o.side_b_mask ? o.side_b_mask : auto_cut(c);
    if (bm & ~all) fail(SF_EINVAL, "side_b_mask has bits beyond the qubit count");
    if (bm == 0 || bm == all) fail(SF_EINVAL, "both halves must be non-empty");
    P->side_b_mask = bm;
    auto inB = [&](int q) { return (bm >> q) & 1; };
    int mB = __builtin_popcountll(bm), mA = n - mB;
    if (mA > 32 || mB > 32) fail(SF_EUNSUPPORTED, "a half of more than 32 qubits");
    if (mA < 1 || mB < 1) fail(SF_EINVAL, "empty half");
    // the pipelined pass kernel holds three tile buffers of 2^k complex64 in
    // shared memory, so k <= 13; with tile_bits 0 each segment takes k = 12
    // (96 KiB per CTA: two CTAs, i.e. two copy/compute pipelines, per SM) or
    // k = 13 (one CTA per SM, fewer passes), whichever is estimated faster
    P->tile_bits = o.tile_bits > 0 ? std::min(o.tile_bits, 13) : 12;
    P->fuse_bits = o.fuse_bits > 0 ? std::min(o.fuse_bits, MAX_R) : 5;
    P->run_bits = o.run_bits > 0 ? std::min(o.run_bits, 8) : 4;
    if (P->tile_bits < 6) P->tile_bits = 6;

    // cross gates in time order (cycle, lower qubit, higher qubit)
    std::vector<int> xg;
    for (size_t i = 0; i < c.gates.size(); i++) {
      const Gate& g = c.gates[i];
      if (g.nq() == 2 && inB(g.q0) != inB(g.q1)) xg.push_back((int)i);
    }
    std::stable_sort(xg.begin(), xg.end(), [&](int a, int b) {
      const Gate &ga = c.gates[a], &gb = c.gates[b];
      if (ga.cycle != gb.cycle) return ga.cycle < gb.cycle;
      int la = std::min(ga.q0, ga.q1), lb = std::min(gb.q0, gb.q1);
      if (la != lb) return la < lb;
      return std::max(ga.q0, ga.q1) < std::max(gb.q0, gb.q1);
    });
    if ((int)xg.size() > MAX_CROSS) fail(SF_EUNSUPPORTED, "more than 64 cross gates");
    std::map<int, int> xindex;
    for (size_t i = 0; i < xg.size(); i++) {
      const Gate& g = c.gates[xg[i]];
      CrossGate x;
      x.gate_index = xg[i];
      x.cycle = g.cycle;
      bool q0a = !inB(g.q0);
      x.qa = q0a ? g.q0 : g.q1;
      x.qb = q0a ? g.q1 : g.q0;
      decompose(g, q0a, o.decomposition, o.projector_side == SF_PROJ_ALTERNATE && (i & 1), x);
      P->cross.push_back(x);
      xindex[xg[i]] = (int)i;
    }
    int total = 0;
    for (auto& x : P->cross) total += x.bits;
    if (total > 63) fail(SF_EUNSUPPORTED, "more than 63 path bits");
    P->path_bits = total;
    int sh = total;
    for (auto& x : P->cross) {
      sh -= x.bits;
      x.shift = sh;
    }
    // levels: cross gates of one cycle
    for (size_t i = 0; i < P->cross.size(); i++) {
      if (P->levels.empty() || P->levels.back().cycle != P->cross[i].cycle) {
        Level L;
        L.cycle = P->cross[i].cycle;
        L.first_cross = (int)i;
        L.n_cross = 0;
        L.bits = 0;
        P->levels.push_back(L);
      }
      Level& L = P->levels.back();
      L.n_cross++;
      L.bits += P->cross[i].bits;
      L.shift = P->cross[i].shift;
    }
    const int nL = (int)P->levels.size();
    P->xs = o.select_prefix_bits >= 0 ? std::min(o.select_prefix_bits, total) : std::max(0, total - 7);

    // layouts: the last level's cut qubits take the lowest positions
    for (int side = 0; side < 2; side++) {
      HalfPlan& H = side ? P->B : P->A;
      H.m = side ? mB : mA;
      H.pos_of.assign(n, -1);
      std::vector<int> order;
      if (nL > 0) {
        const Level& L = P->levels.back();
        for (int i = 0; i < L.n_cross; i++) {
          const CrossGate& x = P->cross[L.first_cross + i];
          order.push_back(side ? x.qb : x.qa);
        }
      }
      for (int q = 0; q < n; q++)
        if ((int)inB(q) == side && std::find(order.begin(), order.end(), q) == order.end())
          order.push_back(q);
      H.qubits = order;
      for (size_t p = 0; p < order.size(); p++) H.pos_of[order[p]] = (int)p;
      H.seg_ops.assign(nL + 1, {});
    }
    // segment of a gate. By cycles: the number of levels whose cycle <= gate
    // cycle (local gates of a level's cycle run after its cross gates). By
    // light cones (default): the deepest level whose cone holds the gate.
    const std::vector<int> cone = o.cycle_segments ? std::vector<int>() : cone_depths(c, *P, inB);
    std::vector<cd> seg_global(2 * (nL + 1), cd(1.0));
    for (size_t i = 0; i < c.gates.size(); i++) {
      const Gate& g = c.gates[i];
      int s = 0;
      while (s < nL && P->levels[s].cycle <= g.cycle) s++;
      if (!cone.empty() && !xindex.count((int)i)) s = cone[i];
      auto it = xindex.find((int)i);
      if (it != xindex.end()) {
        const CrossGate& x = P->cross[it->second];
        // s == level index + 1 for a cross gate
        P->A.seg_ops[s].push_back(cross_op(P->A.pos_of[x.qa], it->second, x.nterm, x.fa));
        P->B.seg_ops[s].push_back(cross_op(P->B.pos_of[x.qb], it->second, x.nterm, x.fb));
        continue;
      }
      int side = inB(g.q0);
      HalfPlan& H = side ? P->B : P->A;
      int p0 = H.pos_of[g.q0], p1 = g.nq() == 2 ? H.pos_of[g.q1] : -1;
      H.seg_ops[s].push_back(local_op(g, p0, p1, seg_global[2 * s + side]));
    }
    // cross ops first within their segment (they commute with the local
    // gates of the same cycle, which act on other qubits)
    for (int side = 0; side < 2; side++) {
      HalfPlan& H = side ? P->B : P->A;
      for (auto& ops : H.seg_ops)
        std::stable_partition(ops.begin(), ops.end(), [](const HOp& o) {
          return o.kind == H_PROJ || o.kind == H_XPHASE || o.kind == H_XSEL ? o.xi >= 0 : false;
        });
    }
    // root: absorb each qubit's leading H into the generated uniform state
    for (int side = 0; side < 2; side++) {
      HalfPlan& H = side ? P->B : P->A;
      H.root_pins.clear();
      int h = 0;
      auto& ops0 = H.seg_ops[0];
      std::vector<bool> erase(ops0.size(), false);
      for (int p = 0; p < H.m; p++) {
        bool absorbed = false;
        for (size_t i = 0; i < ops0.size(); i++) {
          const HOp& op = ops0[i];
          if (op.p0 == p || op.p1 == p) {
            if (op.kind == H_G1 && op.fast == DOP_H) {
              erase[i] = true;
              absorbed = true;
              h++;
            }
            break;
          }
        }
        if (!absorbed) {
          Pin pin;
          pin.pos = p;
          pin.xi = -1;
          pin.v[0] = pin.v[1] = pin.v[2] = pin.v[3] = 0;
          H.root_pins.push_back(pin);
        }
      }
      std::vector<HOp> kept;
      for (size_t i = 0; i < ops0.size(); i++)
        if (!erase[i]) kept.push_back(ops0[i]);
      ops0 = kept;
      H.root_scale = std::pow(2.0, -0.5 * h);
    }
    // deferral of the last level into the gather
    P->deferred = false;
    if (nL > 0 && o.defer_last_level && o.exec_mode != SF_EXEC_PLAIN) {
      const Level& L = P->levels.back();
      bool ok = L.n_cross <= MAX_DEFER;
      int nterm = ok ? P->cross[L.first_cross].nterm : 0;
      for (int i = 0; ok && i < L.n_cross; i++)
        if (P->cross[L.first_cross + i].nterm != nterm || nterm > 4) ok = false;
      std::vector<std::vector<HOp>> kept(2);
      cd Vm[2][MAX_DEFER][4];
      for (int side = 0; side < 2 && ok; side++) {
        HalfPlan& H = side ? P->B : P->A;
        const auto& ops = H.seg_ops[nL];
        std::vector<bool> drop(ops.size(), false);
        for (int i = 0; i < L.n_cross && ok; i++) {
          const CrossGate& x = P->cross[L.first_cross + i];
          int pos = H.pos_of[side ? x.qb : x.qa];
          cd V[4] = {1, 0, 0, 1};
          int phase = 0;  // 0: before, 1: diagonal run, 2: one-qubit tail
          bool factor_diag = true;
          for (int d = 0; d < x.nterm; d++) {
            const cd* f = side ? x.fb[d] : x.fa[d];
            if (!near(f[1], 0) || !near(f[2], 0)) factor_diag = false;
          }
          for (size_t j = 0; j < ops.size() && ok; j++) {
            const HOp& op = ops[j];
            if (op.p0 != pos && op.p1 != pos) continue;
            if (op.xi == L.first_cross + i && phase == 0) {
              drop[j] = true;
              phase = 1;
              continue;
            }
            if (phase == 0) continue;
            bool one_q = op.p1 < 0;
            if (phase == 1 && op.diag() && op.kind != H_XPHASE) {
              if (!factor_diag) ok = false;
              continue;
            }
            if (!one_q || op.xi >= 0) {
              ok = false;
              break;
            }
            // a one-qubit op joins the deferred tail V
            cd g[4];
            if (op.kind == H_G1) {
              for (int t = 0; t < 4; t++) g[t] = op.m[t];
            } else if (op.kind == H_PHASE1) {
              g[0] = 1; g[1] = 0; g[2] = 0; g[3] = omega(op.w);
            } else if (op.kind == H_DMUL) {
              g[0] = op.m[0]; g[1] = 0; g[2] = 0; g[3] = op.m[1];
            } else {
              ok = false;
              break;
            }
            mul2(g, V, V);
            drop[j] = true;
            phase = 2;
          }
          if (phase == 0) ok = false;
          for (int t = 0; t < 4; t++) Vm[side][i][t] = V[t];
        }
        if (!ok) break;
        for (size_t j = 0; j < ops.size(); j++)
          if (!drop[j]) kept[side].push_back(ops[j]);
      }
      if (ok) {
        P->deferred = true;
        P->defer_bits = L.bits;
        std::memset(P->ma, 0, sizeof(P->ma));
        std::memset(P->mb, 0, sizeof(P->mb));
        for (int i = 0; i < L.n_cross; i++) {
          const CrossGate& x = P->cross[L.first_cross + i];
          for (int d = 0; d < x.nterm; d++) {
            cd ma[4], mb[4];
            mul2(Vm[0][i], x.fa[d], ma);
            mul2(Vm[1][i], x.fb[d], mb);
            for (int t = 0; t < 4; t++) {
              P->ma[i][d][2 * t] = (float)ma[t].real();
              P->ma[i][d][2 * t + 1] = (float)ma[t].imag();
              P->mb[i][d][2 * t] = (float)mb[t].real();
              P->mb[i][d][2 * t + 1] = (float)mb[t].imag();
            }
          }
        }
        P->A.seg_ops.push_back(kept[0]);  // index nL + 1: deferred last segment
        P->B.seg_ops.push_back(kept[1]);
      }
    }
    // pass programs
    const bool auto_runs = o.run_bits == 0, auto_tiles = o.tile_bits == 0;
    for (int side = 0; side < 2; side++) {
      HalfPlan& H = side ? P->B : P->A;
      H.seg.assign(nL + 1, SegmentPlan());
      std::vector<Pin> pins = H.root_pins;
      for (int s = 0; s <= nL; s++) {
        plan_segment_auto(H.m, H.seg_ops[s], pins, s == 0, *P, auto_tiles, auto_runs, H.seg[s]);
        H.seg[s].scale *= seg_global[2 * s + side];
        pins = H.seg[s].pins_out;
      }
      if (P->deferred) {
        std::vector<Pin> pin_in = nL >= 1 ? H.seg[nL - 1].pins_out : H.root_pins;
        plan_segment_auto(H.m, H.seg_ops[nL + 1], pin_in, nL == 0, *P, auto_tiles, auto_runs, H.last_deferred);
        H.last_deferred.scale *= seg_global[2 * nL + side];
        if (!o.split_last) {
          // no branching happens at the folded level, so the segment that
          // leads to it and the last segment run as one program per final
          std::vector<HOp> ops = H.seg_ops[nL - 1];
          ops.insert(ops.end(), H.seg_ops[nL + 1].begin(), H.seg_ops[nL + 1].end());
          std::vector<Pin> pin_m = nL >= 2 ? H.seg[nL - 2].pins_out : H.root_pins;
          plan_segment_auto(H.m, ops, pin_m, nL == 1, *P, auto_tiles, auto_runs, H.last_merged);
          H.last_merged.scale *= seg_global[2 * (nL - 1) + side] * seg_global[2 * nL + side];
        }
      }
      P->merged_last = P->deferred && !o.split_last;
      // gather byte tables: bitstring byte -> layout index bits (deferred
      // positions excluded; the gather adds them)
      H.tab.assign(8 * 256, 0);
      int ndef = P->deferred ? P->levels.back().n_cross : 0;
      for (int b = 0; b < 8; b++)
        for (int v = 0; v < 256; v++) {
          uint32_t r = 0;
          for (int t = 0; t < 8; t++) {
            int q = 8 * b + t;
            if (q >= n || !((v >> t) & 1)) continue;
            int pos = H.pos_of[q];
            if (pos < 0 || pos < ndef) continue;
            r |= 1u << pos;
          }
          H.tab[b * 256 + v] = r;
        }
    }
    if (P->A.root_scale == 0.0 || P->B.root_scale == 0.0) fail(SF_EINVAL, "internal scale");
  } catch (...) {
    delete P;
    throw;
  }
  return P;
}

static const char* op_name(int code) {
  switch (code) {
    case DOP_H: return "H";
    case DOP_XH: return "X";
    case DOP_YH: return "Y";
    case DOP_G1: return "U1";
    case DOP_G1SEL: return "XT";
    case DOP_G2: return "U2";
    case DOP_PHASE: return "PH";
    case DOP_DMUL: return "D";
    default: return "?";
  }
}

std::string plan_describe(const Plan& p) {
  std::string o;
  char b[256];
  snprintf(b, sizeof b, "qubits %d (grid %dx%d), half A %d, half B %d, cross gates %zu, path bits %d, levels %zu\n",
           p.circ.n, p.circ.rows, p.circ.cols, p.A.m, p.B.m, p.cross.size(), p.path_bits, p.levels.size());
  o += b;
  for (size_t l = 0; l < p.levels.size(); l++) {
    snprintf(b, sizeof b, "level %zu: cycle %d, %d cross gates, %d bits\n", l + 1, p.levels[l].cycle,
             p.levels[l].n_cross, p.levels[l].bits);
    o += b;
  }
  snprintf(b, sizeof b, "last level folded into the gather: %s; tile bits %d, fusion bits %d\n",
           p.deferred ? "yes" : "no", p.tile_bits, p.fuse_bits);
  o += b;
  for (int side = 0; side < 2; side++) {
    const HalfPlan& H = side ? p.B : p.A;
    const int nseg = (int)H.seg.size() + (p.deferred ? 1 : 0);
    for (int s = 0; s < nseg; s++) {
      const bool fin = s == (int)H.seg.size();
      if (p.merged_last && s == (int)H.seg.size() - 2) continue;  // runs inside the merged program
      const SegmentPlan& sp = !fin ? H.seg[s] : (p.merged_last ? H.last_merged : H.last_deferred);
      snprintf(b, sizeof b, "half %c segment %d%s: %zu passes\n", side ? 'B' : 'A', s,
               fin ? (p.merged_last ? " (the level before the folded last level, and the last segment)"
                                    : " (folded last level)")
                   : "",
               sp.passes.size());
      o += b;
      for (size_t q = 0; q < sp.passes.size(); q++) {
        const PassPlan& pp = sp.passes[q];
        std::string act;
        for (int j = 0; j < pp.dev.k; j++) act += std::to_string(pp.dev.gpos[j]) + (j + 1 < pp.dev.k ? "," : "");
        auto pin_list = [](const DevPin* pins, int n) {
          std::string r;
          for (int i = 0; i < n; i++) r += (i ? "," : " [") + std::to_string(pins[i].pos) + (i + 1 == n ? "]" : "");
          return r;
        };
        snprintf(b, sizeof b, "  pass %zu: active [%s] pins in %d%s out %d%s%s scale 2^%d\n", q, act.c_str(),
                 pp.dev.n_pin_in, pin_list(pp.dev.pin_in, pp.dev.n_pin_in).c_str(), pp.dev.n_pin_out,
                 pin_list(pp.dev.pin_out, pp.dev.n_pin_out).c_str(), pp.dev.gen_input ? " generated" : "",
                 (int)std::lround(std::log2(pp.dev.post_scale)));
        o += b;
        for (size_t t = 0; t < pp.stages.size(); t++) {
          const DevStage& st = pp.stages[t];
          std::string rb, ops;
          for (int j = 0; j < st.r; j++) rb += std::to_string(pp.dev.gpos[st.rbit[j]]) + (j + 1 < st.r ? "," : "");
          for (int x = st.op_begin; x < st.op_end; x++) {
            const DevOp& d = pp.ops[x];
            ops += op_name(d.code);
            if (d.code == DOP_PHASE) {
              const DevPhaseGroup& g = pp.phases[d.arg];
              int ncz = 0;
              for (int j = 0; j < st.r; j++) ncz += __builtin_popcount(g.czq[j]) + __builtin_popcount(g.czf[j]) * 2;
              ops += "(" + std::to_string(g.nsh) + "sh," + std::to_string(g.nsel) + "sel)";
            } else if (d.code != DOP_DMUL) {
              ops += std::to_string(d.a);
            }
            ops += " ";
          }
          snprintf(b, sizeof b, "    stage %zu regs [%s]: %s\n", t, rb.c_str(), ops.c_str());
          o += b;
        }
      }
    }
  }
  return o;
}

void plan_destroy(Plan* p) {
  if (!p) return;
  exec_release_cache(*p);
  delete p;
}

// -------------------------------------------------------------- selection
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Keyed 4-round Feistel permutation of [0, 2^w) with cycle walking.
uint64_t feistel(uint64_t v, int w, uint64_t key) {
  if (w == 0) return 0;
  int h = (w + 1) / 2;
  uint64_t hm = (h >= 64) ? ~0ull : ((1ull << h) - 1);
  uint64_t lim = (w >= 64) ? ~0ull : (1ull << w);
  while (true) {
    uint64_t L = v >> h, R = v & hm;
    for (int r = 0; r < 4; r++) {
      uint64_t f = mix64(key ^ (R + (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ull)) & hm;
      uint64_t nl = R;
      R = L ^ f;
      L = nl;
    }
    v = (L << h) | R;
    if (w >= 64 || v < lim) return v;
  }
}

std::vector<Range> select_ranges(const Plan& p, const sf_path_sel& s, double* f_actual) {
  std::vector<Range> out;
  const int x = p.path_bits;
  const uint64_t total = 1ull << x;
  if (s.mode == SF_SEL_RANGE) {
    if (s.first >= total || s.count > total - s.first) fail(SF_EINVAL, "path range out of bounds");
    if (s.count) out.push_back({s.first, s.first + s.count});
    if (f_actual) *f_actual = (double)s.count / (double)total;
  } else if (s.mode == SF_SEL_FRACTION) {
    if (!(s.fidelity > 0 && s.fidelity <= 1)) fail(SF_EINVAL, "fidelity must be in (0, 1]");
    int xs = p.xs;
    uint64_t np = 1ull << xs;
    double kf = std::floor(s.fidelity * (double)np + 1e-9);
    uint64_t K = (uint64_t)std::max(1.0, kf);
    if (K > np) K = np;
    std::vector<uint64_t> pre(K);
    for (uint64_t i = 0; i < K; i++) pre[i] = feistel(i, xs, s.seed);
    std::sort(pre.begin(), pre.end());
    int sb = x - xs;
    for (uint64_t v : pre) {
      uint64_t lo = v << sb, hi = (v + 1) << sb;
      if (!out.empty() && out.back().hi == lo) out.back().hi = hi;
      else out.push_back({lo, hi});
    }
    if (f_actual) *f_actual = (double)K / (double)np;
  } else if (s.mode == SF_SEL_LIST) {
    if (s.n_list < 0 || (s.n_list > 0 && !s.list)) fail(SF_EINVAL, "bad path list");
    std::vector<uint64_t> ids(s.list, s.list + s.n_list);
    std::sort(ids.begin(), ids.end());
    for (size_t i = 0; i < ids.size(); i++) {
      if (ids[i] >= total) fail(SF_EINVAL, "path id out of range");
      if (i && ids[i] == ids[i - 1]) fail(SF_EINVAL, "duplicate path id in list");
      if (!out.empty() && out.back().hi == ids[i]) out.back().hi++;
      else out.push_back({ids[i], ids[i] + 1});
    }
    if (f_actual) *f_actual = (double)s.n_list / (double)total;
  } else {
    fail(SF_EINVAL, "unknown selection mode");
  }
  return out;
}

}  // namespace sf
