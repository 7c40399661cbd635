// Circuits: gate matrices, validation and the text format.
//
// Gate set of Section 1 (H, CZ, X^1/2, Y^1/2, T) and Section 7 (iSWAP), plus Z,
// S and explicit 2x2 / 4x4 matrices. Matrices follow the readings in sfsim.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <sstream>

#include "sf_internal.h"

namespace sf {

void gate_matrix(Gate& g) {
  const double r = std::sqrt(0.5);
  const cd I(0, 1);
  for (auto& v : g.m) v = 0;
  switch (g.kind) {
    case SF_H: g.m[0] = r; g.m[1] = r; g.m[2] = r; g.m[3] = -r; break;
    case SF_X_HALF:
      g.m[0] = 0.5 * (1.0 + I); g.m[1] = 0.5 * (1.0 - I);
      g.m[2] = 0.5 * (1.0 - I); g.m[3] = 0.5 * (1.0 + I); break;
    case SF_Y_HALF:
      g.m[0] = 0.5 * (1.0 + I); g.m[1] = -0.5 * (1.0 + I);
      g.m[2] = 0.5 * (1.0 + I); g.m[3] = 0.5 * (1.0 + I); break;
    case SF_T: g.m[0] = 1; g.m[3] = cd(r, r); break;
    case SF_Z: g.m[0] = 1; g.m[3] = -1; break;
    case SF_S: g.m[0] = 1; g.m[3] = I; break;
    case SF_CZ: g.m[0] = 1; g.m[5] = 1; g.m[10] = 1; g.m[15] = -1; break;
    case SF_ISWAP: g.m[0] = 1; g.m[6] = I; g.m[9] = I; g.m[15] = 1; break;
    default: break;  // U1/U2 carry their own entries
  }
}

static void validate(Circuit& c) {
  if (c.rows < 1 || c.cols < 1 || c.rows * c.cols > 64)
    fail(SF_EINVAL, "grid must have 1..64 qubits");
  c.n = c.rows * c.cols;
  std::stable_sort(c.gates.begin(), c.gates.end(),
                   [](const Gate& a, const Gate& b) { return a.cycle < b.cycle; });
  std::map<int, uint64_t> used;
  for (size_t i = 0; i < c.gates.size(); i++) {
    const Gate& g = c.gates[i];
    if (g.kind < SF_H || g.kind > SF_U2) fail(SF_EINVAL, "gate " + std::to_string(i) + ": bad kind");
    if (g.q0 < 0 || g.q0 >= c.n) fail(SF_EINVAL, "gate " + std::to_string(i) + ": bad qubit");
    uint64_t bits = 1ull << g.q0;
    if (g.nq() == 2) {
      if (g.q1 < 0 || g.q1 >= c.n || g.q1 == g.q0)
        fail(SF_EINVAL, "gate " + std::to_string(i) + ": bad second qubit");
      bits |= 1ull << g.q1;
    }
    uint64_t& u = used[g.cycle];
    if (u & bits)
      fail(SF_EINVAL, "gate " + std::to_string(i) + ": qubit used twice in cycle " +
                          std::to_string(g.cycle));
    u |= bits;
    for (int k = 0; k < 16; k++)
      if (!std::isfinite(g.m[k].real()) || !std::isfinite(g.m[k].imag()))
        fail(SF_EINVAL, "gate " + std::to_string(i) + ": non-finite matrix entry");
  }
}

Circuit* circuit_from_gates(int rows, int cols, const sf_gate* gates, int64_t n_gates) {
  if (n_gates < 0 || (n_gates > 0 && !gates)) fail(SF_EINVAL, "bad gate array");
  Circuit* c = new Circuit();
  try {
    c->rows = rows;
    c->cols = cols;
    for (int64_t i = 0; i < n_gates; i++) {
      Gate g;
      g.cycle = gates[i].cycle;
      g.kind = gates[i].kind;
      g.q0 = gates[i].q0;
      g.q1 = gates[i].q1;
      if (g.kind == SF_U1) {
        for (int k = 0; k < 4; k++) g.m[k] = cd(gates[i].m[2 * k], gates[i].m[2 * k + 1]);
      } else if (g.kind == SF_U2) {
        for (int k = 0; k < 16; k++) g.m[k] = cd(gates[i].m[2 * k], gates[i].m[2 * k + 1]);
      } else {
        gate_matrix(g);
      }
      if (g.nq() == 1) g.q1 = -1;
      c->gates.push_back(g);
    }
    validate(*c);
  } catch (...) {
    delete c;
    throw;
  }
  return c;
}

Circuit* circuit_parse(const char* text) {
  if (!text) fail(SF_EINVAL, "null text");
  static const std::map<std::string, int> names = {
      {"h", SF_H}, {"x_1_2", SF_X_HALF}, {"y_1_2", SF_Y_HALF}, {"t", SF_T}, {"z", SF_Z},
      {"s", SF_S}, {"cz", SF_CZ}, {"iswap", SF_ISWAP}, {"u1", SF_U1}, {"u2", SF_U2}};
  Circuit* c = new Circuit();
  try {
    std::istringstream in(text);
    std::string line;
    int lineno = 0;
    bool have_grid = false;
    while (std::getline(in, line)) {
      lineno++;
      auto hash = line.find('#');
      if (hash != std::string::npos) line = line.substr(0, hash);
      std::istringstream ls(line);
      std::vector<std::string> tok;
      std::string t;
      while (ls >> t) tok.push_back(t);
      if (tok.empty()) continue;
      auto bad = [&](const char* why) {
        fail(SF_EINVAL, "line " + std::to_string(lineno) + ": " + why);
      };
      if (tok[0] == "grid") {
        if (tok.size() != 3) bad("grid needs R C");
        c->rows = std::atoi(tok[1].c_str());
        c->cols = std::atoi(tok[2].c_str());
        have_grid = true;
        continue;
      }
      if (tok.size() < 3) bad("expected <cycle> <gate> <qubits>");
      auto it = names.find(tok[1]);
      if (it == names.end()) bad("unknown gate");
      Gate g;
      char* end = nullptr;
      g.cycle = (int)std::strtol(tok[0].c_str(), &end, 10);
      if (*end) bad("bad cycle");
      g.kind = it->second;
      int nq = g.nq();
      if ((int)tok.size() < 2 + nq) bad("missing qubit");
      g.q0 = std::atoi(tok[2].c_str());
      g.q1 = nq == 2 ? std::atoi(tok[3].c_str()) : -1;
      size_t nreal = tok.size() - 2 - nq;
      size_t want = g.kind == SF_U1 ? 8 : (g.kind == SF_U2 ? 32 : 0);
      if (nreal != want) bad("wrong number of matrix entries");
      if (want) {
        for (size_t k = 0; k < want / 2; k++) {
          double re = std::strtod(tok[2 + nq + 2 * k].c_str(), &end);
          if (*end) bad("bad real");
          double im = std::strtod(tok[2 + nq + 2 * k + 1].c_str(), &end);
          if (*end) bad("bad real");
          g.m[k] = cd(re, im);
        }
      } else {
        gate_matrix(g);
      }
      c->gates.push_back(g);
    }
    if (!have_grid) fail(SF_EINVAL, "missing 'grid R C' line");
    validate(*c);
  } catch (...) {
    delete c;
    throw;
  }
  return c;
}

// One-sided (Hestenes) Jacobi SVD for a complex 4x4 matrix. Column pairs
// (p, q) of W = R V are rotated until orthogonal; then s_k = |w_k| and
// U = w_k / s_k. Sorted by s descending.
void svd4(const cd R[16], cd U[16], double s[4], cd V[16]) {
  cd W[16];
  for (int i = 0; i < 16; i++) W[i] = R[i];
  for (int i = 0; i < 16; i++) V[i] = (i % 5 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; sweep++) {
    double off = 0;
    for (int p = 0; p < 3; p++)
      for (int q = p + 1; q < 4; q++) {
        double app = 0, aqq = 0;
        cd apq = 0;
        for (int i = 0; i < 4; i++) {
          app += std::norm(W[4 * i + p]);
          aqq += std::norm(W[4 * i + q]);
          apq += std::conj(W[4 * i + p]) * W[4 * i + q];
        }
        double mag = std::abs(apq);
        if (mag <= 1e-300 || mag <= 1e-17 * std::sqrt(app * aqq)) continue;
        off = std::max(off, mag / std::sqrt(app * aqq + 1e-300));
        // rotate so that the (p, q) entry of W^H W vanishes
        cd e = apq / mag;  // phase
        double tau = (aqq - app) / (2 * mag);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        double cs = 1 / std::sqrt(1 + t * t), sn = cs * t;
        for (int i = 0; i < 4; i++) {
          cd wp = W[4 * i + p], wq = W[4 * i + q];
          W[4 * i + p] = cs * wp - sn * std::conj(e) * wq;
          W[4 * i + q] = sn * e * wp + cs * wq;
          cd vp = V[4 * i + p], vq = V[4 * i + q];
          V[4 * i + p] = cs * vp - sn * std::conj(e) * vq;
          V[4 * i + q] = sn * e * vp + cs * vq;
        }
      }
    if (off < 1e-16) break;
  }
  double sv[4];
  int order[4] = {0, 1, 2, 3};
  for (int k = 0; k < 4; k++) {
    double a = 0;
    for (int i = 0; i < 4; i++) a += std::norm(W[4 * i + k]);
    sv[k] = std::sqrt(a);
  }
  std::sort(order, order + 4, [&](int a, int b) { return sv[a] > sv[b]; });
  cd Vs[16];
  for (int kk = 0; kk < 4; kk++) {
    int k = order[kk];
    s[kk] = sv[k];
    for (int i = 0; i < 4; i++) {
      U[4 * i + kk] = sv[k] > 1e-300 ? W[4 * i + k] / sv[k] : cd(0);
      Vs[4 * i + kk] = V[4 * i + k];
    }
  }
  for (int i = 0; i < 16; i++) V[i] = Vs[i];
}

}  // namespace sf
