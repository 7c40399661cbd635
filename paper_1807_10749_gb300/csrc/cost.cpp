// Runtime model of Section 8 (Eq. t_tot): the features of a request and a
// non-negative least-squares fit of the implementation constants from
// measured times.
//
//   T = C0 + C1 f 2^{x_p} (q1 2^{q1} + q2 2^{q2}) (d_p + C2 2^{x_b} d_b)
//       + C3 (selected paths) n_a
//
// C0, a fixed cost per request (kernel launches, table uploads, the final
// copy), is not in the paper's equation, which models long CPU runs; on a GPU
// it dominates requests below a millisecond.
// f 2^{x_p} is the number of selected prefixes of x_p = x_s path bits, x_b =
// x - x_p the bits below them, d_p the cycles before the branch cycle of the
// last prefix cross gate and d_b the cycles from it to the end. The paper's
// last term reads 2^{x_p + x_b} n_a; with a fraction f of the paths summed it
// is the selected path count times n_a. The model is linear in
// (C0, C1, C1 C2, C3), the coefficients the fit returns.
#include <cmath>
#include <cstring>
#include <vector>

#include "sf_internal.h"

namespace sf {
namespace {

void error_to(const Error& e) { set_error(e.msg); }

constexpr int NT = 4;  // model terms

// Least squares on NT unknowns with x >= 0: the best of the 2^NT - 1 active
// sets (solve the normal equations on each support, keep feasible solutions).
bool nnls(const std::vector<std::array<double, NT>>& A, const std::vector<double>& b, double x[NT]) {
  double best = INFINITY;
  bool found = false;
  for (int mask = 1; mask < (1 << NT); mask++) {
    int idx[NT], m = 0;
    for (int j = 0; j < NT; j++)
      if ((mask >> j) & 1) idx[m++] = j;
    // normal equations M y = r on the support (columns scaled to unit norm)
    double sc[NT] = {0};
    for (int a = 0; a < m; a++) {
      double s = 0;
      for (size_t i = 0; i < A.size(); i++) s += A[i][idx[a]] * A[i][idx[a]];
      sc[a] = s > 0 ? 1.0 / std::sqrt(s) : 0.0;
    }
    double M[NT][NT + 1] = {{0}};
    for (int a = 0; a < m; a++) {
      for (int c = 0; c < m; c++) {
        double s = 0;
        for (size_t i = 0; i < A.size(); i++) s += A[i][idx[a]] * A[i][idx[c]];
        M[a][c] = s * sc[a] * sc[c];
      }
      double s = 0;
      for (size_t i = 0; i < A.size(); i++) s += A[i][idx[a]] * b[i];
      M[a][NT] = s * sc[a];
    }
    bool ok = true;
    for (int c = 0; c < m && ok; c++) {  // Gauss-Jordan with partial pivoting
      int pr = c;
      for (int r = c + 1; r < m; r++)
        if (std::fabs(M[r][c]) > std::fabs(M[pr][c])) pr = r;
      if (std::fabs(M[pr][c]) < 1e-12) {
        ok = false;
        break;
      }
      for (int t = 0; t <= NT; t++) std::swap(M[c][t], M[pr][t]);
      for (int r = 0; r < m; r++) {
        if (r == c) continue;
        const double f = M[r][c] / M[c][c];
        for (int t = 0; t <= NT; t++) M[r][t] -= f * M[c][t];
      }
    }
    if (!ok) continue;
    double y[NT] = {0};
    for (int a = 0; a < m; a++) {
      y[idx[a]] = M[a][NT] / M[a][a] * sc[a];
      if (y[idx[a]] < 0) ok = false;
    }
    if (!ok) continue;
    double r2 = 0;
    for (size_t i = 0; i < A.size(); i++) {
      double d = -b[i];
      for (int j = 0; j < NT; j++) d += A[i][j] * y[j];
      r2 += d * d;
    }
    if (r2 < best) {
      best = r2;
      for (int j = 0; j < NT; j++) x[j] = y[j];
      found = true;
    }
  }
  return found;
}

}  // namespace

void cost_terms(const Plan& p, const sf_path_sel& s, int64_t n_a, double t[4]) {
  double fa = 0;
  const auto rs = select_ranges(p, s, &fa);
  const int x = p.path_bits;
  const int xp = std::min(p.xs, x), xb = x - xp;
  uint64_t paths = 0, prefixes = 0;
  uint64_t last = ~0ull;
  for (const auto& r : rs) {
    paths += r.hi - r.lo;
    if (r.hi <= r.lo) continue;
    uint64_t a = r.lo >> xb, b = (r.hi - 1) >> xb;
    if (a == last) a++;  // ranges are sorted: only the previous one can share a prefix
    if (b >= a) prefixes += b - a + 1;
    last = b;
  }
  int d = 0;
  for (const auto& g : p.circ.gates) d = std::max(d, g.cycle + 1);
  int dp = 0;
  if (xp > 0) {
    // the cross gate holding path bit xb (the lowest prefix bit)
    for (const auto& c : p.cross)
      if (c.shift <= xb && xb < c.shift + c.bits) dp = c.cycle;
  }
  const double work = (double)p.A.m * std::ldexp(1.0, p.A.m) + (double)p.B.m * std::ldexp(1.0, p.B.m);
  t[0] = 1.0;
  t[1] = (double)prefixes * work * dp;
  t[2] = (double)prefixes * work * std::ldexp(1.0, xb) * (d - dp);
  t[3] = (double)paths * (double)n_a;
}

}  // namespace sf

extern "C" {

int sf_plan_cost_terms(const sf_plan* h, const sf_path_sel* sel, int64_t n_a, double* terms) {
  try {
    if (!h || !sel || !terms || n_a < 0) sf::fail(SF_EINVAL, "bad argument");
    sf::cost_terms(*h->p, *sel, n_a, terms);
    return SF_OK;
  } catch (const sf::Error& e) {
    sf::error_to(e);
    return e.code;
  } catch (const std::exception& e) {
    sf::set_error(e.what());
    return SF_EINVAL;
  }
}

int sf_cost_fit(const double* terms, const double* seconds, int64_t n, double* coeffs) {
  try {
    if (!terms || !seconds || !coeffs || n < 1) sf::fail(SF_EINVAL, "bad argument");
    std::vector<std::array<double, sf::NT>> A((size_t)n);
    std::vector<double> b((size_t)n);
    for (int64_t i = 0; i < n; i++) {
      if (!(seconds[i] > 0)) sf::fail(SF_EINVAL, "times must be positive");
      // relative error: each row divided by its measured time
      for (int j = 0; j < sf::NT; j++) A[i][j] = terms[sf::NT * i + j] / seconds[i];
      b[i] = 1.0;
    }
    double y[sf::NT];
    if (!sf::nnls(A, b, y)) sf::fail(SF_EINVAL, "degenerate calibration set");
    for (int j = 0; j < sf::NT; j++) coeffs[j] = y[j];  // C0, C1, C1 C2, C3
    return SF_OK;
  } catch (const sf::Error& e) {
    sf::error_to(e);
    return e.code;
  } catch (const std::exception& e) {
    sf::set_error(e.what());
    return SF_EINVAL;
  }
}

double sf_cost_predict(const double* terms, const double* coeffs) {
  if (!terms || !coeffs) return -1.0;
  double t = 0;
  for (int j = 0; j < sf::NT; j++) t += coeffs[j] * terms[j];
  return t;
}

}  // extern "C"
