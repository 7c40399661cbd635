/* FP64 CPU oracle core (test infrastructure only; the CUDA library never
 * links or calls this file, and it includes none of the library's headers).
 *
 * Plain complex128 state-vector arithmetic for arXiv:1807.10749:
 *   oracle_sv  - Schroedinger simulation of the whole circuit (Section 2): every
 *                gate applied in circuit order as a dense 2x2 or 4x4 matrix.
 *   oracle_sf  - the Schroedinger-Feynman path sum (Eq. 2 / Eq. 3): for each
 *                path, both halves start from |0...0> and get their local gates
 *                and, at each cross-cut gate, the path's term (Eq. 1 or the
 *                decompositions of Section 7); then every requested amplitude
 *                gets A[x_A] * B[x_B] added with Neumaier compensation.
 *
 * State index bit k <-> qubit k of the (half) register. A 4x4 matrix acts on the
 * basis index 2*bit(q0) + bit(q1). Matrices are stored as interleaved
 * (re, im) doubles, row-major.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static cplx mget(const double* m, int i) { return m[2 * i] + I * m[2 * i + 1]; }

/* Apply a 2x2 matrix to qubit q of an n-qubit state. */
static void apply1(cplx* psi, int n, int q, const double* m, int par) {
  cplx m00 = mget(m, 0), m01 = mget(m, 1), m10 = mget(m, 2), m11 = mget(m, 3);
  int64_t half = (int64_t)1 << (n - 1);
  int64_t lo = ((int64_t)1 << q) - 1;
#pragma omp parallel for schedule(static) if (par)
  for (int64_t t = 0; t < half; t++) {
    int64_t i0 = ((t & ~lo) << 1) | (t & lo); /* bit q cleared */
    int64_t i1 = i0 | ((int64_t)1 << q);
    cplx a = psi[i0], b = psi[i1];
    psi[i0] = m00 * a + m01 * b;
    psi[i1] = m10 * a + m11 * b;
  }
}

/* Apply a 4x4 matrix to qubits (q0, q1), basis index 2*bit(q0) + bit(q1). */
static void apply2(cplx* psi, int n, int q0, int q1, const double* m, int par) {
  cplx u[16];
  for (int i = 0; i < 16; i++) u[i] = mget(m, i);
  int lo_q = q0 < q1 ? q0 : q1, hi_q = q0 < q1 ? q1 : q0;
  int64_t quarter = (int64_t)1 << (n - 2);
  int64_t mlo = ((int64_t)1 << lo_q) - 1;
  int64_t mhi = ((int64_t)1 << hi_q) - 1;
#pragma omp parallel for schedule(static) if (par)
  for (int64_t t = 0; t < quarter; t++) {
    /* insert zero bits at positions lo_q then hi_q */
    int64_t v = ((t & ~mlo) << 1) | (t & mlo);
    v = ((v & ~mhi) << 1) | (v & mhi);
    int64_t idx[4];
    for (int k = 0; k < 4; k++) {
      int b0 = (k >> 1) & 1, b1 = k & 1;
      idx[k] = v | ((int64_t)b0 << q0) | ((int64_t)b1 << q1);
    }
    cplx in[4], out[4];
    for (int k = 0; k < 4; k++) in[k] = psi[idx[k]];
    for (int r = 0; r < 4; r++) {
      out[r] = 0;
      for (int c = 0; c < 4; c++) out[r] += u[4 * r + c] * in[c];
    }
    for (int k = 0; k < 4; k++) psi[idx[k]] = out[k];
  }
}

/* Full state vector. Gates: nq[g] in {1,2}; q0/q1; mats[g*32..] (2x2 uses 8
 * doubles). out[2*i], out[2*i+1] = amplitude of bitstring xs[i]. */
int oracle_sv(int n, int64_t n_gates, const int32_t* nq, const int32_t* q0, const int32_t* q1,
              const double* mats, int64_t n_x, const uint64_t* xs, double* out) {
  if (n < 1 || n > 34) return -1;
  int64_t dim = (int64_t)1 << n;
  cplx* psi = (cplx*)calloc((size_t)dim, sizeof(cplx));
  if (!psi) return -2;
  psi[0] = 1.0;
  int par = n >= 16;
  for (int64_t g = 0; g < n_gates; g++) {
    if (nq[g] == 1) apply1(psi, n, q0[g], mats + 32 * g, par);
    else apply2(psi, n, q0[g], q1[g], mats + 32 * g, par);
  }
  for (int64_t i = 0; i < n_x; i++) {
    cplx a = psi[xs[i] & (uint64_t)(dim - 1)];
    out[2 * i] = creal(a);
    out[2 * i + 1] = cimag(a);
  }
  free(psi);
  return 0;
}

/* Gather the bits of x at the given qubit positions (ascending) into a dense
 * index: bit k of the result = bit pos[k] of x. */
static int64_t extract(uint64_t x, const int32_t* pos, int m) {
  int64_t r = 0;
  for (int k = 0; k < m; k++) r |= (int64_t)((x >> pos[k]) & 1u) << k;
  return r;
}

/* Evolve one half for one path. ops: nq (1/2), a0/a1 local qubits, xg = -1
 * for a local gate (matrix mats[op*32..]) or the index of the cross gate whose
 * term digits[xg] selects the 2x2 factor mats[op*32 + 8*digit ..]. */
static void evolve_half(cplx* psi, int m, int64_t n_ops, const int32_t* nq, const int32_t* a0,
                        const int32_t* a1, const int32_t* xg, const double* mats,
                        const int32_t* digits, int par) {
  int64_t dim = (int64_t)1 << m;
  memset(psi, 0, (size_t)dim * sizeof(cplx));
  psi[0] = 1.0;
  for (int64_t o = 0; o < n_ops; o++) {
    if (xg[o] >= 0) {
      apply1(psi, m, a0[o], mats + 32 * o + 8 * digits[xg[o]], par);
    } else if (nq[o] == 1) {
      apply1(psi, m, a0[o], mats + 32 * o, par);
    } else {
      apply2(psi, m, a0[o], a1[o], mats + 32 * o, par);
    }
  }
}

/* Neumaier step: (s, c) += v */
static void neumaier(double* s, double* c, double v) {
  double t = *s + v;
  if (((*s) >= 0 ? *s : -*s) >= (v >= 0 ? v : -v)) *c += (*s - t) + v;
  else *c += (v - t) + *s;
  *s = t;
}

/* Schroedinger-Feynman path sum. Half A has mA qubits at global positions
 * posA[0..mA) (ascending), half B likewise. digits: n_paths x n_cross branch
 * digits. out: 2*n_x doubles, the compensated sums over the given paths. */
int oracle_sf(int mA, const int32_t* posA, int64_t nA, const int32_t* nqA, const int32_t* a0A,
              const int32_t* a1A, const int32_t* xgA, const double* matA,
              int mB, const int32_t* posB, int64_t nB, const int32_t* nqB, const int32_t* a0B,
              const int32_t* a1B, const int32_t* xgB, const double* matB,
              int n_cross, int64_t n_paths, const int32_t* digits,
              int64_t n_x, const uint64_t* xs, double* out) {
  if (mA < 1 || mB < 1 || mA > 31 || mB > 31) return -1;
  int64_t* ia = (int64_t*)malloc((size_t)(n_x > 0 ? n_x : 1) * sizeof(int64_t));
  int64_t* ib = (int64_t*)malloc((size_t)(n_x > 0 ? n_x : 1) * sizeof(int64_t));
  double* s = (double*)calloc((size_t)(2 * (n_x > 0 ? n_x : 1)), sizeof(double));
  double* c = (double*)calloc((size_t)(2 * (n_x > 0 ? n_x : 1)), sizeof(double));
  if (!ia || !ib || !s || !c) return -2;
  for (int64_t i = 0; i < n_x; i++) {
    ia[i] = extract(xs[i], posA, mA);
    ib[i] = extract(xs[i], posB, mB);
  }
  int big = (mA >= 18 || mB >= 18);
  if (big) {
    /* large halves: paths in sequence, each gate parallel over amplitudes */
    cplx* A = (cplx*)malloc(((size_t)1 << mA) * sizeof(cplx));
    cplx* B = (cplx*)malloc(((size_t)1 << mB) * sizeof(cplx));
    if (!A || !B) return -2;
    for (int64_t p = 0; p < n_paths; p++) {
      const int32_t* d = digits + (int64_t)n_cross * p;
      evolve_half(A, mA, nA, nqA, a0A, a1A, xgA, matA, d, 1);
      evolve_half(B, mB, nB, nqB, a0B, a1B, xgB, matB, d, 1);
      for (int64_t i = 0; i < n_x; i++) {
        cplx v = A[ia[i]] * B[ib[i]];
        neumaier(&s[2 * i], &c[2 * i], creal(v));
        neumaier(&s[2 * i + 1], &c[2 * i + 1], cimag(v));
      }
    }
    free(A);
    free(B);
  } else {
    /* small halves: paths in parallel, one partial sum per thread, combined
     * in thread order */
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    double* ps = (double*)calloc((size_t)nt * 2 * (n_x > 0 ? n_x : 1), sizeof(double));
    double* pc = (double*)calloc((size_t)nt * 2 * (n_x > 0 ? n_x : 1), sizeof(double));
    if (!ps || !pc) return -2;
#pragma omp parallel
    {
      int tid = 0;
#ifdef _OPENMP
      tid = omp_get_thread_num();
#endif
      cplx* A = (cplx*)malloc(((size_t)1 << mA) * sizeof(cplx));
      cplx* B = (cplx*)malloc(((size_t)1 << mB) * sizeof(cplx));
      double* ms = ps + (size_t)tid * 2 * n_x;
      double* mc = pc + (size_t)tid * 2 * n_x;
#pragma omp for schedule(static)
      for (int64_t p = 0; p < n_paths; p++) {
        const int32_t* d = digits + (int64_t)n_cross * p;
        evolve_half(A, mA, nA, nqA, a0A, a1A, xgA, matA, d, 0);
        evolve_half(B, mB, nB, nqB, a0B, a1B, xgB, matB, d, 0);
        for (int64_t i = 0; i < n_x; i++) {
          cplx v = A[ia[i]] * B[ib[i]];
          neumaier(&ms[2 * i], &mc[2 * i], creal(v));
          neumaier(&ms[2 * i + 1], &mc[2 * i + 1], cimag(v));
        }
      }
      free(A);
      free(B);
    }
    for (int t = 0; t < nt; t++)
      for (int64_t i = 0; i < 2 * n_x; i++) {
        neumaier(&s[i], &c[i], ps[(size_t)t * 2 * n_x + i]);
        neumaier(&s[i], &c[i], pc[(size_t)t * 2 * n_x + i]);
      }
    free(ps);
    free(pc);
  }
  for (int64_t i = 0; i < 2 * n_x; i++) out[i] = s[i] + c[i];
  free(ia);
  free(ib);
  free(s);
  free(c);
  return 0;
}

/* Number of OpenMP threads the oracle runs with. */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
