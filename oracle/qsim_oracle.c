/*
 * FP64 CPU oracle for the full-amplitude state-vector method (test infrastructure).
 *
 * This file is test infrastructure. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it. It shares no code with the CUDA library.
 *
 * The loops below are the plain definitions, written for a reader to check against the
 * paper by eye; no blocking, fusion or reordering. The state is an array of 2^n complex
 * doubles stored as (re, im) pairs, indexed by i = sum_k i_k 2^k, so qubit k is bit k of
 * the index (Eq. 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double re, im;
} cplx;

static inline cplx cmul(cplx a, cplx b) {
  cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}
static inline cplx cadd(cplx a, cplx b) {
  cplx r = {a.re + b.re, a.im + b.im};
  return r;
}

/*
 * Single-qubit gate U on target t, applied where every control bit in cmask is 1
 * (Eq. 2 for cmask = 0; Eq. 3 with control q for cmask = 2^q; several controls
 * are the nested CONTROL block of Appendix A-1). u is row-major [a b; c d].
 * For every i with i_t = 0 (and the controls set): (a_i, a_{i+2^t}) <- U (a_i, a_{i+2^t}).
 */
void or_apply_1q(cplx *psi, int n, int t, uint64_t cmask, const cplx *u) {
  const int64_t N = (int64_t)1 << n;
  const int64_t bt = (int64_t)1 << t;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    if (i & bt) continue;
    if (((uint64_t)i & cmask) != cmask) continue;
    cplx x0 = psi[i], x1 = psi[i + bt];
    psi[i] = cadd(cmul(u[0], x0), cmul(u[1], x1));
    psi[i + bt] = cadd(cmul(u[2], x0), cmul(u[3], x1));
  }
}

/*
 * k-qubit gate M (2^k x 2^k, row-major) on qubits qs[0..k-1], where the controls in
 * cmask are 1. The matrix row/column index r has bit (k-1-j) equal to the bit of qubit
 * qs[j]: the first listed qubit is the most significant, which is how the paper's
 * CNOT, CZ, CR, SWAP, iSWAP and TOFFOLI matrices are written (Appendix A-1).
 * For every base index b with all bits qs[j] = 0: v_r = a_{b + off(r)}, a' = M v.
 */
void or_apply_kq(cplx *psi, int n, const int *qs, int k, uint64_t cmask, const cplx *m) {
  const int64_t N = (int64_t)1 << n;
  const int dim = 1 << k;
  uint64_t qmask = 0;
  for (int j = 0; j < k; ++j) qmask |= (uint64_t)1 << qs[j];
  int64_t *off = (int64_t *)malloc(sizeof(int64_t) * dim);
  for (int r = 0; r < dim; ++r) {
    int64_t o = 0;
    for (int j = 0; j < k; ++j)
      if ((r >> (k - 1 - j)) & 1) o |= (int64_t)1 << qs[j];
    off[r] = o;
  }
#pragma omp parallel
  {
    cplx *v = (cplx *)malloc(sizeof(cplx) * dim);
#pragma omp for schedule(static)
    for (int64_t b = 0; b < N; ++b) {
      if ((uint64_t)b & qmask) continue;
      if (((uint64_t)b & cmask) != cmask) continue;
      for (int r = 0; r < dim; ++r) v[r] = psi[b + off[r]];
      for (int r = 0; r < dim; ++r) {
        cplx acc = {0.0, 0.0};
        for (int c = 0; c < dim; ++c) acc = cadd(acc, cmul(m[r * dim + c], v[c]));
        psi[b + off[r]] = acc;
      }
    }
    free(v);
  }
  free(off);
}

/* Sum of |a_i|^2 over the whole state. */
double or_norm2(const cplx *psi, int n) {
  const int64_t N = (int64_t)1 << n;
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < N; ++i) s += psi[i].re * psi[i].re + psi[i].im * psi[i].im;
  return s;
}

/* Reduced density matrix of the k (<= 3) listed qubits, qs[0] the most significant bit of
 * its row and column index: rho[r][c] = sum over the other qubits' bits (rest) of
 * psi(r, rest) conj(psi(c, rest)). out holds 2^k x 2^k complex numbers, row-major. */
void or_reduced_density(const cplx *psi, int n, const int *qs, int k, double *out) {
  const int64_t N = (int64_t)1 << n;
  const int d = 1 << k;
  int64_t mask = 0, off[8];
  for (int j = 0; j < k; ++j) mask |= (int64_t)1 << qs[j];
  for (int r = 0; r < d; ++r) {
    off[r] = 0;
    for (int j = 0; j < k; ++j)
      if ((r >> (k - 1 - j)) & 1) off[r] |= (int64_t)1 << qs[j];
  }
  double acc[128] = {0};
#pragma omp parallel for reduction(+ : acc[:128]) schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    if (i & mask) continue; /* one term per value of the other qubits */
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        const cplx a = psi[i | off[r]], b = psi[i | off[c]];
        acc[2 * (r * d + c)] += a.re * b.re + a.im * b.im;
        acc[2 * (r * d + c) + 1] += a.im * b.re - a.re * b.im;
      }
  }
  for (int e = 0; e < 2 * d * d; ++e) out[e] = acc[e];
}

/* <a|b> = sum conj(a_i) b_i, written to out[0] (re), out[1] (im). */
void or_inner(const cplx *a, const cplx *b, int n, double *out) {
  const int64_t N = (int64_t)1 << n;
  double re = 0.0, im = 0.0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    re += a[i].re * b[i].re + a[i].im * b[i].im;
    im += a[i].re * b[i].im - a[i].im * b[i].re;
  }
  out[0] = re;
  out[1] = im;
}

/*
 * PMEASURE (Appendix A-1): probability of each outcome s of the listed qubits, without
 * changing the state. out[s] with s = sum_j bit(qs[j]) << (m-1-j): the first listed
 * qubit is the leftmost character of the printed outcome (Appendix A-2 example).
 * Serial loop, so the result does not depend on the thread count.
 */
void or_probabilities(const cplx *psi, int n, const int *qs, int m, double *out) {
  const int64_t N = (int64_t)1 << n;
  memset(out, 0, sizeof(double) * ((size_t)1 << m));
  for (int64_t i = 0; i < N; ++i) {
    int64_t s = 0;
    for (int j = 0; j < m; ++j) s |= ((i >> qs[j]) & 1) << (m - 1 - j);
    out[s] += psi[i].re * psi[i].re + psi[i].im * psi[i].im;
  }
}

/* <Z_q> * norm2 = sum_i (-1)^{i_q} |a_i|^2 for every qubit q (unnormalised). */
void or_z_sums(const cplx *psi, int n, double *out) {
  const int64_t N = (int64_t)1 << n;
  for (int q = 0; q < n; ++q) out[q] = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double p = psi[i].re * psi[i].re + psi[i].im * psi[i].im;
    for (int q = 0; q < n; ++q) out[q] += ((i >> q) & 1) ? -p : p;
  }
}

/*
 * Sampling of full basis indices: for each draw u in [0,1), the smallest index i with
 * u * sum_j |a_j|^2 < sum_{j <= i} |a_j|^2 (running sum in index order). Shots are
 * processed one at a time by a linear scan: slow and plain.
 */
void or_sample(const cplx *psi, int n, const double *u, int64_t shots, uint64_t *out) {
  const int64_t N = (int64_t)1 << n;
  double total = 0.0;
  for (int64_t i = 0; i < N; ++i) total += psi[i].re * psi[i].re + psi[i].im * psi[i].im;
  for (int64_t s = 0; s < shots; ++s) {
    double target = u[s] * total, run = 0.0;
    int64_t pick = N - 1;
    for (int64_t i = 0; i < N; ++i) {
      run += psi[i].re * psi[i].re + psi[i].im * psi[i].im;
      if (target < run) {
        pick = i;
        break;
      }
    }
    out[s] = (uint64_t)pick;
  }
}

/*
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11). Ten rounds of the 4x32 S-box with multipliers 0xD2511F53 and
 * 0xCD9E8D57; the key is bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85
 * between rounds.
 */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* Many Philox blocks at once: ctrs[4*j..4*j+3] -> outs[4*j..4*j+3]. */
void or_philox_many(const uint32_t *ctrs, int64_t count, const uint32_t key[2], uint32_t *outs) {
  for (int64_t j = 0; j < count; ++j) or_philox4x32_10(ctrs + 4 * j, key, outs + 4 * j);
}
