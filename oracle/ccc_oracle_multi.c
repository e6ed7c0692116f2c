/*
 * CPU oracle for the 2-way CCC of markers with s allele states.
 *
 * TEST INFRASTRUCTURE ONLY, like ccc_oracle.c (linked into the same oracle
 * library): loaded only by the tests, the package's smoke check and the
 * benchmark's CPU baseline; it shares nothing with the CUDA path.
 *
 * Sec. 7 item 2 of the paper names the extension of CCC from biallelic SNPs to
 * markers with an arbitrary number of states: a marker with s_1 states against
 * one with s_2 states gives an s_1 x s_2 table of values.  It is written here
 * with the definitions of Sec. 2.1 and Eqs. 1-3 unchanged except for the
 * state set, S = {0, .., s-1}:
 *   v_{i,q} in S x S                          (a pair of allele states)
 *   rho_{i,q}(a) = sum_r chi_a((v_{i,q})_r)   (how many of the two equal a)
 *   f_i(a)       = (1/(2 n_f)) sum_q rho_{i,q}(a)                       (Eq. 1)
 *   f_{i,j}(a,b) = (1/(4 n_f)) sum_q rho_{i,q}(a) rho_{j,q}(b)           (Eq. 2)
 *   CCC_{i,j}(a,b) = f_{i,j}(a,b) (1 - g f_i(a)) (1 - g f_j(b))          (Eq. 3)
 * for a, b in S.  The tally r_{ij}^{ab} is the Eq. 2 numerator.  Here it is
 * accumulated as the expanded product: rho_i(a) rho_j(b) = sum over the two
 * allele slots r of v_i and r' of v_j of chi_a((v_i)_r) chi_b((v_j)_r'), i.e.
 * four unit increments per individual at (x_i, x_j), (x_i, y_j), (y_i, x_j),
 * (y_i, y_j).
 *
 * Readings (also listed in the design notes): an entry is one byte,
 * x | (y << 4); it is missing when x >= s or y >= s (0xFF by convention) and
 * then contributes nothing; missing data are normalised as in ccc_oracle.c
 * (PERSNP: f_i over SNP i's non-missing entries, f_{i,j} over the jointly
 * non-missing ones; JOINT: f_i(a) = sum_b r^{ab} / (4 n_ij)); n_ij = 0 gives
 * zero tallies and zero CCC values.  Output per pair: s*s tallies and s*s
 * values, (a, b) with a (state of the lower SNP index) major.
 */
#include <stdint.h>
#include <stdlib.h>

#define MULTI_NORM_JOINT 1

static int state_lo(uint8_t e) { return e & 15; }
static int state_hi(uint8_t e) { return e >> 4; }
static int multi_missing(uint8_t e, int s) { return state_lo(e) >= s || state_hi(e) >= s; }

/* Per SNP: s_i^a = sum_q rho_{i,q}(a) for a < s, then n_i; counts[i*(s+1) + a]. */
void oracle_multi_counts(const uint8_t *geno, int64_t n_f, int64_t n_v, int64_t ld, int s,
                         int64_t *counts) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
  for (i = 0; i < n_v; ++i) {
    int64_t *c = counts + i * (s + 1);
    int a;
    int64_t q;
    for (a = 0; a <= s; ++a) c[a] = 0;
    for (q = 0; q < n_f; ++q) {
      const uint8_t e = geno[i * ld + q];
      if (multi_missing(e, s)) continue;
      c[state_lo(e)] += 1;
      c[state_hi(e)] += 1;
      c[s] += 1;
    }
  }
}

/* One pair i < j: s*s tallies and s*s CCC values (Eqs. 2-3 over S x S). */
static void multi_pair(const uint8_t *geno, int64_t n_f, int64_t ld, int s, int64_t i, int64_t j,
                       const int64_t *counts, double gamma, int norm, int64_t *tally, double *ccc) {
  const int ss = s * s;
  int64_t n_ij = 0, q;
  int a, b;
  for (a = 0; a < ss; ++a) tally[a] = 0;
  for (q = 0; q < n_f; ++q) {
    const uint8_t ei = geno[i * ld + q], ej = geno[j * ld + q];
    if (multi_missing(ei, s) || multi_missing(ej, s)) continue;
    const int xi = state_lo(ei), yi = state_hi(ei), xj = state_lo(ej), yj = state_hi(ej);
    tally[xi * s + xj] += 1;
    tally[xi * s + yj] += 1;
    tally[yi * s + xj] += 1;
    tally[yi * s + yj] += 1;
    ++n_ij;
  }
  if (n_ij == 0) {
    for (a = 0; a < ss; ++a) ccc[a] = 0.0;
    return;
  }
  double *fi = (double *)malloc(2 * sizeof(double) * (size_t)s);
  double *fj = fi + s;
  const double d = 4.0 * (double)n_ij;
  if (norm == MULTI_NORM_JOINT) {
    for (a = 0; a < s; ++a) {
      int64_t m = 0;
      for (b = 0; b < s; ++b) m += tally[a * s + b];
      fi[a] = (double)m / d;
    }
    for (b = 0; b < s; ++b) {
      int64_t m = 0;
      for (a = 0; a < s; ++a) m += tally[a * s + b];
      fj[b] = (double)m / d;
    }
  } else {
    const int64_t *ci = counts + i * (s + 1), *cj = counts + j * (s + 1);
    for (a = 0; a < s; ++a) {
      fi[a] = ci[s] > 0 ? (double)ci[a] / (2.0 * (double)ci[s]) : 0.0;
      fj[a] = cj[s] > 0 ? (double)cj[a] / (2.0 * (double)cj[s]) : 0.0;
    }
  }
  for (a = 0; a < s; ++a)
    for (b = 0; b < s; ++b)
      ccc[a * s + b] = (double)tally[a * s + b] / d * (1.0 - gamma * fi[a]) * (1.0 - gamma * fj[b]);
  free(fi);
}

/* Every listed row i against all j > i, rows in the given order (upper-triangle
 * order inside a row); returns 0, or 1 when a row is out of range. */
int oracle_multi_rows(const uint8_t *geno, int64_t n_f, int64_t n_v, int64_t ld, int s,
                      const int64_t *rows, int64_t n_rows, double gamma, int norm,
                      int64_t *tally, double *ccc) {
  int64_t *counts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_v * (s + 1)));
  int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_rows + 1));
  int64_t r;
  if (counts == NULL || off == NULL) {
    free(counts);
    free(off);
    return 2;
  }
  off[0] = 0;
  for (r = 0; r < n_rows; ++r) {
    if (rows[r] < 0 || rows[r] >= n_v) {
      free(counts);
      free(off);
      return 1;
    }
    off[r + 1] = off[r] + (n_v - 1 - rows[r]);
  }
  oracle_multi_counts(geno, n_f, n_v, ld, s, counts);
  const int64_t ss = (int64_t)s * s;
#pragma omp parallel for schedule(dynamic, 1)
  for (r = 0; r < n_rows; ++r) {
    const int64_t i = rows[r];
    int64_t j;
    for (j = i + 1; j < n_v; ++j) {
      const int64_t p = off[r] + (j - i - 1);
      multi_pair(geno, n_f, ld, s, i, j, counts, gamma, norm, tally + p * ss, ccc + p * ss);
    }
  }
  free(counts);
  free(off);
  return 0;
}

/* Explicit pairs pi[t] < pj[t]. */
int oracle_multi_pairs(const uint8_t *geno, int64_t n_f, int64_t n_v, int64_t ld, int s,
                       const int64_t *pi, const int64_t *pj, int64_t n, double gamma, int norm,
                       int64_t *tally, double *ccc) {
  int64_t *counts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_v * (s + 1)));
  int64_t t;
  if (counts == NULL) return 2;
  oracle_multi_counts(geno, n_f, n_v, ld, s, counts);
  const int64_t ss = (int64_t)s * s;
#pragma omp parallel for schedule(dynamic, 64)
  for (t = 0; t < n; ++t)
    multi_pair(geno, n_f, ld, s, pi[t], pj[t], counts, gamma, norm, tally + t * ss, ccc + t * ss);
  free(counts);
  return 0;
}
