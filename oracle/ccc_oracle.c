/*
 * CPU oracle for the Custom Correlation Coefficient (CCC) tallies and metrics.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into its own shared library
 * that only the tests, the package's smoke check and the benchmark's CPU
 * baseline load.  It shares no code, header, table or constant with the CUDA
 * path and nothing in the CUDA path may call it.
 *
 * It is deliberately plain: one loop over individuals q per pair (2-way) or
 * per triple (3-way), decoding every packed entry on the fly and forming the
 * products of allele counts exactly as the definitions write them.  Tallies
 * are int64, frequencies and CCC values are double.  OpenMP spreads the
 * listed rows over host threads; nothing else is reordered.
 *
 * Definitions followed (Joubert et al., "Parallel Accelerated Custom
 * Correlation Coefficient Calculations for Genomics Applications"):
 *   Sec. 2.1  vector model v_{i,q} in S x S, S = {0,1};
 *             rho_{i,q}(a) = sum_r chi_a((v_{i,q})_r)        (count of allele a)
 *   Eq. 1     f_i(a)      = (1/(2 n_f)) sum_q rho_{i,q}(a)
 *   Eq. 2     f_{i,j}(a,b) = (1/(4 n_f)) sum_q rho_{i,q}(a) rho_{j,q}(b)
 *   Eq. 3     CCC_{i,j}(a,b) = f_{i,j}(a,b) (1 - g f_i(a)) (1 - g f_j(b)), g = 2/3
 *   Eq. 5     f_{i,j,k}(a,b,c) = (1/(8 n_f)) sum_q rho_i(a) rho_j(b) rho_k(c)
 *   Eq. 4     CCC_{i,j,k}(a,b,c) = f_{i,j,k}(a,b,c) (1-g f_i(a))(1-g f_j(b))(1-g f_k(c))
 *   Sec. 7 item 1: the allele pair (1,0) is reserved to mark a missing entry,
 *             and missing entries are skipped.
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   - code of an entry = 2*(v)_1 + (v)_2, uint64 words, entry q at bits
 *     2*(q%32) of word q/32; bits past n_f are ignored.
 *   - a missing entry contributes rho = 0 for both alleles.
 *   - normalisation with missing data: n_f in Eqs. 1, 2, 5 becomes the count of
 *     non-missing entries involved.  PERSNP (norm 0): f_i over SNP i's own
 *     non-missing entries, f_{i,j} over the jointly non-missing entries.  JOINT
 *     (norm 1): f_i(a) is the marginal of the pair (triple) table itself,
 *     f_i(a) = sum_b r^{ab} / (4 n_ij).  Both equal the paper's definitions when
 *     nothing is missing.
 *   - when no entry is jointly present (n_ij = 0, n_ijk = 0) the tallies are 0
 *     and every CCC value is 0; likewise f_i(a) = 0 when n_i = 0.
 * Output order: 2-way tallies (a,b) with a (allele of the lower SNP index)
 * major: 00,01,10,11.  3-way: abc with a most significant.
 */
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_NORM_PERSNP 0
#define ORACLE_NORM_JOINT 1

/* The 2-bit code of entry q of SNP i. */
static int entry_code(const uint64_t *geno, int64_t ld, int64_t i, int64_t q) {
  uint64_t word = geno[i * ld + q / 32];
  return (int)((word >> (2 * (q % 32))) & 3u);
}

/* The allele pair ((v)_1, (v)_2) stored in a code. */
static int allele_1(int code) { return (code >> 1) & 1; }
static int allele_2(int code) { return code & 1; }

/* Sec. 7 item 1: the pair (1,0) marks a missing entry. */
static int is_missing(int code) { return allele_1(code) == 1 && allele_2(code) == 0; }

/* rho_{i,q}(a) = sum_r chi_a((v_{i,q})_r), Sec. 2.1; 0 for a missing entry. */
static int rho(int code, int a) {
  if (is_missing(code)) return 0;
  return (allele_1(code) == a ? 1 : 0) + (allele_2(code) == a ? 1 : 0);
}

int oracle_version(void) { return 1; }

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Per-SNP allele sums s_i^a = sum_q rho_{i,q}(a) and non-missing count n_i. */
void oracle_allele_counts(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld,
                          int64_t *s0, int64_t *s1, int64_t *n_present) {
  int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
  for (i = 0; i < n_v; ++i) {
    int64_t a0 = 0, a1 = 0, np = 0, q;
    for (q = 0; q < n_f; ++q) {
      int c = entry_code(geno, ld, i, q);
      a0 += rho(c, 0);
      a1 += rho(c, 1);
      np += is_missing(c) ? 0 : 1;
    }
    s0[i] = a0;
    s1[i] = a1;
    n_present[i] = np;
  }
}

/* Eq. 1 with n_f read as SNP i's non-missing count. */
static double freq_single(int64_t s, int64_t n) { return n > 0 ? (double)s / (2.0 * (double)n) : 0.0; }

/* One pair i<j: the four tallies and four CCC values (Eqs. 2-3). */
static void pair_metric(const uint64_t *geno, int64_t n_f, int64_t ld, int64_t i, int64_t j,
                        const int64_t *s0, const int64_t *s1, const int64_t *np, double gamma,
                        int norm, int64_t *tally, double *ccc) {
  int64_t r[2][2] = {{0, 0}, {0, 0}};
  int64_t n_ij = 0, q;
  int a, b;
  for (q = 0; q < n_f; ++q) {
    int ci = entry_code(geno, ld, i, q);
    int cj = entry_code(geno, ld, j, q);
    for (a = 0; a < 2; ++a)
      for (b = 0; b < 2; ++b) r[a][b] += (int64_t)rho(ci, a) * rho(cj, b);
    if (!is_missing(ci) && !is_missing(cj)) ++n_ij;
  }
  for (a = 0; a < 2; ++a)
    for (b = 0; b < 2; ++b) tally[2 * a + b] = r[a][b];
  if (n_ij == 0) {
    for (a = 0; a < 4; ++a) ccc[a] = 0.0;
    return;
  }
  double fi[2], fj[2];
  if (norm == ORACLE_NORM_JOINT) {
    for (a = 0; a < 2; ++a) fi[a] = (double)(r[a][0] + r[a][1]) / (4.0 * (double)n_ij);
    for (b = 0; b < 2; ++b) fj[b] = (double)(r[0][b] + r[1][b]) / (4.0 * (double)n_ij);
  } else {
    fi[0] = freq_single(s0[i], np[i]);
    fi[1] = freq_single(s1[i], np[i]);
    fj[0] = freq_single(s0[j], np[j]);
    fj[1] = freq_single(s1[j], np[j]);
  }
  for (a = 0; a < 2; ++a)
    for (b = 0; b < 2; ++b) {
      double fij = (double)r[a][b] / (4.0 * (double)n_ij);
      ccc[2 * a + b] = fij * (1.0 - gamma * fi[a]) * (1.0 - gamma * fj[b]);
    }
}

/* One triple i<j<k: the eight tallies and eight CCC values (Eqs. 4-5). */
static void triple_metric(const uint64_t *geno, int64_t n_f, int64_t ld, int64_t i, int64_t j,
                          int64_t k, const int64_t *s0, const int64_t *s1, const int64_t *np,
                          double gamma, int norm, int64_t *tally, double *ccc) {
  int64_t r[2][2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
  int64_t n_ijk = 0, q;
  int a, b, c;
  for (q = 0; q < n_f; ++q) {
    int ci = entry_code(geno, ld, i, q);
    int cj = entry_code(geno, ld, j, q);
    int ck = entry_code(geno, ld, k, q);
    for (a = 0; a < 2; ++a)
      for (b = 0; b < 2; ++b)
        for (c = 0; c < 2; ++c) r[a][b][c] += (int64_t)rho(ci, a) * rho(cj, b) * rho(ck, c);
    if (!is_missing(ci) && !is_missing(cj) && !is_missing(ck)) ++n_ijk;
  }
  for (a = 0; a < 2; ++a)
    for (b = 0; b < 2; ++b)
      for (c = 0; c < 2; ++c) tally[4 * a + 2 * b + c] = r[a][b][c];
  if (n_ijk == 0) {
    for (a = 0; a < 8; ++a) ccc[a] = 0.0;
    return;
  }
  double fi[2], fj[2], fk[2];
  if (norm == ORACLE_NORM_JOINT) {
    double d = 8.0 * (double)n_ijk;
    for (a = 0; a < 2; ++a) fi[a] = (double)(r[a][0][0] + r[a][0][1] + r[a][1][0] + r[a][1][1]) / d;
    for (b = 0; b < 2; ++b) fj[b] = (double)(r[0][b][0] + r[0][b][1] + r[1][b][0] + r[1][b][1]) / d;
    for (c = 0; c < 2; ++c) fk[c] = (double)(r[0][0][c] + r[0][1][c] + r[1][0][c] + r[1][1][c]) / d;
  } else {
    fi[0] = freq_single(s0[i], np[i]);
    fi[1] = freq_single(s1[i], np[i]);
    fj[0] = freq_single(s0[j], np[j]);
    fj[1] = freq_single(s1[j], np[j]);
    fk[0] = freq_single(s0[k], np[k]);
    fk[1] = freq_single(s1[k], np[k]);
  }
  for (a = 0; a < 2; ++a)
    for (b = 0; b < 2; ++b)
      for (c = 0; c < 2; ++c) {
        double f = (double)r[a][b][c] / (8.0 * (double)n_ijk);
        ccc[4 * a + 2 * b + c] =
            f * (1.0 - gamma * fi[a]) * (1.0 - gamma * fj[b]) * (1.0 - gamma * fk[c]);
      }
}

typedef struct {
  int64_t *s0, *s1, *np;
} snp_counts;

static int counts_alloc(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, snp_counts *sc) {
  sc->s0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_v > 0 ? n_v : 1));
  sc->s1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_v > 0 ? n_v : 1));
  sc->np = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_v > 0 ? n_v : 1));
  if (!sc->s0 || !sc->s1 || !sc->np) return -1;
  oracle_allele_counts(geno, n_f, n_v, ld, sc->s0, sc->s1, sc->np);
  return 0;
}

static void counts_free(snp_counts *sc) {
  free(sc->s0);
  free(sc->s1);
  free(sc->np);
}

/*
 * 2-way, by rows: for every listed i, all j in (i, n_v) in increasing order.
 * tally[.][4] and ccc[.][4] hold sum over rows of (n_v - 1 - i) entries.
 * Returns 0, or -1 when memory for the per-SNP counts could not be had.
 */
int oracle_ccc2_rows(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld,
                     const int64_t *rows, int64_t n_rows, double gamma, int norm,
                     int64_t *tally, double *ccc) {
  snp_counts sc;
  int64_t *offset, r, t = 0;
  if (counts_alloc(geno, n_f, n_v, ld, &sc)) return -1;
  offset = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_rows + 1));
  if (!offset) {
    counts_free(&sc);
    return -1;
  }
  for (r = 0; r < n_rows; ++r) {
    offset[r] = t;
    t += n_v - 1 - rows[r];
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (r = 0; r < n_rows; ++r) {
    int64_t i = rows[r], j, o = offset[r];
    for (j = i + 1; j < n_v; ++j, ++o)
      pair_metric(geno, n_f, ld, i, j, sc.s0, sc.s1, sc.np, gamma, norm, tally + 4 * o, ccc + 4 * o);
  }
  free(offset);
  counts_free(&sc);
  return 0;
}

/* 2-way, by explicit pairs (pi[t] < pj[t]). */
int oracle_ccc2_pairs(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld,
                      const int64_t *pi, const int64_t *pj, int64_t n_pairs, double gamma,
                      int norm, int64_t *tally, double *ccc) {
  snp_counts sc;
  int64_t t;
  if (counts_alloc(geno, n_f, n_v, ld, &sc)) return -1;
#pragma omp parallel for schedule(dynamic, 64)
  for (t = 0; t < n_pairs; ++t)
    pair_metric(geno, n_f, ld, pi[t], pj[t], sc.s0, sc.s1, sc.np, gamma, norm, tally + 4 * t,
                ccc + 4 * t);
  counts_free(&sc);
  return 0;
}

/*
 * 3-way, by (i, j) rows of a slab: for every listed (i, j) with i < j, all k in
 * (j, n_v) in increasing order; tally[.][8], ccc[.][8].
 */
int oracle_ccc3_rows(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld,
                     const int64_t *ri, const int64_t *rj, int64_t n_rows, double gamma,
                     int norm, int64_t *tally, double *ccc) {
  snp_counts sc;
  int64_t *offset, r, t = 0;
  if (counts_alloc(geno, n_f, n_v, ld, &sc)) return -1;
  offset = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_rows + 1));
  if (!offset) {
    counts_free(&sc);
    return -1;
  }
  for (r = 0; r < n_rows; ++r) {
    offset[r] = t;
    t += n_v - 1 - rj[r];
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (r = 0; r < n_rows; ++r) {
    int64_t i = ri[r], j = rj[r], k, o = offset[r];
    for (k = j + 1; k < n_v; ++k, ++o)
      triple_metric(geno, n_f, ld, i, j, k, sc.s0, sc.s1, sc.np, gamma, norm, tally + 8 * o,
                    ccc + 8 * o);
  }
  free(offset);
  counts_free(&sc);
  return 0;
}

/* 3-way, by explicit triples (pi[t] < pj[t] < pk[t]). */
int oracle_ccc3_triples(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld,
                        const int64_t *pi, const int64_t *pj, const int64_t *pk, int64_t n,
                        double gamma, int norm, int64_t *tally, double *ccc) {
  snp_counts sc;
  int64_t t;
  if (counts_alloc(geno, n_f, n_v, ld, &sc)) return -1;
#pragma omp parallel for schedule(dynamic, 64)
  for (t = 0; t < n; ++t)
    triple_metric(geno, n_f, ld, pi[t], pj[t], pk[t], sc.s0, sc.s1, sc.np, gamma, norm,
                  tally + 8 * t, ccc + 8 * t);
  counts_free(&sc);
  return 0;
}

/*
 * Host twin of the library's result checksum (the paper's extended-precision
 * integer checksum, Sec. 5): C = sum_e h(base + e) * words[e] mod 2^128 over
 * 32-bit words taken as unsigned, h(x) = the SplitMix64 finaliser of
 * (x + 1) * 0x9E3779B97F4A7C15.  out[0] = low 64 bits, out[1] = high.
 */
static uint64_t checksum_hash(uint64_t x) {
  uint64_t z = (x + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void oracle_checksum(const uint32_t *words, int64_t count, int64_t base, uint64_t *out) {
  unsigned __int128 total = 0;
#pragma omp parallel
  {
    unsigned __int128 part = 0;
    int64_t e;
#pragma omp for schedule(static)
    for (e = 0; e < count; ++e)
      part += (unsigned __int128)checksum_hash((uint64_t)(base + e)) * words[e];
#pragma omp critical
    total += part;
  }
  out[0] = (uint64_t)total;
  out[1] = (uint64_t)(total >> 64);
}
