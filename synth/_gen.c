/*
 * Fast packed-panel generator: the same counter-based SplitMix64 draws as the
 * numpy definitions in synth/__init__.py, written straight into packed 2-bit
 * words.  Holds no part of the CCC arithmetic.  Per-SNP genotype thresholds
 * (which involve transcendental functions) are computed by the caller in numpy
 * so that both implementations produce identical panels.
 */
#include <stdint.h>

#define G 0x9E3779B97F4A7C15ull

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double unit(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

static uint64_t snp_key(uint64_t seed, int64_t panel, int64_t i) {
  uint64_t kp = mix64(seed + (uint64_t)(panel + 1) * G);
  return mix64(kp + (uint64_t)(i + 1) * G);
}

/* genotype -> code: 0 -> 00, 1 -> 01, 2 -> 11, missing -> 10 */
static const uint64_t kCode[4] = {0u, 1u, 3u, 2u};

/*
 * Rows snp0 .. snp0+n_rows-1 into out[n_rows][ld] (padding words and bits zero).
 * kind 0: uniform genotypes (t0, t1 ignored); kind 1: thresholds t0[r] < t1[r]
 * give genotype 0 below t0, 1 below t1, else 2.
 */
void synth_pack(int kind, int64_t n_rows, int64_t n_f, int64_t ld, uint64_t seed, int64_t panel,
                int64_t snp0, const double *t0, const double *t1, double p_missing,
                uint64_t *out) {
  int64_t r;
#pragma omp parallel for schedule(static)
  for (r = 0; r < n_rows; ++r) {
    const uint64_t key = snp_key(seed, panel, snp0 + r);
    uint64_t *row = out + r * ld;
    int64_t w;
    for (w = 0; w < ld; ++w) row[w] = 0;
    int64_t q;
    for (q = 0; q < n_f; ++q) {
      const double um = unit(mix64(key + (2u * (uint64_t)q + 1u) * G));
      const double ug = unit(mix64(key + (2u * (uint64_t)q + 2u) * G));
      int g;
      if (kind == 0) {
        g = (int)(ug * 3.0);
        if (g > 2) g = 2;
      } else {
        g = ug < t0[r] ? 0 : (ug < t1[r] ? 1 : 2);
      }
      if (um < p_missing) g = 3;
      row[q / 32] |= kCode[g] << (2 * (q % 32));
    }
  }
}

/*
 * Multi-allelic rows (the numpy definition in synth/__init__.py): entry byte
 * x | (y << 4) with x, y drawn from the cumulative state weights c[r][0..s-1]
 * (computed by the caller), 0xFF when missing; padding bytes zero.
 */
void synth_multi(int64_t n_rows, int64_t n_f, int64_t ld, int s, uint64_t seed, int64_t panel,
                 const double *c, double p_missing, uint8_t *out) {
  int64_t r;
#pragma omp parallel for schedule(static)
  for (r = 0; r < n_rows; ++r) {
    const uint64_t key = snp_key(seed, panel, r);
    const double *cr = c + r * s;
    uint8_t *row = out + r * ld;
    int64_t q;
    for (q = n_f; q < ld; ++q) row[q] = 0;
    for (q = 0; q < n_f; ++q) {
      const double um = unit(mix64(key + (3u * (uint64_t)q + 1u) * G));
      const double u1 = unit(mix64(key + (3u * (uint64_t)q + 2u) * G));
      const double u2 = unit(mix64(key + (3u * (uint64_t)q + 3u) * G));
      int x = 0, y = 0, a;
      for (a = 0; a < s; ++a) {
        x += u1 >= cr[a];
        y += u2 >= cr[a];
      }
      if (x > s - 1) x = s - 1;
      if (y > s - 1) y = s - 1;
      row[q] = um < p_missing ? 0xFF : (uint8_t)(x | (y << 4));
    }
  }
}
