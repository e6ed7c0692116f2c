// Tile order over the upper triangle of a Gram product, shared by the 2-way
// tally kernels (biallelic and multi-allelic), and its K-split form.  The
// triangle orders are host-callable too, so that their coverage can be
// checked without a GPU.
#pragma once

#include "tc_pipeline.cuh"

namespace ccc {
namespace {

// Upper-triangle tiles: I = 64-SNP row block, J = 128-SNP column block,
// J >= I/2 (the first column block holding a j > every i of the row block),
// in groups of `group` column blocks, rows inside a group in increasing order.
struct TriSched {
  struct Params {
    int nI, nJ, group;
    int I0, I1;  // row blocks [I0, I1) (a phase); 0, nI for the whole triangle
    int shift;   // row block I needs column blocks J >= I >> shift (1: 64/128-SNP, 0: square)
  };
  int nI, nJ, nG, G, I0, sh;
  int g, I, J, col_end, row_end;
  bool valid;

  __host__ __device__ void set_group() {
    col_end = min((g + 1) * G, nJ);
    row_end = min(nI, col_end << sh);
  }
  // From group g on, the first group holding a row >= I0; rows start at I0.
  __host__ __device__ void enter_group() {
    while (g < nG) {
      set_group();
      if (I0 < row_end) {
        I = I0;
        J = max(g * G, I >> sh);
        return;
      }
      ++g;
    }
    valid = false;
  }
  __host__ __device__ void init(const Params &p, int64_t start) {
    nI = min(p.nI, p.I1);
    nJ = p.nJ;
    G = p.group;
    I0 = p.I0;
    sh = p.shift;
    nG = (nJ + G - 1) / G;
    valid = nI > I0 && nJ > 0;
    g = (I0 >> sh) / G;
    if (valid) enter_group();
    advance(start);
  }
  __host__ __device__ void advance(int64_t step) {
    while (valid && step > 0) {
      const int64_t rem = col_end - 1 - J;
      if (step <= rem) {
        J += static_cast<int>(step);
        return;
      }
      step -= rem + 1;
      if (++I >= row_end) {
        ++g;
        enter_group();
      } else {
        J = max(g * G, I >> sh);
      }
    }
  }
  __host__ __device__ int map_index() const { return 0; }
  __host__ __device__ int k_blocks(int nkb) const { return nkb; }
  __host__ __device__ int k_begin() const { return 0; }
  __host__ __device__ int a_row() const { return I * tc::BM; }
  __host__ __device__ int b_row() const { return J * tc::BN; }
};

// 256 x 256 tiles on pairs of SMs: I, J count 256-row blocks.
struct TriSchedPair : TriSched {
  __host__ __device__ int a_row() const { return I * 256; }
  __host__ __device__ int b_row() const { return J * 256; }
};

// Upper-triangle tiles of SNPI-SNP row blocks I (256 operand rows, A rows
// 256 I ..) by SNPJ-SNP column blocks J (NB operand rows, B rows NB J ..): the
// narrow-tile FP4 SM-pair kernels (biallelic thresholded: 128 x 120 SNPs,
// NB = 240; s-state markers: 8 PW x 6 PW markers, NB = 192).  A tile holds a
// pair i < j iff its last j exceeds its first i: SNPJ J + SNPJ - 1 > SNPI I,
// i.e. J >= jmin(I) = ceil((SNPI I - SNPJ + 2) / SNPJ).  Order as TriSched:
// groups of `group` column blocks, rows inside a group in increasing order, row
// blocks [I0, I1) only.
template <int SNPI, int SNPJ, int NB>
struct RectSchedT {
  using Params = TriSched::Params;  // nI, nJ, group, I0, I1 (shift unused)
  int nI, nJ, nG, G, I0;
  int g, I, J, col_end, row_end;
  bool valid;

  __host__ __device__ static int jmin(int I) {
    const int x = SNPI * I - SNPJ + 2;
    return x <= 0 ? 0 : (x + SNPJ - 1) / SNPJ;
  }
  // One past the last row block with a column block below col_end.
  __host__ __device__ static int rows_below(int col_end) {
    return (SNPJ * (col_end - 1) + SNPJ - 2) / SNPI + 1;
  }
  __host__ __device__ void set_group() {
    col_end = min((g + 1) * G, nJ);
    row_end = min(nI, rows_below(col_end));
  }
  __host__ __device__ void enter_group() {
    while (g < nG) {
      set_group();
      if (I0 < row_end) {
        I = I0;
        J = max(g * G, jmin(I));
        return;
      }
      ++g;
    }
    valid = false;
  }
  __host__ __device__ void init(const Params &p, int64_t start) {
    nI = min(p.nI, p.I1);
    nJ = p.nJ;
    G = p.group;
    I0 = p.I0;
    nG = (nJ + G - 1) / G;
    valid = nI > I0 && nJ > 0;
    g = jmin(I0) / G;
    if (valid) enter_group();
    advance(start);
  }
  __host__ __device__ void advance(int64_t step) {
    while (valid && step > 0) {
      const int64_t rem = col_end - 1 - J;
      if (step <= rem) {
        J += static_cast<int>(step);
        return;
      }
      step -= rem + 1;
      if (++I >= row_end) {
        ++g;
        enter_group();
      } else {
        J = max(g * G, jmin(I));
      }
    }
  }
  __host__ __device__ int map_index() const { return 0; }
  __host__ __device__ int k_blocks(int nkb) const { return nkb; }
  __host__ __device__ int k_begin() const { return 0; }
  __host__ __device__ int a_row() const { return I * 256; }
  __host__ __device__ int b_row() const { return J * NB; }
};

// Tiles of RectSchedT<SNPI, SNPJ, NB> over nI row and nJ column blocks, row
// blocks [I0, I1) (the host's grid size; the same count the schedule visits).
template <class Rect>
inline int64_t rect_tiles(int nI, int nJ, int I0, int I1) {
  int64_t t = 0;
  for (int I = I0; I < nI && I < I1; ++I) {
    const int jm = Rect::jmin(I);
    if (jm < nJ) t += nJ - jm;
  }
  return t;
}

// Units of a K-split launch, part-major: unit u = (tile u % tiles, part
// u / tiles); part p takes the K stages [p nkb / split, (p + 1) nkb / split)
// of its tile (the host keeps split <= nkb, so no part is empty).  A wave of
// units then covers every tile of a few parts: the tiles that share a row
// block read the same K range at the same time, so its operand blocks come
// from L2 after the first read (tile-major order ran the parts of one tile
// side by side, which share nothing).
struct SplitSchedPair {
  struct Params {
    TriSched::Params tri;
    int split, nkb;
    int64_t tiles;  // tiles of the triangle (or of the row range)
  };
  TriSched::Params tri;
  TriSchedPair t;
  int split, nkb, part, I, J;
  int64_t u, tiles;
  bool valid;

  __device__ void set_unit() {
    valid = u < tiles * split;
    if (!valid) return;
    part = static_cast<int>(u / tiles);
    t.init(tri, u % tiles);
    valid = t.valid;
    I = t.I;
    J = t.J;
  }
  __device__ void init(const Params &p, int64_t start) {
    tri = p.tri;
    split = p.split;
    nkb = p.nkb;
    tiles = p.tiles;
    u = start;
    set_unit();
  }
  __device__ void advance(int64_t step) {
    u += step;
    set_unit();
  }
  __device__ int map_index() const { return 0; }
  __device__ int k_begin() const {
    return static_cast<int>(static_cast<int64_t>(part) * nkb / split);
  }
  __device__ int k_blocks(int) const {
    return static_cast<int>(static_cast<int64_t>(part + 1) * nkb / split) - k_begin();
  }
  __device__ int a_row() const { return t.a_row(); }
  __device__ int b_row() const { return t.b_row(); }
};

}  // namespace
}  // namespace ccc
