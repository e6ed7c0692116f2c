// Host enumeration of the 2-way tile orders, for checks without a GPU.
//
// usage: sched_order KIND n_v I0 I1 group clusters
//   KIND 0: square 128-SNP tiles (TriSchedPair, shift 0); 1: 128 x 120-SNP
//   tiles (RectSchedT<128, 120, 240>); 2, 3: the s-state tiles of 8 PW x 6 PW
//   markers for s = 4 (PW = 8) and s = 3 (PW = 10) (RectSchedT<8 PW, 6 PW, 192>).
//   Cluster c of `clusters` visits the tiles start = c, c + clusters, ... as
//   the persistent kernels do; one line "c I J" per visit, clusters in turn.
#include <cstdio>
#include <cstdlib>

#include "tc_sched.cuh"

using namespace ccc;

template <class S>
static void run(const TriSched::Params &p, int clusters) {
  for (int c = 0; c < clusters; ++c) {
    S s;
    for (s.init(p, c); s.valid; s.advance(clusters)) std::printf("%d %d %d\n", c, s.I, s.J);
  }
}

int main(int argc, char **argv) {
  if (argc != 7) return 2;
  const int kind = std::atoi(argv[1]);
  const long long n_v = std::atoll(argv[2]);
  TriSched::Params p;
  const int snpi = kind <= 1 ? 128 : kind == 2 ? 64 : 80;
  const int snpj = kind == 0 ? 128 : kind == 1 ? 120 : kind == 2 ? 48 : 60;
  p.nI = static_cast<int>((n_v + snpi - 1) / snpi);
  p.nJ = static_cast<int>((n_v + snpj - 1) / snpj);
  p.I0 = std::atoi(argv[3]);
  p.I1 = std::atoi(argv[4]);
  p.group = std::atoi(argv[5]);
  p.shift = 0;
  const int clusters = std::atoi(argv[6]);
  if (kind == 0)
    run<TriSchedPair>(p, clusters);
  else if (kind == 1)
    run<RectSchedT<128, 120, 240>>(p, clusters);
  else if (kind == 2)
    run<RectSchedT<64, 48, 192>>(p, clusters);
  else
    run<RectSchedT<80, 60, 192>>(p, clusters);
  return 0;
}
