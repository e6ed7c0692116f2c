// Host enumeration of the 2-way tile orders, for checks without a GPU.
//
// usage: sched_order KIND n_v I0 I1 group clusters
//   KIND 0: square 128-SNP tiles (TriSchedPair, shift 0), 1: 128 x 120-SNP
//   tiles (RectSchedT<120>).  Cluster c of `clusters` visits the tiles
//   start = c, c + clusters, ... as the persistent kernels do; one line
//   "c I J" per visit, clusters in turn.
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
  const int snpj = kind == 0 ? 128 : 120;
  p.nI = static_cast<int>((n_v + 127) / 128);
  p.nJ = static_cast<int>((n_v + snpj - 1) / snpj);
  p.I0 = std::atoi(argv[3]);
  p.I1 = std::atoi(argv[4]);
  p.group = std::atoi(argv[5]);
  p.shift = 0;
  const int clusters = std::atoi(argv[6]);
  if (kind == 0)
    run<TriSchedPair>(p, clusters);
  else
    run<RectSchedT<120>>(p, clusters);
  return 0;
}
