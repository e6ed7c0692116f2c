// Multi-allelic 2-way tally launches for s = 9..15 states (the kernel is in
// k_multi.cuh; s = 2..8 are instantiated in k_multi.cu).
#include "k_multi.cuh"

namespace ccc {

int launch_tally2_multi_wide(int s, int64_t n_v, const float *w, int32_t *tally, float *out_ccc,
                             int32_t *status, float gamma, int32_t norm, int32_t group,
                             const uint8_t *op, int64_t rows_pad, int64_t kpad, int num_sms,
                             cudaStream_t st, int64_t i_begin, int64_t i_end, int64_t pair0,
                             int split) {
  CUtensorMap tm;
  if (!tc::make_operand_map(&tm, op, rows_pad, kpad, tcp::BMH)) return CCC_ECUDA;
  MultiArgs a{n_v, w, tally, out_ccc, status, gamma, norm, i_begin, i_end, pair0};
  a.out_len = checked_out_len(pairs_in_rows(n_v, i_begin, i_end));
  const int64_t nB = rows_pad / 256;
  const int nkb = static_cast<int>(kpad / tcp::BK);
  if (split > 1) {
    switch (s) {
      case 9: return launch_tally2_multi_split_s<9>(tm, a, nB, group, nkb, split, num_sms, st);
      case 10: return launch_tally2_multi_split_s<10>(tm, a, nB, group, nkb, split, num_sms, st);
      case 11: return launch_tally2_multi_split_s<11>(tm, a, nB, group, nkb, split, num_sms, st);
      case 12: return launch_tally2_multi_split_s<12>(tm, a, nB, group, nkb, split, num_sms, st);
      case 13: return launch_tally2_multi_split_s<13>(tm, a, nB, group, nkb, split, num_sms, st);
      case 14: return launch_tally2_multi_split_s<14>(tm, a, nB, group, nkb, split, num_sms, st);
      case 15: return launch_tally2_multi_split_s<15>(tm, a, nB, group, nkb, split, num_sms, st);
      default: return CCC_EINVAL;
    }
  }
  switch (s) {
    case 9: return launch_tally2_multi_s<9>(tm, a, nB, group, nkb, num_sms, st);
    case 10: return launch_tally2_multi_s<10>(tm, a, nB, group, nkb, num_sms, st);
    case 11: return launch_tally2_multi_s<11>(tm, a, nB, group, nkb, num_sms, st);
    case 12: return launch_tally2_multi_s<12>(tm, a, nB, group, nkb, num_sms, st);
    case 13: return launch_tally2_multi_s<13>(tm, a, nB, group, nkb, num_sms, st);
    case 14: return launch_tally2_multi_s<14>(tm, a, nB, group, nkb, num_sms, st);
    case 15: return launch_tally2_multi_s<15>(tm, a, nB, group, nkb, num_sms, st);
    default: return CCC_EINVAL;
  }
}

}  // namespace ccc
