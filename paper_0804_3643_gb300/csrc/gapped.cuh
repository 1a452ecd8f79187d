// gapped.cuh -- stage 3.1 and the hit and record writers (gapped.cu).
#pragma once
#include "common.cuh"

namespace plast {

// Padded position -> sequence of a bank: pad_off[s] is sequence s's padded
// start (pad_off[n] = the padded length) and blk[i] the last sequence whose
// padded start is at most i * SEQ_BLK (0 if none).  Every padded sequence
// spans at least GAP bytes, so a block holds at most SEQ_BLK / GAP + 1
// sequence starts and the walk from blk[p / SEQ_BLK] is a few steps.
constexpr int SEQ_BLK = 256;
struct SeqMap {
  const int64_t* pad_off;
  const int32_t* blk;
  int32_t n;
};
__device__ __forceinline__ int32_t seq_of(const SeqMap& m, int64_t p) {
  int32_t s = m.blk[p / SEQ_BLK];
  while (s + 1 < m.n && m.pad_off[s + 1] <= p) s++;
  return s;
}

// Stage-2 survivors (padded pos1 << sh | padded pos2, score) as plast_hit
// records in the given order, the ungapped score recomputed exactly from the
// padded codes as a self-check of the packed kernel (*bad |= 2 on a
// mismatch).
cudaError_t launch_expand_hits(const uint64_t* key, const uint32_t* val, int64_t n, int sh, const int8_t* pad1,
                               const SeqMap& s1, const int8_t* pad2, const SeqMap& s2, plast_hit* out, int* bad,
                               cudaStream_t st);

struct GapArgs {
  const int8_t* pad1;
  const int8_t* pad2;
  const uint64_t* key;      // (padded pos1 << sh | padded pos2) per hit
  const uint32_t* val;      // stage-2 score per hit in the low 16 bits
  int64_t n;
  int32_t sh;
  int32_t gap_open, gap_extend, s2;
  int32_t* score;           // out: small gapped score per hit
  uint32_t* ends;           // out: r_i | r_j << 8 | l_i << 16 | l_j << 24
  int32_t* pass;            // out: score >= s2
  const int64_t* n_dev = nullptr;  // optional device copy of the hit count (<= n)
  int64_t out_cap = INT64_MAX;     // records written only below this index
  // launch_compact_pass: the passing hits appended as (key, hit index) to
  // rkey / ridx in any order (slots below out_cap), their number added to
  // *rcount
  uint64_t* rkey = nullptr;
  uint32_t* ridx = nullptr;
  unsigned long long* rcount = nullptr;
};
cudaError_t launch_small_gapped(const GapArgs& a, cudaStream_t st);
cudaError_t launch_gapped_compact(const GapArgs& a, const int64_t* at, const SeqMap& s1, const SeqMap& s2,
                                  plast_gapped* out, cudaStream_t st);
// *n_dev = min(*count, cap): the hit count a planned chain feeds forward.
cudaError_t launch_clamp_count(const unsigned long long* count, int64_t cap, int64_t* n_dev, cudaStream_t st);
// Record sort of a search: the passing hits' keys and indexes compacted,
// then (after sorting the pairs by key) the records written in key order.
cudaError_t launch_compact_pass(const GapArgs& a, cudaStream_t st);
cudaError_t launch_write_sorted(const GapArgs& a, const uint64_t* skey, const uint32_t* sidx, int64_t m,
                                const int64_t* m_dev, const SeqMap& s1, const SeqMap& s2, plast_gapped* out,
                                cudaStream_t st);
cudaError_t launch_hits_to_keys(const plast_hit* in, int64_t n, const int64_t* pad_off1, int32_t n1,
                                const int64_t* pad_off2, int32_t n2, int sh, uint64_t* key, uint32_t* val, int* bad,
                                cudaStream_t st);

}  // namespace plast
