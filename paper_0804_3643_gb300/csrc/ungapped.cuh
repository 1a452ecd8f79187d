// ungapped.cuh -- arguments and launchers of the stage-2 kernels (ungapped.cu).
#pragma once
#include "common.cuh"

namespace plast {

// tile shapes (ungapped.cu): UNG_T1 rows (wide), UNG_NT1 = 8, 4 or 2 rows (narrow)
constexpr int UNG_WIDE = 0;
constexpr int UNG_NARROW = 1;
constexpr int UNG_NARROW4 = 2;
constexpr int UNG_NARROW2 = 3;

// A stage-2 tile: x = key | shape << 14 | rows << 16, y = first bank-1 CSR
// index of its rows, [z, w) = the bank-2 windows it scores, as offsets in
// the key's list (a long list may be cut over several tiles).
__host__ __device__ inline int4 make_tile(int key, int first, int rows, int shape, int vlo, int vhi) {
  return make_int4(key | (shape << 14) | (rows << 16), first, vlo, vhi);
}
__host__ __device__ inline int tile_key(const int4& t) { return t.x & 0x3fff; }
__host__ __device__ inline int tile_shape(const int4& t) { return (t.x >> 14) & 3; }
__host__ __device__ inline int tile_rows(const int4& t) { return (t.x >> 16) & 0xff; }

struct UngArgs {
  const int8_t* nb1;        // bank-1 windows [n_idx1][48]
  const uint32_t* pos1;     // bank-1 padded positions, CSR order
  const int8_t* nb2;        // bank-2 windows [n_idx2][48]
  const uint32_t* pos2;     // bank-2 padded positions, CSR order
  const int64_t* key_off2;  // bank-2 CSR offsets [8801]
  const int4* tiles;        // (key, first bank-1 CSR index, rows, shape UNG_WIDE / UNG_NARROW)
  int32_t n_tiles;          // tiles handled by this launch
  int32_t tile_base;        // first tile of this launch in `tiles`
  int32_t* tile_counter;    // persistent schedule: next tile to take
  int32_t persistent;       // 1: CTAs loop on the counter; 0: one tile per CTA
  int32_t s1;               // ungapped threshold
  uint64_t* out_key;        // hit (padded pos1 << sh | padded pos2)
  uint32_t* out_val;        // hit score (int16 in the low half)
  unsigned long long* out_count;
  int64_t cap;              // capacity of out_key / out_val
  int32_t sh;               // bits of a bank-2 padded position
};

// Wide-tile variants of the stage-2 kernel: how many cells the profile holds
// as int16 (UNG_N16 in ungapped.cu: 0, 12, 14, UNG_MAX_N16).
constexpr int UNG_VARIANTS = 4;
constexpr int UNG_MAX_N16 = 16;
int ungapped_variant();            // the variant launch_ungapped runs
int ungapped_variant_n16(int v);   // its int16 cells (-1 for no such variant)
void set_ungapped_variant(int v);  // -1: the default
// wide tiles (the current variant) / narrow tiles, each a persistent launch
cudaError_t launch_ungapped(const UngArgs& a, int grid, cudaStream_t st);
cudaError_t launch_ungapped_narrow(const UngArgs& a, int grid, cudaStream_t st);
constexpr int UNG_NARROW_CTAS_PER_SM = 2;
constexpr int UNG_NARROW_PASS = 512;  // bank-2 windows a narrow CTA scores per pass
cudaError_t launch_expand_hits(const uint64_t* key, const uint32_t* val, int64_t n, int sh, const int8_t* pad1,
                               const int64_t* pad_off1, int32_t n1, const int8_t* pad2, const int64_t* pad_off2,
                               int32_t n2, plast_hit* out, int* bad, cudaStream_t st);

// gapped.cu
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
};
cudaError_t launch_small_gapped(const GapArgs& a, cudaStream_t st);
cudaError_t launch_gapped_compact(const GapArgs& a, const int64_t* at, const int64_t* pad_off1, int32_t n1,
                                  const int64_t* pad_off2, int32_t n2, plast_gapped* out, cudaStream_t st);
// *n_dev = min(*count, cap): the hit count a planned chain feeds forward.
cudaError_t launch_clamp_count(const unsigned long long* count, int64_t cap, int64_t* n_dev, cudaStream_t st);
cudaError_t launch_clamp_total(const int64_t* total, int64_t cap, int64_t* n_dev, cudaStream_t st);
// Record sort of a search: the passing hits' keys and indexes gathered into
// record slots, then (after sorting the pairs by key) the records written in
// key order.
cudaError_t launch_gather_pass(const GapArgs& a, const int64_t* at, uint64_t* rkey, uint32_t* ridx, cudaStream_t st);
cudaError_t launch_write_sorted(const GapArgs& a, const uint64_t* skey, const uint32_t* sidx, int64_t m,
                                const int64_t* m_dev, const int64_t* pad_off1, int32_t n1, const int64_t* pad_off2,
                                int32_t n2, plast_gapped* out, cudaStream_t st);
cudaError_t launch_hits_to_keys(const plast_hit* in, int64_t n, const int64_t* pad_off1, int32_t n1,
                                const int64_t* pad_off2, int32_t n2, int sh, uint64_t* key, uint32_t* val, int* bad,
                                cudaStream_t st);

}  // namespace plast
