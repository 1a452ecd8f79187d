// ungapped.cuh -- arguments and launchers of the stage-2 kernels (ungapped.cu).
#pragma once
#include "common.cuh"

namespace plast {

// tile shapes (ungapped.cu): UNG_T1 rows (wide); 8, 4, 2 or 16 rows (narrow)
constexpr int UNG_WIDE = 0;
constexpr int UNG_NARROW = 1;
constexpr int UNG_NARROW4 = 2;
constexpr int UNG_NARROW2 = 3;
constexpr int UNG_NARROW16 = 4;
constexpr int UNG_SHAPES = 5;

// A stage-2 tile: x = key | shape << 14 | rows << 17, y = first bank-1 CSR
// index of its rows, [z, w) = the bank-2 windows it scores, as offsets in
// the key's list (a long list may be cut over several tiles).
__host__ __device__ inline int4 make_tile(int key, int first, int rows, int shape, int vlo, int vhi) {
  return make_int4(key | (shape << 14) | (rows << 17), first, vlo, vhi);
}
__host__ __device__ inline int tile_key(const int4& t) { return t.x & 0x3fff; }
__host__ __device__ inline int tile_shape(const int4& t) { return (t.x >> 14) & 7; }
__host__ __device__ inline int tile_rows(const int4& t) { return (t.x >> 17) & 0xff; }

struct UngArgs {
  const int8_t* nb1;        // bank-1 windows [n_idx1][48]
  const uint32_t* pos1;     // bank-1 padded positions, CSR order
  const int8_t* nb2;        // bank-2 windows [n_idx2][48]
  const uint32_t* pos2;     // bank-2 padded positions, CSR order
  const int64_t* key_off2;  // bank-2 CSR offsets [8801]
  const int4* tiles;        // make_tile: key, first bank-1 CSR index, rows, shape, bank-2 range
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
// as int16 (UNG_N16 in ungapped.cu: 0, 12, 14, UNG_MAX_N16) and how many
// passes ahead the bank-2 windows are fetched (the staging depth, 1 or 2).
constexpr int UNG_N16_VARIANTS = 4;
constexpr int UNG_VARIANTS = 2 * UNG_N16_VARIANTS;
constexpr int UNG_MAX_N16 = 16;
int ungapped_variant();              // the variant launch_ungapped runs
int ungapped_variant_n16(int v);     // its int16 cells (-1 for no such variant)
int ungapped_variant_depth(int v);   // its staging depth (-1 for no such variant)
void set_ungapped_variant(int v);    // -1: the default
// wide tiles (the current variant) / narrow tiles, each a persistent launch
cudaError_t launch_ungapped(const UngArgs& a, int grid, cudaStream_t st);
cudaError_t launch_ungapped_narrow(const UngArgs& a, int grid, cudaStream_t st);
constexpr int UNG_NARROW_CTAS_PER_SM = 2;
constexpr int UNG_NARROW_PASS = 512;  // bank-2 windows a narrow CTA scores per pass
}  // namespace plast
