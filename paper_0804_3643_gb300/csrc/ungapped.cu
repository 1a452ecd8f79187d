// ungapped.cu -- stage 2 (Section 3.3.3, the loop of Annex 4) on sm_103a.
//
// Work unit: a TILE = (key, consecutive bank-1 occurrences of that key, shape).
// A CTA builds, in shared memory, the score profile of its bank-1 windows:
// prof[k][b][r] = score(nb1[r][k], b) for cell k < 48, residue code b < 22 and
// tile row r, one signed byte each.  It then streams every bank-2 occurrence
// of the key through the profile.  Per cell a lane loads the bank-2 residue
// (one byte), forms the profile address (one IMAD) and loads its rows' scores
// (one vector load); prmt sign-extends them into int16x2 words, and per pair
// of cells two __vadd2 and one __vimax3_s16x2 update each word's running sums
// and maxima (exact: |sum| <= 48 * 32 < 2^15).  After cell 25 the sums restart
// from the maxima (the reset of Annex 4).
//
// Two tile shapes, each in its own persistent kernel (k_ungapped<N16>,
// k_ungapped_narrow), launched one after the other over the work list:
//  * wide: up to 128 rows.  Lane (g, js) of a warp scores bank-2 window js
//    (4 per warp) against rows 16g .. 16g+15; the 8 lanes of a window read
//    one 128-byte profile row per cell, so a warp's loads come out of shared
//    memory in the minimum number of wavefronts.  Two refinements:
//    - the seed cells.  Positions 1 and 4 of the subset seed have one class
//      per residue (Section 3.3.1), so cells 0 and 3 pair a bank-1 residue
//      with itself and score the diagonal entry d0, d3 > 0 of the row.  The
//      profile folds them into cells 1 and 2: P1 = d0 + s(a1, b),
//      M1 = d0 + max(0, s(a1, b)), P2 = s(a2, b) + d3, and the window starts
//      from sum = P1[b1] + P2[b2] = S3 and max = max(M1[b1], S3), which are
//      the running sum after cell 3 and max(0, S0, S1, S2, S3) (S2 < S3, the
//      empty prefix and S0 are dominated).
//    - N16 of the cells are stored as int16 (two 16-byte loads, no
//      sign extension), trading shared-memory bandwidth, which has headroom,
//      for ALU-pipe work, which has none; the rest are int8.
//  * narrow: up to R = 16, 8, 4 or 2 rows.  Every lane scores its own bank-2
//    window (32 per warp) against the R rows: the profile holds one word per
//    (k, b) and 4 rows (R / 4 planes for R >= 8), or one halfword per (k, b)
//    and 2 rows; the 22 entries of a cell lie in distinct banks, so 32 lanes
//    with any residues read them in one wavefront.  16- and 8-row tiles take
//    the lanes' windows through shared memory; 4- and 2-row tiles, which do too little
//    arithmetic per cell to hide a shared byte load, keep each lane's window
//    in registers.  Narrow tiles serve short lists (a small query bank
//    against a large one, the remainder of a long list), where a wide tile
//    would mostly score padding rows.
// The host picks the shape per key from measured per-cell and per-tile costs.
//
// Pipe balance on sm_103: byte and vector loads go to the LSU, IMAD and
// __vadd2 to the FMA pipe, prmt and the 3-input maxima to the ALU pipe, which
// is the bound.
//
// Hits (score >= s1) are staged in a per-warp shared buffer of 32 records
// and flushed with one global atomic per buffer, as (padded pos1 << sh |
// padded pos2, score).  Tiles come from a device counter (persistent launches, costliest
// tile first) or, in the plain schedule, one launch per key and shape.
#include <atomic>

#include "common.cuh"
#include "ungapped.cuh"

namespace plast {

constexpr int NWARPS = UNG_THREADS / 32;
constexpr int WBUF = 32;
constexpr int PROF_STRIDE = UNG_T1 + 16;                   // bytes per (k, b) row of an int8 plane
constexpr int PROF16_STRIDE = 2 * UNG_T1 + 32;             // bytes per (k, b) row of an int16 plane
constexpr int PLANE8 = NCODE * PROF_STRIDE;                // 3168
constexpr int PLANE16 = NCODE * PROF16_STRIDE;             // 6336
constexpr int SEED_PLANES = 3;                             // P1, M1, P2 (cells 0-3)
constexpr int FIRST_CELL = 4;                              // first cell after the seed
constexpr int TAB_BYTES = 512;                             // int8 [22][22], padded
constexpr int T24_STRIDE = 24;                             // bytes per residue a of the word table
constexpr int T24_BYTES = 544;                             // int8 [22][24] (b = 22, 23 zero), padded
constexpr int ROWS_BYTES = WIN * UNG_T1;                   // 6144, cell-major; shares the staging area
constexpr int WSTAGE_BYTES = NWARPS * 4 * WIN;             // 4 bank-2 windows per warp
constexpr int STAGE_BYTES = WSTAGE_BYTES > WIN * UNG_T1 ? WSTAGE_BYTES : WIN * UNG_T1;  // also the tile's rows
constexpr int WKEY_BYTES = NWARPS * WBUF * 8;              // 8192
constexpr int WVAL_BYTES = NWARPS * WBUF * 4;              // 4096
static_assert(ROWS_BYTES <= STAGE_BYTES, "the tile's bank-1 rows fit the staging area");
constexpr int ROWS_PER_LANE = UNG_T1 / 8;                  // 16

// Wide-tile profile with N16 int16 cells (cells 4 .. 4 + N16 - 1):
// int8 planes P1, M1, P2, then the int8 cells; then the int16 cells.
template <int N16>
struct Wide {
  static_assert(N16 % 2 == 0 && N16 >= 0 && N16 <= WIN - FIRST_CELL, "int16 cells come in pairs");
  static constexpr int N8 = SEED_PLANES + (WIN - FIRST_CELL - N16);
  static constexpr int BASE16 = N8 * PLANE8;
  static constexpr int PROF = BASE16 + N16 * PLANE16;
  static constexpr int SMEM = PROF + TAB_BYTES + T24_BYTES + STAGE_BYTES + WKEY_BYTES + WVAL_BYTES + 2 * 48;
  __host__ __device__ static constexpr bool is16(int k) { return k >= FIRST_CELL && k < FIRST_CELL + N16; }
  // int8 plane of cell k >= FIRST_CELL + N16
  __host__ __device__ static constexpr int plane8(int k) { return SEED_PLANES + (k - FIRST_CELL - N16); }
};

// narrow tiles (their own kernel)
constexpr int NSTRIDE = 52;                                // staged window stride: 13 words, conflict-free bytes
constexpr int NPLANE = WIN * NCODE * 4;                     // 4224: one plane of 4 rows
constexpr int NR_MAX = 16;                                  // rows of the largest narrow tile
constexpr int NPROF_BYTES = (NR_MAX / 4) * NPLANE;          // 16896
constexpr int NROWS_BYTES = WIN * NR_MAX;                   // 768, cell-major
constexpr int NT_THREADS = 512;                            // narrow kernel: 2 CTAs of 16 warps per SM
constexpr int NT_WARPS = NT_THREADS / 32;
constexpr int NSTAGE_BYTES = NT_WARPS * 32 * NSTRIDE;      // 26624: one window per lane
constexpr int NWKEY_BYTES = NT_WARPS * WBUF * 8;           // 4096
constexpr int NWVAL_BYTES = NT_WARPS * WBUF * 4;           // 2048
static_assert(UNG_NARROW_PASS == NT_WARPS * 32, "narrow pass = one window per lane");
static_assert(NPROF_BYTES % 16 == 0 && NROWS_BYTES % 16 == 0 && (32 * NSTRIDE) % 16 == 0, "alignment");
static_assert(Wide<UNG_MAX_N16>::SMEM <= 232448, "shared memory per CTA");

// bytes 2h, 2h+1 of x, sign-extended into the two halves of an int16x2
__device__ __forceinline__ uint32_t sext_pair(uint32_t x, int h) {
  uint32_t r;
  if (h == 0) asm("prmt.b32 %0, %1, 0, 0x9180;" : "=r"(r) : "r"(x));
  else asm("prmt.b32 %0, %1, 0, 0xB3A2;" : "=r"(r) : "r"(x));
  return r;
}

__device__ __forceinline__ void unpack16(const uint4& p, uint32_t (&u)[8]) {
  u[0] = sext_pair(p.x, 0);
  u[1] = sext_pair(p.x, 1);
  u[2] = sext_pair(p.y, 0);
  u[3] = sext_pair(p.y, 1);
  u[4] = sext_pair(p.z, 0);
  u[5] = sext_pair(p.z, 1);
  u[6] = sext_pair(p.w, 0);
  u[7] = sext_pair(p.w, 1);
}

__device__ __forceinline__ void unpack8(uint32_t lo, uint32_t hi, uint32_t (&u)[4]) {
  u[0] = sext_pair(lo, 0);
  u[1] = sext_pair(lo, 1);
  u[2] = sext_pair(hi, 0);
  u[3] = sext_pair(hi, 1);
}

__device__ __forceinline__ void flush_warp(const uint64_t* wk, const uint32_t* wv, int n, int lane,
                                           unsigned long long* out_count, uint64_t* out_key, uint32_t* out_val,
                                           int64_t cap) {
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(out_count, (unsigned long long)n);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int i = lane; i < n; i += 32) {
    unsigned long long d = base + i;
    if ((int64_t)d < cap) {
      out_key[d] = wk[i];
      out_val[d] = wv[i];
    }
  }
}

// The lane's 16 row scores of wide cell K against bank-2 residue b, as eight
// int16x2 words (rows 2w, 2w+1 in word w).  plane = profile + 16 g.
template <int K, int N16>
__device__ __forceinline__ void wide_scores(const unsigned char* plane, uint32_t b, uint32_t (&u)[8]) {
  if constexpr (Wide<N16>::is16(K)) {
    // rows 16g .. 16g+7 at 16g, rows 16g+8 .. 16g+15 at 128 + 16g
    const unsigned char* e = plane + Wide<N16>::BASE16 + (K - FIRST_CELL) * PLANE16 + b * PROF16_STRIDE;
    const uint4 lo = *reinterpret_cast<const uint4*>(e);
    const uint4 hi = *reinterpret_cast<const uint4*>(e + 128);
    u[0] = lo.x;
    u[1] = lo.y;
    u[2] = lo.z;
    u[3] = lo.w;
    u[4] = hi.x;
    u[5] = hi.y;
    u[6] = hi.z;
    u[7] = hi.w;
  } else {
    unpack16(*reinterpret_cast<const uint4*>(plane + Wide<N16>::plane8(K) * PLANE8 + b * PROF_STRIDE), u);
  }
}

// Cells K and K+1 of one bank-2 window against the lane's 16 wide rows, then
// the following pairs (compile-time recursion over K = 4, 6, .., 46).
template <int K, int N16>
__device__ __forceinline__ void wide_pairs(uint32_t row, const unsigned char* plane, uint32_t (&s)[8],
                                           uint32_t (&m)[8]) {
  if constexpr (K < WIN) {
    const uint32_t b0 = lds_u8<K>(row), b1 = lds_u8<K + 1>(row);
    uint32_t u0[8], u1[8];
    wide_scores<K, N16>(plane, b0, u0);
    wide_scores<K + 1, N16>(plane, b1, u1);
#pragma unroll
    for (int w = 0; w < 8; w++) {
      const uint32_t t0 = __vadd2(s[w], u0[w]);
      s[w] = __vadd2(t0, u1[w]);
      m[w] = __vimax3_s16x2(m[w], t0, s[w]);
    }
    if constexpr (K + 1 == RIGHT - 1) {  // the reset of Annex 4
#pragma unroll
      for (int w = 0; w < 8; w++) s[w] = m[w];
    }
    wide_pairs<K + 2, N16>(row, plane, s, m);
  }
}

// The lane's 2 * NW narrow row scores of cell k against bank-2 residue b,
// as NW int16x2 words.  NW >= 2: rows 4p .. 4p+3 the word at
// plane + p * NPLANE + (k * NCODE + b) * 4, p < NW / 2; NW = 1: rows 0-1 the
// halfword at plane + (k * NCODE + b) * 2.
template <int NW>
__device__ __forceinline__ void narrow_scores(const unsigned char* plane, int k, uint32_t b, uint32_t (&u)[NW]) {
  if constexpr (NW == 1) {
    uint32_t h;
    asm("ld.shared.u16 %0, [%1];"
        : "=r"(h)
        : "r"((uint32_t)__cvta_generic_to_shared(plane + (k * NCODE + b) * 2)));
    u[0] = sext_pair(h, 0);
  } else {
    const unsigned char* e = plane + (k * NCODE + b) * 4;
#pragma unroll
    for (int p = 0; p < NW / 2; p++) {
      const uint32_t x = *reinterpret_cast<const uint32_t*>(e + p * NPLANE);
      u[2 * p] = sext_pair(x, 0);
      u[2 * p + 1] = sext_pair(x, 1);
    }
  }
}

template <int K, int NW>
__device__ __forceinline__ void narrow_pairs(uint32_t row, const unsigned char* plane, uint32_t (&s)[NW],
                                             uint32_t (&m)[NW]) {
  if constexpr (K < WIN) {
    const uint32_t b0 = lds_u8<K>(row), b1 = lds_u8<K + 1>(row);
    uint32_t u0[NW], u1[NW];
    narrow_scores<NW>(plane, K, b0, u0);
    narrow_scores<NW>(plane, K + 1, b1, u1);
#pragma unroll
    for (int w = 0; w < NW; w++) {
      const uint32_t t0 = __vadd2(s[w], u0[w]);
      s[w] = __vadd2(t0, u1[w]);
      m[w] = __vimax3_s16x2(m[w], t0, s[w]);
    }
    if constexpr (K + 1 == RIGHT - 1) {
#pragma unroll
      for (int w = 0; w < NW; w++) s[w] = m[w];
    }
    narrow_pairs<K + 2, NW>(row, plane, s, m);
  }
}

// The same with the lane's window in registers (cell k = byte k of win).
template <int K, int NW>
__device__ __forceinline__ void narrow_pairs_reg(const uint32_t (&win)[12], const unsigned char* plane,
                                                 uint32_t (&s)[NW], uint32_t (&m)[NW]) {
  if constexpr (K < WIN) {
    const uint32_t b0 = (win[K >> 2] >> (8 * (K & 3))) & 0xffu;
    const uint32_t b1 = (win[(K + 1) >> 2] >> (8 * ((K + 1) & 3))) & 0xffu;
    uint32_t u0[NW], u1[NW];
    narrow_scores<NW>(plane, K, b0, u0);
    narrow_scores<NW>(plane, K + 1, b1, u1);
#pragma unroll
    for (int w = 0; w < NW; w++) {
      const uint32_t t0 = __vadd2(s[w], u0[w]);
      s[w] = __vadd2(t0, u1[w]);
      m[w] = __vimax3_s16x2(m[w], t0, s[w]);
    }
    if constexpr (K + 1 == RIGHT - 1) {
#pragma unroll
      for (int w = 0; w < NW; w++) s[w] = m[w];
    }
    narrow_pairs_reg<K + 2, NW>(win, plane, s, m);
  }
}

// The lane's rows whose score reaches s1, as a mask with row 4q + j (half
// j & 1 of word 2q + (j >> 1)) at bit 8j + q.  m - s1 is exact in int16
// (-32 <= m <= 48 * 11: m starts at or above the folded seed cell M1 >= -32;
// |s1| <= 30000), so the sign bit of a half is clear where the row reaches
// s1; one prmt gathers the four sign bits of two words.
template <int NW>
__device__ __forceinline__ uint32_t hit_mask(const uint32_t (&m)[NW], uint32_t s1x2) {
  if constexpr (NW == 1) {
    const uint32_t x = ~__vsub2(m[0], s1x2);
    return ((x >> 15) & 0x1u) | ((x >> 23) & 0x100u);
  } else {
    uint32_t mask = 0;
#pragma unroll
    for (int q = 0; q < NW / 2; q++) {
      const uint32_t p = ~__byte_perm(__vsub2(m[2 * q], s1x2), __vsub2(m[2 * q + 1], s1x2), 0x7531u);
      mask |= (p >> (7 - q)) & (0x01010101u << q);  // bits 7, 15, 23, 31: rows 4q .. 4q + 3
    }
    return mask;
  }
}

// m[w] for a run-time w, by a select tree (no indexed register array).
template <int NW>
__device__ __forceinline__ uint32_t pick_word(const uint32_t (&m)[NW], int w) {
  uint32_t v[NW];
#pragma unroll
  for (int i = 0; i < NW; i++) v[i] = m[i];
#pragma unroll
  for (int st = 1; st < NW; st <<= 1) {
    const bool hi = (w & st) != 0;
#pragma unroll
    for (int i = 0; i < NW; i += 2 * st) v[i] = hi ? v[i + st] : v[i];
  }
  return v[0];
}

// Records the rows of this lane whose score reaches s1 against bank-2
// occurrence v: rows r0 + i for i < 2 * NW (row 2w in the low half of m[w],
// row 2w + 1 in the high half), of which the first valid_rows exist.  A warp
// with no hit leaves after one vote; otherwise each lane walks its own set
// bits, and the lanes' slots in the warp buffer come from one ballot when no
// lane has more than one hit (the usual case), else from a shuffle scan.
template <int NW>
__device__ __forceinline__ void emit_hits(const uint32_t (&m)[NW], bool vok, int valid_rows, int64_t r0, int64_t v,
                                          const UngArgs& a, uint32_t s1x2, int lane, uint64_t* my_wk,
                                          uint32_t* my_wv, int& wcnt) {
  uint32_t mx = m[0];
  if constexpr (NW == 8) {
    mx = __vimax3_s16x2(m[0], m[1], m[2]);
    mx = __vimax3_s16x2(mx, m[3], m[4]);
    mx = __vimax3_s16x2(mx, m[5], m[6]);
    mx = __vmaxs2(mx, m[7]);
  } else if constexpr (NW == 4) {
    mx = __vimax3_s16x2(m[0], m[1], m[2]);
    mx = __vmaxs2(mx, m[3]);
  } else if constexpr (NW == 2) {
    mx = __vmaxs2(m[0], m[1]);
  }
  const bool maybe = vok && __vcmpges2(mx, s1x2) != 0u;
  if (!__any_sync(0xffffffffu, maybe)) return;
  uint32_t mask = 0;
  if (maybe) {
    mask = hit_mask<NW>(m, s1x2);
    if (valid_rows < 2 * NW) {
      uint32_t keep = 0;
#pragma unroll
      for (int r = 0; r < 2 * NW; r++)
        if (r < valid_rows) keep |= 1u << (8 * (r & 3) + (r >> 2));
      mask &= keep;
    }
  }
  const int cnt = __popc(mask);
  const unsigned with = __ballot_sync(0xffffffffu, cnt != 0);
  int excl, total;
  if (__ballot_sync(0xffffffffu, cnt > 1) == 0u) {
    excl = __popc(with & ((1u << lane) - 1u));
    total = __popc(with);
  } else {
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    excl = incl - cnt;
    total = __shfl_sync(0xffffffffu, incl, 31);
  }
  if (total == 0) return;
  if (wcnt + total > WBUF) {
    __syncwarp();
    flush_warp(my_wk, my_wv, wcnt, lane, a.out_count, a.out_key, a.out_val, a.cap);
    __syncwarp();
    wcnt = 0;
  }
  const uint64_t p2 = vok ? (uint64_t)a.pos2[v] : 0;
  int64_t at;  // this lane's first slot: in the warp buffer, or global when too many for it
  if (total > WBUF) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.out_count, (unsigned long long)total);
    at = (int64_t)__shfl_sync(0xffffffffu, base, 0) + excl;
  } else {
    at = wcnt + excl;
  }
  while (mask) {
    const int b = __ffs(mask) - 1;
    mask &= mask - 1u;
    const int r = 4 * (b & 7) + (b >> 3);
    const uint32_t wv = pick_word<NW>(m, r >> 1);
    const uint64_t key = ((uint64_t)a.pos1[r0 + r] << a.sh) | p2;
    const uint32_t val = (r & 1) ? (wv >> 16) : (wv & 0xffffu);
    if (total > WBUF) {
      if (at < a.cap) {
        a.out_key[at] = key;
        a.out_val[at] = val;
      }
    } else {
      my_wk[at] = key;
      my_wv[at] = val;
    }
    at++;
  }
  if (total <= WBUF) wcnt += total;
  __syncwarp();
}

// The next tile of a CTA, read by one thread while the CTA works on the
// current one.
struct TileSlot {
  int4 tile;       // the tile (make_tile)
  int64_t v0, v1;  // its bank-2 CSR range
  int t;           // tile index (>= n_tiles: none left)
};
static_assert(sizeof(TileSlot) <= 48, "tile slot size");

__device__ __forceinline__ void fetch_tile(const UngArgs& a, int t, TileSlot* slot) {
  slot->t = t;
  if (t < a.n_tiles) {
    const int4 tl = a.tiles[a.tile_base + t];
    const int64_t base = a.key_off2[tile_key(tl)];
    slot->tile = tl;
    slot->v0 = base + tl.z;
    slot->v1 = base + tl.w;
  }
}

// Four rows against four residue codes: out[j] byte r = score(byte r of
// rows4, 4 * b4 + j).  Four word loads from the [22][24] table (row a holds
// score(a, b) for b = 0 .. 21 and two zero bytes) and a 4 x 4 byte transpose.
__device__ __forceinline__ void score4x4(const uint32_t* t24, uint32_t rows4, int b4, uint32_t (&out)[4]) {
  const uint32_t r0 = t24[__byte_perm(rows4, 0u, 0x4440u) * (T24_STRIDE / 4) + b4];
  const uint32_t r1 = t24[__byte_perm(rows4, 0u, 0x4441u) * (T24_STRIDE / 4) + b4];
  const uint32_t r2 = t24[__byte_perm(rows4, 0u, 0x4442u) * (T24_STRIDE / 4) + b4];
  const uint32_t r3 = t24[__byte_perm(rows4, 0u, 0x4443u) * (T24_STRIDE / 4) + b4];
  const uint32_t t0 = __byte_perm(r0, r1, 0x5140u), t1 = __byte_perm(r0, r1, 0x7362u);
  const uint32_t t2 = __byte_perm(r2, r3, 0x5140u), t3 = __byte_perm(r2, r3, 0x7362u);
  out[0] = __byte_perm(t0, t2, 0x5410u);
  out[1] = __byte_perm(t0, t2, 0x7632u);
  out[2] = __byte_perm(t1, t3, 0x5410u);
  out[3] = __byte_perm(t1, t3, 0x7632u);
}

// Four rows: byte r of the result is score(byte r of src, b).
__device__ __forceinline__ uint32_t pack4(uint32_t src, const int8_t* tab, int b) {
  uint32_t x = 0;
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const int ar = (src >> (8 * r)) & 0xff;
    x |= (uint32_t)(uint8_t)tab[ar * NCODE + b] << (8 * r);
  }
  return x;
}

// A narrow tile of 2 * NW rows: rows cell-major (nrows[k][r], stride
// NR_MAX), the profile (NW >= 2: planes nprof[p][k][b] of rows 4p .. 4p+3,
// p < NW / 2; NW = 1: halfwords of rows 0-1; cells 0-3 folded into P1, M1,
// P2 as in the wide tiles), then every bank-2 window of the key against it,
// one per lane.
template <int NW>
__device__ __forceinline__ void narrow_tile(const UngArgs& a, int rows, int64_t u0, int64_t v0, int64_t v1,
                                            uint8_t* nrows, unsigned char* nprof, const int8_t* tab,
                                            unsigned char* my_nstage, uint32_t my_nrow, uint32_t s1x2,
                                            uint64_t* my_wk, uint32_t* my_wv, int& wcnt) {
  constexpr int NQ = NW >= 2 ? NW / 2 : 1;  // 4-row words per (cell, residue)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint4 sent16 = make_uint4(0x15151515u, 0x15151515u, 0x15151515u, 0x15151515u);
  // only the first 4 * NQ bytes of each cell's row slot are written here; the
  // rest of the slot (up to NR_MAX) may hold a previous, larger tile's rows,
  // which the profile build below reads with its 16-byte load but never uses
  // (it takes the words sx[q], q < NQ, only)
  for (int i = tid; i < WIN * 4 * NQ; i += NT_THREADS) {
    const int r = i % (4 * NQ), k = i / (4 * NQ);
    nrows[k * NR_MAX + r] = r < rows ? (uint8_t)a.nb1[(u0 + r) * WIN + k] : (uint8_t)SENTINEL;
  }
  __syncthreads();
  // cells 4 .. 47 at their own slots; slots 0, 1, 2 hold the folded seed
  // planes P1, M1, P2 (as in the wide tiles); slot 3 is unused
  for (int e = tid; e < WIN * NCODE; e += NT_THREADS) {
    const int k = e / NCODE, b = e - k * NCODE;
    if (k == 3) continue;
    const uint4 cx = *reinterpret_cast<const uint4*>(nrows + (k < 3 ? (k == 2 ? 2 : 1) : k) * NR_MAX);
    const uint32_t sx[4] = {cx.x, cx.y, cx.z, cx.w};
    uint32_t w[NQ];
    if (k >= FIRST_CELL) {
#pragma unroll
      for (int q = 0; q < NQ; q++) w[q] = pack4(sx[q], tab, b);
    } else {
      const uint4 cd = *reinterpret_cast<const uint4*>(nrows + (k == 2 ? 3 : 0) * NR_MAX);
      const uint32_t sd[4] = {cd.x, cd.y, cd.z, cd.w};
#pragma unroll
      for (int q = 0; q < NQ; q++) {
        uint32_t x = 0;
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const int ax = (sx[q] >> (8 * r)) & 0xff, ad = (sd[q] >> (8 * r)) & 0xff;
          int v = tab[ax * NCODE + b];
          if (k == 1) v = max(v, 0);
          v += tab[ad * NCODE + ad];
          x |= (uint32_t)(uint8_t)(int8_t)v << (8 * r);
        }
        w[q] = x;
      }
    }
    if constexpr (NW == 1) {
      *reinterpret_cast<uint16_t*>(nprof + e * 2) = (uint16_t)(w[0] & 0xffffu);
    } else {
#pragma unroll
      for (int q = 0; q < NQ; q++) *reinterpret_cast<uint32_t*>(nprof + q * NPLANE + e * 4) = w[q];
    }
  }
  __syncthreads();

  // window indexes relative to the key's first (32-bit arithmetic)
  if constexpr (NW <= 2) {
    // 2 or 4 rows: few operations per cell, so the lane's own window stays in
    // registers (three 16-byte loads, one iteration ahead) and each cell's
    // residue is a byte of it, not a shared-memory load
    const int n2 = (int)(v1 - v0);
    const uint4* src = reinterpret_cast<const uint4*>(a.nb2 + v0 * WIN);
    uint4 cur[3];
    {
      const int v = warp * 32 + lane;
#pragma unroll
      for (int j = 0; j < 3; j++) cur[j] = v < n2 ? __ldg(src + (int64_t)v * 3 + j) : sent16;
    }
    for (int vb = warp * 32; vb < n2; vb += NT_WARPS * 32) {
      const bool vok = vb + lane < n2;
      uint4 nxt[3];
      {
        const int vn = vb + NT_WARPS * 32 + lane;
#pragma unroll
        for (int j = 0; j < 3; j++) nxt[j] = vn < n2 ? __ldg(src + (int64_t)vn * 3 + j) : sent16;
      }
      const uint32_t win[12] = {cur[0].x, cur[0].y, cur[0].z, cur[0].w, cur[1].x, cur[1].y,
                                cur[1].z, cur[1].w, cur[2].x, cur[2].y, cur[2].z, cur[2].w};
      uint32_t s[NW], m[NW];
      {  // cells 0-3 from the folded seed planes
        const uint32_t bs1 = (win[0] >> 8) & 0xffu, bs2 = (win[0] >> 16) & 0xffu;
        uint32_t up[NW], uq[NW];
        narrow_scores<NW>(nprof, 0, bs1, up);
        narrow_scores<NW>(nprof, 2, bs2, uq);
#pragma unroll
        for (int w = 0; w < NW; w++) s[w] = __vadd2(up[w], uq[w]);
        narrow_scores<NW>(nprof, 1, bs1, up);
#pragma unroll
        for (int w = 0; w < NW; w++) m[w] = __vmaxs2(up[w], s[w]);
      }
      narrow_pairs_reg<FIRST_CELL, NW>(win, nprof, s, m);
      emit_hits<NW>(m, vok, rows, u0, v0 + vb + lane, a, s1x2, lane, my_wk, my_wv, wcnt);
#pragma unroll
      for (int j = 0; j < 3; j++) cur[j] = nxt[j];
    }
    return;
  }
  // the warp's 32 windows are 96 consecutive 16-byte items; lane l moves
  // items l, l + 32, l + 64 (window q / 3, part q % 3), one iteration ahead
  int nw[3], np[3];
#pragma unroll
  for (int j = 0; j < 3; j++) {
    nw[j] = (lane + 32 * j) / 3;
    np[j] = (lane + 32 * j) % 3;
  }
  // window indexes relative to the key's first (32-bit arithmetic)
  const int n2 = (int)(v1 - v0);
  const uint4* src = reinterpret_cast<const uint4*>(a.nb2 + v0 * WIN);
  uint4 pre[3];
#pragma unroll
  for (int j = 0; j < 3; j++) {
    const int v = warp * 32 + nw[j];
    pre[j] = v < n2 ? __ldg(src + (int64_t)v * 3 + np[j]) : sent16;
  }
  for (int vb = warp * 32; vb < n2; vb += NT_WARPS * 32) {
    const bool vok = vb + lane < n2;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 3; j++) {
      uint32_t* d = reinterpret_cast<uint32_t*>(my_nstage + nw[j] * NSTRIDE + np[j] * 16);
      d[0] = pre[j].x;
      d[1] = pre[j].y;
      d[2] = pre[j].z;
      d[3] = pre[j].w;
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 3; j++) {
      const int vn = vb + NT_WARPS * 32 + nw[j];
      pre[j] = vn < n2 ? __ldg(src + (int64_t)vn * 3 + np[j]) : sent16;
    }
    uint32_t s[NW], m[NW];
    {  // cells 0-3 from the folded seed planes
      const uint32_t bs1 = lds_u8<1>(my_nrow), bs2 = lds_u8<2>(my_nrow);
      uint32_t up[NW], uq[NW];
      narrow_scores<NW>(nprof, 0, bs1, up);
      narrow_scores<NW>(nprof, 2, bs2, uq);
#pragma unroll
      for (int w = 0; w < NW; w++) s[w] = __vadd2(up[w], uq[w]);
      narrow_scores<NW>(nprof, 1, bs1, up);
#pragma unroll
      for (int w = 0; w < NW; w++) m[w] = __vmaxs2(up[w], s[w]);
    }
    narrow_pairs<FIRST_CELL, NW>(my_nrow, nprof, s, m);
    emit_hits<NW>(m, vok, rows, u0, v0 + vb + lane, a, s1x2, lane, my_wk, my_wv, wcnt);
  }
}

template <int N16, int DEPTH>
__global__ void __launch_bounds__(UNG_THREADS, 1) k_ungapped(UngArgs a) {
  using L = Wide<N16>;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* prof = smem;
  int8_t* tab = reinterpret_cast<int8_t*>(smem + L::PROF);
  uint32_t* t24 = reinterpret_cast<uint32_t*>(smem + L::PROF + TAB_BYTES);
  unsigned char* stage = smem + L::PROF + TAB_BYTES + T24_BYTES;
  uint8_t* rowsT = stage;  // the tile's bank-1 rows while its profile is built
  uint64_t* wkey = reinterpret_cast<uint64_t*>(stage + STAGE_BYTES);
  uint32_t* wval = reinterpret_cast<uint32_t*>(stage + STAGE_BYTES + WKEY_BYTES);
  TileSlot* slots = reinterpret_cast<TileSlot*>(stage + STAGE_BYTES + WKEY_BYTES + WVAL_BYTES);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane & 7, js = lane >> 3;
  uint64_t* my_wk = wkey + warp * WBUF;
  uint32_t* my_wv = wval + warp * WBUF;
  uint4* my_stage = reinterpret_cast<uint4*>(stage + warp * 4 * WIN);  // 12 x 16 bytes
  const uint32_t my_row = (uint32_t)__cvta_generic_to_shared(stage + warp * 4 * WIN + js * WIN);  // lane's window
  int wcnt = 0;  // warp-uniform fill of this warp's buffer
  const uint4 sent16 = make_uint4(0x15151515u, 0x15151515u, 0x15151515u, 0x15151515u);

  for (int i = tid; i < NCODE * NCODE; i += UNG_THREADS) tab[i] = c_score[i];
  for (int i = tid; i < NCODE * T24_STRIDE; i += UNG_THREADS) {
    const int aa = i / T24_STRIDE, b = i - aa * T24_STRIDE;
    reinterpret_cast<int8_t*>(t24)[i] = b < NCODE ? c_score[aa * NCODE + b] : (int8_t)0;
  }
  const uint32_t s1x2 = ((uint32_t)(uint16_t)a.s1 << 16) | (uint16_t)a.s1;

  // tiles: from the device counter (persistent) or this CTA's own; thread 0
  // fetches the next one into the other slot while the CTA works
  if (tid == 0) fetch_tile(a, a.persistent ? atomicAdd(a.tile_counter, 1) : (int)blockIdx.x, &slots[0]);
  __syncthreads();
  for (int buf = 0;; buf ^= 1) {
    if (slots[buf].t >= a.n_tiles) break;
    const int4 tile = slots[buf].tile;
    const int64_t v0 = slots[buf].v0, v1 = slots[buf].v1;
    if (tid == 0) fetch_tile(a, a.persistent ? atomicAdd(a.tile_counter, 1) : a.n_tiles, &slots[buf ^ 1]);
    const int rows = tile_rows(tile);
    const int64_t u0 = (int64_t)(uint32_t)tile.y;

    {
      // bank-1 windows of the tile, transposed to cell-major (rowsT[k][r])
      for (int i = tid; i < ROWS_BYTES; i += UNG_THREADS) {
        const int r = i & (UNG_T1 - 1), k = i / UNG_T1;
        rowsT[i] = r < rows ? (uint8_t)a.nb1[(u0 + r) * WIN + k] : (uint8_t)SENTINEL;
      }
      __syncthreads();
      // seed planes: 16 rows per 16-byte item, one residue code b per item
      // P1 = d0 + s(a1, b), M1 = d0 + max(0, s(a1, b)), P2 = s(a2, b) + d3
      for (int e = tid; e < SEED_PLANES * NCODE * 8; e += UNG_THREADS) {
        const int p = e / (NCODE * 8);
        const int rem = e - p * (NCODE * 8);
        const int b = rem >> 3, gg = rem & 7;
        const int kx = p == 2 ? 2 : 1, kd = p == 2 ? 3 : 0;
        const uint4 cx = *reinterpret_cast<const uint4*>(rowsT + kx * UNG_T1 + gg * ROWS_PER_LANE);
        const uint4 cd = *reinterpret_cast<const uint4*>(rowsT + kd * UNG_T1 + gg * ROWS_PER_LANE);
        const uint32_t sx[4] = {cx.x, cx.y, cx.z, cx.w}, sd[4] = {cd.x, cd.y, cd.z, cd.w};
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          uint32_t x = 0;
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const int ax = (sx[q] >> (8 * r)) & 0xff, ad = (sd[q] >> (8 * r)) & 0xff;
            int v = tab[ax * NCODE + b];
            if (p == 1) v = max(v, 0);
            v += tab[ad * NCODE + ad];
            x |= (uint32_t)(uint8_t)(int8_t)v << (8 * r);
          }
          w[q] = x;
        }
        *reinterpret_cast<uint4*>(prof + p * PLANE8 + b * PROF_STRIDE + gg * 16) = make_uint4(w[0], w[1], w[2], w[3]);
      }
      // the other planes: 16 rows x 4 residue codes per item, by 4 x 4 transposes
      constexpr int NB4 = (NCODE + 3) / 4;  // 6 groups of 4 codes
      constexpr int N8C = L::N8 - SEED_PLANES;
      for (int e = tid; e < (N8C + N16) * NB4 * 8; e += UNG_THREADS) {
        const int c = e / (NB4 * 8);
        const int rem = e - c * (NB4 * 8);
        const int b4 = rem >> 3, gg = rem & 7;
        const bool i16 = c >= N8C;  // int16 cells first in the cell order, last in this loop
        const int k = i16 ? FIRST_CELL + (c - N8C) : FIRST_CELL + N16 + c;
        const uint4 c16 = *reinterpret_cast<const uint4*>(rowsT + k * UNG_T1 + gg * ROWS_PER_LANE);
        uint32_t o[4][4];  // o[q][j]: rows 4q .. 4q+3 of the group against code 4 * b4 + j
        score4x4(t24, c16.x, b4, o[0]);
        score4x4(t24, c16.y, b4, o[1]);
        score4x4(t24, c16.z, b4, o[2]);
        score4x4(t24, c16.w, b4, o[3]);
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int b = 4 * b4 + j;
          if (b >= NCODE) break;
          if (!i16) {
            *reinterpret_cast<uint4*>(prof + (SEED_PLANES + c) * PLANE8 + b * PROF_STRIDE + gg * 16) =
                make_uint4(o[0][j], o[1][j], o[2][j], o[3][j]);
          } else {
            // int16: rows 0-7 of the group at 16 gg, rows 8-15 128 bytes further
            unsigned char* d = prof + L::BASE16 + (c - N8C) * PLANE16 + b * PROF16_STRIDE + gg * 16;
            *reinterpret_cast<uint4*>(d) = make_uint4(sext_pair(o[0][j], 0), sext_pair(o[0][j], 1),
                                                      sext_pair(o[1][j], 0), sext_pair(o[1][j], 1));
            *reinterpret_cast<uint4*>(d + 128) = make_uint4(sext_pair(o[2][j], 0), sext_pair(o[2][j], 1),
                                                            sext_pair(o[3][j], 0), sext_pair(o[3][j], 1));
          }
        }
      }
      __syncthreads();

      const unsigned char* plane = prof + g * 16;
      // lanes 0..11 fetch the warp's next 4 windows (12 x 16 bytes) DEPTH
      // iterations ahead; sentinel windows past the end of the key.  Window
      // indexes are relative to the key's first (32-bit arithmetic).
      const int n2 = (int)(v1 - v0), lw = lane / 3;
      const uint4* src = reinterpret_cast<const uint4*>(a.nb2 + v0 * WIN) + lane % 3;
      // (DEPTH passes ahead: the staging depth the autotuner picks)
      uint4 pre[DEPTH];
#pragma unroll
      for (int d = 0; d < DEPTH; d++) {
        const int vn = warp * 4 + d * NWARPS * 4 + lw;
        pre[d] = lane < 12 && vn < n2 ? __ldg(src + (int64_t)vn * 3) : sent16;
      }
      for (int vb = warp * 4; vb < n2; vb += NWARPS * 4) {
        const bool vok = vb + js < n2;
        __syncwarp();
        if (lane < 12) my_stage[lane] = pre[0];
        __syncwarp();
        if (lane < 12) {
#pragma unroll
          for (int d = 0; d + 1 < DEPTH; d++) pre[d] = pre[d + 1];
          const int vn = vb + DEPTH * NWARPS * 4 + lw;
          pre[DEPTH - 1] = vn < n2 ? __ldg(src + (int64_t)vn * 3) : sent16;
        }
        uint32_t s[8], m[8];
        {  // cells 0-3 from the folded seed planes
          const uint32_t bs1 = lds_u8<1>(my_row), bs2 = lds_u8<2>(my_row);
          uint32_t up[8], uq[8];
          unpack16(*reinterpret_cast<const uint4*>(plane + bs1 * PROF_STRIDE), up);
          unpack16(*reinterpret_cast<const uint4*>(plane + 2 * PLANE8 + bs2 * PROF_STRIDE), uq);
#pragma unroll
          for (int w = 0; w < 8; w++) s[w] = __vadd2(up[w], uq[w]);
          unpack16(*reinterpret_cast<const uint4*>(plane + PLANE8 + bs1 * PROF_STRIDE), up);
#pragma unroll
          for (int w = 0; w < 8; w++) m[w] = __vmaxs2(up[w], s[w]);
        }
        wide_pairs<FIRST_CELL, N16>(my_row, plane, s, m);
        emit_hits<8>(m, vok, rows - g * ROWS_PER_LANE, u0 + g * ROWS_PER_LANE, v0 + vb + js, a, s1x2, lane, my_wk,
                     my_wv, wcnt);
      }
    }
    __syncthreads();  // the next tile rebuilds the profile
  }
  if (wcnt > 0) {
    __syncwarp();
    flush_warp(my_wk, my_wv, wcnt, lane, a.out_count, a.out_key, a.out_val, a.cap);
  }
}

// Narrow tiles (16, 8, 4 or 2 rows) in their own persistent kernel, so that the
// wide kernel's registers and schedule are its own; two CTAs of 512 threads
// per SM, so that one CTA's tile changes (profile build, barriers) overlap
// the other's scoring.
constexpr int NARROW_SMEM = TAB_BYTES + NROWS_BYTES + NPROF_BYTES + NSTAGE_BYTES + NWKEY_BYTES + NWVAL_BYTES + 2 * 48;
static_assert((TAB_BYTES + NROWS_BYTES + NPROF_BYTES + NSTAGE_BYTES) % 16 == 0, "alignment");
static_assert(2 * NARROW_SMEM <= 228 * 1024, "two narrow CTAs per SM");

__global__ void __launch_bounds__(NT_THREADS, 2) k_ungapped_narrow(UngArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  int8_t* tab = reinterpret_cast<int8_t*>(smem);
  uint8_t* nrows = smem + TAB_BYTES;
  unsigned char* nprof = smem + TAB_BYTES + NROWS_BYTES;
  unsigned char* nstage = smem + TAB_BYTES + NROWS_BYTES + NPROF_BYTES;
  uint64_t* wkey = reinterpret_cast<uint64_t*>(nstage + NSTAGE_BYTES);
  uint32_t* wval = reinterpret_cast<uint32_t*>(nstage + NSTAGE_BYTES + NWKEY_BYTES);
  TileSlot* slots = reinterpret_cast<TileSlot*>(nstage + NSTAGE_BYTES + NWKEY_BYTES + NWVAL_BYTES);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t* my_wk = wkey + warp * WBUF;
  uint32_t* my_wv = wval + warp * WBUF;
  unsigned char* my_nstage = nstage + warp * 32 * NSTRIDE;
  const uint32_t my_nrow = (uint32_t)__cvta_generic_to_shared(my_nstage + lane * NSTRIDE);
  int wcnt = 0;

  for (int i = tid; i < NCODE * NCODE; i += NT_THREADS) tab[i] = c_score[i];
  const uint32_t s1x2 = ((uint32_t)(uint16_t)a.s1 << 16) | (uint16_t)a.s1;
  if (tid == 0) fetch_tile(a, a.persistent ? atomicAdd(a.tile_counter, 1) : (int)blockIdx.x, &slots[0]);
  __syncthreads();
  for (int buf = 0;; buf ^= 1) {
    if (slots[buf].t >= a.n_tiles) break;
    const int4 tile = slots[buf].tile;
    const int64_t v0 = slots[buf].v0, v1 = slots[buf].v1;
    if (tid == 0) fetch_tile(a, a.persistent ? atomicAdd(a.tile_counter, 1) : a.n_tiles, &slots[buf ^ 1]);
    const int rows = tile_rows(tile);
    const int64_t u0 = (int64_t)(uint32_t)tile.y;
    const int shape = tile_shape(tile);
    if (shape == UNG_NARROW16)
      narrow_tile<8>(a, rows, u0, v0, v1, nrows, nprof, tab, my_nstage, my_nrow, s1x2, my_wk, my_wv, wcnt);
    else if (shape == UNG_NARROW)
      narrow_tile<4>(a, rows, u0, v0, v1, nrows, nprof, tab, my_nstage, my_nrow, s1x2, my_wk, my_wv, wcnt);
    else if (shape == UNG_NARROW4)
      narrow_tile<2>(a, rows, u0, v0, v1, nrows, nprof, tab, my_nstage, my_nrow, s1x2, my_wk, my_wv, wcnt);
    else
      narrow_tile<1>(a, rows, u0, v0, v1, nrows, nprof, tab, my_nstage, my_nrow, s1x2, my_wk, my_wv, wcnt);
    __syncthreads();  // the next tile rebuilds the profile
  }
  if (wcnt > 0) {
    __syncwarp();
    flush_warp(my_wk, my_wv, wcnt, lane, a.out_count, a.out_key, a.out_val, a.cap);
  }
}

namespace {
std::atomic<int> g_variant{-1};  // index into the variants (-1: the default)
constexpr int UNG_N16[UNG_N16_VARIANTS] = {0, 12, 14, UNG_MAX_N16};
constexpr int UNG_DEFAULT_VARIANT = 1;  // 12 int16 cells, one pass ahead

template <int N16, int DEPTH>
cudaError_t launch_variant(const UngArgs& a, int grid, cudaStream_t st) {
  static std::atomic<bool> attr_set[64];  // per device; calls may come from several threads
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e =
        cudaFuncSetAttribute(k_ungapped<N16, DEPTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, Wide<N16>::SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  if (grid <= 0) return cudaSuccess;
  note_launch();
  k_ungapped<N16, DEPTH><<<grid, UNG_THREADS, Wide<N16>::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int DEPTH>
cudaError_t launch_depth(int n16v, const UngArgs& a, int grid, cudaStream_t st) {
  switch (n16v) {
    case 0:
      return launch_variant<UNG_N16[0], DEPTH>(a, grid, st);
    case 1:
      return launch_variant<UNG_N16[1], DEPTH>(a, grid, st);
    case 3:
      return launch_variant<UNG_N16[3], DEPTH>(a, grid, st);
    default:
      return launch_variant<UNG_N16[2], DEPTH>(a, grid, st);
  }
}
}  // namespace

int ungapped_variant() {
  const int v = g_variant.load();
  return v < 0 ? UNG_DEFAULT_VARIANT : v;
}

// variant v: int16 cells UNG_N16[v % 4], staging depth 1 + v / 4
int ungapped_variant_n16(int v) { return v >= 0 && v < UNG_VARIANTS ? UNG_N16[v % UNG_N16_VARIANTS] : -1; }
int ungapped_variant_depth(int v) { return v >= 0 && v < UNG_VARIANTS ? 1 + v / UNG_N16_VARIANTS : -1; }

void set_ungapped_variant(int v) { g_variant.store(v); }

cudaError_t launch_ungapped_narrow(const UngArgs& a, int grid, cudaStream_t st) {
  static std::atomic<bool> attr_set[64];  // per device; calls may come from several threads
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_ungapped_narrow, cudaFuncAttributeMaxDynamicSharedMemorySize, NARROW_SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  if (grid <= 0) return cudaSuccess;
  note_launch();
  k_ungapped_narrow<<<grid, NT_THREADS, NARROW_SMEM, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ungapped(const UngArgs& a, int grid, cudaStream_t st) {
  const int v = ungapped_variant();
  return ungapped_variant_depth(v) == 2 ? launch_depth<2>(v % UNG_N16_VARIANTS, a, grid, st)
                                        : launch_depth<1>(v % UNG_N16_VARIANTS, a, grid, st);
}

}  // namespace plast
