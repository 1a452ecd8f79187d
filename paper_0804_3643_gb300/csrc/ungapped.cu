// ungapped.cu -- stage 2 (Section 3.3.3, the loop of Annex 4) on sm_103a.
//
// Work unit: a TILE = (key, up to 128 consecutive bank-1 occurrences of that
// key).  A CTA builds, in shared memory, the score profile of its bank-1
// windows: prof[k][b][r] = score(nb1[r][k], b) for cell k < 48, residue code
// b < 22 and row r < 128, one signed byte each, rows of one (k, b) 144 bytes
// apart (128 used).  It then streams every bank-2 occurrence of the key
// through the profile.  Lane (g, js) of a warp scores bank-2 row js (4 per
// warp, staged in the warp's shared buffer) against bank-1 rows
// 16g .. 16g+15.  Per cell: one byte load fetches the bank-2 residue, one
// IMAD forms the profile address, one 16-byte load fetches the 16 row scores,
// prmt sign-extends them into eight int16x2 words, and per pair of cells two
// __vadd2 and one __vimax3_s16x2 update each word's running sums and maxima
// (exact: |sum| <= 48 * 32 < 2^15).  After cell 25 the sums restart from the
// maxima (the reset of Annex 4).
//
// Pipe balance on sm_103: byte loads and 16-byte loads go to the LSU, IMAD and
// __vadd2 to the FMA pipe, prmt and the 3-input maxima to the ALU pipe, which
// issues at half the FMA rate and is the bound.  The 8 lanes sharing a bank-2
// row read one 128-byte profile row, so a warp's 512 bytes come out of shared
// memory in the minimum 4 wavefronts; each byte read serves one pair-cell.
//
// Hits (score >= s1) are staged in a per-warp shared buffer and flushed with
// one global atomic per 64 records, as (padded pos1 << sh | padded pos2,
// score).  Tiles come from a device counter (persistent launch, largest tile
// first) or, in the plain schedule, one launch per key.
#include "common.cuh"
#include "ungapped.cuh"

namespace plast {

constexpr int NWARPS = UNG_THREADS / 32;
constexpr int WBUF = 64;
constexpr int PROF_STRIDE = UNG_T1 + 16;                   // bytes per (k, b) profile row
constexpr int PROF_BYTES = WIN * NCODE * PROF_STRIDE;      // 152064
constexpr int TAB_BYTES = 512;                             // int8 [22][22], padded
constexpr int ROWS_BYTES = WIN * UNG_T1;                   // 6144, cell-major
constexpr int STAGE_BYTES = NWARPS * 4 * WIN;              // 6144: 4 bank-2 windows per warp
constexpr int WKEY_BYTES = NWARPS * WBUF * 8;              // 16384
constexpr int WVAL_BYTES = NWARPS * WBUF * 4;              // 8192
constexpr int UNG_SMEM = PROF_BYTES + TAB_BYTES + ROWS_BYTES + STAGE_BYTES + WKEY_BYTES + WVAL_BYTES + 16;
constexpr int ROWS_PER_LANE = UNG_T1 / 8;                  // 16

size_t ungapped_smem_bytes() { return (size_t)UNG_SMEM; }

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

// Cells K and K+1 of one bank-2 window against this lane's 16 bank-1 rows,
// then the following pairs (compile-time recursion over K = 0, 2, .., 46).
template <int K>
__device__ __forceinline__ void cell_pairs(uint32_t row, const unsigned char* plane, uint32_t (&s)[8],
                                           uint32_t (&m)[8]) {
  if constexpr (K < WIN) {
    const uint32_t b0 = lds_u8<K>(row), b1 = lds_u8<K + 1>(row);
    uint32_t u0[8], u1[8];
    unpack16(*reinterpret_cast<const uint4*>(plane + (K * NCODE + b0) * PROF_STRIDE), u0);
    unpack16(*reinterpret_cast<const uint4*>(plane + ((K + 1) * NCODE + b1) * PROF_STRIDE), u1);
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
    cell_pairs<K + 2>(row, plane, s, m);
  }
}

__global__ void __launch_bounds__(UNG_THREADS, 1) k_ungapped(UngArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* prof = smem;
  int8_t* tab = reinterpret_cast<int8_t*>(smem + PROF_BYTES);
  uint8_t* rowsT = smem + PROF_BYTES + TAB_BYTES;
  unsigned char* stage = smem + PROF_BYTES + TAB_BYTES + ROWS_BYTES;
  uint64_t* wkey = reinterpret_cast<uint64_t*>(stage + STAGE_BYTES);
  uint32_t* wval = reinterpret_cast<uint32_t*>(stage + STAGE_BYTES + WKEY_BYTES);
  int* s_tile = reinterpret_cast<int*>(stage + STAGE_BYTES + WKEY_BYTES + WVAL_BYTES);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane & 7, js = lane >> 3;
  uint64_t* my_wk = wkey + warp * WBUF;
  uint32_t* my_wv = wval + warp * WBUF;
  uint4* my_stage = reinterpret_cast<uint4*>(stage + warp * 4 * WIN);  // 12 x 16 bytes
  const uint32_t my_row = (uint32_t)__cvta_generic_to_shared(stage + warp * 4 * WIN + js * WIN);  // lane's window
  int wcnt = 0;  // warp-uniform fill of this warp's buffer

  for (int i = tid; i < NCODE * NCODE; i += UNG_THREADS) tab[i] = c_score[i];
  const uint32_t s1x2 = ((uint32_t)(uint16_t)a.s1 << 16) | (uint16_t)a.s1;

  int iter = 0;
  for (;;) {
    int t;
    if (a.persistent) {
      if (tid == 0) *s_tile = atomicAdd(a.tile_counter, 1);
      __syncthreads();
      t = *s_tile;
    } else {
      t = iter == 0 ? (int)blockIdx.x : a.n_tiles;
    }
    iter++;
    if (t >= a.n_tiles) break;
    const int4 tile = a.tiles[a.tile_base + t];
    const int key = tile.x, rows = tile.z;
    const int64_t u0 = (int64_t)(uint32_t)tile.y;

    // bank-1 windows of the tile, transposed to cell-major (rowsT[k][r])
    for (int i = tid; i < ROWS_BYTES; i += UNG_THREADS) {
      const int r = i & (UNG_T1 - 1), k = i / UNG_T1;
      rowsT[i] = r < rows ? (uint8_t)a.nb1[(u0 + r) * WIN + k] : (uint8_t)SENTINEL;
    }
    __syncthreads();
    // score profile prof[k][b][r], 16 rows per 16-byte item
    for (int e = tid; e < WIN * NCODE * 8; e += UNG_THREADS) {
      const int k = e / (NCODE * 8);
      const int rem = e - k * (NCODE * 8);
      const int b = rem >> 3, gg = rem & 7;
      const uint4 c16 = *reinterpret_cast<const uint4*>(rowsT + k * UNG_T1 + gg * ROWS_PER_LANE);
      const uint32_t src[4] = {c16.x, c16.y, c16.z, c16.w};
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        uint32_t x = 0;
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const int ar = (src[q] >> (8 * r)) & 0xff;
          x |= (uint32_t)(uint8_t)tab[ar * NCODE + b] << (8 * r);
        }
        w[q] = x;
      }
      *reinterpret_cast<uint4*>(prof + (k * NCODE + b) * PROF_STRIDE + gg * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();

    const int64_t v0 = a.key_off2[key], v1 = a.key_off2[key + 1];
    const unsigned char* plane = prof + g * 16;
    // lanes 0..11 fetch the warp's next 4 windows (12 x 16 bytes) one
    // iteration ahead; sentinel windows past the end of the key
    uint4 pre = make_uint4(0x15151515u, 0x15151515u, 0x15151515u, 0x15151515u);
    if (lane < 12) {
      const int64_t v = v0 + warp * 4 + lane / 3;
      if (v < v1) pre = __ldg(reinterpret_cast<const uint4*>(a.nb2 + v * WIN) + lane % 3);
    }
    for (int64_t vb = v0 + warp * 4; vb < v1; vb += NWARPS * 4) {
      const int64_t v = vb + js;
      const bool vok = v < v1;
      __syncwarp();
      if (lane < 12) my_stage[lane] = pre;
      __syncwarp();
      if (lane < 12) {
        const int64_t vn = vb + NWARPS * 4 + lane / 3;
        pre = vn < v1 ? __ldg(reinterpret_cast<const uint4*>(a.nb2 + vn * WIN) + lane % 3)
                      : make_uint4(0x15151515u, 0x15151515u, 0x15151515u, 0x15151515u);
      }
      uint32_t s[8], m[8];
#pragma unroll
      for (int w = 0; w < 8; w++) s[w] = m[w] = 0;
      cell_pairs<0>(my_row, plane, s, m);
      // any row of this lane at or above s1?
      uint32_t mx = __vimax3_s16x2(m[0], m[1], m[2]);
      mx = __vimax3_s16x2(mx, m[3], m[4]);
      mx = __vimax3_s16x2(mx, m[5], m[6]);
      mx = __vmaxs2(mx, m[7]);
      const bool maybe = vok && __vcmpges2(mx, s1x2) != 0u;
      if (__any_sync(0xffffffffu, maybe)) {
        // rows 16g + 2w (low half of m[w]) and 16g + 2w + 1 (high half)
        unsigned mask = 0;
        if (maybe) {
#pragma unroll
          for (int w = 0; w < 8; w++) {
            const uint32_t c = __vcmpges2(m[w], s1x2);
            mask |= ((c & 1u) | ((c >> 15) & 2u)) << (2 * w);
          }
          const int valid_rows = rows - g * ROWS_PER_LANE;
          if (valid_rows < ROWS_PER_LANE) mask &= valid_rows <= 0 ? 0u : ((1u << valid_rows) - 1u);
        }
        const int cnt = __popc(mask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (wcnt + total > WBUF) {
          __syncwarp();
          flush_warp(my_wk, my_wv, wcnt, lane, a.out_count, a.out_key, a.out_val, a.cap);
          __syncwarp();
          wcnt = 0;
        }
        const uint64_t p2 = vok ? (uint64_t)a.pos2[v] : 0;
        if (total > WBUF) {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(a.out_count, (unsigned long long)total);
          base = __shfl_sync(0xffffffffu, base, 0) + (incl - cnt);
#pragma unroll
          for (int i = 0; i < ROWS_PER_LANE; i++)
            if (mask & (1u << i)) {
              const uint64_t p1 = a.pos1[u0 + g * ROWS_PER_LANE + i];
              if ((int64_t)base < a.cap) {
                a.out_key[base] = (p1 << a.sh) | p2;
                a.out_val[base] = (m[i >> 1] >> ((i & 1) * 16)) & 0xffffu;
              }
              base++;
            }
        } else {
          int at = wcnt + incl - cnt;
#pragma unroll
          for (int i = 0; i < ROWS_PER_LANE; i++)
            if (mask & (1u << i)) {
              const uint64_t p1 = a.pos1[u0 + g * ROWS_PER_LANE + i];
              my_wk[at] = (p1 << a.sh) | p2;
              my_wv[at] = (m[i >> 1] >> ((i & 1) * 16)) & 0xffffu;
              at++;
            }
          wcnt += total;
        }
        __syncwarp();
      }
    }
    __syncthreads();  // the next tile rebuilds the profile
  }
  if (wcnt > 0) {
    __syncwarp();
    flush_warp(my_wk, my_wv, wcnt, lane, a.out_count, a.out_key, a.out_val, a.cap);
  }
}

cudaError_t launch_ungapped(const UngArgs& a, int grid, cudaStream_t st) {
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_ungapped, cudaFuncAttributeMaxDynamicSharedMemorySize, UNG_SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  if (grid <= 0) return cudaSuccess;
  note_launch();
  k_ungapped<<<grid, UNG_THREADS, UNG_SMEM, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Survivor expansion: padded coordinates -> (sequence, local position), and
// the exact scalar ungapped score with its extents, recomputed per survivor
// as a self-check of the packed kernel (a mismatch raises *bad).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t find_seq_u(const int64_t* off, int32_t n, int64_t p) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int ungapped_exact(const int8_t* pad1, int64_t p1, const int8_t* pad2, int64_t p2,
                                              int* rl, int* ll) {
  int sum = 0, best = 0, r = 0, l = 0;
  for (int t = 0; t < RIGHT; t++) {
    sum += c_score[pad1[p1 + t] * NCODE + pad2[p2 + t]];
    if (sum > best) {
      best = sum;
      r = t + 1;
    }
  }
  sum = best;
  for (int t = 1; t <= LEFT; t++) {
    sum += c_score[pad1[p1 - t] * NCODE + pad2[p2 - t]];
    if (sum > best) {
      best = sum;
      l = t;
    }
  }
  *rl = r;
  *ll = l;
  return best;
}

__global__ void k_expand_hits(const uint64_t* key, const uint32_t* val, int64_t n, int sh, const int8_t* pad1,
                              const int64_t* pad_off1, int32_t n1, const int8_t* pad2, const int64_t* pad_off2,
                              int32_t n2, plast_hit* out, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p1 = (int64_t)(key[i] >> sh), p2 = (int64_t)(key[i] & ((1ull << sh) - 1));
    int rl, ll;
    int u = ungapped_exact(pad1, p1, pad2, p2, &rl, &ll);
    if (u != (int)(int16_t)(val[i] & 0xffffu)) atomicOr(bad, 2);
    int32_t q1 = find_seq_u(pad_off1, n1, p1), q2 = find_seq_u(pad_off2, n2, p2);
    plast_hit h;
    h.seq1 = q1;
    h.pos1 = (int32_t)(p1 - pad_off1[q1]);
    h.seq2 = q2;
    h.pos2 = (int32_t)(p2 - pad_off2[q2]);
    h.score = (int16_t)u;
    h.rlen = (int8_t)rl;
    h.llen = (int8_t)ll;
    out[i] = h;
  }
}

cudaError_t launch_expand_hits(const uint64_t* key, const uint32_t* val, int64_t n, int sh, const int8_t* pad1,
                               const int64_t* pad_off1, int32_t n1, const int8_t* pad2, const int64_t* pad_off2,
                               int32_t n2, plast_hit* out, int* bad, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  note_launch();
  k_expand_hits<<<(unsigned)b, 256, 0, st>>>(key, val, n, sh, pad1, pad_off1, n1, pad2, pad_off2, n2, out, bad);
  return cudaGetLastError();
}

}  // namespace plast
