// ungapped.cu -- stage 2 (Section 3.3.3, the loop of Annex 4) on sm_103a.
//
// Work unit: a TILE = (key, up to 64 consecutive bank-1 occurrences of that
// key).  A CTA builds, in shared memory, the score profile of its 64 bank-1
// windows: prof[k][b][r] = score(nb1[r][k], b) for cell k < 48, residue code
// b < 22 and row r < 64, as int16 (135 KB).  It then streams every bank-2
// occurrence of the key through the profile.  Lane (g, js) of a warp scores
// bank-2 row js (4 per warp) against bank-1 rows 8g .. 8g+7: per cell, one
// 16-byte shared load fetches the 8 row scores and four __vadd2 / __vmaxs2
// pairs update 8 running sums and maxima (int16x2, exact: |sum| <= 48*32).
// After cell 25 the sums restart from the maxima (the reset of Annex 4).
//
// The 8 lanes sharing a bank-2 row read one 128-byte profile row, so the 32
// lanes' 512 bytes come out of shared memory in the minimum 4 wavefronts.
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
constexpr int PROF_BYTES = WIN * NCODE * UNG_T1 * 2;       // 135168
constexpr int TAB_BYTES = 1024;                            // int16 [22][22], padded
constexpr int ROWS_BYTES = WIN * UNG_T1;                   // 3072, cell-major
constexpr int WKEY_BYTES = NWARPS * WBUF * 8;              // 16384
constexpr int WVAL_BYTES = NWARPS * WBUF * 4;              // 8192
constexpr int UNG_SMEM = PROF_BYTES + TAB_BYTES + ROWS_BYTES + WKEY_BYTES + WVAL_BYTES + 16;

size_t ungapped_smem_bytes() { return (size_t)UNG_SMEM; }

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

__global__ void __launch_bounds__(UNG_THREADS, 1) k_ungapped(UngArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint4* prof4 = reinterpret_cast<uint4*>(smem);
  int16_t* tab = reinterpret_cast<int16_t*>(smem + PROF_BYTES);
  uint8_t* rowsT = smem + PROF_BYTES + TAB_BYTES;
  uint64_t* wkey = reinterpret_cast<uint64_t*>(smem + PROF_BYTES + TAB_BYTES + ROWS_BYTES);
  uint32_t* wval = reinterpret_cast<uint32_t*>(smem + PROF_BYTES + TAB_BYTES + ROWS_BYTES + WKEY_BYTES);
  int* s_tile = reinterpret_cast<int*>(smem + PROF_BYTES + TAB_BYTES + ROWS_BYTES + WKEY_BYTES + WVAL_BYTES);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane & 7, js = lane >> 3;
  uint64_t* my_wk = wkey + warp * WBUF;
  uint32_t* my_wv = wval + warp * WBUF;
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
      int r = i & (UNG_T1 - 1), k = i >> 6;
      rowsT[i] = r < rows ? (uint8_t)a.nb1[(u0 + r) * WIN + k] : (uint8_t)SENTINEL;
    }
    __syncthreads();
    // score profile prof[k][b][r], 8 rows per 16-byte item
    for (int e = tid; e < WIN * NCODE * 8; e += UNG_THREADS) {
      int k = e / (NCODE * 8);
      int rem = e - k * (NCODE * 8);
      int b = rem >> 3, gg = rem & 7;
      uint2 c8 = *reinterpret_cast<const uint2*>(rowsT + k * UNG_T1 + gg * 8);
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        uint32_t lo = c8.x, hi = c8.y;
        uint32_t src = q < 2 ? lo : hi;
        int a0 = (src >> ((q & 1) * 16)) & 0xff;
        int a1 = (src >> ((q & 1) * 16 + 8)) & 0xff;
        w[q] = (uint32_t)(uint16_t)tab[a0 * NCODE + b] | ((uint32_t)(uint16_t)tab[a1 * NCODE + b] << 16);
      }
      prof4[e] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();

    const int64_t v0 = a.key_off2[key], v1 = a.key_off2[key + 1];
    const uint4* pbase = prof4 + g;
    for (int64_t vb = v0 + warp * 4; vb < v1; vb += NWARPS * 4) {
      const int64_t v = vb + js;
      const bool vok = v < v1;
      uint32_t win[12];
      if (vok) {
        const uint4* p = reinterpret_cast<const uint4*>(a.nb2 + v * WIN);
        uint4 x0 = __ldg(p), x1 = __ldg(p + 1), x2 = __ldg(p + 2);
        win[0] = x0.x; win[1] = x0.y; win[2] = x0.z; win[3] = x0.w;
        win[4] = x1.x; win[5] = x1.y; win[6] = x1.z; win[7] = x1.w;
        win[8] = x2.x; win[9] = x2.y; win[10] = x2.z; win[11] = x2.w;
      } else {
#pragma unroll
        for (int q = 0; q < 12; q++) win[q] = 0x15151515u;  // sentinel code 21
      }
      uint32_t s0 = 0, s1 = 0, s2 = 0, s3 = 0, m0 = 0, m1 = 0, m2 = 0, m3 = 0;
#pragma unroll
      for (int k = 0; k < WIN; k++) {
        const uint32_t b = (win[k >> 2] >> ((k & 3) * 8)) & 0xffu;
        const uint4 p = pbase[(k * NCODE + (int)b) * 8];
        s0 = __vadd2(s0, p.x);
        m0 = __vmaxs2(m0, s0);
        s1 = __vadd2(s1, p.y);
        m1 = __vmaxs2(m1, s1);
        s2 = __vadd2(s2, p.z);
        m2 = __vmaxs2(m2, s2);
        s3 = __vadd2(s3, p.w);
        m3 = __vmaxs2(m3, s3);
        if (k == RIGHT - 1) {
          s0 = m0;
          s1 = m1;
          s2 = m2;
          s3 = m3;
        }
      }
      // rows of this lane: 8g + 2q (low half of m_q) and 8g + 2q + 1 (high)
      unsigned mask = 0;
      if (vok) {
        uint32_t c0 = __vcmpges2(m0, s1x2), c1 = __vcmpges2(m1, s1x2);
        uint32_t c2 = __vcmpges2(m2, s1x2), c3 = __vcmpges2(m3, s1x2);
        mask = (c0 & 1u) | ((c0 >> 15) & 2u) | ((c1 & 1u) << 2) | ((c1 >> 13) & 8u) | ((c2 & 1u) << 4) |
               ((c2 >> 11) & 32u) | ((c3 & 1u) << 6) | ((c3 >> 9) & 128u);
        int valid_rows = rows - g * 8;
        if (valid_rows < 8) mask &= valid_rows <= 0 ? 0u : ((1u << valid_rows) - 1u);
      }
      if (__any_sync(0xffffffffu, mask != 0)) {
        int cnt = __popc(mask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (wcnt + total > WBUF) {
          __syncwarp();
          flush_warp(my_wk, my_wv, wcnt, lane, a.out_count, a.out_key, a.out_val, a.cap);
          __syncwarp();
          wcnt = 0;
        }
        const uint32_t m[4] = {m0, m1, m2, m3};
        const uint64_t p2 = vok ? (uint64_t)a.pos2[v] : 0;
        if (total > WBUF) {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(a.out_count, (unsigned long long)total);
          base = __shfl_sync(0xffffffffu, base, 0) + (incl - cnt);
#pragma unroll
          for (int i = 0; i < 8; i++)
            if (mask & (1u << i)) {
              uint64_t p1 = a.pos1[u0 + g * 8 + i];
              if ((int64_t)base < a.cap) {
                a.out_key[base] = (p1 << a.sh) | p2;
                a.out_val[base] = (m[i >> 1] >> ((i & 1) * 16)) & 0xffffu;
              }
              base++;
            }
        } else {
          int at = wcnt + incl - cnt;
#pragma unroll
          for (int i = 0; i < 8; i++)
            if (mask & (1u << i)) {
              uint64_t p1 = a.pos1[u0 + g * 8 + i];
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
