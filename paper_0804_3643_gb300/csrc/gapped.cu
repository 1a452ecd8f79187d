// gapped.cu -- stage 3.1 (Section 3.3.4; the two one-sided extensions per hit
// of Section 5.2.2) on sm_103a.
//
// One thread computes one side of one hit: the banded affine dynamic
// programme (Gotoh form, anchored at the seed start, free end, no clamp at
// zero) over LG = 64 residues per sequence and the band |i - j| <= 8.  The
// two threads of a hit are adjacent lanes and add their sides with a
// shuffle.  CTAs stride over the hits.
//
// The thread first copies its side's residues to its own shared segments
// (A_1..A_64 and B_-8..B_74, in reading order, so the left side needs no
// special case).  Per cell the work is then: a byte load of B_j (immediate
// offset), an IMAD for the table address, a load of s(A_i, B_j) from a score
// table replicated per lane (entry (a, b) of lane l at word
// ((b * 23 + a) * 32 + l), so the 32 lanes of a warp never share a bank),
// __viaddmax_s32 for E and F, one 3-input max for H, and a max over the row
// of (33 H + 31 - jb), which keeps the first best cell of the row in
// row-major order.  Adds and IMADs go to the FMA pipe, maxima to the ALU
// pipe, which issues at half the FMA rate on sm_103.  Segment strides are odd
// numbers of words, so the byte loads of a warp hit 32 different banks.  The
// 17 band cells of the previous row (H, H - open - extend, F) live in
// registers and are updated in place.
//
// Reads past a sequence end meet the sentinel padding (score -32): no path
// through a sentinel cell comes back above the best cell of the clipped
// grid, so the fixed band over i <= LG equals the one clipped at the sequence
// ends.  Columns j < 0 start at -2^20 and stay far below zero.  Columns
// j > LG (rows i > LG - BAND) lie outside the grid; they feed no cell of the
// grid and are kept out of the maximum.
#include "common.cuh"
#include "ungapped.cuh"

namespace plast {

constexpr int NEG = -(1 << 20);
constexpr int GAP_THREADS = 256;
constexpr int TAB_A = 23;                                   // padded entries per b
constexpr int TAB_WORDS = NCODE * TAB_A * 32;               // lane-replicated
constexpr int SEG_A = 68;                                   // 17 words: A_1 .. A_64
constexpr int SEG_B = 84;                                   // 21 words: B_-8 .. B_74
constexpr int GAP_SMEM = TAB_WORDS * 4 + GAP_THREADS * (SEG_A + SEG_B);  // 103680 bytes

// One band cell of row i: s from the lane's table, then E, F and H.
template <int JB>
__device__ __forceinline__ int band_cell(const unsigned char* rowbase, uint32_t segb, int (&H)[BW], int (&Hm)[BW],
                                         int (&F)[BW], int& E, int& Hm_left, int goe, int ge) {
  const uint32_t b = lds_u8<JB>(segb);  // B_{i - BAND + JB}
  const int sc = *reinterpret_cast<const int*>(rowbase + b * (TAB_A * 128));
  const int up_m = JB + 1 < BW ? Hm[JB + 1 < BW ? JB + 1 : 0] : NEG;
  const int up_f = JB + 1 < BW ? F[JB + 1 < BW ? JB + 1 : 0] : NEG;
  const int e = __viaddmax_s32(E, -ge, Hm_left);   // max(E - ge, H_left - open - ge)
  const int f = __viaddmax_s32(up_f, -ge, up_m);   // max(F_up - ge, H_up - open - ge)
  const int hv = __vimax3_s32(H[JB] + sc, e, f);
  H[JB] = hv;
  Hm_left = hv - goe;
  Hm[JB] = Hm_left;
  F[JB] = f;
  E = e;
  return hv;
}

// Row i of the band.  The first best cell of the row in row-major order is
// the largest (H * 33 + 31 - jb): 33 > 31 keeps H's order, ties go to the
// smaller jb.  Cells with j > LG (EDGE rows) stay out of the maximum.
template <bool EDGE>
__device__ __forceinline__ void gapped_row(int i, const unsigned char* rowbase, uint32_t segb, int (&H)[BW],
                                           int (&Hm)[BW], int (&F)[BW], int goe, int ge, int& best, int& bi,
                                           int& bj) {
  int E = NEG, Hm_left = NEG;
  const int jlim = LG + BAND - i;  // cells jb <= jlim have j <= LG
  int enc[BW];
#define PLAST_CELL(JB)                                                                   \
  {                                                                                      \
    const int hv = band_cell<JB>(rowbase, segb, H, Hm, F, E, Hm_left, goe, ge);          \
    enc[JB] = (EDGE && JB > jlim) ? NEG * 33 : hv * 33 + (31 - JB);                      \
  }
  PLAST_CELL(0) PLAST_CELL(1) PLAST_CELL(2) PLAST_CELL(3) PLAST_CELL(4) PLAST_CELL(5) PLAST_CELL(6)
  PLAST_CELL(7) PLAST_CELL(8) PLAST_CELL(9) PLAST_CELL(10) PLAST_CELL(11) PLAST_CELL(12) PLAST_CELL(13)
  PLAST_CELL(14) PLAST_CELL(15) PLAST_CELL(16)
#undef PLAST_CELL
  int r = __vimax3_s32(enc[0], enc[1], enc[2]);
  r = __vimax3_s32(r, enc[3], enc[4]);
  r = __vimax3_s32(r, enc[5], enc[6]);
  r = __vimax3_s32(r, enc[7], enc[8]);
  r = __vimax3_s32(r, enc[9], enc[10]);
  r = __vimax3_s32(r, enc[11], enc[12]);
  r = __vimax3_s32(r, enc[13], enc[14]);
  r = __vimax3_s32(r, enc[15], enc[16]);
  if (r >= (best + 1) * 33) {  // a strictly larger H (r >= 0 here)
    const int rb = r / 33;
    best = rb;
    bi = i;
    bj = i - BAND + (31 - (r - rb * 33));
  }
}

__global__ void __launch_bounds__(GAP_THREADS, 2) k_small_gapped(GapArgs a) {
  extern __shared__ __align__(16) unsigned char gsm[];
  int* tab32 = reinterpret_cast<int*>(gsm);
  unsigned char* sega = gsm + TAB_WORDS * 4 + threadIdx.x * SEG_A;
  unsigned char* segb = gsm + TAB_WORDS * 4 + GAP_THREADS * SEG_A + threadIdx.x * SEG_B;
  const uint32_t segb_s = (uint32_t)__cvta_generic_to_shared(segb);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = warp; e < NCODE * TAB_A; e += GAP_THREADS / 32) {
    const int b = e / TAB_A, aa = e - b * TAB_A;
    tab32[e * 32 + lane] = aa < NCODE ? (int)c_score[aa * NCODE + b] : 0;
  }
  __syncthreads();
  const unsigned char* tlane = reinterpret_cast<const unsigned char*>(tab32) + lane * 4;
  const int go = a.gap_open, ge = a.gap_extend, goe = go + ge;
  const int64_t total = 2 * a.n;
  const int64_t stride = (int64_t)gridDim.x * GAP_THREADS;
  for (int64_t base = (int64_t)blockIdx.x * GAP_THREADS + warp * 32; base < total; base += stride) {
    const int64_t t = base + lane;
    const int64_t h = t >> 1;
    const int side = (int)(t & 1);  // 0: right of the seed start, 1: left of it
    const bool active = t < total;
    int best = 0, bi = 0, bj = 0;
    if (active) {
      const uint64_t key = a.key[h];
      const int64_t p1 = (int64_t)(key >> a.sh), p2 = (int64_t)(key & ((1ull << a.sh) - 1));
      // residue i (1-based) of each side: right A_i = pad1[p1 + i - 1],
      // left A_i = pad1[p1 - i]; the same for B with p2
      if (side == 0) {
        for (int i = 0; i < LG; i++) sega[i] = (unsigned char)a.pad1[p1 + i];
        for (int j = -BAND; j <= LG + BAND + 2; j++) segb[j + BAND] = (unsigned char)a.pad2[p2 + j - 1];
      } else {
        for (int i = 0; i < LG; i++) sega[i] = (unsigned char)a.pad1[p1 - 1 - i];
        for (int j = -BAND; j <= LG + BAND + 2; j++) segb[j + BAND] = (unsigned char)a.pad2[p2 - j];
      }
      int H[BW], Hm[BW], F[BW];
#pragma unroll
      for (int jb = 0; jb < BW; jb++) {  // row 0
        const int j = jb - BAND;
        H[jb] = j < 0 ? NEG : (j == 0 ? 0 : -(go + j * ge));
        Hm[jb] = H[jb] - goe;
        F[jb] = NEG;
      }
      // row i reads B_{i - BAND + jb} = segb[i + jb]
      for (int i = 1; i <= LG - BAND; i++) {
        const unsigned char* rowbase = tlane + (uint32_t)sega[i - 1] * 128u;
        gapped_row<false>(i, rowbase, segb_s + i, H, Hm, F, goe, ge, best, bi, bj);
      }
      for (int i = LG - BAND + 1; i <= LG; i++) {
        const unsigned char* rowbase = tlane + (uint32_t)sega[i - 1] * 128u;
        gapped_row<true>(i, rowbase, segb_s + i, H, Hm, F, goe, ge, best, bi, bj);
      }
    }
    const int other = __shfl_xor_sync(0xffffffffu, best, 1);
    const int obi = __shfl_xor_sync(0xffffffffu, bi, 1);
    const int obj = __shfl_xor_sync(0xffffffffu, bj, 1);
    if (active && side == 0) {
      const int g = best + other;
      a.score[h] = g;
      a.ends[h] = (uint32_t)bi | ((uint32_t)bj << 8) | ((uint32_t)obi << 16) | ((uint32_t)obj << 24);
      a.pass[h] = g >= a.s2;
    }
  }
}

cudaError_t launch_small_gapped(const GapArgs& a, cudaStream_t st) {
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_small_gapped, cudaFuncAttributeMaxDynamicSharedMemorySize, GAP_SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  if (a.n <= 0) return cudaSuccess;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (2 * a.n + GAP_THREADS - 1) / GAP_THREADS;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 2 * 16;
  if (blocks > cap) blocks = cap;
  note_launch();
  k_small_gapped<<<(unsigned)blocks, GAP_THREADS, GAP_SMEM, st>>>(a);
  return cudaGetLastError();
}

__device__ __forceinline__ int32_t find_seq_g(const int64_t* off, int32_t n, int64_t p) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_gapped_compact(GapArgs a, const int64_t* at, const int64_t* pad_off1, int32_t n1,
                                 const int64_t* pad_off2, int32_t n2, plast_gapped* out) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < a.n; h += (int64_t)gridDim.x * blockDim.x) {
    if (!a.pass[h]) continue;
    const uint64_t key = a.key[h];
    const int64_t p1 = (int64_t)(key >> a.sh), p2 = (int64_t)(key & ((1ull << a.sh) - 1));
    const int32_t q1 = find_seq_g(pad_off1, n1, p1), q2 = find_seq_g(pad_off2, n2, p2);
    const uint32_t e = a.ends[h];
    plast_gapped r;
    r.seq1 = q1;
    r.pos1 = (int32_t)(p1 - pad_off1[q1]);
    r.seq2 = q2;
    r.pos2 = (int32_t)(p2 - pad_off2[q2]);
    r.score = (int16_t)a.score[h];
    r.ungapped = (int16_t)(a.val[h] & 0xffffu);
    r.r_i = (int16_t)(e & 0xff);
    r.r_j = (int16_t)((e >> 8) & 0xff);
    r.l_i = (int16_t)((e >> 16) & 0xff);
    r.l_j = (int16_t)((e >> 24) & 0xff);
    out[at[h]] = r;
  }
}

cudaError_t launch_gapped_compact(const GapArgs& a, const int64_t* at, const int64_t* pad_off1, int32_t n1,
                                  const int64_t* pad_off2, int32_t n2, plast_gapped* out, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  int64_t b = (a.n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  note_launch();
  k_gapped_compact<<<(unsigned)b, 256, 0, st>>>(a, at, pad_off1, n1, pad_off2, n2, out);
  return cudaGetLastError();
}

// Hits given by (sequence, local position) -> padded coordinates, with the
// positions checked against the sequence lengths (bad |= 1 otherwise).
__global__ void k_hits_to_keys(const plast_hit* in, int64_t n, const int64_t* pad_off1, int32_t n1,
                               const int64_t* pad_off2, int32_t n2, int sh, uint64_t* key, uint32_t* val, int* bad) {
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n; h += (int64_t)gridDim.x * blockDim.x) {
    const plast_hit x = in[h];
    bool ok = x.seq1 >= 0 && x.seq1 < n1 && x.seq2 >= 0 && x.seq2 < n2;
    int64_t p1 = 0, p2 = 0;
    if (ok) {
      const int64_t l1 = pad_off1[x.seq1 + 1] - pad_off1[x.seq1] - GAP;
      const int64_t l2 = pad_off2[x.seq2 + 1] - pad_off2[x.seq2] - GAP;
      ok = x.pos1 >= 0 && x.pos1 < l1 && x.pos2 >= 0 && x.pos2 < l2;
      p1 = pad_off1[x.seq1] + x.pos1;
      p2 = pad_off2[x.seq2] + x.pos2;
    }
    if (!ok) {
      atomicOr(bad, 1);
      p1 = pad_off1[0];
      p2 = pad_off2[0];
    }
    key[h] = ((uint64_t)p1 << sh) | (uint64_t)p2;
    val[h] = (uint32_t)(uint16_t)x.score;
  }
}

cudaError_t launch_hits_to_keys(const plast_hit* in, int64_t n, const int64_t* pad_off1, int32_t n1,
                                const int64_t* pad_off2, int32_t n2, int sh, uint64_t* key, uint32_t* val, int* bad,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  note_launch();
  k_hits_to_keys<<<(unsigned)b, 256, 0, st>>>(in, n, pad_off1, n1, pad_off2, n2, sh, key, val, bad);
  return cudaGetLastError();
}

}  // namespace plast
