// gapped.cu -- stage 3.1 (Section 3.3.4; the two one-sided extensions per hit
// of Section 5.2.2) on sm_103a.
//
// One thread computes one side (right or left of the seed start) of TWO hits
// at once, one per int16 half: the banded affine dynamic programme (Gotoh
// form, anchored at the seed start, free end, no clamp at zero) over
// LG = 64 residues per sequence and the band |i - j| <= 8.  The two threads
// holding the two sides of the same hits are adjacent lanes and add their
// sides with shuffles.  CTAs stride over the hits.
//
// Per cell (two hits): two byte loads of B_j from the thread's shared
// segments, two IMADs and two loads of s(A_i, B_j) - go from a lane-replicated
// table (entry (a, b) of lane l at word (b * 23 + a) * 32 + l: the lanes of a
// warp never share a bank), one IMAD packing the two entries, then four
// three-operand maxima.  Row i's values are kept offset by i * ge, and F and
// DF also shifted down by goe = go + ge:
//   H'  = H + i ge,  E' = E + i ge,  Gg = F + i ge - goe,  DFg = DF + i ge - goe
// so that, with up = (i - 1, j) and diag = (i - 1, j - 1),
//   Gg  = max(H'_up - go - goe, Gg_up)            __viaddmax_s16x2
//   DFg = max(H'_diag + (s - go), Gg)             __viaddmax_s16x2
//   H'  = max(DFg + goe, E')                      __viaddmax_s16x2
//   E'  = max(E' - ge, DFg)   (E' of the next cell)  __viaddmax_s16x2
// which restate F = max(H_up - go - ge, F_up - ge), DF = max(H_diag + s, F),
// H = max(DF, E), E_next = max(E - ge, DF - go - ge) with no other operation.
// Only DF feeds the next E: since go >= 0, H - go - ge is never above E - ge
// when H = E.  Values are exact in int16 (|H| <= 64 * 11 on the grid; cells
// off the grid stay below -14000 and above -16000 - 64 * 24).
//
// The A residues of a side reach the thread four rows at a time: aligned
// 32-bit loads of pad1 (byte-reversed for the left side) funnel-shifted into
// place, one word per hit per four rows, fetched a group ahead; each row
// takes its byte with one prmt.  (Byte loads, one per row, cost a memory
// transaction per lane when the hits of a warp are scattered over bank 1, as
// they are in the order stage 2 writes them.)
//
// The end cell (first maximum in row-major order): after each row the row
// maximum is compared with the best so far per half; the halves that improve
// copy the row's H values into a best-row array (LOP3 masks) and record the
// row.  At the end the first column of the best row holding the best value
// is the end column.
//
// Reads past a sequence end meet the sentinel padding (score -32): no path
// through a sentinel cell comes back above the best cell of the clipped
// grid, so the fixed band over i <= LG equals the one clipped at the sequence
// ends.  Columns j < 0 start at -16000 and stay far below zero.  Columns
// j > LG (rows i > LG - BAND) lie outside the grid and feed no cell of it
// (a cell reads only cells of its own or a smaller column), so they are not
// computed (compile-time column limits); the stale values left in their
// slots are read only by other such cells.
#include <atomic>

#include "gapped.cuh"

#include "common.cuh"

namespace plast {

constexpr int NEG16 = -16000;
constexpr int GAP_THREADS = 256;
constexpr int TAB_A = 23;                                   // padded entries per b
constexpr int TAB_WORDS = NCODE * TAB_A * 32;               // lane-replicated
constexpr int SEG_W = 22;                                   // words staged per hit: B_-8 .. B_74 + slack
constexpr int SEG_B = SEG_W * 4;                            // 88 bytes
constexpr int SEG_T = 2 * SEG_B + 4;                        // 45 words per thread: odd, no bank conflict
constexpr int GAP_SMEM = TAB_WORDS * 4 + GAP_THREADS * SEG_T;  // 110848 bytes

__device__ __forceinline__ uint32_t x2(int v) { return ((uint32_t)(uint16_t)v << 16) | (uint16_t)v; }

struct Band {
  uint32_t H[BW], Gg[BW], bestH[BW];  // H' and Gg of the previous row, H' of the best row
  uint32_t best, bi;                 // per half (best without the row offset)
};

struct GapConst {
  uint32_t nge2, goe2, ngg2;  // -ge, go + ge, -(go + goe) in both halves
  int ge;
};

// Cell JB of row i for both hits.
template <int JB>
__device__ __forceinline__ uint32_t band_cell(Band& B, const unsigned char* row0, const unsigned char* row1,
                                              uint32_t sb0, uint32_t sb1, uint32_t& E, const GapConst& k) {
  const uint32_t b0 = lds_u8<JB>(sb0), b1 = lds_u8<JB>(sb1);  // B_{i - BAND + JB} of each hit
  const uint32_t s0 = *reinterpret_cast<const uint32_t*>(row0 + b0 * (TAB_A * 128));
  const uint32_t s1 = *reinterpret_cast<const uint32_t*>(row1 + b1 * (TAB_A * 128));
  const uint32_t sc = s1 * 65536u + s0;  // entries are zero-extended int16 s - go
  const uint32_t up_h = JB + 1 < BW ? B.H[JB + 1 < BW ? JB + 1 : 0] : x2(NEG16);
  const uint32_t up_g = JB + 1 < BW ? B.Gg[JB + 1 < BW ? JB + 1 : 0] : x2(NEG16);
  const uint32_t gg = __viaddmax_s16x2(up_h, k.ngg2, up_g);  // Gg
  const uint32_t dfg = __viaddmax_s16x2(B.H[JB], sc, gg);    // DFg
  const uint32_t h = __viaddmax_s16x2(dfg, k.goe2, E);        // H'
  E = __viaddmax_s16x2(E, k.nge2, dfg);                        // E' of the next cell
  B.H[JB] = h;
  B.Gg[JB] = gg;
  return h;
}

// Cells 0 .. JLIM of row i (the cells JB > JLIM have j > LG, see below).
template <int JB, int JLIM>
__device__ __forceinline__ void band_cells(Band& B, const unsigned char* row0, const unsigned char* row1,
                                           uint32_t sb0, uint32_t sb1, uint32_t& E, const GapConst& k) {
  if constexpr (JB <= JLIM) {
    band_cell<JB>(B, row0, row1, sb0, sb1, E, k);
    band_cells<JB + 1, JLIM>(B, row0, row1, sb0, sb1, E, k);
  }
}

// Maximum of H'[0 .. JLIM], three at a time.
template <int JB, int JLIM>
__device__ __forceinline__ uint32_t row_max(const Band& B, uint32_t m) {
  if constexpr (JB + 1 <= JLIM) return row_max<JB + 2, JLIM>(B, __vimax3_s16x2(m, B.H[JB], B.H[JB + 1]));
  else if constexpr (JB <= JLIM) return __vmaxs2(m, B.H[JB]);
  else return m;
}

// Row i; columns jb > JLIM have j > LG: they are neither computed nor in the
// maximum.
template <int JLIM>
__device__ __forceinline__ void gapped_row(Band& B, int i, const unsigned char* row0, const unsigned char* row1,
                                           uint32_t sb0, uint32_t sb1, const GapConst& k) {
  uint32_t E = x2(NEG16);
  band_cells<0, JLIM>(B, row0, row1, sb0 + i, sb1 + i, E, k);
  const uint32_t rmax = __vsub2(row_max<1, JLIM>(B, B.H[0]), x2(i * k.ge));  // without the row offset
  const uint32_t up = __vcmpgts2(rmax, B.best);  // 0xffff in the halves that improve
  B.best = __vmaxs2(B.best, rmax);
  B.bi = (x2(i) & up) | (B.bi & ~up);
#pragma unroll
  for (int jb = 0; jb < BW; jb++) B.bestH[jb] = (B.H[jb] & up) | (B.bestH[jb] & ~up);
}

// First column of the best row holding the best value, for half q.
__device__ __forceinline__ int end_column(const Band& B, int q, int ge) {
  const int sh = 16 * q;
  const int bi = (int16_t)(B.bi >> sh);
  const int best = (int16_t)(B.best >> sh) + bi * ge;  // with the best row's offset
  const int jlim = min(BW - 1, LG + BAND - bi);
  int found = -1;
#pragma unroll
  for (int jb = BW - 1; jb >= 0; jb--)
    if (jb <= jlim && (int16_t)(B.bestH[jb] >> sh) == best) found = jb;
  return bi - BAND + found;
}

// Copy B_-8 .. B_74 of one hit side into a thread's segment in reading
// order with aligned 32-bit loads, B_-8 landing on the segment's first byte
// (so the byte loads of a warp stay conflict-free); returns its shared address.
// Right side: B_j = pad2[p2 + j - 1], the bytes [p2 - 9, p2 + 73] forwards.
// Left side:  B_j = pad2[p2 - j],     the bytes [p2 - 74, p2 + 8] backwards,
// each word byte-reversed.
__device__ __forceinline__ uint32_t stage_b(const int8_t* pad2, int64_t p2, int side, uint32_t* dst,
                                            uint32_t dst_s) {
  const int64_t lo = p2 - 9, hi = p2 + BAND;
  const int64_t first = side ? ((hi | 3) - 3) : (lo & ~(int64_t)3);  // byte address of the first word
  const uint32_t sel = side ? 0x0123u : 0x3210u;
  const uint32_t sh = 8u * (side ? (uint32_t)(3 - (hi & 3)) : (uint32_t)(lo & 3));
  const uint32_t* src = reinterpret_cast<const uint32_t*>(pad2 + first);
  uint32_t w[SEG_W + 1];
#pragma unroll
  for (int k = 0; k <= SEG_W; k++) w[k] = __byte_perm(__ldg(src + (side ? -k : k)), 0u, sel);
#pragma unroll
  for (int k = 0; k < SEG_W; k++) dst[k] = __funnelshift_r(w[k], w[k + 1], sh);
  return dst_s;
}

// Consecutive bytes of pad1 from address `start`, forwards (dir 0) or
// backwards (dir 1), delivered four per call in reading order (byte 0 first).
struct ByteRun {
  const uint32_t* src;
  uint32_t prev, sel, sh;
  int dir, k;
  __device__ __forceinline__ void init(const int8_t* base, int64_t start, int d) {
    dir = d;
    const int64_t first = start & ~(int64_t)3;
    sel = d ? 0x0123u : 0x3210u;
    sh = 8u * (d ? (uint32_t)(3 - (start & 3)) : (uint32_t)(start & 3));
    src = reinterpret_cast<const uint32_t*>(base + first);
    prev = __byte_perm(__ldg(src), 0u, sel);
    k = 1;
  }
  __device__ __forceinline__ uint32_t next() {
    const uint32_t nxt = __byte_perm(__ldg(src + (dir ? -k : k)), 0u, sel);
    const uint32_t out = __funnelshift_r(prev, nxt, sh);
    prev = nxt;
    k++;
    return out;
  }
};

__global__ void __launch_bounds__(GAP_THREADS, 2) k_small_gapped(GapArgs a) {
  extern __shared__ __align__(16) unsigned char gsm[];
  uint32_t* tab32 = reinterpret_cast<uint32_t*>(gsm);
  unsigned char* seg = gsm + TAB_WORDS * 4 + threadIdx.x * SEG_T;
  const uint32_t seg_s = (uint32_t)__cvta_generic_to_shared(seg);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int go = a.gap_open, ge = a.gap_extend, goe = go + ge;
  for (int e = warp; e < NCODE * TAB_A; e += GAP_THREADS / 32) {
    const int b = e / TAB_A, aa = e - b * TAB_A;
    tab32[e * 32 + lane] = aa < NCODE ? (uint32_t)(uint16_t)(int16_t)(c_score[aa * NCODE + b] - go) : 0u;
  }
  __syncthreads();
  const unsigned char* tlane = reinterpret_cast<const unsigned char*>(tab32) + lane * 4;
  GapConst kc;
  kc.nge2 = x2(-ge);
  kc.goe2 = x2(goe);
  kc.ngg2 = x2(-(go + goe));
  kc.ge = ge;
  const int64_t n = a.n_dev ? min(a.n, max(*a.n_dev, (int64_t)0)) : a.n;
  const int64_t npairs = (n + 1) / 2;  // hits 2p and 2p+1 share a thread
  const int64_t total = 2 * npairs;      // (pair, side) threads
  const int64_t stride = (int64_t)gridDim.x * GAP_THREADS;
  for (int64_t base = (int64_t)blockIdx.x * GAP_THREADS + warp * 32; base < total; base += stride) {
    const int64_t t = base + lane;
    const int64_t pr = t >> 1;
    const int side = (int)(t & 1);  // 0: right of the seed start, 1: left of it
    const bool active = t < total;
    const int64_t h0 = 2 * pr, h1 = 2 * pr + 1 < n ? 2 * pr + 1 : 2 * pr;
    Band B;
    if (active) {
      const uint64_t k0 = a.key[h0], k1 = a.key[h1];
      const uint64_t mask = (1ull << a.sh) - 1;
      const int64_t p10 = (int64_t)(k0 >> a.sh), p20 = (int64_t)(k0 & mask);
      const int64_t p11 = (int64_t)(k1 >> a.sh), p21 = (int64_t)(k1 & mask);
      // residue i (1-based): right A_i = pad1[p1 + i - 1], B_j = pad2[p2 + j - 1];
      // left A_i = pad1[p1 - i], B_j = pad2[p2 - j].
      // B_-8 .. B_74 of each hit in reading order: aligned words of pad2,
      // taken backwards and byte-reversed for the left side; sbX points at B_-8
      const uint32_t sb0 = stage_b(a.pad2, p20, side, reinterpret_cast<uint32_t*>(seg), seg_s);
      const uint32_t sb1 = stage_b(a.pad2, p21, side, reinterpret_cast<uint32_t*>(seg + SEG_B), seg_s + SEG_B);
#pragma unroll
      for (int jb = 0; jb < BW; jb++) {  // row 0
        const int j = jb - BAND;
        const int v = j < 0 ? NEG16 : (j == 0 ? 0 : -(go + j * ge));
        B.H[jb] = x2(v);
        B.Gg[jb] = x2(NEG16);
        B.bestH[jb] = B.H[jb];
      }
      B.best = 0;
      B.bi = 0;
      // A_i of both hits, four rows per word (byte r = row 4g + 1 + r),
      // fetched a group ahead; right: A_i = pad1[p1 + i - 1] forwards from
      // p1, left: A_i = pad1[p1 - i] backwards from p1 - 1
      ByteRun ra0, ra1;
      ra0.init(a.pad1, p10 - side, side);
      ra1.init(a.pad1, p11 - side, side);
      uint32_t aw0 = ra0.next(), aw1 = ra1.next();
#define PLAST_ROW(I, R, JLIM)                                                                          \
  {                                                                                                    \
    const unsigned char* r0 = tlane + __byte_perm(c0, 0u, 0x4440u + (R)) * 128u;                       \
    const unsigned char* r1 = tlane + __byte_perm(c1, 0u, 0x4440u + (R)) * 128u;                       \
    gapped_row<JLIM>(B, (I), r0, r1, sb0, sb1, kc);                                                    \
  }
      for (int g = 0; g < (LG - BAND) / 4; g++) {  // rows 1 .. 56: the whole band on the grid
        const uint32_t c0 = aw0, c1 = aw1;
        aw0 = ra0.next();
        aw1 = ra1.next();
        const int i = 4 * g + 1;
        PLAST_ROW(i, 0, BW - 1)
        PLAST_ROW(i + 1, 1, BW - 1)
        PLAST_ROW(i + 2, 2, BW - 1)
        PLAST_ROW(i + 3, 3, BW - 1)
      }
      {  // rows 57 .. 60
        const uint32_t c0 = aw0, c1 = aw1;
        aw0 = ra0.next();
        aw1 = ra1.next();
        PLAST_ROW(LG - BAND + 1, 0, 15)
        PLAST_ROW(LG - BAND + 2, 1, 14)
        PLAST_ROW(LG - BAND + 3, 2, 13)
        PLAST_ROW(LG - BAND + 4, 3, 12)
      }
      {  // rows 61 .. 64
        const uint32_t c0 = aw0, c1 = aw1;
        PLAST_ROW(LG - BAND + 5, 0, 11)
        PLAST_ROW(LG - BAND + 6, 1, 10)
        PLAST_ROW(LG - BAND + 7, 2, 9)
        PLAST_ROW(LG - BAND + 8, 3, 8)
      }
#undef PLAST_ROW
    } else {
      B.best = 0;
      B.bi = 0;
#pragma unroll
      for (int jb = 0; jb < BW; jb++) B.bestH[jb] = 0;
    }
    // per hit: this side's (score, end row, end column)
    int bi0 = 0, bj0 = 0, bi1 = 0, bj1 = 0;
    if (active) {
      bi0 = (int16_t)(B.bi & 0xffff);
      bj0 = end_column(B, 0, ge);
      bi1 = (int16_t)(B.bi >> 16);
      bj1 = end_column(B, 1, ge);
    }
    const uint32_t ob = __shfl_xor_sync(0xffffffffu, B.best, 1);
    const int obi0 = __shfl_xor_sync(0xffffffffu, bi0, 1), obj0 = __shfl_xor_sync(0xffffffffu, bj0, 1);
    const int obi1 = __shfl_xor_sync(0xffffffffu, bi1, 1), obj1 = __shfl_xor_sync(0xffffffffu, bj1, 1);
    if (active && side == 0) {
      const int g0 = (int16_t)(B.best & 0xffff) + (int16_t)(ob & 0xffff);
      a.score[h0] = g0;
      a.ends[h0] = (uint32_t)bi0 | ((uint32_t)bj0 << 8) | ((uint32_t)obi0 << 16) | ((uint32_t)obj0 << 24);
      a.pass[h0] = g0 >= a.s2;
      if (2 * pr + 1 < n) {
        const int g1 = (int16_t)(B.best >> 16) + (int16_t)(ob >> 16);
        a.score[h1] = g1;
        a.ends[h1] = (uint32_t)bi1 | ((uint32_t)bj1 << 8) | ((uint32_t)obi1 << 16) | ((uint32_t)obj1 << 24);
        a.pass[h1] = g1 >= a.s2;
      }
    }
  }
}

// The passing hits as (key, hit index) appended to rkey / ridx (slots below
// out_cap written), their number added to *rcount.  A CTA takes 4,096
// consecutive hits, 16 per thread; a block-wide scan of the per-thread
// counts places them behind one atomic per CTA (a single counter taking one
// atomic per warp would serialise on it).
constexpr int CP_THREADS = 256;
constexpr int CP_PER = 16;
__global__ void __launch_bounds__(CP_THREADS) k_compact_pass(GapArgs a) {
  __shared__ int wsum[CP_THREADS / 32];
  __shared__ unsigned long long block_at;
  const int64_t n = a.n_dev ? min(a.n, max(*a.n_dev, (int64_t)0)) : a.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = (int64_t)blockIdx.x * CP_THREADS * CP_PER; base < n;
       base += (int64_t)gridDim.x * CP_THREADS * CP_PER) {
    const int64_t h0 = base + (int64_t)threadIdx.x * CP_PER;
    uint32_t bits = 0;
#pragma unroll
    for (int j = 0; j < CP_PER; j++)
      if (h0 + j < n && a.pass[h0 + j]) bits |= 1u << j;
    const int c = __popc(bits);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < CP_THREADS / 32; w++) t += wsum[w];
      block_at = t ? atomicAdd(a.rcount, (unsigned long long)t) : 0;
    }
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; w++) before += wsum[w];
    unsigned long long at = block_at + before + x - c;
    for (; bits; bits &= bits - 1, at++) {
      const int64_t h = h0 + __ffs(bits) - 1;
      if ((int64_t)at < a.out_cap) {
        a.rkey[at] = a.key[h];
        a.ridx[at] = (uint32_t)h;
      }
    }
    __syncthreads();  // wsum and block_at are reused
  }
}

cudaError_t launch_compact_pass(const GapArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  int64_t b = (a.n + CP_THREADS * CP_PER - 1) / (CP_THREADS * CP_PER);
  if (b > 152 * 16) b = 152 * 16;
  note_launch();
  k_compact_pass<<<(unsigned)b, CP_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_small_gapped(const GapArgs& a, cudaStream_t st) {
  static std::atomic<bool> attr_set[64];  // per device; calls may come from several threads
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
  int64_t blocks = (2 * ((a.n + 1) / 2) + GAP_THREADS - 1) / GAP_THREADS;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 2 * 16;
  if (blocks > cap) blocks = cap;
  note_launch();
  k_small_gapped<<<(unsigned)blocks, GAP_THREADS, GAP_SMEM, st>>>(a);
  return cudaGetLastError();
}

__device__ __forceinline__ plast_gapped make_record(const GapArgs& a, int64_t h, uint64_t key, const SeqMap& s1,
                                                    const SeqMap& s2) {
  const int64_t p1 = (int64_t)(key >> a.sh), p2 = (int64_t)(key & ((1ull << a.sh) - 1));
  const int32_t q1 = seq_of(s1, p1), q2 = seq_of(s2, p2);
  const int64_t* pad_off1 = s1.pad_off;
  const int64_t* pad_off2 = s2.pad_off;
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
  return r;
}

__global__ void k_gapped_compact(GapArgs a, const int64_t* at, SeqMap s1, SeqMap s2, plast_gapped* out) {
  const int64_t n = a.n_dev ? min(a.n, max(*a.n_dev, (int64_t)0)) : a.n;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n; h += (int64_t)gridDim.x * blockDim.x) {
    if (!a.pass[h] || at[h] >= a.out_cap) continue;
    out[at[h]] = make_record(a, h, a.key[h], s1, s2);
  }
}

// Records in key order: out[r] from hit sidx[r] (key skey[r]), r < m (or
// < *m_dev, at most m).
__global__ void k_write_sorted(GapArgs a, const uint64_t* skey, const uint32_t* sidx, int64_t m, const int64_t* m_dev,
                               SeqMap s1, SeqMap s2, plast_gapped* out) {
  if (m_dev) m = min(m, max(*m_dev, (int64_t)0));
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
    out[r] = make_record(a, sidx[r], skey[r], s1, s2);
}

cudaError_t launch_gapped_compact(const GapArgs& a, const int64_t* at, const SeqMap& s1, const SeqMap& s2,
                                  plast_gapped* out, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  int64_t b = (a.n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  note_launch();
  k_gapped_compact<<<(unsigned)b, 256, 0, st>>>(a, at, s1, s2, out);
  return cudaGetLastError();
}

__global__ void k_clamp_count(const unsigned long long* count, int64_t cap, int64_t* n_dev) {
  const unsigned long long c = *count;
  *n_dev = c > (unsigned long long)cap ? cap : (int64_t)c;
}

cudaError_t launch_clamp_count(const unsigned long long* count, int64_t cap, int64_t* n_dev, cudaStream_t st) {
  note_launch();
  k_clamp_count<<<1, 1, 0, st>>>(count, cap, n_dev);
  return cudaGetLastError();
}

cudaError_t launch_write_sorted(const GapArgs& a, const uint64_t* skey, const uint32_t* sidx, int64_t m,
                                const int64_t* m_dev, const SeqMap& s1, const SeqMap& s2, plast_gapped* out,
                                cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  int64_t b = (m + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  note_launch();
  k_write_sorted<<<(unsigned)b, 256, 0, st>>>(a, skey, sidx, m, m_dev, s1, s2, out);
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

// ---------------------------------------------------------------------------
// Survivor expansion: padded coordinates -> (sequence, local position), and
// the exact scalar ungapped score with its extents, recomputed per survivor
// as a self-check of the packed kernel (a mismatch raises *bad).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ungapped_exact(const int8_t* tab, const int8_t* pad1, int64_t p1, const int8_t* pad2,
                                              int64_t p2, int* rl, int* ll) {
  int sum = 0, best = 0, r = 0, l = 0;
  for (int t = 0; t < RIGHT; t++) {
    sum += tab[pad1[p1 + t] * NCODE + pad2[p2 + t]];
    if (sum > best) {
      best = sum;
      r = t + 1;
    }
  }
  sum = best;
  for (int t = 1; t <= LEFT; t++) {
    sum += tab[pad1[p1 - t] * NCODE + pad2[p2 - t]];
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
                              SeqMap s1, const int8_t* pad2, SeqMap s2, plast_hit* out, int* bad) {
  __shared__ int8_t tab[NCODE * NCODE];  // lanes look up different entries
  for (int i = threadIdx.x; i < NCODE * NCODE; i += blockDim.x) tab[i] = c_score[i];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p1 = (int64_t)(key[i] >> sh), p2 = (int64_t)(key[i] & ((1ull << sh) - 1));
    int rl, ll;
    int u = ungapped_exact(tab, pad1, p1, pad2, p2, &rl, &ll);
    if (u != (int)(int16_t)(val[i] & 0xffffu)) atomicOr(bad, 2);
    const int32_t q1 = seq_of(s1, p1), q2 = seq_of(s2, p2);
    const int64_t* pad_off1 = s1.pad_off;
    const int64_t* pad_off2 = s2.pad_off;
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
                               const SeqMap& s1, const int8_t* pad2, const SeqMap& s2, plast_hit* out, int* bad,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  note_launch();
  k_expand_hits<<<(unsigned)b, 256, 0, st>>>(key, val, n, sh, pad1, s1, pad2, s2, out, bad);
  return cudaGetLastError();
}

}  // namespace plast
