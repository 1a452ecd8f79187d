// gapped.cu -- stage 3.1 (Section 3.3.4; the two one-sided extensions per hit
// of Section 5.2.2) on sm_103a.
//
// One thread computes one side of one hit: the banded affine dynamic
// programme (Gotoh form, anchored at the seed start, free end, no clamp at
// zero) over LG = 64 residues per sequence and the band |i - j| <= 8.  The
// 17 band cells of the previous row (H and F) live in registers; the row is
// walked left to right so E is a scalar.  Reads past a sequence end meet the
// sentinel padding (score -32), and no path through a sentinel cell can come
// back above the best in-sequence cell, so the fixed band over i, j <= LG
// equals the one clipped at the sequence ends.  The two threads of a hit are adjacent lanes and add their
// sides with a shuffle.
#include "common.cuh"
#include "ungapped.cuh"

namespace plast {

constexpr int NEG = -(1 << 20);
constexpr int GAP_THREADS = 256;

__global__ void __launch_bounds__(GAP_THREADS) k_small_gapped(GapArgs a) {
  __shared__ int8_t tab[NCODE * NCODE];
  for (int i = threadIdx.x; i < NCODE * NCODE; i += GAP_THREADS) tab[i] = c_score[i];
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * GAP_THREADS + threadIdx.x;
  const int64_t h = t >> 1;
  const int side = (int)(t & 1);  // 0: right of the seed start, 1: left of it
  const bool active = h < a.n;
  const int go = a.gap_open, ge = a.gap_extend;
  int best = 0, bi = 0, bj = 0;
  if (active) {
    const uint64_t key = a.key[h];
    const int64_t p1 = (int64_t)(key >> a.sh), p2 = (int64_t)(key & ((1ull << a.sh) - 1));
    const int step = side ? -1 : 1;
    // residue i (1-based) of each side: A_i = A[(i - 1) * step]
    const int8_t* A = a.pad1 + p1 - side;
    const int8_t* B = a.pad2 + p2 - side;
    int H[BW], F[BW];
#pragma unroll
    for (int jb = 0; jb < BW; jb++) {
      const int j = jb - BAND;
      H[jb] = j < 0 ? NEG : (j == 0 ? 0 : -(go + j * ge));
      F[jb] = NEG;
    }
    for (int i = 1; i <= LG; i++) {
      const int8_t* trow = tab + A[(i - 1) * step] * NCODE;
      int E = NEG, Hleft = NEG;
      int Hn[BW], Fn[BW];
#pragma unroll
      for (int jb = 0; jb < BW; jb++) {
        const int j = i - BAND + jb;
        const int diag = H[jb];
        const int upH = jb + 1 < BW ? H[jb + 1] : NEG;
        const int upF = jb + 1 < BW ? F[jb + 1] : NEG;
        int e = max(E - ge, Hleft - go - ge);
        int f = max(upF - ge, upH - go - ge);
        int hv = max(diag + trow[B[(j - 1) * step]], max(e, f));
        if (j < 0 || j > LG) {  // outside the grid: j runs over 0..LG only
          hv = NEG;
          e = NEG;
          f = NEG;
        }
        Hn[jb] = hv;
        Fn[jb] = f;
        E = e;
        Hleft = hv;
        if (hv > best) {
          best = hv;
          bi = i;
          bj = j;
        }
      }
#pragma unroll
      for (int jb = 0; jb < BW; jb++) {
        H[jb] = Hn[jb];
        F[jb] = Fn[jb];
      }
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

cudaError_t launch_small_gapped(const GapArgs& a, cudaStream_t st) {
  if (a.n <= 0) return cudaSuccess;
  int64_t threads = 2 * a.n;
  int64_t blocks = (threads + GAP_THREADS - 1) / GAP_THREADS;
  note_launch();
  k_small_gapped<<<(unsigned)blocks, GAP_THREADS, 0, st>>>(a);
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
