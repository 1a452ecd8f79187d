// index.cu -- stage 0 (Section 3.3.1) and the six-frame translation of
// Section 6, as device kernels.
//
// A bank lives on the device as
//   pad      codes with GAP sentinel bytes before, between and after the
//            sequences: sequence s starts at pad_off[s] = seq_off[s] + GAP*(s+1)
//   pos      padded start of every indexed word, grouped by key (CSR by
//            key_off[8801]), increasing within a key
//   nb       the 48-residue neighbourhood of every indexed word, in the
//            order stage 2 consumes it: the 26 residues from the seed start
//            rightwards, then the 22 residues left of it walking leftwards
//            (Section 3.3.2's neighbourhood blocks, built once per bank).
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "gapped.cuh"
#include "index.cuh"

namespace plast {

__global__ void k_check_codes(const int8_t* codes, int64_t n, int lo, int hi, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int c = codes[i];
    if (c < lo || c > hi) atomicOr(bad, 1);
  }
}

// last s in [0, n) with off[s] <= p (off non-decreasing, off[0] <= p)
__device__ __forceinline__ int32_t find_seq(const int64_t* off, int32_t n, int64_t p) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// True in every byte lane of w whose byte, read unsigned, is above hi
// (0 <= hi < 127): adding 127 - hi to the low seven bits carries into bit 7
// exactly when the byte exceeds hi, and bytes of 128 or more have bit 7 set.
__device__ __forceinline__ uint32_t bytes_above(uint32_t w, uint32_t hi) {
  return (((w & 0x7f7f7f7fu) + 0x01010101u * (127u - hi)) | w) & 0x80808080u;
}

// Padded bank, one thread per 16-byte chunk of codes: the chunk's sequence by
// one binary search; a chunk inside one sequence moves with one 16-byte load
// and store (sequence s moves by GAP * (s + 1), a multiple of 16, into a
// 16-byte aligned pad), the others byte by byte.  Every code is checked
// against [0, hi]; *bad is raised if one is outside.
static_assert(GAP % 16 == 0, "sequences move by whole 16-byte chunks");
__global__ void k_build_pad(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, int64_t n_res, int hi,
                            int8_t* pad, int* bad) {
  const bool vec = (reinterpret_cast<uintptr_t>(codes) & 15) == 0;
  const int64_t n_chunks = (n_res + 15) >> 4;
  uint32_t b = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_chunks; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = c << 4, p1 = min(p0 + 16, n_res);
    int32_t s = find_seq(seq_off, n_seqs, p0);
    if (vec && p1 - p0 == 16 && seq_off[s + 1] >= p1) {
      const uint4 v = *reinterpret_cast<const uint4*>(codes + p0);
      b |= bytes_above(v.x, hi) | bytes_above(v.y, hi) | bytes_above(v.z, hi) | bytes_above(v.w, hi);
      *reinterpret_cast<uint4*>(pad + p0 + (int64_t)GAP * (s + 1)) = v;
    } else {
      for (int64_t p = p0; p < p1; p++) {
        while (seq_off[s + 1] <= p) s++;  // seq_off[n_seqs] = n_res > p ends the walk
        const int8_t x = codes[p];
        if (x < 0 || x > hi) b = 1;
        pad[p + (int64_t)GAP * (s + 1)] = x;
      }
    }
  }
  if (b) atomicOr(bad, 1);
}

// Stage 0's lookup table and lists (Section 3.3.1) as a stable counting
// sort of the padded positions by key.  A word is indexed when its four
// letters are residues (codes below 20: no stop, no sentinel, so no word
// crosses a sequence end).  The padded bank is cut into tiles of T positions
// (a multiple of 4096, chosen so that the tiles keep the GPU busy); pass 1
// counts each tile's words per key, an exclusive scan of the counts in
// key-major order gives every (key, tile) its first slot (and, at (k, 0), the
// CSR offset of key k), pass 2 walks each tile in position order with one
// warp and writes each word's position into its key's slots, so positions
// increase within a key.
constexpr int IX_THREADS = 256;
constexpr int IX_PER = 16;                      // positions per thread and chunk
constexpr int IX_CHUNK = IX_THREADS * IX_PER;   // 4096

// Keys of the 16 words at p0 .. p0 + 15 from five aligned words of pad (p0 is
// a multiple of 16; a thread at or past n_pad reads nothing, the others at
// most 19 bytes past p0, inside the bank's trailing slack); bit j of the
// result says whether word p0 + j is indexed.
__device__ __forceinline__ uint32_t keys16_from(const uint32_t w[5], const int8_t* cls2, const int8_t* cls3,
                                                int32_t key[IX_PER]) {
  uint32_t by[IX_PER + 3];
#pragma unroll
  for (int j = 0; j < IX_PER + 3; j++) by[j] = (w[j >> 2] >> (8 * (j & 3))) & 0xffu;
  uint32_t valid = 0;
#pragma unroll
  for (int j = 0; j < IX_PER; j++) {
    const uint32_t a0 = by[j], a1 = by[j + 1], a2 = by[j + 2], a3 = by[j + 3];
    const bool ok = a0 < NAA && a1 < NAA && a2 < NAA && a3 < NAA;
    key[j] = ok ? (((int)(a0 * 2) + cls2[ok ? a1 : 0]) * 11 + cls3[ok ? a2 : 0]) * 20 + (int)a3 : -1;
    valid |= (uint32_t)ok << j;
  }
  return valid;
}

// The 20 bytes pad[p0 .. p0 + 20) as five words (p0 a multiple of 16); all
// sentinels at or past n_pad (nothing is read there; below it at most 19
// bytes past p0 are read, inside the bank's trailing slack).
__device__ __forceinline__ void load20(const int8_t* pad, int64_t p0, int64_t n_pad, uint32_t w[5]) {
  if (p0 < n_pad) {
    const uint4 v = *reinterpret_cast<const uint4*>(pad + p0);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
    w[4] = *reinterpret_cast<const uint32_t*>(pad + p0 + 16);
  } else {
#pragma unroll
    for (int k = 0; k < 5; k++) w[k] = 0x01010101u * SENTINEL;
  }
}

// Keys of the 16 words at p0 .. p0 + 15; bit j of the result says whether
// word p0 + j is indexed.
__device__ __forceinline__ uint32_t word_keys16(const int8_t* pad, int64_t p0, int64_t n_pad, const int8_t* cls2,
                                                const int8_t* cls3, int32_t key[IX_PER]) {
  uint32_t w[5];
  load20(pad, p0, n_pad, w);
  return keys16_from(w, cls2, cls3, key);
}

__device__ __forceinline__ void load_classes(int8_t* cls2, int8_t* cls3) {
  if (threadIdx.x < NAA) {
    cls2[threadIdx.x] = c_cls2[threadIdx.x];
    cls3[threadIdx.x] = c_cls3[threadIdx.x];
  }
}

// Pass 1: hist[k * n_tiles + t] = words of key k in tile t.
__global__ void __launch_bounds__(IX_THREADS) k_index_hist(const int8_t* pad, int64_t n_pad, int64_t tile,
                                                           int64_t n_tiles, int32_t* hist) {
  __shared__ int32_t cnt[NKEYS];
  __shared__ int8_t cls2[NAA], cls3[NAA];
  for (int k = threadIdx.x; k < NKEYS; k += IX_THREADS) cnt[k] = 0;
  load_classes(cls2, cls3);
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * tile;
  for (int64_t c = 0; c < tile; c += IX_CHUNK) {
    int32_t key[IX_PER];
    const uint32_t valid = word_keys16(pad, base + c + (int64_t)threadIdx.x * IX_PER, n_pad, cls2, cls3, key);
#pragma unroll
    for (int j = 0; j < IX_PER; j++)
      if (valid >> j & 1) atomicAdd(&cnt[key[j]], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NKEYS; k += IX_THREADS) hist[(int64_t)k * n_tiles + blockIdx.x] = cnt[k];
}

// offT[t * NKEYS + k] = off[k * n_tiles + t]: the scanned slots tile-major,
// so that each tile of pass 2 reads its keys' slots contiguously (32 x 32
// blocks through shared memory, reads and writes coalesced).
__global__ void k_index_transpose(const int64_t* off, int64_t n_tiles, int64_t* offT) {
  __shared__ int64_t blk[32][33];
  const int64_t k0 = (int64_t)blockIdx.y * 32, t0 = (int64_t)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t k = k0 + r, t = t0 + threadIdx.x;
    if (k < NKEYS && t < n_tiles) blk[r][threadIdx.x] = off[k * n_tiles + t];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t t = t0 + r, k = k0 + threadIdx.x;
    if (k < NKEYS && t < n_tiles) offT[t * NKEYS + k] = blk[threadIdx.x][r];
  }
}

// key_off[k] = first slot of key k (its tile-0 slot), key_off[NKEYS] = total.
__global__ void k_index_key_off(const int64_t* off, int64_t n_tiles, const int64_t* total, int64_t* key_off) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NKEYS) key_off[k] = off[(int64_t)k * n_tiles];
  if (k == NKEYS) key_off[k] = *total;
}

// Pass 2: one warp per tile, in blocks of 512 positions: each lane computes
// the keys of 16 consecutive positions from one 16-byte load (the next
// block's load in flight meanwhile) and parks them in shared memory; the
// block is then ranked 32 positions at a time in position order, lanes
// holding the same key taking consecutive slots in lane order.  The 16 match
// masks of a block are formed before the slots are taken, so only the
// per-key slot counter orders the steps.  (The scattered 4-byte position
// stores bound this kernel: more, smaller tiles shorten each key's run of
// slots per tile and make it slower, not faster.)
constexpr int IX_BLOCK = 32 * IX_PER;  // 512 positions
__global__ void __launch_bounds__(32) k_index_scatter(const int8_t* pad, int64_t n_pad, int64_t tile,
                                                      const int64_t* offT, uint32_t* pos) {
  __shared__ int32_t next[NKEYS];
  __shared__ int16_t kb[IX_BLOCK];
  __shared__ int8_t cls2[NAA], cls3[NAA];
  const int lane = threadIdx.x;
  const int64_t* my_off = offT + (int64_t)blockIdx.x * NKEYS;
#pragma unroll 8
  for (int k = lane; k < NKEYS; k += 32) next[k] = (int32_t)my_off[k];
  load_classes(cls2, cls3);
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * tile, end = min(base + tile, n_pad);
  uint32_t w[5];
  load20(pad, base + (int64_t)lane * IX_PER, n_pad, w);
  for (int64_t q0 = base; q0 < end; q0 += IX_BLOCK) {
    {
      uint32_t wn[5];
      load20(pad, q0 + IX_BLOCK < end ? q0 + IX_BLOCK + (int64_t)lane * IX_PER : n_pad, n_pad, wn);
      const int64_t p0 = q0 + (int64_t)lane * IX_PER;
      int32_t key[IX_PER];
      const uint32_t valid = keys16_from(w, cls2, cls3, key);
#pragma unroll
      for (int j = 0; j < IX_PER; j++)
        kb[lane * IX_PER + j] = (int16_t)((valid >> j & 1) && p0 + j < end ? key[j] : -1);
#pragma unroll
      for (int c = 0; c < 5; c++) w[c] = wn[c];
    }
    __syncwarp();
    int k[IX_PER];
    unsigned peers[IX_PER];
#pragma unroll
    for (int j = 0; j < IX_PER; j++) {
      k[j] = kb[32 * j + lane];
      peers[j] = __match_any_sync(0xffffffffu, k[j] >= 0 ? k[j] : NKEYS + lane);
    }
#pragma unroll
    for (int j = 0; j < IX_PER; j++) {
      const int leader = __ffs(peers[j]) - 1;
      int slot = 0;
      if (k[j] >= 0 && lane == leader) {
        slot = next[k[j]];
        next[k[j]] = slot + __popc(peers[j]);
      }
      slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(peers[j] & ((1u << lane) - 1u));
      if (k[j] >= 0) pos[slot] = (uint32_t)(q0 + 32 * j + lane);
    }
    __syncwarp();
  }
}

// Window of indexed word i: cells 0..25 = pad[p .. p+25], cells 26..47 =
// pad[p-1], pad[p-2], .., pad[p-22]; one thread per window.  The thread reads
// the 48 bytes S[j] = pad[p - 22 + j] as four aligned 16-byte loads (pad is
// 16-byte aligned with slack on both sides, so the 64-byte cover stays inside
// it), selects and funnel-shifts their 12 words into place, and assembles the
// window: cells 0-25 are S[22..47], cells 26-47 are S[21], S[20], .., S[0].
// A warp's 32 windows are consecutive in nb: they pass through shared memory
// and leave as 16-byte stores of consecutive addresses.
constexpr int NB_THREADS = 256;
__global__ void __launch_bounds__(NB_THREADS) k_neighbourhoods(const int8_t* pad, const uint32_t* pos, int64_t n,
                                                               int8_t* nb) {
  __shared__ uint4 stage[NB_THREADS / 32][32 * 3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint4* my = stage[warp];
  for (int64_t w0 = ((int64_t)blockIdx.x * NB_THREADS + warp * 32); w0 < n; w0 += (int64_t)gridDim.x * NB_THREADS) {
    const int64_t i = w0 + lane;
    if (i < n) {
      const int64_t s0 = (int64_t)pos[i] - 22;
      const int64_t a = s0 & ~(int64_t)15;
      const int off = (int)(s0 - a), q = off >> 2;
      const uint32_t sh = 8u * (uint32_t)(off & 3);
      const uint4* src = reinterpret_cast<const uint4*>(pad + a);
      uint32_t raw[16];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const uint4 v = __ldg(src + c);
        raw[4 * c] = v.x;
        raw[4 * c + 1] = v.y;
        raw[4 * c + 2] = v.z;
        raw[4 * c + 3] = v.w;
      }
      uint32_t W[13], S[12];
#pragma unroll
      for (int k = 0; k < 13; k++) W[k] = q == 0 ? raw[k] : q == 1 ? raw[k + 1] : q == 2 ? raw[k + 2] : raw[k + 3];
#pragma unroll
      for (int k = 0; k < 12; k++) S[k] = __funnelshift_r(W[k], W[k + 1], sh);
      uint32_t o[12];
#pragma unroll
      for (int k = 0; k < 6; k++) o[k] = __funnelshift_r(S[5 + k], S[6 + k], 16);  // S[22 + 4k ..]
      o[6] = __byte_perm(S[11], S[5], 0x4532u);                                   // S46 S47 S21 S20
#pragma unroll
      for (int k = 7; k < 12; k++) o[k] = __byte_perm(S[11 - k], 0u, 0x0123u);    // S[4(11-k)+3] .. S[4(11-k)]
      my[3 * lane] = make_uint4(o[0], o[1], o[2], o[3]);
      my[3 * lane + 1] = make_uint4(o[4], o[5], o[6], o[7]);
      my[3 * lane + 2] = make_uint4(o[8], o[9], o[10], o[11]);
    }
    __syncwarp();
    const int cnt = (int)min((int64_t)32, n - w0);
    uint4* dst = reinterpret_cast<uint4*>(nb + w0 * WIN);
#pragma unroll
    for (int r = 0; r < 3; r++) {
      const int e = lane + 32 * r;
      if (e < 3 * cnt) dst[e] = my[e];
    }
    __syncwarp();
  }
}

__global__ void k_block_seq(const int64_t* pad_off, int32_t n_seqs, int64_t n_blk, int32_t* blk) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_blk; i += (int64_t)gridDim.x * blockDim.x)
    blk[i] = n_seqs > 0 ? find_seq(pad_off, n_seqs, i * SEQ_BLK) : 0;
}

__global__ void k_export_pos(const uint32_t* pos, int64_t n, const int64_t* pad_off, int32_t n_seqs, int32_t* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = pos[i];
    int32_t s = find_seq(pad_off, n_seqs, p);
    out[i] = (int32_t)(p - (int64_t)GAP * (s + 1));
  }
}

// ---------------------------------------------------------------------------
// Six-frame translation.  Standard genetic code, codons indexed by
// n1*16 + n2*4 + n3 with A C G T = 0 1 2 3.
// ---------------------------------------------------------------------------
__constant__ char c_code[65] = "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF";
__constant__ int8_t c_aa_of_letter[26];

// One thread per 16 consecutive translated residues: one binary search for
// the sequence (contig, frame) of the first, then a walk forward.
constexpr int TR_PER = 16;
__global__ void k_translate6(const uint8_t* dna, const int64_t* contig_off, int32_t n_contigs, const int64_t* seq_off,
                             int64_t n_aa, int8_t* aa) {
  // codon -> residue code, in shared memory (lanes read different entries,
  // which constant memory would serialise)
  __shared__ int8_t code_of[64];
  if (threadIdx.x < 64) {
    const char letter = c_code[threadIdx.x];
    code_of[threadIdx.x] = letter == '*' ? (int8_t)STOP : c_aa_of_letter[letter - 'A'];
  }
  __syncthreads();
  const int32_t n_seqs = 6 * n_contigs;
  const int64_t n_chunks = (n_aa + TR_PER - 1) / TR_PER;
  for (int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < n_chunks;
       ch += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t0 = ch * TR_PER, t1 = min(t0 + TR_PER, n_aa);
    // the last sequence with seq_off[s] <= t that is not empty holds t
    int32_t s = find_seq(seq_off, n_seqs, t0);
    for (int64_t t = t0; t < t1; t++) {
      while (s + 1 < n_seqs && seq_off[s + 1] <= t) s++;
      const int32_t c = s / 6, f = s % 6;
      const int64_t i = t - seq_off[s];
      const int64_t c0 = contig_off[c], L = contig_off[c + 1] - c0;
      const int64_t q = (f % 3) + 3 * i;
      int n1, n2, n3;
      if (f < 3) {
        n1 = dna[c0 + q];
        n2 = dna[c0 + q + 1];
        n3 = dna[c0 + q + 2];
      } else {
        n1 = 3 - dna[c0 + L - 1 - q];
        n2 = 3 - dna[c0 + L - 2 - q];
        n3 = 3 - dna[c0 + L - 3 - q];
      }
      aa[t] = code_of[n1 * 16 + n2 * 4 + n3];
    }
  }
}

cudaError_t upload_code_letters_once() {
  static std::atomic<bool> done[64];  // per device; calls may come from several threads
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && done[dev]) return cudaSuccess;
  int8_t m[26];
  for (int i = 0; i < 26; i++) m[i] = -1;
  for (int i = 0; i < NAA; i++) m[ALPHABET[i] - 'A'] = (int8_t)i;
  cudaError_t e = cudaMemcpyToSymbol(c_aa_of_letter, m, sizeof(m));
  if (e == cudaSuccess && dev < 64) done[dev] = true;
  return e;
}

static unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t launch_check_codes(const int8_t* codes, int64_t n, int lo, int hi, int* bad, cudaStream_t st) {
  if (n > 0) {
    note_launch();
    k_check_codes<<<grid_for(n, 256), 256, 0, st>>>(codes, n, lo, hi, bad);
  }
  return cudaGetLastError();
}

cudaError_t launch_build_pad(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, int64_t n_res, int hi,
                             int8_t* pad, int* bad, cudaStream_t st) {
  if (n_res > 0) {
    note_launch();
    k_build_pad<<<grid_for((n_res + 15) / 16, 256), 256, 0, st>>>(codes, seq_off, n_seqs, n_res, hi, pad, bad);
  }
  return cudaGetLastError();
}

int64_t index_tile(int64_t n_pad) {
  // about six one-warp CTAs on each of 152 SMs
  int64_t t = (n_pad + 912 - 1) / 912;
  t = (t + IX_CHUNK - 1) / IX_CHUNK * IX_CHUNK;
  return std::min<int64_t>(std::max<int64_t>(t, IX_CHUNK), 16 * IX_CHUNK);
}

cudaError_t launch_index_hist(const int8_t* pad, int64_t n_pad, int64_t tile, int64_t n_tiles, int32_t* hist,
                              cudaStream_t st) {
  if (n_tiles > 0) {
    note_launch();
    k_index_hist<<<(unsigned)n_tiles, IX_THREADS, 0, st>>>(pad, n_pad, tile, n_tiles, hist);
  }
  return cudaGetLastError();
}

cudaError_t launch_index_finish(const int8_t* pad, int64_t n_pad, int64_t tile, int64_t n_tiles, const int64_t* off,
                                int64_t* offT, const int64_t* total, int64_t* key_off, uint32_t* pos,
                                cudaStream_t st) {
  // one-warp CTAs with 35 KB of shared memory each: ask for the largest
  // shared-memory carveout so that six of them share an SM
  static std::atomic<bool> carveout_set[64];  // per device; calls may come from several threads
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !carveout_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_index_scatter, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    carveout_set[dev] = true;
  }
  note_launch();
  k_index_key_off<<<(NKEYS + 1 + 255) / 256, 256, 0, st>>>(off, n_tiles, total, key_off);
  if (n_tiles > 0) {
    note_launch();
    k_index_transpose<<<dim3((unsigned)((n_tiles + 31) / 32), (NKEYS + 31) / 32), dim3(32, 8), 0, st>>>(off, n_tiles,
                                                                                                     offT);
    note_launch();
    k_index_scatter<<<(unsigned)n_tiles, 32, 0, st>>>(pad, n_pad, tile, offT, pos);
  }
  return cudaGetLastError();
}

cudaError_t launch_neighbourhoods(const int8_t* pad, const uint32_t* pos, int64_t n, int8_t* nb, cudaStream_t st) {
  if (n > 0) {
    note_launch();
    k_neighbourhoods<<<grid_for(n, NB_THREADS), NB_THREADS, 0, st>>>(pad, pos, n, nb);
  }
  return cudaGetLastError();
}

cudaError_t launch_block_seq(const int64_t* pad_off, int32_t n_seqs, int64_t n_pad, int32_t* blk, cudaStream_t st) {
  const int64_t n_blk = n_pad / SEQ_BLK + 1;
  note_launch();
  k_block_seq<<<grid_for(n_blk, 256), 256, 0, st>>>(pad_off, n_seqs, n_blk, blk);
  return cudaGetLastError();
}

cudaError_t launch_export_pos(const uint32_t* pos, int64_t n, const int64_t* pad_off, int32_t n_seqs, int32_t* out,
                              cudaStream_t st) {
  if (n > 0) {
    note_launch();
    k_export_pos<<<grid_for(n, 256), 256, 0, st>>>(pos, n, pad_off, n_seqs, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_translate6(const uint8_t* dna, const int64_t* contig_off, int32_t n_contigs, const int64_t* seq_off,
                              int64_t n_aa, int8_t* aa, cudaStream_t st) {
  cudaError_t e = upload_code_letters_once();
  if (e != cudaSuccess) return e;
  if (n_aa > 0) {
    note_launch();
    k_translate6<<<grid_for((n_aa + TR_PER - 1) / TR_PER, 256), 256, 0, st>>>(dna, contig_off, n_contigs, seq_off,
                                                                              n_aa, aa);
  }
  return cudaGetLastError();
}

}  // namespace plast
