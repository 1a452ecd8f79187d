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
#include "common.cuh"
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

__global__ void k_scatter_codes(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, int64_t n_res,
                                int8_t* pad) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_res; p += (int64_t)gridDim.x * blockDim.x) {
    int32_t s = find_seq(seq_off, n_seqs, p);
    pad[p + (int64_t)GAP * (s + 1)] = codes[p];
  }
}

// Key of the word starting at every padded position; -1 where the word holds
// a stop or a sentinel (so no word crosses a sequence end).
__global__ void k_word_keys(const int8_t* pad, int64_t n_pad, int32_t* key, int32_t* flag) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    int k = -1;
    if (p + 3 < n_pad) k = seed_key(pad[p], pad[p + 1], pad[p + 2], pad[p + 3]);
    key[p] = k;
    flag[p] = k >= 0;
  }
}

__global__ void k_compact_words(const int32_t* key, const int64_t* at, int64_t n_pad, uint64_t* okey, uint32_t* opos) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * blockDim.x) {
    int k = key[p];
    if (k >= 0) {
      int64_t d = at[p];
      okey[d] = (uint64_t)k;
      opos[d] = (uint32_t)p;
    }
  }
}

__global__ void k_key_offsets(const uint64_t* skey, int64_t n, int64_t* key_off) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    int prev = i == 0 ? -1 : (int)skey[i - 1];
    int cur = i == n ? NKEYS : (int)skey[i];
    for (int k = prev + 1; k <= cur; k++) key_off[k] = i;
  }
}

// Window of indexed word i: cells 0..25 = pad[p .. p+25], cells 26..47 =
// pad[p-1], pad[p-2], .., pad[p-22]; one thread per window.  The thread reads
// the 48 bytes S[j] = pad[p - 22 + j] with 13 aligned word loads (pad has
// slack on both sides, so the rounded range stays inside it), forms their 12
// words with funnel shifts, and writes the window as three 16-byte stores:
// cells 0-25 are S[22..47], cells 26-47 are S[21], S[20], .., S[0].
__global__ void k_neighbourhoods(const int8_t* pad, const uint32_t* pos, int64_t n, int8_t* nb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = (int64_t)pos[i] - 22;
    const uint32_t* w = reinterpret_cast<const uint32_t*>(pad + (s0 & ~(int64_t)3));
    const uint32_t sh = 8u * (uint32_t)(s0 & 3);
    uint32_t raw[13], S[12];
#pragma unroll
    for (int k = 0; k < 13; k++) raw[k] = __ldg(w + k);
#pragma unroll
    for (int k = 0; k < 12; k++) S[k] = __funnelshift_r(raw[k], raw[k + 1], sh);
    uint32_t o[12];
#pragma unroll
    for (int q = 0; q < 6; q++) o[q] = __funnelshift_r(S[5 + q], S[6 + q], 16);  // S[22 + 4q ..]
    o[6] = __byte_perm(S[11], S[5], 0x4532u);                                   // S46 S47 S21 S20
#pragma unroll
    for (int q = 7; q < 12; q++) o[q] = __byte_perm(S[11 - q], 0u, 0x0123u);    // S[4(11-q)+3] .. S[4(11-q)]
    uint4* d = reinterpret_cast<uint4*>(nb + i * WIN);
    d[0] = make_uint4(o[0], o[1], o[2], o[3]);
    d[1] = make_uint4(o[4], o[5], o[6], o[7]);
    d[2] = make_uint4(o[8], o[9], o[10], o[11]);
  }
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

__global__ void k_translate6(const uint8_t* dna, const int64_t* contig_off, int32_t n_contigs, const int64_t* seq_off,
                             int64_t n_aa, int8_t* aa) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_aa; t += (int64_t)gridDim.x * blockDim.x) {
    int32_t s = find_seq(seq_off, 6 * n_contigs, t);
    // the last sequence with seq_off[s] <= t that is not empty holds t
    int32_t c = s / 6, f = s % 6;
    int64_t i = t - seq_off[s];
    int64_t c0 = contig_off[c], L = contig_off[c + 1] - c0;
    int64_t q = (f % 3) + 3 * i;
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
    char letter = c_code[n1 * 16 + n2 * 4 + n3];
    aa[t] = letter == '*' ? (int8_t)STOP : c_aa_of_letter[letter - 'A'];
  }
}

cudaError_t upload_code_letters_once() {
  static bool done[64] = {false};
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

cudaError_t launch_build_pad(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, int64_t n_res, int8_t* pad,
                             int64_t n_pad, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(pad, SENTINEL, (size_t)n_pad, st);
  if (e != cudaSuccess) return e;
  if (n_res > 0) {
    note_launch();
    k_scatter_codes<<<grid_for(n_res, 256), 256, 0, st>>>(codes, seq_off, n_seqs, n_res, pad);
  }
  return cudaGetLastError();
}

cudaError_t launch_word_keys(const int8_t* pad, int64_t n_pad, int32_t* key, int32_t* flag, cudaStream_t st) {
  note_launch();
  k_word_keys<<<grid_for(n_pad, 256), 256, 0, st>>>(pad, n_pad, key, flag);
  return cudaGetLastError();
}

cudaError_t launch_compact_words(const int32_t* key, const int64_t* at, int64_t n_pad, uint64_t* okey, uint32_t* opos,
                                 cudaStream_t st) {
  note_launch();
  k_compact_words<<<grid_for(n_pad, 256), 256, 0, st>>>(key, at, n_pad, okey, opos);
  return cudaGetLastError();
}

cudaError_t launch_key_offsets(const uint64_t* skey, int64_t n, int64_t* key_off, cudaStream_t st) {
  note_launch();
  k_key_offsets<<<grid_for(n + 1, 256), 256, 0, st>>>(skey, n, key_off);
  return cudaGetLastError();
}

cudaError_t launch_neighbourhoods(const int8_t* pad, const uint32_t* pos, int64_t n, int8_t* nb, cudaStream_t st) {
  if (n > 0) {
    note_launch();
    k_neighbourhoods<<<grid_for(n, 256), 256, 0, st>>>(pad, pos, n, nb);
  }
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
    k_translate6<<<grid_for(n_aa, 256), 256, 0, st>>>(dna, contig_off, n_contigs, seq_off, n_aa, aa);
  }
  return cudaGetLastError();
}

}  // namespace plast
