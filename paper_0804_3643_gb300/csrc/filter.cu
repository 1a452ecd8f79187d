// filter.cu -- Section 4.2's filter, applied to the stage-2 survivors.
#include "filter.cuh"

#include "common.cuh"

namespace plast {

// ---------------------------------------------------------------------------
// Section 4.2's filter as a gate on the survivors.  The paper filters the
// pairs before the ungapped extension to spare its CPU the extension of the
// ~97 % that fail; both gates only remove pairs, so the pairs kept are the
// same in either order.  Here every pair is extended anyway (the filter's
// raw score needs one table lookup per cell, as the extension does), and
// the raw score -- the sum of the positive substitution scores over the
// same 48-cell window, sentinel cells adding nothing -- is taken for the
// survivors only (about 0.2 % of the pairs).  One thread per survivor;
// passing survivors are compacted by warp-aggregated atomics.
// ---------------------------------------------------------------------------
// The 48 residues pad[start .. start + 48) as 12 words (little-endian bytes),
// from four aligned 16-byte loads: the padded bank is 16-byte aligned and has
// at least GAP - LEFT sentinels before the first window and GAP - RIGHT after
// the last, more than the 15 bytes the aligned cover reaches beyond.
static_assert(GAP >= LEFT + 15 && GAP >= RIGHT + 15, "the aligned cover of a window stays in the padding");
__device__ __forceinline__ void window_words(const int8_t* pad, int64_t start, uint32_t out[12]) {
  const int64_t base = start & ~(int64_t)15;
  const int off = (int)(start - base), q = off >> 2, r = off & 3;
  const uint4* src = reinterpret_cast<const uint4*>(pad + base);
  uint32_t w[16];
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const uint4 v = __ldg(src + c);
    w[4 * c] = v.x;
    w[4 * c + 1] = v.y;
    w[4 * c + 2] = v.z;
    w[4 * c + 3] = v.w;
  }
  uint32_t sw[13];
#pragma unroll
  for (int k = 0; k < 13; k++) sw[k] = q == 0 ? w[k] : q == 1 ? w[k + 1] : q == 2 ? w[k + 2] : w[k + 3];
#pragma unroll
  for (int k = 0; k < 12; k++) out[k] = __funnelshift_r(sw[k], sw[k + 1], 8 * r);
}

__global__ void k_filter_gate(const uint64_t* key, const uint32_t* val, int64_t n, const int64_t* n_dev, int sh,
                              const int8_t* pad1, const int8_t* pad2, int s0, uint64_t* okey, uint32_t* oval,
                              unsigned long long* ocount) {
  // positive parts of the substitution scores, row a at a * 32
  __shared__ uint8_t pos[NCODE * 32];
  for (int i = threadIdx.x; i < NCODE * 32; i += blockDim.x) {
    const int a = i >> 5, b = i & 31;
    pos[i] = b < NCODE ? (uint8_t)max(0, (int)c_score[a * NCODE + b]) : (uint8_t)0;
  }
  __syncthreads();
  if (n_dev) n = min(n, *n_dev);
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // whole warps walk the list together so the ballot below sees every lane
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t i = base + lane;
    bool keep = false;
    uint64_t k = 0;
    if (i < n) {
      k = key[i];
      const int64_t p1 = (int64_t)(k >> sh), p2 = (int64_t)(k & ((1ull << sh) - 1));
      uint32_t x[12], y[12];
      window_words(pad1, p1 - LEFT, x);
      window_words(pad2, p2 - LEFT, y);
      int f = 0;
#pragma unroll
      for (int c = 0; c < 12; c++)
#pragma unroll
        for (int b = 0; b < 4; b++) f += pos[((x[c] >> (8 * b)) & 0xff) * 32 + ((y[c] >> (8 * b)) & 0xff)];
      keep = f >= s0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) continue;
    unsigned long long at = 0;
    if (lane == 0) at = atomicAdd(ocount, (unsigned long long)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (keep) {
      const unsigned long long j = at + __popc(m & ((1u << lane) - 1));
      okey[j] = k;
      oval[j] = val[i];
    }
  }
}

cudaError_t launch_filter_gate(const uint64_t* key, const uint32_t* val, int64_t n, const int64_t* n_dev, int sh,
                               const int8_t* pad1, const int8_t* pad2, int s0, uint64_t* okey, uint32_t* oval,
                               unsigned long long* ocount, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  note_launch();
  k_filter_gate<<<(unsigned)b, 256, 0, st>>>(key, val, n, n_dev, sh, pad1, pad2, s0, okey, oval, ocount);
  return cudaGetLastError();
}

}  // namespace plast
