// prims.cu -- scoring tables, a device-wide exclusive scan and a stable LSD
// radix sort of (uint64 key, uint32 value) pairs.  The sort gives stage 0 its
// CSR order (positions stay increasing within a key because the sort is
// stable) and stage 2 its canonical record order.
#include <atomic>
#include <mutex>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"

namespace plast {

std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_total() { return g_launches.load(); }

__constant__ int8_t c_score[NCODE * NCODE];
__constant__ int8_t c_cls2[NAA];
__constant__ int8_t c_cls3[NAA];

static int code_of(char c) {
  const char* p = strchr(ALPHABET, c);
  return p ? (int)(p - ALPHABET) : -1;
}

void build_tables(Tables* t) {
  for (int a = 0; a < NCODE; a++)
    for (int b = 0; b < NCODE; b++) {
      int v;
      if (a == SENTINEL || b == SENTINEL) v = SENT_SCORE;
      else if (a == STOP && b == STOP) v = 1;
      else if (a == STOP || b == STOP) v = -4;
      else v = 0;  // filled from the transcription below
      t->score[a * NCODE + b] = (int8_t)v;
    }
  for (int a = 0; a < NAA; a++) {
    const char* s = B62_UPPER[a];
    for (int b = a; b < NAA; b++) {
      char* end;
      long v = strtol(s, &end, 10);
      s = end;
      t->score[a * NCODE + b] = t->score[b * NCODE + a] = (int8_t)v;
    }
  }
  for (int k = 0; k < 2; k++)
    for (const char* p = SEED_POS2[k]; *p; p++) {
      int c = code_of(*p);
      if (c >= 0) t->cls2[c] = (int8_t)k;
    }
  for (int k = 0; k < 11; k++)
    for (const char* p = SEED_POS3[k]; *p; p++) {
      int c = code_of(*p);
      if (c >= 0) t->cls3[c] = (int8_t)k;
    }
}

cudaError_t upload_tables_once() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  if (dev < 64 && done[dev]) return cudaSuccess;
  // keep freed stream-ordered memory in the pool: scratch and banks are
  // re-allocated on every call
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  Tables t;
  build_tables(&t);
  if ((e = cudaMemcpyToSymbol(c_score, t.score, sizeof(t.score))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_cls2, t.cls2, sizeof(t.cls2))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_cls3, t.cls3, sizeof(t.cls3))) != cudaSuccess) return e;
  if (dev < 64) done[dev] = true;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Exclusive scan, int32 in -> int64 out, in three passes over tiles of
// SCAN_TILE elements: tile sums, a one-CTA scan of the sums, tile scans.
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t s_warp[SCAN_THREADS / 32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < SCAN_THREADS / 32 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < SCAN_THREADS / 32) s_warp[lane] = w;
  }
  __syncthreads();
  int64_t before = warp ? s_warp[warp - 1] : 0;
  if (total) *total = s_warp[SCAN_THREADS / 32 - 1];
  int64_t r = before + x - v;
  __syncthreads();
  return r;
}

// n_dev (optional): the element count lives in device memory, at most n.
__device__ __forceinline__ int64_t count_of(int64_t n, const int64_t* n_dev) {
  return n_dev ? min(n, max(*n_dev, (int64_t)0)) : n;
}

__global__ void k_scan_tile_sums(const int32_t* in, int64_t n, int64_t* sums, const int64_t* n_dev) {
  n = count_of(n, n_dev);
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t acc = 0;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; r++) {
    int64_t i = base + r * SCAN_THREADS + threadIdx.x;
    if (i < n) acc += in[i];
  }
  int64_t tot;
  block_exclusive_scan(acc, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* sums, int64_t nt, int64_t* d_total) {
  int64_t carry = 0;
  for (int64_t b = 0; b < nt; b += SCAN_THREADS) {
    int64_t i = b + threadIdx.x;
    int64_t v = i < nt ? sums[i] : 0;
    int64_t tot;
    int64_t ex = block_exclusive_scan(v, &tot);
    if (i < nt) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void k_scan_tiles(const int32_t* in, int64_t n, const int64_t* sums, int64_t* out, const int64_t* n_dev) {
  n = count_of(n, n_dev);
  // thread t owns the contiguous items [t*ITEMS, t*ITEMS + ITEMS) of the tile
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int32_t v[SCAN_ITEMS];
  int64_t acc = 0;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; r++) {
    int64_t i = base + r;
    v[r] = i < n ? in[i] : 0;
    acc += v[r];
  }
  int64_t ex = block_exclusive_scan(acc, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; r++) {
    int64_t i = base + r;
    if (i < n) out[i] = ex;
    ex += v[r];
  }
}

size_t scan_tmp_bytes(int64_t n) {
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  return (size_t)(nt + 1) * sizeof(int64_t);
}

cudaError_t scan_exclusive(const int32_t* in, int64_t* out, int64_t n, int64_t* d_total, void* tmp,
                           size_t tmp_bytes, cudaStream_t st, const int64_t* n_dev) {
  if (n <= 0) {
    if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(int64_t), st);
    return cudaSuccess;
  }
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tmp_bytes < scan_tmp_bytes(n)) return cudaErrorInvalidValue;
  int64_t* sums = (int64_t*)tmp;
  note_launch();
  k_scan_tile_sums<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, n, sums, n_dev);
  note_launch();
  k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(sums, nt, d_total);
  note_launch();
  k_scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, n, sums, out, n_dev);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.  Per pass: tile histograms (digit-major
// so that one flat exclusive scan gives every tile's base per digit), the
// scan, then a stable scatter that ranks equal digits in element order.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void k_radix_hist(const uint64_t* keys, int64_t n, int shift, int32_t* hist, int64_t nt,
                             const int64_t* n_dev) {
  __shared__ int h[256];
  n = count_of(n, n_dev);
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; r++) {
    int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nt + blockIdx.x] = h[threadIdx.x];
}

// Scatter of one tile: ranks by digit as in a stable counting sort, the tile
// reordered by digit in shared memory, then written out digit run by digit
// run (consecutive threads write consecutive addresses).
__global__ void k_radix_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, int64_t n,
                                int shift, const int32_t* hist, const int64_t* off, int64_t nt,
                                const int64_t* n_dev) {
  n = count_of(n, n_dev);
  __shared__ int64_t s_base[256];  // global start of this tile's run of digit d
  __shared__ int s_start[256];     // start of digit d within the tile
  __shared__ int s_cnt[RS_WARPS][256];
  __shared__ int s_run[256];
  __shared__ int s_wsum[RS_WARPS];
  __shared__ uint64_t s_key[RS_TILE];
  __shared__ uint32_t s_val[RS_TILE];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  s_base[tid] = off[(int64_t)tid * nt + blockIdx.x];
  {  // exclusive scan of the tile's histogram over the digits (thread = digit)
    const int c = hist[(int64_t)tid * nt + blockIdx.x];
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; w++) before += s_wsum[w];
    s_start[tid] = before + x - c;
  }
  s_run[tid] = 0;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; r++) {
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) s_cnt[w][tid] = 0;
    __syncthreads();
    const int64_t i = base + r * RS_THREADS + tid;
    const bool valid = i < n;
    const uint64_t k = valid ? kin[i] : 0;
    const uint32_t v = valid ? vin[i] : 0;
    const int d = valid ? (int)((k >> shift) & 255) : 256 + lane;  // padding lanes get unique dummies
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) s_cnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      int run = s_run[tid];
#pragma unroll
      for (int w = 0; w < RS_WARPS; w++) {
        const int c = s_cnt[w][tid];
        s_cnt[w][tid] = run;
        run += c;
      }
      s_run[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const int lp = s_start[d] + s_cnt[warp][d] + rank;
      s_key[lp] = k;
      s_val[lp] = v;
    }
    __syncthreads();
  }
  const int in_tile = (int)min((int64_t)RS_TILE, n - base);
  for (int j = tid; j < in_tile; j += RS_THREADS) {
    const uint64_t k = s_key[j];
    const int d = (int)((k >> shift) & 255);
    const int64_t dst = s_base[d] + (j - s_start[d]);
    kout[dst] = k;
    vout[dst] = s_val[j];
  }
}

size_t radix_tmp_bytes(int64_t n) {
  int64_t nt = (n + RS_TILE - 1) / RS_TILE;
  size_t h = (size_t)256 * nt;
  return h * sizeof(int32_t) + h * sizeof(int64_t) + scan_tmp_bytes((int64_t)h) + 64;
}

cudaError_t radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                             int bits, void* tmp, size_t tmp_bytes, cudaStream_t st, bool* result_in_alt,
                             const int64_t* n_dev) {
  *result_in_alt = false;
  if ((n <= 1 && !n_dev) || n <= 0 || bits <= 0) return cudaSuccess;
  if (tmp_bytes < radix_tmp_bytes(n)) return cudaErrorInvalidValue;
  int64_t nt = (n + RS_TILE - 1) / RS_TILE;
  size_t h = (size_t)256 * nt;
  int32_t* hist = (int32_t*)tmp;
  int64_t* off = (int64_t*)((char*)tmp + ((h * sizeof(int32_t) + 15) & ~(size_t)15));
  void* stmp = (char*)off + h * sizeof(int64_t);
  size_t stmp_bytes = scan_tmp_bytes((int64_t)h);
  uint64_t *ki = keys, *ko = keys_alt;
  uint32_t *vi = vals, *vo = vals_alt;
  bool alt = false;
  for (int shift = 0; shift < bits; shift += 8) {
    note_launch();
    k_radix_hist<<<(unsigned)nt, RS_THREADS, 0, st>>>(ki, n, shift, hist, nt, n_dev);
    cudaError_t e = scan_exclusive(hist, off, (int64_t)h, nullptr, stmp, stmp_bytes, st);
    if (e != cudaSuccess) return e;
    note_launch();
    k_radix_scatter<<<(unsigned)nt, RS_THREADS, 0, st>>>(ki, vi, ko, vo, n, shift, hist, off, nt, n_dev);
    uint64_t* tk = ki;
    ki = ko;
    ko = tk;
    uint32_t* tv = vi;
    vi = vo;
    vo = tv;
    alt = !alt;
  }
  *result_in_alt = alt;
  return cudaGetLastError();
}

}  // namespace plast
