// api.cu -- the C ABI declared in include/plast.h.
//
// Host code only: argument checks, bank lifecycle, the stage-2 work list
// (tiles of bank-1 occurrences of one key, wide or narrow by measured cost,
// costliest first for the persistent queue), the tile-cost calibration,
// stream-ordered scratch, and the launch sequences of the calls.  Every step
// of the computation runs in the kernels of index.cu, ungapped.cu, gapped.cu
// and prims.cu.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <new>
#include <stdio.h>
#include <string.h>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bank.cuh"
#include "common.cuh"
#include "gapped.cuh"
#include "filter.cuh"
#include "full.cuh"
#include "index.cuh"
#include "ungapped.cuh"

namespace {

using namespace plast;

std::atomic<int> g_schedule{0};
std::atomic<int> g_timing{0};

// CUDA events recorded on the call's stream at the stage boundaries of the
// last stage-2 / stage-3.1 call of this thread (when timing is on).
struct StageTimer {
  cudaEvent_t ev[PLAST_MAX_STAGES + 1] = {};
  bool rec[PLAST_MAX_STAGES + 1] = {};
  void reset() {
    for (bool& r : rec) r = false;
  }
  void mark(int i, cudaStream_t st) {
    if (!g_timing.load(std::memory_order_relaxed) || i > PLAST_MAX_STAGES) return;
    if (!ev[i] && cudaEventCreate(&ev[i]) != cudaSuccess) return;
    if (cudaEventRecord(ev[i], st) == cudaSuccess) rec[i] = true;
  }
};
thread_local StageTimer t_timer;

// NVTX range over a scope (host timeline of the calls and their stages, for
// profilers; header-only, inert without one).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Fault injection for the failure paths: any single device allocation of
// the library above this many bytes fails as if the device were out of
// memory (0: no limit).
std::atomic<int64_t> g_alloc_limit{0};

cudaError_t dev_alloc_async(void** p, size_t bytes, cudaStream_t st) {
  const int64_t lim = g_alloc_limit.load(std::memory_order_relaxed);
  if (lim > 0 && (int64_t)bytes > lim) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, st);
}

cudaError_t dev_alloc(void** p, size_t bytes) {
  const int64_t lim = g_alloc_limit.load(std::memory_order_relaxed);
  if (lim > 0 && (int64_t)bytes > lim) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

int rc_of(cudaError_t e) {
  if (e == cudaSuccess) return PLAST_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return PLAST_E_OOM;
  }
  return PLAST_E_CUDA;
}

#define CK(x)                              \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return rc_of(e_); \
  } while (0)

// Stream-ordered scratch that is returned when the call ends.
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
  template <class T>
  cudaError_t get(T** out, size_t count) {
    void* p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = dev_alloc_async(&p, (bytes + 255) & ~(size_t)255, st);
    if (e != cudaSuccess) return e;
    ptrs.push_back(p);
    *out = (T*)p;
    return cudaSuccess;
  }
  void release(void* p) {
    for (auto& q : ptrs)
      if (q == p) {
        cudaFreeAsync(q, st);
        q = nullptr;
      }
    ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), nullptr), ptrs.end());
  }
};

int bits_for(int64_t v) {
  int b = 1;
  while (b < 62 && ((int64_t)1 << b) <= v) b++;
  return b;
}

int num_sms() {
  static std::atomic<int> sms[64];  // per device, 0 until first asked (calls may come from several threads)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64) {
    const int v = sms[dev].load(std::memory_order_relaxed);
    if (v) return v;
  }
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (n <= 0) n = 1;
  if (dev >= 0 && dev < 64) sms[dev].store(n, std::memory_order_relaxed);
  return n;
}

// Stage-2 tile costs in SM-nanoseconds: per slot (a bank-1 row of the tile's
// shape against a bank-2 window: 48 cells, whatever the tile's fill) and per
// tile.  A CTA moves through a key's bank-2 windows a pass at a time (32 warps
// x 4 windows wide, x 32 narrow), so a tile is charged its shape's rows x n2
// rounded up to that granularity.  Defaults from a GB300; plast_autotune
// measures them on the current device.
std::mutex g_cost_mu;
plast_tile_costs g_costs = {0.317, 2960.0, 0.479, 566.0, 0.616, 1101.0, 1.094, 1090.0, 12, 0, 0.416, 314.0};
// 0: by cost; 1: wide only; 2, 3, 4, 5: narrow tiles of 8, 4, 2, 16 rows only
std::atomic<int> g_shape{0};
constexpr int64_t WIDE_PASS = (UNG_THREADS / 32) * 4;     // bank-2 windows per CTA pass, wide tile
constexpr int64_t NARROW_PASS = UNG_NARROW_PASS;           // narrow tiles
int64_t round_up(int64_t n, int64_t g) { return (n + g - 1) / g * g; }

int shape_rows(int shape) {
  switch (shape) {
    case UNG_WIDE:
      return UNG_T1;
    case UNG_NARROW:
      return UNG_NT1;
    case UNG_NARROW4:
      return UNG_NT1 / 2;
    case UNG_NARROW16:
      return 2 * UNG_NT1;
    default:
      return UNG_NT1 / 4;
  }
}

double shape_slots(int shape, int64_t n2) {
  return (double)shape_rows(shape) * (double)round_up(n2, shape == UNG_WIDE ? WIDE_PASS : NARROW_PASS);
}

double tile_cost(const plast_tile_costs& c, int shape, int64_t n2) {
  const double slots = shape_slots(shape, n2);
  switch (shape) {
    case UNG_WIDE:
      return c.wide_slot * slots + c.wide_tile;
    case UNG_NARROW:
      return c.narrow_slot * slots + c.narrow_tile;
    case UNG_NARROW4:
      return c.narrow4_slot * slots + c.narrow4_tile;
    case UNG_NARROW16:
      return c.narrow16_slot * slots + c.narrow16_tile;
    default:
      return c.narrow2_slot * slots + c.narrow2_tile;
  }
}

// Stage-2 work list: for every key present in both banks, tiles of
// consecutive bank-1 occurrences.  Full wide tiles of UNG_T1 rows; the
// remainder (or a short list) goes to one wide tile or to narrow tiles,
// whichever the cost model says is cheaper: narrow tiles of 16 rows while 16
// or more rows remain (of 8 if those cost less per row), the last rows by the
// cheapest cover with tiles of 16, 8, 4 and 2 rows.
struct TileList {
  std::vector<int4> tiles;        // (key, first CSR index of bank 1, rows, shape)
  int64_t n_wide = 0;             // persistent order: the wide tiles come first
  int64_t pairs = 0;
};

// When a launch has too few tiles to keep its CTAs busy to the end (a small
// query bank: a few hundred keys with one or two bank-1 occurrences), the
// costliest tiles are cut along their bank-2 lists into pieces of whole
// passes, so that no piece costs more than about 1/4 of a CTA's share; the
// pieces re-sorted costliest first.  v[lo, hi) is one launch's tile list.
void split_long_tiles(const plast_tile_costs& c, std::vector<int4>& v, int64_t lo, int64_t hi, int64_t ctas) {
  if (hi <= lo || ctas <= 0) return;
  // the list is costliest first: a tile above twice the target exists only if
  // the first one is above it, and the target is at most the first tile's
  // cost times the tile count over 4 * ctas
  if (hi - lo > 8 * ctas) {
    const double c0 = tile_cost(c, tile_shape(v[lo]), (int64_t)v[lo].w - v[lo].z);
    double total = 0;
    for (int64_t i = lo; i < hi; i++) total += tile_cost(c, tile_shape(v[i]), (int64_t)v[i].w - v[i].z);
    if (c0 <= 2 * total / (4.0 * (double)ctas)) return;
  }
  auto cost = [&](const int4& t) { return tile_cost(c, tile_shape(t), (int64_t)t.w - t.z); };
  double total = 0;
  for (int64_t i = lo; i < hi; i++) total += cost(v[i]);
  const double target = total / (4.0 * (double)ctas);
  bool any = false;
  for (int64_t i = lo; i < hi && !any; i++) any = cost(v[i]) > 2 * target;
  if (!any) return;
  std::vector<std::pair<double, int4>> out;
  out.reserve((size_t)(hi - lo) * 2);
  for (int64_t i = lo; i < hi; i++) {
    const int4 t = v[i];
    const double ct = cost(t);
    const int shape = tile_shape(t);
    const int64_t pass = shape == UNG_WIDE ? WIDE_PASS : NARROW_PASS, n2 = (int64_t)t.w - t.z;
    const int64_t pieces = std::min<int64_t>((int64_t)std::ceil(ct / target), (n2 + pass - 1) / pass);
    if (ct <= 2 * target || pieces < 2) {
      out.push_back({ct, t});
      continue;
    }
    const int64_t chunk = round_up((n2 + pieces - 1) / pieces, pass);
    for (int64_t a = 0; a < n2; a += chunk) {
      const int4 p = make_tile(tile_key(t), t.y, tile_rows(t), shape, t.z + (int)a,
                               t.z + (int)std::min<int64_t>(a + chunk, n2));
      out.push_back({cost(p), p});
    }
  }
  std::stable_sort(out.begin(), out.end(),
                   [](const std::pair<double, int4>& x, const std::pair<double, int4>& y) { return x.first > y.first; });
  std::vector<int4> nv(v.begin(), v.begin() + lo);
  for (const auto& x : out) nv.push_back(x.second);
  nv.insert(nv.end(), v.begin() + hi, v.end());
  v.swap(nv);
}

void build_tiles_from(const int64_t* ko1, const int64_t* ko2, bool largest_first, TileList* tl,
                      const std::vector<char>* key_mask, int shape_override, int n_sms) {
  tl->tiles.clear();
  tl->pairs = 0;
  tl->n_wide = 0;
  plast_tile_costs c;
  {
    std::lock_guard<std::mutex> lk(g_cost_mu);
    c = g_costs;
  }
  const int mode = shape_override >= 0 ? shape_override : g_shape.load();
  // Keys in launch order: the persistent schedule takes them by decreasing
  // n2, which orders the tiles of each shape by decreasing cost (a tile's
  // cost depends on its shape and n2 only), so the tiles need no sort.
  std::vector<int> keys;
  keys.reserve(NKEYS);
  for (int k = 0; k < NKEYS; k++) {
    if (key_mask && !(*key_mask)[k]) continue;
    if (ko1[k + 1] == ko1[k] || ko2[k + 1] == ko2[k]) continue;
    keys.push_back(k);
  }
  if (largest_first) {
    // counting sort by decreasing ceil(n2 / 128), the quantity every tile
    // cost depends on (monotonically), stable in key order
    int64_t bmax = 0;
    for (const int k : keys) bmax = std::max<int64_t>(bmax, ko2[k + 1] - ko2[k]);
    const int NB = (int)std::min<int64_t>(round_up(bmax, WIDE_PASS) / WIDE_PASS + 1, 1 << 20);
    static thread_local std::vector<int32_t> count;
    count.assign((size_t)NB + 1, 0);
    auto bucket = [&](int k) {
      const int64_t b = round_up(ko2[k + 1] - ko2[k], WIDE_PASS) / WIDE_PASS;
      return NB - 1 - (int)std::min<int64_t>(b, NB - 1);
    };
    for (const int k : keys) count[bucket(k) + 1]++;
    for (int b = 0; b < NB; b++) count[b + 1] += count[b];
    std::vector<int> sorted(keys.size());
    for (const int k : keys) sorted[count[bucket(k)]++] = k;
    keys.swap(sorted);
  }
  // wide tiles, then narrow tiles of 16, 8, 4 and 2 rows, each in key order
  // (narrow tiles with their cost, for the merge)
  int64_t rows_total = 0;
  for (const int k : keys) rows_total += ko1[k + 1] - ko1[k];
  std::vector<int4> wide;
  std::vector<std::pair<float, int4>> by_shape[UNG_SHAPES];
  std::vector<int4>* out = largest_first ? nullptr : &tl->tiles;  // plain schedule: key by key
  if (out) {
    out->reserve((size_t)(rows_total / UNG_T1 + 4 * keys.size()));
  } else {
    wide.reserve((size_t)(rows_total / UNG_T1 + keys.size()));
    by_shape[UNG_NARROW16].reserve((size_t)(std::min<int64_t>(rows_total / 16, 8 * (int64_t)keys.size()) + 16));
    by_shape[UNG_NARROW].reserve(keys.size());
    by_shape[UNG_NARROW4].reserve(keys.size());
    by_shape[UNG_NARROW2].reserve(keys.size());
  }
  double cost_now[UNG_SHAPES] = {};  // tile costs of the current key's n2
  int32_t n2_now = 0;
  // cheapest cover of the last t < 16 rows of a key by narrow tiles (a tile
  // may hold fewer rows than its shape); the costs, hence the cover, depend
  // on n2 only through its pass count, so it is kept while that repeats
  constexpr int TAIL = 16;
  double best[TAIL];
  int pick[TAIL];
  int64_t cover_passes = -1;
  auto emit = [&](int k, int64_t first, int64_t rows, int shape) {
    const int4 t = make_tile(k, (int)first, (int)rows, shape, 0, n2_now);
    if (out) out->push_back(t);
    else if (shape == UNG_WIDE) wide.push_back(t);
    else by_shape[shape].push_back({(float)cost_now[shape], t});
  };
  for (const int k : keys) {
    const int64_t n1 = ko1[k + 1] - ko1[k];
    const int64_t n2 = ko2[k + 1] - ko2[k];
    tl->pairs += n1 * n2;
    n2_now = (int32_t)n2;
    for (int shape = UNG_NARROW; shape < UNG_SHAPES; shape++) cost_now[shape] = tile_cost(c, shape, n2);
    int64_t u = ko1[k];
    const int64_t end = ko1[k + 1];
    if (mode >= 2) {  // one narrow shape only
      const int shape = mode - 1, r = shape_rows(shape);
      for (; u < end; u += r) emit(k, u, std::min<int64_t>(r, end - u), shape);
      continue;
    }
    for (; end - u >= UNG_T1; u += UNG_T1) emit(k, u, UNG_T1, UNG_WIDE);
    const int64_t rem = end - u;
    if (rem <= 0) continue;
    if (mode == 1) {
      emit(k, u, rem, UNG_WIDE);
      continue;
    }
    if (round_up(n2, NARROW_PASS) != cover_passes) {
      cover_passes = round_up(n2, NARROW_PASS);
      best[0] = 0;
      pick[0] = 0;
      for (int t = 1; t < TAIL; t++) {
        best[t] = 0;
        pick[t] = -1;
        for (const int shape : {UNG_NARROW16, UNG_NARROW, UNG_NARROW4, UNG_NARROW2}) {
          const double v = cost_now[shape] + best[std::max(t - shape_rows(shape), 0)];
          if (pick[t] < 0 || v < best[t]) best[t] = v, pick[t] = shape;
        }
      }
    }
    // full tiles of 16 rows (or of 8 where those cost less per row), then
    // the cheapest cover of the rest; against one wide tile for it all
    const int bulk = cost_now[UNG_NARROW16] <= 2 * cost_now[UNG_NARROW] ? UNG_NARROW16 : UNG_NARROW;
    const int br = shape_rows(bulk);
    const int64_t full = rem / br;
    const int tail = (int)(rem % br);
    const double narrow_cost = (double)full * cost_now[bulk] + best[tail];
    if (!(narrow_cost < tile_cost(c, UNG_WIDE, n2))) {
      emit(k, u, rem, UNG_WIDE);
      continue;
    }
    for (int64_t i = 0; i < full; i++, u += br) emit(k, u, br, bulk);
    for (int t = tail; t > 0;) {
      const int shape = pick[t], r = std::min(shape_rows(shape), t);
      emit(k, u, r, shape);
      u += r;
      t -= r;
    }
  }
  if (!largest_first) {
    for (const int4& t : tl->tiles) tl->n_wide += tile_shape(t) == UNG_WIDE;
    return;
  }
  // wide tiles (one launch), then the narrow ones (another), costliest first:
  // a merge of the per-shape narrow lists, each already in cost order
  size_t total = wide.size();
  for (const auto& v : by_shape) total += v.size();
  tl->tiles.reserve(total);
  tl->tiles.insert(tl->tiles.end(), wide.begin(), wide.end());
  tl->n_wide = (int64_t)wide.size();
  size_t at[UNG_SHAPES] = {};
  for (;;) {
    int pickd = -1;
    float bestc = 0;
    for (int shape = UNG_NARROW; shape < UNG_SHAPES; shape++) {
      if (at[shape] >= by_shape[shape].size()) continue;
      const float v = by_shape[shape][at[shape]].first;
      if (pickd < 0 || v > bestc) pickd = shape, bestc = v;
    }
    if (pickd < 0) break;
    tl->tiles.push_back(by_shape[pickd][at[pickd]++].second);
  }
  if (n_sms > 0) {
    std::vector<int4> wide(tl->tiles.begin(), tl->tiles.begin() + tl->n_wide);
    std::vector<int4> narrow(tl->tiles.begin() + tl->n_wide, tl->tiles.end());
    split_long_tiles(c, wide, 0, (int64_t)wide.size(), (int64_t)n_sms);
    split_long_tiles(c, narrow, 0, (int64_t)narrow.size(), (int64_t)UNG_NARROW_CTAS_PER_SM * n_sms);
    tl->tiles.assign(wide.begin(), wide.end());
    tl->n_wide = (int64_t)wide.size();
    tl->tiles.insert(tl->tiles.end(), narrow.begin(), narrow.end());
  }
}

// Queues stage 2 over the tile list (its device copy is a.tiles): in the
// persistent schedule the wide kernel over the wide tiles and the narrow
// kernel over the rest, each on its own counter (counters[0], counters[1],
// zeroed by the caller); in the plain schedule, per key one launch of each
// kernel its tiles need.
cudaError_t launch_tiles(const TileList& tl, UngArgs a, int32_t* counters, bool persistent, cudaStream_t st) {
  const int64_t nt = (int64_t)tl.tiles.size();
  auto run = [&](int64_t lo, int64_t hi, bool wide, int32_t* counter) -> cudaError_t {
    if (hi <= lo) return cudaSuccess;
    a.tile_base = (int32_t)lo;
    a.n_tiles = (int32_t)(hi - lo);
    a.tile_counter = counter;
    a.persistent = persistent ? 1 : 0;
    const int per_sm = wide ? 1 : UNG_NARROW_CTAS_PER_SM;
    const int grid = persistent ? (int)std::min<int64_t>((int64_t)per_sm * num_sms(), hi - lo) : (int)(hi - lo);
    return wide ? launch_ungapped(a, grid, st) : launch_ungapped_narrow(a, grid, st);
  };
  if (persistent) {
    cudaError_t e = run(0, tl.n_wide, true, counters);
    return e != cudaSuccess ? e : run(tl.n_wide, nt, false, counters + 1);
  }
  for (int64_t i = 0; i < nt;) {
    int64_t j = i;
    const int key = tile_key(tl.tiles[i]);
    while (j < nt && tile_key(tl.tiles[j]) == key && tile_shape(tl.tiles[j]) == UNG_WIDE) j++;
    int64_t k = j;
    while (k < nt && tile_key(tl.tiles[k]) == key) k++;
    cudaError_t e = run(i, j, true, counters);
    if (e == cudaSuccess) e = run(j, k, false, counters + 1);
    if (e != cudaSuccess) return e;
    i = k;
  }
  return cudaSuccess;
}

void build_tiles(const plast_bank* b1, const plast_bank* b2, bool largest_first, TileList* tl,
                 const std::vector<char>* key_mask = nullptr, int shape_override = -1) {
  build_tiles_from(b1->h_key_off.data(), b2->h_key_off.data(), largest_first, tl, key_mask, shape_override,
                   largest_first ? num_sms() : 0);
}

// The survivor rate of the last stage 2 of each pair of banks, to size the
// next one's survivor buffer.  The first guess, pairs / 128, holds for
// ordinary protein banks (about 1 / 570 at S1 = 38), but keys with
// low-complexity runs pass far more often, and an overflowing first run is
// run again with the exact count; with the rate of the pair's last search
// the buffer fits at once.  Sizing only: no result depends on it.
struct RateHint {
  const plast_bank* b1;
  const plast_bank* b2;
  double rate;
};
std::mutex g_hint_mu;
RateHint g_hints[32] = {};
int g_hint_next = 0;

double rate_hint(const plast_bank* b1, const plast_bank* b2) {
  std::lock_guard<std::mutex> lk(g_hint_mu);
  for (const RateHint& h : g_hints)
    if (h.b1 == b1 && h.b2 == b2) return h.rate;
  return 0.0;
}

void set_rate_hint(const plast_bank* b1, const plast_bank* b2, double rate) {
  std::lock_guard<std::mutex> lk(g_hint_mu);
  for (RateHint& h : g_hints)
    if (h.b1 == b1 && h.b2 == b2) {
      h.rate = rate;
      return;
    }
  g_hints[g_hint_next] = RateHint{b1, b2, rate};
  g_hint_next = (g_hint_next + 1) % 32;
}

void forget_rate_hints(const plast_bank* b) {
  std::lock_guard<std::mutex> lk(g_hint_mu);
  for (RateHint& h : g_hints)
    if (h.b1 == b || h.b2 == b) h = RateHint{nullptr, nullptr, 0.0};
}

// Device state shared by the stage-2 calls: sorted survivor keys and values.
struct Survivors {
  uint64_t* key = nullptr;
  uint32_t* val = nullptr;
  int64_t n = 0;
  int sh = 0;  // key = padded pos1 << sh | padded pos2
};

// Stage 2 into scratch; the survivors come back in canonical (key) order
// when `sort`, else in the order the kernel wrote them.
int run_ungapped(const plast_bank* b1, const plast_bank* b2, const plast_params& prm, int32_t s0, cudaStream_t st,
                 Scratch& sc, Survivors* sv, const std::vector<char>* key_mask = nullptr, bool sort = true) {
  NvtxRange nvtx_("stage 2: tiles, ungapped kernels, survivors");
  sv->n = 0;
  sv->sh = b2->pad_bits;
  TileList tl;
  const int mode = g_schedule.load();
  build_tiles(b1, b2, mode == 0, &tl, key_mask);
  t_timer.mark(0, st);
  if (tl.tiles.empty()) return PLAST_OK;
  const int64_t nt = (int64_t)tl.tiles.size();
  if (nt > 0x7fffffff) return PLAST_E_INVALID;

  int4* d_tiles;
  int32_t* d_counter;
  unsigned long long* d_count;
  CK(sc.get(&d_tiles, nt));
  CK(sc.get(&d_counter, 2));
  CK(sc.get(&d_count, 1));
  CK(cudaMemcpyAsync(d_tiles, tl.tiles.data(), nt * sizeof(int4), cudaMemcpyHostToDevice, st));

  int64_t cap = tl.pairs / 128 + (1 << 20);
  const double hint = rate_hint(b1, b2);
  if (hint > 0.0) cap = std::max<int64_t>(cap, (int64_t)(hint * 1.1 * (double)tl.pairs) + (1 << 20));
  for (int attempt = 0; attempt < 2; attempt++) {
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    CK(sc.get(&k0, cap));
    CK(sc.get(&v0, cap));
    CK(cudaMemsetAsync(d_counter, 0, 2 * sizeof(int32_t), st));
    CK(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st));
    UngArgs a;
    a.nb1 = b1->nb;
    a.pos1 = b1->pos;
    a.nb2 = b2->nb;
    a.pos2 = b2->pos;
    a.key_off2 = b2->key_off;
    a.tiles = d_tiles;
    a.tile_counter = d_counter;
    a.s1 = prm.s1;
    a.out_key = k0;
    a.out_val = v0;
    a.out_count = d_count;
    a.cap = cap;
    a.sh = sv->sh;
    t_timer.mark(1, st);
    CK(launch_tiles(tl, a, d_counter, mode == 0, st));
    t_timer.mark(2, st);
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, d_count, sizeof(n), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (tl.pairs > 0) set_rate_hint(b1, b2, (double)n / (double)tl.pairs);
    if ((int64_t)n > cap) {
      sc.release(k0);
      sc.release(v0);
      cap = (int64_t)n + 1024;
      continue;
    }
    if (s0 > 0 && n > 0) {
      // Section 4.2's filter on the survivors
      uint64_t* kf;
      uint32_t* vf;
      CK(sc.get(&kf, (int64_t)n));
      CK(sc.get(&vf, (int64_t)n));
      CK(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st));
      CK(launch_filter_gate(k0, v0, (int64_t)n, nullptr, sv->sh, b1->pad, b2->pad, s0, kf, vf, d_count, st));
      CK(cudaMemcpyAsync(&n, d_count, sizeof(n), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      sc.release(k0);
      sc.release(v0);
      k0 = kf;
      v0 = vf;
    }
    sv->n = (int64_t)n;
    if (n == 0) return PLAST_OK;
    if (!sort) {
      t_timer.mark(3, st);
      sv->key = k0;
      sv->val = v0;
      return PLAST_OK;
    }
    CK(sc.get(&k1, n));
    CK(sc.get(&v1, n));
    void* tmp;
    size_t tb = radix_tmp_bytes((int64_t)n);
    CK(sc.get((char**)&tmp, tb));
    bool alt = false;
    CK(radix_sort_pairs(k0, v0, k1, v1, (int64_t)n, b1->pad_bits + sv->sh, tmp, tb, st, &alt));
    t_timer.mark(3, st);
    sv->key = alt ? k1 : k0;
    sv->val = alt ? v1 : v0;
    return PLAST_OK;
  }
  return PLAST_E_CUDA;
}

int check_bad(int* d_bad, cudaStream_t st, int* h_bad) {
  CK(cudaMemcpyAsync(h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PLAST_OK;
}

}  // namespace

extern "C" {

void plast_default_params(plast_params* p) {
  if (!p) return;
  p->w = 4;
  p->nl = 22;
  p->nr = 22;
  p->s1 = 38;
  p->lg = 64;
  p->band = 8;
  p->gap_open = 11;
  p->gap_extend = 1;
  p->s2 = 47;
}

const char* plast_strerror(int code) {
  switch (code) {
    case PLAST_OK: return "ok";
    case PLAST_E_INVALID: return "invalid argument";
    case PLAST_E_OOM: return "device allocation failed";
    case PLAST_E_CAPACITY: return "output capacity too small";
    case PLAST_E_CUDA: return "CUDA error";
    case PLAST_E_TIMEOUT: return "device-side wait timed out";
    default: return "unknown error";
  }
}

int plast_set_timing(int on) {
  g_timing.store(on ? 1 : 0);
  return PLAST_OK;
}

int plast_stage_times(double* ms, int n) {
  if (!ms || n < 0) return PLAST_E_INVALID;
  for (int i = 0; i < n; i++) {
    ms[i] = -1.0;
    if (i + 1 > PLAST_MAX_STAGES || !t_timer.rec[i] || !t_timer.rec[i + 1]) continue;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, t_timer.ev[i], t_timer.ev[i + 1]) == cudaSuccess) ms[i] = f;
  }
  return PLAST_OK;
}

long long plast_kernel_launches(void) { return plast::launch_total(); }

int plast_set_alloc_limit(int64_t bytes) {
  if (bytes < 0) return PLAST_E_INVALID;
  g_alloc_limit.store(bytes);
  return PLAST_OK;
}

int plast_set_schedule(int mode) {
  if (mode != 0 && mode != 1) return PLAST_E_INVALID;
  g_schedule.store(mode);
  return PLAST_OK;
}

void plast_bank_free(plast_bank* b) {
  if (!b) return;
  forget_rate_hints(b);
  if (b->ready) {
    cudaEventSynchronize(b->ready);  // the build may still be running on its stream
    cudaEventDestroy(b->ready);
  }
  // pool memory, returned in order with the legacy default stream
  for (void* p : {(void*)b->pad_alloc, (void*)b->pad_off, (void*)b->blk_seq, (void*)b->key_off, (void*)b->pos,
                  (void*)b->nb})
    if (p) cudaFreeAsync(p, 0);
  delete b;
}

int plast_bank_stats(const plast_bank* b, int32_t* n_seqs, int64_t* n_residues, int64_t* n_positions) {
  if (!b) return PLAST_E_INVALID;
  if (n_seqs) *n_seqs = b->n_seqs;
  if (n_residues) *n_residues = b->n_res;
  if (n_positions) *n_positions = b->n_idx;
  return PLAST_OK;
}

int64_t plast_pair_count(const plast_bank* b1, const plast_bank* b2) {
  if (!b1 || !b2) return -1;
  int64_t s = 0;
  for (int k = 0; k < NKEYS; k++)
    s += (b1->h_key_off[k + 1] - b1->h_key_off[k]) * (b2->h_key_off[k + 1] - b2->h_key_off[k]);
  return s;
}

int plast_index_bank(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, const plast_params* params,
                     void* stream, plast_bank** out) {
  NvtxRange nvtx_("plast_index_bank (stage 0)");
  if (!out || !seq_off || n_seqs < 0 || !params_ok(params)) return PLAST_E_INVALID;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  CK(upload_tables_once());
  std::vector<int64_t> h_off((size_t)n_seqs + 1);
  CK(cudaMemcpyAsync(h_off.data(), seq_off, h_off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h_off[0] != 0) return PLAST_E_INVALID;
  for (int32_t s = 0; s < n_seqs; s++)
    if (h_off[s + 1] < h_off[s]) return PLAST_E_INVALID;
  const int64_t n_res = h_off[n_seqs];
  const int64_t n_pad = n_res + (int64_t)GAP * (n_seqs + 1);
  if (n_pad >= ((int64_t)1 << 31)) return PLAST_E_INVALID;
  if (n_res > 0 && !codes) return PLAST_E_INVALID;

  plast_bank* b = new (std::nothrow) plast_bank();
  if (!b) return PLAST_E_OOM;
  cudaGetDevice(&b->device);
  b->n_seqs = n_seqs;
  b->n_res = n_res;
  b->n_pad = n_pad;
  b->pad_bits = bits_for(n_pad);
  b->h_pad_off.resize((size_t)n_seqs + 1);
  for (int32_t s = 0; s <= n_seqs; s++) b->h_pad_off[s] = h_off[s] + (int64_t)GAP * (s + 1);

  auto fail = [&](int rc) {
    plast_bank_free(b);
    return rc;
  };
  auto ck = [&](cudaError_t e) { return e == cudaSuccess ? PLAST_OK : rc_of(e); };
  int rc;
  {
    Scratch sc(st);
    int* d_bad;
    int64_t* d_seq_off;
    if ((rc = ck(sc.get(&d_bad, 1)))) return fail(rc);
    if ((rc = ck(cudaMemsetAsync(d_bad, 0, sizeof(int), st)))) return fail(rc);
    if ((rc = ck(dev_alloc_async((void**)&b->pad_alloc, (size_t)(n_pad + 2 * PAD_SLACK), st)))) return fail(rc);
    b->pad = b->pad_alloc + PAD_SLACK;
    if ((rc = ck(cudaMemsetAsync(b->pad_alloc, SENTINEL, (size_t)(n_pad + 2 * PAD_SLACK), st)))) return fail(rc);
    if ((rc = ck(dev_alloc_async((void**)&b->pad_off, ((size_t)n_seqs + 1) * sizeof(int64_t), st)))) return fail(rc);
    if ((rc = ck(dev_alloc_async((void**)&b->key_off, (NKEYS + 1) * sizeof(int64_t), st)))) return fail(rc);
    if ((rc = ck(cudaMemcpyAsync(b->pad_off, b->h_pad_off.data(), b->h_pad_off.size() * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, st))))
      return fail(rc);
    if ((rc = ck(dev_alloc_async((void**)&b->blk_seq, ((size_t)(n_pad / SEQ_BLK) + 1) * sizeof(int32_t), st))))
      return fail(rc);
    if ((rc = ck(launch_block_seq(b->pad_off, n_seqs, n_pad, b->blk_seq, st)))) return fail(rc);
    if ((rc = ck(sc.get(&d_seq_off, (size_t)n_seqs + 1)))) return fail(rc);
    if ((rc = ck(cudaMemcpyAsync(d_seq_off, seq_off, ((size_t)n_seqs + 1) * sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, st))))
      return fail(rc);
    if ((rc = ck(launch_build_pad(codes, d_seq_off, n_seqs, n_res, 20, b->pad, d_bad, st)))) return fail(rc);
    const int64_t ix_tile = index_tile(n_pad), n_tiles = (n_pad + ix_tile - 1) / ix_tile;
    const int64_t n_cells = (int64_t)NKEYS * n_tiles;
    int32_t* d_hist;
    int64_t *d_off, *d_total;
    if ((rc = ck(sc.get(&d_hist, n_cells)))) return fail(rc);
    if ((rc = ck(sc.get(&d_off, n_cells)))) return fail(rc);
    if ((rc = ck(sc.get(&d_total, 1)))) return fail(rc);
    if ((rc = ck(launch_index_hist(b->pad, n_pad, ix_tile, n_tiles, d_hist, st)))) return fail(rc);
    void* stmp;
    size_t stb = scan_tmp_bytes(n_cells);
    if ((rc = ck(sc.get((char**)&stmp, stb)))) return fail(rc);
    if ((rc = ck(scan_exclusive(d_hist, d_off, n_cells, d_total, stmp, stb, st)))) return fail(rc);
    int64_t n_idx = 0;
    int h_bad = 0;
    if ((rc = ck(cudaMemcpyAsync(&n_idx, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, st)))) return fail(rc);
    if ((rc = ck(cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st)))) return fail(rc);
    if ((rc = ck(cudaStreamSynchronize(st)))) return fail(rc);
    if (h_bad) return fail(PLAST_E_INVALID);
    b->n_idx = n_idx;
    if ((rc = ck(dev_alloc_async((void**)&b->pos, (size_t)std::max<int64_t>(n_idx, 1) * sizeof(uint32_t), st))))
      return fail(rc);
    int64_t* d_offT;
    if ((rc = ck(sc.get(&d_offT, n_cells)))) return fail(rc);
    if ((rc = ck(launch_index_finish(b->pad, n_pad, ix_tile, n_tiles, d_off, d_offT, d_total, b->key_off, b->pos,
                                     st))))
      return fail(rc);
    b->h_key_off.resize(NKEYS + 1);
    if ((rc = ck(cudaMemcpyAsync(b->h_key_off.data(), b->key_off, (NKEYS + 1) * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st))))
      return fail(rc);
    if ((rc = ck(cudaStreamSynchronize(st)))) return fail(rc);
    // the windows are laid out while the caller goes on (later calls wait on
    // b->ready)
    if ((rc = ck(dev_alloc_async((void**)&b->nb, (size_t)std::max<int64_t>(n_idx, 1) * WIN, st)))) return fail(rc);
    if ((rc = ck(launch_neighbourhoods(b->pad, b->pos, n_idx, b->nb, st)))) return fail(rc);
    if ((rc = ck(cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming)))) return fail(rc);
    if ((rc = ck(cudaEventRecord(b->ready, st)))) return fail(rc);
  }
  *out = b;
  return PLAST_OK;
}

int plast_bank_export_index(const plast_bank* b, int64_t* key_off, int32_t* pos, int64_t cap, int64_t* n_out,
                            void* stream) {
  if (!b || !n_out || !key_off) return PLAST_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  CK(bank_wait(b, st));
  *n_out = b->n_idx;
  if (cap < b->n_idx) return PLAST_E_CAPACITY;
  if (b->n_idx > 0 && !pos) return PLAST_E_INVALID;
  CK(cudaMemcpyAsync(key_off, b->key_off, (NKEYS + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  CK(launch_export_pos(b->pos, b->n_idx, b->pad_off, b->n_seqs, pos, st));
  CK(cudaStreamSynchronize(st));
  return PLAST_OK;
}

static int ungapped_impl(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                         const std::vector<char>* mask, plast_hit* out, int64_t cap, int64_t* n_out, void* stream);

// Key list -> mask (NULL: every key); false on a key outside 0..8799.
static bool key_mask(const int32_t* keys, int32_t n_keys, std::vector<char>* mask) {
  if (!keys) return true;
  mask->assign(NKEYS, 0);
  for (int32_t i = 0; i < n_keys; i++) {
    if (keys[i] < 0 || keys[i] >= NKEYS) return false;
    (*mask)[keys[i]] = 1;
  }
  return true;
}

int plast_ungapped(const plast_bank* b1, const plast_bank* b2, const plast_params* params, plast_hit* out,
                   int64_t cap, int64_t* n_out, void* stream) {
  return ungapped_impl(b1, b2, params, 0, nullptr, out, cap, n_out, stream);
}

int plast_ungapped_ex(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                      const int32_t* keys, int32_t n_keys, plast_hit* out, int64_t cap, int64_t* n_out,
                      void* stream) {
  if (n_keys < 0 || !s0_ok(s0)) return PLAST_E_INVALID;
  std::vector<char> mask;
  if (!key_mask(keys, n_keys, &mask)) return PLAST_E_INVALID;
  return ungapped_impl(b1, b2, params, s0, keys ? &mask : nullptr, out, cap, n_out, stream);
}

static int ungapped_impl(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                         const std::vector<char>* mask, plast_hit* out, int64_t cap, int64_t* n_out, void* stream) {
  NvtxRange nvtx_("plast_ungapped (stages 1-2)");
  if (!b1 || !b2 || !n_out || cap < 0 || !params_ok(params)) return PLAST_E_INVALID;
  const plast_params prm = resolve(params);
  cudaStream_t st = (cudaStream_t)stream;
  CK(bank_wait(b1, st));
  CK(bank_wait(b2, st));
  *n_out = 0;
  CK(upload_tables_once());
  t_timer.reset();
  Scratch sc(st);
  Survivors sv;
  int rc = run_ungapped(b1, b2, prm, s0, st, sc, &sv, mask);
  if (rc) return rc;
  *n_out = sv.n;
  if (sv.n > cap) return PLAST_E_CAPACITY;
  if (sv.n == 0) return PLAST_OK;
  if (!out) return PLAST_E_INVALID;
  int* d_bad;
  CK(sc.get(&d_bad, 1));
  CK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  CK(launch_expand_hits(sv.key, sv.val, sv.n, sv.sh, b1->pad, seq_map(b1), b2->pad, seq_map(b2), out, d_bad, st));
  int h_bad = 0;
  if ((rc = check_bad(d_bad, st, &h_bad))) return rc;
  return h_bad ? PLAST_E_CUDA : PLAST_OK;
}

namespace {

int run_gapped(const plast_bank* b1, const plast_bank* b2, const plast_params& prm, const uint64_t* key,
               const uint32_t* val, int64_t n, int sh, plast_gapped* out, int64_t cap, int64_t* n_out,
               cudaStream_t st, Scratch& sc) {
  *n_out = 0;
  if (n == 0) return PLAST_OK;
  GapArgs g;
  g.pad1 = b1->pad;
  g.pad2 = b2->pad;
  g.key = key;
  g.val = val;
  g.n = n;
  g.sh = sh;
  g.gap_open = prm.gap_open;
  g.gap_extend = prm.gap_extend;
  g.s2 = prm.s2;
  int64_t *at, *total;
  CK(sc.get(&g.score, n));
  CK(sc.get(&g.ends, n));
  CK(sc.get(&g.pass, n));
  CK(sc.get(&at, n));
  CK(sc.get(&total, 1));
  CK(launch_small_gapped(g, st));
  t_timer.mark(4, st);
  void* stmp;
  size_t stb = scan_tmp_bytes(n);
  CK(sc.get((char**)&stmp, stb));
  CK(scan_exclusive(g.pass, at, n, total, stmp, stb, st));
  int64_t m = 0;
  CK(cudaMemcpyAsync(&m, total, sizeof(m), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *n_out = m;
  if (m > cap) return PLAST_E_CAPACITY;
  if (m == 0) return PLAST_OK;
  if (!out) return PLAST_E_INVALID;
  CK(launch_gapped_compact(g, at, seq_map(b1), seq_map(b2), out, st));
  t_timer.mark(5, st);
  CK(cudaStreamSynchronize(st));
  return PLAST_OK;
}

// Stage 3.1 of a search: the survivors in any order; the passing ones are
// compacted, sorted by key (fewer than the survivors) and written as records
// in canonical order.
int run_gapped_search(const plast_bank* b1, const plast_bank* b2, const plast_params& prm, const Survivors& sv,
                      plast_gapped* out, int64_t cap, int64_t* n_out, cudaStream_t st, Scratch& sc) {
  NvtxRange nvtx_("stage 3.1 and the record sort");
  *n_out = 0;
  const int64_t n = sv.n;
  if (n == 0) return PLAST_OK;
  if (n > (int64_t)UINT32_MAX) return PLAST_E_CAPACITY;
  GapArgs g;
  g.pad1 = b1->pad;
  g.pad2 = b2->pad;
  g.key = sv.key;
  g.val = sv.val;
  g.n = n;
  g.sh = sv.sh;
  g.gap_open = prm.gap_open;
  g.gap_extend = prm.gap_extend;
  g.s2 = prm.s2;
  // the passing hits come out of stage 3.1 as (key, hit index), in any order
  uint64_t *rk0, *rk1;
  uint32_t *ri0, *ri1;
  CK(sc.get(&g.score, n));
  CK(sc.get(&g.ends, n));
  CK(sc.get(&g.pass, n));
  CK(sc.get(&rk0, n));
  CK(sc.get(&ri0, n));
  CK(sc.get(&g.rcount, 1));
  g.rkey = rk0;
  g.ridx = ri0;
  CK(cudaMemsetAsync(g.rcount, 0, sizeof(unsigned long long), st));
  CK(launch_small_gapped(g, st));
  t_timer.mark(4, st);
  CK(launch_compact_pass(g, st));
  unsigned long long mc = 0;
  CK(cudaMemcpyAsync(&mc, g.rcount, sizeof(mc), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int64_t m = (int64_t)mc;
  *n_out = m;
  if (m > cap) return PLAST_E_CAPACITY;
  if (m == 0) return PLAST_OK;
  if (!out) return PLAST_E_INVALID;
  CK(sc.get(&rk1, m));
  CK(sc.get(&ri1, m));
  void* rtmp;
  size_t rtb = radix_tmp_bytes(m);
  CK(sc.get((char**)&rtmp, rtb));
  bool alt = false;
  CK(radix_sort_pairs(rk0, ri0, rk1, ri1, m, b1->pad_bits + sv.sh, rtmp, rtb, st, &alt));
  CK(launch_write_sorted(g, alt ? rk1 : rk0, alt ? ri1 : ri0, m, nullptr, seq_map(b1), seq_map(b2), out, st));
  t_timer.mark(5, st);
  CK(cudaStreamSynchronize(st));
  return PLAST_OK;
}

}  // namespace

int plast_small_gapped(const plast_bank* b1, const plast_bank* b2, const plast_params* params, const plast_hit* in,
                       int64_t n_in, plast_gapped* out, int64_t cap, int64_t* n_out, void* stream) {
  NvtxRange nvtx_("plast_small_gapped (stage 3.1)");
  if (!b1 || !b2 || !n_out || n_in < 0 || cap < 0 || !params_ok(params)) return PLAST_E_INVALID;
  if (n_in > 0 && !in) return PLAST_E_INVALID;
  const plast_params prm = resolve(params);
  cudaStream_t st = (cudaStream_t)stream;
  CK(bank_wait(b1, st));
  CK(bank_wait(b2, st));
  *n_out = 0;
  CK(upload_tables_once());
  t_timer.reset();
  if (n_in == 0) return PLAST_OK;
  if (b1->n_seqs == 0 || b2->n_seqs == 0) return PLAST_E_INVALID;
  Scratch sc(st);
  uint64_t* key;
  uint32_t* val;
  int* d_bad;
  CK(sc.get(&key, n_in));
  CK(sc.get(&val, n_in));
  CK(sc.get(&d_bad, 1));
  CK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  const int sh = b2->pad_bits;
  CK(launch_hits_to_keys(in, n_in, b1->pad_off, b1->n_seqs, b2->pad_off, b2->n_seqs, sh, key, val, d_bad, st));
  int h_bad = 0;
  int rc = check_bad(d_bad, st, &h_bad);
  if (rc) return rc;
  if (h_bad) return PLAST_E_INVALID;
  return run_gapped(b1, b2, prm, key, val, n_in, sh, out, cap, n_out, st, sc);
}

static int search_impl(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                       const int32_t* keys, int32_t n_keys, plast_gapped* out, int64_t cap, int64_t* n_out,
                       int64_t* n_ungapped_out, void* stream) {
  NvtxRange nvtx_("plast_search");
  if (!b1 || !b2 || !n_out || cap < 0 || n_keys < 0 || !params_ok(params) || !s0_ok(s0)) return PLAST_E_INVALID;
  std::vector<char> mask;
  if (!key_mask(keys, n_keys, &mask)) return PLAST_E_INVALID;
  const plast_params prm = resolve(params);
  cudaStream_t st = (cudaStream_t)stream;
  CK(bank_wait(b1, st));
  CK(bank_wait(b2, st));
  *n_out = 0;
  if (n_ungapped_out) *n_ungapped_out = 0;
  CK(upload_tables_once());
  t_timer.reset();
  Scratch sc(st);
  Survivors sv;
  int rc = run_ungapped(b1, b2, prm, s0, st, sc, &sv, keys ? &mask : nullptr, false);
  if (rc) return rc;
  if (n_ungapped_out) *n_ungapped_out = sv.n;
  return run_gapped_search(b1, b2, prm, sv, out, cap, n_out, st, sc);
}

int plast_search(const plast_bank* b1, const plast_bank* b2, const plast_params* params, plast_gapped* out,
                 int64_t cap, int64_t* n_out, void* stream) {
  return search_impl(b1, b2, params, 0, nullptr, 0, out, cap, n_out, nullptr, stream);
}

int plast_search_ex(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                    const int32_t* keys, int32_t n_keys, plast_gapped* out, int64_t cap, int64_t* n_out,
                    int64_t* n_ungapped_out, void* stream) {
  return search_impl(b1, b2, params, s0, keys, n_keys, out, cap, n_out, n_ungapped_out, stream);
}

static thread_local int64_t t_full_cells = 0;  // cells of this thread's last plast_full_gapped

int64_t plast_full_gapped_cells(void) { return t_full_cells; }

int plast_full_gapped(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t xdrop,
                      int32_t s3, const plast_gapped* in, int64_t n_in, plast_alignment* out, int64_t cap,
                      int64_t* n_out, int64_t* n_extended_out, void* stream) {
  NvtxRange nvtx_("plast_full_gapped (stage 3.2)");
  t_full_cells = 0;
  if (!b1 || !b2 || !n_out || n_in < 0 || cap < 0 || !params_ok(params) || xdrop < 0 || xdrop > 30000)
    return PLAST_E_INVALID;
  if ((n_in > 0 && !in) || n_in > (int64_t)UINT32_MAX) return PLAST_E_INVALID;
  const plast_params prm = resolve(params);
  cudaStream_t st = (cudaStream_t)stream;
  CK(bank_wait(b1, st));
  CK(bank_wait(b2, st));
  *n_out = 0;
  if (n_extended_out) *n_extended_out = 0;
  CK(upload_tables_once());
  if (n_in == 0) return PLAST_OK;
  if (b1->n_seqs == 0 || b2->n_seqs == 0) return PLAST_E_INVALID;
  const int q1 = bits_for(b1->n_seqs), q2 = bits_for(b2->n_seqs);
  if (q1 > 24 || q2 > 24) return PLAST_E_INVALID;
  const int64_t n = n_in;
  Scratch sc(st);
  // canonical order of the records (padded positions), then the processing
  // order (pair of sequences, decreasing small gapped score; ties keep the
  // canonical order: the sort is stable)
  uint64_t *k0, *k1;
  uint32_t *v0, *v1, *canon, *proc;
  int* d_bad;
  CK(sc.get(&k0, n));
  CK(sc.get(&k1, n));
  CK(sc.get(&v0, n));
  CK(sc.get(&v1, n));
  CK(sc.get(&canon, n));
  CK(sc.get(&d_bad, 1));
  void* rtmp;
  const size_t rtb = radix_tmp_bytes(n);
  CK(sc.get((char**)&rtmp, rtb));
  CK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  const int sh = b2->pad_bits;
  CK(launch_full_canon(in, n, b1->pad_off, b1->n_seqs, b2->pad_off, b2->n_seqs, sh, k0, v0, d_bad, st));
  int h_bad = 0;
  int rc = check_bad(d_bad, st, &h_bad);
  if (rc) return rc;
  if (h_bad) return PLAST_E_INVALID;
  bool alt = false;
  CK(radix_sort_pairs(k0, v0, k1, v1, n, b1->pad_bits + sh, rtmp, rtb, st, &alt));
  CK(cudaMemcpyAsync(canon, alt ? v1 : v0, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  CK(launch_full_proc(in, canon, n, q2, k0, v0, st));
  CK(radix_sort_pairs(k0, v0, k1, v1, n, q1 + q2 + 16, rtmp, rtb, st, &alt));
  proc = alt ? v1 : v0;
  // pairs of sequences: their first positions in processing order
  int32_t *flag, *done, *keep;
  int64_t *at, *gstart, *ng, *m_dev, *ext_dev;
  CK(sc.get(&flag, n));
  CK(sc.get(&at, n));
  CK(sc.get(&gstart, n + 1));
  CK(sc.get(&ng, 1));
  void* stmp;
  const size_t stb = scan_tmp_bytes(n);
  CK(sc.get((char**)&stmp, stb));
  CK(launch_full_groups(in, proc, n, flag, nullptr, nullptr, nullptr, 0, st));
  CK(scan_exclusive(flag, at, n, ng, stmp, stb, st));
  CK(launch_full_groups(in, proc, n, flag, at, ng, gstart, 1, st));
  // the extensions
  const int64_t warps = std::min<int64_t>(full_gapped_warps(num_sms()), (n + 3) / 4 * 4);
  plast_alignment* res;
  uint8_t* arena;
  int32_t* segs;
  int* d_err;
  unsigned long long* d_cells;
  CK(sc.get(&res, n));
  CK(sc.get(&done, n));
  CK(sc.get(&arena, (size_t)warps * FG_ARENA));
  CK(sc.get(&segs, (size_t)warps * 3 * FG_SEGS));
  CK(sc.get(&d_err, 1));
  CK(sc.get(&d_cells, 2));  // the cell count, then the kernel's work counter
  CK(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  CK(cudaMemsetAsync(d_cells, 0, 2 * sizeof(unsigned long long), st));
  FullArgs fa;
  fa.pad1 = b1->pad;
  fa.pad2 = b2->pad;
  fa.pad_off1 = b1->pad_off;
  fa.pad_off2 = b2->pad_off;
  fa.in = in;
  fa.proc = proc;
  fa.gstart = gstart;
  fa.ng_dev = ng;
  fa.go = prm.gap_open;
  fa.ge = prm.gap_extend;
  fa.xdrop = xdrop;
  fa.res = res;
  fa.done = done;
  fa.arena = arena;
  fa.segs = segs;
  fa.err = d_err;
  fa.cells = d_cells;
  fa.next = reinterpret_cast<unsigned*>(d_cells + 1);
  t_timer.reset();
  t_timer.mark(0, st);
  CK(launch_full_gapped(fa, warps, st));
  t_timer.mark(1, st);
  // the alignments kept, in canonical order
  CK(sc.get(&keep, n));
  CK(sc.get(&m_dev, 1));
  CK(sc.get(&ext_dev, 1));
  CK(launch_full_keep(canon, n, done, res, s3, keep, st));
  CK(scan_exclusive(keep, at, n, m_dev, stmp, stb, st));
  CK(scan_exclusive(done, gstart, n, ext_dev, stmp, stb, st));
  int64_t m = 0, ext = 0;
  int h_err = 0;
  unsigned long long cells = 0;
  CK(cudaMemcpyAsync(&cells, d_cells, sizeof(cells), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&m, m_dev, sizeof(m), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ext, ext_dev, sizeof(ext), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&h_err, d_err, sizeof(h_err), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h_err) return PLAST_E_CAPACITY;
  t_full_cells = (int64_t)cells;
  *n_out = m;
  if (n_extended_out) *n_extended_out = ext;
  if (m > cap) return PLAST_E_CAPACITY;
  if (m == 0) return PLAST_OK;
  if (!out) return PLAST_E_INVALID;
  CK(launch_full_write(canon, n, keep, at, res, out, st));
  t_timer.mark(2, st);
  CK(cudaStreamSynchronize(st));
  return PLAST_OK;
}

int plast_translate6(const uint8_t* dna, const int64_t* contig_off, int32_t n_contigs, int8_t* aa_out,
                     int64_t aa_cap, int64_t* seq_off_out, int32_t* frame_meta_out, int64_t* n_aa_out,
                     void* stream) {
  NvtxRange nvtx_("plast_translate6");
  if (!contig_off || n_contigs < 0 || !n_aa_out) return PLAST_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  *n_aa_out = 0;
  std::vector<int64_t> h_off((size_t)n_contigs + 1);
  CK(cudaMemcpyAsync(h_off.data(), contig_off, h_off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h_off[0] != 0) return PLAST_E_INVALID;
  for (int32_t c = 0; c < n_contigs; c++)
    if (h_off[c + 1] < h_off[c]) return PLAST_E_INVALID;
  const int64_t n_nt = h_off[n_contigs];
  if (n_nt > 0 && !dna) return PLAST_E_INVALID;
  std::vector<int64_t> so((size_t)6 * n_contigs + 1);
  std::vector<int32_t> meta((size_t)12 * n_contigs);
  so[0] = 0;
  for (int32_t c = 0; c < n_contigs; c++) {
    const int64_t L = h_off[c + 1] - h_off[c];
    for (int f = 0; f < 6; f++) {
      const int64_t start = f % 3;
      const int64_t len = L > start ? (L - start) / 3 : 0;
      const size_t s = (size_t)6 * c + f;
      so[s + 1] = so[s] + len;
      meta[2 * s] = c;
      meta[2 * s + 1] = f < 3 ? f + 1 : -(f - 2);
    }
  }
  const int64_t n_aa = so.back();
  *n_aa_out = n_aa;
  if (n_aa > aa_cap) return PLAST_E_CAPACITY;
  if (!seq_off_out || (n_contigs > 0 && !frame_meta_out) || (n_aa > 0 && !aa_out)) return PLAST_E_INVALID;
  Scratch sc(st);
  int* d_bad;
  CK(sc.get(&d_bad, 1));
  CK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  CK(launch_check_codes((const int8_t*)dna, n_nt, 0, 3, d_bad, st));
  int h_bad = 0;
  int rc = check_bad(d_bad, st, &h_bad);
  if (rc) return rc;
  if (h_bad) return PLAST_E_INVALID;
  CK(cudaMemcpyAsync(seq_off_out, so.data(), so.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (n_contigs > 0)
    CK(cudaMemcpyAsync(frame_meta_out, meta.data(), meta.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CK(launch_translate6(dna, contig_off, n_contigs, seq_off_out, n_aa, aa_out, st));
  CK(cudaStreamSynchronize(st));
  return PLAST_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Planned search: every buffer sized up front, so the chain of stages 1-3.1
// runs with no allocation and no host synchronisation and can be captured in
// a CUDA graph.  The survivor count flows between kernels in device memory.
// ---------------------------------------------------------------------------
struct plast_plan {
  const plast_bank* b1 = nullptr;
  const plast_bank* b2 = nullptr;
  plast_params prm{};
  int32_t s0 = 0;  // Section 4.2's filter threshold (0: off)
  int device = 0;
  int64_t max_hits = 0, max_records = 0, n_tiles = 0;
  TileList tl;  // host copy of the work list (launch split)
  int sh = 0, bits = 0;
  int4* tiles = nullptr;
  int32_t* counter = nullptr;
  unsigned long long* count = nullptr;
  int64_t* n_dev = nullptr;   // survivors, clamped to max_hits
  int64_t* m_dev = nullptr;   // records, clamped to max_records
  uint64_t* k0 = nullptr;     // survivors (kernel order)
  uint32_t* v0 = nullptr;
  uint64_t* kf = nullptr;     // survivors through the S0 filter (when s0 > 0)
  uint32_t* vf = nullptr;
  unsigned long long* count_f = nullptr;
  uint64_t *rk0 = nullptr, *rk1 = nullptr;  // record keys and hit indexes, sorted
  uint32_t *ri0 = nullptr, *ri1 = nullptr;
  void* rtmp = nullptr;
  size_t rtb = 0;
  int32_t* score = nullptr;
  uint32_t* ends = nullptr;
  int32_t* pass = nullptr;
  int64_t* total = nullptr;   // passing hits (an unsigned long long counter)
  plast_gapped* out = nullptr;  // caller's buffer
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

void plast_plan_free(plast_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (void* q : {(void*)p->tiles, (void*)p->counter, (void*)p->count, (void*)p->n_dev, (void*)p->m_dev,
                  (void*)p->k0, (void*)p->v0, (void*)p->rk0, (void*)p->rk1, (void*)p->ri0, (void*)p->ri1, p->rtmp,
                  (void*)p->score, (void*)p->ends, (void*)p->pass, (void*)p->total,
                  (void*)p->kf, (void*)p->vf, (void*)p->count_f})
    if (q) cudaFree(q);
  delete p;
}

int plast_plan_create(const plast_bank* b1, const plast_bank* b2, const plast_params* params, int32_t s0,
                      int64_t max_hits, plast_gapped* records, int64_t max_records, void* stream,
                      plast_plan** out) {
  if (!b1 || !b2 || !out || !records || max_hits < 1 || max_records < 1 || !params_ok(params) || !s0_ok(s0))
    return PLAST_E_INVALID;
  if (max_hits > (int64_t)UINT32_MAX) return PLAST_E_INVALID;
  max_records = std::min(max_records, max_hits);  // a search never has more records than hits
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  CK(upload_tables_once());
  // the banks are complete before any run (runs may be captured in a graph)
  if (b1->ready) CK(cudaEventSynchronize(b1->ready));
  if (b2->ready) CK(cudaEventSynchronize(b2->ready));
  plast_plan* p = new (std::nothrow) plast_plan();
  if (!p) return PLAST_E_OOM;
  cudaGetDevice(&p->device);
  p->b1 = b1;
  p->b2 = b2;
  p->prm = resolve(params);
  p->s0 = s0;
  p->max_hits = max_hits;
  p->max_records = max_records;
  p->out = records;
  p->sh = b2->pad_bits;
  p->bits = b1->pad_bits + p->sh;
  auto fail = [&](cudaError_t e) {
    plast_plan_free(p);
    return rc_of(e);
  };
  TileList& tl = p->tl;
  build_tiles(b1, b2, true, &tl);
  p->n_tiles = (int64_t)tl.tiles.size();
  cudaError_t e;
  auto alloc = [&](void** q, size_t bytes) { return dev_alloc(q, bytes < 16 ? 16 : bytes); };
  p->rtb = radix_tmp_bytes(max_records);
  if ((e = alloc((void**)&p->tiles, sizeof(int4) * (size_t)std::max<int64_t>(p->n_tiles, 1))) ||
      (e = alloc((void**)&p->counter, 2 * sizeof(int32_t))) ||
      (e = alloc((void**)&p->count, sizeof(unsigned long long))) ||
      (e = alloc((void**)&p->n_dev, sizeof(int64_t))) || (e = alloc((void**)&p->m_dev, sizeof(int64_t))) ||
      (e = alloc((void**)&p->k0, 8 * (size_t)max_hits)) || (e = alloc((void**)&p->v0, 4 * (size_t)max_hits)) ||
      (e = alloc((void**)&p->rk0, 8 * (size_t)max_records)) || (e = alloc((void**)&p->rk1, 8 * (size_t)max_records)) ||
      (e = alloc((void**)&p->ri0, 4 * (size_t)max_records)) || (e = alloc((void**)&p->ri1, 4 * (size_t)max_records)) ||
      (e = alloc(&p->rtmp, p->rtb)) ||
      (e = alloc((void**)&p->score, 4 * (size_t)max_hits)) || (e = alloc((void**)&p->ends, 4 * (size_t)max_hits)) ||
      (e = alloc((void**)&p->pass, 4 * (size_t)max_hits)) ||
      (e = alloc((void**)&p->total, sizeof(unsigned long long))))
    return fail(e);
  if (p->s0 > 0 &&
      ((e = alloc((void**)&p->kf, 8 * (size_t)max_hits)) || (e = alloc((void**)&p->vf, 4 * (size_t)max_hits)) ||
       (e = alloc((void**)&p->count_f, sizeof(unsigned long long)))))
    return fail(e);
  if (p->n_tiles > 0 &&
      (e = cudaMemcpyAsync(p->tiles, tl.tiles.data(), sizeof(int4) * p->n_tiles, cudaMemcpyHostToDevice, st)))
    return fail(e);
  // set the kernels' shared-memory attributes now, outside any capture
  UngArgs none{};
  GapArgs gnone{};
  gnone.n = 0;
  if ((e = launch_ungapped(none, 0, st)) || (e = launch_ungapped_narrow(none, 0, st)) ||
      (e = launch_small_gapped(gnone, st)))
    return fail(e);
  if ((e = cudaStreamSynchronize(st))) return fail(e);
  *out = p;
  return PLAST_OK;
}

int plast_plan_run(plast_plan* p, void* stream) {
  NvtxRange nvtx_("plast_plan_run");
  if (!p) return PLAST_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(p->counter, 0, 2 * sizeof(int32_t), st));
  CK(cudaMemsetAsync(p->count, 0, sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(p->total, 0, sizeof(int64_t), st));
  if (p->n_tiles > 0) {
    UngArgs a;
    a.nb1 = p->b1->nb;
    a.pos1 = p->b1->pos;
    a.nb2 = p->b2->nb;
    a.pos2 = p->b2->pos;
    a.key_off2 = p->b2->key_off;
    a.tiles = p->tiles;
    a.n_tiles = (int32_t)p->n_tiles;
    a.tile_base = 0;
    a.tile_counter = p->counter;
    a.persistent = 1;
    a.s1 = p->prm.s1;
    a.out_key = p->k0;
    a.out_val = p->v0;
    a.out_count = p->count;
    a.cap = p->max_hits;
    a.sh = p->sh;
    CK(launch_tiles(p->tl, a, p->counter, true, st));
  }
  CK(launch_clamp_count(p->count, p->max_hits, p->n_dev, st));
  const bool filter = p->s0 > 0;
  if (filter) {
    CK(cudaMemsetAsync(p->count_f, 0, sizeof(unsigned long long), st));
    CK(launch_filter_gate(p->k0, p->v0, p->max_hits, p->n_dev, p->sh, p->b1->pad, p->b2->pad, p->s0, p->kf,
                          p->vf, p->count_f, st));
    CK(launch_clamp_count(p->count_f, p->max_hits, p->n_dev, st));
  }
  GapArgs g;
  g.pad1 = p->b1->pad;
  g.pad2 = p->b2->pad;
  g.key = filter ? p->kf : p->k0;
  g.val = filter ? p->vf : p->v0;
  g.n = p->max_hits;
  g.sh = p->sh;
  g.gap_open = p->prm.gap_open;
  g.gap_extend = p->prm.gap_extend;
  g.s2 = p->prm.s2;
  g.score = p->score;
  g.ends = p->ends;
  g.pass = p->pass;
  g.n_dev = p->n_dev;
  g.out_cap = p->max_records;
  g.rkey = p->rk0;  // the passing hits, appended in any order (sorted below)
  g.ridx = p->ri0;
  g.rcount = reinterpret_cast<unsigned long long*>(p->total);
  CK(launch_small_gapped(g, st));
  CK(launch_compact_pass(g, st));
  CK(launch_clamp_count(g.rcount, p->max_records, p->m_dev, st));
  bool alt = false;
  CK(radix_sort_pairs(p->rk0, p->ri0, p->rk1, p->ri1, p->max_records, p->bits, p->rtmp, p->rtb, st, &alt, p->m_dev));
  CK(launch_write_sorted(g, alt ? p->rk1 : p->rk0, alt ? p->ri1 : p->ri0, p->max_records, p->m_dev, seq_map(p->b1),
                         seq_map(p->b2), p->out, st));
  return PLAST_OK;
}

int plast_plan_capture(plast_plan* p, void* stream) {
  if (!p || !stream) return PLAST_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  if (p->graph) {
    cudaGraphDestroy(p->graph);
    p->graph = nullptr;
  }
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = plast_plan_run(p, stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return rc_of(e);
  p->graph = g;
  CK(cudaGraphInstantiate(&p->exec, g, 0));
  return PLAST_OK;
}

int plast_plan_launch(plast_plan* p, void* stream) {
  if (!p || !p->exec) return PLAST_E_INVALID;
  CK(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
  return PLAST_OK;
}

int plast_plan_result(const plast_plan* p, int64_t* n_records, int64_t* n_hits, void* stream) {
  if (!p || !n_records) return PLAST_E_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long hits = 0, kept = 0;
  int64_t recs = 0;
  CK(cudaMemcpyAsync(&hits, p->count, sizeof(hits), cudaMemcpyDeviceToHost, st));
  if (p->count_f) CK(cudaMemcpyAsync(&kept, p->count_f, sizeof(kept), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&recs, p->total, sizeof(recs), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (n_hits) *n_hits = (int64_t)(p->count_f && hits <= (unsigned long long)p->max_hits ? kept : hits);
  if ((int64_t)hits > p->max_hits) {
    *n_records = (int64_t)hits;
    return PLAST_E_CAPACITY;
  }
  *n_records = recs;
  return recs > p->max_records ? PLAST_E_CAPACITY : PLAST_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Tile-cost calibration: the stage-2 kernel timed on random banks with every
// tile wide, then every tile narrow, against a long and a short bank 2; a
// two-point fit per shape gives the cost per row slot x window and per tile.
// ---------------------------------------------------------------------------
namespace {

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// n_seqs random proteins of `len` residues (codes 0..19 uniform), indexed
int random_bank(int32_t n_seqs, int len, uint64_t seed, cudaStream_t st, plast_bank** out) {
  std::vector<int8_t> codes((size_t)n_seqs * len);
  std::vector<int64_t> off((size_t)n_seqs + 1);
  uint64_t x = seed;
  for (auto& c : codes) c = (int8_t)(splitmix(x) % 20);
  for (int32_t i = 0; i <= n_seqs; i++) off[i] = (int64_t)i * len;
  int8_t* d_codes = nullptr;
  int64_t* d_off = nullptr;
  CK(cudaMalloc(&d_codes, codes.size()));
  cudaError_t e = cudaMalloc(&d_off, off.size() * sizeof(int64_t));
  int rc = PLAST_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_codes, codes.data(), codes.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) rc = plast_index_bank(d_codes, d_off, n_seqs, nullptr, st, out);
  else rc = rc_of(e);
  cudaStreamSynchronize(st);
  cudaFree(d_codes);
  if (d_off) cudaFree(d_off);
  return rc;
}

// median device time (ms) of the stage-2 kernel over `reps` runs of the
// given shape; *slots = sum over tiles of the charged slots, *tiles = count
int time_stage2(const plast_bank* b1, const plast_bank* b2, int shape, cudaStream_t st, int reps, double* ms,
                double* slots, double* tiles) {
  TileList tl;
  CK(bank_wait(b1, st));
  CK(bank_wait(b2, st));
  build_tiles(b1, b2, true, &tl, nullptr, shape);
  *slots = 0;
  for (const int4& t : tl.tiles) {
    *slots += shape_slots(tile_shape(t), (int64_t)t.w - t.z);
  }
  *tiles = (double)tl.tiles.size();
  *ms = 0;
  if (tl.tiles.empty()) return PLAST_OK;
  Scratch sc(st);
  int4* d_tiles;
  int32_t* d_counter;
  unsigned long long* d_count;
  uint64_t* k0;
  uint32_t* v0;
  const int64_t cap = tl.pairs / 64 + (1 << 16);
  CK(sc.get(&d_tiles, tl.tiles.size()));
  CK(sc.get(&d_counter, 2));
  CK(sc.get(&d_count, 1));
  CK(sc.get(&k0, cap));
  CK(sc.get(&v0, cap));
  CK(cudaMemcpyAsync(d_tiles, tl.tiles.data(), tl.tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  UngArgs a;
  a.nb1 = b1->nb;
  a.pos1 = b1->pos;
  a.nb2 = b2->nb;
  a.pos2 = b2->pos;
  a.key_off2 = b2->key_off;
  a.tiles = d_tiles;
  a.n_tiles = (int32_t)tl.tiles.size();
  a.tile_base = 0;
  a.tile_counter = d_counter;
  a.persistent = 1;
  plast_params dp;
  plast_default_params(&dp);
  a.s1 = dp.s1;
  a.out_key = k0;
  a.out_val = v0;
  a.out_count = d_count;
  a.cap = cap;
  a.sh = b2->pad_bits;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PLAST_E_CUDA;
  }
  std::vector<float> t;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r <= reps && e == cudaSuccess; r++) {
    e = cudaMemsetAsync(d_counter, 0, 2 * sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_tiles(tl, a, d_counter, true, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float x = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
    if (r > 0) t.push_back(x);  // run 0 warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return rc_of(e);
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return PLAST_OK;
}

}  // namespace

extern "C" {

int plast_get_tile_costs(plast_tile_costs* out) {
  if (!out) return PLAST_E_INVALID;
  std::lock_guard<std::mutex> lk(g_cost_mu);
  *out = g_costs;
  out->wide_int16_cells = ungapped_variant_n16(ungapped_variant());
  out->wide_stage_depth = ungapped_variant_depth(ungapped_variant());
  return PLAST_OK;
}

int plast_set_tile_costs(const plast_tile_costs* c) {
  if (!c) return PLAST_E_INVALID;
  const double slot[UNG_SHAPES] = {c->wide_slot, c->narrow_slot, c->narrow4_slot, c->narrow2_slot, c->narrow16_slot};
  const double tile[UNG_SHAPES] = {c->wide_tile, c->narrow_tile, c->narrow4_tile, c->narrow2_tile, c->narrow16_tile};
  for (int i = 0; i < UNG_SHAPES; i++)
    if (!(slot[i] > 0) || !(tile[i] >= 0) || slot[i] > 1e6 || tile[i] > 1e12) return PLAST_E_INVALID;
  int variant = -1;
  const int depth = c->wide_stage_depth ? c->wide_stage_depth : 1;
  for (int v = 0; v < UNG_VARIANTS; v++)
    if (ungapped_variant_n16(v) == c->wide_int16_cells && ungapped_variant_depth(v) == depth) variant = v;
  if (variant < 0) return PLAST_E_INVALID;
  std::lock_guard<std::mutex> lk(g_cost_mu);
  g_costs = *c;
  g_costs.wide_stage_depth = depth;
  set_ungapped_variant(variant);
  return PLAST_OK;
}

int plast_stage2_tiles(const int64_t* key_off1, const int64_t* key_off2, int32_t n_sms, int32_t* tiles, int64_t cap,
                       int64_t* n_tiles) {
  if (!key_off1 || !key_off2 || !n_tiles || cap < 0 || n_sms < 0 || (cap > 0 && !tiles)) return PLAST_E_INVALID;
  for (int k = 0; k < NKEYS; k++)
    if (key_off1[k + 1] < key_off1[k] || key_off2[k + 1] < key_off2[k] || key_off1[k + 1] > INT32_MAX ||
        key_off2[k + 1] - key_off2[k] > INT32_MAX)
      return PLAST_E_INVALID;
  TileList tl;
  const bool persistent = g_schedule.load() == 0;
  build_tiles_from(key_off1, key_off2, persistent, &tl, nullptr, -1, persistent ? n_sms : 0);
  *n_tiles = (int64_t)tl.tiles.size();
  if (*n_tiles > cap) return PLAST_E_CAPACITY;
  for (size_t i = 0; i < tl.tiles.size(); i++) {
    const int4 t = tl.tiles[i];
    int32_t* o = tiles + 6 * i;
    o[0] = tile_key(t);
    o[1] = t.y;
    o[2] = tile_rows(t);
    o[3] = tile_shape(t);
    o[4] = t.z;
    o[5] = t.w;
  }
  return PLAST_OK;
}

int plast_set_tile_shape(int mode) {
  if (mode < 0 || mode > UNG_SHAPES) return PLAST_E_INVALID;
  g_shape.store(mode);
  return PLAST_OK;
}

int plast_autotune(void* stream, plast_tile_costs* out) {
  cudaStream_t st = (cudaStream_t)stream;
  CK(upload_tables_once());
  plast_bank *b1 = nullptr, *b2l = nullptr, *b2s = nullptr;
  // bank 1: ~10 occurrences per key; bank 2: ~4,100 (four narrow passes)
  // and ~300 (two wide passes, a fraction of a narrow one) per key
  int rc = random_bank(300, 300, 11, st, &b1);
  if (rc == PLAST_OK) rc = random_bank(120000, 300, 12, st, &b2l);
  if (rc == PLAST_OK) rc = random_bank(9000, 300, 13, st, &b2s);
  plast_tile_costs c;
  plast_get_tile_costs(&c);
  const double sms = (double)num_sms();
  // slot and tile cost of a shape from its times on the long and short bank 2
  auto fit = [&](int shape, double* slot, double* tile, double* t_long) {
    double t_l, s_l, n_l, t_s, s_s, n_s;
    int r = time_stage2(b1, b2l, shape, st, 3, &t_l, &s_l, &n_l);
    if (r == PLAST_OK) r = time_stage2(b1, b2s, shape, st, 3, &t_s, &s_s, &n_s);
    if (r != PLAST_OK) return r;
    // SM-nanoseconds = slot cost x slots + tile cost x tiles, for both banks
    const double y_l = t_l * 1e6 * sms, y_s = t_s * 1e6 * sms;
    const double det = s_l * n_s - s_s * n_l;
    *slot = det != 0 ? (y_l * n_s - y_s * n_l) / det : 0;
    *tile = det != 0 ? (s_l * y_s - s_s * y_l) / det : 0;
    if (!(*slot > 0) || !(*tile >= 0)) {
      *slot = y_l / std::max(s_l, 1.0);
      *tile = 0;
    }
    *t_long = t_l;
    return PLAST_OK;
  };
  const int saved_variant = ungapped_variant();
  double best_t = 0;
  int best_v = saved_variant;
  // the int16 cells at staging depth 1, then the staging depths of the best
  auto try_variant = [&](int v, bool first) {
    set_ungapped_variant(v);
    double slot, tile, t_long;
    rc = fit(1, &slot, &tile, &t_long);
    if (rc == PLAST_OK && (first || t_long < best_t)) {
      best_t = t_long;
      best_v = v;
      c.wide_slot = slot;
      c.wide_tile = tile;
      c.wide_int16_cells = ungapped_variant_n16(v);
      c.wide_stage_depth = ungapped_variant_depth(v);
    }
  };
  for (int v = 0; v < UNG_N16_VARIANTS && rc == PLAST_OK; v++) try_variant(v, v == 0);
  for (int v = best_v % UNG_N16_VARIANTS + UNG_N16_VARIANTS; v < UNG_VARIANTS && rc == PLAST_OK;
       v += UNG_N16_VARIANTS)
    try_variant(v, false);
  set_ungapped_variant(rc == PLAST_OK ? best_v : saved_variant);
  double t_long;
  if (rc == PLAST_OK) rc = fit(2, &c.narrow_slot, &c.narrow_tile, &t_long);
  if (rc == PLAST_OK) rc = fit(3, &c.narrow4_slot, &c.narrow4_tile, &t_long);
  if (rc == PLAST_OK) rc = fit(4, &c.narrow2_slot, &c.narrow2_tile, &t_long);
  if (rc == PLAST_OK) rc = fit(5, &c.narrow16_slot, &c.narrow16_tile, &t_long);
  plast_bank_free(b1);
  plast_bank_free(b2l);
  plast_bank_free(b2s);
  if (rc != PLAST_OK) return rc;
  rc = plast_set_tile_costs(&c);
  if (rc == PLAST_OK && out) *out = c;
  return rc;
}

}  // extern "C"
