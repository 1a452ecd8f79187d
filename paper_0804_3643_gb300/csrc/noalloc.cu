// noalloc.cu -- plast_small_gapped_noalloc: the small gapped extension
// (stage 3.1) for callers that must not allocate device memory.
//
// plast_small_gapped takes its working buffers (hit keys, per-hit scores,
// end cells, pass flags, scan offsets) from the stream-ordered allocator on
// every call.  Some callers cannot let a library allocate: a framework that
// has reserved the GPU's memory for its own allocator up front, or a
// latency-bound serving loop that must not risk an allocation's implicit
// synchronisation or an out-of-memory failure in the middle of a request.
// This entry point runs the same kernels on a fixed scratch area that lives
// in this file as a static device array, sized for at most
// PLAST_NOALLOC_MAX_HITS hits, which every GPU that loads the library holds
// until the process exits.  It calls no cudaMalloc, cudaFree or allocating
// library routine.
#include <mutex>

#include "bank.cuh"
#include "common.cuh"
#include "gapped.cuh"
#include "ungapped.cuh"

namespace {

using namespace plast;

constexpr int64_t NMAX = PLAST_NOALLOC_MAX_HITS;

// Byte offsets of the scratch arrays, each 256-byte aligned.
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_KEY = 0;
constexpr size_t OFF_VAL = OFF_KEY + align256(NMAX * sizeof(uint64_t));
constexpr size_t OFF_SCORE = OFF_VAL + align256(NMAX * sizeof(uint32_t));
constexpr size_t OFF_ENDS = OFF_SCORE + align256(NMAX * sizeof(int32_t));
constexpr size_t OFF_PASS = OFF_ENDS + align256(NMAX * sizeof(uint32_t));
constexpr size_t OFF_AT = OFF_PASS + align256(NMAX * sizeof(int32_t));
constexpr size_t OFF_TOTAL = OFF_AT + align256(NMAX * sizeof(int64_t));
constexpr size_t OFF_BAD = OFF_TOTAL + 256;
constexpr size_t OFF_SCAN = OFF_BAD + 256;
constexpr size_t SCAN_BYTES = 4096;  // >= scan_tmp_bytes(NMAX), checked at run time
constexpr size_t SCRATCH_BYTES = OFF_SCAN + SCAN_BYTES;
static_assert(SCRATCH_BYTES <= (size_t)PLAST_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

// The scratch area.  In host code this name is only a handle for the runtime:
// kernels get its device address from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PLAST_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current and kept for the life of the process (a device reset, which
// gives the device a new context, invalidates it; the header says so).
unsigned char* scratch_on_current_device(cudaError_t* err) {
  static std::mutex mu;
  static unsigned char* addr[64] = {nullptr};
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = (unsigned char*)p;
  }
  return addr[dev];
}

int rc_of(cudaError_t e) { return e == cudaSuccess ? PLAST_OK : PLAST_E_CUDA; }

#define CKN(x)                                \
  do {                                        \
    cudaError_t e_ = (x);                     \
    if (e_ != cudaSuccess) return rc_of(e_);  \
  } while (0)

}  // namespace

extern "C" int plast_small_gapped_noalloc(const plast_bank* b1, const plast_bank* b2, const plast_params* params,
                                          const plast_hit* in, int64_t n_in, plast_gapped* out, int64_t cap,
                                          int64_t* n_out, void* stream) {
  if (!b1 || !b2 || !n_out || n_in < 0 || cap < 0) return PLAST_E_INVALID;
  if (n_in > NMAX) return PLAST_E_INVALID;
  if (n_in > 0 && !in) return PLAST_E_INVALID;
  // the same parameter checks as plast_small_gapped
  if (!params_ok(params)) return PLAST_E_INVALID;
  const plast_params prm = resolve(params);
  *n_out = 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (bank_wait(b1, st) != cudaSuccess || bank_wait(b2, st) != cudaSuccess) return PLAST_E_CUDA;

  cudaError_t err;
  unsigned char* base = scratch_on_current_device(&err);
  if (!base) return rc_of(err);
  CKN(upload_tables_once());
  if (n_in == 0) return PLAST_OK;
  if (b1->n_seqs == 0 || b2->n_seqs == 0) return PLAST_E_INVALID;
  if (scan_tmp_bytes(n_in) > SCAN_BYTES) return PLAST_E_INVALID;

  uint64_t* key = (uint64_t*)(base + OFF_KEY);
  uint32_t* val = (uint32_t*)(base + OFF_VAL);
  int64_t* at = (int64_t*)(base + OFF_AT);
  int64_t* total = (int64_t*)(base + OFF_TOTAL);
  int* bad = (int*)(base + OFF_BAD);

  // The array keeps the previous call's contents: the flag that must start
  // at zero is cleared here; every other array is fully written before it
  // is read.
  CKN(cudaMemsetAsync(bad, 0, sizeof(int), st));
  const int sh = b2->pad_bits;
  CKN(launch_hits_to_keys(in, n_in, b1->pad_off, b1->n_seqs, b2->pad_off, b2->n_seqs, sh, key, val, bad, st));
  int h_bad = 0;
  CKN(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKN(cudaStreamSynchronize(st));
  if (h_bad) return PLAST_E_INVALID;

  GapArgs g;
  g.pad1 = b1->pad;
  g.pad2 = b2->pad;
  g.key = key;
  g.val = val;
  g.n = n_in;
  g.sh = sh;
  g.gap_open = prm.gap_open;
  g.gap_extend = prm.gap_extend;
  g.s2 = prm.s2;
  g.score = (int32_t*)(base + OFF_SCORE);
  g.ends = (uint32_t*)(base + OFF_ENDS);
  g.pass = (int32_t*)(base + OFF_PASS);
  CKN(launch_small_gapped(g, st));
  CKN(scan_exclusive(g.pass, at, n_in, total, base + OFF_SCAN, SCAN_BYTES, st));
  int64_t m = 0;
  CKN(cudaMemcpyAsync(&m, total, sizeof(m), cudaMemcpyDeviceToHost, st));
  CKN(cudaStreamSynchronize(st));
  *n_out = m;
  if (m > cap) return PLAST_E_CAPACITY;
  if (m == 0) return PLAST_OK;
  if (!out) return PLAST_E_INVALID;
  CKN(launch_gapped_compact(g, at, seq_map(b1), seq_map(b2), out, st));
  CKN(cudaStreamSynchronize(st));
  return PLAST_OK;
}
