// bank.cuh -- the device-resident indexed bank behind the opaque plast_bank
// handle of include/plast.h (library-internal).
#pragma once
#include <vector>

#include "common.cuh"
#include "gapped.cuh"

// Sentinel bytes allocated before and after a bank's padded codes, beyond
// GAP: kernels that read whole aligned words around a hit may touch a few
// bytes outside [0, n_pad).
constexpr int64_t PAD_SLACK = 256;

struct plast_bank {
  int device = 0;
  int32_t n_seqs = 0;
  int64_t n_res = 0, n_pad = 0, n_idx = 0;
  int8_t* pad = nullptr;       // [n_pad] padded codes (PAD_SLACK more sentinel bytes on both sides)
  int8_t* pad_alloc = nullptr; // the allocation: pad - PAD_SLACK
  int64_t* pad_off = nullptr;  // [n_seqs + 1] padded start of each sequence; [n_seqs] = n_pad
  int32_t* blk_seq = nullptr;  // [n_pad / SEQ_BLK + 1] sequence at each block start (SeqMap)
  int64_t* key_off = nullptr;  // [8801]
  uint32_t* pos = nullptr;     // [n_idx] padded word starts in CSR order
  int8_t* nb = nullptr;        // [n_idx][48] neighbourhoods
  int pad_bits = 1;            // bits needed by a padded position
  std::vector<int64_t> h_key_off;
  std::vector<int64_t> h_pad_off;
  cudaEvent_t ready = nullptr;  // recorded after the last kernel that builds the bank
};

inline plast::SeqMap seq_map(const plast_bank* b) { return plast::SeqMap{b->pad_off, b->blk_seq, b->n_seqs}; }

// Orders work queued on st after the bank's construction (which may still be
// running on the stream it was built on).
inline cudaError_t bank_wait(const plast_bank* b, cudaStream_t st) {
  return b && b->ready ? cudaStreamWaitEvent(st, b->ready, 0) : cudaSuccess;
}
