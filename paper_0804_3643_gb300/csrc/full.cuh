// full.cuh -- stage 3.2 and the trace-back fields of stage 4 (full.cu).
#pragma once
#include "common.cuh"

namespace plast {

constexpr int FG_W = 1024;                  // computed columns of one row a warp can hold
constexpr int64_t FG_ARENA = 1 << 20;       // row table + H values (int16) of one side, per warp
constexpr int FG_SEGS = 8192;               // gap-free segments kept for one pair of sequences
constexpr int FG_ERR_WIDTH = 1, FG_ERR_ARENA = 2, FG_ERR_SEGS = 4, FG_ERR_PATH = 8;

struct FullArgs {
  const int8_t* pad1;
  const int8_t* pad2;
  const int64_t* pad_off1;  // padded sequence starts of each bank
  const int64_t* pad_off2;
  const plast_gapped* in;   // stage-3.1 records
  const uint32_t* proc;     // record indexes in processing order
  const int64_t* gstart;    // first processing position of each pair of sequences, [ng + 1]
  const int64_t* ng_dev;    // number of pairs of sequences
  int32_t go, ge, xdrop;
  plast_alignment* res;     // per record index
  int32_t* done;            // per record index: 1 extended, 0 on a segment of an earlier alignment
  uint8_t* arena;           // FG_ARENA bytes per warp
  int32_t* segs;            // 3 * FG_SEGS ints per warp
  int* err;                 // FG_ERR_* bits
  unsigned long long* cells;  // computed dynamic-programming cells, summed
  unsigned* next;             // the next pair of sequences to take (zero at launch)
};

// Warps the stage-3.2 kernel runs with on a GPU of n_sms SMs (the arena and
// segment buffers are sized for them).
int64_t full_gapped_warps(int n_sms);
cudaError_t launch_full_gapped(const FullArgs& a, int64_t warps, cudaStream_t st);
cudaError_t launch_full_canon(const plast_gapped* in, int64_t n, const int64_t* po1, int32_t n1, const int64_t* po2,
                              int32_t n2, int sh, uint64_t* key, uint32_t* val, int* bad, cudaStream_t st);
cudaError_t launch_full_proc(const plast_gapped* in, const uint32_t* canon, int64_t n, int b2, uint64_t* key,
                             uint32_t* val, cudaStream_t st);
// phase 0: head flags of the pairs of sequences in processing order; phase 1:
// their start positions from the scanned flags (gstart[*ng] = n)
cudaError_t launch_full_groups(const plast_gapped* in, const uint32_t* proc, int64_t n, int32_t* flag,
                               const int64_t* at, const int64_t* ng, int64_t* gstart, int phase, cudaStream_t st);
cudaError_t launch_full_keep(const uint32_t* canon, int64_t n, const int32_t* done, const plast_alignment* res,
                             int32_t s3, int32_t* keep, cudaStream_t st);
cudaError_t launch_full_write(const uint32_t* canon, int64_t n, const int32_t* keep, const int64_t* at,
                              const plast_alignment* res, plast_alignment* out, cudaStream_t st);

}  // namespace plast
