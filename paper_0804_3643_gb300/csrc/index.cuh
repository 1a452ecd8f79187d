// index.cuh -- launchers of the stage-0 and translation kernels (index.cu).
#pragma once
#include "common.cuh"

namespace plast {

cudaError_t launch_check_codes(const int8_t* codes, int64_t n, int lo, int hi, int* bad, cudaStream_t st);
// Codes into the sentinel-filled padded bank, checked against [0, hi].
cudaError_t launch_build_pad(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, int64_t n_res, int hi,
                             int8_t* pad, int* bad, cudaStream_t st);
// Stage-0 index as a counting sort over tiles of index_tile(n_pad) padded
// positions: per-tile key counts hist[k * n_tiles + t]; after their
// exclusive scan `off` (with the total), the CSR offsets and the positions
// (offT: scratch of NKEYS * n_tiles for the offsets tile-major).
int64_t index_tile(int64_t n_pad);
cudaError_t launch_index_hist(const int8_t* pad, int64_t n_pad, int64_t tile, int64_t n_tiles, int32_t* hist,
                              cudaStream_t st);
cudaError_t launch_index_finish(const int8_t* pad, int64_t n_pad, int64_t tile, int64_t n_tiles, const int64_t* off,
                                int64_t* offT, const int64_t* total, int64_t* key_off, uint32_t* pos,
                                cudaStream_t st);
cudaError_t launch_neighbourhoods(const int8_t* pad, const uint32_t* pos, int64_t n, int8_t* nb, cudaStream_t st);
// blk[i] = the sequence at padded position i * SEQ_BLK, i <= n_pad / SEQ_BLK
cudaError_t launch_block_seq(const int64_t* pad_off, int32_t n_seqs, int64_t n_pad, int32_t* blk, cudaStream_t st);
cudaError_t launch_export_pos(const uint32_t* pos, int64_t n, const int64_t* pad_off, int32_t n_seqs, int32_t* out,
                              cudaStream_t st);
cudaError_t launch_translate6(const uint8_t* dna, const int64_t* contig_off, int32_t n_contigs, const int64_t* seq_off,
                              int64_t n_aa, int8_t* aa, cudaStream_t st);

}  // namespace plast
