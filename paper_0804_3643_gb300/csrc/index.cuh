// index.cuh -- launchers of the stage-0 and translation kernels (index.cu).
#pragma once
#include "common.cuh"

namespace plast {

cudaError_t launch_check_codes(const int8_t* codes, int64_t n, int lo, int hi, int* bad, cudaStream_t st);
cudaError_t launch_build_pad(const int8_t* codes, const int64_t* seq_off, int32_t n_seqs, int64_t n_res, int8_t* pad,
                             int64_t n_pad, cudaStream_t st);
cudaError_t launch_word_keys(const int8_t* pad, int64_t n_pad, int32_t* key, int32_t* flag, cudaStream_t st);
cudaError_t launch_compact_words(const int32_t* key, const int64_t* at, int64_t n_pad, uint64_t* okey, uint32_t* opos,
                                 cudaStream_t st);
cudaError_t launch_key_offsets(const uint64_t* skey, int64_t n, int64_t* key_off, cudaStream_t st);
cudaError_t launch_neighbourhoods(const int8_t* pad, const uint32_t* pos, int64_t n, int8_t* nb, cudaStream_t st);
cudaError_t launch_export_pos(const uint32_t* pos, int64_t n, const int64_t* pad_off, int32_t n_seqs, int32_t* out,
                              cudaStream_t st);
cudaError_t launch_translate6(const uint8_t* dna, const int64_t* contig_off, int32_t n_contigs, const int64_t* seq_off,
                              int64_t n_aa, int8_t* aa, cudaStream_t st);

}  // namespace plast
