// filter.cuh -- Section 4.2's filter on the stage-2 survivors (filter.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace plast {

// Survivors (padded pos1 << sh | padded pos2, stage-2 value) whose sum of
// positive substitution scores over the 48-cell window reaches s0 are
// appended to okey/oval, their count added to *ocount; the first n
// survivors, or the first min(n, *n_dev) when n_dev is given.
cudaError_t launch_filter_gate(const uint64_t* key, const uint32_t* val, int64_t n, const int64_t* n_dev, int sh,
                               const int8_t* pad1, const int8_t* pad2, int s0, uint64_t* okey, uint32_t* oval,
                               unsigned long long* ocount, cudaStream_t st);

}  // namespace plast
