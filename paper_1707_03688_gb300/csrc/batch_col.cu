// Batched column passes (see batch.cuh).
#include "batch.cuh"

namespace nslct {
int launch_batch_col(int grid, int threads, const PassDesc* descs, const BatchItem* items, int nitems, int* counter,
                     cudaStream_t s) {
  return launch_batch<true>(grid, threads, descs, items, nitems, counter, s);
}
int prepare_batch_col() { return prepare_batch<true>(); }
}  // namespace nslct
