// Batched row passes (see batch.cuh).
#include "batch.cuh"

namespace nslct {
int batch_panel_lines(int L) { return batch_lines_of(L); }
int launch_batch_row(int grid, const PassDesc* descs, const BatchItem* items, int nitems, int* counter,
                     cudaStream_t s) {
  return launch_batch<false>(grid, descs, items, nitems, counter, s);
}
int prepare_batch_row() { return prepare_batch<false>(); }
}  // namespace nslct
