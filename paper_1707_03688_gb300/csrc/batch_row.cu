// Batched row passes (see batch.cuh).
#include "batch.cuh"

namespace nslct {
int batch_panel_lines(int L, int threads) {
  return threads == kB3K  ? batch_lines_of<kB3K>(L)
         : threads == 128 ? batch_lines_of<128>(L)
         : threads == 256 ? batch_lines_of<256>(L)
         : threads == 512 ? batch_lines_of<512>(L)
                          : 0;
}
int launch_batch_row(int grid, int threads, const PassDesc* descs, const BatchItem* items, int nitems, int* counter,
                     cudaStream_t s) {
  return launch_batch<false>(grid, threads, descs, items, nitems, counter, s);
}
int prepare_batch_row() { return prepare_batch<false>(); }
}  // namespace nslct
