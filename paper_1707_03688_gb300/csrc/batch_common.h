// Host-side declarations of the batched pass kernels (see batch.cuh).
#pragma once

#include "internal.h"

namespace nslct {

struct BatchItem {
  int field;  // index into the batch
  int panel;  // panel of that field's pass
};

// Lines per panel of the batched kernels for line length L with `threads`-thread
// CTAs (128, 256 or 512; 0 if that CTA size does not handle L).
int batch_panel_lines(int L, int threads);

int launch_batch_row(int grid, int threads, const PassDesc* descs, const BatchItem* items, int nitems, int* counter,
                     cudaStream_t s);
int launch_batch_col(int grid, int threads, const PassDesc* descs, const BatchItem* items, int nitems, int* counter,
                     cudaStream_t s);
int prepare_batch_row();
int prepare_batch_col();

}  // namespace nslct
