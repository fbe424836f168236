// Host-side declarations of the batched pass kernels (see batch.cuh).
#pragma once

#include "internal.h"

namespace nslct {

// The configuration code of the batched kernel for 3*2^a lines packed in pairs
// (128 threads, three CTAs per SM); 128, 256 and 512 are the plain CTA sizes.
constexpr int kB3K = 1128;

struct BatchItem {
  int field;  // index into the batch
  int panel;  // panel of that field's pass
};

// Lines per panel of the batched kernels for line length L with `threads`-thread
// CTAs (128, 256 or 512) or the kB3K configuration; 0 if it does not handle L.
int batch_panel_lines(int L, int threads);

int launch_batch_row(int grid, int threads, const PassDesc* descs, const BatchItem* items, int nitems, int* counter,
                     cudaStream_t s);
int launch_batch_col(int grid, int threads, const PassDesc* descs, const BatchItem* items, int nitems, int* counter,
                     cudaStream_t s);
int prepare_batch_row();
int prepare_batch_col();

}  // namespace nslct
