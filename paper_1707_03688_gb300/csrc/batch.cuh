// Batched passes: one persistent launch per pass covers every field of a batch
// of fields with uneven sizes (each with its own ABCD plan).
//
// Work items are (field, panel) pairs, ordered largest line first, and handed
// out dynamically through an atomic counter, so a CTA that finishes a small
// panel takes the next one. Each item's panel is copied global -> shared with
// 16-byte cp.async while the CTA still computes the previous item, exactly as
// in the single-field kernels; the line length (a template parameter there) is
// dispatched per item here. Five such launches (plus one counter reset) make
// one batched transform; they can be captured into one CUDA graph.
#pragma once

#include "batch_common.h"
#include "fft_pass.cuh"

namespace nslct {

// lengths the batched kernels handle (line length along the pass axis)
#define NSLCT_BATCH_LENGTHS(X) \
  X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(96) X(192) X(384) X(768) X(1536)

template <int L> struct BShape {
  static constexpr int E = elems_per_thread(L);  // the plans' tw16 tables
  static constexpr int T_LINE = L / E;
  static constexpr int THREADS = 512;
  static constexpr int P = THREADS / T_LINE;   // lines per panel
  static_assert(P >= 2 && P % 2 == 0, "panel width");
  static constexpr int XSM = P * (L + L / 16);
  static constexpr int STG_ROW = P * (L + 8);  // row-major rows are padded in staging
  static constexpr int STG_TILED = P * L;
};

constexpr int kBatchThreads = 512;

// exchange-buffer and staging-buffer entries for the largest need among the lengths
__host__ __device__ constexpr int batch_xsm() {
  int m = 0;
#define NSLCT_BSM(LL) m = BShape<LL>::XSM > m ? BShape<LL>::XSM : m;
  NSLCT_BATCH_LENGTHS(NSLCT_BSM)
#undef NSLCT_BSM
  return m;
}
__host__ __device__ constexpr int batch_stg() {
  int m = 0;
#define NSLCT_BSM(LL) m = BShape<LL>::STG_ROW > m ? BShape<LL>::STG_ROW : m;
  NSLCT_BATCH_LENGTHS(NSLCT_BSM)
#undef NSLCT_BSM
  return m;
}
constexpr int kBatchXsm = batch_xsm();
constexpr size_t kBatchSmem = (size_t)(batch_xsm() + batch_stg()) * sizeof(float2);
static_assert(kBatchSmem <= 227 * 1024, "batched kernel shared memory");

__host__ __device__ constexpr int batch_lines_of(int L) {
#define NSLCT_BP(LL) \
  if (L == LL) return BShape<LL>::P;
  NSLCT_BATCH_LENGTHS(NSLCT_BP)
#undef NSLCT_BP
  return 0;
}

template <int L, bool COL>
__device__ __forceinline__ int bstg_index(int p, int e, int tiled) {
  constexpr int P = BShape<L>::P;
  if (COL) return (e >> 1) * (2 * P) + (p >> 1) * 4 + (e & 1) * 2 + (p & 1);
  if (tiled) return (p >> 1) * (2 * L) + (e >> 1) * 4 + (p & 1) * 2 + (e & 1);
  return p * (L + 8) + e;
}

// Issue the 16-byte copies of one panel (every thread takes part).
template <int L, bool COL>
__device__ __forceinline__ void bstage_panel(float2* stg, const PassDesc& d, int panel) {
  constexpr int P = BShape<L>::P;
  constexpr int CHUNKS = P * L / 2;
  const float2* __restrict__ in = reinterpret_cast<const float2*>(d.in);
  const int first = panel * P;
  if (COL) {
    const int tiles_valid = min(P, d.Ny - first) / 2;
    for (int c = threadIdx.x; c < CHUNKS; c += kBatchThreads) {
      const int a = c / P, k = c % P;
      if ((k >> 1) < tiles_valid)
        cp_async16(stg + a * (2 * P) + k * 2, in + (size_t)a * (2 * d.Ny) + (first >> 1) * 4 + k * 2);
    }
  } else if (d.in_tiled) {
    const int rows_valid = min(P, d.Nx - first);
    for (int c = threadIdx.x; c < CHUNKS; c += kBatchThreads) {
      const int q = c / L, k = c % L;
      if (2 * q < rows_valid) cp_async16(stg + q * (2 * L) + k * 2, in + (size_t)((first >> 1) + q) * (2 * L) + k * 2);
    }
  } else {
    constexpr int CPR = L / 2;
    const int rows_valid = min(P, d.Nx - first);
    for (int c = threadIdx.x; c < CHUNKS; c += kBatchThreads) {
      const int q = c / CPR, k = c % CPR;
      if (q < rows_valid) cp_async16(stg + q * (L + 8) + k * 2, in + (size_t)(first + q) * L + k * 2);
    }
  }
}

template <bool COL>
__device__ __forceinline__ void bstage_any(float2* stg, const PassDesc& d, int panel) {
  const int L = COL ? d.Nx : d.Ny;
  switch (L) {
#define NSLCT_BCASE(LL) \
  case LL: bstage_panel<LL, COL>(stg, d, panel); break;
    NSLCT_BATCH_LENGTHS(NSLCT_BCASE)
#undef NSLCT_BCASE
    default: break;
  }
  cp_async_commit();
}

// Compute one item whose panel sits in `stg`; prefetch `next` (if any) into
// `stg` once the panel is in registers.
template <int L, bool COL>
__device__ __forceinline__ void bprocess(const PassDesc& d, int panel, float2* stg, float2* xs,
                                         const PassDesc* __restrict__ descs, const BatchItem* __restrict__ items,
                                         int next, int nitems) {
  using Sh = BShape<L>;
  constexpr int E = Sh::E;
  constexpr int T_LINE = Sh::T_LINE;
  constexpr int P = Sh::P;
  const int tid = threadIdx.x;
  const int p = tid % P;
  const int t = tid / P;
  const int nlines = COL ? d.Ny : d.Nx;
  const int line = panel * P + p;
  const bool valid = line < nlines;
  float2 v[E];
#pragma unroll
  for (int s = 0; s < E; ++s) v[s] = stg[bstg_index<L, COL>(p, t + T_LINE * s, d.in_tiled)];
  __syncthreads();  // staging consumed
  if (next < nitems) {
    const BatchItem it = items[next];
    bstage_any<COL>(stg, descs[it.field], it.panel);
  }
  const float2* __restrict__ tw = reinterpret_cast<const float2*>(d.tw);
  if (d.t1 != kNone) LineFft<float, L, P, E>::run(v, xs, t, p, tw, d.t1 == kInv);
  if (d.has_chirp) {
    apply_chirp<float, L, COL, E>(v, d, t, line, d.fscale);
  } else if (d.scale_only) {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = make_float2(v[s].x * d.fscale, v[s].y * d.fscale);
  }
  if (d.t2 != kNone) LineFft<float, L, P, E>::run(v, xs, t, p, tw, d.t2 == kInv);
  float2* out = reinterpret_cast<float2*>(d.out);
  if (valid) {
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int e = t + T_LINE * s;
      const int i = COL ? e : line;
      const int j = COL ? line : e;
      out[elem_index(i, j, d.Ny, d.out_tiled)] = v[s];
    }
  }
}

// One pass of the batch. descs[f] is field f's descriptor for this pass;
// items[0..nitems) the work list; *counter must be 0 at launch.
template <bool COL>
__global__ void __launch_bounds__(kBatchThreads, 1)
batch_pass_kernel(const PassDesc* __restrict__ descs, const BatchItem* __restrict__ items, int nitems, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item[2];
  float2* xs = reinterpret_cast<float2*>(smem_raw);
  // the exchange buffer (sized for the largest need) comes first, staging after it
  float2* stg = xs + kBatchXsm;
  if (threadIdx.x == 0) s_item[0] = atomicAdd(counter, 1);
  __syncthreads();
  int cur = s_item[0];
  if (cur < nitems) {
    const BatchItem it = items[cur];
    bstage_any<COL>(stg, descs[it.field], it.panel);
  }
  while (cur < nitems) {
    if (threadIdx.x == 0) s_item[1] = atomicAdd(counter, 1);
    cp_async_wait_all();
    __syncthreads();
    const int next = s_item[1];
    const BatchItem it = items[cur];
    const PassDesc& d = descs[it.field];
    const int L = COL ? d.Nx : d.Ny;
    switch (L) {
#define NSLCT_BCASE(LL) \
  case LL: bprocess<LL, COL>(d, it.panel, stg, xs, descs, items, next, nitems); break;
      NSLCT_BATCH_LENGTHS(NSLCT_BCASE)
#undef NSLCT_BCASE
      default: break;
    }
    __syncthreads();  // everyone is done with s_item[1] and the exchange buffer
    cur = next;
  }
  cp_async_wait_all();
}

template <bool COL>
inline int launch_batch(int grid, const PassDesc* descs, const BatchItem* items, int nitems, int* counter,
                        cudaStream_t s) {
  batch_pass_kernel<COL><<<grid, kBatchThreads, kBatchSmem, s>>>(descs, items, nitems, counter);
  return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
}

template <bool COL>
inline int prepare_batch() {
  return cudaFuncSetAttribute(batch_pass_kernel<COL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kBatchSmem) == cudaSuccess
             ? NSLCT_OK
             : NSLCT_E_CUDA;
}

}  // namespace nslct
