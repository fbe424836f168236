// Compile-time FFT schedule shared by the kernels and the host twiddle builder.
#pragma once

namespace nslct {

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Elements per thread of the FP32 forward/inverse kernels for the largest
// power-of-two lines (2048, 4096): 16 (radix-16 stages, 512-thread CTAs).
// Measured at 4096^2 (Gsamples/s): 16 -> 26.4, 8 (radix-8, 1024 threads, one
// more exchange) -> 23.4, 64 (radix-64, 128 threads, one exchange fewer, 255
// registers) -> 20.6. Overridable at build time.
#ifndef NSLCT_E_LARGE
#define NSLCT_E_LARGE 16
#endif

// default elements per thread: 16 for 2^a lines, 24 for 3*2^a lines (capped by L)
__host__ __device__ constexpr int elems_per_thread(int L) {
  return is_pow2(L) ? (L >= 16 ? 16 : L) : (L >= 24 ? 24 : L);
}
// elements per thread of the forward/inverse kernel that runs length L (FP32 or FP64);
// the adjoint, batched and split-precision kernels use elems_per_thread(L)
__host__ __device__ constexpr int kernel_elems(int L, bool f32) {
  return (f32 && is_pow2(L) && L >= 2048) ? NSLCT_E_LARGE : elems_per_thread(L);
}
// shared-memory padding: one slot per 2^pad_shift elements keeps the
// stride-E stage writes conflict-free
__host__ __device__ constexpr int pad_shift(int E) { return E >= 64 ? 6 : 4; }
// largest power of two <= n that divides e
__host__ __device__ constexpr int pow2_radix(int n, int e) {
  int r = 1;
  while (r * 2 <= n && e % (r * 2) == 0) r *= 2;
  return r;
}
// radix of stage `st` when each thread holds E elements: E first, then the
// largest power of two dividing E that fits the rest
__host__ __device__ constexpr int stage_radix(int L, int E, int st) {
  int rem = L;
  int r = E;
  for (int i = 0; i <= st; ++i) {
    r = (i == 0) ? E : pow2_radix(rem, E);
    if (i < st) rem /= r;
  }
  return r;
}
__host__ __device__ constexpr int num_stages(int L, int E) {
  int rem = L, s = 0;
  while (rem > 1) { rem /= stage_radix(L, E, s); ++s; }
  return s;
}
__host__ __device__ constexpr int stage_ns(int L, int E, int st) {  // product of the radices before `st`
  int ns = 1;
  for (int i = 0; i < st; ++i) ns *= stage_radix(L, E, i);
  return ns;
}

// Size (in complex entries) of the per-stage twiddle table of length L: for
// every stage st >= 1 with radix RD and NS = product of the earlier radices,
// NS * RD entries W_{NS*RD}^{jm*r} laid out [jm][r].
__host__ __device__ constexpr int stage_table_offset(int L, int E, int st) {
  int off = 0;
  for (int i = 1; i < st; ++i) off += stage_ns(L, E, i) * stage_radix(L, E, i);
  return off;
}
// After the [jm][r] tables, a compact table per stage st >= 1 of the NS
// base twiddles W_{NS*RD}^{jm} alone (the line-pair kernel forms the powers
// r = 2 .. RD-1 in registers from these).
__host__ __device__ constexpr int compact_table_offset(int L, int E, int st) {
  int off = stage_table_offset(L, E, num_stages(L, E));
  for (int i = 1; i < st; ++i) off += stage_ns(L, E, i);
  return off;
}
__host__ __device__ constexpr int twiddle_table_size(int L, int E) {
  return compact_table_offset(L, E, num_stages(L, E));
}

}  // namespace nslct
