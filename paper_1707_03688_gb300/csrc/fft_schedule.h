// Compile-time FFT schedule shared by the kernels and the host twiddle builder.
#pragma once

namespace nslct {

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// elements per thread
__host__ __device__ constexpr int elems_per_thread(int L) {
  return is_pow2(L) ? (L >= 16 ? 16 : L) : (L >= 24 ? 24 : L);
}
// radix of stage `st`: the largest allowed radix first, then powers of two
__host__ __device__ constexpr int stage_radix(int L, int st) {
  int rem = L;
  int first = is_pow2(L) ? (L >= 16 ? 16 : L) : (L >= 24 ? 24 : L);
  int r = first;
  for (int i = 0; i <= st; ++i) {
    if (i == 0) {
      r = first;
    } else {
      int big = is_pow2(L) ? 16 : 8;
      r = rem >= big ? big : rem;
    }
    if (i < st) rem /= r;
  }
  return r;
}
__host__ __device__ constexpr int num_stages(int L) {
  int rem = L, s = 0;
  while (rem > 1) { rem /= stage_radix(L, s); ++s; }
  return s;
}
__host__ __device__ constexpr int stage_ns(int L, int st) {  // product of the radices before `st`
  int ns = 1;
  for (int i = 0; i < st; ++i) ns *= stage_radix(L, i);
  return ns;
}


// Size (in complex entries) of the per-stage twiddle table of length L: for
// every stage st >= 1 with radix RD and NS = product of the earlier radices,
// NS * RD entries W_{NS*RD}^{jm*r} laid out [jm][r].
__host__ __device__ constexpr int stage_table_offset(int L, int st) {
  int off = 0;
  for (int i = 1; i < st; ++i) off += stage_ns(L, i) * stage_radix(L, i);
  return off;
}
__host__ __device__ constexpr int twiddle_table_size(int L) { return stage_table_offset(L, num_stages(L)); }

}  // namespace nslct
