// Instantiations of the fused FFT pass kernels for one element type and one
// group of lengths. The build compiles this file once per (type, group) so the
// translation units compile in parallel; the groups together cover every
// supported length 2^a (8..4096) and 3*2^a (12..1536).
#include "fft_pass.cuh"

#if !defined(NSLCT_REAL) || !defined(NSLCT_GROUP) || !defined(NSLCT_SUFFIX)
#error "compile with -DNSLCT_REAL=float|double -DNSLCT_GROUP=0..3 -DNSLCT_SUFFIX=f32_g0|..."
#endif
#define NSLCT_CAT2(a, b) a##b
#define NSLCT_CAT(a, b) NSLCT_CAT2(a, b)

#if NSLCT_GROUP == 0
#define NSLCT_LENGTHS(X) X(4096) X(2048)
#elif NSLCT_GROUP == 1
#define NSLCT_LENGTHS(X) X(1024) X(512) X(256)
#elif NSLCT_GROUP == 2
#define NSLCT_LENGTHS(X) X(128) X(64) X(32) X(16) X(8)
#elif NSLCT_GROUP == 3
#define NSLCT_LENGTHS(X) X(1536) X(768) X(384) X(192) X(96) X(48) X(24) X(12)
#else
#error "unknown NSLCT_GROUP"
#endif

namespace nslct {

int NSLCT_CAT(launch_, NSLCT_SUFFIX)(bool col, const PassDesc& d, cudaStream_t s) {
  const int L = col ? d.Nx : d.Ny;
  switch (L) {
#define NSLCT_CASE(LL) \
  case LL: return col ? launch_one<NSLCT_REAL, LL, true>(d, s) : launch_one<NSLCT_REAL, LL, false>(d, s);
    NSLCT_LENGTHS(NSLCT_CASE)
#undef NSLCT_CASE
    default: return NSLCT_E_SIZE;
  }
}

int NSLCT_CAT(prepare_, NSLCT_SUFFIX)(int L) {
  switch (L) {
#define NSLCT_CASE(LL) \
  case LL: {                                        \
    const int rc = prepare_one<NSLCT_REAL, LL>();    \
    return rc != NSLCT_OK ? rc : prepare_dual_one<NSLCT_REAL, LL>(); \
  }
    NSLCT_LENGTHS(NSLCT_CASE)
#undef NSLCT_CASE
    default: return NSLCT_E_SIZE;
  }
}

int NSLCT_CAT(launch_dual_, NSLCT_SUFFIX)(bool col, const PassDesc& d, const void* in_y, void* out_y,
                                         double* partials, int accumulate, cudaStream_t s) {
  const int L = col ? d.Nx : d.Ny;
  switch (L) {
#define NSLCT_CASE(LL)                                                                               \
  case LL:                                                                                           \
    return col ? launch_dual_one<NSLCT_REAL, LL, true>(d, in_y, out_y, partials, accumulate, s)      \
               : launch_dual_one<NSLCT_REAL, LL, false>(d, in_y, out_y, partials, accumulate, s);
    NSLCT_LENGTHS(NSLCT_CASE)
#undef NSLCT_CASE
    default: return NSLCT_E_SIZE;
  }
}

int NSLCT_CAT(dual_blocks_, NSLCT_SUFFIX)(int L, int nlines) {
  switch (L) {
#define NSLCT_CASE(LL) \
  case LL: return dual_blocks<NSLCT_REAL, LL>(nlines);
    NSLCT_LENGTHS(NSLCT_CASE)
#undef NSLCT_CASE
    default: return -1;
  }
}

}  // namespace nslct
