// Routes a pass to the translation unit that instantiates its length.
#include "internal.h"

namespace nslct {

int launch_f32_g0(bool, const PassDesc&, cudaStream_t);
int prepare_f32_g0(int);
int launch_dual_f32_g0(bool, const PassDesc&, const void*, void*, double*, int, cudaStream_t);
int dual_blocks_f32_g0(int, int);
int launch_f32_g1(bool, const PassDesc&, cudaStream_t);
int prepare_f32_g1(int);
int launch_dual_f32_g1(bool, const PassDesc&, const void*, void*, double*, int, cudaStream_t);
int dual_blocks_f32_g1(int, int);
int launch_f32_g2(bool, const PassDesc&, cudaStream_t);
int prepare_f32_g2(int);
int launch_dual_f32_g2(bool, const PassDesc&, const void*, void*, double*, int, cudaStream_t);
int dual_blocks_f32_g2(int, int);
int launch_f32_g3(bool, const PassDesc&, cudaStream_t);
int prepare_f32_g3(int);
int launch_dual_f32_g3(bool, const PassDesc&, const void*, void*, double*, int, cudaStream_t);
int dual_blocks_f32_g3(int, int);
int launch_f64_g0(bool, const PassDesc&, cudaStream_t);
int prepare_f64_g0(int);
int launch_dual_f64_g0(bool, const PassDesc&, const void*, void*, double*, int, cudaStream_t);
int dual_blocks_f64_g0(int, int);
int launch_f64_g1(bool, const PassDesc&, cudaStream_t);
int prepare_f64_g1(int);
int launch_dual_f64_g1(bool, const PassDesc&, const void*, void*, double*, int, cudaStream_t);
int dual_blocks_f64_g1(int, int);
int launch_f64_g2(bool, const PassDesc&, cudaStream_t);
int prepare_f64_g2(int);
int launch_dual_f64_g2(bool, const PassDesc&, const void*, void*, double*, int, cudaStream_t);
int dual_blocks_f64_g2(int, int);
int launch_f64_g3(bool, const PassDesc&, cudaStream_t);
int prepare_f64_g3(int);
int launch_dual_f64_g3(bool, const PassDesc&, const void*, void*, double*, int, cudaStream_t);
int dual_blocks_f64_g3(int, int);

static int group_of(int L) {
  switch (L) {
    case 4096: case 2048: return 0;
    case 1024: case 512: case 256: return 1;
    case 128: case 64: case 32: case 16: case 8: return 2;
    case 1536: case 768: case 384: case 192: case 96: case 48: case 24: case 12: return 3;
    default: return -1;
  }
}

int launch_pass_f32(bool col, const PassDesc& d, cudaStream_t s) {
  switch (group_of(col ? d.Nx : d.Ny)) {
    case 0: return launch_f32_g0(col, d, s);
    case 1: return launch_f32_g1(col, d, s);
    case 2: return launch_f32_g2(col, d, s);
    case 3: return launch_f32_g3(col, d, s);
    default: return NSLCT_E_SIZE;
  }
}

int prepare_pass_f32(int L) {
  switch (group_of(L)) {
    case 0: return prepare_f32_g0(L);
    case 1: return prepare_f32_g1(L);
    case 2: return prepare_f32_g2(L);
    case 3: return prepare_f32_g3(L);
    default: return NSLCT_E_SIZE;
  }
}

int launch_dual_f32(bool col, const PassDesc& d, const void* in_y, void* out_y, double* partials, int accumulate, cudaStream_t s) {
  switch (group_of(col ? d.Nx : d.Ny)) {
    case 0: return launch_dual_f32_g0(col, d, in_y, out_y, partials, accumulate, s);
    case 1: return launch_dual_f32_g1(col, d, in_y, out_y, partials, accumulate, s);
    case 2: return launch_dual_f32_g2(col, d, in_y, out_y, partials, accumulate, s);
    case 3: return launch_dual_f32_g3(col, d, in_y, out_y, partials, accumulate, s);
    default: return NSLCT_E_SIZE;
  }
}

int dual_blocks_f32(int L, int nlines) {
  switch (group_of(L)) {
    case 0: return dual_blocks_f32_g0(L, nlines);
    case 1: return dual_blocks_f32_g1(L, nlines);
    case 2: return dual_blocks_f32_g2(L, nlines);
    case 3: return dual_blocks_f32_g3(L, nlines);
    default: return -1;
  }
}

int launch_pass_f64(bool col, const PassDesc& d, cudaStream_t s) {
  switch (group_of(col ? d.Nx : d.Ny)) {
    case 0: return launch_f64_g0(col, d, s);
    case 1: return launch_f64_g1(col, d, s);
    case 2: return launch_f64_g2(col, d, s);
    case 3: return launch_f64_g3(col, d, s);
    default: return NSLCT_E_SIZE;
  }
}

int prepare_pass_f64(int L) {
  switch (group_of(L)) {
    case 0: return prepare_f64_g0(L);
    case 1: return prepare_f64_g1(L);
    case 2: return prepare_f64_g2(L);
    case 3: return prepare_f64_g3(L);
    default: return NSLCT_E_SIZE;
  }
}

int launch_dual_f64(bool col, const PassDesc& d, const void* in_y, void* out_y, double* partials, int accumulate, cudaStream_t s) {
  switch (group_of(col ? d.Nx : d.Ny)) {
    case 0: return launch_dual_f64_g0(col, d, in_y, out_y, partials, accumulate, s);
    case 1: return launch_dual_f64_g1(col, d, in_y, out_y, partials, accumulate, s);
    case 2: return launch_dual_f64_g2(col, d, in_y, out_y, partials, accumulate, s);
    case 3: return launch_dual_f64_g3(col, d, in_y, out_y, partials, accumulate, s);
    default: return NSLCT_E_SIZE;
  }
}

int dual_blocks_f64(int L, int nlines) {
  switch (group_of(L)) {
    case 0: return dual_blocks_f64_g0(L, nlines);
    case 1: return dual_blocks_f64_g1(L, nlines);
    case 2: return dual_blocks_f64_g2(L, nlines);
    case 3: return dual_blocks_f64_g3(L, nlines);
    default: return -1;
  }
}

}  // namespace nslct
