// Internal declarations shared by the host plan, the C-ABI and the kernel passes.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "nslct.h"

struct nslct_plan_s;

namespace nslct {

// A quadratic chirp phase in turns, stored as Q0.64 fixed point:
//   turns(a, b) = k11 a^2 + k12 a b + k22 b^2   (mod 1, exact in uint64 arithmetic)
// where (a, b) are the integer indices along x and y of the domain the chirp
// acts in (centred sample indices in space, centred bin indices in frequency).
// Because a^2, a*b, b^2 are integers, only the fractional part of each real
// coefficient matters, so the 64-bit wrap-around IS the reduction modulo 2*pi.
struct Chirp {
  uint64_t k11, k12, k22;
};

enum Transform : int { kNone = 0, kFwd = 1, kInv = 2 };

// A pass of the packed line-pair kernel as a program: transforms T_0 ..
// T_{ntr-1} of alternating direction, an optional step before T_0, one step in
// each gap between transforms and up to two after the last. A step multiplies
// by a chirp (times scale) or by scale alone; kind 0 is no step. Filled by the
// launcher from the generic fields of PassDesc.
struct X2Step {
  int kind;            // 0 none, 1 chirp x scale, 2 scale
  int freq;            // chirp indices: 0 = centred samples, 1 = centred bins
  float scale;
  Chirp c;
};
struct X2Prog {
  int ntr;
  X2Step pre;
  X2Step gap[2];
  X2Step post[2];
};

// One kernel pass: a batch of 1D transforms of length L along one axis, each
// optionally followed by a chirp multiply and a second 1D transform.
//   row pass: lines are rows i (length Ny), elements are columns j
//   col pass: lines are columns j (length Nx), elements are rows i
// Layouts: 0 = row-major [Nx][Ny]; 1 = 2x2-tiled, element (i, j) at
//   (i/2)*2*Ny + (j/2)*4 + (i%2)*2 + (j%2), which keeps a row pair AND a column
//   pair of the field in whole 32-byte sectors.
struct PassDesc {
  const void* in;
  void* out;
  int Nx, Ny;
  int in_tiled, out_tiled;
  int t1, t2;          // Transform before / after the chirp
  int has_chirp;
  int freq_domain;     // chirp indices: 0 = centred samples, 1 = centred bins
  Chirp chirp;
  double scale;        // real factor applied with the chirp (or alone)
  float fscale;        // the same factor in FP32
  int scale_only;      // no chirp but scale != 1
  int num_sms;         // persistent-grid size for the FP32 kernels
  const void* tw;      // per-stage twiddle table of the pass axis length (see fft_schedule.h)
  unsigned int* err;   // device status word: bit 0 = a bounded wait expired
  int mixed;           // radix-16 stages as split-FP16 tensor-core DFTs (FP32 data)
  // optional tail: after t2, a second chirp (x scale2) and a third transform
  int t3;
  int has_chirp2;
  int freq_domain2;
  Chirp chirp2;
  float fscale2;       // applied with chirp2 (or alone when != 1)
  // zero padding (Secs. 2.A, 5.A): a pass with row-major input and pad_in set
  // reads the caller's in_rows x in_cols array as the region starting at
  // (in_r0, in_c0) of the Nx x Ny grid, zeros elsewhere; a pass with row-major
  // output and pad_out set writes only the region at (out_r0, out_c0) to an
  // out_rows x out_cols array
  int pad_in, in_rows, in_cols, in_r0, in_c0;
  int pad_out, out_rows, out_cols, out_r0, out_c0;
  // a row-major output pass multiplies each stored value by the same element
  // of this caller array (the output's shape and type) when non-null
  const void* post_mask;
  // same-plan batches: nbatch fields (<= 1: one), field b at in + b * in_bstride
  // and out + b * out_bstride (elements); the adjoint's value path uses the
  // same strides
  int nbatch;
  long long in_bstride, out_bstride;
  // bounded waits: give up after wait_us microseconds (0: one second); a
  // self-test arms the first panel's barrier for test_extra_tx more bytes than
  // are copied, so that its wait must expire
  unsigned int wait_us;
  unsigned int test_extra_tx;
  // the same pass as a program for the packed line-pair kernel (set by its launcher)
  X2Prog x2;
  // split-precision tensor-core kernel: its constant operands (DFT matrix
  // halves and twiddles, see tc_pass.cu) and whether the program's first
  // transform is an inverse (set by its launcher)
  const void* tc_tab;
  int x2_first_inv;
};

// FP32 lines of 256..4096 points run in the line-pair kernel (which also
// walks a whole same-plan batch in one launch); 0 at build time disables it.
#ifndef NSLCT_PAIR
#define NSLCT_PAIR 1
#endif
inline bool pair_kernel_length(int L) { return NSLCT_PAIR && L >= 256 && L <= 4096 && (L & (L - 1)) == 0; }

// Enqueue one pass. `col` selects the axis. Returns an NSLCT_* code.
int launch_pass_f32(bool col, const PassDesc& d, cudaStream_t s);
int launch_pass_f64(bool col, const PassDesc& d, cudaStream_t s);
// Prepare kernel attributes (dynamic shared memory) for length L on the current device.
int prepare_pass_f32(int L);
int prepare_pass_f64(int L);

// Dual (adjoint) passes: gradient path d.in -> d.out and value path in_y -> out_y
// through the same pass; with `accumulate`, per-CTA sums S_aa, S_ab, S_bb go to
// partials[cta][3]. dual_blocks_* gives the CTA count of such a pass.
int launch_dual_f32(bool col, const PassDesc& d, const void* in_y, void* out_y, double* partials, int accumulate,
                    cudaStream_t s);
int launch_dual_f64(bool col, const PassDesc& d, const void* in_y, void* out_y, double* partials, int accumulate,
                    cudaStream_t s);
int dual_blocks_f32(int L, int nlines);
int dual_blocks_f64(int L, int nlines);

// The five pass descriptors of the forward or inverse chain (see api.cpp).
void build_chain_descs(const nslct_plan_s* p, const void* in, void* out, bool inverse, PassDesc d[5]);
bool chain_pass_is_column(int k);
// The plan's own schedule: 5 passes, or 3 when H acts along y only. Returns
// the pass count; cols[k] tells the axis of pass k.
int build_schedule(const nslct_plan_s* p, const void* in, void* out, bool inverse, PassDesc d[5], bool cols[5]);

// True when L is a length the kernels are instantiated for.
bool supported_length(int L);

// Split-precision passes on the tensor cores (tc_pass.cu): the line lengths
// the kernel runs, the size of its constant table and the table's bytes,
// kernel attributes, and one pass (NSLCT_E_UNSUPPORTED when the pass is not
// one it runs: the caller then uses the FP32 kernels).
bool tc_length(int L);
size_t tc_table_bytes();
void tc_build_table(unsigned char* host);
int prepare_pass_tc();
int launch_pass_tc(bool col, const PassDesc& d, cudaStream_t s);

}  // namespace nslct

struct nslct_plan_s;

// The opaque plan (one ABCD matrix, one field size).
struct nslct_plan_s {
  int Nx, Ny;
  double dx, dy;
  unsigned flags;
  int prec;            // 0 = fp32, 1 = fp64
  int mixed;           // NSLCT_PREC_SPLIT_F16: FP32 data, split-FP16 tensor-core DFT-16 stages
  int y_only_h;        // H = (0,0;0,h): CC^H acts along y only and the chain runs in 3 passes
  int type2;           // CC-CM-CC-CM chain: the factors below are the type-1 ones of M^-1
  int device;
  double M[16];        // the (possibly projected) ABCD matrix
  double H[4], Bp[4], C1[4], C2[4];
  // Forward chain chirps (application order): chi_H (frequency, -H),
  // cm_C2 (space), chi_Bp (frequency, -B'), cm_C1 (space).
  nslct::Chirp fwd_chi_h, fwd_cm_c2, fwd_chi_bp, fwd_cm_c1;
  // Inverse chain chirps: cm_-C1, chi_+B', cm_-C2, chi_+H.
  nslct::Chirp inv_cm_c1, inv_chi_bp, inv_cm_c2, inv_chi_h;
  int num_sms;         // multiprocessors of `device`
  int has_theta;       // A invertible: theta and its chirp Jacobian are defined
  double theta[10];    // (c11,c12,c22, l11,l12,l21,l22, b11,b12,b22), see grad_math.cpp
  int has_h0;          // made by nslct_plan_theta with an H anchor: nslct_plan_theta_set applies
  double h0[4];        // that anchor of the H(theta) rule
  double jac[120];     // d(H, B', C1, C2 entries)/d theta, 12 x 10
  void* ws;            // backward value-path field(s) (made on first use, grown for batches)
  long long ws_elems;  // elements `ws` holds
  double* partials;    // backward per-CTA sums (made on first use)
  int partials_stride; // rows per pass in `partials`
  unsigned int* err;   // device status word shared by the plan's kernels
  void* tw_x;          // device twiddles for length Nx, forward/inverse kernels
  void* tw_y;          // device twiddles for length Ny (tables may alias each other)
  void* tw16_x;        // twiddles for elems_per_thread(Nx): adjoint and batched kernels
  void* tw16_y;
  void* tc_tab;        // split-precision plans with a 4096-point axis: tensor-core kernel constants
  // zero padding: the caller's input field is the in_rows x in_cols region at
  // (in_r0, in_c0) of the Nx x Ny grid the chain runs on; the output is the
  // out_* region (the whole grid unless cropped). pad_ws holds the tiled grid
  // between passes when the caller's output is smaller than the grid.
  int padded;
  int in_rows, in_cols, in_r0, in_c0;
  int out_rows, out_cols, out_r0, out_c0;
  void* pad_ws;
};
