// nslct_backward: adjoint of the chain plus chirp/ABCD parameter gradients.
//
// For a real loss l(y), y = L x, and gbar = dl/dRe y + j dl/dIm y:
//   * grad_in = L^H gbar = L^{-1} gbar: L is unitary (Sec. 6.B), so the exact
//     inverse chain of Eq. CCCMCCCM04 is the adjoint;
//   * each chirp stage v_out = e^{j phi(c)} v_in of Eq. HA28 contributes
//     dl/dc = -sum (d phi/dc) Im(conj(gbar_s) v_out), with gbar_s the gradient
//     pulled back to that stage and v_out the forward value there.
// Both are obtained in one sweep of the five inverse passes over the pair
// (gbar, y): the same inverse operators that carry gbar back to each stage also
// carry y back to that stage's forward value, so nothing from the forward
// call is stored. The sweep's intermediate values differ from (gbar_s, v_out)
// by known constants (the -1/(Nx Ny) of each chirp convolution and the
// unnormalised FFTs); those are folded into the per-stage factors below.
#include <cmath>
#include <cstring>
#include <new>

#include "grad_math.h"
#include "internal.h"

namespace nslct {

// Reduce the per-CTA sums in a fixed order (deterministic) and form the
// 12 chirp gradients and, optionally, the 10 theta gradients. Each thread
// sums whole rows (S_aa, S_ab, S_bb) of every slot, rows t, t + T, ... in
// four independent chains (loads in flight) added in a fixed order; then the
// warps and the block reduce in a fixed tree.
constexpr int kFinalizeThreads = 1024;
__global__ void __launch_bounds__(kFinalizeThreads) grad_finalize_kernel(const double* __restrict__ partials,
                                                                         GradFinal f, double* grad_chirp,
                                                                         double* grad_theta) {
  __shared__ double red[kFinalizeThreads / 32][12];
  __shared__ double sums[12];
  double acc[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) acc[q] = 0.0;
#pragma unroll
  for (int slot = 0; slot < 4; ++slot) {
    const double* __restrict__ rows = partials + (size_t)slot * f.stride * 3;
    double c[4][3] = {};
    int b = threadIdx.x;
    for (; b + 3 * kFinalizeThreads < f.nblk[slot]; b += 4 * kFinalizeThreads)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < 3; ++k) c[u][k] += rows[(size_t)(b + u * kFinalizeThreads) * 3 + k];
    for (; b < f.nblk[slot]; b += kFinalizeThreads)
#pragma unroll
      for (int k = 0; k < 3; ++k) c[0][k] += rows[(size_t)b * 3 + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[slot * 3 + k] = (c[0][k] + c[1][k]) + (c[2][k] + c[3][k]);
  }
#pragma unroll
  for (int q = 0; q < 12; ++q)
    for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 12; ++q) red[warp][q] = acc[q];
  __syncthreads();
  if (threadIdx.x < 12) {
    double tot = 0.0;
    for (int w = 0; w < kFinalizeThreads / 32; ++w) tot += red[w][threadIdx.x];
    sums[threadIdx.x] = tot * f.factor[threadIdx.x / 3][threadIdx.x % 3];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // slots: 0 = C1, 1 = B', 2 = C2, 3 = H; output order H, B', C1, C2
    double g[12];
    const int order[4] = {3, 1, 0, 2};
    for (int o = 0; o < 4; ++o)
      for (int k = 0; k < 3; ++k) g[o * 3 + k] = sums[order[o] * 3 + k];
    if (grad_chirp)
      for (int r = 0; r < 12; ++r) grad_chirp[r] = g[r];
    if (grad_theta && f.want_theta)
      for (int c = 0; c < 10; ++c) {
        double acc = 0.0;
        for (int r = 0; r < 12; ++r) acc += f.jac[r * 10 + c] * g[r];
        grad_theta[c] = acc;
      }
  }
}

}  // namespace nslct

using namespace nslct;

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

int dual_launch(const nslct_plan_s* p, bool col, const PassDesc& d, const void* in_y, void* out_y, double* partials,
                int acc, cudaStream_t s) {
  return p->prec == 1 ? launch_dual_f64(col, d, in_y, out_y, partials, acc, s)
                      : launch_dual_f32(col, d, in_y, out_y, partials, acc, s);
}

int dual_rows(const nslct_plan_s* p, int L, int nlines) {
  return p->prec == 1 ? dual_blocks_f64(L, nlines) : dual_blocks_f32(L, nlines);
}

}  // namespace

// Shared by nslct_backward and its variants: the five dual passes (writing
// per-CTA sums to `partials`, `stride` rows per pass) and the finalisation.
// only_pass in 0..4: that dual pass alone, without the finalisation.
int nslct_backward_impl(nslct_plan_t p, const void* grad_out, const void* y, void* grad_in, double* grad_theta,
                        double* grad_chirp, void* ws, double* partials, int stride, cudaStream_t s, int nbatch,
                        long long fstride, int only_pass) {
  const double nn = (double)p->Nx * (double)p->Ny;
  const double ccs = -1.0 / nn;
  PassDesc base{};
  base.Nx = p->Nx;
  base.Ny = p->Ny;
  base.scale = 1.0;
  base.fscale2 = 1.0f;
  PassDesc d[5];
  for (auto& x : d) x = base;
  // the inverse chain (Eq. CCCMCCCM04), as in nslct_inverse
  d[0].in = grad_out; d[0].out = grad_in; d[0].in_tiled = 0; d[0].out_tiled = 1; d[0].tw = p->tw16_y;
  for (int k = 1; k < 5; ++k) { d[k].in = grad_in; d[k].out = grad_in; d[k].in_tiled = 1; d[k].out_tiled = 1; }
  d[4].out_tiled = 0;
  d[1].tw = p->tw16_x; d[2].tw = p->tw16_y; d[3].tw = p->tw16_x; d[4].tw = p->tw16_y;
  d[1].freq_domain = d[3].freq_domain = 1;
  d[0].has_chirp = 1; d[0].chirp = p->inv_cm_c1; d[0].t2 = kFwd;
  d[1].has_chirp = 1; d[1].chirp = p->inv_chi_bp; d[1].t1 = kFwd; d[1].t2 = kInv;
  d[2].has_chirp = 1; d[2].chirp = p->inv_cm_c2; d[2].t1 = kInv; d[2].t2 = kFwd; d[2].scale = ccs;
  d[3].has_chirp = 1; d[3].chirp = p->inv_chi_h; d[3].t1 = kFwd; d[3].t2 = kInv;
  d[4].t1 = kInv; d[4].scale = ccs;
  for (auto& x : d) {
    x.fscale = (float)x.scale;
    x.scale_only = (!x.has_chirp && x.scale != 1.0) ? 1 : 0;
    x.num_sms = p->num_sms;
    x.err = p->err;
    // a same-plan batch: every array is nbatch fields fstride elements apart,
    // and the CTA sums of all fields add into the (shared) parameter gradients
    x.nbatch = nbatch;
    x.in_bstride = x.out_bstride = fstride;
  }
  const bool cols[5] = {false, true, false, true, false};
  const bool want = grad_theta || grad_chirp;
  GradFinal f{};
  for (int k = 0; k < 5; ++k) {
    if (only_pass >= 0 && k != only_pass) continue;
    const int acc = (want && k < 4) ? 1 : 0;
    if (acc) {
      const int L = cols[k] ? p->Nx : p->Ny;
      f.nblk[k] = (nbatch > 1 ? nbatch : 1) * dual_rows(p, L, cols[k] ? p->Ny : p->Nx);
      if (f.nblk[k] < 0 || f.nblk[k] > stride) return NSLCT_E_SIZE;
    }
    const void* in_y = k == 0 ? y : ws;
    const int rc = dual_launch(p, cols[k], d[k], in_y, ws, acc ? partials + (size_t)k * stride * 3 : nullptr, acc, s);
    if (rc != NSLCT_OK) return rc;
  }
  if (!want || only_pass >= 0) return NSLCT_OK;
  // d loss / d chirp entry = -factor_s * sign_s * w_k * S_k, with w = (d1^2/2, d1 d2, d2^2/2)
  const double dwx = kTwoPi / (p->Nx * p->dx), dwy = kTwoPi / (p->Ny * p->dy);
  const double fs[4] = {1.0, 1.0 / nn, 1.0 / (nn * nn), 1.0 / nn};   // C1, B', C2, H
  const double sg[4] = {+1.0, -1.0, +1.0, -1.0};                      // CM^{C} vs CM^{-B} in frequency
  const double d1[4] = {p->dx, dwx, p->dx, dwx};
  const double d2[4] = {p->dy, dwy, p->dy, dwy};
  for (int sl = 0; sl < 4; ++sl) {
    f.factor[sl][0] = -fs[sl] * sg[sl] * 0.5 * d1[sl] * d1[sl];
    f.factor[sl][1] = -fs[sl] * sg[sl] * d1[sl] * d2[sl];
    f.factor[sl][2] = -fs[sl] * sg[sl] * 0.5 * d2[sl] * d2[sl];
  }
  f.stride = stride;
  f.want_theta = (grad_theta && p->has_theta) ? 1 : 0;
  std::memcpy(f.jac, p->jac, sizeof(f.jac));
  grad_finalize_kernel<<<1, kFinalizeThreads, 0, s>>>(partials, f, grad_chirp, grad_theta);
  return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
}

// nslct_backward over a same-plan batch of nbatch fields fstride elements apart
// (one field: nbatch = 1). The value-path workspace and the CTA partial sums
// are the plan's unless the caller passes a workspace; both grow on demand.
static int backward_batch(nslct_plan_t p, int nbatch, long long fstride, const void* grad_out, const void* y,
                          void* grad_in, double* grad_theta, double* grad_chirp, void* workspace,
                          nslct_stream_t stream, int only_pass = -1) {
  if (!p || !grad_out || !y || !grad_in || nbatch < 1 || only_pass > 4) return NSLCT_E_ARG;
  if (p->padded || p->type2) return NSLCT_E_UNSUPPORTED;
  if (grad_theta && !p->has_theta) return NSLCT_E_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(grad_out) | reinterpret_cast<uintptr_t>(y) |
       reinterpret_cast<uintptr_t>(grad_in) | reinterpret_cast<uintptr_t>(workspace)) & 15u)
    return NSLCT_E_ARG;
  const size_t esz = p->prec == 1 ? 16 : 8;
  const long long n = (long long)p->Nx * p->Ny;
  if (nbatch > 1 && (fstride < n || ((size_t)fstride * esz) % 16)) return NSLCT_E_ARG;
  const long long span = nbatch > 1 ? (long long)(nbatch - 1) * fstride + n : n;  // elements a batch array covers
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return NSLCT_E_CUDA;
  if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return NSLCT_E_CUDA;
  int rc = NSLCT_OK;
  if (!workspace && p->ws_elems < span) {
    if (p->ws) cudaFree(p->ws);
    p->ws = nullptr;
    p->ws_elems = 0;
    if (cudaMalloc(&p->ws, esz * (size_t)span) != cudaSuccess) { p->ws = nullptr; rc = NSLCT_E_NOMEM; }
    else p->ws_elems = span;
  }
  const int rows = nbatch * ((p->Nx > p->Ny ? p->Nx : p->Ny) / 2 + 1);
  if (rc == NSLCT_OK && (!p->partials || p->partials_stride < rows)) {
    if (p->partials) cudaFree(p->partials);
    p->partials = nullptr;
    p->partials_stride = rows;
    if (cudaMalloc(&p->partials, sizeof(double) * 3 * 4 * (size_t)rows) != cudaSuccess) {
      p->partials = nullptr;
      p->partials_stride = 0;
      rc = NSLCT_E_NOMEM;
    }
  }
  if (rc == NSLCT_OK)
    rc = nslct_backward_impl(p, grad_out, y, grad_in, grad_theta, grad_chirp, workspace ? workspace : p->ws,
                             p->partials, p->partials_stride, reinterpret_cast<cudaStream_t>(stream), nbatch, fstride,
                             only_pass);
  if (prev != p->device) cudaSetDevice(prev);
  return rc;
}

extern "C" int nslct_backward(nslct_plan_t p, const void* grad_out, const void* y, void* grad_in, double* grad_theta,
                              double* grad_chirp, void* workspace, nslct_stream_t stream) {
  return backward_batch(p, 1, 0, grad_out, y, grad_in, grad_theta, grad_chirp, workspace, stream);
}

extern "C" int nslct_backward_many(nslct_plan_t p, int nbatch, long long stride, const void* grad_out, const void* y,
                                   void* grad_in, double* grad_theta, double* grad_chirp, void* workspace,
                                   nslct_stream_t stream) {
  return backward_batch(p, nbatch, stride, grad_out, y, grad_in, grad_theta, grad_chirp, workspace, stream);
}

extern "C" int nslct_backward_pass(nslct_plan_t p, int pass, int nbatch, long long stride, const void* grad_out,
                                   const void* y, void* grad_in, void* workspace, nslct_stream_t stream) {
  if (pass < 0 || pass > 4) return NSLCT_E_ARG;
  return backward_batch(p, nbatch, stride, grad_out, y, grad_in, nullptr, nullptr, workspace, stream, pass);
}
