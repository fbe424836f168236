// Packed FP32x2 arithmetic for the line-pair kernel.
//
// The line-pair kernel runs the same 1D transform on two lines at once, so
// every butterfly, twiddle product and chirp product is done twice with the
// same operation sequence. Here the two lines share one 64-bit register pair
// per quantity: re = (line0.re, line1.re), im = (line0.im, line1.im). One
// add/sub/mul/fma.f32x2 then does both lines' work. Its lane throughput is
// that of scalar FP32 (a packed instruction holds the FMA pipe for two
// cycles); what halves is the number of issued instructions.
//
// Inverse transforms use J(z) = i conj(z), the swap of the real and imaginary
// parts: IDFT = J DFT J, and a chirp product commutes with J up to
// conjugation, J(x) conj(c) = J(x c). The kernel therefore only contains the
// forward DFT. Data held "in the J domain" (parts swapped) is transformed
// inversely by that same code. Within one pass the transforms alternate in
// direction (FFT, chirp, IFFT, ...), so every chirp between two transforms
// also switches domain, which costs nothing: its two results are simply
// written to the other registers. Only the domain at the pass's load and
// store depends on the first and last direction; these are template
// parameters of the kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "fft_schedule.h"

namespace nslct {

typedef unsigned long long f32x2;  // (lane 0, lane 1) = (low, high) FP32 halves

__device__ __forceinline__ f32x2 x2_pack(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void x2_unpack(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 x2_bcast(float v) { return x2_pack(v, v); }
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// a * b + c with one rounding per lane
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// complex values of the two lines at one position
struct cx2 {
  f32x2 re, im;
};
__device__ __forceinline__ cx2 c2_add(cx2 a, cx2 b) { return {x2_add(a.re, b.re), x2_add(a.im, b.im)}; }
__device__ __forceinline__ cx2 c2_sub(cx2 a, cx2 b) { return {x2_sub(a.re, b.re), x2_sub(a.im, b.im)}; }

// Constants of the radix-8 and radix-16 codelets, in both lanes:
// c = cos(pi/8), s = sin(pi/8), h = 1/sqrt(2), and their negatives.
struct X2Const {
  f32x2 c, s, ns, nc, h, nh, m1;
  __device__ __forceinline__ X2Const()
      : c(x2_bcast(0.92387953251128675613f)),
        s(x2_bcast(0.38268343236508977173f)),
        ns(x2_bcast(-0.38268343236508977173f)),
        nc(x2_bcast(-0.92387953251128675613f)),
        h(x2_bcast(0.70710678118654752440f)),
        nh(x2_bcast(-0.70710678118654752440f)),
        m1(x2_bcast(-1.0f)) {}
};

// x * W16^k, W16 = e^{-2 pi i / 16}, for the k a radix-16 (or radix-8) codelet needs
__device__ __forceinline__ cx2 x2_w16_1(cx2 x, const X2Const& K) {  // c - i s
  return {x2_fma(x.re, K.c, x2_mul(x.im, K.s)), x2_fma(x.im, K.c, x2_mul(x.re, K.ns))};
}
__device__ __forceinline__ cx2 x2_w16_2(cx2 x, const X2Const& K) {  // h (1 - i)
  return {x2_mul(x2_add(x.re, x.im), K.h), x2_mul(x2_sub(x.im, x.re), K.h)};
}
__device__ __forceinline__ cx2 x2_w16_3(cx2 x, const X2Const& K) {  // s - i c
  return {x2_fma(x.re, K.s, x2_mul(x.im, K.c)), x2_fma(x.im, K.s, x2_mul(x.re, K.nc))};
}
__device__ __forceinline__ cx2 x2_w16_6(cx2 x, const X2Const& K) {  // h (-1 - i)
  return {x2_mul(x2_sub(x.im, x.re), K.h), x2_mul(x2_add(x.re, x.im), K.nh)};
}
__device__ __forceinline__ cx2 x2_w16_9(cx2 x, const X2Const& K) {  // -c + i s
  return {x2_fma(x.re, K.nc, x2_mul(x.im, K.ns)), x2_fma(x.im, K.nc, x2_mul(x.re, K.s))};
}

// Radix-2 DFT in place; ROT1: a1 enters multiplied by -i (folded into the
// additions: -i a1 = (a1.im, -a1.re)).
template <bool ROT1>
__device__ __forceinline__ void x2_dft2(cx2& a0, cx2& a1) {
  if constexpr (ROT1) {
    const cx2 r0 = {x2_add(a0.re, a1.im), x2_sub(a0.im, a1.re)};
    a1 = {x2_sub(a0.re, a1.im), x2_add(a0.im, a1.re)};
    a0 = r0;
  } else {
    const cx2 r0 = c2_add(a0, a1);
    a1 = c2_sub(a0, a1);
    a0 = r0;
  }
}

// Radix-4 DFT in place (W4 = -i); ROT2: a2 enters multiplied by -i.
template <bool ROT2>
__device__ __forceinline__ void x2_dft4(cx2& a0, cx2& a1, cx2& a2, cx2& a3) {
  cx2 t0, t1;
  if constexpr (ROT2) {
    t0 = {x2_add(a0.re, a2.im), x2_sub(a0.im, a2.re)};
    t1 = {x2_sub(a0.re, a2.im), x2_add(a0.im, a2.re)};
  } else {
    t0 = c2_add(a0, a2);
    t1 = c2_sub(a0, a2);
  }
  const cx2 t2 = c2_add(a1, a3);
  const cx2 dd = c2_sub(a1, a3);  // a1 - a3; times -i is (dd.im, -dd.re)
  a0 = c2_add(t0, t2);
  a2 = c2_sub(t0, t2);
  a1 = {x2_add(t1.re, dd.im), x2_sub(t1.im, dd.re)};
  a3 = {x2_sub(t1.re, dd.im), x2_add(t1.im, dd.re)};
}

// Forward unnormalised DFT of RD points in place, natural order in and out.
template <int RD> struct X2Dft;

template <> struct X2Dft<2> {
  static __device__ __forceinline__ void run(cx2* x, const X2Const&) { x2_dft2<false>(x[0], x[1]); }
};
template <> struct X2Dft<4> {
  static __device__ __forceinline__ void run(cx2* x, const X2Const&) { x2_dft4<false>(x[0], x[1], x[2], x[3]); }
};
// 8 = 4 x 2: n = 2 n1 + n2, k = k1 + 4 k2
template <> struct X2Dft<8> {
  static __device__ __forceinline__ void run(cx2* x, const X2Const& K) {
    x2_dft4<false>(x[0], x[2], x[4], x[6]);  // n2 = 0 -> Y[0][k1] in slot 2 k1
    x2_dft4<false>(x[1], x[3], x[5], x[7]);  // n2 = 1 -> Y[1][k1] in slot 2 k1 + 1
    x[3] = x2_w16_2(x[3], K);                // W8^1
    x[7] = x2_w16_6(x[7], K);                // W8^3; W8^2 = -i is folded below
    x2_dft2<false>(x[0], x[1]);
    x2_dft2<false>(x[2], x[3]);
    x2_dft2<true>(x[4], x[5]);
    x2_dft2<false>(x[6], x[7]);
    // X[k1 + 4 k2] sits in slot 2 k1 + k2
    const cx2 y1 = x[2], y2 = x[4], y3 = x[6], y4 = x[1], y5 = x[3], y6 = x[5];
    x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6;
  }
};
// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
template <> struct X2Dft<16> {
  static __device__ __forceinline__ void run(cx2* x, const X2Const& K) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) x2_dft4<false>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
    // slot 4 k1 + n2 holds Y[n2][k1]; multiply by W16^{n2 k1}
    x[5] = x2_w16_1(x[5], K);
    x[9] = x2_w16_2(x[9], K);
    x[13] = x2_w16_3(x[13], K);
    x[6] = x2_w16_2(x[6], K);
    x[14] = x2_w16_6(x[14], K);   // slot 10 (W16^4 = -i) is folded below
    x[7] = x2_w16_3(x[7], K);
    x[11] = x2_w16_6(x[11], K);
    x[15] = x2_w16_9(x[15], K);
    x2_dft4<false>(x[0], x[1], x[2], x[3]);
    x2_dft4<false>(x[4], x[5], x[6], x[7]);
    x2_dft4<true>(x[8], x[9], x[10], x[11]);
    x2_dft4<false>(x[12], x[13], x[14], x[15]);
    // X[k1 + 4 k2] sits in slot 4 k1 + k2: transpose the 4 x 4 slots
    cx2 y[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) y[i] = x[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = y[4 * k1 + k2];
  }
};

// Radix-3 DFT in place, W3 = e^{-2 pi i / 3} = -1/2 - i sqrt(3)/2:
// X0 = a + (b + c), X1,2 = a - (b + c)/2 -/+ i sqrt(3)/2 (b - c).
__device__ __forceinline__ void x2_dft3(cx2& a, cx2& b, cx2& c) {
  const f32x2 mh = x2_bcast(-0.5f);
  const f32x2 r3 = x2_bcast(0.86602540378443864676f), nr3 = x2_bcast(-0.86602540378443864676f);
  const cx2 t = c2_add(b, c), d = c2_sub(b, c);
  const cx2 m = {x2_fma(t.re, mh, a.re), x2_fma(t.im, mh, a.im)};
  a = c2_add(a, t);
  b = {x2_fma(d.im, r3, m.re), x2_fma(d.re, nr3, m.im)};
  c = {x2_fma(d.im, nr3, m.re), x2_fma(d.re, r3, m.im)};
}
// 24 = 3 x 8 by the prime-factor (Good-Thomas) mapping, which needs no
// twiddles between the two layers: n = (8 n1 + 3 n2) mod 24 and
// k = (16 k1 + 9 k2) mod 24, so that W24^{nk} = W3^{n1 k1} W8^{n2 k2}.
template <> struct X2Dft<24> {
  static __device__ __forceinline__ void run(cx2* x, const X2Const& K) {
    // radix 3 over n1 for each n2: slots (3 n2, 3 n2 + 8, 3 n2 + 16) mod 24
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) x2_dft3(x[(3 * n2) % 24], x[(3 * n2 + 8) % 24], x[(3 * n2 + 16) % 24]);
    // radix 8 over n2 for each k1 (the slots (8 k1 + 3 n2) mod 24 of n1 = k1);
    // X[(16 k1 + 9 k2) mod 24] is output k2 of group k1
    cx2 t[3][8];
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
      for (int n2 = 0; n2 < 8; ++n2) t[k1][n2] = x[(8 * k1 + 3 * n2) % 24];
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) X2Dft<8>::run(t[k1], K);
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) x[(16 * k1 + 9 * k2) % 24] = t[k1][k2];
  }
};

// A twiddle factor in both lanes, with its negated sine.
struct tw2 {
  f32x2 c, s, ns;
};
__device__ __forceinline__ tw2 tw2_mul(const tw2& a, const tw2& b, const X2Const& K) {
  tw2 r;
  r.c = x2_fma(a.c, b.c, x2_mul(a.ns, b.s));
  r.s = x2_fma(a.c, b.s, x2_mul(a.s, b.c));
  r.ns = x2_mul(r.s, K.m1);
  return r;
}
__device__ __forceinline__ cx2 tw2_apply(cx2 x, const tw2& w) {
  return {x2_fma(x.re, w.c, x2_mul(x.im, w.ns)), x2_fma(x.re, w.s, x2_mul(x.im, w.c))};
}

// A scalar twiddle (c, s) in both lanes: the copies and the sign flip of s
// are integer moves, off the FP32 pipe.
__device__ __forceinline__ tw2 tw2_from(float2 w) {
  const float ns = __int_as_float(__float_as_int(w.y) ^ 0x80000000);
  return {x2_pack(w.x, w.x), x2_pack(w.y, w.y), x2_pack(ns, ns)};
}

// x[r] *= w1^r for r = 1 .. RD-1 with the powers computed once as scalars
// (each product is the same for both lines; in packed form both lanes would
// repeat it) as w^{2^k} * w^{r - 2^k}, w^{2^k} by repeated squaring.
template <int RD>
__device__ __forceinline__ void x2_twiddle_scalar_powers(cx2* x, float2 wb) {
  float2 w[RD];
  w[1] = wb;
#pragma unroll
  for (int r = 2; r < RD; ++r) {
    const int hi = (r & (r - 1)) == 0 ? r / 2 : (1 << (31 - __clz(r)));
    const int lo = (r & (r - 1)) == 0 ? r / 2 : r - hi;
    w[r] = make_float2(w[hi].x * w[lo].x - w[hi].y * w[lo].y, w[hi].x * w[lo].y + w[hi].y * w[lo].x);
  }
#pragma unroll
  for (int r = 1; r < RD; ++r) x[r] = tw2_apply(x[r], tw2_from(w[r]));
}

// x[r] *= w1^r for r = 1 .. RD-1, each power as w^{2^k} * w^{r - 2^k} with
// w^{2^k} by repeated squaring (the products and their rounding depth are
// those of the scalar kernels' twiddle powers). Powers are made just before
// use so that few of them are live at once.
template <int RD>
__device__ __forceinline__ void x2_twiddle(cx2* x, float2 wb, const X2Const& K) {
  const tw2 w1 = {x2_bcast(wb.x), x2_bcast(wb.y), x2_bcast(-wb.y)};
  x[1] = tw2_apply(x[1], w1);
  if constexpr (RD >= 4) {
    const tw2 w2 = tw2_mul(w1, w1, K);
    x[2] = tw2_apply(x[2], w2);
    const tw2 w3 = tw2_mul(w2, w1, K);
    x[3] = tw2_apply(x[3], w3);
    if constexpr (RD >= 8) {
      const tw2 w4 = tw2_mul(w2, w2, K);
      x[4] = tw2_apply(x[4], w4);
      tw2 w8;
      if constexpr (RD >= 16) {
        w8 = tw2_mul(w4, w4, K);
        x[8] = tw2_apply(x[8], w8);
        x[9] = tw2_apply(x[9], tw2_mul(w8, w1, K));
        x[10] = tw2_apply(x[10], tw2_mul(w8, w2, K));
        x[11] = tw2_apply(x[11], tw2_mul(w8, w3, K));
        x[12] = tw2_apply(x[12], tw2_mul(w8, w4, K));
      }
      const tw2 w5 = tw2_mul(w4, w1, K);
      x[5] = tw2_apply(x[5], w5);
      if constexpr (RD >= 16) x[13] = tw2_apply(x[13], tw2_mul(w8, w5, K));
      const tw2 w6 = tw2_mul(w4, w2, K);
      x[6] = tw2_apply(x[6], w6);
      if constexpr (RD >= 16) x[14] = tw2_apply(x[14], tw2_mul(w8, w6, K));
      const tw2 w7 = tw2_mul(w4, w3, K);
      x[7] = tw2_apply(x[7], w7);
      if constexpr (RD >= 16) x[15] = tw2_apply(x[15], tw2_mul(w8, w7, K));
    }
  }
}

}  // namespace nslct
