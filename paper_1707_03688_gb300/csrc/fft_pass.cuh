// Fused FFT pass kernels for the CM-CC-CM-CC chain.
//
// Every pass of the chain (Eq. HA28 applied right to left, split into five
// passes over HBM) has the shape
//     load panel -> [1D FFT or IFFT] -> [chirp x scale] -> [1D FFT or IFFT] -> store
// along rows (row pass) or columns (column pass). A CTA owns a panel of P whole
// lines, so a chirp convolution's FFT -> chirp -> IFFT along one axis never
// leaves the chip.
//
// 1D FFTs are unnormalised mixed-radix Stockham transforms (radices 2,3,4,8,16,24)
// in registers with shared-memory exchanges between stages. Each thread owns
// E elements of a line, e = t + T_LINE * s (s = 0..E-1), both at the start and
// at the end of every 1D transform, so the chirp multiply between two
// transforms happens in registers and the global loads/stores are coalesced.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "fft_schedule.h"
#include "pair_x2.cuh"

namespace nslct {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename R> struct Cpx;
template <> struct Cpx<float> { using T = float2; };
template <> struct Cpx<double> { using T = double2; };
template <typename R> using cpx = typename Cpx<R>::T;

template <typename R> __device__ __forceinline__ cpx<R> mk(R x, R y) { cpx<R> c; c.x = x; c.y = y; return c; }
template <typename R> __device__ __forceinline__ cpx<R> cadd(cpx<R> a, cpx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ cpx<R> csub(cpx<R> a, cpx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i: (x + iy)(-i) = y - ix
template <typename R> __device__ __forceinline__ cpx<R> mul_negi(cpx<R> a) { return mk<R>(a.y, -a.x); }
template <typename R> __device__ __forceinline__ cpx<R> mul_posi(cpx<R> a) { return mk<R>(-a.y, a.x); }

// ---------------------------------------------------------------------------
// compile-time roots of unity: W_N^k = exp(-2 pi i k / N)
// Own Taylor-series evaluation of cos/sin on [-pi/4, pi/4] after an exact
// octant reduction of the rational angle k/N.
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 14; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 14; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
// cos(2 pi k / n) and sin(2 pi k / n) with exact reduction of k/n to [0, 1/8].
__host__ __device__ constexpr double cos2pi(long k, long n) {
  k %= n; if (k < 0) k += n;
  // angle = 2 pi k / n; use symmetry in eighths: 8k vs n
  if (8 * k <= n) return taylor_cos(2.0 * kPi * (double)k / (double)n);
  if (8 * k <= 2 * n) return taylor_sin(2.0 * kPi * (double)(n - 4 * k) / (4.0 * (double)n));   // cos(pi/2 - y) = sin y
  if (8 * k <= 4 * n) return -cos2pi(n - 2 * k, 2 * n);                                          // cos(pi - y) = -cos y
  return cos2pi(n - k, n);                                                                       // cos(2pi - y) = cos y
}
__host__ __device__ constexpr double sin2pi(long k, long n) {
  k %= n; if (k < 0) k += n;
  if (8 * k <= n) return taylor_sin(2.0 * kPi * (double)k / (double)n);
  if (8 * k <= 2 * n) return taylor_cos(2.0 * kPi * (double)(n - 4 * k) / (4.0 * (double)n));
  if (8 * k <= 4 * n) return sin2pi(n - 2 * k, 2 * n);                                           // sin(pi - y) = sin y
  return -sin2pi(n - k, n);                                                                      // sin(2pi - y) = -sin y
}

// x *= W_N^K, specialised for the trivial roots.
template <typename R, int N, int K>
__device__ __forceinline__ cpx<R> twc(cpx<R> x) {
  constexpr int k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    return x;
  } else if constexpr (4 * k == N) {
    return mul_negi<R>(x);
  } else if constexpr (2 * k == N) {
    return mk<R>(-x.x, -x.y);
  } else if constexpr (4 * k == 3 * N) {
    return mul_posi<R>(x);
  } else if constexpr (8 * k == N) {          // (1 - i)/sqrt2
    constexpr R h = (R)0.70710678118654752440084436210485;
    return mk<R>(h * (x.x + x.y), h * (x.y - x.x));
  } else if constexpr (8 * k == 3 * N) {      // (-1 - i)/sqrt2
    constexpr R h = (R)0.70710678118654752440084436210485;
    return mk<R>(h * (x.y - x.x), -h * (x.x + x.y));
  } else {
    constexpr R c = (R)cos2pi(k, N);
    constexpr R s = (R)(-sin2pi(k, N));
    return mk<R>(x.x * c - x.y * s, x.x * s + x.y * c);
  }
}

// ---------------------------------------------------------------------------
// forward DFT codelets in registers (unnormalised, W = e^{-2 pi i / N})
// ---------------------------------------------------------------------------
template <typename R, int N> struct Dft;

template <typename R> struct Dft<R, 1> {
  static __device__ __forceinline__ void run(cpx<R>*) {}
};

template <typename R> struct Dft<R, 2> {
  static __device__ __forceinline__ void run(cpx<R>* a) {
    cpx<R> t = a[0];
    a[0] = cadd<R>(t, a[1]);
    a[1] = csub<R>(t, a[1]);
  }
};

template <typename R> struct Dft<R, 3> {
  static __device__ __forceinline__ void run(cpx<R>* a) {
    constexpr R s3 = (R)0.86602540378443864676372317075294;  // sin(2 pi / 3)
    cpx<R> t = cadd<R>(a[1], a[2]);
    cpx<R> d = csub<R>(a[1], a[2]);
    cpx<R> m = mk<R>(a[0].x - (R)0.5 * t.x, a[0].y - (R)0.5 * t.y);
    // -i * s3 * d = (s3 d.y, -s3 d.x)
    cpx<R> r = mk<R>(s3 * d.y, -s3 * d.x);
    a[0] = cadd<R>(a[0], t);
    a[1] = cadd<R>(m, r);
    a[2] = csub<R>(m, r);
  }
};

template <typename R> struct Dft<R, 4> {
  static __device__ __forceinline__ void run(cpx<R>* a) {
    cpx<R> t0 = cadd<R>(a[0], a[2]);
    cpx<R> t1 = csub<R>(a[0], a[2]);
    cpx<R> t2 = cadd<R>(a[1], a[3]);
    cpx<R> t3 = mul_negi<R>(csub<R>(a[1], a[3]));
    a[0] = cadd<R>(t0, t2);
    a[2] = csub<R>(t0, t2);
    a[1] = cadd<R>(t1, t3);
    a[3] = csub<R>(t1, t3);
  }
};

// Composite N = N1 * N2 (Cooley-Tukey inside one thread):
//   n = N2 n1 + n2, k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_n2 W_N2^{n2 k2} W_N^{n2 k1} sum_n1 x[N2 n1 + n2] W_N1^{n1 k1}
template <typename R, int N1, int N2>
struct DftComposite {
  static __device__ __forceinline__ void run(cpx<R>* a) {
    constexpr int N = N1 * N2;
    cpx<R> t[N];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      cpx<R> col[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) col[n1] = a[N2 * n1 + n2];
      Dft<R, N1>::run(col);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) t[n2 * N1 + k1] = col[k1];
    }
    apply_tw<0>(t);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      cpx<R> row[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) row[n2] = t[n2 * N1 + k1];
      Dft<R, N2>::run(row);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) a[k1 + N1 * k2] = row[k2];
    }
  }
  // t[n2 * N1 + k1] *= W_N^{n2 k1}, unrolled at compile time
  template <int I>
  static __device__ __forceinline__ void apply_tw(cpx<R>* t) {
    if constexpr (I < N1 * N2) {
      constexpr int n2 = I / N1, k1 = I % N1;
      t[I] = twc<R, N1 * N2, n2 * k1>(t[I]);
      apply_tw<I + 1>(t);
    }
  }
};

template <typename R> struct Dft<R, 6> : DftComposite<R, 3, 2> {};
template <typename R> struct Dft<R, 8> : DftComposite<R, 4, 2> {};
template <typename R> struct Dft<R, 12> : DftComposite<R, 4, 3> {};
template <typename R> struct Dft<R, 16> : DftComposite<R, 4, 4> {};
template <typename R> struct Dft<R, 24> : DftComposite<R, 8, 3> {};
template <typename R> struct Dft<R, 32> : DftComposite<R, 8, 4> {};
template <typename R> struct Dft<R, 64> : DftComposite<R, 8, 8> {};

__device__ __forceinline__ int padded(int e) { return e + (e >> 4); }
template <int SH> __device__ __forceinline__ int padded_by(int e) { return e + (e >> SH); }

// LM (line-major): the T_LINE threads of line p are threads p*T_LINE .. ,
// whole warps, so each line keeps its exchange buffer to itself
// (p*(L + L/16) + padded(e)) and synchronises on its own named barrier
// (1 + p) instead of the whole CTA. Otherwise lines are interleaved thread by
// thread (padded(e)*P + p) and share __syncthreads.
// w[r] = w1^r for r = 1 .. RD-1 (w[0] unused), each as w[2^k] * w[r - 2^k] with
// w[2^k] by repeated squaring: at most four roundings deep for RD = 16. This
// replaces RD-1 table loads per butterfly by one load of the base twiddle
// W_{NS*RD}^{jm} (the compact table) and RD-2 complex products.
template <typename R, int RD>
__device__ __forceinline__ void twiddle_powers(cpx<R> w1, cpx<R>* w) {
  w[1] = w1;
#pragma unroll
  for (int r = 2; r < RD; ++r) {
    const int hi = (r & (r - 1)) == 0 ? r / 2 : (1 << (31 - __clz(r)));
    const int lo = (r & (r - 1)) == 0 ? r / 2 : r - hi;
    w[r] = cmul<R>(w[hi], w[lo]);
  }
}

// Twiddles of stage ST for butterfly jm from the full table,
// tab[OFF + jm*RD + r] = W_{NS*RD}^{jm*r}: each correctly rounded (used where
// the extra rounding of the register powers matters, the adjoint kernels).
template <typename R, int RD>
__device__ __forceinline__ void load_twiddles(const cpx<R>* __restrict__ row, cpx<R>* w) {
  if constexpr (sizeof(R) == 4 && RD % 2 == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(row);  // rows start at even entries
#pragma unroll
    for (int r = 0; r < RD; r += 2) {
      const float4 q = __ldg(p4 + r / 2);
      w[r] = mk<R>(q.x, q.y);
      w[r + 1] = mk<R>(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int r = 0; r < RD; ++r) w[r] = row[r];
  }
}

// EXACT = true: table twiddles (load_twiddles); false: one base twiddle per
// butterfly and its powers in registers (twiddle_powers).
template <typename R, int L, int P, int E_ = elems_per_thread(L), bool LM = false, bool EXACT = false>
struct LineFft {
  static constexpr int E = E_;
  static constexpr int T_LINE = L / E;
  static constexpr int S = num_stages(L, E);
  static constexpr int SH = pad_shift(E);
  static constexpr int LS = L + (L >> SH);
  static_assert(L % E == 0, "bad E");
  static_assert(!LM || (T_LINE % 32 == 0 && P <= 15), "line-major needs whole warps per line");

  static __device__ __forceinline__ void sync(int p) {
    if constexpr (LM) {
      asm volatile("bar.sync %0, %1;\n" ::"r"(p + 1), "n"(T_LINE) : "memory");
    } else {
      __syncthreads();
    }
  }
  static __device__ __forceinline__ int sidx(int p, int e) {
    if constexpr (LM) return p * LS + padded_by<SH>(e);
    return padded_by<SH>(e) * P + p;
  }

  // One Stockham stage; FIRST stage reads the registers, later stages read the
  // shared-memory line; the LAST stage leaves its result in registers.
  template <int ST>
  static __device__ __forceinline__ void stage(cpx<R>* v, cpx<R>* sm, int t, int p, const cpx<R>* __restrict__ tw) {
    constexpr int RD = stage_radix(L, E, ST);
    constexpr int NS = stage_ns(L, E, ST);
    constexpr bool FIRST = (ST == 0);
    constexpr bool LAST = (ST == S - 1);
    constexpr int NB = E / RD;  // butterflies per thread
    static_assert(E % RD == 0, "radix must divide E");
    if constexpr (!FIRST) {
      sync(p);
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = sm[sidx(p, t + T_LINE * s)];
      if constexpr (!LAST) sync(p);
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      cpx<R> x[RD];
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = v[u + r * NB];
      const int j = t + u * T_LINE;
      const int jm = j % NS;
      if constexpr (NS > 1) {
        cpx<R> w[RD];
        if constexpr (EXACT) load_twiddles<R, RD>(tw + stage_table_offset(L, E, ST) + jm * RD, w);
        else twiddle_powers<R, RD>(tw[compact_table_offset(L, E, ST) + jm], w);
#pragma unroll
        for (int r = 1; r < RD; ++r) x[r] = cmul<R>(x[r], w[r]);
      }
      Dft<R, RD>::run(x);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < RD; ++r) v[u + r * NB] = x[r];
      } else {
        const int base = (j / NS) * NS * RD + jm;
#pragma unroll
        for (int r = 0; r < RD; ++r) sm[sidx(p, base + r * NS)] = x[r];
      }
    }
  }

  template <int ST>
  static __device__ __forceinline__ void stages(cpx<R>* v, cpx<R>* sm, int t, int p, const cpx<R>* __restrict__ tw) {
    if constexpr (ST < S) {
      stage<ST>(v, sm, t, p, tw);
      stages<ST + 1>(v, sm, t, p, tw);
    }
  }

  // Unnormalised forward (inverse = false) or inverse DFT of the thread's line.
  // The inverse uses conj(DFT(conj(x))).
  static __device__ __forceinline__ void run(cpx<R>* v, cpx<R>* sm, int t, int p, const cpx<R>* __restrict__ tw,
                                             bool inverse) {
    if (inverse) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s].y = -v[s].y;
    }
    if constexpr (S > 1) sync(p);  // the previous user of `sm` is done
    stages<0>(v, sm, t, p, tw);
    if (inverse) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s].y = -v[s].y;
    }
  }
};

// Two FP32 fields' copies of the same line through one FFT schedule (the
// adjoint's gradient and value paths): the exchanges move (a[e], b[e]) as one
// 16-byte entry and each (correctly rounded) twiddle load serves both.
template <int L, int P, int E_ = elems_per_thread(L)>
struct LineFft2 {
  static constexpr int E = E_;
  static constexpr int T_LINE = L / E;
  static constexpr int S = num_stages(L, E);
  static constexpr int SH = pad_shift(E);
  static __device__ __forceinline__ int sidx(int p, int e) { return padded_by<SH>(e) * P + p; }

  template <int ST>
  static __device__ __forceinline__ void stage(float2* a, float2* b, float4* sm, int t, int p,
                                               const float2* __restrict__ tw) {
    constexpr int RD = stage_radix(L, E, ST);
    constexpr int NS = stage_ns(L, E, ST);
    constexpr bool FIRST = (ST == 0);
    constexpr bool LAST = (ST == S - 1);
    constexpr int NB = E / RD;
    if constexpr (!FIRST) {
      __syncthreads();
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const float4 q = sm[sidx(p, t + T_LINE * s)];
        a[s] = make_float2(q.x, q.y);
        b[s] = make_float2(q.z, q.w);
      }
      if constexpr (!LAST) __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      float2 xa[RD], xb[RD];
#pragma unroll
      for (int r = 0; r < RD; ++r) {
        xa[r] = a[u + r * NB];
        xb[r] = b[u + r * NB];
      }
      const int j = t + u * T_LINE;
      const int jm = j % NS;
      if constexpr (NS > 1) {
        float2 w[RD];
        load_twiddles<float, RD>(tw + stage_table_offset(L, E, ST) + jm * RD, w);
#pragma unroll
        for (int r = 1; r < RD; ++r) {
          xa[r] = cmul<float>(xa[r], w[r]);
          xb[r] = cmul<float>(xb[r], w[r]);
        }
      }
      Dft<float, RD>::run(xa);
      Dft<float, RD>::run(xb);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < RD; ++r) {
          a[u + r * NB] = xa[r];
          b[u + r * NB] = xb[r];
        }
      } else {
        const int base = (j / NS) * NS * RD + jm;
#pragma unroll
        for (int r = 0; r < RD; ++r) sm[sidx(p, base + r * NS)] = make_float4(xa[r].x, xa[r].y, xb[r].x, xb[r].y);
      }
    }
  }

  template <int ST>
  static __device__ __forceinline__ void stages(float2* a, float2* b, float4* sm, int t, int p,
                                                const float2* __restrict__ tw) {
    if constexpr (ST < S) {
      stage<ST>(a, b, sm, t, p, tw);
      stages<ST + 1>(a, b, sm, t, p, tw);
    }
  }

  static __device__ __forceinline__ void run(float2* a, float2* b, float4* sm, int t, int p,
                                             const float2* __restrict__ tw, bool inverse) {
    if (inverse) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        a[s].y = -a[s].y;
        b[s].y = -b[s].y;
      }
    }
    if constexpr (S > 1) __syncthreads();
    stages<0>(a, b, sm, t, p, tw);
    if (inverse) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        a[s].y = -a[s].y;
        b[s].y = -b[s].y;
      }
    }
  }
};

// ---------------------------------------------------------------------------
// Split-precision tensor-core DFT-16 (the mixed mode, NSLCT_PREC_SPLIT_F16)
//
// A radix-16 Stockham stage applied to 8 butterflies at a time is the complex
// product D = W X of the 16 x 16 DFT matrix W (W[m][k] = e^{-2 pi i mk/16})
// with X (16 points x 8 butterflies). In real-block form
//     Re D = Wr Xr - Wi Xi,   Im D = Wi Xr + Wr Xi,
// and every real operand is split into FP16 halves, v = v_hi + v_lo, so
//     A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi      (FP32 accumulation)
// keeps ~22 significant bits. Each product is one warp-level
// mma.m16n8k16 (f16 inputs, f32 accumulators): 12 per 8 butterflies.
// Twiddles between stages stay FP32. The data move through shared memory at
// every stage (the MMA fragments do not match the one-butterfly-per-thread
// register layout), so the line visits shared memory S + 1 times instead of
// S - 1.
// ---------------------------------------------------------------------------
template <int R> struct W16c {
  static constexpr float c = (float)cos2pi(R, 16);
  static constexpr float s = (float)(-sin2pi(R, 16));
};
__constant__ float kW16re[16] = {W16c<0>::c, W16c<1>::c, W16c<2>::c, W16c<3>::c, W16c<4>::c, W16c<5>::c,
                                 W16c<6>::c, W16c<7>::c, W16c<8>::c, W16c<9>::c, W16c<10>::c, W16c<11>::c,
                                 W16c<12>::c, W16c<13>::c, W16c<14>::c, W16c<15>::c};
__constant__ float kW16im[16] = {W16c<0>::s, W16c<1>::s, W16c<2>::s, W16c<3>::s, W16c<4>::s, W16c<5>::s,
                                 W16c<6>::s, W16c<7>::s, W16c<8>::s, W16c<9>::s, W16c<10>::s, W16c<11>::s,
                                 W16c<12>::s, W16c<13>::s, W16c<14>::s, W16c<15>::s};

__device__ __forceinline__ uint32_t h2bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
// FP16 halves of (a, b): hi = fp16(v), lo = fp16(v - hi), packed low = a
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  hi = h2bits(h);
  lo = h2bits(__floats2half2_rn(a - hf.x, b - hf.y));
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Constant A fragments of W (row-major 16 x 16) for this lane: register q holds
// rows g + 8 (q & 1), columns 2c + 8 (q >> 1) + {0, 1}, g = lane / 4, c = lane % 4.
struct DftFrags {
  uint32_t re_hi[4], re_lo[4], im_hi[4], im_lo[4], nim_hi[4], nim_lo[4];
  __device__ __forceinline__ void init(int lane) {
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = g + 8 * (q & 1), k0 = 2 * c + 8 * (q >> 1);
      const int r0 = (m * k0) & 15, r1 = (m * (k0 + 1)) & 15;
      split_pair(kW16re[r0], kW16re[r1], re_hi[q], re_lo[q]);
      split_pair(kW16im[r0], kW16im[r1], im_hi[q], im_lo[q]);
      split_pair(-kW16im[r0], -kW16im[r1], nim_hi[q], nim_lo[q]);
    }
  }
};

template <int L, int P, int E>
struct MixedLineFft {
  using Base = LineFft<float, L, P, E, false>;
  static constexpr int T_LINE = L / E;
  static constexpr int S = num_stages(L, E);
  static constexpr int NBF = L / 16;                   // radix-16 butterflies per line
  static constexpr int THREADS = T_LINE * P;
  static_assert(E == 16, "the split-precision mode runs with 16 elements per thread");

  static __device__ __forceinline__ int sidx(int p, int e) { return padded(e) * P + p; }

  // One radix-16 stage on tensor cores, shared memory -> shared memory.
  template <int ST>
  static __device__ __forceinline__ void mma_stage(float2* sm, const float2* __restrict__ tw, const DftFrags& W) {
    constexpr int NS = stage_ns(L, E, ST);
    constexpr int NG = NBF / 8;                          // 8-butterfly groups per line
    constexpr int GPW = (P * NG) / (THREADS / 32);       // groups per warp (4)
    static_assert((P * NG) % (THREADS / 32) == 0, "groups per warp");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, c = lane & 3;
    uint32_t xr_hi[GPW][2], xr_lo[GPW][2], xi_hi[GPW][2], xi_lo[GPW][2];
    float inv_scale[GPW];  // 2^e of the butterfly this lane fed in (vector g)
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GPW; ++q) {
      const int G = warp * GPW + q;
      const int p = G / NG, j = (G % NG) * 8 + g;
      float2 x[4];
      const int ks[4] = {2 * c, 2 * c + 1, 2 * c + 8, 2 * c + 9};
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = sm[sidx(p, j + ks[u] * NBF)];
      if constexpr (NS > 1) {
        const float4* row = reinterpret_cast<const float4*>(tw + stage_table_offset(L, E, ST) + (j % NS) * 16);
        const float4 w01 = __ldg(row + c), w89 = __ldg(row + c + 4);
        x[0] = cmul<float>(x[0], make_float2(w01.x, w01.y));
        x[1] = cmul<float>(x[1], make_float2(w01.z, w01.w));
        x[2] = cmul<float>(x[2], make_float2(w89.x, w89.y));
        x[3] = cmul<float>(x[3], make_float2(w89.z, w89.w));
      }
      // Scale the butterfly (held by the 4 lanes with this g) by an exact power
      // of two so its largest component lies in [0.5, 1): FP16 neither
      // overflows (unnormalised FFT values grow to ~N |x|) nor drops the small
      // split halves into subnormals.
      float mx = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) mx = fmaxf(mx, fmaxf(fabsf(x[u].x), fabsf(x[u].y)));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      // clamped so that both 2^-ex and 2^ex stay finite: subnormal inputs (the
      // underflowed tails of a field) would otherwise ask for 2^+132
      const int ex = mx > 0.f ? min(max(ilogbf(mx) + 1, -125), 127) : 0;
      const float sc = ldexpf(1.0f, -ex);
      inv_scale[q] = ldexpf(1.0f, ex);
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = make_float2(x[u].x * sc, x[u].y * sc);
      split_pair(x[0].x, x[1].x, xr_hi[q][0], xr_lo[q][0]);
      split_pair(x[2].x, x[3].x, xr_hi[q][1], xr_lo[q][1]);
      split_pair(x[0].y, x[1].y, xi_hi[q][0], xi_lo[q][0]);
      split_pair(x[2].y, x[3].y, xi_hi[q][1], xi_lo[q][1]);
    }
    __syncthreads();  // every input read before any output lands
#pragma unroll
    for (int q = 0; q < GPW; ++q) {
      const int G = warp * GPW + q;
      const int p = G / NG, gbase = (G % NG) * 8;
      float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
      mma16816(dr, W.re_hi, xr_hi[q][0], xr_hi[q][1]);
      mma16816(dr, W.re_hi, xr_lo[q][0], xr_lo[q][1]);
      mma16816(dr, W.re_lo, xr_hi[q][0], xr_hi[q][1]);
      mma16816(dr, W.nim_hi, xi_hi[q][0], xi_hi[q][1]);
      mma16816(dr, W.nim_hi, xi_lo[q][0], xi_lo[q][1]);
      mma16816(dr, W.nim_lo, xi_hi[q][0], xi_hi[q][1]);
      mma16816(di, W.im_hi, xr_hi[q][0], xr_hi[q][1]);
      mma16816(di, W.im_hi, xr_lo[q][0], xr_lo[q][1]);
      mma16816(di, W.im_lo, xr_hi[q][0], xr_hi[q][1]);
      mma16816(di, W.re_hi, xi_hi[q][0], xi_hi[q][1]);
      mma16816(di, W.re_hi, xi_lo[q][0], xi_lo[q][1]);
      mma16816(di, W.re_lo, xi_hi[q][0], xi_hi[q][1]);
      // d[v]: output point m = g + 8 (v >> 1) of butterfly (vector) n = 2c + (v & 1),
      // whose scale sits with the lanes 4n .. 4n + 3
      const float us0 = __shfl_sync(0xffffffffu, inv_scale[q], 8 * c);
      const float us1 = __shfl_sync(0xffffffffu, inv_scale[q], 8 * c + 4);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int m = g + 8 * (v >> 1);
        const int j = gbase + 2 * c + (v & 1);
        const int base = (j / NS) * NS * 16 + (j % NS);
        const float us = (v & 1) ? us1 : us0;
        sm[sidx(p, base + m * NS)] = make_float2(dr[v] * us, di[v] * us);
      }
    }
  }

  // A non-radix-16 stage, FP32, shared memory -> shared memory.
  template <int ST>
  static __device__ __forceinline__ void fp32_stage(float2* sm, const float2* __restrict__ tw, int t, int p) {
    constexpr int RD = stage_radix(L, E, ST);
    constexpr int NS = stage_ns(L, E, ST);
    constexpr int NB = E / RD;
    float2 v[E];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = sm[sidx(p, t + T_LINE * s)];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      float2 x[RD];
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = v[u + r * NB];
      const int j = t + u * T_LINE;
      const int jm = j % NS;
      if constexpr (NS > 1) {
        float2 w[RD];
        twiddle_powers<float, RD>(__ldg(tw + compact_table_offset(L, E, ST) + jm), w);
#pragma unroll
        for (int r = 1; r < RD; ++r) x[r] = cmul<float>(x[r], w[r]);
      }
      Dft<float, RD>::run(x);
      const int base = (j / NS) * NS * RD + jm;
#pragma unroll
      for (int r = 0; r < RD; ++r) sm[sidx(p, base + r * NS)] = x[r];
    }
  }

  template <int ST>
  static __device__ __forceinline__ void stages(float2* sm, const float2* __restrict__ tw, int t, int p,
                                                const DftFrags& W) {
    if constexpr (ST < S) {
      if constexpr (stage_radix(L, E, ST) == 16) mma_stage<ST>(sm, tw, W);
      else fp32_stage<ST>(sm, tw, t, p);
      stages<ST + 1>(sm, tw, t, p, W);
    }
  }

  static __device__ __forceinline__ void run(float2* v, float2* sm, int t, int p, const float2* __restrict__ tw,
                                             bool inverse) {
    DftFrags W;
    W.init(threadIdx.x & 31);
    __syncthreads();  // the previous user of `sm` is done
#pragma unroll
    for (int s = 0; s < E; ++s) sm[sidx(p, t + T_LINE * s)] = make_float2(v[s].x, inverse ? -v[s].y : v[s].y);
    stages<0>(sm, tw, t, p, W);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const float2 z = sm[sidx(p, t + T_LINE * s)];
      v[s] = make_float2(z.x, inverse ? -z.y : z.y);
    }
  }
};

// ---------------------------------------------------------------------------
// chirp evaluation
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t chirp_turns(const Chirp& c, long long a, long long b) {
  return c.k11 * (uint64_t)(a * a) + c.k12 * (uint64_t)(a * b) + c.k22 * (uint64_t)(b * b);
}

// e^{2 pi i turns} * scale; turns is a Q0.64 fraction of a full turn
__device__ __forceinline__ float2 chirp_value(uint64_t q, float scale) {
  // top 32 bits as a signed fraction in [-1/2, 1/2)
  const float tt = (float)(int)(unsigned)(q >> 32) * 2.3283064365386963e-10f;  // 2^-32
  float s, c;
  __sincosf(6.28318530717958647692f * tt, &s, &c);
  return make_float2(c * scale, s * scale);
}
__device__ __forceinline__ double2 chirp_value(uint64_t q, double scale) {
  const double tt = (double)(long long)q * 5.421010862427522170037264e-20;  // 2^-64
  double s, c;
  sincospi(2.0 * tt, &s, &c);
  return make_double2(c * scale, s * scale);
}

__device__ __forceinline__ int centred_bin(int b, int n) { return b < (n + 1) / 2 ? b : b - n; }

// Output-domain mask of a row-major output pass: value (i, j) of the grid is
// multiplied by the mask element at the same output position (the output
// region's coordinates for a cropped padded plan); positions outside the
// stored region are left alone.
template <typename R>
__device__ __forceinline__ cpx<R> apply_post_mask(const PassDesc& d, int i, int j, cpx<R> v) {
  const int rows = d.pad_out ? d.out_rows : d.Nx, cols = d.pad_out ? d.out_cols : d.Ny;
  const int r = d.pad_out ? i - d.out_r0 : i, c = d.pad_out ? j - d.out_c0 : j;
  if ((unsigned)r >= (unsigned)rows || (unsigned)c >= (unsigned)cols) return v;
  return cmul<R>(v, reinterpret_cast<const cpx<R>*>(d.post_mask)[(size_t)r * cols + c]);
}

// element (i, j) of an Nx x Ny field in the given layout
__device__ __forceinline__ int elem_index(int i, int j, int Ny, int tiled) {
  if (!tiled) return i * Ny + j;
  return (i >> 1) * (2 * Ny) + (j >> 1) * 4 + (i & 1) * 2 + (j & 1);
}

// Multiply the thread's E elements of line `line` by the pass chirp.
// Element s sits at index e = t + T_LINE s along the line. The phase is a
// quadratic in the element's integer coordinate a(s), which is linear in s
// (centred samples: a = e - N/2; centred bins: a = e for e < N/2, e - N
// after, and e < N/2 exactly when s < E/2 because N/2 is a multiple of
// T_LINE). So the Q0.64 phase is advanced with two 64-bit additions per
// element: q(s+1) = q(s) + D(s), D(s+1) = D(s) + 2 k T^2, all exact mod 2^64.
template <typename R, int L, bool COL, int E = elems_per_thread(L)>
__device__ __forceinline__ void apply_chirp_c(cpx<R>* v, const PassDesc& d, const Chirp& ch, int freq, int t,
                                              int line, R scale);

template <typename R, int L, bool COL, int E = elems_per_thread(L)>
__device__ __forceinline__ void apply_chirp(cpx<R>* v, const PassDesc& d, int t, int line, R scale) {
  apply_chirp_c<R, L, COL, E>(v, d, d.chirp, d.freq_domain, t, line, scale);
}

template <typename R, int L, bool COL, int E>
__device__ __forceinline__ void apply_chirp_c(cpx<R>* v, const PassDesc& d, const Chirp& ch, int freq, int t,
                                              int line, R scale) {
  constexpr int T = L / E;
  const int nl = COL ? d.Ny : d.Nx;   // length of the other axis
  // coordinate of the line and of element 0
  long long b, a0;
  if (freq) {
    b = centred_bin(line, nl);
    a0 = t;
  } else {
    b = (long long)line - nl / 2;
    a0 = (long long)t - L / 2;
  }
  // phase = ka a^2 + kab a b + kb b^2 with (ka, kb) the element/line coefficients
  const uint64_t ka = COL ? ch.k11 : ch.k22;
  const uint64_t kb = COL ? ch.k22 : ch.k11;
  const uint64_t kab_b = ch.k12 * (uint64_t)b;
  const uint64_t base = kb * (uint64_t)(b * b);
  auto phase_at = [&](long long a) -> uint64_t { return ka * (uint64_t)(a * a) + kab_b * (uint64_t)a + base; };
  const uint64_t dd = 2ull * ka * (uint64_t)((long long)T * T);
  uint64_t q = phase_at(a0);
  uint64_t dq = ka * (uint64_t)(2 * a0 * T + (long long)T * T) + kab_b * (uint64_t)T;
#pragma unroll
  for (int s = 0; s < E; ++s) {
    if (freq && s == E / 2) {
      const long long a = a0 + (long long)T * s - L;
      q = phase_at(a);
      dq = ka * (uint64_t)(2 * a * T + (long long)T * T) + kab_b * (uint64_t)T;
    }
    v[s] = cmul<R>(v[s], chirp_value(q, scale));
    q += dq;
    dq += dd;
  }
}

// ---------------------------------------------------------------------------
// v1: one panel per CTA, global loads straight into registers (FP64 plans)
// ---------------------------------------------------------------------------
template <typename R, int L> struct PassShape {
  static constexpr int E = elems_per_thread(L);
  static constexpr int T_LINE = L / E;
  static constexpr int MAX_THREADS = 512;
  static constexpr int P0 = MAX_THREADS / T_LINE;
  static constexpr int P = P0 < 2 ? 2 : (P0 > 32 ? 32 : P0);
  static constexpr int THREADS = T_LINE * P;
  static constexpr int XSM = P * (L + L / 16);          // exchange buffer (complex entries)
  static constexpr size_t SMEM = (size_t)XSM * sizeof(cpx<R>);
};

template <typename R, int L, bool COL>
__global__ void __launch_bounds__(PassShape<R, L>::THREADS, 1)
pass_kernel(PassDesc d) {
  using Sh = PassShape<R, L>;
  constexpr int E = Sh::E;
  constexpr int T_LINE = Sh::T_LINE;
  constexpr int P = Sh::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);

  const int tid = threadIdx.x;
  const int p = tid % P;
  const int t = tid / P;
  const int nlines = COL ? d.Ny : d.Nx;
  const int line = blockIdx.x * P + p;
  const bool valid = line < nlines;
  const cpx<R>* __restrict__ in = reinterpret_cast<const cpx<R>*>(d.in);
  cpx<R>* out = reinterpret_cast<cpx<R>*>(d.out);
  const cpx<R>* __restrict__ tw = reinterpret_cast<const cpx<R>*>(d.tw);

  cpx<R> v[E];
#pragma unroll
  for (int s = 0; s < E; ++s) {
    const int e = t + T_LINE * s;
    const int i = COL ? e : line;
    const int j = COL ? line : e;
    if (!COL && !d.in_tiled && d.pad_in) {
      // zero padding: the caller's array is the region at (in_r0, in_c0)
      const int r = i - d.in_r0, c = j - d.in_c0;
      v[s] = (valid && (unsigned)r < (unsigned)d.in_rows && (unsigned)c < (unsigned)d.in_cols)
                 ? in[(size_t)r * d.in_cols + c]
                 : mk<R>((R)0, (R)0);
    } else {
      v[s] = valid ? in[elem_index(i, j, d.Ny, d.in_tiled)] : mk<R>((R)0, (R)0);
    }
  }

  if (d.t1 != kNone) LineFft<R, L, P>::run(v, sm, t, p, tw, d.t1 == kInv);
  if (d.has_chirp) {
    apply_chirp<R, L, COL>(v, d, t, line, (R)d.scale);
  } else if (d.scale != 1.0) {
    const R scale = (R)d.scale;
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = mk<R>(v[s].x * scale, v[s].y * scale);
  }
  if (d.t2 != kNone) LineFft<R, L, P>::run(v, sm, t, p, tw, d.t2 == kInv);
  if (!COL && !d.out_tiled && d.post_mask && valid) {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = apply_post_mask<R>(d, line, t + T_LINE * s, v[s]);
  }

  // In-place passes: every thread of the CTA must have loaded its inputs before
  // any thread stores (the FFT stages already synchronise when S > 1).
  if (LineFft<R, L, P>::S <= 1 || (d.t1 == kNone && d.t2 == kNone)) __syncthreads();

  if (valid) {
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int e = t + T_LINE * s;
      const int i = COL ? e : line;
      const int j = COL ? line : e;
      if (!COL && !d.out_tiled && d.pad_out) {
        const int r = i - d.out_r0, c = j - d.out_c0;
        if ((unsigned)r < (unsigned)d.out_rows && (unsigned)c < (unsigned)d.out_cols) out[(size_t)r * d.out_cols + c] = v[s];
      } else {
        out[elem_index(i, j, d.Ny, d.out_tiled)] = v[s];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// v3 (FP32): persistent CTAs, one per SM, with TMA.
//   * the NEXT panel streams global -> shared (stg_in) through the Tensor
//     Memory Accelerator while the current one is in registers going through
//     the FFTs: a 1D bulk copy per row / row pair for row passes, a 2D tiled
//     tensor copy (boxes of 2P complex x up to 256 row pairs) for the strided
//     column panels; completion is tracked by an mbarrier with a transaction
//     byte count;
//   * results go registers -> shared (stg_out) -> global by TMA stores, so a
//     column panel's 32-byte sectors leave as a few bulk operations instead of
//     thousands of scattered 8-byte stores.
// Every wait on the mbarrier is bounded: on expiry the CTA sets bit 0 of the
// plan's device status word (d.err) and leaves; nslct_status reports it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }

// 16-byte asynchronous global -> shared copies (used by the batched kernels)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const void* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(map), "r"(x),
               "r"(y), "r"(z), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(map), "r"(x),
               "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// Bounded wait (one thread) for the mbarrier phase with the given parity:
// false once wait_us microseconds (0: one second) have passed on the global
// timer. try_wait may suspend the thread for a while on each call, so the
// bound is on elapsed time, not on the number of calls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned int wait_us) {
  const uint64_t limit = (uint64_t)(wait_us ? wait_us : 1000000u) * 1000ull;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit) return false;
  }
}

template <int L, bool COL, int E_ = kernel_elems(L, true)> struct PShape {
  static constexpr int E = E_;
  static constexpr int T_LINE = L / E;
  // panel of ~8192 complex per CTA (~4096 for 24-element threads) keeps the
  // exchange buffer and the staging buffers within 227 KB of shared memory
  static constexpr int MAXT = E >= 64 ? 128 : (E > 16 ? 256 : (E < 16 ? 1024 : 512));
  static constexpr int P0 = MAXT / T_LINE;
  static constexpr int P = P0 < 2 ? 2 : (P0 > 32 ? 32 : P0);
  static constexpr int THREADS = T_LINE * P;
  static constexpr int XSM = P * (L + (L >> pad_shift(E)));      // exchange buffer entries
  static constexpr int STG = COL ? P * L : P * (L + 8);          // one staging buffer (row-major rows padded)
  // Column panels leave through an output staging buffer and TMA stores; row
  // panels are whole contiguous rows, stored straight from registers. One
  // input buffer each: a second one for row passes (two panels in flight) was
  // measured slower (25.4 vs 26.4 Gsamples/s at 4096^2).
  static constexpr int NIN = 1;
  static constexpr int NSTG = COL ? 2 : 1;
  static constexpr size_t SMEM = (size_t)(XSM + NSTG * STG) * sizeof(float2) + 64;
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
  // TMA boxes start on 128-byte boundaries of shared memory
  static_assert((XSM * sizeof(float2)) % 128 == 0 && (STG * sizeof(float2)) % 128 == 0, "staging alignment");
};

// Row pairs per TMA box of a column panel: all of them up to 256, else a
// divisor of the row-pair count (every supported Nx/2 above 256 is a multiple
// of 128), so the boxes tile the panel exactly.
__host__ __device__ __forceinline__ int col_box_rows(int rows) {
  return rows <= 256 ? rows : (rows % 256 == 0 ? 256 : 128);
}

// staging index of element e of panel line p
template <int L, bool COL, int P>
__device__ __forceinline__ int stg_index(int p, int e, int tiled) {
  if (COL) return (e >> 1) * (2 * P) + (p >> 1) * 4 + (e & 1) * 2 + (p & 1);
  if (tiled) return (p >> 1) * (2 * L) + (e >> 1) * 4 + (p & 1) * 2 + (e & 1);
  return p * (L + 8) + e;
}

// Thread 0: start the copies of one panel into `stg`, arming the mbarrier.
template <int L, bool COL, int P>
__device__ __forceinline__ void tma_load_panel(float2* stg, const float2* in, const CUtensorMap* map,
                                               const PassDesc& d, int panel, uint64_t* bar) {
  const int first = panel * P;
  if (COL) {
    const int rows = d.Nx >> 1;                      // row pairs
    const int box = col_box_rows(rows);
    mbar_arrive_expect_tx(bar, (uint32_t)(rows * 2 * P * sizeof(float2)));
    for (int y0 = 0; y0 < rows; y0 += box) tma_load_2d(stg + y0 * (2 * P), map, 2 * first, y0, bar);
  } else {
    const int valid = min(P, d.Nx - first);
    if (d.in_tiled) {
      mbar_arrive_expect_tx(bar, (uint32_t)((valid >> 1) * 2 * L * sizeof(float2)));
      for (int q = 0; q < (valid >> 1); ++q)
        bulk_load(stg + q * (2 * L), in + (size_t)((first >> 1) + q) * (2 * L), 2 * L * sizeof(float2), bar);
    } else if (!d.pad_in) {
      mbar_arrive_expect_tx(bar, (uint32_t)(valid * L * sizeof(float2)));
      for (int q = 0; q < valid; ++q) bulk_load(stg + q * (L + 8), in + (size_t)(first + q) * L, L * sizeof(float2), bar);
    } else {
      // zero padding: only the caller's rows, copied to the 16-byte boundary
      // at or below the column offset (read back shifted)
      uint32_t bytes = 0;
      for (int q = 0; q < valid; ++q)
        if ((unsigned)(first + q - d.in_r0) < (unsigned)d.in_rows) bytes += d.in_cols * sizeof(float2);
      mbar_arrive_expect_tx(bar, bytes);
      for (int q = 0; q < valid; ++q) {
        const int r = first + q - d.in_r0;
        if ((unsigned)r < (unsigned)d.in_rows)
          bulk_load(stg + q * (L + 8) + (d.in_c0 & ~1), in + (size_t)r * d.in_cols, d.in_cols * sizeof(float2), bar);
      }
    }
  }
}

// Thread 0: send one finished panel from `stg` to global memory.
template <int L, bool COL, int P>
__device__ __forceinline__ void tma_store_panel(const float2* stg, float2* out, const CUtensorMap* map,
                                                const PassDesc& d, int panel) {
  const int first = panel * P;
  if (COL) {
    const int rows = d.Nx >> 1;
    const int box = col_box_rows(rows);
    for (int y0 = 0; y0 < rows; y0 += box) tma_store_2d(map, 2 * first, y0, stg + y0 * (2 * P));
  } else {
    const int valid = min(P, d.Nx - first);
    if (d.out_tiled) {
      for (int q = 0; q < (valid >> 1); ++q)
        bulk_store(out + (size_t)((first >> 1) + q) * (2 * L), stg + q * (2 * L), 2 * L * sizeof(float2));
    } else {
      for (int q = 0; q < valid; ++q) bulk_store(out + (size_t)(first + q) * L, stg + q * (L + 8), L * sizeof(float2));
    }
  }
  bulk_commit();
}

template <int L, bool COL, bool MIXED = false>
__global__ void __launch_bounds__(PShape<L, COL, MIXED ? elems_per_thread(L) : kernel_elems(L, true)>::THREADS, 1)
pass_kernel_tma(PassDesc d, const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_out) {
  using Sh = PShape<L, COL, MIXED ? elems_per_thread(L) : kernel_elems(L, true)>;
  constexpr int E = Sh::E;
  constexpr int T_LINE = Sh::T_LINE;
  constexpr int P = Sh::P;
  // Line-major threads with per-line named barriers were measured slower
  // (18.9 vs 26.4 Gsamples/s at 4096^2): lines stay interleaved per thread.
  constexpr bool LM = false;
  using Fft = typename std::conditional<MIXED, MixedLineFft<L, P, E>, LineFft<float, L, P, E, LM>>::type;
  constexpr int NIN = Sh::NIN;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* xs = reinterpret_cast<float2*>(smem_raw);
  float2* stg_in = xs + Sh::XSM;                     // NIN input buffers of STG entries
  float2* stg_out = stg_in + Sh::STG;                 // column passes: the output buffer
  uint64_t* bar = reinterpret_cast<uint64_t*>(stg_in + Sh::NSTG * Sh::STG);  // one per input buffer
  volatile int& s_ok = *reinterpret_cast<volatile int*>(bar + NIN);

  const int tid = threadIdx.x;
  const int p = LM ? tid / T_LINE : tid % P;
  const int t = LM ? tid % T_LINE : tid / P;
  const int nlines = COL ? d.Ny : d.Nx;
  const int npanels = (nlines + P - 1) / P;
  const float2* in = reinterpret_cast<const float2*>(d.in);
  float2* out = reinterpret_cast<float2*>(d.out);
  const float2* __restrict__ tw = reinterpret_cast<const float2*>(d.tw);
  const float scale = d.fscale;

  if (tid == 0) {
    for (int b = 0; b < NIN; ++b) mbar_init(bar + b, 1);
    mbar_fence_init();
    for (int b = 0; b < NIN; ++b) {
      const int pb = blockIdx.x + b * gridDim.x;
      if (pb < npanels) tma_load_panel<L, COL, P>(stg_in + b * Sh::STG, in, &map_in, d, pb, bar + b);
    }
  }
  __syncthreads();
  int it = 0;
  for (int panel = blockIdx.x; panel < npanels; panel += gridDim.x, ++it) {
    const int line = panel * P + p;
    const bool valid = line < nlines;
    const int b = NIN == 1 ? 0 : (it % NIN);
    const uint32_t parity = (uint32_t)((it / NIN) & 1);
    float2* buf = stg_in + b * Sh::STG;
    if (tid == 0) {
      s_ok = mbar_wait_bounded(bar + b, parity, d.wait_us) ? 1 : 0;
      if (COL) bulk_wait_read_all();  // the previous panel's stores have left stg_out
    }
    __syncthreads();
    if (!s_ok) {
      if (tid == 0) {
        if (d.err) atomicOr(d.err, 1u);
        for (int k = 0; k < NIN; ++k) mbar_wait_bounded(bar + k, (uint32_t)(((it + k) / NIN) & 1), d.wait_us);
        bulk_wait_all();
      }
      return;
    }
    float2 v[E];
    if (COL || d.in_tiled || !d.pad_in) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = buf[stg_index<L, COL, P>(p, t + T_LINE * s, d.in_tiled)];
    } else {
      const bool rv = (unsigned)(line - d.in_r0) < (unsigned)d.in_rows;
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const int e = t + T_LINE * s;
        v[s] = (rv && (unsigned)(e - d.in_c0) < (unsigned)d.in_cols) ? buf[p * (L + 8) + e - (d.in_c0 & 1)]
                                                                       : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();  // this input buffer is consumed
    const int next = panel + NIN * gridDim.x;
    if (tid == 0 && next < npanels) {
      fence_proxy_async();
      tma_load_panel<L, COL, P>(buf, in, &map_in, d, next, bar + b);
    }

    if (d.t1 != kNone) Fft::run(v, xs, t, p, tw, d.t1 == kInv);
    if (d.has_chirp) {
      apply_chirp<float, L, COL, E>(v, d, t, line, scale);
    } else if (d.scale_only) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = make_float2(v[s].x * scale, v[s].y * scale);
    }
    if (d.t2 != kNone) Fft::run(v, xs, t, p, tw, d.t2 == kInv);
    if (d.has_chirp2) {
      apply_chirp_c<float, L, COL, E>(v, d, d.chirp2, d.freq_domain2, t, line, d.fscale2);
    } else if (d.fscale2 != 1.0f) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = make_float2(v[s].x * d.fscale2, v[s].y * d.fscale2);
    }
    if (d.t3 != kNone) Fft::run(v, xs, t, p, tw, d.t3 == kInv);
    if (!COL && !d.out_tiled && d.post_mask) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = apply_post_mask<float>(d, line, t + T_LINE * s, v[s]);
    }

    if constexpr (COL) {
#pragma unroll
      for (int s = 0; s < E; ++s) stg_out[stg_index<L, COL, P>(p, t + T_LINE * s, 1)] = v[s];
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) tma_store_panel<L, COL, P>(stg_out, out, &map_out, d, panel);
    } else if (!d.out_tiled && d.pad_out) {
      const int r = line - d.out_r0;
      if ((unsigned)r < (unsigned)d.out_rows) {
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const int c = t + T_LINE * s - d.out_c0;
          if ((unsigned)c < (unsigned)d.out_cols) out[(size_t)r * d.out_cols + c] = v[s];
        }
      }
    } else if (valid) {
#pragma unroll
      for (int s = 0; s < E; ++s) out[elem_index(line, t + T_LINE * s, d.Ny, d.out_tiled)] = v[s];
    }
  }
  if (COL && tid == 0) bulk_wait_all();
}

// Host: 2D tensor map of the 2x2-tiled field for column panels: rows are row
// pairs (2 Ny complex, 16 Ny bytes apart), the box is 2P complex wide (P/2
// tiles) and up to 256 row pairs tall. Complex64 values are 8-byte elements.
bool encode_column_map(CUtensorMap* map, const void* base, int Nx, int Ny, int P);
// The same as a 3D map over a batch of nbatch fields bstride elements apart
// (the batch index is the third coordinate).
bool encode_column_map_batched(CUtensorMap* map, const void* base, int Nx, int Ny, int P, int nbatch,
                               long long bstride, int box_rows);

// ---------------------------------------------------------------------------
// v4 (FP32, power-of-two lines of 256..4096): line-pair kernel.
//
// A CTA of 256 threads owns G = 256 / (L/16) line PAIRS (a row pair, or a
// column pair: the unit of the 2x2-tiled layout); thread t of a pair holds the
// elements e = t + (L/16) s, s < 16, of BOTH lines. So
//   * every shared-memory exchange of a Stockham stage moves (line0[e], line1[e])
//     as one 16-byte access instead of two 8-byte ones, and each twiddle load
//     serves both lines;
//   * a column pair's TMA box lands as exactly that layout (per row pair the
//     tile holds line0[2r], line1[2r], line0[2r+1], line1[2r+1]), and leaves
//     from it.
// The panel lands by TMA in the exchange buffer itself (no separate staging
// buffer): one CTA needs ~70 KB of shared memory and 128 registers a thread,
// so two CTAs share an SM and overlap each other's loads, stores and barriers.
// Waits are bounded as in v3.
// ---------------------------------------------------------------------------
// (NSLCT_PAIR: see internal.h)
// packed pair kernel, row passes: the next panel's load is issued as soon as
// the last FFT stage has read the buffer (1), or after the panel's work (0).
// (Column passes load the next panel's halves as their TMA stores drain: an
// early load of the lower half measured 1 % slower there.)
#ifndef NSLCT_PAIR_EARLY_LOAD
#define NSLCT_PAIR_EARLY_LOAD 1
#endif
// row passes of the pair kernel: 16-byte tiled loads and stores with a lane-pair shuffle
#ifndef NSLCT_PAIR_SHFL
#define NSLCT_PAIR_SHFL 1
#endif
// column passes of the pair kernel: leave through the buffer by TMA stores (1)
// or by 16-byte stores from registers with the next load issued first (0)
#ifndef NSLCT_PAIR_COL_TMA_STORE
#define NSLCT_PAIR_COL_TMA_STORE 1
#endif
// column passes with TMA stores: the upper half of each column pair leaves from
// the landing buffer, the lower half from a separate 32 KB buffer, so the next
// panel's lower half can be loaded while the stores drain (1), or the whole
// panel leaves from the landing buffer and the next load waits for it (0)
#ifndef NSLCT_PAIR_SPLIT_STORE
#define NSLCT_PAIR_SPLIT_STORE 1
#endif

// Row pairs per TMA box of a pair-kernel column panel: half the panel or less,
// so that the two halves load and store separately.
__host__ __device__ __forceinline__ int pair_box_rows(int rows) {
  if (!NSLCT_PAIR_SPLIT_STORE) return rows <= 256 ? rows : (rows % 256 == 0 ? 256 : 128);
  return rows / 2 < 256 ? rows / 2 : 256;
}

// CTA size of the pair kernel for lines of up to 2048 points: 128 threads, four
// CTAs per SM (256 threads and two CTAs per SM for 4096-point lines, whose pair
// takes 256 threads)
#ifndef NSLCT_PAIR_SMALL_THREADS
#define NSLCT_PAIR_SMALL_THREADS 128
#endif
template <int L> struct PairShape {
  static constexpr int E = 16;
  static constexpr int T = L / E;                 // threads per line pair
  static constexpr int THREADS = L <= 2048 ? NSLCT_PAIR_SMALL_THREADS : 256;
  static constexpr int CTAS = 512 / THREADS;      // per SM (128 registers a thread)
  static constexpr int G = THREADS / T;           // line pairs per CTA
  static constexpr int P = 2 * G;                 // lines per CTA
  static constexpr int SH = pad_shift(E);
  static constexpr int LS = L + (L >> SH);        // float4 entries per pair region (padded)
  static constexpr size_t SMEM = (size_t)G * LS * sizeof(float4) + 64;
  // column passes: the separate output buffer of the lower halves (G L/2 entries)
  static constexpr int OSTG = NSLCT_PAIR_SPLIT_STORE ? G * (L / 2) : 0;
  static constexpr size_t SMEM_COL = SMEM + (size_t)OSTG * sizeof(float4);
  static_assert(is_pow2(L) && L >= 256 && L <= 4096, "pair kernel lengths");
  static_assert(CTAS * (SMEM_COL + 1024) <= 228 * 1024, "CTAS CTAs per SM");
  static_assert((LS * sizeof(float4)) % 128 == 0, "TMA destinations on 128-byte boundaries");
  static_assert(2 * (L + 8) <= 2 * LS, "row landing fits the pair region");
};

// w[r] = w1^r for r = 1 .. RD-1 (w[0] unused), each as w[2^k] * w[r - 2^k] with
// w[2^k] by repeated squaring: at most four roundings deep for RD = 16.

template <int L> struct PairFft {
  using Sh = PairShape<L>;
  static constexpr int E = Sh::E;
  static constexpr int T = Sh::T;
  static constexpr int S = num_stages(L, E);
  static constexpr int SH = Sh::SH;

  static __device__ __forceinline__ int sidx(int g, int e) { return g * Sh::LS + padded_by<SH>(e); }

  template <int ST>
  static __device__ __forceinline__ void stage(float2* v0, float2* v1, float4* sm, int t, int g,
                                               const float2* __restrict__ tw) {
    constexpr int RD = stage_radix(L, E, ST);
    constexpr int NS = stage_ns(L, E, ST);
    constexpr bool FIRST = (ST == 0);
    constexpr bool LAST = (ST == S - 1);
    constexpr int NB = E / RD;
    static_assert(E % RD == 0, "radix must divide E");
    if constexpr (!FIRST) {
      __syncthreads();
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const float4 q = sm[sidx(g, t + T * s)];
        v0[s] = make_float2(q.x, q.y);
        v1[s] = make_float2(q.z, q.w);
      }
      if constexpr (!LAST) __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      float2 x0[RD], x1[RD];
#pragma unroll
      for (int r = 0; r < RD; ++r) {
        x0[r] = v0[u + r * NB];
        x1[r] = v1[u + r * NB];
      }
      const int j = t + u * T;
      const int jm = j % NS;
      if constexpr (NS > 1) {
        // one coalesced load of the base twiddle; its powers in registers
        float2 w[RD];
        twiddle_powers<float, RD>(__ldg(tw + compact_table_offset(L, E, ST) + jm), w);
#pragma unroll
        for (int r = 1; r < RD; ++r) {
          x0[r] = cmul<float>(x0[r], w[r]);
          x1[r] = cmul<float>(x1[r], w[r]);
        }
      }
      Dft<float, RD>::run(x0);
      Dft<float, RD>::run(x1);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < RD; ++r) {
          v0[u + r * NB] = x0[r];
          v1[u + r * NB] = x1[r];
        }
      } else {
        const int base = (j / NS) * NS * RD + jm;
#pragma unroll
        for (int r = 0; r < RD; ++r)
          sm[sidx(g, base + r * NS)] = make_float4(x0[r].x, x0[r].y, x1[r].x, x1[r].y);
      }
    }
  }

  template <int ST>
  static __device__ __forceinline__ void stages(float2* v0, float2* v1, float4* sm, int t, int g,
                                                const float2* __restrict__ tw) {
    if constexpr (ST < S) {
      stage<ST>(v0, v1, sm, t, g, tw);
      stages<ST + 1>(v0, v1, sm, t, g, tw);
    }
  }

  // Unnormalised DFT (or inverse, as conj(DFT(conj x))) of both lines.
  static __device__ __forceinline__ void run(float2* v0, float2* v1, float4* sm, int t, int g,
                                             const float2* __restrict__ tw, bool inverse) {
    if (inverse) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        v0[s].y = -v0[s].y;
        v1[s].y = -v1[s].y;
      }
    }
    __syncthreads();  // the previous user of `sm` is done
    stages<0>(v0, v1, sm, t, g, tw);
    if (inverse) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        v0[s].y = -v0[s].y;
        v1[s].y = -v1[s].y;
      }
    }
  }
};

// packed line-pair FFT: twiddle powers as scalars broadcast to both lanes (1)
// or computed in packed form (0)
#ifndef NSLCT_X2_SCALAR_POWERS
#define NSLCT_X2_SCALAR_POWERS 1
#endif
// The line-pair FFT on packed pairs (pair_x2.cuh): the stages of PairFft with
// each butterfly and twiddle product done once for both lines. Entry e of a
// pair region is (re pair, im pair), 16 bytes as in PairFft. Always the
// forward DFT; an inverse is this code on data held in the J domain.
template <int L> struct X2Fft {
  using Sh = PairShape<L>;
  static constexpr int E = Sh::E;
  static constexpr int T = Sh::T;
  static constexpr int S = num_stages(L, E);
  static constexpr int SH = Sh::SH;

  static __device__ __forceinline__ int sidx(int g, int e) { return g * Sh::LS + padded_by<SH>(e); }

  template <int ST, class Hook>
  static __device__ __forceinline__ void stage(cx2* v, ulonglong2* sm, int t, int g, const float2* __restrict__ tw,
                                               const X2Const& K, const Hook& freed, bool call) {
    constexpr int RD = stage_radix(L, E, ST);
    constexpr int NS = stage_ns(L, E, ST);
    constexpr bool FIRST = (ST == 0);
    constexpr bool LAST = (ST == S - 1);
    constexpr int NB = E / RD;
    static_assert(E % RD == 0, "radix must divide E");
    if constexpr (!FIRST) {
      __syncthreads();
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const ulonglong2 q = sm[sidx(g, t + T * s)];
        v[s] = cx2{q.x, q.y};
      }
      if constexpr (!LAST) {
        __syncthreads();
      } else if (call) {
        __syncthreads();  // every thread has read the buffer for the last time
        freed();
      }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      cx2 x[RD];
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = v[u + r * NB];
      const int j = t + u * T;
      const int jm = j % NS;
      if constexpr (NS > 1) {
        const float2 wb = __ldg(tw + compact_table_offset(L, E, ST) + jm);
        if constexpr (NSLCT_X2_SCALAR_POWERS) x2_twiddle_scalar_powers<RD>(x, wb);
        else x2_twiddle<RD>(x, wb, K);
      }
      X2Dft<RD>::run(x, K);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < RD; ++r) v[u + r * NB] = x[r];
      } else {
        const int base = (j / NS) * NS * RD + jm;
#pragma unroll
        for (int r = 0; r < RD; ++r) sm[sidx(g, base + r * NS)] = make_ulonglong2(x[r].re, x[r].im);
      }
    }
  }

  template <int ST, class Hook>
  static __device__ __forceinline__ void stages(cx2* v, ulonglong2* sm, int t, int g, const float2* __restrict__ tw,
                                                const X2Const& K, const Hook& freed, bool call) {
    if constexpr (ST < S) {
      stage<ST>(v, sm, t, g, tw, K, freed, call);
      stages<ST + 1>(v, sm, t, g, tw, K, freed, call);
    }
  }

  // With `call`, freed() runs in every thread, after a barrier, as soon as the
  // last stage has read the buffer (the caller reuses it, e.g. for the next
  // panel's load, while the last stage computes).
  template <class Hook>
  static __device__ __forceinline__ void run(cx2* v, ulonglong2* sm, int t, int g, const float2* __restrict__ tw,
                                             const Hook& freed, bool call) {
    const X2Const K;
    __syncthreads();  // the previous user of `sm` is done
    stages<0>(v, sm, t, g, tw, K, freed, call);
  }
};

#ifndef NSLCT_X2_HALFWARP
#define NSLCT_X2_HALFWARP 1
#endif
// A pair of 4096-point line-pair FFTs with one CTA-wide exchange each (the
// two transforms of a column pass or of row pass 3). With n = n0 + 16 n1 + 256
// n2 and k = k0 + 16 k1 + 256 k2, nk = 256 n2 k0 + 16 n1 (k0 + 16 k1) + n0 (k0
// + 16 k1 + 256 k2) mod 4096, so the first transform runs
//   A  thread n0 + 16 n1 (natural order): DFT-16 over n2 -> k0;
//   B  thread 16 k0 + n0: twiddle W_256^{n1 k0}, DFT-16 over n1 -> k1;
//   C  thread 16 k0 + k1: twiddle W_4096^{n0 (k0 + 16 k1)}, DFT-16 over n0 -> k2,
// leaving thread t with X[sw(t) + 256 k2], sw(t) = (t >> 4) + 16 (t & 15).
// A -> B is an all-to-all (CTA barriers); B -> C stays inside the half-warp of
// k0, in the very entries that half-warp read in A -> B, so it needs only
// __syncwarp. The second transform is the transpose of the first (the DFT
// matrix is symmetric): from that swapped order back to the natural one, the
// half-warp exchange first and the all-to-all last, each twiddle after its
// DFT. Two CTA barriers per transform instead of four; the twiddle bases are
// the compact table's stage 1 and 2 entries.
struct X2Fft4096H {
  static constexpr int L = 4096;
  static constexpr int E = 16;
  static constexpr int SH = pad_shift(E);
  static __device__ __forceinline__ int sw(int t) { return (t >> 4) + 16 * (t & 15); }
  static __device__ __forceinline__ int px(int p) { return padded_by<SH>(p); }
  static __device__ __forceinline__ float2 w256(const float2* __restrict__ tw, int j) {
    return __ldg(tw + compact_table_offset(L, E, 1) + j);
  }
  static __device__ __forceinline__ float2 w4096(const float2* __restrict__ tw, int j) {
    return __ldg(tw + compact_table_offset(L, E, 2) + j);
  }

  // v: the thread's elements t + 256 s; on return X[sw(t) + 256 s].
  static __device__ __forceinline__ void run_b(cx2* v, ulonglong2* sm, int t, const float2* __restrict__ tw) {
    const X2Const K;
    X2Dft<16>::run(v, K);  // A: over n2
    const int n0 = t & 15, n1 = t >> 4;
    __syncthreads();  // the previous user of `sm` is done
#pragma unroll
    for (int k0 = 0; k0 < 16; ++k0) sm[px(256 * k0 + 16 * n0 + n1)] = make_ulonglong2(v[k0].re, v[k0].im);
    __syncthreads();
    const int k0 = t >> 4, m = t & 15;  // B: this thread is (k0, n0 = m)
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const ulonglong2 q = sm[px(256 * k0 + 16 * m + r)];
      v[r] = cx2{q.x, q.y};
    }
    x2_twiddle_scalar_powers<16>(v, w256(tw, k0));
    X2Dft<16>::run(v, K);
    __syncwarp();  // the half-warp has read its entries; they now take its B -> C exchange
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) sm[px(256 * k0 + 16 * k1 + m)] = make_ulonglong2(v[k1].re, v[k1].im);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) {  // C: this thread is (k0, k1 = m)
      const ulonglong2 q = sm[px(256 * k0 + 16 * m + r)];
      v[r] = cx2{q.x, q.y};
    }
    x2_twiddle_scalar_powers<16>(v, w4096(tw, k0 + 16 * m));
    X2Dft<16>::run(v, K);
  }

  // v: the thread's elements sw(t) + 256 s, the order run_b leaves (its
  // half-warp's entries of `sm` last touched by its own run_b); on return the
  // transform's elements t + 256 s. With `call`, freed() runs in every thread
  // after a barrier once the buffer has been read for the last time.
  template <class Hook>
  static __device__ __forceinline__ void run_t(cx2* v, ulonglong2* sm, int t, const float2* __restrict__ tw,
                                               const Hook& freed, bool call) {
    const X2Const K;
    const int k0 = t >> 4, m = t & 15;  // C^T: this thread is (k0, k1 = m)
    X2Dft<16>::run(v, K);                // over k2 -> n0
    x2_twiddle_scalar_powers<16>(v, w4096(tw, k0 + 16 * m));
    __syncwarp();
#pragma unroll
    for (int n0 = 0; n0 < 16; ++n0) sm[px(256 * k0 + 16 * n0 + m)] = make_ulonglong2(v[n0].re, v[n0].im);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) {  // B^T: this thread is (k0, n0 = m)
      const ulonglong2 q = sm[px(256 * k0 + 16 * m + r)];
      v[r] = cx2{q.x, q.y};
    }
    X2Dft<16>::run(v, K);  // over k1 -> n1
    x2_twiddle_scalar_powers<16>(v, w256(tw, k0));
    __syncthreads();  // every half-warp has read its entries
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) sm[px(256 * n1 + 16 * m + k0)] = make_ulonglong2(v[n1].re, v[n1].im);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) {  // A^T: this thread is (n0, n1) = (t & 15, t >> 4)
      const ulonglong2 q = sm[px(16 * t + r)];
      v[r] = cx2{q.x, q.y};
    }
    if (call) {
      __syncthreads();  // every thread has read the buffer for the last time
      freed();
    }
    X2Dft<16>::run(v, K);  // over k0 -> n2
  }
};

// One step of a packed pass program on the thread's E positions of lines
// line0 and line0 + 1: multiply by the chirp (its phases exactly as in
// apply_chirp_c, one Q0.64 phase per line) times scale, or by scale alone.
// conj: the data is held in the J domain, so the chirp is conjugated. SWAP:
// the results go to the other parts (the step also switches domain); a swap
// with no step is a multiply by one.
template <int L, int E, bool COL, bool SWAP>
__device__ __forceinline__ void x2_step_e(cx2* v, const X2Step& st, bool conj, const PassDesc& d, int t, int line0) {
  constexpr int T = L / E;
  if (st.kind == 1) {
    const int nl = COL ? d.Ny : d.Nx;  // length of the other axis
    const uint64_t ka = COL ? st.c.k11 : st.c.k22;
    const uint64_t kb = COL ? st.c.k22 : st.c.k11;
    const long long a0 = st.freq ? (long long)t : (long long)t - L / 2;
    const uint64_t dd = 2ull * ka * (uint64_t)((long long)T * T);
    uint64_t q[2], dq[2], kab[2], base[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long b = st.freq ? (long long)centred_bin(line0 + h, nl) : (long long)(line0 + h) - nl / 2;
      kab[h] = st.c.k12 * (uint64_t)b;
      base[h] = kb * (uint64_t)(b * b);
      q[h] = ka * (uint64_t)(a0 * a0) + kab[h] * (uint64_t)a0 + base[h];
      dq[h] = ka * (uint64_t)(2 * a0 * T + (long long)T * T) + kab[h] * (uint64_t)T;
    }
    const float sc = st.scale, ssc = conj ? -st.scale : st.scale;
#pragma unroll
    for (int s = 0; s < E; ++s) {
      if (s == E / 2 && st.freq) {
        // centred bins: the second half of the line holds the negative bins
        const long long a = a0 + (long long)T * s - L;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          q[h] = ka * (uint64_t)(a * a) + kab[h] * (uint64_t)a + base[h];
          dq[h] = ka * (uint64_t)(2 * a * T + (long long)T * T) + kab[h] * (uint64_t)T;
        }
      }
      float sn[2], cs[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        // top 32 bits as a signed fraction of a turn in [-1/2, 1/2)
        const float tt = (float)(int)(unsigned)(q[h] >> 32) * 2.3283064365386963e-10f;  // 2^-32
        __sincosf(6.28318530717958647692f * tt, &sn[h], &cs[h]);
        q[h] += dq[h];
        dq[h] += dd;
      }
      // scaled (and for conj negated) sine per line; its negation by an integer XOR
      const float s0 = sn[0] * ssc, s1 = sn[1] * ssc;
      const f32x2 cc = x2_pack(cs[0] * sc, cs[1] * sc);
      const f32x2 ss = x2_pack(s0, s1);
      const f32x2 nss = x2_pack(__int_as_float(__float_as_int(s0) ^ 0x80000000),
                                __int_as_float(__float_as_int(s1) ^ 0x80000000));
      const f32x2 re = x2_fma(v[s].re, cc, x2_mul(v[s].im, nss));
      const f32x2 im = x2_fma(v[s].re, ss, x2_mul(v[s].im, cc));
      v[s] = SWAP ? cx2{im, re} : cx2{re, im};
    }
  } else if (SWAP || st.kind == 2) {
    const f32x2 sc = x2_bcast(st.kind == 2 ? st.scale : 1.0f);
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const f32x2 re = x2_mul(v[s].re, sc), im = x2_mul(v[s].im, sc);
      v[s] = SWAP ? cx2{im, re} : cx2{re, im};
    }
  }
}

// x2_step with the line-pair kernel's elements per thread
template <int L, bool COL, bool SWAP>
__device__ __forceinline__ void x2_step(cx2* v, const X2Step& st, bool conj, const PassDesc& d, int t, int line0) {
  x2_step_e<L, PairShape<L>::E, COL, SWAP>(v, st, conj, d, t, line0);
}

// Thread 0: copies of one panel (G line pairs from line `first`) into the
// pair regions of `x`, arming the mbarrier. Column pairs: one 2D box column
// (4 complex wide) per pair; row pairs: one or two 1D bulk copies per pair.
// half (column panels): 0 = the whole panel; 1 = arm the barrier for the
// whole panel and load the lower row pairs; 2 = load the upper row pairs.
template <int L, bool COL>
__device__ __forceinline__ void pair_load_panel(float4* x, const float2* in, const CUtensorMap* map,
                                                const PassDesc& d, int first, uint64_t* bar, int b, int half = 0) {
  using Sh = PairShape<L>;
  const int nlines = COL ? d.Ny : d.Nx;
  const int pairs = min(Sh::G, (nlines - first) >> 1);
  if (COL) {
    const int rows = d.Nx >> 1;
    const int box = pair_box_rows(rows);
    if (half != 2) mbar_arrive_expect_tx(bar, (uint32_t)(pairs * rows * 4 * sizeof(float2)) + d.test_extra_tx);
    const int r0 = half == 2 ? rows / 2 : 0, r1 = half == 1 ? rows / 2 : rows;
    for (int g = 0; g < pairs; ++g)
      for (int y0 = r0; y0 < r1; y0 += box)
        tma_load_3d(reinterpret_cast<float2*>(x + g * Sh::LS) + y0 * 4, map, 2 * (first + 2 * g), y0, b, bar);
  } else if (d.in_tiled) {
    mbar_arrive_expect_tx(bar, (uint32_t)(pairs * 2 * L * sizeof(float2)) + d.test_extra_tx);
    for (int g = 0; g < pairs; ++g)
      bulk_load(x + g * Sh::LS, in + (size_t)((first >> 1) + g) * (2 * L), 2 * L * sizeof(float2), bar);
  } else if (!d.pad_in) {
    mbar_arrive_expect_tx(bar, (uint32_t)(pairs * 2 * L * sizeof(float2)) + d.test_extra_tx);
    for (int g = 0; g < pairs; ++g)
      for (int h = 0; h < 2; ++h)
        bulk_load(reinterpret_cast<float2*>(x + g * Sh::LS) + h * (L + 8), in + (size_t)(first + 2 * g + h) * L,
                  L * sizeof(float2), bar);
  } else {
    // zero padding: only the caller's rows, each copied to the 16-byte
    // boundary at or below its column offset (read back shifted)
    uint32_t bytes = 0;
    for (int g = 0; g < pairs; ++g)
      for (int h = 0; h < 2; ++h)
        if ((unsigned)(first + 2 * g + h - d.in_r0) < (unsigned)d.in_rows) bytes += d.in_cols * sizeof(float2);
    mbar_arrive_expect_tx(bar, bytes + d.test_extra_tx);
    for (int g = 0; g < pairs; ++g)
      for (int h = 0; h < 2; ++h) {
        const int r = first + 2 * g + h - d.in_r0;
        if ((unsigned)r < (unsigned)d.in_rows)
          bulk_load(reinterpret_cast<float2*>(x + g * Sh::LS) + h * (L + 8) + (d.in_c0 & ~1),
                    in + (size_t)r * d.in_cols, d.in_cols * sizeof(float2), bar);
      }
  }
}

// MODE 0: scalar arithmetic, any sequence of transforms. MODE 1..4: packed
// FP32x2 (pair_x2.cuh) running the pass program d.x2, whose first and last
// transforms are (1) forward, forward, (2) inverse, forward, (3) inverse,
// inverse, (4) forward, inverse; MODE 5 is mode 1 for programs of more than
// one transform (4096-point rows: their first two run as X2Fft4096H's pair).
template <int L, bool COL, int MODE = 0>
__global__ void __launch_bounds__(PairShape<L>::THREADS, PairShape<L>::CTAS)
pass_kernel_pair(PassDesc d, const __grid_constant__ CUtensorMap map_in, const __grid_constant__ CUtensorMap map_out) {
  using Sh = PairShape<L>;
  using Fft = PairFft<L>;
  constexpr int E = Sh::E;
  constexpr int T = Sh::T;
  constexpr int P = Sh::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4* xs = reinterpret_cast<float4*>(smem_raw);
  // the mbarrier after the exchange buffer (and, for column passes, after the
  // output buffer of the lower halves)
  uint64_t* bar = reinterpret_cast<uint64_t*>(xs + Sh::G * Sh::LS + (COL ? Sh::OSTG : 0));
  volatile int& s_ok = *reinterpret_cast<volatile int*>(bar + 1);

  const int tid = threadIdx.x;
  const int g = tid / T;
  const int t = tid % T;
  const int nlines = COL ? d.Ny : d.Nx;
  const int npf = (nlines + P - 1) / P;                 // panels per field
  const int nb = d.nbatch > 1 ? d.nbatch : 1;
  const int npanels = npf * nb;                          // over the whole batch
  const float2* in0 = reinterpret_cast<const float2*>(d.in);
  float2* out0 = reinterpret_cast<float2*>(d.out);
  const float2* __restrict__ tw = reinterpret_cast<const float2*>(d.tw);
  float4* xg = xs + g * Sh::LS;                 // this thread's pair region
  float2* xg2 = reinterpret_cast<float2*>(xg);

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
    if ((int)blockIdx.x < npanels) {
      const int b0 = blockIdx.x / npf;
      pair_load_panel<L, COL>(xs, in0 + b0 * d.in_bstride, &map_in, d, (blockIdx.x % npf) * P, bar, b0);
    }
  }
  __syncthreads();
  int it = 0;
  for (int gp = blockIdx.x; gp < npanels; gp += gridDim.x, ++it) {
    const int bf = gp / npf;                             // field of the batch
    const int panel = gp % npf;
    const float2* in = in0 + bf * d.in_bstride;
    float2* out = out0 + bf * d.out_bstride;
    const int first = panel * P;
    const int line0 = first + 2 * g;
    const bool valid = line0 < nlines;          // lines come in pairs (even counts)
    if (tid == 0) s_ok = mbar_wait_bounded(bar, (uint32_t)(it & 1), d.wait_us) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {
      if (tid == 0) {
        if (d.err) atomicOr(d.err, 1u);
        // every copy of this panel was issued before the wait: give them one
        // more bounded wait to land before the shared memory is released,
        // then drain the stores
        mbar_wait_bounded(bar, (uint32_t)(it & 1), d.wait_us);
        bulk_wait_all();
      }
      return;
    }
    const int next = gp + gridDim.x;
    const int nbf = next / npf;                          // the next panel's field
    // thread 0 issues the next panel's copies into the freed buffer (row
    // passes of the packed kernel: as soon as the last FFT stage has read it)
    constexpr bool EARLY = MODE != 0 && NSLCT_PAIR_EARLY_LOAD && !COL;
    auto load_next = [&]() {
      if (tid == 0 && next < npanels) {
        fence_proxy_async();
        pair_load_panel<L, COL>(xs, in0 + nbf * d.in_bstride, &map_in, d, (next % npf) * P, bar, nbf);
      }
    };
    float2 v0[E], v1[E];
    int eb = t;            // the thread's elements are eb + T s
    bool swapped = false;  // eb = X2Fft4096H::sw(t), between the two transforms of a pair
    if (COL) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const float4 q = xg[t + T * s];
        v0[s] = make_float2(q.x, q.y);
        v1[s] = make_float2(q.z, q.w);
      }
    } else if (d.in_tiled) {
      if constexpr (NSLCT_PAIR_SHFL) {
        // float4 e of a tiled row pair is (line0[e], line0[e+1]) for even e and
        // (line1[e-1], line1[e]) for odd e: one 16-byte load per lane, then
        // lanes e and e^1 swap the half the other one needs
        const bool odd = (t & 1) != 0;
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const float4 q = xg[t + T * s];
          const float2 mine = odd ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
          const float2 give = odd ? make_float2(q.x, q.y) : make_float2(q.z, q.w);
          const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, give.x, 1), __shfl_xor_sync(0xffffffffu, give.y, 1));
          v0[s] = odd ? got : mine;
          v1[s] = odd ? mine : got;
        }
      } else {
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const int e = t + T * s;
          v0[s] = xg2[(e >> 1) * 4 + (e & 1)];
          v1[s] = xg2[(e >> 1) * 4 + 2 + (e & 1)];
        }
      }
    } else if (!d.pad_in) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        v0[s] = xg2[t + T * s];
        v1[s] = xg2[(L + 8) + t + T * s];
      }
    } else {
      const bool r0 = (unsigned)(line0 - d.in_r0) < (unsigned)d.in_rows;
      const bool r1 = (unsigned)(line0 + 1 - d.in_r0) < (unsigned)d.in_rows;
      const int shift = d.in_c0 & 1;
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const int e = t + T * s;
        const bool c = (unsigned)(e - d.in_c0) < (unsigned)d.in_cols;
        v0[s] = (c && r0) ? xg2[e - shift] : make_float2(0.f, 0.f);
        v1[s] = (c && r1) ? xg2[(L + 8) + e - shift] : make_float2(0.f, 0.f);
      }
    }

    if constexpr (MODE == 0) {
      const float scale = d.fscale;
      if (d.t1 != kNone) Fft::run(v0, v1, xs, t, g, tw, d.t1 == kInv);
      if (d.has_chirp) {
        apply_chirp_c<float, L, COL, E>(v0, d, d.chirp, d.freq_domain, t, line0, scale);
        apply_chirp_c<float, L, COL, E>(v1, d, d.chirp, d.freq_domain, t, line0 + 1, scale);
      } else if (d.scale_only) {
#pragma unroll
        for (int s = 0; s < E; ++s) {
          v0[s] = make_float2(v0[s].x * scale, v0[s].y * scale);
          v1[s] = make_float2(v1[s].x * scale, v1[s].y * scale);
        }
      }
      if (d.t2 != kNone) Fft::run(v0, v1, xs, t, g, tw, d.t2 == kInv);
      if (d.has_chirp2) {
        apply_chirp_c<float, L, COL, E>(v0, d, d.chirp2, d.freq_domain2, t, line0, d.fscale2);
        apply_chirp_c<float, L, COL, E>(v1, d, d.chirp2, d.freq_domain2, t, line0 + 1, d.fscale2);
      } else if (d.fscale2 != 1.0f) {
#pragma unroll
        for (int s = 0; s < E; ++s) {
          v0[s] = make_float2(v0[s].x * d.fscale2, v0[s].y * d.fscale2);
          v1[s] = make_float2(v1[s].x * d.fscale2, v1[s].y * d.fscale2);
        }
      }
      if (d.t3 != kNone) Fft::run(v0, v1, xs, t, g, tw, d.t3 == kInv);
    } else {
      // packed pass program: load in the domain of the first transform (J
      // for an inverse: the parts swapped), one forward-FFT body for every
      // transform, each gap's step switching domain, store from the domain
      // of the last transform
      constexpr bool FINV = MODE == 2 || MODE == 3;
      constexpr bool LINV = MODE == 3 || MODE == 4;
      cx2 v[E];
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const f32x2 re = x2_pack(v0[s].x, v1[s].x), im = x2_pack(v0[s].y, v1[s].y);
        v[s] = FINV ? cx2{im, re} : cx2{re, im};
      }
      if (d.x2.pre.kind) x2_step<L, COL, false>(v, d.x2.pre, FINV, d, eb, line0);
      ulonglong2* xs2 = reinterpret_cast<ulonglong2*>(xs);
#pragma unroll 1
      for (int k = 0; k < d.x2.ntr; ++k) {
        if (k > 0) {
          // the gap after transform k-1, whose domain is J when it was an inverse
          const X2Step st = k == 1 ? d.x2.gap[0] : d.x2.gap[1];
          x2_step<L, COL, true>(v, st, FINV != (((k - 1) & 1) != 0), d, eb, line0);
        }
        const bool early = EARLY && k == d.x2.ntr - 1;
        if constexpr (L == 4096 && NSLCT_X2_HALFWARP && !COL && (MODE == 2 || MODE == 5)) {
          // row passes of two or more transforms (mode 2, and mode 5: mode 1's
          // program with more than one transform): X2Fft4096H's pair (natural
          // -> swapped -> natural); a lone one, or the third of three: the
          // Stockham FFT. (Measured: row pass 3 at 4096^2 89.0 against 92.4 us;
          // the column pass's pair gained nothing, 95.9 against 95.5 us, and
          // compiling the pair into the one-transform passes' kernels slowed
          // them by 3-4 us, hence the separate mode 5.)
          if (swapped) {
            X2Fft4096H::run_t(v, xs2, t, tw, load_next, early);
            eb = t;
            swapped = false;
          } else if (k + 1 < d.x2.ntr) {
            X2Fft4096H::run_b(v, xs2, t, tw);
            eb = X2Fft4096H::sw(t);
            swapped = true;
          } else {
            X2Fft<L>::run(v, xs2, t, g, tw, load_next, early);
          }
        } else {
          X2Fft<L>::run(v, xs2, t, g, tw, load_next, early);
        }
      }
      if (d.x2.post[0].kind) x2_step<L, COL, false>(v, d.x2.post[0], LINV, d, eb, line0);
      if (d.x2.post[1].kind) x2_step<L, COL, false>(v, d.x2.post[1], LINV, d, eb, line0);
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const cx2 w = LINV ? cx2{v[s].im, v[s].re} : v[s];
        x2_unpack(w.re, v0[s].x, v1[s].x);
        x2_unpack(w.im, v0[s].y, v1[s].y);
      }
    }
    if (!COL && !d.out_tiled && d.post_mask) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        v0[s] = apply_post_mask<float>(d, line0, eb + T * s, v0[s]);
        v1[s] = apply_post_mask<float>(d, line0 + 1, eb + T * s, v1[s]);
      }
    }
    if constexpr (!EARLY) __syncthreads();  // every thread has finished reading the buffer

    if constexpr (COL && !NSLCT_PAIR_COL_TMA_STORE) {
      // next panel's load first (already issued when EARLY), then 16-byte
      // stores of (line0[e], line1[e]), one tile row of the column pair each
      if constexpr (!EARLY) load_next();
      if (valid) {
        float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const int e = eb + T * s;
          o4[((size_t)(e >> 1) * (2 * d.Ny) + (line0 >> 1) * 4 + (e & 1) * 2) >> 1] =
              make_float4(v0[s].x, v0[s].y, v1[s].x, v1[s].y);
        }
      }
    } else if constexpr (COL && NSLCT_PAIR_SPLIT_STORE) {
      // lower half (e < L/2) to the separate buffer, upper half stays in place;
      // the next panel's lower half is loaded while both halves are stored
      float4* ostg = xs + Sh::G * Sh::LS;
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const int e = eb + T * s;
        const float4 q = make_float4(v0[s].x, v0[s].y, v1[s].x, v1[s].y);
        if (e < L / 2) ostg[g * (L / 2) + e] = q;
        else xg[e] = q;
      }
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        const int pairs = min(Sh::G, (nlines - first) >> 1);
        const int rows = d.Nx >> 1;
        const int box = pair_box_rows(rows);
        for (int q = 0; q < pairs; ++q) {
          for (int y0 = 0; y0 < rows / 2; y0 += box)
            tma_store_3d(&map_out, 2 * (first + 2 * q), y0, bf, reinterpret_cast<float2*>(ostg + q * (L / 2)) + y0 * 4);
          for (int y0 = rows / 2; y0 < rows; y0 += box)
            tma_store_3d(&map_out, 2 * (first + 2 * q), y0, bf, reinterpret_cast<float2*>(xs + q * Sh::LS) + y0 * 4);
        }
        bulk_commit();
        if (next < npanels)
          pair_load_panel<L, COL>(xs, in0 + nbf * d.in_bstride, &map_in, d, (next % npf) * P, bar, nbf, 1);
        bulk_wait_read_all();  // both output halves have left shared memory
        if (next < npanels)
          pair_load_panel<L, COL>(xs, in0 + nbf * d.in_bstride, &map_in, d, (next % npf) * P, bar, nbf, 2);
      }
    } else if constexpr (COL) {
      // leave through the buffer: the box layout is (line0[e], line1[e]) per e
#pragma unroll
      for (int s = 0; s < E; ++s)
        xg[eb + T * s] = make_float4(v0[s].x, v0[s].y, v1[s].x, v1[s].y);
      fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        const int pairs = min(Sh::G, (nlines - first) >> 1);
        const int rows = d.Nx >> 1;
        const int box = pair_box_rows(rows);
        for (int q = 0; q < pairs; ++q)
          for (int y0 = 0; y0 < rows; y0 += box)
            tma_store_3d(&map_out, 2 * (first + 2 * q), y0, bf, reinterpret_cast<float2*>(xs + q * Sh::LS) + y0 * 4);
        bulk_commit();
        bulk_wait_read_all();  // the buffer is free again
        if (next < npanels)
          pair_load_panel<L, COL>(xs, in0 + nbf * d.in_bstride, &map_in, d, (next % npf) * P, bar, nbf);
      }
    } else {
      if constexpr (!EARLY) load_next();
      if (!d.out_tiled && d.pad_out) {
        // zero padding: store the output region alone
        const int r = line0 - d.out_r0;
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const int c = eb + T * s - d.out_c0;
          if ((unsigned)c < (unsigned)d.out_cols) {
            if ((unsigned)r < (unsigned)d.out_rows) out[(size_t)r * d.out_cols + c] = v0[s];
            if ((unsigned)(r + 1) < (unsigned)d.out_rows) out[(size_t)(r + 1) * d.out_cols + c] = v1[s];
          }
        }
      } else if constexpr (NSLCT_PAIR_SHFL) {
        // lanes e (even) and e^1 swap halves so that each lane stores one
        // 16-byte vector: tiled, float4 e; row-major, (line0[e], line0[e+1])
        // from the even lane and (line1[e-1], line1[e]) from the odd one
        // (every lane shuffles: with 16 threads per pair a warp can straddle
        // a valid and an invalid pair)
        // (the neighbouring element's thread: lane ^ 1, or lane ^ 16 in the
        // swapped order of X2Fft4096H)
        const bool odd = (eb & 1) != 0;
        const int pm = swapped ? 16 : 1;
        float4* o4 = reinterpret_cast<float4*>(d.out_tiled ? out + (size_t)(line0 >> 1) * (2 * L)
                                                           : out + (size_t)line0 * L);
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const int e = eb + T * s;
          const float2 give = odd ? v0[s] : v1[s];
          const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, give.x, pm), __shfl_xor_sync(0xffffffffu, give.y, pm));
          const float4 q = odd ? make_float4(got.x, got.y, v1[s].x, v1[s].y) : make_float4(v0[s].x, v0[s].y, got.x, got.y);
          if (valid) o4[d.out_tiled ? e : (odd ? (L + e - 1) / 2 : e / 2)] = q;
        }
      } else if (valid) {
        if (d.out_tiled) {
          float2* o = out + (size_t)(line0 >> 1) * (2 * L);
#pragma unroll
          for (int s = 0; s < E; ++s) {
            const int e = eb + T * s;
            o[(e >> 1) * 4 + (e & 1)] = v0[s];
            o[(e >> 1) * 4 + 2 + (e & 1)] = v1[s];
          }
        } else {
          float2* o = out + (size_t)line0 * L;
#pragma unroll
          for (int s = 0; s < E; ++s) {
            o[eb + T * s] = v0[s];
            o[L + eb + T * s] = v1[s];
          }
        }
      }
    }
  }
  if (COL && tid == 0) bulk_wait_all();
}


// Pass program of the packed line-pair kernel from the generic descriptor
// fields: the sequence t1, step 1, t2, step 2, t3 with absent parts skipped
// (step 1 is the chirp or the lone scale, step 2 chirp2 or fscale2). Returns
// the kernel mode 1..4 (see pass_kernel_pair) or 0 when the transforms do not
// alternate in direction, two steps share a gap, or there is no transform.
inline int x2_program(const PassDesc& d, X2Prog& pg) {
  X2Step st[2] = {};
  if (d.has_chirp) st[0] = X2Step{1, d.freq_domain, d.fscale, d.chirp};
  else if (d.scale_only) st[0] = X2Step{2, 0, d.fscale, Chirp{}};
  if (d.has_chirp2) st[1] = X2Step{1, d.freq_domain2, d.fscale2, d.chirp2};
  else if (d.fscale2 != 1.0f) st[1] = X2Step{2, 0, d.fscale2, Chirp{}};
  const int tr[3] = {d.t1, d.t2, d.t3};
  pg = X2Prog{};
  int dirs[3] = {}, n = 0, npend = 0;
  X2Step pend[2] = {};
  for (int k = 0; k < 3; ++k) {
    if (tr[k] != kNone) {
      if (npend > 1) return 0;
      if (n == 0) {
        if (npend) pg.pre = pend[0];
      } else {
        pg.gap[n - 1] = npend ? pend[0] : X2Step{};
      }
      dirs[n++] = tr[k];
      npend = 0;
    }
    if (k < 2 && st[k].kind) pend[npend++] = st[k];
  }
  if (n == 0) return 0;
  for (int i = 1; i < n; ++i)
    if (dirs[i] == dirs[i - 1]) return 0;
  for (int i = 0; i < npend; ++i) pg.post[i] = pend[i];
  pg.ntr = n;
  const bool fi = dirs[0] == kInv, li = dirs[n - 1] == kInv;
  return !fi && !li ? 1 : fi && !li ? 2 : fi && li ? 3 : 4;
}

// packed line-pair kernel modes built: rows (1) F..F, (2) I..F, (3) I..I;
// columns (4) F..I; 0 builds the scalar kernel instead
#ifndef NSLCT_PAIR_X2
#define NSLCT_PAIR_X2 1
#endif
template <bool COL>
inline bool pair_mode_built(int mode) {
  if (!NSLCT_PAIR_X2) return mode == 0;
  return COL ? mode == 4 : (mode >= 1 && mode <= 3);
}

template <int L, bool COL, int MODE>
inline void launch_pair(const PassDesc& d, const CUtensorMap& mi, const CUtensorMap& mo, int blocks, cudaStream_t s) {
  using Sh = PairShape<L>;
  pass_kernel_pair<L, COL, MODE><<<blocks, Sh::THREADS, COL ? Sh::SMEM_COL : Sh::SMEM, s>>>(d, mi, mo);
}

template <typename R, int L, bool COL>
inline int launch_one(const PassDesc& d, cudaStream_t s) {
  const int nlines = COL ? d.Ny : d.Nx;
  if constexpr (sizeof(R) == 4) {
    alignas(64) CUtensorMap mi{}, mo{};
    if constexpr (is_pow2(L) && L >= 256) {
      if (d.mixed) {
        using Sh = PShape<L, COL, elems_per_thread(L)>;
        const int npanels = (nlines + Sh::P - 1) / Sh::P;
        const int blocks = npanels < d.num_sms ? npanels : d.num_sms;
        if (COL && (!encode_column_map(&mi, d.in, d.Nx, d.Ny, Sh::P) ||
                    !encode_column_map(&mo, d.out, d.Nx, d.Ny, Sh::P)))
          return NSLCT_E_CUDA;
        pass_kernel_tma<L, COL, true><<<blocks, Sh::THREADS, Sh::SMEM, s>>>(d, mi, mo);
        return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
      }
    }
    using ShT = PShape<L, COL>;
    // the general FP32 kernel, one field
    auto launch_tma = [&](const PassDesc& e) -> int {
      const int npanels = (nlines + ShT::P - 1) / ShT::P;
      const int blocks = npanels < e.num_sms ? npanels : e.num_sms;
      if (COL && (!encode_column_map(&mi, e.in, e.Nx, e.Ny, ShT::P) ||
                  !encode_column_map(&mo, e.out, e.Nx, e.Ny, ShT::P)))
        return NSLCT_E_CUDA;
      pass_kernel_tma<L, COL><<<blocks, ShT::THREADS, ShT::SMEM, s>>>(e, mi, mo);
      return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
    };
    if constexpr (NSLCT_PAIR && is_pow2(L) && L >= 256) {
      using Sh = PairShape<L>;
      const int nb = d.nbatch > 1 ? d.nbatch : 1;
      PassDesc dx = d;
      const int mode = NSLCT_PAIR_X2 ? x2_program(d, dx.x2) : 0;
      if (pair_mode_built<COL>(mode)) {
        const long long npanels = (long long)((nlines + Sh::P - 1) / Sh::P) * nb;
        const int blocks = npanels < Sh::CTAS * d.num_sms ? (int)npanels : Sh::CTAS * d.num_sms;
        const int box = pair_box_rows(d.Nx / 2);
        if (COL && (!encode_column_map_batched(&mi, d.in, d.Nx, d.Ny, 2, nb, d.in_bstride, box) ||
                    !encode_column_map_batched(&mo, d.out, d.Nx, d.Ny, 2, nb, d.out_bstride, box)))
          return NSLCT_E_CUDA;
        if constexpr (!NSLCT_PAIR_X2) launch_pair<L, COL, 0>(dx, mi, mo, blocks, s);
        else if constexpr (COL) launch_pair<L, true, 4>(dx, mi, mo, blocks, s);
        else if (mode == 1) {
          if constexpr (L == 4096 && NSLCT_X2_HALFWARP) {
            if (dx.x2.ntr > 1) launch_pair<L, false, 5>(dx, mi, mo, blocks, s);
            else launch_pair<L, false, 1>(dx, mi, mo, blocks, s);
          } else {
            launch_pair<L, false, 1>(dx, mi, mo, blocks, s);
          }
        }
        else if (mode == 2) launch_pair<L, false, 2>(dx, mi, mo, blocks, s);
        else launch_pair<L, false, 3>(dx, mi, mo, blocks, s);
        return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
      }
      // a pass program the packed kernel is not built for: the general
      // kernel, one launch per field of the batch
      for (int b = 0; b < nb; ++b) {
        PassDesc e = d;
        e.nbatch = 1;
        e.in = static_cast<const float2*>(d.in) + b * d.in_bstride;
        e.out = static_cast<float2*>(d.out) + b * d.out_bstride;
        const int rc = launch_tma(e);
        if (rc != NSLCT_OK) return rc;
      }
      return NSLCT_OK;
    }
    return launch_tma(d);
  } else {
    using Sh = PassShape<R, L>;
    const int blocks = (nlines + Sh::P - 1) / Sh::P;
    pass_kernel<R, L, COL><<<blocks, Sh::THREADS, Sh::SMEM, s>>>(d);
  }
  return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
}

template <int L, bool COL, int MODE>
inline cudaError_t prepare_pair() {
  using Sh = PairShape<L>;
  return cudaFuncSetAttribute(pass_kernel_pair<L, COL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(COL ? Sh::SMEM_COL : Sh::SMEM));
}

template <typename R, int L>
inline int prepare_one() {
  cudaError_t e1, e2;
  if constexpr (sizeof(R) == 4) {
    e1 = cudaFuncSetAttribute(pass_kernel_tma<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PShape<L, false>::SMEM);
    e2 = cudaFuncSetAttribute(pass_kernel_tma<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PShape<L, true>::SMEM);
    if constexpr (NSLCT_PAIR && is_pow2(L) && L >= 256) {
      if constexpr (NSLCT_PAIR_X2) {
        if (e1 == cudaSuccess) e1 = prepare_pair<L, false, 1>();
        if constexpr (L == 4096 && NSLCT_X2_HALFWARP)
          if (e1 == cudaSuccess) e1 = prepare_pair<L, false, 5>();
        if (e1 == cudaSuccess) e1 = prepare_pair<L, false, 2>();
        if (e1 == cudaSuccess) e1 = prepare_pair<L, false, 3>();
        if (e2 == cudaSuccess) e2 = prepare_pair<L, true, 4>();
      } else {
        if (e1 == cudaSuccess) e1 = prepare_pair<L, false, 0>();
        if (e2 == cudaSuccess) e2 = prepare_pair<L, true, 0>();
      }
    }
    if constexpr (is_pow2(L) && L >= 256) {
      if (e1 == cudaSuccess)
        e1 = cudaFuncSetAttribute(pass_kernel_tma<L, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)PShape<L, false, elems_per_thread(L)>::SMEM);
      if (e2 == cudaSuccess)
        e2 = cudaFuncSetAttribute(pass_kernel_tma<L, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)PShape<L, true, elems_per_thread(L)>::SMEM);
    }
  } else {
    using Sh = PassShape<R, L>;
    e1 = cudaFuncSetAttribute(pass_kernel<R, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    e2 = cudaFuncSetAttribute(pass_kernel<R, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  }
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? NSLCT_OK : NSLCT_E_CUDA;
}

}  // namespace nslct

namespace nslct {

// The adjoint's two paths through one packed FFT (pair_x2.cuh): lane 0 holds a
// line of the gradient path, lane 1 the same line of the value path, P lines
// interleaved thread by thread as in LineFft2. Twiddles come from the full
// table (correctly rounded, as in LineFft2), broadcast to both lanes.
#ifndef NSLCT_DUAL_X2
#define NSLCT_DUAL_X2 1
#endif
// EXACT: every twiddle from the full table (the adjoint); otherwise one base
// twiddle from the compact table and its powers formed as scalars (batches).
template <int L, int P, int E_, bool EXACT = true>
struct LineFftX2 {
  static constexpr int E = E_;
  static constexpr int T_LINE = L / E;
  static constexpr int S = num_stages(L, E);
  static constexpr int SH = pad_shift(E);
  static __device__ __forceinline__ int sidx(int p, int e) { return padded_by<SH>(e) * P + p; }

  template <int ST>
  static __device__ __forceinline__ void stage(cx2* v, ulonglong2* sm, int t, int p, const float2* __restrict__ tw,
                                               const X2Const& K) {
    constexpr int RD = stage_radix(L, E, ST);
    constexpr int NS = stage_ns(L, E, ST);
    constexpr bool FIRST = (ST == 0);
    constexpr bool LAST = (ST == S - 1);
    constexpr int NB = E / RD;
    if constexpr (!FIRST) {
      __syncthreads();
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const ulonglong2 q = sm[sidx(p, t + T_LINE * s)];
        v[s] = cx2{q.x, q.y};
      }
      if constexpr (!LAST) __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      cx2 x[RD];
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = v[u + r * NB];
      const int j = t + u * T_LINE;
      const int jm = j % NS;
      if constexpr (NS > 1) {
        if constexpr (EXACT) {
          float2 w[RD];
          load_twiddles<float, RD>(tw + stage_table_offset(L, E, ST) + jm * RD, w);
#pragma unroll
          for (int r = 1; r < RD; ++r) x[r] = tw2_apply(x[r], tw2_from(w[r]));
        } else {
          x2_twiddle_scalar_powers<RD>(x, __ldg(tw + compact_table_offset(L, E, ST) + jm));
        }
      }
      X2Dft<RD>::run(x, K);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < RD; ++r) v[u + r * NB] = x[r];
      } else {
        const int base = (j / NS) * NS * RD + jm;
#pragma unroll
        for (int r = 0; r < RD; ++r) sm[sidx(p, base + r * NS)] = make_ulonglong2(x[r].re, x[r].im);
      }
    }
  }

  template <int ST>
  static __device__ __forceinline__ void stages(cx2* v, ulonglong2* sm, int t, int p, const float2* __restrict__ tw,
                                                const X2Const& K) {
    if constexpr (ST < S) {
      stage<ST>(v, sm, t, p, tw, K);
      stages<ST + 1>(v, sm, t, p, tw, K);
    }
  }

  // unnormalised DFT, or the inverse as conj(DFT(conj x)), of both paths
  static __device__ __forceinline__ void run(float2* a, float2* b, ulonglong2* sm, int t, int p,
                                             const float2* __restrict__ tw, bool inverse) {
    const X2Const K;
    const f32x2 sg = x2_bcast(inverse ? -1.0f : 1.0f);
    cx2 v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = cx2{x2_pack(a[s].x, b[s].x), x2_mul(x2_pack(a[s].y, b[s].y), sg)};
    if constexpr (S > 1) __syncthreads();
    stages<0>(v, sm, t, p, tw, K);
#pragma unroll
    for (int s = 0; s < E; ++s) {
      x2_unpack(v[s].re, a[s].x, b[s].x);
      x2_unpack(x2_mul(v[s].im, sg), a[s].y, b[s].y);
    }
  }
};

// dual kernels whose line length the packed codelets cover
template <int L> __host__ __device__ constexpr bool dual_x2_length() {
  if constexpr (!NSLCT_DUAL_X2 || !is_pow2(L) || L < 16) return false;
  else {
    constexpr int E = elems_per_thread(L);
    bool ok = true;
    for (int st = 0; st < num_stages(L, E); ++st) {
      const int r = stage_radix(L, E, st);
      ok = ok && (r == 2 || r == 4 || r == 8 || r == 16);
    }
    return ok;
  }
}

// Multiply both paths' values of one line by the pass chirp times scale: one
// chirp value per element (phases exactly as in apply_chirp_c), broadcast to
// both lanes.
template <int L, bool COL, int E>
__device__ __forceinline__ void x2_dual_chirp(float2* a, float2* b, const PassDesc& d, int t, int line, float scale) {
  constexpr int T = L / E;
  const Chirp& ch = d.chirp;
  const int nl = COL ? d.Ny : d.Nx;
  const long long bl = d.freq_domain ? (long long)centred_bin(line, nl) : (long long)line - nl / 2;
  const long long a0 = d.freq_domain ? (long long)t : (long long)t - L / 2;
  const uint64_t ka = COL ? ch.k11 : ch.k22;
  const uint64_t kb = COL ? ch.k22 : ch.k11;
  const uint64_t kab_b = ch.k12 * (uint64_t)bl;
  const uint64_t base = kb * (uint64_t)(bl * bl);
  const uint64_t dd = 2ull * ka * (uint64_t)((long long)T * T);
  uint64_t q = ka * (uint64_t)(a0 * a0) + kab_b * (uint64_t)a0 + base;
  uint64_t dq = ka * (uint64_t)(2 * a0 * T + (long long)T * T) + kab_b * (uint64_t)T;
#pragma unroll
  for (int s = 0; s < E; ++s) {
    if (d.freq_domain && s == E / 2) {
      const long long av = a0 + (long long)T * s - L;
      q = ka * (uint64_t)(av * av) + kab_b * (uint64_t)av + base;
      dq = ka * (uint64_t)(2 * av * T + (long long)T * T) + kab_b * (uint64_t)T;
    }
    const float tt = (float)(int)(unsigned)(q >> 32) * 2.3283064365386963e-10f;  // 2^-32
    float sn, cs;
    __sincosf(6.28318530717958647692f * tt, &sn, &cs);
    q += dq;
    dq += dd;
    const float2 w = make_float2(cs * scale, sn * scale);
    const cx2 x = {x2_pack(a[s].x, b[s].x), x2_pack(a[s].y, b[s].y)};
    const cx2 y = tw2_apply(x, tw2_from(w));
    x2_unpack(y.re, a[s].x, b[s].x);
    x2_unpack(y.im, a[s].y, b[s].y);
  }
}

// ---------------------------------------------------------------------------
// Dual passes for the adjoint (nslct_backward). Two fields go through the same
// pass of the inverse chain: the gradient path g (-> grad_in) and the value
// path y (-> workspace), which recomputes the forward intermediates by
// inverting the chain instead of storing them. At the pass's chirp point,
// before the chirp, the CTA accumulates
//     S_aa = sum a^2 q,  S_ab = sum a b q,  S_bb = sum b^2 q,  q = Im(conj(g) y)
// with (a, b) the chirp's integer coordinates along (x, y); the host turns
// these into d loss / d chirp entries. One panel per CTA; partial sums per CTA
// go to `partials[blockIdx.x][3]` (FP64), reduced later in a fixed order.
// ---------------------------------------------------------------------------
#ifndef NSLCT_DUAL_THREADS
#define NSLCT_DUAL_THREADS 256
#endif
template <typename R, int L> struct DualShape {
  static constexpr int E = elems_per_thread(L);  // the plan's tw16 tables
  static constexpr int T_LINE = L / E;
  // NSLCT_DUAL_THREADS-thread CTAs (at least two lines): 256 gives twice the
  // CTAs of 512 and lets two share an SM
  static constexpr int P0 = NSLCT_DUAL_THREADS / T_LINE;
  static constexpr int P = P0 < 2 ? 2 : (P0 > 32 ? 32 : P0);
  static constexpr int THREADS = T_LINE * P;
  static constexpr int XSM = P * (L + L / 16);
  // FP32: the two paths share each exchange (16-byte entries)
  static constexpr size_t SMEM = (size_t)XSM * sizeof(cpx<R>) * (sizeof(R) == 4 ? 2 : 1) + 32 * 3 * sizeof(double);
  static_assert(SMEM <= 227 * 1024, "adjoint kernel shared memory");
};

template <typename R, int L, bool COL>
__global__ void __launch_bounds__(DualShape<R, L>::THREADS, DualShape<R, L>::THREADS <= 256 ? 2 : 1)
dual_pass_kernel(PassDesc d, const void* in_y, void* out_y, double* partials, int accumulate) {
  using Sh = DualShape<R, L>;
  constexpr int E = Sh::E;
  constexpr int T_LINE = Sh::T_LINE;
  constexpr int P = Sh::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw + (size_t)Sh::XSM * sizeof(cpx<R>) * (sizeof(R) == 4 ? 2 : 1));

  const int tid = threadIdx.x;
  const int p = tid % P;
  const int t = tid / P;
  const int nlines = COL ? d.Ny : d.Nx;
  // same-plan batches: CTA b * (CTAs per field) + k takes panel k of field b
  const int cpf = (nlines + P - 1) / P;
  const int bf = blockIdx.x / cpf;
  const int line = (blockIdx.x % cpf) * P + p;
  const bool valid = line < nlines;
  const cpx<R>* __restrict__ gin = reinterpret_cast<const cpx<R>*>(d.in) + bf * d.in_bstride;
  const cpx<R>* __restrict__ yin = reinterpret_cast<const cpx<R>*>(in_y) + bf * d.in_bstride;
  cpx<R>* gout = reinterpret_cast<cpx<R>*>(d.out) + bf * d.out_bstride;
  cpx<R>* yout = reinterpret_cast<cpx<R>*>(out_y) + bf * d.out_bstride;
  const cpx<R>* __restrict__ tw = reinterpret_cast<const cpx<R>*>(d.tw);

  cpx<R> vg[E], vy[E];
#pragma unroll
  for (int s = 0; s < E; ++s) {
    const int e = t + T_LINE * s;
    const int i = COL ? e : line;
    const int j = COL ? line : e;
    const int k = elem_index(i, j, d.Ny, d.in_tiled);
    vg[s] = valid ? gin[k] : mk<R>((R)0, (R)0);
    vy[s] = valid ? yin[k] : mk<R>((R)0, (R)0);
  }
  constexpr bool X2 = sizeof(R) == 4 && dual_x2_length<L>();
  if (d.t1 != kNone) {
    if constexpr (X2) {
      LineFftX2<L, P, E>::run(vg, vy, reinterpret_cast<ulonglong2*>(sm), t, p, tw, d.t1 == kInv);
    } else if constexpr (sizeof(R) == 4) {
      LineFft2<L, P, E>::run(vg, vy, reinterpret_cast<float4*>(sm), t, p, tw, d.t1 == kInv);
    } else {
      LineFft<R, L, P, E, false, true>::run(vg, sm, t, p, tw, d.t1 == kInv);
      LineFft<R, L, P, E, false, true>::run(vy, sm, t, p, tw, d.t1 == kInv);
    }
  }
  if (accumulate) {
    // coordinates as in apply_chirp
    const int nl = COL ? d.Ny : d.Nx;
    const int lc = d.freq_domain ? centred_bin(line, nl) : line - nl / 2;
    // per-thread sums in the plan's precision; FP32 sums carry their rounding
    // error along (TwoSum), since the weighted terms cancel heavily
    R sum[3] = {(R)0, (R)0, (R)0}, err[3] = {(R)0, (R)0, (R)0};
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int e = t + T_LINE * s;
      const int ec = d.freq_domain ? centred_bin(e, L) : e - L / 2;
      const int a = COL ? ec : lc;   // x coordinate
      const int b = COL ? lc : ec;   // y coordinate
      const R q = vg[s].x * vy[s].y - vg[s].y * vy[s].x;
      const R term[3] = {(R)(a * a) * q, (R)(a * b) * q, (R)(b * b) * q};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if constexpr (sizeof(R) == 4) {
          const R tsum = sum[k] + term[k];
          const R bp = tsum - sum[k];
          err[k] += (sum[k] - (tsum - bp)) + (term[k] - bp);
          sum[k] = tsum;
        } else {
          sum[k] += term[k];
        }
      }
    }
    double acc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] = valid ? (double)sum[k] + (double)err[k] : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    const int warp = tid >> 5, lane = tid & 31;
    __syncthreads();
    if (lane == 0)
      for (int k = 0; k < 3; ++k) red[warp * 3 + k] = acc[k];
    __syncthreads();
    if (tid == 0) {
      double tot[3] = {0.0, 0.0, 0.0};
      for (int w = 0; w < Sh::THREADS / 32; ++w)
        for (int k = 0; k < 3; ++k) tot[k] += red[w * 3 + k];
      for (int k = 0; k < 3; ++k) partials[blockIdx.x * 3 + k] = tot[k];
    }
  }
  if (d.has_chirp) {
    if constexpr (X2) {
      x2_dual_chirp<L, COL, E>(vg, vy, d, t, line, (float)d.scale);
    } else {
      apply_chirp<R, L, COL, E>(vg, d, t, line, (R)d.scale);
      apply_chirp<R, L, COL, E>(vy, d, t, line, (R)d.scale);
    }
  } else if (d.scale != 1.0) {
    const R scale = (R)d.scale;
#pragma unroll
    for (int s = 0; s < E; ++s) {
      vg[s] = mk<R>(vg[s].x * scale, vg[s].y * scale);
      vy[s] = mk<R>(vy[s].x * scale, vy[s].y * scale);
    }
  }
  if (d.t2 != kNone) {
    if constexpr (X2) {
      LineFftX2<L, P, E>::run(vg, vy, reinterpret_cast<ulonglong2*>(sm), t, p, tw, d.t2 == kInv);
    } else if constexpr (sizeof(R) == 4) {
      LineFft2<L, P, E>::run(vg, vy, reinterpret_cast<float4*>(sm), t, p, tw, d.t2 == kInv);
    } else {
      LineFft<R, L, P, E, false, true>::run(vg, sm, t, p, tw, d.t2 == kInv);
      LineFft<R, L, P, E, false, true>::run(vy, sm, t, p, tw, d.t2 == kInv);
    }
  }
  __syncthreads();  // in-place: all loads of the panel happened before any store
  if (valid) {
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int e = t + T_LINE * s;
      const int i = COL ? e : line;
      const int j = COL ? line : e;
      const int k = elem_index(i, j, d.Ny, d.out_tiled);
      gout[k] = vg[s];
      yout[k] = vy[s];
    }
  }
}

// number of CTAs (and partial-sum rows) a dual pass along this axis uses
template <typename R, int L>
inline int dual_blocks(int nlines) { return (nlines + DualShape<R, L>::P - 1) / DualShape<R, L>::P; }

template <typename R, int L, bool COL>
inline int launch_dual_one(const PassDesc& d, const void* in_y, void* out_y, double* partials, int accumulate,
                           cudaStream_t s) {
  using Sh = DualShape<R, L>;
  const int nlines = COL ? d.Ny : d.Nx;
  const int nb = d.nbatch > 1 ? d.nbatch : 1;
  dual_pass_kernel<R, L, COL><<<nb * dual_blocks<R, L>(nlines), Sh::THREADS, Sh::SMEM, s>>>(d, in_y, out_y, partials,
                                                                                           accumulate);
  return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
}

template <typename R, int L>
inline int prepare_dual_one() {
  using Sh = DualShape<R, L>;
  cudaError_t e1 = cudaFuncSetAttribute(dual_pass_kernel<R, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)Sh::SMEM);
  cudaError_t e2 = cudaFuncSetAttribute(dual_pass_kernel<R, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)Sh::SMEM);
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? NSLCT_OK : NSLCT_E_CUDA;
}

}  // namespace nslct
