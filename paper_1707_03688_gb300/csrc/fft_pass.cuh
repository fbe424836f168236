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
#include <cuda_runtime.h>

#include "internal.h"

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

// ---------------------------------------------------------------------------
// per-length FFT schedule
// ---------------------------------------------------------------------------
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

__device__ __forceinline__ int padded(int e) { return e + (e >> 4); }

template <typename R, int L, int P>
struct LineFft {
  static constexpr int E = elems_per_thread(L);
  static constexpr int T_LINE = L / E;
  static constexpr int S = num_stages(L);
  static_assert(L % E == 0, "bad E");

  // One Stockham stage; FIRST stage reads the registers, later stages read the
  // shared-memory line; the LAST stage leaves its result in registers.
  template <int ST>
  static __device__ __forceinline__ void stage(cpx<R>* v, cpx<R>* sm, int t, int p, const cpx<R>* __restrict__ tw) {
    constexpr int RD = stage_radix(L, ST);
    constexpr int NS = stage_ns(L, ST);
    constexpr bool FIRST = (ST == 0);
    constexpr bool LAST = (ST == S - 1);
    constexpr int NB = E / RD;  // butterflies per thread
    static_assert(E % RD == 0, "radix must divide E");
    if constexpr (!FIRST) {
      __syncthreads();
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = sm[padded(t + T_LINE * s) * P + p];
      if constexpr (!LAST) __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      cpx<R> x[RD];
#pragma unroll
      for (int r = 0; r < RD; ++r) x[r] = v[u + r * NB];
      const int j = t + u * T_LINE;
      const int jm = j % NS;
      if constexpr (NS > 1) {
        constexpr int STRIDE = L / (NS * RD);
#pragma unroll
        for (int r = 1; r < RD; ++r) x[r] = cmul<R>(x[r], tw[jm * r * STRIDE]);
      }
      Dft<R, RD>::run(x);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < RD; ++r) v[u + r * NB] = x[r];
      } else {
        const int base = (j / NS) * NS * RD + jm;
#pragma unroll
        for (int r = 0; r < RD; ++r) sm[padded(base + r * NS) * P + p] = x[r];
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
    if constexpr (S > 1) __syncthreads();  // the previous user of `sm` is done
    stages<0>(v, sm, t, p, tw);
    if (inverse) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s].y = -v[s].y;
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
  const float tt = (float)(int)(q >> 32) * 2.3283064365386963e-10f;  // 2^-32
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

// element (i, j) of an Nx x Ny field in the given layout
__device__ __forceinline__ size_t elem_index(int i, int j, int Ny, int tiled) {
  if (!tiled) return (size_t)i * Ny + j;
  return (size_t)(i >> 1) * (2 * (size_t)Ny) + (size_t)(j >> 1) * 4 + (i & 1) * 2 + (j & 1);
}

template <typename R, int L> struct PassShape {
  static constexpr int E = elems_per_thread(L);
  static constexpr int T_LINE = L / E;
  static constexpr int MAX_THREADS = 512;
  static constexpr int P0 = MAX_THREADS / T_LINE;
  static constexpr int P = P0 < 2 ? 2 : (P0 > 32 ? 32 : P0);
  static constexpr int THREADS = T_LINE * P;
  static constexpr int MIN_BLOCKS = sizeof(R) == 4 ? (THREADS >= 512 ? 2 : 1) : 1;
  static constexpr size_t SMEM = (size_t)P * (L + L / 16) * sizeof(cpx<R>);
};

template <typename R, int L, bool COL>
__global__ void __launch_bounds__(PassShape<R, L>::THREADS, PassShape<R, L>::MIN_BLOCKS)
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
    v[s] = valid ? in[elem_index(i, j, d.Ny, d.in_tiled)] : mk<R>((R)0, (R)0);
  }

  if (d.t1 != kNone) LineFft<R, L, P>::run(v, sm, t, p, tw, d.t1 == kInv);

  if (d.has_chirp) {
    const R scale = (R)d.scale;
    if (d.freq_domain) {
      // column passes: a = bin along x (element), b = bin along y (line)
      // row passes:    a = bin along x (line),    b = bin along y (element)
      const long long lb = COL ? centred_bin(line, d.Ny) : centred_bin(line, d.Nx);
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const int e = t + T_LINE * s;
        const long long eb = COL ? centred_bin(e, d.Nx) : centred_bin(e, d.Ny);
        const uint64_t q = COL ? chirp_turns(d.chirp, eb, lb) : chirp_turns(d.chirp, lb, eb);
        v[s] = cmul<R>(v[s], chirp_value(q, scale));
      }
    } else {
      const long long lc = COL ? (long long)line - d.Ny / 2 : (long long)line - d.Nx / 2;
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const int e = t + T_LINE * s;
        const long long ec = COL ? (long long)e - d.Nx / 2 : (long long)e - d.Ny / 2;
        const uint64_t q = COL ? chirp_turns(d.chirp, ec, lc) : chirp_turns(d.chirp, lc, ec);
        v[s] = cmul<R>(v[s], chirp_value(q, scale));
      }
    }
  } else if (d.scale != 1.0) {
    const R scale = (R)d.scale;
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = mk<R>(v[s].x * scale, v[s].y * scale);
  }

  if (d.t2 != kNone) LineFft<R, L, P>::run(v, sm, t, p, tw, d.t2 == kInv);

  // In-place passes: every thread of the CTA must have loaded its inputs before
  // any thread stores (the FFT stages already synchronise when S > 1).
  if (LineFft<R, L, P>::S <= 1 || (d.t1 == kNone && d.t2 == kNone)) __syncthreads();

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

template <typename R, int L, bool COL>
inline int launch_one(const PassDesc& d, cudaStream_t s) {
  using Sh = PassShape<R, L>;
  const int nlines = COL ? d.Ny : d.Nx;
  const int blocks = (nlines + Sh::P - 1) / Sh::P;
  pass_kernel<R, L, COL><<<blocks, Sh::THREADS, Sh::SMEM, s>>>(d);
  return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
}

template <typename R, int L>
inline int prepare_one() {
  using Sh = PassShape<R, L>;
  cudaError_t e1 = cudaFuncSetAttribute(pass_kernel<R, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  cudaError_t e2 = cudaFuncSetAttribute(pass_kernel<R, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? NSLCT_OK : NSLCT_E_CUDA;
}

}  // namespace nslct
