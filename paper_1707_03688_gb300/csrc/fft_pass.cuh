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
#include "fft_schedule.h"

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

__device__ __forceinline__ int padded(int e) { return e + (e >> 4); }

// Twiddles of stage ST for butterfly jm: tab[OFF + jm*RD + r] = W_{NS*RD}^{jm*r}.
template <typename R, int RD>
__device__ __forceinline__ void load_twiddles(const cpx<R>* __restrict__ row, cpx<R>* w) {
  if constexpr (sizeof(R) == 4 && RD % 2 == 0) {
    // two complex64 per 16-byte load; rows start at even entries
    const float4* p4 = reinterpret_cast<const float4*>(row);
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
        cpx<R> w[RD];
        load_twiddles<R, RD>(tw + stage_table_offset(L, ST) + jm * RD, w);
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
template <typename R, int L, bool COL>
__device__ __forceinline__ void apply_chirp(cpx<R>* v, const PassDesc& d, int t, int line, R scale) {
  constexpr int E = elems_per_thread(L);
  constexpr int T = L / E;
  const int nl = COL ? d.Ny : d.Nx;   // length of the other axis
  // coordinate of the line and of element 0
  long long b, a0;
  if (d.freq_domain) {
    b = centred_bin(line, nl);
    a0 = t;
  } else {
    b = (long long)line - nl / 2;
    a0 = (long long)t - L / 2;
  }
  // phase = ka a^2 + kab a b + kb b^2 with (ka, kb) the element/line coefficients
  const uint64_t ka = COL ? d.chirp.k11 : d.chirp.k22;
  const uint64_t kb = COL ? d.chirp.k22 : d.chirp.k11;
  const uint64_t kab_b = d.chirp.k12 * (uint64_t)b;
  const uint64_t base = kb * (uint64_t)(b * b);
  auto phase_at = [&](long long a) -> uint64_t { return ka * (uint64_t)(a * a) + kab_b * (uint64_t)a + base; };
  const uint64_t dd = 2ull * ka * (uint64_t)((long long)T * T);
  uint64_t q = phase_at(a0);
  uint64_t dq = ka * (uint64_t)(2 * a0 * T + (long long)T * T) + kab_b * (uint64_t)T;
#pragma unroll
  for (int s = 0; s < E; ++s) {
    if (d.freq_domain && s == E / 2) {
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
    v[s] = valid ? in[elem_index(i, j, d.Ny, d.in_tiled)] : mk<R>((R)0, (R)0);
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

// ---------------------------------------------------------------------------
// v2 (FP32): persistent CTAs, one per SM. The next panel is copied
// global -> shared with 16-byte cp.async while the current one is in registers
// going through the FFTs, so HBM reads overlap the arithmetic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int L, bool COL> struct PShape {
  static constexpr int E = elems_per_thread(L);
  static constexpr int T_LINE = L / E;
  static constexpr int P0 = 512 / T_LINE;
  static constexpr int P = P0 < 2 ? 2 : (P0 > 32 ? 32 : P0);
  static constexpr int THREADS = T_LINE * P;
  static constexpr int XSM = P * (L + L / 16);                   // exchange buffer entries
  static constexpr int STG = COL ? P * L : P * (L + 8);          // staging buffer entries (row-major rows padded)
  static constexpr size_t SMEM = (size_t)(XSM + STG) * sizeof(float2);
};

// staging index of element e of panel line p
template <int L, bool COL, int P>
__device__ __forceinline__ int stg_index(int p, int e, int in_tiled) {
  if (COL) return (e >> 1) * (2 * P) + (p >> 1) * 4 + (e & 1) * 2 + (p & 1);
  if (in_tiled) return (p >> 1) * (2 * L) + (e >> 1) * 4 + (p & 1) * 2 + (e & 1);
  return p * (L + 8) + e;
}

// Issue the 16-byte copies of one panel into the staging buffer.
template <int L, bool COL>
__device__ __forceinline__ void stage_panel(float2* stg, const float2* __restrict__ in, const PassDesc& d, int panel) {
  using Sh = PShape<L, COL>;
  constexpr int P = Sh::P;
  constexpr int CHUNKS = P * L / 2;  // 16-byte chunks per panel
  const int first = panel * P;
  if (COL) {
    // row pair a: P/2 tiles (2P complex, P chunks) starting at tile first/2
    const int tiles_valid = min(P, d.Ny - first) / 2;
    for (int c = threadIdx.x; c < CHUNKS; c += Sh::THREADS) {
      const int a = c / P, k = c % P;
      if ((k >> 1) < tiles_valid)
        cp_async16(stg + a * (2 * P) + k * 2, in + a * (2 * d.Ny) + (first >> 1) * 4 + k * 2);
    }
  } else if (d.in_tiled) {
    // P/2 row pairs, each 2L complex contiguous (L chunks)
    const int rows_valid = min(P, d.Nx - first);
    for (int c = threadIdx.x; c < CHUNKS; c += Sh::THREADS) {
      const int q = c / L, k = c % L;
      if (2 * q < rows_valid) cp_async16(stg + q * (2 * L) + k * 2, in + ((first >> 1) + q) * (2 * L) + k * 2);
    }
  } else {
    constexpr int CPR = L / 2;  // chunks per row
    const int rows_valid = min(P, d.Nx - first);
    for (int c = threadIdx.x; c < CHUNKS; c += Sh::THREADS) {
      const int p = c / CPR, k = c % CPR;
      if (p < rows_valid) cp_async16(stg + p * (L + 8) + k * 2, in + (first + p) * L + k * 2);
    }
  }
  cp_async_commit();
}

template <int L, bool COL>
__global__ void __launch_bounds__(PShape<L, COL>::THREADS, 1)
pass_kernel_v2(PassDesc d) {
  using Sh = PShape<L, COL>;
  constexpr int E = Sh::E;
  constexpr int T_LINE = Sh::T_LINE;
  constexpr int P = Sh::P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* xs = reinterpret_cast<float2*>(smem_raw);
  float2* stg = xs + Sh::XSM;

  const int tid = threadIdx.x;
  const int p = tid % P;
  const int t = tid / P;
  const int nlines = COL ? d.Ny : d.Nx;
  const int npanels = (nlines + P - 1) / P;
  const float2* __restrict__ in = reinterpret_cast<const float2*>(d.in);
  float2* out = reinterpret_cast<float2*>(d.out);
  const float2* __restrict__ tw = reinterpret_cast<const float2*>(d.tw);
  const float scale = d.fscale;

  int panel = blockIdx.x;
  if (panel < npanels) stage_panel<L, COL>(stg, in, d, panel);
  for (; panel < npanels; panel += gridDim.x) {
    const int line = panel * P + p;
    const bool valid = line < nlines;
    cp_async_wait_all();
    __syncthreads();
    float2 v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = stg[stg_index<L, COL, P>(p, t + T_LINE * s, d.in_tiled)];
    __syncthreads();  // staging buffer free again
    const int next = panel + gridDim.x;
    if (next < npanels) stage_panel<L, COL>(stg, in, d, next);

    if (d.t1 != kNone) LineFft<float, L, P>::run(v, xs, t, p, tw, d.t1 == kInv);
    if (d.has_chirp) {
      apply_chirp<float, L, COL>(v, d, t, line, scale);
    } else if (d.scale_only) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = make_float2(v[s].x * scale, v[s].y * scale);
    }
    if (d.t2 != kNone) LineFft<float, L, P>::run(v, xs, t, p, tw, d.t2 == kInv);

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
  cp_async_wait_all();
}

template <typename R, int L, bool COL>
inline int launch_one(const PassDesc& d, cudaStream_t s) {
  const int nlines = COL ? d.Ny : d.Nx;
  if constexpr (sizeof(R) == 4) {
    using Sh = PShape<L, COL>;
    const int npanels = (nlines + Sh::P - 1) / Sh::P;
    const int blocks = npanels < d.num_sms ? npanels : d.num_sms;
    pass_kernel_v2<L, COL><<<blocks, Sh::THREADS, Sh::SMEM, s>>>(d);
  } else {
    using Sh = PassShape<R, L>;
    const int blocks = (nlines + Sh::P - 1) / Sh::P;
    pass_kernel<R, L, COL><<<blocks, Sh::THREADS, Sh::SMEM, s>>>(d);
  }
  return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
}

template <typename R, int L>
inline int prepare_one() {
  cudaError_t e1, e2;
  if constexpr (sizeof(R) == 4) {
    e1 = cudaFuncSetAttribute(pass_kernel_v2<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PShape<L, false>::SMEM);
    e2 = cudaFuncSetAttribute(pass_kernel_v2<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PShape<L, true>::SMEM);
  } else {
    using Sh = PassShape<R, L>;
    e1 = cudaFuncSetAttribute(pass_kernel<R, L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    e2 = cudaFuncSetAttribute(pass_kernel<R, L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  }
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? NSLCT_OK : NSLCT_E_CUDA;
}

}  // namespace nslct
