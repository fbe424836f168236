// Batched passes: one persistent launch per pass covers every field of a batch
// of fields with uneven sizes (each with its own ABCD plan).
//
// Work items are (field, panel) pairs, ordered largest line first, and handed
// out through an atomic counter, so a CTA that finishes a small panel takes
// the next one. A CTA takes its item indices three items ahead of use, reads
// the item records two ahead and copies the descriptors one ahead (cp.async,
// three shared slots), so that starting an item waits on no global load but
// its panel, which is copied global -> shared with 16-byte cp.async while the
// CTA still computes the previous item. The line length (a template parameter
// in the single-field kernels) is dispatched per item here. Five passes make
// one batched transform; they can be captured into one CUDA graph.
#pragma once

#include "batch_common.h"
#include "fft_pass.cuh"

namespace nslct {

// lengths the batched kernels handle (line length along the pass axis)
#define NSLCT_BATCH_LENGTHS(X) \
  X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(96) X(192) X(384) X(768) X(1536)

// CTA configurations (the template parameter TH below): 512 threads (one CTA
// per SM, every length), 256 threads (two CTAs per SM with independent
// barriers, lines up to 2048: a panel needs at least two lines of L/E threads
// each), 128 threads (four CTAs per SM) and kB3K (batch_common.h): 128 threads
// for 3*2^a lines alone (three CTAs per SM). Packed configurations hold the
// same positions of two lines in each thread as the two FP32x2 lanes
// (pair_x2.cuh, LineFftX2), so a panel has twice the lines of its threads:
// 128 threads pack power-of-two lines up to 2048 (16 positions per line;
// 3*2^a lines run one per thread), kB3K packs 3*2^a lines up to 1536 (24
// positions per line: the registers of three CTAs per SM, not four).
// bthreads gives a configuration's thread count.
__host__ __device__ constexpr int bthreads(int TH) { return TH % 1000; }
template <int L> __host__ __device__ constexpr bool x2_3k_length() {
  if constexpr (is_pow2(L) || L % 24 != 0 || L > 2048) return false;
  else {
    constexpr int E = elems_per_thread(L);
    bool ok = E == 24 && stage_radix(L, E, 0) == 24;
    for (int st = 1; st < num_stages(L, E); ++st) {
      const int r = stage_radix(L, E, st);
      ok = ok && (r == 2 || r == 4 || r == 8);
    }
    return ok;
  }
}
template <int L, int TH> __host__ __device__ constexpr bool batch_packed() {
  return TH == kB3K ? x2_3k_length<L>() : (TH == 128 && dual_x2_length<L>() && L <= 2048);
}
template <int L, int TH> struct BShape {
  static constexpr int E = elems_per_thread(L);  // the plans' tw16 tables
  static constexpr int T_LINE = L / E;
  static constexpr int THREADS = bthreads(TH);
  static constexpr bool PACKED = batch_packed<L, TH>();
  static constexpr int P = (PACKED ? 2 : 1) * THREADS / T_LINE;  // lines per panel
  static constexpr bool ok = (TH != kB3K || PACKED) && P >= 2 && P % 2 == 0 &&
                             (PACKED ? P / 2 : P) * T_LINE == THREADS;
  static constexpr int XSM = P * (L + L / 16);
  static constexpr int STG_ROW = P * (L + 8);  // row-major rows are padded in staging
  static constexpr int STG_TILED = P * L;
};

// exchange-buffer and staging-buffer entries for the largest need among the lengths
template <int TH>
__host__ __device__ constexpr int batch_xsm() {
  int m = 0;
#define NSLCT_BSM(LL) \
  if (BShape<LL, TH>::ok && BShape<LL, TH>::XSM > m) m = BShape<LL, TH>::XSM;
  NSLCT_BATCH_LENGTHS(NSLCT_BSM)
#undef NSLCT_BSM
  return m;
}
template <int TH>
__host__ __device__ constexpr int batch_stg() {
  int m = 0;
#define NSLCT_BSM(LL) \
  if (BShape<LL, TH>::ok && BShape<LL, TH>::STG_ROW > m) m = BShape<LL, TH>::STG_ROW;
  NSLCT_BATCH_LENGTHS(NSLCT_BSM)
#undef NSLCT_BSM
  return m;
}
// 128-thread CTAs stage each panel in the exchange buffer itself (four CTAs
// per SM; the next panel is copied in once the item's last FFT has read the
// buffer); the larger CTAs keep a separate staging buffer, filled while they
// compute.
template <int TH> __host__ __device__ constexpr bool batch_single_buffer() { return bthreads(TH) == 128; }
template <int TH> __host__ __device__ constexpr int batch_ctas_per_sm() {
  return TH == kB3K ? 3 : (TH == 128 ? 4 : (TH == 256 ? 2 : 1));
}
template <int TH> constexpr size_t batch_smem() {
  return (size_t)(batch_single_buffer<TH>() ? (batch_xsm<TH>() > batch_stg<TH>() ? batch_xsm<TH>() : batch_stg<TH>())
                                            : batch_xsm<TH>() + batch_stg<TH>()) *
         sizeof(float2);
}
static_assert(batch_smem<512>() <= 227 * 1024, "batched kernel shared memory");
static_assert(batch_smem<256>() <= 113 * 1024, "two 256-thread batched CTAs per SM");
static_assert(batch_smem<128>() <= 52 * 1024, "four 128-thread batched CTAs per SM");
static_assert(batch_smem<kB3K>() <= 70 * 1024, "three packed 3*2^a CTAs per SM");

// lines per panel for line length L with TH-thread CTAs (0: not handled)
template <int TH>
__host__ __device__ constexpr int batch_lines_of(int L) {
#define NSLCT_BP(LL) \
  if (L == LL) return BShape<LL, TH>::ok ? BShape<LL, TH>::P : 0;
  NSLCT_BATCH_LENGTHS(NSLCT_BP)
#undef NSLCT_BP
  return 0;
}

template <int L, bool COL, int TH>
__device__ __forceinline__ int bstg_index(int p, int e, int tiled) {
  constexpr int P = BShape<L, TH>::P;
  if (COL) return (e >> 1) * (2 * P) + (p >> 1) * 4 + (e & 1) * 2 + (p & 1);
  if (tiled) return (p >> 1) * (2 * L) + (e >> 1) * 4 + (p & 1) * 2 + (e & 1);
  return p * (L + 8) + e;
}

// Issue the 16-byte copies of one panel (every thread takes part).
template <int L, bool COL, int TH>
__device__ __forceinline__ void bstage_panel(float2* stg, const PassDesc& d, int panel) {
  constexpr int P = BShape<L, TH>::P;
  constexpr int CHUNKS = P * L / 2;
  const float2* __restrict__ in = reinterpret_cast<const float2*>(d.in);
  const int first = panel * P;
  if (COL) {
    const int tiles_valid = min(P, d.Ny - first) / 2;
    for (int c = threadIdx.x; c < CHUNKS; c += bthreads(TH)) {
      const int a = c / P, k = c % P;
      if ((k >> 1) < tiles_valid)
        cp_async16(stg + a * (2 * P) + k * 2, in + (size_t)a * (2 * d.Ny) + (first >> 1) * 4 + k * 2);
    }
  } else if (d.in_tiled) {
    const int rows_valid = min(P, d.Nx - first);
    for (int c = threadIdx.x; c < CHUNKS; c += bthreads(TH)) {
      const int q = c / L, k = c % L;
      if (2 * q < rows_valid) cp_async16(stg + q * (2 * L) + k * 2, in + (size_t)((first >> 1) + q) * (2 * L) + k * 2);
    }
  } else {
    constexpr int CPR = L / 2;
    const int rows_valid = min(P, d.Nx - first);
    for (int c = threadIdx.x; c < CHUNKS; c += bthreads(TH)) {
      const int q = c / CPR, k = c % CPR;
      if (q < rows_valid) cp_async16(stg + q * (L + 8) + k * 2, in + (size_t)(first + q) * L + k * 2);
    }
  }
}

// Copy a pass descriptor global -> shared with 8-byte cp.async (every thread
// takes part; committed with the next cp_async_commit).
template <int TH>
__device__ __forceinline__ void bdesc_copy(PassDesc* dst, const PassDesc* src) {
  static_assert(sizeof(PassDesc) % 8 == 0 && alignof(PassDesc) >= 8, "descriptor copy by 8-byte words");
  constexpr int W = (int)(sizeof(PassDesc) / 8);
  for (int w = threadIdx.x; w < W; w += bthreads(TH))
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(reinterpret_cast<uint64_t*>(dst) + w)),
                 "l"(reinterpret_cast<const uint64_t*>(src) + w)
                 : "memory");
}

// What an item does for the pipeline once its panel is in registers: stage the
// next item's panel (its descriptor `nd` already in shared memory; null: no
// next item) and copy the descriptor of the item after it (`cs`, null: none)
// into the free slot `cd`.
struct BNext {
  const PassDesc* nd;
  int npanel;
  const PassDesc* cs;
  PassDesc* cd;
};

template <bool COL, int TH>
__device__ __forceinline__ void bstage_any(float2* stg, const PassDesc& d, int panel);

template <bool COL, int TH>
__device__ __forceinline__ void bprefetch(float2* stg, const BNext& nx) {
  if (nx.cs) bdesc_copy<TH>(nx.cd, nx.cs);
  if (nx.nd) bstage_any<COL, TH>(stg, *nx.nd, nx.npanel);
  else cp_async_commit();
}

template <bool COL, int TH>
__device__ __forceinline__ void bstage_any(float2* stg, const PassDesc& d, int panel) {
  const int L = COL ? d.Nx : d.Ny;
  switch (L) {
#define NSLCT_BCASE(LL) \
  case LL:                                                \
    if constexpr (BShape<LL, TH>::ok) bstage_panel<LL, COL, TH>(stg, d, panel); \
    break;
    NSLCT_BATCH_LENGTHS(NSLCT_BCASE)
#undef NSLCT_BCASE
    default: break;
  }
  cp_async_commit();
}

// Compute one item whose panel sits in `stg`; prefetch `next` (if any) into
// `stg` once the panel is in registers.
template <int L, bool COL, int TH>
__device__ __forceinline__ void bprocess(const PassDesc& d, int panel, float2* stg, float2* xs, const BNext& nx) {
  using Sh = BShape<L, TH>;
  constexpr int E = Sh::E;
  constexpr int T_LINE = Sh::T_LINE;
  constexpr int P = Sh::P;
  const int tid = threadIdx.x;
  const int p = tid % P;
  const int t = tid / P;
  const int nlines = COL ? d.Ny : d.Nx;
  const int line = panel * P + p;
  const bool valid = line < nlines;
  float2 v[E];
#pragma unroll
  for (int s = 0; s < E; ++s) v[s] = stg[bstg_index<L, COL, TH>(p, t + T_LINE * s, d.in_tiled)];
  __syncthreads();  // staging consumed
  if constexpr (!batch_single_buffer<TH>()) bprefetch<COL, TH>(stg, nx);
  const float2* __restrict__ tw = reinterpret_cast<const float2*>(d.tw);
  if (d.t1 != kNone) LineFft<float, L, P, E>::run(v, xs, t, p, tw, d.t1 == kInv);
  if (d.has_chirp) {
    apply_chirp<float, L, COL, E>(v, d, t, line, d.fscale);
  } else if (d.scale_only) {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = make_float2(v[s].x * d.fscale, v[s].y * d.fscale);
  }
  if (d.t2 != kNone) LineFft<float, L, P, E>::run(v, xs, t, p, tw, d.t2 == kInv);
  if constexpr (batch_single_buffer<TH>()) {
    __syncthreads();  // the last FFT has read the buffer
    bprefetch<COL, TH>(stg, nx);
  }
  float2* out = reinterpret_cast<float2*>(d.out);
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

// bprocess for packed panels: thread (pair q, position group t) holds lines
// 2q and 2q + 1 at positions t + T_LINE s in the two FP32x2 lanes from load
// to store. A pass program (d.x2.ntr > 0) runs as in the line-pair kernel;
// any other pass unpacks into the generic packed FFT's operands.
template <int L, bool COL, int TH>
__device__ __forceinline__ void bprocess_x2(const PassDesc& d, int panel, float2* stg, float2* xs, const BNext& nx) {
  using Sh = BShape<L, TH>;
  constexpr int E = Sh::E;
  constexpr int T_LINE = Sh::T_LINE;
  constexpr int P = Sh::P;
  constexpr int PP = P / 2;  // line pairs per panel
  const int tid = threadIdx.x;
  const int q = tid % PP;
  const int t = tid / PP;
  const int nlines = COL ? d.Ny : d.Nx;
  const int line0 = panel * P + 2 * q;
  const bool prog = d.x2.ntr > 0;
  // the pass program starts in the domain of its first transform (J for an
  // inverse: parts swapped) and ends in that of its last
  const bool finv = prog && d.x2_first_inv != 0;
  const bool linv = prog && (finv != (((d.x2.ntr - 1) & 1) != 0));
  cx2 v[E];
#pragma unroll
  for (int s = 0; s < E; ++s) {
    const float2 a = stg[bstg_index<L, COL, TH>(2 * q, t + T_LINE * s, d.in_tiled)];
    const float2 b = stg[bstg_index<L, COL, TH>(2 * q + 1, t + T_LINE * s, d.in_tiled)];
    const f32x2 re = x2_pack(a.x, b.x), im = x2_pack(a.y, b.y);
    v[s] = finv ? cx2{im, re} : cx2{re, im};
  }
  __syncthreads();  // staging consumed
  if constexpr (!batch_single_buffer<TH>()) bprefetch<COL, TH>(stg, nx);
  const float2* __restrict__ tw = reinterpret_cast<const float2*>(d.tw);
  ulonglong2* xs2 = reinterpret_cast<ulonglong2*>(xs);
  if (prog) {
    // inverses run in the J domain on the forward codelets, each step between
    // transforms switches domain, chirp products packed
    using F = LineFftX2<L, PP, E, false>;
    const X2Const K;
    if (d.x2.pre.kind) x2_step_e<L, E, COL, false>(v, d.x2.pre, finv, d, t, line0);
#pragma unroll 1
    for (int k = 0; k < d.x2.ntr; ++k) {
      if (k > 0) {
        const X2Step st = k == 1 ? d.x2.gap[0] : d.x2.gap[1];
        x2_step_e<L, E, COL, true>(v, st, finv != (((k - 1) & 1) != 0), d, t, line0);
      }
      if constexpr (F::S > 1) __syncthreads();  // the previous user of the exchange buffer is done
      F::template stages<0>(v, xs2, t, q, tw, K);
    }
    if (d.x2.post[0].kind) x2_step_e<L, E, COL, false>(v, d.x2.post[0], linv, d, t, line0);
    if (d.x2.post[1].kind) x2_step_e<L, E, COL, false>(v, d.x2.post[1], linv, d, t, line0);
  } else {
    float2 a[E], b[E];
#pragma unroll
    for (int s = 0; s < E; ++s) {
      x2_unpack(v[s].re, a[s].x, b[s].x);
      x2_unpack(v[s].im, a[s].y, b[s].y);
    }
    if (d.t1 != kNone) LineFftX2<L, PP, E, false>::run(a, b, xs2, t, q, tw, d.t1 == kInv);
    if (d.has_chirp) {
      apply_chirp<float, L, COL, E>(a, d, t, line0, d.fscale);
      apply_chirp<float, L, COL, E>(b, d, t, line0 + 1, d.fscale);
    } else if (d.scale_only) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        a[s] = make_float2(a[s].x * d.fscale, a[s].y * d.fscale);
        b[s] = make_float2(b[s].x * d.fscale, b[s].y * d.fscale);
      }
    }
    if (d.t2 != kNone) LineFftX2<L, PP, E, false>::run(a, b, xs2, t, q, tw, d.t2 == kInv);
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = cx2{x2_pack(a[s].x, b[s].x), x2_pack(a[s].y, b[s].y)};
  }
  if constexpr (batch_single_buffer<TH>()) {
    __syncthreads();  // the last FFT has read the buffer
    bprefetch<COL, TH>(stg, nx);
  }
  float2* out = reinterpret_cast<float2*>(d.out);
  if (COL && d.out_tiled && line0 + 1 < nlines) {
    // the two lines of a column pair at one row are one 16-byte half of a tile sector
    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int e = t + T_LINE * s;
      const cx2 w = linv ? cx2{v[s].im, v[s].re} : v[s];
      float a0, a1, b0, b1;
      x2_unpack(w.re, a0, a1);
      x2_unpack(w.im, b0, b1);
      o4[((size_t)(e >> 1) * (2 * d.Ny) + (line0 >> 1) * 4 + (e & 1) * 2) >> 1] = make_float4(a0, b0, a1, b1);
    }
    return;
  }
  if constexpr (!COL && PP < 32) {
    // rows: the thread of the neighbouring position e^1 (same line pair) is
    // lane ^ PP; the two swap halves so that each stores one 16-byte vector:
    // tiled, float4 e of the row pair; row-major, (line0[e], line0[e+1]) from
    // the even position and (line1[e-1], line1[e]) from the odd one
    // (every lane shuffles: a warp can hold a valid and an invalid pair; line
    // counts are even, so a pair is valid as a whole)
    const bool valid = line0 < nlines;
    const bool odd = (t & 1) != 0;
    float4* o4 = reinterpret_cast<float4*>(d.out_tiled ? out + (size_t)(line0 >> 1) * (2 * d.Ny)
                                                       : out + (size_t)line0 * d.Ny);
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int e = t + T_LINE * s;
      const cx2 w = linv ? cx2{v[s].im, v[s].re} : v[s];
      float r0, r1, i0, i1;
      x2_unpack(w.re, r0, r1);
      x2_unpack(w.im, i0, i1);
      const float2 give = odd ? make_float2(r0, i0) : make_float2(r1, i1);
      const float2 got = make_float2(__shfl_xor_sync(0xffffffffu, give.x, PP), __shfl_xor_sync(0xffffffffu, give.y, PP));
      const float4 o = odd ? make_float4(got.x, got.y, r1, i1) : make_float4(r0, i0, got.x, got.y);
      if (valid) o4[d.out_tiled ? e : (odd ? (d.Ny + e - 1) / 2 : e / 2)] = o;
    }
    return;
  }
#pragma unroll
  for (int s = 0; s < E; ++s) {
    const int e = t + T_LINE * s;
    const cx2 w = linv ? cx2{v[s].im, v[s].re} : v[s];
    float r0, r1, i0, i1;
    x2_unpack(w.re, r0, r1);
    x2_unpack(w.im, i0, i1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int line = line0 + h;
      if (line < nlines) {
        const int i = COL ? e : line;
        const int j = COL ? line : e;
        out[elem_index(i, j, d.Ny, d.out_tiled)] = h ? make_float2(r1, i1) : make_float2(r0, i0);
      }
    }
  }
}

// One pass of the batch. descs[f] is field f's descriptor for this pass;
// items[0..nitems) the work list; *counter must be 0 at launch. Item indices
// come from the counter three items ahead of use, item records two ahead and
// descriptors one ahead, so that an item starts without a global load.
template <bool COL, int TH>
__global__ void __launch_bounds__(bthreads(TH), batch_ctas_per_sm<TH>())
batch_pass_kernel(const PassDesc* __restrict__ descs, const BatchItem* __restrict__ items, int nitems, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // descriptors of the current item, the next one (its panel is staged from
  // it) and the one after (being copied)
  __shared__ __align__(16) PassDesc s_desc[3];
  __shared__ int s_idx[4];
  float2* xs = reinterpret_cast<float2*>(smem_raw);
  // the exchange buffer (sized for the largest need) comes first, staging after
  // it or (single buffer) in it
  float2* stg = batch_single_buffer<TH>() ? xs : xs + batch_xsm<TH>();
  if (threadIdx.x == 0) {
    const int base = atomicAdd(counter, 3);  // the first three items, consecutive
    s_idx[0] = base;
    s_idx[1] = base + 1;
    s_idx[2] = base + 2;
    s_idx[3] = atomicAdd(counter, 1);
  }
  __syncthreads();
  auto item_at = [&](int k) { return k < nitems ? items[k] : BatchItem{-1, 0}; };
  if (s_idx[0] >= nitems) return;
  BatchItem it0 = items[s_idx[0]], it1 = item_at(s_idx[1]), it2 = item_at(s_idx[2]);
  int idx3 = s_idx[3];
  bdesc_copy<TH>(&s_desc[0], descs + it0.field);
  if (it1.field >= 0) bdesc_copy<TH>(&s_desc[1], descs + it1.field);
  bstage_any<COL, TH>(stg, descs[it0.field], it0.panel);
  for (int i = 0; it0.field >= 0; ++i) {
    // thread 0: the index of the item four on (stored once this item's
    // barriers have passed); every thread: the record of the item three on
    int idx4 = 0;
    if (threadIdx.x == 0) idx4 = atomicAdd(counter, 1);
    const BatchItem it3 = item_at(idx3);
    cp_async_wait_all();
    __syncthreads();
    const int slot = i % 3;
    const PassDesc& d = s_desc[slot];
    const BNext nx{it1.field >= 0 ? &s_desc[(slot + 1) % 3] : nullptr, it1.panel,
                   it2.field >= 0 ? descs + it2.field : nullptr, &s_desc[(slot + 2) % 3]};
    const int L = COL ? d.Nx : d.Ny;
    switch (L) {
#define NSLCT_BCASE(LL)                                                   \
  case LL:                                                                \
    if constexpr (BShape<LL, TH>::ok) {                                   \
      if constexpr (BShape<LL, TH>::PACKED)                               \
        bprocess_x2<LL, COL, TH>(d, it0.panel, stg, xs, nx);              \
      else                                                                \
        bprocess<LL, COL, TH>(d, it0.panel, stg, xs, nx);                 \
    }                                                                     \
    break;
      NSLCT_BATCH_LENGTHS(NSLCT_BCASE)
#undef NSLCT_BCASE
      default: break;
    }
    // every thread read s_idx[3] before this item's first barrier
    if (threadIdx.x == 0) s_idx[3] = idx4;
    __syncthreads();  // everyone is done with the exchange buffer, this item's descriptor slot and s_idx
    idx3 = s_idx[3];
    it0 = it1;
    it1 = it2;
    it2 = it3;
  }
  cp_async_wait_all();
}

template <bool COL>
inline int launch_batch(int grid, int threads, const PassDesc* descs, const BatchItem* items, int nitems,
                        int* counter, cudaStream_t s) {
  if (threads == kB3K) {
    // column passes only (the batch's scheduler sends row passes' 3*2^a lines
    // to the four-CTA kernel)
    if constexpr (COL) batch_pass_kernel<COL, kB3K><<<grid, 128, batch_smem<kB3K>(), s>>>(descs, items, nitems, counter);
    else return NSLCT_E_UNSUPPORTED;
  } else if (threads == 128)
    batch_pass_kernel<COL, 128><<<grid, 128, batch_smem<128>(), s>>>(descs, items, nitems, counter);
  else if (threads == 256)
    batch_pass_kernel<COL, 256><<<grid, 256, batch_smem<256>(), s>>>(descs, items, nitems, counter);
  else
    batch_pass_kernel<COL, 512><<<grid, 512, batch_smem<512>(), s>>>(descs, items, nitems, counter);
  return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
}

template <bool COL>
inline int prepare_batch() {
  if constexpr (COL)
    if (cudaFuncSetAttribute(batch_pass_kernel<COL, kB3K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_smem<kB3K>()) != cudaSuccess)
      return NSLCT_E_CUDA;
  const bool ok = cudaFuncSetAttribute(batch_pass_kernel<COL, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batch_smem<128>()) == cudaSuccess &&
                  cudaFuncSetAttribute(batch_pass_kernel<COL, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batch_smem<256>()) == cudaSuccess &&
                  cudaFuncSetAttribute(batch_pass_kernel<COL, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batch_smem<512>()) == cudaSuccess;
  return ok ? NSLCT_OK : NSLCT_E_CUDA;
}

}  // namespace nslct
