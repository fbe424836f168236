// Split-precision pass kernel on the fifth-generation tensor cores (tcgen05,
// accumulators in tensor memory) for 4096-point lines: the mixed mode
// (NSLCT_PREC_SPLIT_F16) of the chain's passes (Sec. 4.B, Eq. HA28; the FFTs
// of Eqs. BasicDFT16/20 are 92 % of the multiplications, Eq. HA32).
//
// Each 1D transform of length L = R * R (R = 64) is a four-step DFT:
//     x[R n1 + n2]  --DFT_R over n1-->  Y[k1, n2]
//     Y'[k1, n2] = Y[k1, n2] W_L^{n2 k1}                      (twiddle, FP32)
//     Y'        --DFT_R over n2-->  X[k1 + R k2]
// and each DFT_R stage is one real GEMM on the tensor cores: the 128 data
// vectors of a tile (two lines x 64) are the rows of A, the DFT matrix in
// real-block form (cos and sin of 2 pi n k / R) is B, and D = A B^T lands in
// TMEM. The real K and N indices of a complex index k and part c (0 = re,
// 1 = im) are 4 (k >> 1) + 2 c + (k & 1): the real parts of k and k + 1 are
// neighbours, then their imaginary parts, so that an accumulator row read
// from TMEM is already in packed FP32x2 pairs (re_k, re_k+1), (im_k, im_k+1)
// and an A row is written from such pairs with one FP16x2 conversion each.
// Operands are FP16 splits: a = a_hi + a_lo, w = w_hi + w_lo, and
// a_lo w_hi + a_hi w_lo + a_hi w_hi accumulates in FP32 (about 22 significant
// bits; the dropped a_lo w_lo is below 2^-22 relative). FP16's range is
// handled by exact power-of-two scales: each data row before a stage whose A
// is one thread group's row (the first stage of a transform) is scaled so its
// largest component lies in [1/2, 1); the second stage's A mixes the rows of
// a line, so the first stage's outputs are brought to the line's common scale
// (the largest row maximum of the line) before they are split, which bounds
// them by R.
//
// Layouts (tcgen05 canonical layouts, no swizzle, 16-bit elements):
//   * the first stage of each transform reads A from TMEM: row m of the tile
//     is TMEM lane m, K pairs packed two FP16 per 32-bit column;
//   * the second stage reads A from shared memory MN-major (8 consecutive
//     rows of one K index per 16 bytes), so the thread that owns data row n2
//     after the first stage writes its outputs into column n2 with 16-byte
//     stores: the four-step transposition is free;
//   * B (the DFT matrix, hi and lo) is K-major in shared memory for the whole
//     kernel.
// Row m of a tile is (line m / 64, index m % 64). Warp w handles TMEM lane
// quarter w % 4 and the quarter w / 4 of each row's 64 complex values.
//
// CTA: 16 warps, one CTA per SM, persistent over tiles; every warp runs the
// epilogue work (loads, conversion, twiddles, chirps, stores) and the last
// warp to finish an operand issues that stage's MMAs. Two tiles are in flight
// (two TMEM slots of 256 columns, two shared-memory A buffers) so that the
// tensor cores run one tile's stage while the warps prepare the other's.
//
// Every wait on an mbarrier is bounded in time; on expiry the kernel sets bit
// 0 of the plan's status word, stops issuing MMAs, lets every thread run to
// the end without waiting, drains its MMAs with bounded waits, frees its TMEM
// and returns.
#include <cmath>
#include <cstring>

#include "fft_pass.cuh"

namespace nslct {
namespace tcp {

constexpr int R = 64;               // DFT size of each tensor-core stage
constexpr int L = R * R;            // line length
constexpr int LPT = 128 / R;        // lines per tile
constexpr int KD = 2 * R;           // real K (= real N) of each stage GEMM
constexpr int NWARP = 16;
constexpr int THREADS = 32 * NWARP;
constexpr int VPT = R / 4;          // complex values a thread handles per job (16)
constexpr int NP = VPT / 2;         // ... as packed pairs (8)

// shared memory
constexpr uint32_t B_CK = 128;                   // K-major B: byte stride of core matrices along K
constexpr uint32_t B_CMN = (KD / 8) * 128;       // ... along N
constexpr uint32_t B_BYTES = KD * KD * 2;        // one of B_hi, B_lo
constexpr uint32_t A_CMN = 128;                  // MN-major A: byte stride of core matrices along M
constexpr uint32_t A_CK = (KD / 8) * 128 + 16;   // ... along K (padded against bank conflicts)
constexpr uint32_t A_BYTES = (KD / 8) * A_CK;    // one of A_hi, A_lo of one slot
constexpr uint32_t OFF_B = 0;
// twiddles: T[a][n2] = W_L^{8 a n2} (float2), then P as float4 pairs
// (re_b, re_b+1, im_b, im_b+1) of W_L^{b n2} at [b / 2][n2] (a, b < 8)
constexpr uint32_t OFF_TW = 2 * B_BYTES;
constexpr uint32_t TW_BYTES = 8 * R * 8 + 4 * R * 16;
constexpr uint32_t TAB_BYTES = 2 * B_BYTES + TW_BYTES;  // the host-built table, copied as is
constexpr uint32_t OFF_A = TAB_BYTES;            // [slot][hi, lo]
constexpr uint32_t OFF_X = OFF_A + 4 * A_BYTES;  // scratch
// barriers: table, mma_done[2], drain[NWARP]
constexpr int BAR_TAB = 0, BAR_DONE = 1, BAR_DRAIN = 3, NBAR = 3 + NWARP;
// then: TMEM base, abort flag, arrival counters [2]; then two buffers of the
// scale exchange, each [4][128] quarter-row maxima and [NWARP][2] per-line
// warp maxima
constexpr uint32_t OFF_SCALE = OFF_X + NBAR * 8 + 16;
constexpr uint32_t SCALE_FLOATS = 4 * 128 + 2 * NWARP;
constexpr uint32_t SMEM = OFF_SCALE + 2 * SCALE_FLOATS * 4;
static_assert(SMEM <= 227 * 1024, "one CTA per SM");

// TMEM columns (512 allocated): slot s holds D at 256 s, A_hi at 256 s + 128, A_lo at 256 s + 192
constexpr uint32_t TMEM_COLS = 512;

// Descriptor fields. LBO/SBO of the no-swizzle canonical layouts: the byte
// stride between core matrices along K (leading) and along M or N (stride).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family
  return d;               // base offset 0, no swizzle
}
// kind::f16 instruction descriptor: FP32 accumulator, FP16 A and B, M = 128, N = KD
__host__ __device__ constexpr uint32_t instr_desc(int a_mn) {
  return (1u << 4) | ((uint32_t)a_mn << 15) | ((uint32_t)(KD >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
               ::"r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive TMEM columns of this warp's lane quarter into r[0..31]
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// barrier of all warps (id 1; id 0 is __syncthreads)
__device__ __forceinline__ void cta_sync() { asm volatile("bar.sync 1, %0;\n" ::"r"(THREADS) : "memory"); }

__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;\n" : "=r"(old) : "r"(smem_u32(p)), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ float pow2f(int s) { return __int_as_float((s + 127) << 23); }
// exponent s with max * 2^s in [1/2, 1) (clamped so that 2^s is a normal float)
__device__ __forceinline__ int scale_exp(float mx) {
  const int e = (__float_as_int(mx) >> 23) & 0xff;
  int s = e == 0 ? 126 : 126 - e;
  return s < -126 ? -126 : s;
}
// FP16 pair (lo, hi halves) of two FP32 values, rounded to nearest
__device__ __forceinline__ uint32_t f16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// the FP32 values of an FP16 pair
__device__ __forceinline__ f32x2 f16x2_to_f32x2(uint32_t h) {
  const __half2 hh = *reinterpret_cast<const __half2*>(&h);
  const float2 f = __half22float2(hh);
  return x2_pack(f.x, f.y);
}
// hi/lo FP16 split of a packed pair: hi is v with the low 13 mantissa bits
// cleared (an FP16 value as it stands for |v| in FP16's normal range), lo the
// exact FP32 remainder rounded to FP16: v = hi + lo + O(2^-21 |v|), or
// O(2^-24) in FP16's subnormal range
__device__ __forceinline__ void split2(f32x2 v, uint32_t& hi, uint32_t& lo) {
  const f32x2 t = v & 0xFFFFE000FFFFE000ull;
  float a, b, c, e;
  x2_unpack(t, a, b);
  hi = f16x2(a, b);
  x2_unpack(x2_sub(v, t), c, e);
  lo = f16x2(c, e);
}

// Bounded wait for an mbarrier phase (see mbar_wait_bounded) that suspends
// the thread between checks instead of spinning
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, unsigned int wait_us) {
  const uint64_t limit = (uint64_t)(wait_us ? wait_us : 1000000u) * 1000ull;
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > limit) return false;
  }
}

// element (i, j) of the field in the given layout (float2 units)
__device__ __forceinline__ long long elem_at(bool col, int tiled, int ln, int e, int Ny) {
  const int i = col ? e : ln, j = col ? ln : e;
  return tiled ? (long long)(i >> 1) * (2 * Ny) + (j >> 1) * 4 + (i & 1) * 2 + (j & 1) : (long long)i * Ny + j;
}
// distance (float2 units) from element e to element e + R of a line: the
// same for every even step in both layouts
__device__ __forceinline__ long long elem_step(bool col, int tiled, int Ny) {
  return col ? (long long)R * Ny : (tiled ? 2 * R : R);
}

// The thread's 16 values of one job as 8 packed pairs: v[p] holds values 2p
// and 2p + 1 (re pair, im pair). Value j sits at element e0 + R j of its line.
struct Vals {
  cx2 v[NP];
};

__device__ __forceinline__ f32x2 x2_neg(f32x2 a) { return a ^ 0x8000000080000000ull; }
// a * b for packed complex pairs
__device__ __forceinline__ cx2 c2_mul(cx2 a, cx2 b) {
  return {x2_fma(a.re, b.re, x2_mul(a.im, x2_neg(b.im))), x2_fma(a.re, b.im, x2_mul(a.im, b.re))};
}
__device__ __forceinline__ cx2 c2_scale(cx2 a, f32x2 s) { return {x2_mul(a.re, s), x2_mul(a.im, s)}; }

// e^{2 pi i turns} for a Q0.64 fraction of a turn (top 32 bits), times scale
__device__ __forceinline__ float2 turn_phasor(uint64_t q, float scale) {
  const float tt = (float)(int)(unsigned)(q >> 32) * 2.3283064365386963e-10f;  // 2^-32
  float s, c;
  __sincosf(6.28318530717958647692f * tt, &s, &c);
  return make_float2(c * scale, s * scale);
}

// One step of the pass program (X2Step) on the thread's values of line ln,
// value j at element e0 + R j, all in one half of the line (a centred bin is
// e or e - L for all of them), times an extra factor f:
//   kind 1: the chirp e^{2 pi i phi(a, b)} * scale * f, phi the Q0.64 quadratic
//           of the chirp's coefficients; the phasors of values j and j + 1 are
//           two recurrences c_{j+2} = c_j rho_j, rho_{j+2} = rho_j delta whose
//           seeds c_0, c_1, rho_0, rho_1 and delta are evaluated from the
//           exact integer phases;
//   kind 2 (or 0 with f != 1): the scale alone.
__device__ __forceinline__ void step_x2(Vals& x, const X2Step& st, float f, bool col, const PassDesc& d, int ln,
                                        int e0) {
  if (st.kind == 1) {
    const int nl = col ? d.Ny : d.Nx;
    const uint64_t ka = col ? st.c.k11 : st.c.k22;
    const uint64_t kb = col ? st.c.k22 : st.c.k11;
    const long long b = st.freq ? (long long)centred_bin(ln, nl) : (long long)ln - nl / 2;
    const long long a0 = st.freq ? (e0 < L / 2 ? (long long)e0 : (long long)e0 - L) : (long long)e0 - L / 2;
    const uint64_t kab = st.c.k12 * (uint64_t)b;
    const uint64_t base = kb * (uint64_t)(b * b);
    auto phase = [&](long long a) { return ka * (uint64_t)(a * a) + kab * (uint64_t)a + base; };
    const uint64_t q0 = phase(a0), q1 = phase(a0 + R), q2 = phase(a0 + 2 * R), q3 = phase(a0 + 3 * R);
    const float sc = st.scale * f;
    const float2 c0 = turn_phasor(q0, sc), c1 = turn_phasor(q1, sc);
    const float2 r0 = turn_phasor(q2 - q0, 1.0f), r1 = turn_phasor(q3 - q1, 1.0f);
    const float2 dl = turn_phasor(ka * (uint64_t)(8 * R * R), 1.0f);  // phi(a + 4R) - 2 phi(a + 2R) + phi(a)
    cx2 c = {x2_pack(c0.x, c1.x), x2_pack(c0.y, c1.y)};
    cx2 rho = {x2_pack(r0.x, r1.x), x2_pack(r0.y, r1.y)};
    const cx2 delta = {x2_bcast(dl.x), x2_bcast(dl.y)};
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      x.v[p] = c2_mul(x.v[p], c);
      if (p + 1 < NP) {
        c = c2_mul(c, rho);
        rho = c2_mul(rho, delta);
      }
    }
  } else if (st.kind == 2 || f != 1.0f) {
    const f32x2 s = x2_bcast((st.kind == 2 ? st.scale : 1.0f) * f);
#pragma unroll
    for (int p = 0; p < NP; ++p) x.v[p] = c2_scale(x.v[p], s);
  }
}

// J(z) = i conj(z): the parts swapped (an inverse DFT is J DFT J)
__device__ __forceinline__ void jswap(Vals& x) {
#pragma unroll
  for (int p = 0; p < NP; ++p) x.v[p] = cx2{x.v[p].im, x.v[p].re};
}

// largest |re| or |im| of the thread's values
__device__ __forceinline__ float max_abs(const Vals& x) {
  float m[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    float a, b, c, e;
    x2_unpack(x.v[p].re, a, b);
    x2_unpack(x.v[p].im, c, e);
    m[p] = fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(c), fabsf(e)));
  }
#pragma unroll
  for (int w = NP / 2; w > 0; w >>= 1)
#pragma unroll
    for (int p = 0; p < w; ++p) m[p] = fmaxf(m[p], m[p + w]);
  return m[0];
}

struct Slot {
  int tile;    // tile index over the batch, or -1
  int s_row;   // exponent of the row scale (first stage of the current transform)
  int s_line;  // exponent of the line's common scale
};

struct Ctx {
  const PassDesc* d;
  int w, q, h, lane, m, line, r;  // warp, lane quarter, quarter of the row, lane, tile row, line, index in line
  uint32_t tbase;
  uint32_t sbase;                 // shared-memory address of the dynamic buffer
  unsigned char* smem;
  float* scale;                   // two exchange buffers
  uint32_t* arrive;               // per-slot arrival counters of the warps
  uint64_t* bars;
  volatile int* abort;            // set by any thread whose bounded wait expired
  uint32_t ph0, ph1;              // parities of mma_done[0], mma_done[1]
  uint32_t kjob;                  // K-major jobs so far (exchange buffer parity)
  int issued;                     // this thread issued MMAs
  int tpf;                        // tiles per field
};

// Issue the 24 MMAs of one stage of `slot` and commit them to mma_done[slot]:
// K-major stages read A (hi, lo) from TMEM, MN-major ones from shared memory.
__device__ __forceinline__ void issue_stage(Ctx& c, int slot, bool kmajor) {
  fence_after();
  const uint32_t dcol = c.tbase + 256u * slot;
  const uint64_t bhi0 = smem_desc(c.sbase + OFF_B, B_CK, B_CMN);
  const uint64_t blo0 = smem_desc(c.sbase + OFF_B + B_BYTES, B_CK, B_CMN);
  const uint64_t kstep_b = (2 * B_CK) >> 4;  // 16 K elements: two core matrices along K
  if (kmajor) {
    const uint32_t id = instr_desc(0);
#pragma unroll
    for (int kc = 0; kc < KD / 16; ++kc) {
      const uint32_t ahi = dcol + 128u + 8u * kc, alo = dcol + 192u + 8u * kc;
      mma_ts(dcol, alo, bhi0 + kc * kstep_b, id, kc > 0);
      mma_ts(dcol, ahi, blo0 + kc * kstep_b, id, 1);
      mma_ts(dcol, ahi, bhi0 + kc * kstep_b, id, 1);
    }
  } else {
    const uint32_t id = instr_desc(1);
    const uint64_t ahi0 = smem_desc(c.sbase + OFF_A + (2 * slot) * A_BYTES, A_CK, A_CMN);
    const uint64_t alo0 = smem_desc(c.sbase + OFF_A + (2 * slot + 1) * A_BYTES, A_CK, A_CMN);
    const uint64_t kstep_a = (2 * A_CK) >> 4;
#pragma unroll
    for (int kc = 0; kc < KD / 16; ++kc) {
      mma_ss(dcol, alo0 + kc * kstep_a, bhi0 + kc * kstep_b, id, kc > 0);
      mma_ss(dcol, ahi0 + kc * kstep_a, blo0 + kc * kstep_b, id, 1);
      mma_ss(dcol, ahi0 + kc * kstep_a, bhi0 + kc * kstep_b, id, 1);
    }
  }
  mma_commit(&c.bars[BAR_DONE + slot]);
  c.issued = 1;
}

// A warp has written its part of the slot's next A operand: count it; the
// last warp to arrive issues the stage (the atomic's release/acquire orders
// every warp's writes before the MMAs).
__device__ __forceinline__ void operand_ready(Ctx& c, int slot, bool kmajor) {
  __syncwarp();
  if (c.lane == 0) {
    // the counter only grows: every NWARP-th arrival completes an operand
    const uint32_t old = atom_add_acq_rel(&c.arrive[slot], 1u);
    if (old % NWARP == NWARP - 1 && !*c.abort) issue_stage(c, slot, kmajor);
  }
  __syncwarp();
}

// Scale the thread's values (a quarter of row m) by the row's power of two,
// split them into FP16 halves and write them as the K-major A operand of the
// slot in TMEM (row m = lane, K pairs = columns 16 h .. 16 h + 15); record the
// row and line exponents. `mx` is the largest |re| or |im| of these values
// before the factor `pre` that the caller still has to apply (a power of
// two, folded into the row scale here).
__device__ __forceinline__ void write_kmajor(Ctx& c, Slot& sl, int slot, const Vals& x, float mx) {
  // the warp's maximum per line: its lanes with the same bit 3 hold one line
  float wm = mx;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    if (o != 8) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
  float* qmax = c.scale + (c.kjob & 1u) * SCALE_FLOATS;  // alternate buffers: the previous
  float* wmax = qmax + 4 * 128;                          // exchange may still be read
  c.kjob++;
  qmax[c.h * 128 + c.m] = mx;
  if ((c.lane & ~8) == 0) wmax[2 * c.w + c.line] = wm;
  cta_sync();
  const float rowmax = fmaxf(fmaxf(qmax[c.m], qmax[128 + c.m]), fmaxf(qmax[256 + c.m], qmax[384 + c.m]));
  float linemax = 0.f;
#pragma unroll
  for (int w = 0; w < NWARP; ++w) linemax = fmaxf(linemax, wmax[2 * w + c.line]);
  sl.s_row = scale_exp(rowmax);
  sl.s_line = scale_exp(linemax);
  const f32x2 f = x2_bcast(pow2f(sl.s_row));
  uint32_t hi[2 * NP], lo[2 * NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    split2(x2_mul(x.v[p].re, f), hi[2 * p], lo[2 * p]);
    split2(x2_mul(x.v[p].im, f), hi[2 * p + 1], lo[2 * p + 1]);
  }
  const uint32_t ta = c.tbase + ((uint32_t)(32 * c.q) << 16) + 256u * slot + 128u + 16u * c.h;
  tmem_st16(ta, hi);
  tmem_st16(ta + 64, lo);
  tmem_st_wait();
  fence_before();
}

// Wait (bounded; skipped once the kernel is aborting) for the slot's MMAs,
// then load this thread's quarter of row m of D (columns 32 h .. 32 h + 31)
// as packed pairs. After an expired wait every thread still runs every step
// and barrier, on whatever the accumulator holds, so the warps stay in step.
__device__ __forceinline__ void read_d(Ctx& c, int slot, Vals& x) {
  uint32_t& ph = slot == 0 ? c.ph0 : c.ph1;
  if (!*c.abort && !wait_phase(&c.bars[BAR_DONE + slot], ph, c.d->wait_us)) *c.abort = 1;
  ph ^= 1u;
  fence_after();
  uint32_t r[2 * VPT];
  tmem_ld32(c.tbase + ((uint32_t)(32 * c.q) << 16) + 256u * slot + 32u * c.h, r);
  tmem_ld_wait();
#pragma unroll
  for (int p = 0; p < NP; ++p)
    x.v[p] = cx2{x2_pack(__uint_as_float(r[4 * p]), __uint_as_float(r[4 * p + 1])),
                 x2_pack(__uint_as_float(r[4 * p + 2]), __uint_as_float(r[4 * p + 3]))};
}

// After a transform's first stage: row n2's outputs Y[k1], k1 = 16 h + j, to
// the line scale and times W_L^{n2 k1} = T[k1 / 8][n2] P[k1 % 8][n2] (the scale
// folded into T), split, and written MN-major into column K(n2, re/im) of the
// slot's shared-memory A operand, at the row that holds (line, k1): 16 (k1 / 8)
// + 8 line + k1 % 8 (the thread mapping of pass_kernel_tc).
__device__ __forceinline__ void job_mid(Ctx& c, Slot& sl, int slot) {
  Vals x;
  read_d(c, slot, x);
  const float f = pow2f(sl.s_line - sl.s_row);
  const float2* T = reinterpret_cast<const float2*>(c.smem + OFF_TW);
  const float4* P = reinterpret_cast<const float4*>(c.smem + OFF_TW + 8 * R * 8);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const float2 t = T[(2 * c.h + a) * R + c.r];
    const f32x2 tr = x2_bcast(t.x * f), ti = x2_bcast(t.y * f), nti = x2_bcast(-t.y * f);
#pragma unroll
    for (int bp = 0; bp < 4; ++bp) {
      const float4 pw = P[bp * R + c.r];
      const f32x2 pr = x2_pack(pw.x, pw.y), pi = x2_pack(pw.z, pw.w);
      const cx2 w = {x2_fma(tr, pr, x2_mul(nti, pi)), x2_fma(tr, pi, x2_mul(ti, pr))};
      x.v[4 * a + bp] = c2_mul(x.v[4 * a + bp], w);
    }
  }
  unsigned char* ahi = c.smem + OFF_A + (2 * slot) * A_BYTES;
  unsigned char* alo = ahi + A_BYTES;
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    // k1 = 16 h + 8 g + 0..7: rows 16 (2 h + g) + 8 line + 0..7, core-matrix
    // row group 4 h + 2 g + line
    const uint32_t rowg = (uint32_t)(4 * c.h + 2 * g + c.line) * A_CMN;
#pragma unroll
    for (int comp = 0; comp < 2; ++comp) {
      const int K = 4 * (c.r >> 1) + 2 * comp + (c.r & 1);
      uint32_t ph[4], pl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) split2(comp ? x.v[4 * g + i].im : x.v[4 * g + i].re, ph[i], pl[i]);
      const uint32_t off = rowg + (uint32_t)(K >> 3) * A_CK + (uint32_t)(K & 7) * 16;
      *reinterpret_cast<uint4*>(ahi + off) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
      *reinterpret_cast<uint4*>(alo + off) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
    }
  }
  fence_proxy_async();
  fence_before();
  operand_ready(c, slot, false);
}

// The first job of a tile: its input x[R n1 + n2] (n1 = 16 h + j, n2 = r) of
// row m's line, the program's step before the first transform, the J swap
// for an inverse first transform, and the first stage's K-major A operand.
template <bool COL>
__device__ __forceinline__ void job_in(Ctx& c, Slot& sl, int slot, int e_q) {
  const PassDesc& d = *c.d;
  const int f = sl.tile / c.tpf;
  const int ln = (sl.tile % c.tpf) * LPT + c.line;
  const int e0 = c.r + e_q;
  const float2* src = reinterpret_cast<const float2*>(d.in) + (long long)f * d.in_bstride + elem_at(COL, d.in_tiled, ln, e0, d.Ny);
  const long long stp = elem_step(COL, d.in_tiled, d.Ny);
  Vals x;
  float2 t[VPT];
#pragma unroll
  for (int j = 0; j < VPT; ++j) t[j] = src[j * stp];
#pragma unroll
  for (int p = 0; p < NP; ++p) x.v[p] = cx2{x2_pack(t[2 * p].x, t[2 * p + 1].x), x2_pack(t[2 * p].y, t[2 * p + 1].y)};
  if (d.x2.pre.kind) step_x2(x, d.x2.pre, 1.0f, COL, d, ln, e0);
  if (d.x2_first_inv) jswap(x);
  write_kmajor(c, sl, slot, x, max_abs(x));
  operand_ready(c, slot, true);
}

// The job after transform t: the values X[k1 + R k2] (k1 = r, k2 = 16 h + j)
// back to true scale and out of the J domain for an inverse; then the gap step
// and the next transform's K-major A operand, or the post steps and the store.
template <bool COL>
__device__ __forceinline__ void job_after(Ctx& c, Slot& sl, int slot, int t, int e_q) {
  const PassDesc& d = *c.d;
  const X2Prog& pg = d.x2;
  const bool inv = ((d.x2_first_inv ? 1 : 0) ^ (t & 1)) != 0;
  Vals x;
  read_d(c, slot, x);
  if (inv) jswap(x);
  const int ln = (sl.tile % c.tpf) * LPT + c.line;
  const int e0 = c.r + e_q;
  const float f = pow2f(-sl.s_line);
  if (t + 1 < pg.ntr) {
    // a chirp keeps every magnitude, so the row maximum can be taken first
    const X2Step& st = t == 0 ? pg.gap[0] : pg.gap[1];
    const float mx = max_abs(x) * fabsf(f * (st.kind ? st.scale : 1.0f));
    step_x2(x, st, f, COL, d, ln, e0);
    if (!inv) jswap(x);  // the next transform runs the other way
    write_kmajor(c, sl, slot, x, mx);
    operand_ready(c, slot, true);
  } else {
    step_x2(x, pg.post[0], f, COL, d, ln, e0);
    if (pg.post[1].kind) step_x2(x, pg.post[1], 1.0f, COL, d, ln, e0);
    const int fi = sl.tile / c.tpf;
    float2* dst = reinterpret_cast<float2*>(d.out) + (long long)fi * d.out_bstride + elem_at(COL, d.out_tiled, ln, e0, d.Ny);
    const long long stp = elem_step(COL, d.out_tiled, d.Ny);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      float a, b, e, g;
      x2_unpack(x.v[p].re, a, b);
      x2_unpack(x.v[p].im, e, g);
      dst[(2 * p) * stp] = make_float2(a, e);
      dst[(2 * p + 1) * stp] = make_float2(b, g);
    }
  }
}

// Issue an L2 prefetch of a tile's input from one thread: a row tile is two
// contiguous rows in both layouts (one bulk prefetch); a column tile is one
// column pair of the 2x2-tiled field, fetched as boxes of the column tensor
// map (8-byte elements, 4 wide, PF_ROWS row pairs high) when the launcher
// made one (col_map).
constexpr int PF_ROWS = 256;
template <bool COL>
__device__ __forceinline__ void prefetch_tile(const PassDesc& d, const CUtensorMap* map, int col_map, int tpf, int tile) {
  const int f = tile / tpf;
  const int ln = (tile % tpf) * LPT;
  if (COL) {
    if (!col_map) return;
    for (int y0 = 0; y0 < d.Nx / 2; y0 += PF_ROWS)
      asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(map), "r"(2 * ln),
                   "r"(y0), "r"(f)
                   : "memory");
  } else {
    const float2* src = reinterpret_cast<const float2*>(d.in) + (long long)f * d.in_bstride + elem_at(false, d.in_tiled, ln, 0, d.Ny);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"((uint32_t)(LPT * L * sizeof(float2)))
                 : "memory");
  }
}

template <bool COL>
__global__ void __launch_bounds__(THREADS, 1)
pass_kernel_tc(PassDesc d, const __grid_constant__ CUtensorMap map_in, int col_map) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_X);
  uint32_t* s_tbase = reinterpret_cast<uint32_t*>(bars + NBAR);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tbase + 1);
  uint32_t* s_arrive = s_tbase + 2;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int nb = d.nbatch > 1 ? d.nbatch : 1;
  const int nlines = COL ? d.Ny : d.Nx;
  const int tpf = nlines / LPT;
  const int ntiles = tpf * nb;
  const int G = (int)gridDim.x;

  if (tid == 0) {
    for (int i = 0; i < NBAR; ++i) mbar_init(&bars[i], 1);
    *s_abort = 0;
    s_arrive[0] = s_arrive[1] = 0u;
    mbar_fence_init();
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(s_tbase)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    if (lane == 0) {
      // the DFT matrix halves and the twiddle factors, laid out by the host
      mbar_arrive_expect_tx(&bars[BAR_TAB], TAB_BYTES);
      bulk_load(smem + OFF_B, d.tc_tab, TAB_BYTES, &bars[BAR_TAB]);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();

  Ctx c;
  c.d = &d;
  c.w = warp;
  c.q = warp & 3;
  c.h = warp >> 2;
  c.lane = lane;
  // Tile row m (the thread's TMEM lane) holds index r of line `line`, m = 16 (r / 8)
  // + 8 line + r % 8: a warp holds 16 consecutive indices of both lines of the
  // tile, so that its global accesses cover whole 32-byte sectors of the 2x2-
  // tiled layout (both lines of a pair at two consecutive indices) in row and
  // column passes alike. Both stages use this order for their rows.
  c.m = 32 * c.q + lane;
  c.line = (c.m >> 3) & 1;
  c.r = 8 * (c.m >> 4) + (c.m & 7);
  c.tbase = *s_tbase;
  c.sbase = smem_u32(smem);
  c.smem = smem;
  c.scale = reinterpret_cast<float*>(smem + OFF_SCALE);
  c.arrive = s_arrive;
  c.bars = bars;
  c.abort = s_abort;
  c.ph0 = c.ph1 = 0u;
  c.kjob = 0u;
  c.issued = 0;
  c.tpf = tpf;
  const int e_q = 16 * R * c.h;  // first element of this thread's quarter: e = r + R (16 h + j)
  if (!wait_phase(&bars[BAR_TAB], 0, d.wait_us)) *s_abort = 1;
  const int ntr = d.x2.ntr;

  // software pipeline over tile pairs (slot 0: tile t0, slot 1: t0 + G): the
  // next pair's first job follows each slot's last, and row inputs are
  // prefetched into L2 one pair ahead
  Slot sl[2];
  sl[0].tile = blockIdx.x < ntiles ? (int)blockIdx.x : -1;
  sl[1].tile = (int)blockIdx.x + G < ntiles ? (int)blockIdx.x + G : -1;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (sl[s].tile >= 0) {
      if (tid == 0 && sl[s].tile + 2 * G < ntiles) prefetch_tile<COL>(d, &map_in, col_map, tpf, sl[s].tile + 2 * G);
      job_in<COL>(c, sl[s], s, e_q);
    }
  }
  while (sl[0].tile >= 0) {
    for (int t = 0; t < ntr; ++t) {
#pragma unroll
      for (int s = 0; s < 2; ++s)
        if (sl[s].tile >= 0) job_mid(c, sl[s], s);
      if (t + 1 < ntr) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
          if (sl[s].tile >= 0) job_after<COL>(c, sl[s], s, t, e_q);
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (sl[s].tile >= 0) {
        job_after<COL>(c, sl[s], s, ntr - 1, e_q);
        const int nt = sl[s].tile + 2 * G;
        sl[s].tile = nt < ntiles ? nt : -1;
        if (sl[s].tile >= 0) {
          if (tid == 0 && nt + 2 * G < ntiles) prefetch_tile<COL>(d, &map_in, col_map, tpf, nt + 2 * G);
          job_in<COL>(c, sl[s], s, e_q);
        }
      }
    }
  }
  // every MMA this thread issued has completed before the TMEM is released
  if (c.issued) {
    mma_commit(&bars[BAR_DRAIN + warp]);
    wait_phase(&bars[BAR_DRAIN + warp], 0, d.wait_us);
  }
  if (*s_abort && tid == 0 && d.err) atomicOr(d.err, 1u);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(c.tbase), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace tcp

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

bool tc_length(int L) { return L == tcp::L; }

size_t tc_table_bytes() { return tcp::TAB_BYTES; }

// The constant operands of the tensor-core kernel, as the bytes the kernel
// copies to shared memory: B_hi and B_lo (the real-block DFT_R matrix in the
// permuted real index order, K-major canonical layout, FP16 halves of the
// FP64 values), then the FP32 twiddle factors T[a][n2] = W_L^{8 a n2} and the
// pairs (W_L^{b n2}, W_L^{(b+1) n2}) for even b, whose products give W_L^{n2 k1}
// for k1 = 8 a + b.
void tc_build_table(unsigned char* host) {
  using namespace tcp;
  constexpr double two_pi = 6.283185307179586476925286766559;
  auto ridx = [](int k, int part) { return 4 * (k >> 1) + 2 * part + (k & 1); };
  for (int k1 = 0; k1 < R; ++k1)
    for (int n1 = 0; n1 < R; ++n1) {
      const double th = two_pi * (double)((k1 * n1) % R) / (double)R;
      // W = e^{-i th}: out_re = sum x_re cos + x_im sin, out_im = sum -x_re sin + x_im cos
      const double w[2][2] = {{std::cos(th), std::sin(th)}, {-std::sin(th), std::cos(th)}};
      for (int po = 0; po < 2; ++po)
        for (int pi = 0; pi < 2; ++pi) {
          const int n = ridx(k1, po), k = ridx(n1, pi);
          const __half hi = __double2half(w[po][pi]);
          const __half lo = __double2half(w[po][pi] - (double)__half2float(hi));
          const uint32_t off = (uint32_t)(n >> 3) * B_CMN + (uint32_t)(k >> 3) * B_CK + (n & 7) * 16 + (k & 7) * 2;
          std::memcpy(host + off, &hi, 2);
          std::memcpy(host + B_BYTES + off, &lo, 2);
        }
    }
  auto tw = [&](int n2, int k1) {
    const double th = two_pi * (double)((n2 * k1) % L) / (double)L;
    return make_float2((float)std::cos(th), (float)-std::sin(th));
  };
  float2* T = reinterpret_cast<float2*>(host + OFF_TW);
  float4* P = reinterpret_cast<float4*>(host + OFF_TW + 8 * R * 8);
  for (int n2 = 0; n2 < R; ++n2) {
    for (int a = 0; a < 8; ++a) T[a * R + n2] = tw(n2, 8 * a);
    for (int bp = 0; bp < 4; ++bp) {
      const float2 w0 = tw(n2, 2 * bp), w1 = tw(n2, 2 * bp + 1);
      P[bp * R + n2] = make_float4(w0.x, w1.x, w0.y, w1.y);
    }
  }
}

int prepare_pass_tc() {
  cudaError_t e1 = cudaFuncSetAttribute(tcp::pass_kernel_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tcp::SMEM);
  cudaError_t e2 = cudaFuncSetAttribute(tcp::pass_kernel_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tcp::SMEM);
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? NSLCT_OK : NSLCT_E_CUDA;
}

// Launch one pass on the tensor-core kernel; NSLCT_E_UNSUPPORTED when the
// pass is not one it runs (the caller then uses the FP32 kernels).
int launch_pass_tc(bool col, const PassDesc& d, cudaStream_t s) {
  const int L = col ? d.Nx : d.Ny;
  const int nlines = col ? d.Ny : d.Nx;
  if (!tc_length(L) || !d.tc_tab || nlines % tcp::LPT != 0) return NSLCT_E_UNSUPPORTED;
  if (d.pad_in || d.pad_out || d.post_mask) return NSLCT_E_UNSUPPORTED;
  PassDesc dx = d;
  const int mode = x2_program(d, dx.x2);
  if (mode == 0) return NSLCT_E_UNSUPPORTED;
  dx.x2_first_inv = (mode == 2 || mode == 3) ? 1 : 0;
  const int nb = d.nbatch > 1 ? d.nbatch : 1;
  const long long ntiles = (long long)(nlines / tcp::LPT) * nb;
  const int blocks = ntiles < d.num_sms ? (int)ntiles : d.num_sms;
  alignas(64) CUtensorMap mi{};
  int col_map = 0;
  if (col && (d.Nx / 2) % tcp::PF_ROWS == 0)
    col_map = encode_column_map_batched(&mi, d.in, d.Nx, d.Ny, 2, nb, d.in_bstride, tcp::PF_ROWS) ? 1 : 0;
  if (col) tcp::pass_kernel_tc<true><<<blocks, tcp::THREADS, tcp::SMEM, s>>>(dx, mi, col_map);
  else tcp::pass_kernel_tc<false><<<blocks, tcp::THREADS, tcp::SMEM, s>>>(dx, mi, 0);
  return cudaGetLastError() == cudaSuccess ? NSLCT_OK : NSLCT_E_CUDA;
}

}  // namespace nslct
