// C ABI of libnslct (declared in include/nslct.h).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fft_schedule.h"
#include "grad_math.h"
#include "plan_math.h"

using namespace nslct;

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Per-stage twiddle table of length L (layout in fft_schedule.h): for stage
// st >= 1 with radix RD and NS earlier points, entry [jm][r] = W_{NS RD}^{jm r}.
// Per-stage twiddle table of length L for kernels holding E elements per
// thread (layout in fft_schedule.h): for stage st >= 1 with radix RD and NS
// earlier points, entry [jm][r] = W_{NS RD}^{jm r}.
template <typename R>
int upload_twiddles(int L, int E, void** dev) {
  struct C2 { R x, y; };
  const int n = twiddle_table_size(L, E) > 0 ? twiddle_table_size(L, E) : 1;
  std::vector<C2> host(n, C2{(R)1, (R)0});
  for (int st = 1; st < num_stages(L, E); ++st) {
    const int rd = stage_radix(L, E, st), ns = stage_ns(L, E, st), off = stage_table_offset(L, E, st);
    for (int jm = 0; jm < ns; ++jm)
      for (int r = 0; r < rd; ++r) {
        const long num = (long)jm * r, den = (long)ns * rd;
        const double a = kTwoPi * (double)(num % den) / (double)den;
        host[off + jm * rd + r].x = (R)std::cos(a);
        host[off + jm * rd + r].y = (R)(-std::sin(a));
      }
    const int coff = compact_table_offset(L, E, st);
    for (int jm = 0; jm < ns; ++jm) {
      const double a = kTwoPi * (double)jm / ((double)ns * rd);
      host[coff + jm].x = (R)std::cos(a);
      host[coff + jm].y = (R)(-std::sin(a));
    }
  }
  if (cudaMalloc(dev, sizeof(C2) * n) != cudaSuccess) { *dev = nullptr; return NSLCT_E_NOMEM; }
  if (cudaMemcpy(*dev, host.data(), sizeof(C2) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(*dev);
    *dev = nullptr;
    return NSLCT_E_CUDA;
  }
  return NSLCT_OK;
}

void free_plan(nslct_plan_s* p) {
  if (!p) return;
  if (p->ws) cudaFree(p->ws);
  if (p->pad_ws) cudaFree(p->pad_ws);
  if (p->err) cudaFree(p->err);
  if (p->partials) cudaFree(p->partials);
  if (p->tc_tab) cudaFree(p->tc_tab);
  // the four twiddle pointers may alias each other: free each table once
  void* tabs[4] = {p->tw_x, p->tw_y, p->tw16_x, p->tw16_y};
  for (int i = 0; i < 4; ++i) {
    bool seen = !tabs[i];
    for (int k = 0; k < i && !seen; ++k) seen = tabs[k] == tabs[i];
    if (!seen) cudaFree(tabs[i]);
  }
  delete p;
}

int launch(const nslct_plan_s* p, bool col, const PassDesc& d, cudaStream_t s) {
  if (p->mixed && p->tc_tab) {
    // split-precision plans: the tensor-core kernel where it runs the pass
    const int rc = launch_pass_tc(col, d, s);
    if (rc != NSLCT_E_UNSUPPORTED) return rc;
  }
  if (d.nbatch > 1 && !(p->prec == 0 && !p->mixed && pair_kernel_length(col ? d.Nx : d.Ny))) {
    // a kernel without a batch dimension: one launch per field
    const size_t esz = p->prec == 1 ? 16 : 8;
    for (int b = 0; b < d.nbatch; ++b) {
      PassDesc e = d;
      e.nbatch = 1;
      e.in = static_cast<const char*>(d.in) + (size_t)b * d.in_bstride * esz;
      e.out = static_cast<char*>(d.out) + (size_t)b * d.out_bstride * esz;
      const int rc = p->prec == 1 ? launch_pass_f64(col, e, s) : launch_pass_f32(col, e, s);
      if (rc != NSLCT_OK) return rc;
    }
    return NSLCT_OK;
  }
  return p->prec == 1 ? launch_pass_f64(col, d, s) : launch_pass_f32(col, d, s);
}

// Enqueue passes [first, last] of the forward (or inverse) chain.
int run_chain(nslct_plan_t p, const void* in, void* out, nslct_stream_t stream, bool inverse, int first = 0,
              int last = 4, const void* mask = nullptr, int nbatch = 1, long long in_stride = 0,
              long long out_stride = 0) {
  if (!p || !in || !out || first < 0 || last > 4 || first > last) return NSLCT_E_ARG;
  // 16-byte copies need 16-byte aligned fields
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) return NSLCT_E_ARG;
  // a padded plan's input and output have different shapes: no in-place calls
  if (p->padded && in == out) return NSLCT_E_ARG;
  DeviceGuard g(p->device);
  if (!g.ok) return NSLCT_E_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  PassDesc d[5];
  bool cols[5];
  // a type-2 plan stores the type-1 factors of M^-1: its forward transform is
  // that plan's inverse chain and vice versa
  const int npass = build_schedule(p, in, out, inverse != (p->type2 != 0), d, cols);
  if (last >= npass) return NSLCT_E_ARG;
  if (mask) {
    if (reinterpret_cast<uintptr_t>(mask) & 15u) return NSLCT_E_ARG;
    d[npass - 1].post_mask = mask;
  }
  if (nbatch > 1) {
    // the first pass reads the caller's input; every other access is to the
    // output (the intermediate lives there)
    for (int k = 0; k < npass; ++k) {
      d[k].nbatch = nbatch;
      d[k].in_bstride = k == 0 ? in_stride : out_stride;
      d[k].out_bstride = out_stride;
    }
  }
  for (int k = first; k <= last; ++k) {
    const int rc = launch(p, cols[k], d[k], s);
    if (rc != NSLCT_OK) return rc;
  }
  return NSLCT_OK;
}

}  // namespace

namespace nslct {

bool chain_pass_is_column(int k) { return k == 1 || k == 3; }

// The five passes of the forward chain (Eq. HA28, right to left) or of the
// inverse chain (Eq. CCCMCCCM04) from `in` (row-major) to `out` (row-major),
// with `out` holding the tiled intermediate field between passes.
// The tiled grid between passes: the caller's output buffer, unless the
// caller's output is smaller than the grid (padded plans).
void* chain_mid(const nslct_plan_s* p, void* out, bool inverse) {
  if (!p->padded) return out;
  const bool small_out = inverse ? (p->in_rows != p->Nx || p->in_cols != p->Ny)
                                 : (p->out_rows != p->Nx || p->out_cols != p->Ny);
  return small_out ? p->pad_ws : out;
}

// Set the zero-padding regions of a chain's first (row-major input) and last
// (row-major output) pass: the forward reads the input region and writes the
// output region, the inverse the other way round.
void set_pad_regions(const nslct_plan_s* p, bool inverse, PassDesc& first, PassDesc& last) {
  if (!p->padded) return;
  const int* src = inverse ? &p->out_rows : &p->in_rows;
  const int* dst = inverse ? &p->in_rows : &p->out_rows;
  first.pad_in = (src[0] != p->Nx || src[1] != p->Ny) ? 1 : 0;
  first.in_rows = src[0]; first.in_cols = src[1]; first.in_r0 = src[2]; first.in_c0 = src[3];
  last.pad_out = (dst[0] != p->Nx || dst[1] != p->Ny) ? 1 : 0;
  last.out_rows = dst[0]; last.out_cols = dst[1]; last.out_r0 = dst[2]; last.out_c0 = dst[3];
}

void build_chain_descs(const nslct_plan_s* p, const void* in, void* out, bool inverse, PassDesc d[5]) {
  const double ccs = -1.0 / ((double)p->Nx * (double)p->Ny);  // each CC's constant, Eq. BasicDFT16/20
  PassDesc base{};
  base.Nx = p->Nx;
  base.Ny = p->Ny;
  base.scale = 1.0;
  base.fscale2 = 1.0f;
  for (int k = 0; k < 5; ++k) d[k] = base;
  void* mid = chain_mid(p, out, inverse);
  // pass 1: row pass, caller layout -> tiled layout in `mid`
  d[0].in = in; d[0].out = mid; d[0].in_tiled = 0; d[0].out_tiled = 1; d[0].tw = p->tw_y;
  // passes 2..4 in place on the tiled field; pass 5 back to the caller layout in `out`
  for (int k = 1; k < 5; ++k) { d[k].in = mid; d[k].out = mid; d[k].in_tiled = 1; d[k].out_tiled = 1; }
  d[4].out = out;
  d[4].out_tiled = 0;
  set_pad_regions(p, inverse, d[0], d[4]);
  d[1].tw = p->tw_x; d[2].tw = p->tw_y; d[3].tw = p->tw_x; d[4].tw = p->tw_y;
  d[1].freq_domain = d[3].freq_domain = 1;
  d[1].has_chirp = d[2].has_chirp = d[3].has_chirp = 1;
  d[1].t1 = kFwd; d[1].t2 = kInv;
  d[2].t1 = kInv; d[2].t2 = kFwd; d[2].scale = ccs;
  d[3].t1 = kFwd; d[3].t2 = kInv;
  d[4].t1 = kInv; d[4].scale = ccs;
  if (!inverse) {
    // CC^H, CM^{C2}, CC^{B'}, CM^{C1}
    d[0].t1 = kFwd;
    d[1].chirp = p->fwd_chi_h;
    d[2].chirp = p->fwd_cm_c2;
    d[3].chirp = p->fwd_chi_bp;
    d[4].has_chirp = 1; d[4].chirp = p->fwd_cm_c1;
  } else {
    // CM^{-C1}, CC^{-B'}, CM^{-C2}, CC^{-H}
    d[0].has_chirp = 1; d[0].chirp = p->inv_cm_c1; d[0].t2 = kFwd;
    d[1].chirp = p->inv_chi_bp;
    d[2].chirp = p->inv_cm_c2;
    d[3].chirp = p->inv_chi_h;
  }
  for (int k = 0; k < 5; ++k) {
    d[k].fscale = (float)d[k].scale;
    d[k].scale_only = (!d[k].has_chirp && d[k].scale != 1.0) ? 1 : 0;
    d[k].num_sms = p->num_sms;
    d[k].err = p->err;
    d[k].mixed = p->mixed;
    d[k].tc_tab = p->tc_tab;
  }
}

// When H = (0,0;0,h) (the closed form of Eq. LC10, or H = 0), CC^H only
// convolves along y:
//   CC^H = -(1/(Nx Ny)) IFFT2(chi_H FFT2(.)) = -(1/Ny) IFFT_y(chi_H(k_y) FFT_y(.)),
// because the x transforms of FFT2 and IFFT2 then cancel to Nx I. CC^H and
// CM^{C2} and the row half of the next CC then share one row pass:
//   forward: row [FFT_y, chi_{-H} -1/Ny, IFFT_y, CM^{C2}, FFT_y]
//            col [FFT_x, chi_{-B'}, IFFT_x]
//            row [IFFT_y, CM^{C1} -1/(Nx Ny)]
//   inverse: row [CM^{-C1}, FFT_y]
//            col [FFT_x, chi_{+B'}, IFFT_x]
//            row [IFFT_y, CM^{-C2} -1/(Nx Ny), FFT_y, chi_{+H} -1/Ny, IFFT_y]
// Three passes instead of five (48 instead of 80 bytes per sample).
int build_schedule(const nslct_plan_s* p, const void* in, void* out, bool inverse, PassDesc d[5], bool cols[5]) {
  build_chain_descs(p, in, out, inverse, d);
  for (int k = 0; k < 5; ++k) cols[k] = chain_pass_is_column(k);
  if (!p->y_only_h) return 5;
  const float cy = -1.0f / (float)p->Ny;
  const double ccs = -1.0 / ((double)p->Nx * (double)p->Ny);
  PassDesc r1 = d[0], c2 = d[1], r3 = d[4];
  if (!inverse) {
    r1.t1 = kFwd;
    r1.has_chirp = 1; r1.freq_domain = 1; r1.chirp = p->fwd_chi_h; r1.scale = cy;
    r1.t2 = kInv;
    r1.has_chirp2 = 1; r1.freq_domain2 = 0; r1.chirp2 = p->fwd_cm_c2; r1.fscale2 = 1.0f;
    r1.t3 = kFwd;
    c2 = d[3];  // FFT_x, chi_{-B'}, IFFT_x
    r3 = d[4];  // IFFT_y, CM^{C1} x -1/(Nx Ny)
  } else {
    r1 = d[0];  // CM^{-C1}, FFT_y
    c2 = d[1];  // FFT_x, chi_{+B'}, IFFT_x
    r3 = d[4];
    r3.t1 = kInv;
    r3.has_chirp = 1; r3.freq_domain = 0; r3.chirp = p->inv_cm_c2; r3.scale = ccs;
    r3.t2 = kFwd;
    r3.has_chirp2 = 1; r3.freq_domain2 = 1; r3.chirp2 = p->inv_chi_h; r3.fscale2 = cy;
    r3.t3 = kInv;
  }
  for (PassDesc* x : {&r1, &c2, &r3}) {
    x->fscale = (float)x->scale;
    x->scale_only = (!x->has_chirp && x->scale != 1.0) ? 1 : 0;
  }
  // r1 reads the caller's field and writes the tiled one; c2 works in place;
  // r3 returns to the caller's layout in `out`
  void* mid = chain_mid(p, out, inverse);
  r1.in = in; r1.out = mid; r1.in_tiled = 0; r1.out_tiled = 1;
  c2.in = mid; c2.out = mid; c2.in_tiled = 1; c2.out_tiled = 1;
  r3.in = mid; r3.out = out; r3.in_tiled = 1; r3.out_tiled = 0;
  c2.pad_in = c2.pad_out = 0;
  r1.pad_out = 0;
  r3.pad_in = 0;
  set_pad_regions(p, inverse, r1, r3);
  d[0] = r1; d[1] = c2; d[2] = r3;
  cols[0] = false; cols[1] = true; cols[2] = false;
  return 3;
}

bool supported_length(int L) {
  switch (L) {
    case 8: case 16: case 32: case 64: case 128: case 256: case 512: case 1024: case 2048: case 4096:
    case 12: case 24: case 48: case 96: case 192: case 384: case 768: case 1536:
      return true;
    default:
      return false;
  }
}
}  // namespace nslct

extern "C" {

// Host-only part of planning: validation, H choice and decomposition.
// Whether the plan runs the CC-CM-CC-CM chain (Eq. CCCMCCCM16): on request, or
// by the tr(B) rule of Eq. Reversible08 (type 2 for tr B < 0; tr B = 0 is
// left open by the equation and taken as type 1).
static bool wants_type2(const double m[16], unsigned flags) {
  if (flags & NSLCT_TYPE2) return true;
  if (flags & NSLCT_TYPE_BY_TRACE) return m[2] + m[7] < 0.0;  // b11 + b22
  return false;
}

// (A, B; C, D)^-1 = (D^T, -B^T; -C^T, A^T) (Eq. CCCMCCCM20), exact for symplectic M
static void symplectic_inverse(const double m[16], double r[16]) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      r[i * 4 + j] = m[(j + 2) * 4 + (i + 2)];            // D^T
      r[i * 4 + j + 2] = -m[j * 4 + (i + 2)];             // -B^T
      r[(i + 2) * 4 + j] = -m[(j + 2) * 4 + i];           // -C^T
      r[(i + 2) * 4 + j + 2] = m[j * 4 + i];              // A^T
    }
}

static int derive_type1(const double m[16], unsigned flags, const double* h_user, Decomp* dc);

// Validate (and optionally project) the caller's ABCD into m, choose H and
// decompose. For type-2 plans the stored factors are the type-1 factors of
// M^-1 with H = -H1: by Eqs. CCCMCCCM20-30 the type-2 chain of M with H1 is
// exactly the inverse chain of that type-1 plan, and the type-2 HA criterion
// (the gamma factors of its four chirps) equals the type-1 one of M^-1 at -H1.
static int derive(const double abcd[16], unsigned flags, const double* h_user, double m[16], Decomp* dc,
                  int* type2 = nullptr) {
  if (!abcd) return NSLCT_E_ARG;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(abcd[i])) return NSLCT_E_ARG;
  const unsigned hsel = flags & NSLCT_H_MASK;
  if (hsel == NSLCT_H_USER && !h_user) return NSLCT_E_ARG;
  std::memcpy(m, abcd, 16 * sizeof(double));
  double mmax = 1.0;
  for (int i = 0; i < 16; ++i) mmax = std::fmax(mmax, std::fabs(m[i]));
  if (flags & NSLCT_PROJECT_SP4) {
    if (!project_sp4(abcd, m)) return NSLCT_E_NOT_SYMPLECTIC;
  }
  if (symplectic_residual(m) > 1e-9 * mmax * mmax) return NSLCT_E_NOT_SYMPLECTIC;
  const bool t2 = wants_type2(m, flags);
  if (type2) *type2 = t2 ? 1 : 0;
  if (!t2) return derive_type1(m, flags, h_user, dc);
  double mi[16];
  symplectic_inverse(m, mi);
  double hneg[4];
  if (hsel == NSLCT_H_USER) {
    for (int i = 0; i < 4; ++i) hneg[i] = -h_user[i];
  }
  return derive_type1(mi, flags, hsel == NSLCT_H_USER ? hneg : nullptr, dc);
}

static int derive_type1(const double m[16], unsigned flags, const double* h_user, Decomp* dc) {
  const unsigned hsel = flags & NSLCT_H_MASK;
  Mat2 h{};
  int rc = NSLCT_OK;
  if (hsel == NSLCT_H_USER) {
    for (int i = 0; i < 4; ++i)
      if (!std::isfinite(h_user[i])) return NSLCT_E_ARG;
    h = mat2_symmetrise({h_user[0], h_user[1], h_user[2], h_user[3]});
    Mat2 a, b, c, d;
    split_blocks(m, a, b, c, d);
    const Mat2 bp = mat2_sub(b, mat2_mul(a, h));
    double scale = 1.0;
    for (double v : {bp.m00, bp.m01, bp.m10, bp.m11}) scale = std::fmax(scale, std::fabs(v));
    if (std::fabs(bp.m01 - bp.m10) > 1e-9 * scale) return NSLCT_E_INFEASIBLE;
  } else if (hsel == NSLCT_H_LC) {
    rc = choose_h_lc(m, &h);
    if (rc != NSLCT_OK) rc = choose_h_ha(m, &h);  // Sec. 4.B.2: fall back to the HA choice
  } else if (hsel == NSLCT_H_LC_Y) {
    rc = choose_h_lc_y(m, &h);
    if (rc != NSLCT_OK) rc = choose_h_lc(m, &h);
    if (rc != NSLCT_OK) rc = choose_h_ha(m, &h);
  } else {
    rc = choose_h_ha(m, &h);
  }
  if (rc != NSLCT_OK) return rc;
  *dc = decompose(m, h);
  if (!(std::fabs(dc->det_bp) >= kDetFloor)) return NSLCT_E_INFEASIBLE;
  return NSLCT_OK;
}

// The host fields of a plan that follow from its (validated) ABCD and
// decomposition: flags, M, H, B', C1, C2, the Q0.64 chirps, the three-pass
// choice and theta with its chirp Jacobian. Touches no device.
static void set_derived(nslct_plan_s* p, const double m[16], const Decomp& dc, int type2, unsigned flags) {
  p->type2 = type2;
  p->flags = (flags & ~NSLCT_TYPE2) | (type2 ? NSLCT_TYPE2 : 0u);
  std::memcpy(p->M, m, 16 * sizeof(double));
  const Mat2* src[4] = {&dc.H, &dc.Bp, &dc.C1, &dc.C2};
  double* dst[4] = {p->H, p->Bp, p->C1, p->C2};
  for (int k = 0; k < 4; ++k) {
    dst[k][0] = src[k]->m00; dst[k][1] = src[k]->m01; dst[k][2] = src[k]->m10; dst[k][3] = src[k]->m11;
  }
  fill_chirps(p);
  p->y_only_h = (p->prec == 0 && !(flags & NSLCT_FULL_CHAIN) && p->H[0] == 0.0 && p->H[1] == 0.0 && p->H[2] == 0.0)
                    ? 1 : 0;
  // theta gradients follow the type-1 chain of M only
  p->has_theta = (!p->type2 && theta_from_abcd(p->M, p->theta)) ? 1 : 0;
  // the Jacobian of the H(theta) rule about its anchor (the plan's own H
  // when it was not made from an anchor h0)
  if (p->has_theta) chirp_jacobian(p->theta, p->has_h0 ? p->h0 : p->H, p->jac);
}

int nslct_plan_ex(nslct_plan_t* out, const double abcd[16], int Nx, int Ny, double dx, double dy,
                  unsigned flags, const double* h_user) {
  if (!out) return NSLCT_E_ARG;
  *out = nullptr;
  if (!abcd || Nx < 2 || Ny < 2 || !(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy))
    return NSLCT_E_ARG;
  const unsigned prec_flag = flags & NSLCT_PREC_MASK;
  if (prec_flag != NSLCT_PREC_FP32 && prec_flag != NSLCT_PREC_FP64 && prec_flag != NSLCT_PREC_SPLIT_F16)
    return NSLCT_E_UNSUPPORTED;
  if (!supported_length(Nx) || !supported_length(Ny)) return NSLCT_E_SIZE;
  double m[16];
  Decomp dc{};
  int type2 = 0;
  int rc = derive(abcd, flags, h_user, m, &dc, &type2);
  if (rc != NSLCT_OK) return rc;

  nslct_plan_s* p = new (std::nothrow) nslct_plan_s();
  if (!p) return NSLCT_E_NOMEM;
  p->Nx = Nx; p->Ny = Ny; p->dx = dx; p->dy = dy;
  p->prec = prec_flag == NSLCT_PREC_FP64 ? 1 : 0;
  p->mixed = prec_flag == NSLCT_PREC_SPLIT_F16 ? 1 : 0;
  set_derived(p, m, dc, type2, flags);

  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    free_plan(p);
    return NSLCT_E_CUDA;
  }
  if (cudaMalloc(&p->err, sizeof(unsigned int)) != cudaSuccess) { p->err = nullptr; free_plan(p); return NSLCT_E_NOMEM; }
  if (cudaMemset(p->err, 0, sizeof(unsigned int)) != cudaSuccess) { free_plan(p); return NSLCT_E_CUDA; }
  const bool f32 = p->prec == 0;
  // forward/inverse kernels: kernel_elems (split-precision plans: 16 per thread);
  // adjoint and batched kernels: elems_per_thread
  auto fwd_e = [&](int L) { return p->mixed ? elems_per_thread(L) : kernel_elems(L, f32); };
  auto upload = [&](int L, int E, void** dst) {
    return f32 ? upload_twiddles<float>(L, E, dst) : upload_twiddles<double>(L, E, dst);
  };
  rc = upload(Nx, fwd_e(Nx), &p->tw_x);
  if (rc == NSLCT_OK) {
    if (Ny == Nx) p->tw_y = p->tw_x;
    else rc = upload(Ny, fwd_e(Ny), &p->tw_y);
  }
  if (rc == NSLCT_OK) {
    if (fwd_e(Nx) == elems_per_thread(Nx)) p->tw16_x = p->tw_x;
    else rc = upload(Nx, elems_per_thread(Nx), &p->tw16_x);
  }
  if (rc == NSLCT_OK) {
    if (Ny == Nx) p->tw16_y = p->tw16_x;
    else if (fwd_e(Ny) == elems_per_thread(Ny)) p->tw16_y = p->tw_y;
    else rc = upload(Ny, elems_per_thread(Ny), &p->tw16_y);
  }
  if (rc == NSLCT_OK) rc = p->prec ? prepare_pass_f64(Nx) : prepare_pass_f32(Nx);
  if (rc == NSLCT_OK && Ny != Nx) rc = p->prec ? prepare_pass_f64(Ny) : prepare_pass_f32(Ny);
  if (rc == NSLCT_OK && p->mixed && (tc_length(Nx) || tc_length(Ny))) {
    // the tensor-core kernel's constants (DFT matrix halves and twiddles)
    std::vector<unsigned char> tab(tc_table_bytes(), 0);
    tc_build_table(tab.data());
    if (cudaMalloc(&p->tc_tab, tab.size()) != cudaSuccess) {
      p->tc_tab = nullptr;
      rc = NSLCT_E_NOMEM;
    } else if (cudaMemcpy(p->tc_tab, tab.data(), tab.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = NSLCT_E_CUDA;
    } else {
      rc = prepare_pass_tc();
    }
  }
  if (rc != NSLCT_OK) { free_plan(p); return rc; }
  *out = p;
  return NSLCT_OK;
}

int nslct_derive(const double abcd[16], unsigned flags, const double* h_user, double abcd_used[16], double H[4],
                 double Bp[4], double C1[4], double C2[4], double* objective) {
  double m[16];
  Decomp dc{};
  int type2 = 0;
  const int rc = derive(abcd, flags, h_user, m, &dc, &type2);
  if (rc != NSLCT_OK) return rc;
  const Mat2* src[4] = {&dc.H, &dc.Bp, &dc.C1, &dc.C2};
  double* dst[4] = {H, Bp, C1, C2};
  for (int k = 0; k < 4; ++k) {
    if (!dst[k]) continue;
    dst[k][0] = src[k]->m00; dst[k][1] = src[k]->m01; dst[k][2] = src[k]->m10; dst[k][3] = src[k]->m11;
  }
  if (abcd_used) std::memcpy(abcd_used, m, sizeof(m));
  if (objective) {
    double mi[16];
    if (type2) symplectic_inverse(m, mi);
    *objective = ha_objective(type2 ? mi : m, dc.H);
  }
  return NSLCT_OK;
}

int nslct_plan_theta(nslct_plan_t* out, const double theta[10], const double h0[4], int Nx, int Ny, double dx,
                     double dy, unsigned flags) {
  if (!out) return NSLCT_E_ARG;
  *out = nullptr;
  if (!theta) return NSLCT_E_ARG;
  for (int i = 0; i < 10; ++i)
    if (!std::isfinite(theta[i])) return NSLCT_E_ARG;
  if (flags & (NSLCT_TYPE2 | NSLCT_TYPE_BY_TRACE)) return NSLCT_E_UNSUPPORTED;
  const double det_l = theta[3] * theta[6] - theta[4] * theta[5];
  if (!(std::fabs(det_l) > 1e-12)) return NSLCT_E_ARG;
  double m[16];
  abcd_from_theta(theta, m);
  flags &= ~(unsigned)(NSLCT_H_MASK | NSLCT_PROJECT_SP4);
  if (!h0) return nslct_plan_ex(out, m, Nx, Ny, dx, dy, flags, nullptr);
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(h0[i])) return NSLCT_E_ARG;
  double h[4];
  h_of_theta(theta, h0, h);
  const int rc = nslct_plan_ex(out, m, Nx, Ny, dx, dy, flags | NSLCT_H_USER, h);
  if (rc == NSLCT_OK) {
    nslct_plan_s* p = *out;
    std::memcpy(p->h0, h0, sizeof(p->h0));
    p->has_h0 = 1;
    if (p->has_theta) chirp_jacobian(p->theta, p->h0, p->jac);
  }
  return rc;
}

int nslct_plan_theta_set(nslct_plan_t p, const double theta[10]) {
  if (!p || !theta) return NSLCT_E_ARG;
  if (!p->has_h0 || p->padded || p->type2) return NSLCT_E_UNSUPPORTED;
  for (int i = 0; i < 10; ++i)
    if (!std::isfinite(theta[i])) return NSLCT_E_ARG;
  const double det_l = theta[3] * theta[6] - theta[4] * theta[5];
  if (!(std::fabs(det_l) > 1e-12)) return NSLCT_E_ARG;
  double m[16], h[4], mm[16];
  abcd_from_theta(theta, m);
  h_of_theta(theta, p->h0, h);
  const unsigned flags = (p->flags & ~(unsigned)(NSLCT_H_MASK | NSLCT_PROJECT_SP4 | NSLCT_TYPE2)) | NSLCT_H_USER;
  Decomp dc{};
  int type2 = 0;
  const int rc = derive(m, flags, h, mm, &dc, &type2);
  if (rc != NSLCT_OK) return rc;  // the plan is left as it was
  set_derived(p, mm, dc, type2, flags);
  return NSLCT_OK;
}

int nslct_plan_theta_get(nslct_plan_t p, double theta[10]) {
  if (!p || !theta) return NSLCT_E_ARG;
  if (!p->has_theta) return NSLCT_E_UNSUPPORTED;
  std::memcpy(theta, p->theta, sizeof(p->theta));
  return NSLCT_OK;
}

int nslct_plan_padded(nslct_plan_t* out, const double abcd[16], int Nx, int Ny, int Nx_pad, int Ny_pad, double dx,
                      double dy, unsigned flags) {
  if (!out) return NSLCT_E_ARG;
  *out = nullptr;
  if ((flags & NSLCT_H_MASK) == NSLCT_H_USER) return NSLCT_E_ARG;
  if (Nx < 2 || Ny < 2 || (Nx & 1) || (Ny & 1) || Nx > Nx_pad || Ny > Ny_pad) return NSLCT_E_ARG;
  const bool crop = (flags & NSLCT_CROP_OUTPUT) != 0;
  if (flags & (NSLCT_TYPE2 | NSLCT_TYPE_BY_TRACE)) return NSLCT_E_UNSUPPORTED;
  int rc = nslct_plan_ex(out, abcd, Nx_pad, Ny_pad, dx, dy, flags & ~NSLCT_CROP_OUTPUT, nullptr);
  if (rc != NSLCT_OK) return rc;
  nslct_plan_s* p = *out;
  p->flags = flags;
  p->padded = 1;
  // centred placement: index i of the field sits at i - floor(N/2) of the
  // centred grid, i.e. at row i + floor(N'/2) - floor(N/2)
  p->in_rows = Nx; p->in_cols = Ny;
  p->in_r0 = Nx_pad / 2 - Nx / 2; p->in_c0 = Ny_pad / 2 - Ny / 2;
  if (crop) {
    p->out_rows = Nx; p->out_cols = Ny; p->out_r0 = p->in_r0; p->out_c0 = p->in_c0;
  } else {
    p->out_rows = Nx_pad; p->out_cols = Ny_pad; p->out_r0 = 0; p->out_c0 = 0;
  }
  const size_t esz = p->prec == 1 ? 16 : 8;
  DeviceGuard g(p->device);
  if (!g.ok || cudaMalloc(&p->pad_ws, esz * (size_t)Nx_pad * Ny_pad) != cudaSuccess) {
    p->pad_ws = nullptr;
    free_plan(p);
    *out = nullptr;
    return NSLCT_E_NOMEM;
  }
  return NSLCT_OK;
}

int nslct_plan_shape(nslct_plan_t p, int* in_rows, int* in_cols, int* out_rows, int* out_cols) {
  if (!p) return NSLCT_E_ARG;
  if (in_rows) *in_rows = p->padded ? p->in_rows : p->Nx;
  if (in_cols) *in_cols = p->padded ? p->in_cols : p->Ny;
  if (out_rows) *out_rows = p->padded ? p->out_rows : p->Nx;
  if (out_cols) *out_cols = p->padded ? p->out_cols : p->Ny;
  return NSLCT_OK;
}

int nslct_plan(nslct_plan_t* out, const double abcd[16], int Nx, int Ny, double dx, double dy, unsigned flags) {
  if ((flags & NSLCT_H_MASK) == NSLCT_H_USER) return NSLCT_E_ARG;
  return nslct_plan_ex(out, abcd, Nx, Ny, dx, dy, flags, nullptr);
}

int nslct_plan_params(nslct_plan_t p, int field, double H[4], double Bp[4], double C1[4], double C2[4]) {
  if (!p || field != 0) return NSLCT_E_ARG;
  if (H) std::memcpy(H, p->H, 4 * sizeof(double));
  if (Bp) std::memcpy(Bp, p->Bp, 4 * sizeof(double));
  if (C1) std::memcpy(C1, p->C1, 4 * sizeof(double));
  if (C2) std::memcpy(C2, p->C2, 4 * sizeof(double));
  return NSLCT_OK;
}

int nslct_plan_info(nslct_plan_t p, int* Nx, int* Ny, unsigned* flags, double abcd[16]) {
  if (!p) return NSLCT_E_ARG;
  if (Nx) *Nx = p->Nx;
  if (Ny) *Ny = p->Ny;
  if (flags) *flags = p->flags;
  if (abcd) std::memcpy(abcd, p->M, 16 * sizeof(double));
  return NSLCT_OK;
}

int nslct_forward(nslct_plan_t p, const void* in, void* out, nslct_stream_t stream) {
  return run_chain(p, in, out, stream, false, 0, p ? nslct_plan_passes(p) - 1 : 4);
}

int nslct_inverse(nslct_plan_t p, const void* in, void* out, nslct_stream_t stream) {
  return run_chain(p, in, out, stream, true, 0, p ? nslct_plan_passes(p) - 1 : 4);
}

int nslct_plan_passes(nslct_plan_t p) { return !p ? 0 : (p->y_only_h ? 3 : 5); }

// Field strides of a same-plan batch: at least one field, 16-byte aligned
// fields, and in-place only with equal strides.
static int check_many(nslct_plan_t p, int nbatch, const void* in, long long in_stride, const void* out,
                      long long out_stride) {
  if (!p || nbatch < 1 || p->padded) return p && p->padded ? NSLCT_E_UNSUPPORTED : NSLCT_E_ARG;
  const long long n = (long long)p->Nx * p->Ny;
  const size_t esz = p->prec == 1 ? 16 : 8;
  if (nbatch > 1 && (in_stride < n || out_stride < n)) return NSLCT_E_ARG;
  if (((size_t)in_stride * esz) % 16 || ((size_t)out_stride * esz) % 16) return NSLCT_E_ARG;
  if (in == out && in_stride != out_stride) return NSLCT_E_ARG;
  return NSLCT_OK;
}

int nslct_forward_many(nslct_plan_t p, int nbatch, const void* in, long long in_stride, void* out,
                       long long out_stride, nslct_stream_t stream) {
  const int rc = check_many(p, nbatch, in, in_stride, out, out_stride);
  if (rc != NSLCT_OK) return rc;
  return run_chain(p, in, out, stream, false, 0, nslct_plan_passes(p) - 1, nullptr, nbatch, in_stride, out_stride);
}

int nslct_inverse_many(nslct_plan_t p, int nbatch, const void* in, long long in_stride, void* out,
                       long long out_stride, nslct_stream_t stream) {
  const int rc = check_many(p, nbatch, in, in_stride, out, out_stride);
  if (rc != NSLCT_OK) return rc;
  return run_chain(p, in, out, stream, true, 0, nslct_plan_passes(p) - 1, nullptr, nbatch, in_stride, out_stride);
}

// One side stream and a pair of fork/join events per device, made on first
// use, for nslct_forward_group.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
// streams nslct_forward_group spreads its transforms over (the caller's + side streams)
#ifndef NSLCT_GROUP_STREAMS
#define NSLCT_GROUP_STREAMS 2
#endif
static_assert(NSLCT_GROUP_STREAMS >= 2 && NSLCT_GROUP_STREAMS <= 8, "group streams");
static std::mutex g_side_mu;
static SideStream g_side[64][NSLCT_GROUP_STREAMS - 1];

int nslct_forward_group(int n, const nslct_plan_t* plans, const void* const* in, void* const* out,
                        nslct_stream_t stream) {
  if (n < 1 || !plans || !in || !out) return NSLCT_E_ARG;
  for (int k = 0; k < n; ++k)
    if (!plans[k] || !in[k] || !out[k] || plans[k]->device != plans[0]->device) return NSLCT_E_ARG;
  const int dev = plans[0]->device;
  if (dev < 0 || dev >= 64) return NSLCT_E_ARG;
  DeviceGuard g(dev);
  if (!g.ok) return NSLCT_E_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n == 1) return nslct_forward(plans[0], in[0], out[0], stream);
  const int nside = std::min(n, NSLCT_GROUP_STREAMS) - 1;
  SideStream* ss = g_side[dev];
  {
    std::lock_guard<std::mutex> lock(g_side_mu);
    for (int i = 0; i < nside; ++i) {
      if (ss[i].s) continue;
      if (cudaStreamCreateWithFlags(&ss[i].s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ss[i].fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ss[i].join, cudaEventDisableTiming) != cudaSuccess)
        return NSLCT_E_CUDA;
    }
  }
  // transform k on stream k mod (nside + 1): the caller's stream, then the
  // side streams, each forked from and joined back to the caller's stream
  for (int i = 0; i < nside; ++i)
    if (cudaEventRecord(ss[i].fork, s) != cudaSuccess || cudaStreamWaitEvent(ss[i].s, ss[i].fork, 0) != cudaSuccess)
      return NSLCT_E_CUDA;
  int rc = NSLCT_OK;
  for (int k = 0; k < n && rc == NSLCT_OK; ++k) {
    const int j = k % (nside + 1);
    rc = nslct_forward(plans[k], in[k], out[k], j == 0 ? stream : reinterpret_cast<nslct_stream_t>(ss[j - 1].s));
  }
  for (int i = 0; i < nside; ++i)
    if (cudaEventRecord(ss[i].join, ss[i].s) != cudaSuccess || cudaStreamWaitEvent(s, ss[i].join, 0) != cudaSuccess)
      return NSLCT_E_CUDA;
  return rc;
}

int nslct_forward_masked(nslct_plan_t p, const void* in, const void* mask, void* out, nslct_stream_t stream) {
  if (!mask) return NSLCT_E_ARG;
  return run_chain(p, in, out, stream, false, 0, p ? nslct_plan_passes(p) - 1 : 4, mask);
}

int nslct_forward_pass(nslct_plan_t p, int pass, const void* in, void* out, nslct_stream_t stream) {
  if (!p || pass < 0 || pass >= nslct_plan_passes(p)) return NSLCT_E_ARG;
  return run_chain(p, in, out, stream, false, pass, pass);
}

int nslct_selftest_timeout(nslct_plan_t p, const void* in, void* out, nslct_stream_t stream) {
  if (!p || !in || !out || in == out) return NSLCT_E_ARG;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) return NSLCT_E_ARG;
  if (p->prec != 0 || p->mixed || p->padded || !pair_kernel_length(p->Ny)) return NSLCT_E_UNSUPPORTED;
  DeviceGuard g(p->device);
  if (!g.ok) return NSLCT_E_CUDA;
  PassDesc d[5];
  bool cols[5];
  build_schedule(p, in, out, false, d, cols);
  // the first pass, with each panel's barrier armed for 16 bytes more than
  // its copies bring and a 1 ms limit: every wait expires, every copy lands
  d[0].test_extra_tx = 16;
  d[0].wait_us = 1000;
  return launch(p, cols[0], d[0], reinterpret_cast<cudaStream_t>(stream));
}

int nslct_status(nslct_plan_t p) {
  if (!p) return NSLCT_E_ARG;
  DeviceGuard g(p->device);
  if (!g.ok) return NSLCT_E_CUDA;
  unsigned int word = 0;
  if (cudaMemcpy(&word, p->err, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return NSLCT_E_CUDA;
  if (word) {
    const unsigned int zero = 0;
    cudaMemcpy(p->err, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    return NSLCT_E_TIMEOUT;
  }
  return NSLCT_OK;
}

int nslct_destroy(nslct_plan_t p) {
  if (!p) return NSLCT_OK;
  DeviceGuard g(p->device);
  free_plan(p);
  return NSLCT_OK;
}

const char* nslct_strerror(int code) {
  switch (code) {
    case NSLCT_OK: return "success";
    case NSLCT_E_ARG: return "invalid argument";
    case NSLCT_E_NOT_SYMPLECTIC: return "ABCD matrix is not symplectic (Eq. Intro12)";
    case NSLCT_E_INFEASIBLE: return "no symmetric H gives a symmetric invertible B' = B - AH";
    case NSLCT_E_SIZE: return "unsupported field size (need 2^a or 3*2^a, 8..4096)";
    case NSLCT_E_CUDA: return "CUDA runtime error";
    case NSLCT_E_NOMEM: return "out of memory";
    case NSLCT_E_TIMEOUT: return "bounded device wait expired";
    case NSLCT_E_UNSUPPORTED: return "unsupported flag combination";
    default: return "unknown error code";
  }
}

const char* nslct_version(void) { return "nslct-gb300 0.1"; }

}  // extern "C"
