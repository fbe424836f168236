// Host-side plan: FP64 derivation of the CM-CC-CM-CC chain parameters.
//
// Steps (Sec. 4.B):
//   1. check the ABCD matrix against Eq. Intro12 (or project it onto Sp(4));
//   2. choose the symmetric H: the high-accuracy criterion of Eq. HA24, the
//      low-complexity closed forms of Eqs. LC08/LC10, or a caller-given H;
//   3. B' = B - AH, D' = D - CH, C2 = B'^{-1}(A - I), C1 = (D' - I)B'^{-1}
//      (Eq. Bnonsym08);
//   4. turn every chirp matrix into exact fixed-point phase coefficients.
#include <cmath>
#include <cstring>
#include <limits>

#include "plan_math.h"

namespace nslct {

static constexpr double kTwoPi = 6.283185307179586476925286766559;

// ---------------------------------------------------------------- 2x2 helpers

Mat2 mat2_mul(const Mat2& a, const Mat2& b) {
  return {a.m00 * b.m00 + a.m01 * b.m10, a.m00 * b.m01 + a.m01 * b.m11,
          a.m10 * b.m00 + a.m11 * b.m10, a.m10 * b.m01 + a.m11 * b.m11};
}
Mat2 mat2_sub(const Mat2& a, const Mat2& b) { return {a.m00 - b.m00, a.m01 - b.m01, a.m10 - b.m10, a.m11 - b.m11}; }
double mat2_det(const Mat2& a) { return a.m00 * a.m11 - a.m01 * a.m10; }
Mat2 mat2_inv(const Mat2& a) {
  const double d = mat2_det(a);
  return {a.m11 / d, -a.m01 / d, -a.m10 / d, a.m00 / d};
}
Mat2 mat2_symmetrise(const Mat2& a) {
  const double o = 0.5 * (a.m01 + a.m10);
  return {a.m00, o, o, a.m11};
}
static const Mat2 kEye = {1, 0, 0, 1};

void split_blocks(const double* m, Mat2& a, Mat2& b, Mat2& c, Mat2& d) {
  a = {m[0], m[1], m[4], m[5]};
  b = {m[2], m[3], m[6], m[7]};
  c = {m[8], m[9], m[12], m[13]};
  d = {m[10], m[11], m[14], m[15]};
}

// ---------------------------------------------------------------- symplectic check / projection

// max |M^T J M - J| with J = (0, I; -I, 0); zero iff Eq. Intro16 holds.
double symplectic_residual(const double* m) {
  double j[16] = {0};
  j[2] = 1; j[7] = 1; j[8] = -1; j[13] = -1;
  double jm[16], r = 0;
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) {
      double s = 0;
      for (int l = 0; l < 4; ++l) s += j[i * 4 + l] * m[l * 4 + k];
      jm[i * 4 + k] = s;
    }
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) {
      double s = 0;
      for (int l = 0; l < 4; ++l) s += m[l * 4 + i] * jm[l * 4 + k];
      r = std::fmax(r, std::fabs(s - j[i * 4 + k]));
    }
  return r;
}

// Gauss-Jordan inverse of a 4x4 with partial pivoting; false if singular.
static bool inv4(const double* m, double* out) {
  double a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 8; ++k) a[i][k] = k < 4 ? m[i * 4 + k] : (k - 4 == i ? 1.0 : 0.0);
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    if (std::fabs(a[piv][c]) < 1e-300) return false;
    if (piv != c)
      for (int k = 0; k < 8; ++k) std::swap(a[c][k], a[piv][k]);
    const double s = 1.0 / a[c][c];
    for (int k = 0; k < 8; ++k) a[c][k] *= s;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      const double f = a[r][c];
      if (f != 0.0)
        for (int k = 0; k < 8; ++k) a[r][k] -= f * a[c][k];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) out[i * 4 + k] = a[i][k + 4];
  return true;
}

// Nearest-symplectic clean-up: X <- (X + J^T X^{-T} J) / 2 until it stops moving.
// Every symplectic matrix is a fixed point (J^T X^{-T} J = X when X^T J X = J).
bool project_sp4(const double* m, double* out) {
  double x[16];
  std::memcpy(x, m, sizeof(x));
  for (int it = 0; it < 100; ++it) {
    double xi[16];
    if (!inv4(x, xi)) return false;
    // y = J^T X^{-T} J ; (X^{-T})_{ik} = xi[k][i]
    // J = [[0, I], [-I, 0]] acts on 2x2 blocks: with X^{-T} = [[P, Q], [R, S]],
    // J^T X^{-T} J = [[S, -R], [-Q, P]].
    double t[16];
    for (int i = 0; i < 4; ++i)
      for (int k = 0; k < 4; ++k) t[i * 4 + k] = xi[k * 4 + i];
    double y[16];
    for (int i = 0; i < 2; ++i)
      for (int k = 0; k < 2; ++k) {
        const double P = t[i * 4 + k], Q = t[i * 4 + k + 2];
        const double R = t[(i + 2) * 4 + k], S = t[(i + 2) * 4 + k + 2];
        y[i * 4 + k] = S;
        y[i * 4 + k + 2] = -R;
        y[(i + 2) * 4 + k] = -Q;
        y[(i + 2) * 4 + k + 2] = P;
      }
    double delta = 0;
    for (int i = 0; i < 16; ++i) {
      const double nx = 0.5 * (x[i] + y[i]);
      delta = std::fmax(delta, std::fabs(nx - x[i]));
      x[i] = nx;
    }
    if (delta < 1e-17) break;
  }
  std::memcpy(out, x, sizeof(x));
  return true;
}

// ---------------------------------------------------------------- decomposition

Decomp decompose(const double* m, const Mat2& h_in) {
  Mat2 a, b, c, d;
  split_blocks(m, a, b, c, d);
  Decomp r;
  r.H = mat2_symmetrise(h_in);
  const Mat2 bp = mat2_sub(b, mat2_mul(a, r.H));
  const Mat2 dp = mat2_sub(d, mat2_mul(c, r.H));
  r.det_bp = mat2_det(bp);
  r.bp_asym = std::fabs(bp.m01 - bp.m10);
  r.Bp = mat2_symmetrise(bp);
  if (r.det_bp == 0.0 || !std::isfinite(r.det_bp)) {
    r.C1 = r.C2 = {0, 0, 0, 0};
    return r;
  }
  const Mat2 bpi = mat2_inv(bp);
  const Mat2 c2 = mat2_mul(bpi, mat2_sub(a, kEye));
  const Mat2 c1 = mat2_mul(mat2_sub(dp, kEye), bpi);
  r.C1 = mat2_symmetrise(c1);
  r.C2 = mat2_symmetrise(c2);
  return r;
}

// Eq. HA16
double gamma_ratio(const Mat2& c) {
  const double o = std::fabs(0.5 * (c.m01 + c.m10));
  return (std::fabs(c.m00) + o + 1.0) * (o + std::fabs(c.m11) + 1.0);
}

// Eq. HA24 objective; +inf when B' is (numerically) singular.
double ha_objective(const double* m, const Mat2& h) {
  const Decomp r = decompose(m, h);
  if (!(std::fabs(r.det_bp) >= kDetFloor)) return std::numeric_limits<double>::infinity();
  return gamma_ratio(r.C1) * gamma_ratio(r.Bp) * gamma_ratio(r.C2) * gamma_ratio(r.H);
}

static Mat2 h_of(const double v[3]) { return {v[0], v[1], v[1], v[2]}; }

namespace {

// Search space for H: either the 2D feasible plane h = h0 + s e1 + t e2, or all
// of R^3 when every symmetric H is feasible.
struct HSpace {
  int dim;
  double h0[3], e1[3], e2[3];
  void point(const double* c, double* v) const {
    if (dim == 3) { v[0] = c[0]; v[1] = c[1]; v[2] = c[2]; return; }
    for (int i = 0; i < 3; ++i) v[i] = h0[i] + c[0] * e1[i] + c[1] * e2[i];
  }
  double eval(const double* m, const double* c) const {
    double v[3];
    point(c, v);
    return ha_objective(m, h_of(v));
  }
};

struct Cand {
  double f;
  double c[3];
};

}  // namespace

// Symmetric H for which B - AH is symmetric lie on the plane r . (h11, h12, h22) = rhs
// with r = (-a21, a11 - a22, a12), rhs = b12 - b21 (the (1,2) and (2,1) entries of
// B - AH equal each other). The criterion of Eq. HA24 is minimised over that set:
//   1. a lattice over [-R, R]^dim, R = 6 max(1, max|M|) (241^2 on the plane,
//      41^3 when r = 0 and rhs = 0), infeasible points (|det B'| < 1e-3) skipped;
//   2. from each of the best few lattice points that lie apart, a shrinking
//      window: evaluate a full grid of offsets around the current point, move
//      to its best entry, quarter the window; stop below 1e-11. A full window
//      is used because the absolute values of Eq. HA16 give the objective kinks
//      that defeat moves along fixed axes.
int choose_h_ha(const double* m, Mat2* h_out) {
  Mat2 a, b, c, d;
  split_blocks(m, a, b, c, d);
  const double r[3] = {-a.m10, a.m00 - a.m11, a.m01};
  const double rhs = b.m01 - b.m10;
  const double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  double mmax = 1.0;
  for (int i = 0; i < 16; ++i) mmax = std::fmax(mmax, std::fabs(m[i]));
  const double R = 6.0 * mmax;

  HSpace sp{};
  int G, W;
  if (rn > 1e-12) {
    sp.dim = 2;
    const double n0[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    for (int i = 0; i < 3; ++i) sp.h0[i] = n0[i] * rhs / rn;
    // e1: Gram-Schmidt of the coordinate axis least aligned with r; e2 = n0 x e1
    int ax = 0;
    for (int i = 1; i < 3; ++i)
      if (std::fabs(n0[i]) < std::fabs(n0[ax])) ax = i;
    double e1[3] = {0, 0, 0};
    e1[ax] = 1.0;
    const double dp = e1[0] * n0[0] + e1[1] * n0[1] + e1[2] * n0[2];
    for (int i = 0; i < 3; ++i) e1[i] -= dp * n0[i];
    const double e1n = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; ++i) sp.e1[i] = e1[i] / e1n;
    sp.e2[0] = n0[1] * sp.e1[2] - n0[2] * sp.e1[1];
    sp.e2[1] = n0[2] * sp.e1[0] - n0[0] * sp.e1[2];
    sp.e2[2] = n0[0] * sp.e1[1] - n0[1] * sp.e1[0];
    G = kGrid2D;
    W = kZoom2D;
  } else {
    if (std::fabs(rhs) > 1e-12) return NSLCT_E_INFEASIBLE;
    sp.dim = 3;
    G = kGrid3D;
    W = kZoom3D;
  }
  const double step0 = 2.0 * R / (G - 1);

  // 1. lattice; keep the kStarts best points that are > 2.5 steps apart
  Cand best[kStarts];
  int nbest = 0;
  const long total = sp.dim == 2 ? (long)G * G : (long)G * G * G;
  for (long idx = 0; idx < total; ++idx) {
    double cc[3];
    long rem = idx;
    for (int k = sp.dim - 1; k >= 0; --k) { cc[k] = -R + step0 * (double)(rem % G); rem /= G; }
    const double f = sp.eval(m, cc);
    if (!std::isfinite(f)) continue;
    // replace a near neighbour if this point is better, else insert by rank
    int near = -1;
    for (int q = 0; q < nbest; ++q) {
      double dmax = 0;
      for (int k = 0; k < sp.dim; ++k) dmax = std::fmax(dmax, std::fabs(cc[k] - best[q].c[k]));
      if (dmax <= 2.5 * step0) { near = q; break; }
    }
    if (near >= 0) {
      if (f < best[near].f) {
        best[near].f = f;
        for (int k = 0; k < 3; ++k) best[near].c[k] = cc[k];
      }
    } else if (nbest < kStarts) {
      best[nbest].f = f;
      for (int k = 0; k < 3; ++k) best[nbest].c[k] = cc[k];
      ++nbest;
    } else {
      int worst = 0;
      for (int q = 1; q < nbest; ++q)
        if (best[q].f > best[worst].f) worst = q;
      if (f < best[worst].f) {
        best[worst].f = f;
        for (int k = 0; k < 3; ++k) best[worst].c[k] = cc[k];
      }
    }
  }
  if (nbest == 0) return NSLCT_E_INFEASIBLE;

  // 2. shrinking-window refinement of every start
  double fbest = std::numeric_limits<double>::infinity();
  double cbest[3] = {0, 0, 0};
  for (int q = 0; q < nbest; ++q) {
    double cur[3] = {best[q].c[0], best[q].c[1], best[q].c[2]};
    double fcur = best[q].f;
    double half = step0;
    while (half > kStepMin) {
      double cand_best[3] = {cur[0], cur[1], cur[2]};
      double fc = fcur;
      const long wtotal = sp.dim == 2 ? (long)W * W : (long)W * W * W;
      for (long idx = 0; idx < wtotal; ++idx) {
        double cc[3] = {cur[0], cur[1], cur[2]};
        long rem = idx;
        for (int k = sp.dim - 1; k >= 0; --k) {
          const double off = -1.0 + 2.0 * (double)(rem % W) / (double)(W - 1);
          cc[k] = cur[k] + half * off;
          rem /= W;
        }
        const double f = sp.eval(m, cc);
        if (f < fc) { fc = f; cand_best[0] = cc[0]; cand_best[1] = cc[1]; cand_best[2] = cc[2]; }
      }
      fcur = fc;
      cur[0] = cand_best[0]; cur[1] = cand_best[1]; cur[2] = cand_best[2];
      half *= 0.25;
    }
    if (fcur < fbest) { fbest = fcur; cbest[0] = cur[0]; cbest[1] = cur[1]; cbest[2] = cur[2]; }
  }
  double v[3];
  sp.point(cbest, v);
  *h_out = h_of(v);
  return NSLCT_OK;
}

// Eqs. LC08/LC10: one-parameter H; the candidate with the lower Eq. HA24 value wins.
// Returns NSLCT_E_INFEASIBLE when neither candidate exists or gives |det B'| >= floor.
int choose_h_lc(const double* m, Mat2* h_out) {
  Mat2 a, b, c, d;
  split_blocks(m, a, b, c, d);
  double best = std::numeric_limits<double>::infinity();
  Mat2 bh = {0, 0, 0, 0};
  if (std::fabs(a.m10) > 1e-12) {
    const Mat2 h = {(b.m10 - b.m01) / a.m10, 0, 0, 0};
    const double f = ha_objective(m, h);
    if (f < best) { best = f; bh = h; }
  }
  if (std::fabs(a.m01) > 1e-12) {
    const Mat2 h = {0, 0, 0, (b.m01 - b.m10) / a.m01};
    const double f = ha_objective(m, h);
    if (f < best) { best = f; bh = h; }
  }
  if (!std::isfinite(best)) return NSLCT_E_INFEASIBLE;
  *h_out = bh;
  return NSLCT_OK;
}

// Eq. LC10 only: H = (0,0;0,h), h = (b12 - b21)/a12, when a12 != 0 and B' is invertible.
int choose_h_lc_y(const double* m, Mat2* h_out) {
  Mat2 a, b, c, d;
  split_blocks(m, a, b, c, d);
  if (!(std::fabs(a.m01) > 1e-12)) return NSLCT_E_INFEASIBLE;
  const Mat2 h = {0, 0, 0, (b.m01 - b.m10) / a.m01};
  if (!std::isfinite(ha_objective(m, h))) return NSLCT_E_INFEASIBLE;
  *h_out = h;
  return NSLCT_OK;
}

// ---------------------------------------------------------------- fixed-point chirps

// x mod 1 as a Q0.64 fraction of a turn, in two's complement. The fraction
// is split off with trunc (x - trunc(x) is exact) and scaled as it is; taking
// x - floor(x) instead would compute 1 + x for negative x and round away the
// low bits of a small coefficient, which a^2 ~ 4e6 then multiplies.
uint64_t turns_q64(double x) {
  if (!std::isfinite(x)) return 0;
  const double xf = x - std::trunc(x);  // exact, |xf| < 1, sign of x
  if (xf >= 0.0) return (uint64_t)std::ldexp(xf, 64);
  return (uint64_t)0 - (uint64_t)std::ldexp(-xf, 64);
}

// chirp exp(j/2 (c11 a^2 da^2 + 2 c12 a b da db + c22 b^2 db^2)) in turns
Chirp chirp_from(const Mat2& c, double da, double db) {
  const double c12 = 0.5 * (c.m01 + c.m10);
  Chirp r;
  r.k11 = turns_q64(c.m00 * da * da / (2.0 * kTwoPi));
  r.k12 = turns_q64(c12 * da * db / kTwoPi);
  r.k22 = turns_q64(c.m11 * db * db / (2.0 * kTwoPi));
  return r;
}

Mat2 mat2_neg(const Mat2& a) { return {-a.m00, -a.m01, -a.m10, -a.m11}; }

void fill_chirps(nslct_plan_s* p) {
  const double dwx = kTwoPi / (p->Nx * p->dx);
  const double dwy = kTwoPi / (p->Ny * p->dy);
  const Mat2 H = {p->H[0], p->H[1], p->H[2], p->H[3]};
  const Mat2 Bp = {p->Bp[0], p->Bp[1], p->Bp[2], p->Bp[3]};
  const Mat2 C1 = {p->C1[0], p->C1[1], p->C1[2], p->C1[3]};
  const Mat2 C2 = {p->C2[0], p->C2[1], p->C2[2], p->C2[3]};
  // forward: CC^H uses CM^{-H} at the frequency spacing (Eq. BasicCC20)
  p->fwd_chi_h = chirp_from(mat2_neg(H), dwx, dwy);
  p->fwd_cm_c2 = chirp_from(C2, p->dx, p->dy);
  p->fwd_chi_bp = chirp_from(mat2_neg(Bp), dwx, dwy);
  p->fwd_cm_c1 = chirp_from(C1, p->dx, p->dy);
  // inverse (Eq. CCCMCCCM04): CM^{-C1}, CC^{-B'} (= F^-1 CM^{+B'} F), CM^{-C2}, CC^{-H}
  p->inv_cm_c1 = chirp_from(mat2_neg(C1), p->dx, p->dy);
  p->inv_chi_bp = chirp_from(Bp, dwx, dwy);
  p->inv_cm_c2 = chirp_from(mat2_neg(C2), p->dx, p->dy);
  p->inv_chi_h = chirp_from(H, dwx, dwy);
}

}  // namespace nslct
