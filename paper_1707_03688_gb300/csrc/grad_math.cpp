// Host FP64 math for the parameter gradients of nslct_backward.
//
// Parametrisation (the 10 degrees of freedom of an ABCD matrix, Sec. 1): for
// invertible A,
//   M(theta) = (I,0; C,I) (L,0; 0,L^-T) (I,B; 0,I) = (L, L B; C L, C L B + L^-T)
// with C, B symmetric and L = A; theta = (c11,c12,c22, l11,l12,l21,l22, b11,b12,b22).
// H follows theta by moving a reference H0 along the normal r of the feasible
// plane r.h = b12 - b21 (r = (-a21, a11 - a22, a12), the condition that
// B - AH be symmetric): h = h0 + r (rhs - r.h0) / (r.r). That map is smooth, and
// the chirp matrices (H, B', C1, C2) of Eq. Bnonsym08 are smooth functions of
// theta, whose 12 x 10 Jacobian is taken by the complex-step derivative
// Im f(theta + i s e_k) / s, exact to rounding because every step is analytic.
#include <complex>
#include <cmath>
#include <cstring>

#include "grad_math.h"

namespace nslct {

namespace {

template <typename T>
struct M2 {
  T a, b, c, d;  // [[a, b], [c, d]]
};
template <typename T> M2<T> mul(const M2<T>& x, const M2<T>& y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
template <typename T> M2<T> sub(const M2<T>& x, const M2<T>& y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }
template <typename T> M2<T> add(const M2<T>& x, const M2<T>& y) { return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
template <typename T> M2<T> inv(const M2<T>& x) {
  const T det = x.a * x.d - x.b * x.c;
  return {x.d / det, -x.b / det, -x.c / det, x.a / det};
}
template <typename T> M2<T> transpose(const M2<T>& x) { return {x.a, x.c, x.b, x.d}; }

// ABCD blocks of M(theta)
template <typename T>
void blocks_of_theta(const T* th, M2<T>& A, M2<T>& B, M2<T>& C, M2<T>& D) {
  const M2<T> c = {th[0], th[1], th[1], th[2]};
  const M2<T> l = {th[3], th[4], th[5], th[6]};
  const M2<T> b = {th[7], th[8], th[8], th[9]};
  A = l;
  B = mul(l, b);
  C = mul(c, l);
  D = add(mul(C, b), transpose(inv(l)));
}

template <typename T>
M2<T> h_rule(const M2<T>& A, const M2<T>& B, const double* h0) {
  const T r0 = -A.c, r1 = A.a - A.d, r2 = A.b;
  const T rhs = B.b - B.c;
  const T h11 = T(h0[0]), h12 = T(0.5 * (h0[1] + h0[2])), h22 = T(h0[3]);
  const T rr = r0 * r0 + r1 * r1 + r2 * r2;  // r.r without conjugation (analytic)
  if (std::abs(rr) < 1e-24) return {h11, h12, h12, h22};
  const T lam = (rhs - (r0 * h11 + r1 * h12 + r2 * h22)) / rr;
  const T v0 = h11 + lam * r0, v1 = h12 + lam * r1, v2 = h22 + lam * r2;
  return {v0, v1, v1, v2};
}

// (H, B', C1, C2) symmetric entries in the order h11 h12 h22, b'11 b'12 b'22,
// c1_11 c1_12 c1_22, c2_11 c2_12 c2_22.
template <typename T>
void chirp_vec(const T* th, const double* h0, T* out) {
  M2<T> A, B, C, D;
  blocks_of_theta(th, A, B, C, D);
  const M2<T> H = h_rule(A, B, h0);
  const M2<T> I = {T(1), T(0), T(0), T(1)};
  const M2<T> bp = sub(B, mul(A, H));
  const M2<T> dp = sub(D, mul(C, H));
  const M2<T> bpi = inv(bp);
  const M2<T> c2 = mul(bpi, sub(A, I));
  const M2<T> c1 = mul(sub(dp, I), bpi);
  const M2<T>* mats[4] = {&H, &bp, &c1, &c2};
  for (int k = 0; k < 4; ++k) {
    out[3 * k + 0] = mats[k]->a;
    out[3 * k + 1] = T(0.5) * (mats[k]->b + mats[k]->c);
    out[3 * k + 2] = mats[k]->d;
  }
}

}  // namespace

bool theta_from_abcd(const double* m, double* th) {
  const double a = m[0], b = m[1], c = m[4], d = m[5];
  const double det = a * d - b * c;
  if (!(std::fabs(det) > 1e-12)) return false;
  const M2<double> A = {a, b, c, d};
  const M2<double> Bm = {m[2], m[3], m[6], m[7]};
  const M2<double> Cm = {m[8], m[9], m[12], m[13]};
  const M2<double> Ai = inv(A);
  const M2<double> cs = mul(Cm, Ai);  // C A^-1 (symmetric for symplectic M)
  const M2<double> bs = mul(Ai, Bm);  // A^-1 B (symmetric for symplectic M)
  th[0] = cs.a; th[1] = 0.5 * (cs.b + cs.c); th[2] = cs.d;
  th[3] = a; th[4] = b; th[5] = c; th[6] = d;
  th[7] = bs.a; th[8] = 0.5 * (bs.b + bs.c); th[9] = bs.d;
  return true;
}

void abcd_from_theta(const double* th, double* m) {
  M2<double> A, B, C, D;
  blocks_of_theta(th, A, B, C, D);
  const double out[16] = {A.a, A.b, B.a, B.b, A.c, A.d, B.c, B.d, C.a, C.b, D.a, D.b, C.c, C.d, D.c, D.d};
  std::memcpy(m, out, sizeof(out));
}

void h_of_theta(const double* th, const double* h0, double* h) {
  M2<double> A, B, C, D;
  blocks_of_theta(th, A, B, C, D);
  const M2<double> H = h_rule(A, B, h0);
  h[0] = H.a; h[1] = H.b; h[2] = H.c; h[3] = H.d;
}

void chirp_jacobian(const double* th, const double* h0, double* jac) {
  using Z = std::complex<double>;
  const double step = 1e-30;
  for (int k = 0; k < 10; ++k) {
    Z tz[10];
    for (int i = 0; i < 10; ++i) tz[i] = Z(th[i], i == k ? step : 0.0);
    Z out[12];
    chirp_vec(tz, h0, out);
    for (int r = 0; r < 12; ++r) jac[r * 10 + k] = out[r].imag() / step;
  }
}

}  // namespace nslct
