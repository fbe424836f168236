// Host FP64 math behind the parameter gradients (see grad_math.cpp).
#pragma once

namespace nslct {

// theta (10) of an ABCD matrix with invertible A; false when A is singular.
bool theta_from_abcd(const double* m, double* th);
// row-major 4x4 M(theta)
void abcd_from_theta(const double* th, double* m);
// H following theta from the reference h0 (row-major 2x2)
void h_of_theta(const double* th, const double* h0, double* h);
// d(H, B', C1, C2 symmetric entries)/d theta, row-major 12 x 10
void chirp_jacobian(const double* th, const double* h0, double* jac);

// Constants the FP64 finalisation kernel needs (by value).
struct GradFinal {
  double factor[4][3];  // slot s, entry k: d loss/d chirp entry = factor * S_k
  double jac[120];      // chirp_jacobian at the plan's theta
  int nblk[4];          // CTAs (partial-sum rows) of each accumulating pass
  int stride;           // rows reserved per pass in the partials buffer
  int want_theta;       // write the 10 theta gradients
};

}  // namespace nslct
