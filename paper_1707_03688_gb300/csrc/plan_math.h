// FP64 host math of the plan (see plan.cpp).
#pragma once

#include <cstdint>

#include "internal.h"

namespace nslct {

struct Mat2 {
  double m00, m01, m10, m11;  // row-major 2x2
};

struct Decomp {
  Mat2 H, Bp, C1, C2;
  double det_bp;    // det(B - AH) before symmetrisation
  double bp_asym;   // |(B - AH)_12 - (B - AH)_21|
};

constexpr double kDetFloor = 1e-3;   // |det B'| below this counts as singular
constexpr int kGrid2D = 241;         // lattice per axis on the feasible plane
constexpr int kGrid3D = 41;          // lattice per axis when every symmetric H is feasible
constexpr int kZoom2D = 21;          // refinement window points per axis on the plane
constexpr int kZoom3D = 9;           // refinement window points per axis in 3D
constexpr int kStarts = 6;           // lattice minima refined independently
constexpr double kStepMin = 1e-11;   // refinement stops below this window half-width

Mat2 mat2_mul(const Mat2& a, const Mat2& b);
Mat2 mat2_sub(const Mat2& a, const Mat2& b);
Mat2 mat2_neg(const Mat2& a);
double mat2_det(const Mat2& a);
Mat2 mat2_inv(const Mat2& a);
Mat2 mat2_symmetrise(const Mat2& a);
void split_blocks(const double* m, Mat2& a, Mat2& b, Mat2& c, Mat2& d);

double symplectic_residual(const double* m);
bool project_sp4(const double* m, double* out);
Decomp decompose(const double* m, const Mat2& h);
double gamma_ratio(const Mat2& c);
double ha_objective(const double* m, const Mat2& h);
int choose_h_ha(const double* m, Mat2* h_out);
int choose_h_lc(const double* m, Mat2* h_out);
int choose_h_lc_y(const double* m, Mat2* h_out);
uint64_t turns_q64(double x);
Chirp chirp_from(const Mat2& c, double da, double db);
void fill_chirps(nslct_plan_s* p);

}  // namespace nslct
