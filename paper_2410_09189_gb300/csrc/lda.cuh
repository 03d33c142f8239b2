#pragma once
// LDA (Slater exchange + PZ81 correlation, spin-unpolarised) at one point, and the mixed
// path's float32 increment of its potential; shared by the xc kernels and the persistent
// Hartree solve's closing phase.

#include <math.h>

#include "rmgtd_internal.cuh"

namespace rmgtd {

// ---------------------------------------------------------------------------------------
// LDA (Slater exchange + Perdew-Zunger 1981 correlation, spin-unpolarised), float64.
// The roots and the reciprocal are Newton iterations in float64 seeded from float32:
//   z = rho^(-1/3):   z <- z (4 - rho z^3) / 3        (one step from rcbrtf)
//   u = r_s^(-1/2):   u <- u (3 - r_s u^2) / 2        (one step from rsqrtf)
//   q = 1/den:        q <- q (2 - den q)              (one step from 1/float)
// each step squares the relative error e -> ~2 e^2 (cube root), 1.5 e^2 (inverse square
// root), e^2 (reciprocal): from float32 seeds (e <= 2^-22) one step leaves <= 2^-43 ~ 1e-13,
// far below anything the SCF threshold resolves, at a third of the float64 operations.
// Then rho^(1/3) = rho z^2, r_s = (3/(4 pi))^(1/3) z, 1/r_s = rho z^2 / (3/(4 pi))^(1/3).
__device__ __forceinline__ void lda_point(double rho, double& vxc, double& exc) {
  if (!(rho >= kRhoFloor)) {
    vxc = 0.0;
    exc = 0.0;
    return;
  }
  constexpr double kC3pi = 0.98474502184269641;   // (3/pi)^(1/3)
  constexpr double kCrs = 0.62035049089940009;    // (3/(4 pi))^(1/3)
  double z = (double)rcbrtf((float)rho);
  z = z * (4.0 - rho * z * z * z) * (1.0 / 3.0);
  const double c13 = rho * z * z;                 // rho^(1/3)
  const double t = kC3pi * c13;
  const double ex = -0.75 * t, vx = -t;
  const double rs = kCrs * z;
  double ec, dec;
  if (rs >= 1.0) {
    double u = (double)rsqrtf((float)rs);
    u = u * (3.0 - rs * u * u) * 0.5;
    const double sq = rs * u;                     // sqrt(r_s)
    const double den = 1.0 + 1.0529 * sq + 0.3334 * rs;
    double q = (double)(1.0f / (float)den);
    q = q * (2.0 - den * q);
    ec = -0.1423 * q;
    dec = 0.1423 * (0.5 * 1.0529 * u + 0.3334) * q * q;
  } else {
    const double lr = log(rs);
    const double irs = c13 * (1.0 / kCrs);        // 1 / r_s
    ec = 0.0311 * lr - 0.048 + 0.0020 * rs * lr - 0.0116 * rs;
    dec = 0.0311 * irs + 0.0020 * (lr + 1.0) - 0.0116;
  }
  vxc = vx + ec - rs * (1.0 / 3.0) * dec;
  exc = ex + ec;
}

// Increment V_xc(rho0 + d) - V_xc(rho0) of the mixed path in float32 arithmetic on the
// increment itself.  Every difference of the functional is rewritten as d times a smooth
// factor, so float32 rounding is relative to the increment, not to V_xc:
//   c = rho^(1/3):  c - c0 = d / (c^2 + c c0 + c0^2)            (c^3 - c0^3 = d)
//   r_s = k / c:    r_s - r_s0 = -k (c - c0) / (c c0)
//   r_s >= 1:  V_c = gamma Nn / Dd^2, Nn = 1 + 7/6 b1 s + 4/3 b2 r_s, Dd = 1 + b1 s + b2 r_s,
//              s = sqrt(r_s), s - s0 = (r_s - r_s0) / (s + s0),
//              Nn/Dd^2 - Nn0/Dd0^2 = (dNn Dd0^2 - Nn0 dDd (Dd + Dd0)) / (Dd^2 Dd0^2)
//   r_s <  1:  V_c = A ln r_s + (B - A/3) + 2/3 C r_s ln r_s + (2D - C)/3 r_s,
//              ln r_s - ln r_s0 = log1p((r_s - r_s0) / r_s0),
//              r_s ln r_s - r_s0 ln r_s0 = (r_s - r_s0) ln r_s + r_s0 (ln r_s - ln r_s0)
// (the PZ81 potential of lda_point, V_c = eps_c - (r_s/3) d eps_c/d r_s, regrouped).  Points
// within a factor 2 of the density floor or whose two densities sit on different sides of
// r_s = 1 (or within float32 rounding of it) take both float64 evaluations instead; points
// whose two densities are both well below the floor give 0.
// r0 = (float)rho0 (rounded to nearest); rho0 itself is read only on the float64 path.
__device__ __forceinline__ float dvxc_increment(const double* rho0p, float r0, float d) {
  constexpr float kC3pi = 0.98474502f, kCrs = 0.62035049f;
  constexpr float b1 = 1.0529f, b2 = 0.3334f, gam = -0.1423f;
  constexpr float A = 0.0311f, C = 0.0020f, D = -0.0116f;
  // the floor decision of float64 is certain outside +-1e-4 of the floor (float32 rounding
  // of r0 and r1 is ~1e-7 relative)
  constexpr float kLo = (float)(kRhoFloor * (1.0 - 1e-4)), kHi = (float)(kRhoFloor * (1.0 + 1e-4));
  const float r1 = r0 + d;
  // both densities below the floor (vacuum): V_xc = 0 on both sides
  if (r0 < kLo && r1 < kLo) return 0.0f;
  bool easy = r0 > kHi && r1 > kHi;
  float out = 0.0f;
  if (easy) {
    const float c0 = cbrtf(r0), c1 = cbrtf(r1);
    const float dc = d / (c1 * c1 + c1 * c0 + c0 * c0);
    const float rs0 = kCrs / c0, rs1 = kCrs / c1;
    const float drs = -kCrs * dc / (c1 * c0);
    const bool hi0 = rs0 >= 1.0f;
    easy = (hi0 == (rs1 >= 1.0f)) && fabsf(rs0 - 1.0f) > 1e-5f && fabsf(rs1 - 1.0f) > 1e-5f;
    float dvc;
    if (hi0) {
      const float s0 = sqrtf(rs0), s1 = sqrtf(rs1);
      const float ds = drs / (s1 + s0);
      const float D0 = 1.0f + b1 * s0 + b2 * rs0, D1 = 1.0f + b1 * s1 + b2 * rs1;
      const float N0 = 1.0f + (7.0f / 6.0f) * b1 * s0 + (4.0f / 3.0f) * b2 * rs0;
      const float dN = (7.0f / 6.0f) * b1 * ds + (4.0f / 3.0f) * b2 * drs;
      const float dD = b1 * ds + b2 * drs;
      dvc = gam * (dN * D0 * D0 - N0 * dD * (D1 + D0)) / (D1 * D1 * D0 * D0);
    } else {
      const float lr0 = logf(rs0);
      const float dlr = log1pf(drs / rs0);
      dvc = A * dlr + (2.0f / 3.0f) * C * (drs * (lr0 + dlr) + rs0 * dlr) +
            ((2.0f * D - C) / 3.0f) * drs;
    }
    out = -kC3pi * dc + dvc;
  }
  if (!easy) {
    const double rho0 = *rho0p;
    double v1, v0, e;
    lda_point(rho0 + (double)d, v1, e);
    lda_point(rho0, v0, e);
    out = (float)(v1 - v0);
  }
  return out;
}

}  // namespace rmgtd
