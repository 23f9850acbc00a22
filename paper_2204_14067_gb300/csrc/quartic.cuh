// Device form of the exact line search's step rule: the minimiser over
// s >= 0 of the quartic c0 + c1 s + c2 s^2 + c3 s^3 + c4 s^4, among 0 and the
// positive real roots of its derivative (closed-form cubic roots, Newton
// polished).  Shared by the batched PR+ phase and the distance-geometry BM
// phase, which keep their control scalars on the device.
#pragma once

namespace bm {

__device__ inline double poly4d(const double* c, double s) { return (((c[4] * s + c[3]) * s + c[2]) * s + c[1]) * s + c[0]; }
__device__ inline double dpoly4d(const double* c, double s) { return ((4 * c[4] * s + 3 * c[3]) * s + 2 * c[2]) * s + c[1]; }
__device__ inline double ddpoly4d(const double* c, double s) { return (12 * c[4] * s + 6 * c[3]) * s + 2 * c[2]; }

// argmin over s >= 0 of the quartic: candidates 0 and the positive real roots
// of its derivative (Cardano / trigonometric form, Newton-polished)
__device__ inline double quartic_argmin_d(const double* c) {
  double roots[3];
  int nr = 0;
  const double a3 = 4 * c[4], a2 = 3 * c[3], a1 = 2 * c[2], a0 = c[1];
  const double scale = fmax(fmax(fabs(a3), fabs(a2)), fmax(fmax(fabs(a1), fabs(a0)), 1e-300));
  if (fabs(a3) > 1e-14 * scale) {
    const double p2 = a2 / a3, p1 = a1 / a3, p0 = a0 / a3;
    const double q = (3 * p1 - p2 * p2) / 9.0;
    const double r = (9 * p2 * p1 - 27 * p0 - 2 * p2 * p2 * p2) / 54.0;
    const double disc = q * q * q + r * r;
    if (disc > 0) {
      const double sq = sqrt(disc);
      roots[nr++] = cbrt(r + sq) + cbrt(r - sq) - p2 / 3.0;
    } else {
      const double th = acos(fmax(-1.0, fmin(1.0, q < 0 ? r / sqrt(-q * q * q) : 0.0)));
      const double mm = 2.0 * sqrt(fmax(0.0, -q));
      for (int t = 0; t < 3; ++t) roots[nr++] = mm * cos((th + 2.0 * 3.141592653589793 * t) / 3.0) - p2 / 3.0;
    }
  } else if (fabs(a2) > 1e-14 * scale) {
    const double dd = a1 * a1 - 4 * a2 * a0;
    if (dd >= 0) {
      const double sq = sqrt(dd);
      const double qq = -0.5 * (a1 + (a1 >= 0 ? sq : -sq));
      if (qq != 0) {
        roots[nr++] = qq / a2;
        roots[nr++] = a0 / qq;
      }
    }
  } else if (fabs(a1) > 0) {
    roots[nr++] = -a0 / a1;
  }
  double best_s = 0.0, best = poly4d(c, 0.0);
  for (int t = 0; t < nr; ++t) {
    double s = roots[t];
    for (int it = 0; it < 3; ++it) {
      const double d2 = ddpoly4d(c, s);
      if (d2 == 0) break;
      s -= dpoly4d(c, s) / d2;
    }
    if (!(s > 0) || !isfinite(s)) continue;
    const double v = poly4d(c, s);
    if (v < best) best = v, best_s = s;
  }
  return best_s;
}


}  // namespace bm
