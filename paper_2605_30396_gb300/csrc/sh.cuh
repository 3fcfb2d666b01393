// Real spherical harmonics of degrees 1-3 (the 15 view-dependent bases of a
// Gaussian's colour, Sec. 2.2), in Cartesian form for a unit direction.
// Basis order b = l*l + l + m - 1 (l = 1..3, m = -l..l); the constants carry
// N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), the sqrt(2) of the real forms,
// the Condon-Shortley phase and the leading factors of the associated Legendre
// polynomials.  Used by the decode and the splatting preprocess.
#pragma once

#include <math.h>

namespace dlsh {

struct ShConst {
  float c[15];
};

// Y_b(v) for unit v = (x, y, z); c points at the 15 constants of make_sh_constants.
__device__ __forceinline__ void sh_basis(const float* c, float x, float y, float z, float (&Y)[15]) {
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = c[0] * y;
  Y[1] = c[1] * z;
  Y[2] = c[2] * x;
  Y[3] = c[3] * x * y;
  Y[4] = c[4] * y * z;
  Y[5] = c[5] * (3.f * zz - 1.f);
  Y[6] = c[6] * x * z;
  Y[7] = c[7] * (xx - yy);
  Y[8] = c[8] * y * (3.f * xx - yy);
  Y[9] = c[9] * x * y * z;
  Y[10] = c[10] * y * (5.f * zz - 1.f);
  Y[11] = c[11] * z * (5.f * zz - 3.f);
  Y[12] = c[12] * x * (5.f * zz - 1.f);
  Y[13] = c[13] * z * (xx - yy);
  Y[14] = c[14] * x * (xx - 3.f * yy);
}

inline double sh_factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

inline double sh_nlm(int l, int m) {
  const int am = m < 0 ? -m : m;
  return sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * sh_factorial(l - am) / sh_factorial(l + am));
}

// Constants of the Cartesian forms in sh_basis.  With P_l^m carrying the
// Condon-Shortley phase: P_1^1 = -sin, P_2^1 = -3z sin, P_2^2 = 3 sin^2,
// P_3^1 = -1.5 (5z^2-1) sin, P_3^2 = 15 z sin^2, P_3^3 = -15 sin^3, and
// sin^m(theta) {cos,sin}(m phi) expands to the x/y polynomials of sh_basis.
inline ShConst make_sh_constants() {
  const double r2 = sqrt(2.0);
  ShConst k;
  k.c[0] = static_cast<float>(-r2 * sh_nlm(1, -1));             // y
  k.c[1] = static_cast<float>(sh_nlm(1, 0));                    // z
  k.c[2] = static_cast<float>(-r2 * sh_nlm(1, 1));              // x
  k.c[3] = static_cast<float>(r2 * sh_nlm(2, -2) * 3.0 * 2.0);  // xy   (sin^2 sin 2phi = 2xy)
  k.c[4] = static_cast<float>(-r2 * sh_nlm(2, -1) * 3.0);       // yz
  k.c[5] = static_cast<float>(sh_nlm(2, 0) * 0.5);              // 3z^2 - 1
  k.c[6] = static_cast<float>(-r2 * sh_nlm(2, 1) * 3.0);        // xz
  k.c[7] = static_cast<float>(r2 * sh_nlm(2, 2) * 3.0);         // x^2 - y^2
  k.c[8] = static_cast<float>(-r2 * sh_nlm(3, -3) * 15.0);      // y(3x^2 - y^2)
  k.c[9] = static_cast<float>(r2 * sh_nlm(3, -2) * 15.0 * 2.0); // xyz
  k.c[10] = static_cast<float>(-r2 * sh_nlm(3, -1) * 1.5);      // y(5z^2 - 1)
  k.c[11] = static_cast<float>(sh_nlm(3, 0) * 0.5);             // z(5z^2 - 3)
  k.c[12] = static_cast<float>(-r2 * sh_nlm(3, 1) * 1.5);       // x(5z^2 - 1)
  k.c[13] = static_cast<float>(r2 * sh_nlm(3, 2) * 15.0);       // z(x^2 - y^2)
  k.c[14] = static_cast<float>(-r2 * sh_nlm(3, 3) * 15.0);      // x(x^2 - 3y^2)
  return k;
}

}  // namespace dlsh
