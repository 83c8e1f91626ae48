// Boundary-lowered stencils at the cells next to a non-periodic end
// (Sec. 2.2, boundary paragraph): the fourth cell from the end (k = 3) uses
// 6th-order centred stencils, the third (k = 2) 4th-order ones, the second
// (k = 1) the centred 2nd-order diffusion and a biased 3rd-order first
// derivative, the end cell (k = 0) a completely biased 2nd-order diffusion
// and a completely biased 3rd-order first derivative.  Values are passed
// as v[j], j = 0..6, the cells counted from the end inward (mirrored at the
// high end, where first derivatives change sign).
#pragma once

namespace smc {

// h * d/dx at the cell k from the end (low-end orientation).  The one-sided
// stencils are written on differences (their weights sum to zero), so
// rounding follows the variation of v rather than its size:
//   k = 0: (-11 v0 + 18 v1 - 9 v2 + 2 v3) / 6,  k = 1: (-2 v0 - 3 v1 + 6 v2 - v3) / 6
__device__ __forceinline__ double lowered_d(const double *v, int k) {
  switch (k) {
    case 0:
      return (18.0 * (v[1] - v[0]) - 9.0 * (v[2] - v[0]) + 2.0 * (v[3] - v[0])) * (1.0 / 6.0);
    case 1:
      return (-2.0 * (v[0] - v[1]) + 6.0 * (v[2] - v[1]) - (v[3] - v[1])) * (1.0 / 6.0);
    case 2: return (2.0 / 3.0) * (v[3] - v[1]) - (1.0 / 12.0) * (v[4] - v[0]);
    default:
      return 0.75 * (v[4] - v[2]) - 0.15 * (v[5] - v[1]) + (1.0 / 60.0) * (v[6] - v[0]);
  }
}

// The 6th-order narrow matrix (free parameter 281/3600), rows and columns
// -2..3 of H_{j+1/2} = sum a_{j+m} M_mn u_{j+n}, and the 4th-order one
// (rows/columns -1..2, free parameters -1/9 and 1/72).  Zero row sums.
struct LoweredM {
  double M6[6][6];
  double M4[4][4];
};

__host__ __device__ inline LoweredM lowered_matrices() {
  LoweredM L;
  const double c = 281.0 / 3600.0;
  const double r1[6] = {-11.0 / 180 + c, 1.0 / 9 - 2 * c, -1.0 / 18 + c, 1.0 / 180, 0.0, 0.0};
  const double r2[6] = {7.0 / 60 - 3 * c, -1.0 / 120 + 5 * c, -17.0 / 90 - 2 * c, 5.0 / 72 + c,
                        1.0 / 90 - c, 0.0};
  const double r3[6] = {-1.0 / 15 + 3 * c, -11.0 / 60 - 3 * c, -101.0 / 360, 137.0 / 180 - 2 * c,
                        -83.0 / 360 + c, c};
  for (int n = 0; n < 6; ++n) {
    L.M6[0][n] = r1[n];
    L.M6[1][n] = r2[n];
    L.M6[2][n] = r3[n];
    L.M6[3][n] = -r3[5 - n];
    L.M6[4][n] = -r2[5 - n];
    L.M6[5][n] = -r1[5 - n];
  }
  const double M4[4][4] = {{-1.0 / 72, 8.0 / 72, -7.0 / 72, 0.0},
                           {8.0 / 72, -57.0 / 72, 48.0 / 72, 1.0 / 72},
                           {-1.0 / 72, -48.0 / 72, 57.0 / 72, -8.0 / 72},
                           {0.0, 7.0 / 72, -8.0 / 72, 1.0 / 72}};
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) L.M4[m][n] = M4[m][n];
  return L;
}

// h^2 (a u_x)_x at the cell k from the end (either end: the operator is
// symmetric under reflection).  Face fluxes in difference-first form
// (every row sums to zero): sum_m a_m sum_n M_mn (u_n - u_ref).
__device__ __forceinline__ double lowered_n(const LoweredM &L, const double *a, const double *u,
                                            int k) {
  if (k == 0) {
    // a u_xx + a_x u_x, one-sided: u_xx h^2 ~ 2 u0 - 5 u1 + 4 u2 - u3,
    // 2 h u_x ~ -3 u0 + 4 u1 - u2 (same for a), on differences from u0, a0
    const double d1 = u[1] - u[0], d2 = u[2] - u[0], d3 = u[3] - u[0];
    const double uxx = -5.0 * d1 + 4.0 * d2 - d3;
    const double ux = 4.0 * d1 - d2;
    const double ax = 4.0 * (a[1] - a[0]) - (a[2] - a[0]);
    return a[0] * uxx + 0.25 * ax * ux;
  }
  if (k == 1) return 0.5 * (a[1] + a[2]) * (u[2] - u[1]) - 0.5 * (a[0] + a[1]) * (u[1] - u[0]);
  double H[2];
  for (int o = 0; o < 2; ++o) {
    double acc = 0.0;
    if (k == 2) {
      const int j = 1 + o;                          // faces 1+1/2 and 2+1/2
      for (int m = 0; m < 4; ++m) {
        double w = 0.0;
        for (int n = 0; n < 4; ++n) w += L.M4[m][n] * (u[j - 1 + n] - u[j]);
        acc += a[j - 1 + m] * w;
      }
    } else {
      const int j = 2 + o;                          // faces 2+1/2 and 3+1/2
      for (int m = 0; m < 6; ++m) {
        double w = 0.0;
        for (int n = 0; n < 6; ++n) w += L.M6[m][n] * (u[j - 2 + n] - u[j]);
        acc += a[j - 2 + m] * w;
      }
    }
    H[o] = acc;
  }
  return H[1] - H[0];
}

}  // namespace smc
