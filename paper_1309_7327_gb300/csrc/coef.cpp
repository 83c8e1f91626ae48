// Host construction of the 8th-order narrow-stencil matrix of Sec. 2.2.
#include "smc_internal.h"

namespace smc {

// M[8][8], rows m = -3..4 and columns n = -3..4 of the face flux
// H_{i+1/2} = sum_{m,n} a_{i+m} M_mn u_{i+n} (unscaled; divide by h^2), from
// the two free parameters m47 and m48.  The lower four rows follow from the
// upper four by the antisymmetry M_{-m+1,-n+1} = -M_mn.
void narrow8_matrix(double m47, double m48, double M[8][8]) {
  const double a = m47, b = m48;
  double m[5][9] = {};
  m[1][1] = 5.0 / 336 + b;
  m[1][2] = -83.0 / 3600 - a / 5 - 14.0 * b / 5;
  m[1][3] = 299.0 / 50400 + 2.0 * a / 5 + 13.0 * b / 5;
  m[1][4] = 17.0 / 12600 - a / 5 - 4.0 * b / 5;
  m[1][5] = 1.0 / 1120;
  m[2][1] = -11.0 / 560 - 2 * b;
  m[2][2] = -31.0 / 360 + a + 3 * b;
  m[2][3] = 41.0 / 200 - 9.0 * a / 5 + 4.0 * b / 5;
  m[2][4] = -5927.0 / 50400 + 4.0 * a / 5 - 9.0 * b / 5;
  m[2][5] = 17.0 / 600 - a / 5 - 4.0 * b / 5;
  m[2][6] = -503.0 / 50400 + a / 5 + 4.0 * b / 5;
  m[3][1] = -1.0 / 280;
  m[3][2] = 1097.0 / 5040 - 2 * a + 6 * b;
  m[3][3] = -1349.0 / 10080 + 3 * a - 12 * b;
  m[3][4] = -887.0 / 5040 - a + 6 * b;
  m[3][5] = 3613.0 / 50400 + 4.0 * a / 5 - 9.0 * b / 5;
  m[3][6] = 467.0 / 25200 - 3.0 * a / 5 + 18.0 * b / 5;
  m[3][7] = 139.0 / 25200 - a / 5 - 9.0 * b / 5;
  m[4][1] = 17.0 / 1680 + 2 * b;
  m[4][2] = -319.0 / 2520 + 2 * a - 8 * b;
  m[4][3] = -919.0 / 5040 - 2 * a + 6 * b;
  m[4][4] = -445.0 / 2016;
  m[4][5] = 583.0 / 720 - a + 6 * b;
  m[4][6] = -65.0 / 224 - 7 * b;
  m[4][7] = a;
  m[4][8] = b;
  for (int r = 0; r < 8; ++r)
    for (int c = 0; c < 8; ++c) M[r][c] = 0.0;
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) {
      M[r][c] = m[r + 1][c + 1];
      M[7 - r][7 - c] = -m[r + 1][c + 1];
    }
}

}  // namespace smc
