// Collocation nodes and integration matrices for SDC (Sec. 3.1) and
// multirate SDC (Sec. 3.2), computed in long double on the host.
//
// Gauss-Lobatto nodes: the end points and the roots of P'_N, N = n - 1,
// found by Newton's method on P'_N with P''_N from Legendre's equation.
// Integration matrices: the Lagrange basis through the nodes is obtained by
// solving the Vandermonde system V C = I (Gaussian elimination with partial
// pivoting), and each basis polynomial is integrated exactly term by term.
#include <cmath>
#include <vector>

#include "smc_internal.h"

namespace smc {

typedef long double ld;

static void legendre(int N, ld x, ld &P, ld &dP) {
  // P_N(x) and P'_N(x) by the three-term recurrence
  ld p0 = 1.0L, p1 = x;
  if (N == 0) { P = 1.0L; dP = 0.0L; return; }
  for (int k = 2; k <= N; ++k) {
    const ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = N * (p0 - x * p1) / (1.0L - x * x);
}

void lobatto_nodes(int n, std::vector<double> &out) {
  const int N = n - 1;
  std::vector<ld> x(n);
  x[0] = -1.0L;
  x[N] = 1.0L;
  for (int j = 1; j < N; ++j) {
    ld xi = -cosl(3.14159265358979323846264338327950288L * j / N);
    for (int it = 0; it < 100; ++it) {
      ld P, dP;
      legendre(N, xi, P, dP);
      const ld d2P = (2.0L * xi * dP - N * (N + 1) * P) / (1.0L - xi * xi);
      const ld step = dP / d2P;
      xi -= step;
      if (fabsl(step) < 1e-30L) break;
    }
    x[j] = xi;
  }
  out.resize(n);
  for (int j = 0; j < n; ++j) out[j] = (double)(0.5L * (x[j] + 1.0L));
}

// C[k][j]: coefficient of t^k in the Lagrange polynomial L_j through nodes t.
static void lagrange_coeffs(const std::vector<ld> &t, std::vector<ld> &C) {
  const int n = (int)t.size();
  std::vector<ld> A(n * 2 * n, 0.0L);
  for (int i = 0; i < n; ++i) {
    ld pw = 1.0L;
    for (int k = 0; k < n; ++k) {
      A[i * 2 * n + k] = pw;
      pw *= t[i];
    }
    A[i * 2 * n + n + i] = 1.0L;
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabsl(A[r * 2 * n + col]) > fabsl(A[piv * 2 * n + col])) piv = r;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) std::swap(A[col * 2 * n + c], A[piv * 2 * n + c]);
    const ld inv = 1.0L / A[col * 2 * n + col];
    for (int c = 0; c < 2 * n; ++c) A[col * 2 * n + c] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const ld f = A[r * 2 * n + col];
      if (f == 0.0L) continue;
      for (int c = 0; c < 2 * n; ++c) A[r * 2 * n + c] -= f * A[col * 2 * n + c];
    }
  }
  // V C = I  =>  C = V^-1, stored row k (power), column j (basis index)
  C.assign(n * n, 0.0L);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) C[k * n + j] = A[k * 2 * n + n + j];
}

static ld integral(const std::vector<ld> &C, int n, int j, ld a, ld b) {
  ld acc = 0.0L, pa = a, pb = b;
  for (int k = 0; k < n; ++k) {
    acc += C[k * n + j] * (pb - pa) / (k + 1);
    pa *= a;
    pb *= b;
  }
  return acc;
}

void node_to_node_matrix(const std::vector<double> &nodes, std::vector<double> &S) {
  const int n = (int)nodes.size();
  std::vector<ld> t(nodes.begin(), nodes.end());
  std::vector<ld> C;
  lagrange_coeffs(t, C);
  S.assign((n - 1) * n, 0.0);
  for (int m = 0; m < n - 1; ++m)
    for (int j = 0; j < n; ++j) S[m * n + j] = (double)integral(C, n, j, t[m], t[m + 1]);
}

// Type (b) multirate nodes: `fine` Gauss-Lobatto nodes in each interval of the
// `coarse` Gauss-Lobatto nodes.  S21 integrates the coarse interpolant between
// fine nodes; S22 integrates the piecewise (per coarse interval) interpolant
// of the fine values.
void multirate_matrices(int coarse, int fine, int repeat, std::vector<double> &t1,
                        std::vector<double> &t2, std::vector<double> &S21,
                        std::vector<double> &S22) {
  std::vector<double> g;
  lobatto_nodes(coarse, t1);
  lobatto_nodes(fine, g);
  // every coarse interval holds `repeat` consecutive groups of `fine`
  // Gauss-Lobatto nodes (type (b) for repeat = 1, type (c) otherwise);
  // neighbouring groups share their end nodes
  const int M1 = coarse - 1, sub = fine - 1, per = sub * repeat, M2 = M1 * per;
  std::vector<ld> T2(M2 + 1);
  for (int p = 0; p < M1; ++p)
    for (int r = 0; r < repeat; ++r)
      for (int s = 0; s <= sub; ++s)
        T2[p * per + r * sub + s] =
            (ld)t1[p] + ((ld)t1[p + 1] - (ld)t1[p]) * ((ld)r + (ld)g[s]) / (ld)repeat;
  t2.resize(M2 + 1);
  for (int q = 0; q <= M2; ++q) t2[q] = (double)T2[q];
  std::vector<ld> T1(t1.begin(), t1.end()), C1;
  lagrange_coeffs(T1, C1);
  S21.assign(M2 * (M1 + 1), 0.0);
  S22.assign(M2 * (M2 + 1), 0.0);
  for (int q = 0; q < M2; ++q)
    for (int j = 0; j <= M1; ++j)
      S21[q * (M1 + 1) + j] = (double)integral(C1, M1 + 1, j, T2[q], T2[q + 1]);
  // the fine basis of one group, in the group's own coordinate
  // sigma = (t - start) / width (the Lagrange basis is invariant under this
  // affine map; it keeps the Vandermonde system well conditioned)
  std::vector<ld> G(g.begin(), g.end()), Cg;
  lagrange_coeffs(G, Cg);
  for (int p = 0; p < M1; ++p) {
    const ld width = ((ld)t1[p + 1] - (ld)t1[p]) / (ld)repeat;
    for (int r = 0; r < repeat; ++r) {
      const int q0 = p * per + r * sub;
      for (int s = 0; s < sub; ++s)
        for (int t = 0; t <= sub; ++t)
          S22[(q0 + s) * (M2 + 1) + q0 + t] = (double)(width * integral(Cg, sub + 1, t, G[s], G[s + 1]));
    }
  }
}

}  // namespace smc
