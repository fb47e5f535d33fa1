// weights.cpp -- differentiation-weight tables of the ACAT step, computed in
// exact rational arithmetic and rounded once to double.
//
// On the 2p nodes r = -p+1..p (unit spacing) the k-th derivative at q of the
// Lagrange interpolant is sum_r gamma^{k,q}_{p,r} f_r (Eq. 2.10). Each basis
// polynomial l_r(x) = prod_{m != r} (x - m) / (r - m) is expanded into integer
// coefficients, differentiated k times and evaluated at q; every value is a
// fraction of 64-bit integers until the final division.
//
// The flux weights gamma^{0,1/2}_{p,.} of Eq. 2.14 are the weights for which
// Eq. 2.11 holds at k = 1, D^1_{p,i} = (A^{0,1/2}_{p,i} - A^{0,1/2}_{p,i-1})/dx,
// with D^1_p the centred (2p+1)-point first derivative (Eq. 2.5): matching the
// coefficient of f_{i+l} gives gamma_m = -sum_{l=-p}^{m-1} delta^1_{p,l}.
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "acat_internal.h"

namespace {

struct Q {  // exact rational n/d, d > 0, reduced
  int64_t n, d;
};

int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a ? a : 1;
}

Q mk(int64_t n, int64_t d) {
  if (d < 0) {
    n = -n;
    d = -d;
  }
  int64_t g = gcd64(n, d);
  return Q{n / g, d / g};
}
Q add(Q a, Q b) {
  int64_t g = gcd64(a.d, b.d);
  return mk(a.n * (b.d / g) + b.n * (a.d / g), a.d / g * b.d);
}
Q mul(Q a, Q b) {
  int64_t g1 = gcd64(a.n, b.d), g2 = gcd64(b.n, a.d);
  return mk((a.n / g1) * (b.n / g2), (a.d / g2) * (b.d / g1));
}
Q neg(Q a) { return Q{-a.n, a.d}; }
double to_d(Q a) { return (double)a.n / (double)a.d; }

// Weights of the k-th derivative at q (rational) over the integer nodes
// x[0..n-1]; w[r] exact.
void lagrange_deriv(int n, const int *x, int k, Q q, Q *w) {
  for (int r = 0; r < n; r++) {
    // numerator polynomial prod_{m != r} (t - x_m), integer coefficients
    int64_t c[ACAT_MAXN + 2];
    std::memset(c, 0, sizeof c);
    c[0] = 1;
    int deg = 0;
    int64_t den = 1;
    for (int m = 0; m < n; m++) {
      if (m == r) continue;
      for (int e = deg + 1; e >= 1; e--) c[e] = c[e - 1] - x[m] * c[e];
      c[0] = -x[m] * c[0];
      deg++;
      den *= (int64_t)(x[r] - x[m]);
    }
    // k-th derivative at q: sum_e c_e e!/(e-k)! q^(e-k)
    Q v{0, 1};
    for (int e = k; e <= deg; e++) {
      int64_t ff = 1;
      for (int t = e - k + 1; t <= e; t++) ff *= t;
      Q qp{1, 1};
      for (int t = 0; t < e - k; t++) qp = mul(qp, q);
      v = add(v, mul(mk(c[e] * ff, 1), qp));
    }
    w[r] = mul(v, mk(1, den));
  }
}

}  // namespace

void acat_build_tables(AcatTables *T) {
  std::memset(T, 0, sizeof *T);
  for (int p = 1; p <= ACAT_MAXP; p++) {
    const int n = 2 * p;
    int nodes[ACAT_MAXN + 1];
    for (int r = 0; r < n; r++) nodes[r] = r - p + 1;
    Q w[ACAT_MAXN + 1];
    // gamma^{1,j}_{p,r}: first derivative at each node j
    for (int j = 0; j < n; j++) {
      lagrange_deriv(n, nodes, 1, mk(nodes[j], 1), w);
      for (int r = 0; r < n; r++) T->g1[p][j][r] = to_d(w[r]);
    }
    // gamma^{k,0}_{p,r}: k-th derivative at 0 (time derivatives), k < 2p
    for (int k = 0; k < n; k++) {
      lagrange_deriv(n, nodes, k, mk(0, 1), w);
      for (int r = 0; r < n; r++) T->gk[p][k][r] = to_d(w[r]);
    }
    // gamma^{2p-1,1/2}: the binomial (2p-1)-th difference (Eq. 3.12)
    lagrange_deriv(n, nodes, n - 1, mk(1, 2), w);
    for (int r = 0; r < n; r++) T->gd[p][r] = to_d(w[r]);
    // flux weights: Eq. 2.11 at k = 1 from the centred first derivative
    int cen[ACAT_MAXN + 1];
    for (int r = 0; r <= n; r++) cen[r] = r - p;
    Q d[ACAT_MAXN + 1];
    lagrange_deriv(n + 1, cen, 1, mk(0, 1), d);
    Q s{0, 1};
    for (int m = 0; m < n; m++) {
      s = add(s, neg(d[m]));
      T->gh[p][m] = to_d(s);
    }
    // Taylor coefficients r^l / l! at the 2p time levels
    for (int rr = 0; rr < n; rr++) {
      const int r = rr - p + 1;
      Q v{1, 1};
      T->taylor[p][rr][0] = 1.0;
      for (int l = 1; l < n; l++) {
        v = mul(v, mk(r, l));
        T->taylor[p][rr][l] = to_d(v);
      }
    }
    // (2p-1)! for tau_p
    int64_t f = 1;
    for (int t = 2; t <= n - 1; t++) f *= t;
    T->fact[p] = (double)f;
  }
  int64_t f = 1;
  T->invfact[0] = 1.0;
  for (int k = 1; k <= ACAT_MAXN; k++) {
    f *= k;
    T->invfact[k] = 1.0 / (double)f;
  }
  for (int p = 0; p <= ACAT_MAXP; p++) {
    for (int a = 0; a < ACAT_MAXN; a++) {
      T->ghf[p][a] = (float)T->gh[p][a];
      for (int b = 0; b < ACAT_MAXN; b++) {
        T->g1f[p][a][b] = (float)T->g1[p][a][b];
        T->gkf[p][a][b] = (float)T->gk[p][a][b];
        T->taylorf[p][a][b] = (float)T->taylor[p][a][b];
      }
    }
  }
  for (int k = 0; k <= ACAT_MAXN; k++) T->invfactf[k] = (float)T->invfact[k];
}
