// Host-side generation of the 1D operators of the nodal Gauss-Legendre basis
// (Sec. 2.1 Eq. ansatz.uh, Sec. 2.2 Eq. pde.nc.dg2), of the subcell
// projection / reconstruction (Sec. 4.2 Eqs. subcell.p, subcell.r) and of the
// WENO3 stencil matrices.  Arithmetic in long double; results rounded to double.
#include <cmath>
#include <cstring>

#include "adg_internal.h"

namespace adg {
namespace {

typedef long double ld;

// Legendre P_n and P_n' on [-1, 1]
void legendre(int n, ld x, ld* p, ld* dp) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) {
    *p = 1.0L;
    *dp = 0.0L;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0L);
}

// n Gauss-Legendre points and weights on [0, 1], ascending
void gauss(int n, ld* x, ld* w) {
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    ld z = cosl(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(n, z, &p, &dp);
      ld dz = p / dp;
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    ld p, dp;
    legendre(n, z, &p, &dp);
    // store mapped to [0,1]; the cosine guess gives descending z
    x[n - 1 - i] = 0.5L * (z + 1.0L);
    w[n - 1 - i] = 1.0L / ((1.0L - z * z) * dp * dp);
  }
}

ld lagrange(const ld* nodes, int n, int a, ld x) {
  ld r = 1.0L;
  for (int b = 0; b < n; ++b)
    if (b != a) r *= (x - nodes[b]) / (nodes[a] - nodes[b]);
  return r;
}

ld lagrange_deriv(const ld* nodes, int n, int a, ld x) {
  ld s = 0.0L;
  for (int c = 0; c < n; ++c) {
    if (c == a) continue;
    ld t = 1.0L / (nodes[a] - nodes[c]);
    for (int b = 0; b < n; ++b)
      if (b != a && b != c) t *= (x - nodes[b]) / (nodes[a] - nodes[b]);
    s += t;
  }
  return s;
}

// In-place Gauss-Jordan inverse of an m x m matrix (partial pivoting).
void invert(ld* A, int m) {
  ld I[32 * 32];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) I[i * m + j] = (i == j) ? 1.0L : 0.0L;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabsl(A[r * m + c]) > fabsl(A[piv * m + c])) piv = r;
    if (piv != c)
      for (int j = 0; j < m; ++j) {
        ld t = A[c * m + j];
        A[c * m + j] = A[piv * m + j];
        A[piv * m + j] = t;
        t = I[c * m + j];
        I[c * m + j] = I[piv * m + j];
        I[piv * m + j] = t;
      }
    const ld d = A[c * m + c];
    for (int j = 0; j < m; ++j) {
      A[c * m + j] /= d;
      I[c * m + j] /= d;
    }
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const ld f = A[r * m + c];
      if (f == 0.0L) continue;
      for (int j = 0; j < m; ++j) {
        A[r * m + j] -= f * A[c * m + j];
        I[r * m + j] -= f * I[c * m + j];
      }
    }
  }
  for (int i = 0; i < m * m; ++i) A[i] = I[i];
}

// Basis operators of one degree: nodes, weights, D, Ktau, phi(0), phi(1)
void basis_ops(int N, ld* xi, ld* w, ld* D, ld* Kt, ld* phi0, ld* phi1) {
  const int n = N + 1;
  gauss(n, xi, w);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) D[a * n + b] = lagrange_deriv(xi, n, b, xi[a]);
  for (int a = 0; a < n; ++a) {
    phi0[a] = lagrange(xi, n, a, 0.0L);
    phi1[a] = lagrange(xi, n, a, 1.0L);
  }
  // K1[m][l] = phi_m(1) phi_l(1) - w_l D[l][m];  Ktau = K1^{-1} diag(w)
  ld K1[MAXN * MAXN];
  for (int m = 0; m < n; ++m)
    for (int l = 0; l < n; ++l) K1[m * n + l] = phi1[m] * phi1[l] - w[l] * D[l * n + m];
  invert(K1, n);
  for (int m = 0; m < n; ++m)
    for (int j = 0; j < n; ++j) Kt[m * n + j] = K1[m * n + j] * w[j];
}

}  // namespace

void build_ops(int N, Ops* o) {
  std::memset(o, 0, sizeof(Ops));
  const int n = N + 1, Ns = 2 * N + 1;
  o->N = N;
  o->n = n;
  o->Ns = Ns;
  ld xi[MAXN], w[MAXN], D[MAXN * MAXN], Kt[MAXN * MAXN], p0[MAXN], p1[MAXN];
  basis_ops(N, xi, w, D, Kt, p0, p1);
  for (int a = 0; a < n; ++a) {
    o->xi[a] = (double)xi[a];
    o->w[a] = (double)w[a];
    o->phi0[a] = (double)p0[a];
    o->phi1[a] = (double)p1[a];
    o->phi0w[a] = (double)(p0[a] / w[a]);
    o->phi1w[a] = (double)(p1[a] / w[a]);
  }
  for (int i = 0; i < n * n; ++i) {
    o->D[i] = (double)D[i];
    o->Kt[i] = (double)Kt[i];
    o->Df[i] = (float)D[i];
    o->Ktf[i] = (float)Kt[i];
  }
  for (int a = 0; a < n; ++a) o->wf[a] = (float)o->w[a];   // the FP64 weight rounded to FP32
  for (int a = 0; a < n; ++a)
    for (int j = 0; j < n; ++j) o->Mvol[a * n + j] = (double)(w[j] * D[j * n + a] / w[a]);
  // subcell projection: n-point GL rule per subinterval is exact for degree N
  ld P1[MAXNS * MAXN];
  {
    ld xq[MAXN], wq[MAXN];
    gauss(n, xq, wq);
    for (int s = 0; s < Ns; ++s)
      for (int a = 0; a < n; ++a) {
        ld acc = 0.0L;
        for (int q = 0; q < n; ++q) acc += wq[q] * lagrange(xi, n, a, (s + xq[q]) / Ns);
        P1[s * n + a] = acc;
      }
  }
  // R1 = (P1^T P1)^{-1} P1^T
  ld NtN[MAXN * MAXN];
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      ld acc = 0.0L;
      for (int s = 0; s < Ns; ++s) acc += P1[s * n + a] * P1[s * n + b];
      NtN[a * n + b] = acc;
    }
  invert(NtN, n);
  for (int a = 0; a < n; ++a)
    for (int s = 0; s < Ns; ++s) {
      ld acc = 0.0L;
      for (int b = 0; b < n; ++b) acc += NtN[a * n + b] * P1[s * n + b];
      o->R1[a * Ns + s] = (double)acc;
    }
  for (int s = 0; s < Ns; ++s)
    for (int a = 0; a < n; ++a) {
      o->P1[s * n + a] = (double)P1[s * n + a];
      o->Mt[a * Ns + s] = (double)(P1[s * n + a] / (Ns * w[a]));
    }
  // composite rule of the initial projection: Ns subintervals x (N+2) points
  {
    ld xq[MAXN + 1], wq[MAXN + 1];
    gauss(N + 2, xq, wq);
    for (int s = 0; s < Ns; ++s)
      for (int q = 0; q < N + 2; ++q) {
        const int p = s * (N + 2) + q;
        const ld x = (s + xq[q]) / Ns;
        o->cq_x[p] = (double)x;
        o->cq_w[p] = (double)(wq[q] / Ns);
        for (int a = 0; a < n; ++a) o->cq_phi[p * n + a] = (double)lagrange(xi, n, a, x);
      }
  }
  // degree-2 subcell basis
  {
    ld x3[3], w3[3], D3[9], K3[9], q0[3], q1[3];
    basis_ops(2, x3, w3, D3, K3, q0, q1);
    for (int a = 0; a < 3; ++a) {
      o->xi3[a] = (double)x3[a];
      o->w3[a] = (double)w3[a];
      o->phi03[a] = (double)q0[a];
      o->phi13[a] = (double)q1[a];
    }
    for (int i = 0; i < 9; ++i) {
      o->D3[i] = (double)D3[i];
      o->Kt3[i] = (double)K3[i];
    }
    for (int j = 0; j < 3; ++j)
      for (int p = 0; p < 3; ++p) o->E[j * 3 + p] = (double)powl(x3[j], (ld)p);
  }
  // WENO3 stencils {s-2..s}, {s-1..s+1}, {s..s+2}: A[r][p] = int_o^{o+1} xi^p
  for (int k = 0; k < 3; ++k) {
    const int o0 = k - 2;
    ld A[9];
    for (int r = 0; r < 3; ++r) {
      const ld lo = (ld)(o0 + r), hi = lo + 1.0L;
      for (int p = 0; p < 3; ++p) A[r * 3 + p] = (powl(hi, (ld)(p + 1)) - powl(lo, (ld)(p + 1))) / (p + 1);
    }
    invert(A, 3);   // A^{-1}[p][r]: monomial p from cell r
    for (int i = 0; i < 9; ++i) o->C[k][i] = (double)A[i];
    for (int r = 0; r < 3; ++r) {
      o->Cf[k][r] = (float)A[3 + r];
      o->Cf[k][3 + r] = (float)A[6 + r];
    }
    // nodes of the degree-2 subcell basis (3 GL points on [0, 1])
    const ld x3n[3] = {0.5L - sqrtl(0.15L), 0.5L, 0.5L + sqrtl(0.15L)};
    for (int j = 0; j < 3; ++j)
      for (int r = 0; r < 3; ++r) {
        ld v = 0.0L;
        for (int q = 0; q < 3; ++q) v += powl(x3n[j], (ld)q) * A[q * 3 + r];
        o->Wf[k][j * 3 + r] = (float)v;
      }
  }
}

}  // namespace adg
