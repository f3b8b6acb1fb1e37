// Reference element of the nodal DG space (Section 5.2.2: "expanded in the
// nodal basis of P_q"), built on the unit tetrahedron (0,0,0), (1,0,0),
// (0,1,0), (0,0,1) at equispaced nodes:
//   * nodal basis phi_j = sum_n C[n][j] x^a_n y^b_n z^c_n with C = V^{-1},
//     V[i][n] = monomial n at node i;
//   * mass M[i][j] = int phi_i phi_j from the exact simplex integral
//     int x^a y^b z^c = a! b! c! / (a + b + c + 3)!;
//   * D_r[i][j] = d phi_j / d r at node i (likewise s, t);
//   * face mass by a collapsed (Duffy) Gauss-Legendre rule, 4 x 4 points, exact
//     for the degree 2q <= 6 integrands;
//   * LIFT = M^{-1} E_f for each face.
#include <cmath>
#include <mutex>
#include <stdexcept>

#include "common.h"

namespace cmcg {
namespace {

struct Mono {
  int a, b, c;
};

std::vector<Mono> monomials(int q) {
  std::vector<Mono> m;
  for (int a = 0; a <= q; ++a)
    for (int b = 0; b <= q - a; ++b)
      for (int c = 0; c <= q - a - b; ++c) m.push_back({a, b, c});
  return m;
}

double fact(int n) {
  double r = 1;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

double ipow(double x, int e) {
  double r = 1;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// Gauss-Jordan inverse with partial pivoting (n <= 20).
std::vector<double> invert(const std::vector<double>& A, int n) {
  std::vector<double> a(A), inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[r * n + col]) > std::fabs(a[piv * n + col])) piv = r;
    if (std::fabs(a[piv * n + col]) < 1e-300) throw std::runtime_error("singular matrix");
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[piv * n + k], a[col * n + k]);
        std::swap(inv[piv * n + k], inv[col * n + k]);
      }
    double d = a[col * n + col];
    for (int k = 0; k < n; ++k) {
      a[col * n + k] /= d;
      inv[col * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = a[r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[r * n + k] -= f * a[col * n + k];
        inv[r * n + k] -= f * inv[col * n + k];
      }
    }
  }
  return inv;
}

}  // namespace

// Gauss-Legendre nodes / weights on [0, 1] by Newton iteration on P_n.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1;
      dp = n * (z * p1 - p0) / (z * z - 1);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged root
    double p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1);
    x[i] = 0.5 * (z + 1);
    w[i] = 1.0 / ((1 - z * z) * dp * dp);  // = 0.5 * 2 / ((1 - z^2) P'^2)
  }
}

namespace {

RefMats build(int q) {
  RefMats r;
  r.q = q;
  r.np = np_of(q);
  r.nfp = nfp_of(q);
  const int np = r.np, nfp = r.nfp;
  auto mono = monomials(q);
  // nodes in boundary order
  std::vector<double> X(np), Y(np), Z(np);
  for (int k = 0; k <= q; ++k)
    for (int j = 0; j <= q - k; ++j)
      for (int i = 0; i <= q - k - j; ++i) {
        int n = lattice_index(q, i, j, k);
        X[n] = double(i) / q;
        Y[n] = double(j) / q;
        Z[n] = double(k) / q;
      }
  std::vector<double> V(np * np);
  for (int i = 0; i < np; ++i)
    for (int n = 0; n < np; ++n) V[i * np + n] = ipow(X[i], mono[n].a) * ipow(Y[i], mono[n].b) * ipow(Z[i], mono[n].c);
  std::vector<double> C = invert(V, np);  // phi_j = sum_n C[n][j] m_n

  auto phi = [&](int j, double x, double y, double z) {
    double s = 0;
    for (int n = 0; n < np; ++n) s += C[n * np + j] * ipow(x, mono[n].a) * ipow(y, mono[n].b) * ipow(z, mono[n].c);
    return s;
  };

  r.M.assign(np * np, 0.0);
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j) {
      double s = 0;
      for (int n = 0; n < np; ++n)
        for (int m = 0; m < np; ++m) {
          int a = mono[n].a + mono[m].a, b = mono[n].b + mono[m].b, c = mono[n].c + mono[m].c;
          s += C[n * np + i] * C[m * np + j] * fact(a) * fact(b) * fact(c) / fact(a + b + c + 3);
        }
      r.M[i * np + j] = s;
    }
  r.Minv = invert(r.M, np);

  r.Dr.assign(np * np, 0.0);
  r.Ds.assign(np * np, 0.0);
  r.Dt.assign(np * np, 0.0);
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j) {
      double dr = 0, ds = 0, dt = 0;
      for (int n = 0; n < np; ++n) {
        const Mono& m = mono[n];
        double c = C[n * np + j];
        if (m.a) dr += c * m.a * ipow(X[i], m.a - 1) * ipow(Y[i], m.b) * ipow(Z[i], m.c);
        if (m.b) ds += c * m.b * ipow(X[i], m.a) * ipow(Y[i], m.b - 1) * ipow(Z[i], m.c);
        if (m.c) dt += c * m.c * ipow(X[i], m.a) * ipow(Y[i], m.b) * ipow(Z[i], m.c - 1);
      }
      r.Dr[i * np + j] = dr;
      r.Ds[i * np + j] = ds;
      r.Dt[i * np + j] = dt;
    }

  // face-local node order
  const FaceTab fm = make_fmask(q);
  r.fmask.assign(4 * nfp, 0);
  for (int f = 0; f < 4; ++f)
    for (int jf = 0; jf < nfp; ++jf) r.fmask[f * nfp + jf] = fm.v[f][jf];

  // face masses by Duffy-collapsed Gauss-Legendre quadrature
  const double VX[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  std::vector<double> gx, gw;
  gauss_legendre01(4, gx, gw);
  r.LIFT.assign(np * 4 * nfp, 0.0);
  for (int f = 0; f < 4; ++f) {
    const double* P0 = VX[FACE_VERTS[f][0]];
    const double* P1 = VX[FACE_VERTS[f][1]];
    const double* P2 = VX[FACE_VERTS[f][2]];
    double e1[3], e2[3], cr[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = P1[d] - P0[d];
      e2[d] = P2[d] - P0[d];
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double area = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    r.face_ref_area[f] = area;
    std::vector<double> Ef(np * np, 0.0);
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double u = gx[a], v = gx[b] * (1 - gx[a]);
        double wq = gw[a] * gw[b] * (1 - gx[a]) * 2.0 * area;
        double x = P0[0] + u * e1[0] + v * e2[0];
        double y = P0[1] + u * e1[1] + v * e2[1];
        double z = P0[2] + u * e1[2] + v * e2[2];
        std::vector<double> pv(np);
        for (int j = 0; j < np; ++j) pv[j] = phi(j, x, y, z);
        for (int i = 0; i < np; ++i)
          for (int j = 0; j < np; ++j) Ef[i * np + j] += wq * pv[i] * pv[j];
      }
    for (int i = 0; i < np; ++i)
      for (int jf = 0; jf < nfp; ++jf) {
        int col = r.fmask[f * nfp + jf];
        double s = 0;
        for (int k = 0; k < np; ++k) s += r.Minv[i * np + k] * Ef[k * np + col];
        r.LIFT[i * (4 * nfp) + f * nfp + jf] = s;
      }
  }

  // neighbour node tables: own face-local node jf with weights (w0, w1, w2) is
  // the neighbour face-local node with weights w'[sigma[s]] = w[s].
  r.nbrnode.assign(4 * 6 * nfp, 0);
  for (int nf = 0; nf < 4; ++nf)
    for (int p = 0; p < 6; ++p) {
      int jf = 0;
      for (int w2 = 0; w2 <= q; ++w2)
        for (int w1 = 0; w1 <= q - w2; ++w1) {
          int w[3] = {q - w1 - w2, w1, w2}, wn[3];
          for (int s = 0; s < 3; ++s) wn[PERMS[p][s]] = w[s];
          // canonical index of (wn1, wn2): w2 outermost, w1 fastest
          int idx = 0;
          for (int t = 0; t < wn[2]; ++t) idx += q - t + 1;
          idx += wn[1];
          r.nbrnode[(nf * 6 + p) * nfp + jf] = fm.v[nf][idx];
          ++jf;
        }
    }
  return r;
}

}  // namespace

const RefMats& ref_mats(int q) {
  static std::once_flag once[4];
  static RefMats cache[4];
  if (q < 1 || q > 3) throw std::runtime_error("order out of range");
  std::call_once(once[q], [q] { cache[q] = build(q); });
  return cache[q];
}

}  // namespace cmcg
