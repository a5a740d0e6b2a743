// Reference-tetrahedron operators (host, FP64).
//
// Basis: the orthonormal collapsed-coordinate polynomials of the reference
// tetrahedron (the "orthonormal polynomial basis" phi_i that defines the
// generalized Vandermonde matrices V and V_I of eq. 20), evaluated with the
// three-term recurrence of the normalised Jacobi polynomials.
// Nodes: equispaced, node (i,j,k) at r = -1 + 2(i,j,k)/N, enumerated with k
// outermost, then j, then i.
// Face mass matrices (eq. 17) are integrated with a collapsed Gauss rule on
// each face; LIFT = M^{-1} F.  Volume quadrature (eq. 19): the conical
// product of Gauss-Jacobi rules with N+1 points per direction (degree
// 2N+1), nodes from Sturm-sequence bisection of the Jacobi matrix and
// weights from the Christoffel function.
#include "refelem.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace wadg {

const int kFacePerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                             {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
const int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

int n_nodes(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
int n_face_nodes(int N) { return (N + 1) * (N + 2) / 2; }

namespace {

// ---------------------------------------------------------- Jacobi family
double jacobi_norm0(double al, double be) {
  // integral of (1-x)^al (1+x)^be over [-1, 1]
  return std::pow(2.0, al + be + 1) * std::tgamma(al + 1) * std::tgamma(be + 1) /
         std::tgamma(al + be + 2);
}

// a_n of x P_n = a_{n+1} P_{n+1} + b_n P_n + a_n P_{n-1} (orthonormal family)
double rec_a(int n, double al, double be) {
  double h = 2.0 * n + al + be;
  return 2.0 / h *
         std::sqrt(n * (n + al + be) * (n + al) * (n + be) / ((h - 1.0) * (h + 1.0)));
}
double rec_b(int n, double al, double be) {
  if (n == 0) return (be - al) / (al + be + 2.0);
  double h = 2.0 * n + al + be;
  return -(al * al - be * be) / (h * (h + 2.0));
}

// orthonormal Jacobi polynomial P_n^(al,be)(x)
double jacobi(double x, double al, double be, int n) {
  double p0 = 1.0 / std::sqrt(jacobi_norm0(al, be));
  if (n == 0) return p0;
  double a1 = rec_a(1, al, be);
  double p1 = (x - rec_b(0, al, be)) * p0 / a1;
  double pm = p0, pc = p1;
  for (int k = 1; k < n; ++k) {
    double an = rec_a(k, al, be), an1 = rec_a(k + 1, al, be);
    double pn = ((x - rec_b(k, al, be)) * pc - an * pm) / an1;
    pm = pc;
    pc = pn;
  }
  return pc;
}

double jacobi_deriv(double x, double al, double be, int n) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + al + be + 1.0)) * jacobi(x, al + 1, be + 1, n - 1);
}

// Gauss-Jacobi nodes and weights with n points
void gauss_jacobi(int n, double al, double be, std::vector<double>& x,
                  std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  std::vector<double> d(n), o(n > 1 ? n - 1 : 1);
  for (int k = 0; k < n; ++k) d[k] = rec_b(k, al, be);
  for (int k = 0; k + 1 < n; ++k) o[k] = rec_a(k + 1, al, be);
  auto count_below = [&](double s) {  // eigenvalues of the Jacobi matrix < s
    int c = 0;
    double q = d[0] - s;
    if (q < 0) ++c;
    for (int k = 1; k < n; ++k) {
      if (q == 0.0) q = 1e-300;
      q = (d[k] - s) - o[k - 1] * o[k - 1] / q;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int k = 0; k < n; ++k) {
    double lo = -1.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (count_below(mid) > k) hi = mid; else lo = mid;
      if (hi - lo < 1e-17) break;
    }
    double r = 0.5 * (lo + hi);
    for (int it = 0; it < 3; ++it) {  // Newton polish on P_n
      double f = jacobi(r, al, be, n), df = jacobi_deriv(r, al, be, n);
      if (df != 0.0) r -= f / df;
    }
    x[k] = r;
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      double p = jacobi(r, al, be, j);
      s += p * p;
    }
    w[k] = 1.0 / s;
  }
}

// ------------------------------------------------------- tetrahedron basis
struct Mode { int i, j, k; };

std::vector<Mode> modes(int N) {
  std::vector<Mode> m;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; i + j <= N; ++j)
      for (int k = 0; i + j + k <= N; ++k) m.push_back({i, j, k});
  return m;
}

void collapse(double r, double s, double t, double& a, double& b, double& c) {
  double den = -(s + t);
  a = std::fabs(den) > 1e-14 ? 2.0 * (1.0 + r) / den - 1.0 : -1.0;
  b = std::fabs(1.0 - t) > 1e-14 ? 2.0 * (1.0 + s) / (1.0 - t) - 1.0 : -1.0;
  c = t;
}

double ipow(double x, int e) {
  if (e < 0) return 0.0;
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// value and gradient of phi_m at (r,s,t)
void basis_eval(const Mode& md, double r, double s, double t, double* val,
                double* dr, double* ds, double* dt) {
  const double C = 2.0 * std::sqrt(2.0);
  double a, b, c;
  collapse(r, s, t, a, b, c);
  int i = md.i, j = md.j, k = md.k;
  double fa = jacobi(a, 0, 0, i), dfa = jacobi_deriv(a, 0, 0, i);
  double gb = jacobi(b, 2 * i + 1, 0, j), dgb = jacobi_deriv(b, 2 * i + 1, 0, j);
  double hc = jacobi(c, 2 * i + 2 * j + 2, 0, k);
  double dhc = jacobi_deriv(c, 2 * i + 2 * j + 2, 0, k);
  if (val) *val = C * fa * gb * ipow(1 - b, i) * hc * ipow(1 - c, i + j);
  if (!dr) return;
  // d(gb (1-b)^i)/db and d(hc (1-c)^(i+j))/dc
  double g_full = dgb * ipow(1 - b, i) - (i > 0 ? i * gb * ipow(1 - b, i - 1) : 0.0);
  double h_full = dhc * ipow(1 - c, i + j) -
                  (i + j > 0 ? (i + j) * hc * ipow(1 - c, i + j - 1) : 0.0);
  // r enters through a only: da/dr = 4/((1-b)(1-c))
  double vr = (i > 0) ? 4.0 * dfa * gb * ipow(1 - b, i - 1) * hc * ipow(1 - c, i + j - 1) : 0.0;
  // s: through a (da/ds = 2(1+a)/((1-b)(1-c))) and b (db/ds = 2/(1-c))
  double sa = (i > 0) ? 2.0 * (1 + a) * dfa * gb * ipow(1 - b, i - 1) * hc *
                            ipow(1 - c, i + j - 1)
                      : 0.0;
  double sb = (i + j > 0) ? 2.0 * fa * g_full * hc * ipow(1 - c, i + j - 1) : 0.0;
  // t: through a (as for s), b (db/dt = (1+b)/(1-c)) and c
  double tb = (i + j > 0) ? fa * g_full * (1 + b) * hc * ipow(1 - c, i + j - 1) : 0.0;
  double tc = fa * gb * ipow(1 - b, i) * h_full;
  *dr = C * vr;
  *ds = C * (sa + sb);
  *dt = C * (sa + tb + tc);
}

// --------------------------------------------------------- dense algebra
// in-place inverse by Gauss-Jordan elimination with partial pivoting
bool invert(std::vector<double>& A, int n) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r * n + col]) > std::fabs(A[piv * n + col])) piv = r;
    if (A[piv * n + col] == 0.0) return false;
    if (piv != col)
      for (int c = 0; c < n; ++c) {
        std::swap(A[piv * n + c], A[col * n + c]);
        std::swap(I[piv * n + c], I[col * n + c]);
      }
    double d = 1.0 / A[col * n + col];
    for (int c = 0; c < n; ++c) {
      A[col * n + c] *= d;
      I[col * n + c] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = A[r * n + col];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        A[r * n + c] -= f * A[col * n + c];
        I[r * n + c] -= f * I[col * n + c];
      }
    }
  }
  A.swap(I);
  return true;
}

// C[m][n] = A[m][k] * B[k][n]
std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B,
                           int m, int k, int n) {
  std::vector<double> C(static_cast<size_t>(m) * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < k; ++l) {
      double a = A[i * k + l];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[i * n + j] += a * B[l * n + j];
    }
  return C;
}

}  // namespace

std::vector<double> RefOps::lagrange_at(double rr, double ss, double tt) const {
  auto md = modes(N);
  std::vector<double> phi(Np), out(Np, 0.0);
  for (int m = 0; m < Np; ++m) basis_eval(md[m], rr, ss, tt, &phi[m], nullptr, nullptr, nullptr);
  for (int i = 0; i < Np; ++i)
    for (int m = 0; m < Np; ++m) out[i] += phi[m] * Vinv[m * Np + i];
  return out;
}

void stroud_rule(int n, std::vector<double>& r, std::vector<double>& s, std::vector<double>& t,
                 std::vector<double>& w) {
  // conical product of Gauss-Jacobi rules with weights (1-x)^0, (1-x)^1,
  // (1-x)^2 on the collapsed coordinates: n^3 points, degree 2n - 1
  std::vector<double> xa, wa, xb, wb, xc, wc;
  gauss_jacobi(n, 0, 0, xa, wa);
  gauss_jacobi(n, 1, 0, xb, wb);
  gauss_jacobi(n, 2, 0, xc, wc);
  r.clear(); s.clear(); t.clear(); w.clear();
  for (int ia = 0; ia < n; ++ia)
    for (int ib = 0; ib < n; ++ib)
      for (int ic = 0; ic < n; ++ic) {
        const double a = xa[ia], b = xb[ib], c = xc[ic];
        r.push_back(0.25 * (1 + a) * (1 - b) * (1 - c) - 1.0);
        s.push_back(0.5 * (1 + b) * (1 - c) - 1.0);
        t.push_back(c);
        w.push_back(wa[ia] * wb[ib] * wc[ic] / 8.0);
      }
}

bool set_volume_rule(RefOps& o, const std::vector<double>& r, const std::vector<double>& s,
                     const std::vector<double>& t, const std::vector<double>& w, int pad_to,
                     const char** err) {
  const int Np = o.Np;
  const int n = static_cast<int>(w.size());
  if (n < 1 || r.size() != w.size() || s.size() != w.size() || t.size() != w.size()) {
    *err = "empty or inconsistent quadrature rule";
    return false;
  }
  for (int q = 0; q < n; ++q) {
    // barycentric coordinates of the point on the reference tetrahedron
    const double l1 = 0.5 * (1.0 + r[q]), l2 = 0.5 * (1.0 + s[q]), l3 = 0.5 * (1.0 + t[q]);
    const double l0 = 1.0 - l1 - l2 - l3;
    if (!(w[q] > 0.0) || l0 < -1e-12 || l1 < -1e-12 || l2 < -1e-12 || l3 < -1e-12) {
      *err = "quadrature weights must be positive and points inside the tetrahedron";
      return false;
    }
  }
  const int Nq = pad_to > n ? pad_to : n;
  // padding points: zero weight at the centroid (no contribution to P_q)
  std::vector<double> rr(r), ss(s), tt(t), ww(w);
  for (int q = n; q < Nq; ++q) {
    rr.push_back(-0.5);
    ss.push_back(-0.5);
    tt.push_back(-0.5);
    ww.push_back(0.0);
  }
  std::vector<double> Vq(static_cast<size_t>(Nq) * Np), Pq(static_cast<size_t>(Np) * Nq);
  for (int q = 0; q < Nq; ++q) {
    std::vector<double> l = o.lagrange_at(rr[q], ss[q], tt[q]);
    for (int i = 0; i < Np; ++i) Vq[static_cast<size_t>(q) * Np + i] = l[i];
  }
  // P_q = M^{-1} V_q^T W
  for (int i = 0; i < Np; ++i)
    for (int q = 0; q < Nq; ++q) {
      double a = 0.0;
      for (int j = 0; j < Np; ++j) a += o.Minv[i * Np + j] * Vq[static_cast<size_t>(q) * Np + j];
      Pq[static_cast<size_t>(i) * Nq + q] = a * ww[q];
    }
  // the rule must integrate products of two degree-N polynomials exactly:
  // P_q V_q = M^{-1} (V_q^T W V_q) is then the identity
  double dev = 0.0;
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double a = 0.0;
      for (int q = 0; q < Nq; ++q)
        a += Pq[static_cast<size_t>(i) * Nq + q] * Vq[static_cast<size_t>(q) * Np + j];
      dev = std::max(dev, std::fabs(a - (i == j ? 1.0 : 0.0)));
    }
  if (!(dev < 1e-10)) {
    *err = "the quadrature rule is not exact for polynomials of degree 2N (P_q V_q != I)";
    return false;
  }
  o.rq = rr;
  o.sq = ss;
  o.tq = tt;
  o.wq = ww;
  o.Nq = Nq;
  o.Nq_rule = n;
  o.Vq = Vq;
  o.Pq = Pq;
  return true;
}

bool build_ref_ops(int N, RefOps& o, const char** err) {
  if (N < 1 || N > 6) {
    *err = "polynomial order N must be in 1..6";
    return false;
  }
  o.N = N;
  o.Np = n_nodes(N);
  o.Nfp = n_face_nodes(N);
  const int Np = o.Np, Nfp = o.Nfp;
  o.r.clear(); o.s.clear(); o.t.clear(); o.bary.clear();
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j + k <= N; ++j)
      for (int i = 0; i + j + k <= N; ++i) {
        o.r.push_back(-1.0 + 2.0 * i / N);
        o.s.push_back(-1.0 + 2.0 * j / N);
        o.t.push_back(-1.0 + 2.0 * k / N);
        o.bary.insert(o.bary.end(), {N - i - j - k, i, j, k});
      }
  auto md = modes(N);
  o.V.assign(Np * Np, 0.0);
  std::vector<double> Vr(Np * Np), Vs(Np * Np), Vt(Np * Np);
  for (int p = 0; p < Np; ++p)
    for (int m = 0; m < Np; ++m)
      basis_eval(md[m], o.r[p], o.s[p], o.t[p], &o.V[p * Np + m], &Vr[p * Np + m],
                 &Vs[p * Np + m], &Vt[p * Np + m]);
  o.Vinv = o.V;
  if (!invert(o.Vinv, Np)) {
    *err = "singular Vandermonde matrix";
    return false;
  }
  // M^{-1} = V V^T for an orthonormal basis
  o.Minv.assign(Np * Np, 0.0);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      double a = 0.0;
      for (int m = 0; m < Np; ++m) a += o.V[i * Np + m] * o.V[j * Np + m];
      o.Minv[i * Np + j] = a;
    }
  o.Dr = matmul(Vr, o.Vinv, Np, Np, Np);
  o.Ds = matmul(Vs, o.Vinv, Np, Np, Np);
  o.Dt = matmul(Vt, o.Vinv, Np, Np, Np);
  // face node lists: barycentric coordinate of the opposite vertex is zero
  const int opp[4] = {3, 2, 0, 1};
  o.Fmask.clear();
  for (int f = 0; f < 4; ++f)
    for (int p = 0; p < Np; ++p)
      if (o.bary[p * 4 + opp[f]] == 0) o.Fmask.push_back(p);
  if (static_cast<int>(o.Fmask.size()) != 4 * Nfp) {
    *err = "face node count mismatch";
    return false;
  }
  // face mass matrices on the reference triangle (-1,-1),(1,-1),(-1,1) of
  // area 2 in each face's own pair of coordinates, by a collapsed Gauss rule
  std::vector<double> xa, wa, xb, wb;
  gauss_jacobi(N + 1, 0, 0, xa, wa);
  gauss_jacobi(N + 1, 1, 0, xb, wb);
  std::vector<double> E(static_cast<size_t>(Np) * 4 * Nfp, 0.0);
  for (int f = 0; f < 4; ++f) {
    for (int qa = 0; qa <= N; ++qa)
      for (int qb = 0; qb <= N; ++qb) {
        double u = 0.5 * (1 + xa[qa]) * (1 - xb[qb]) - 1.0;
        double v = xb[qb];
        double w = wa[qa] * wb[qb] * 0.5;
        double rr, ss, tt;
        switch (f) {
          case 0: rr = u; ss = v; tt = -1.0; break;
          case 1: rr = u; ss = -1.0; tt = v; break;
          case 2: rr = u; ss = v; tt = -1.0 - u - v; break;
          default: rr = -1.0; ss = u; tt = v; break;
        }
        std::vector<double> l = o.lagrange_at(rr, ss, tt);
        for (int i = 0; i < Np; ++i)
          for (int m = 0; m < Nfp; ++m)
            E[static_cast<size_t>(i) * 4 * Nfp + f * Nfp + m] +=
                w * l[i] * l[o.Fmask[f * Nfp + m]];
      }
  }
  o.LIFT = matmul(o.Minv, E, Np, Np, 4 * Nfp);
  // default volume quadrature: the conical-product rule of degree 2N+1
  {
    std::vector<double> qr, qs, qt, qw;
    stroud_rule(N + 1, qr, qs, qt, qw);
    if (!set_volume_rule(o, qr, qs, qt, qw, 0, err)) return false;
  }
  // face-node permutation table
  o.fperm.assign(4 * 24 * Nfp, -1);
  o.fmap.assign(4 * 24 * Nfp, 0);
  for (int f = 0; f < 4; ++f)
    for (int nf = 0; nf < 4; ++nf)
      for (int rot = 0; rot < 6; ++rot)
        for (int m = 0; m < Nfp; ++m) {
          int node = o.Fmask[f * Nfp + m];
          int mu[3];
          for (int i = 0; i < 3; ++i) mu[i] = o.bary[node * 4 + kFaceVerts[f][i]];
          // neighbour local face vertex i sits on our face vertex kFacePerm[rot][i]
          int want[4] = {0, 0, 0, 0};
          for (int i = 0; i < 3; ++i) want[kFaceVerts[nf][i]] = mu[kFacePerm[rot][i]];
          for (int p = 0; p < Np; ++p) {
            const int* bb = &o.bary[p * 4];
            if (bb[0] == want[0] && bb[1] == want[1] && bb[2] == want[2] && bb[3] == want[3]) {
              o.fperm[(f * 24 + nf * 6 + rot) * Nfp + m] = p;
              for (int m2 = 0; m2 < Nfp; ++m2)
                if (o.Fmask[nf * Nfp + m2] == p) o.fmap[(f * 24 + nf * 6 + rot) * Nfp + m] = m2;
              break;
            }
          }
        }
  return true;
}

}  // namespace wadg
