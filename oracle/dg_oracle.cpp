// Plain FP64 CPU oracle for the discontinuous Galerkin discretisation of the
// incompressible Navier-Stokes equations (artificial-compressibility Riemann
// flux, BR2 viscous lifting, orthonormal modal P^k basis on boxes) of
// Franciolini, Botti, Colombo, Crivellini, "p-Multigrid matrix-free
// discontinuous Galerkin solution strategies for the under-resolved
// simulation of incompressible turbulent flows" (arXiv 1809.00866).
//
// TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
// legs of the benchmark load this library. It shares no code, header, table or
// helper with the CUDA path.
//
// Everything is computed from its definition, in the order the paper states
// it: basis functions are evaluated from Legendre polynomials at every point,
// integrals are Gauss sums, the fluxes are evaluated point by point, the
// Jacobian action is the exact forward-mode derivative of the residual
// (dual numbers), and the Riemann star state is found by bisection. No tables,
// no sum factorisation, no fusion.
//
// Readings of the paper that this file fixes:
//  * basis: normalised tensor Legendre polynomials of total degree <= k on each
//    box, ordered by total degree, then first index descending, then second
//    index descending (Sec. 2.4.1: hierarchical orthonormal modal basis);
//  * quadrature: Gauss-Legendre with k+1 points per direction;
//  * lifting sign: the lifting r^s([v]) is defined by
//      int_{K u K'} r . tau = + int_s [v] {tau} . n
//    so that grad v - R^K(v) is the consistent (distributional) gradient of
//    Sec. 2.1 and the BR2 fluxes of Eq. (vflux) read as printed;
//  * n^s points from K (lower index along the face axis) to K'; [v] = v_K - v_K';
//  * the artificial-compressibility Riemann problem (Sec. 2.1) is solved
//    exactly from the 1D system p_t + c^2 (u_n)_x = 0,
//    (u_n)_t + (u_n^2 + p)_x = 0, (u_t)_t + (u_n u_t)_x = 0, including the
//    change of the tangential velocity across the two acoustic waves;
//    when |u*| is within a rounding band of zero the two contact sides are
//    averaged;
//  * walls (optional, at y = yn[0] and y = yn[ny], no-slip data f = 0; Sec. 2.1,
//    Dirichlet viscous flux and ghost boundary state): the ghost state keeps the
//    Riemann invariants of the interior and makes the interface velocity the data,
//    (u_gb, p_gb) = (2 f - u_K, p_K); the same exact Riemann solver then gives
//    u* = f.n, so no mass crosses a wall; the jump is [u] = u_K - f; the lifting of
//    a wall face lives on K alone, int_K r . tau = int_s [u] tau . n (the one-sided
//    average), and the viscous flux is F^nu(grad u_K - eta r([u])).

#include <omp.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace orc {

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
static inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
static inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
static inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
static inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
static inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
static inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
static inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
static inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
static inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
static inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
static inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
static inline Dual asinh(Dual a) { return Dual(std::asinh(a.v), a.d / std::sqrt(1.0 + a.v * a.v)); }
static inline double val(double x) { return x; }
static inline double val(const Dual& x) { return x.v; }
using std::sqrt;
using std::asinh;

// ------------------------------------------------------ Legendre and quadrature
// L_n(x) by the three-term recurrence (n+1) L_{n+1} = (2n+1) x L_n - n L_{n-1}.
static double legendre(int n, double x) {
  if (n == 0) return 1.0;
  double a = 1.0, b = x;
  for (int j = 1; j < n; ++j) {
    double c = ((2.0 * j + 1.0) * x * b - j * a) / (j + 1.0);
    a = b;
    b = c;
  }
  return b;
}
// L_n'(x) from L'_{j+1} = L'_{j-1} + (2j+1) L_j.
static double dlegendre(int n, double x) {
  if (n == 0) return 0.0;
  double dm1 = 0.0, d0 = 1.0;  // L_0', L_1'
  for (int j = 1; j < n; ++j) {
    double d1 = dm1 + (2.0 * j + 1.0) * legendre(j, x);
    dm1 = d0;
    d0 = d1;
  }
  return d0;
}
// Gauss-Legendre nodes (ascending) and weights on [-1,1]: Newton on L_n.
static void gauss(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double t = std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double dt = legendre(n, t) / dlegendre(n, t);
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double dp = dlegendre(n, t);
    x[n - 1 - i] = t;
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// --------------------------------------------------------------------- basis
struct Mode { int e[3]; };
static std::vector<Mode> modes(int k) {
  std::vector<Mode> m;
  for (int t = 0; t <= k; ++t)
    for (int a = t; a >= 0; --a)
      for (int b = t - a; b >= 0; --b) m.push_back(Mode{{a, b, t - a - b}});
  return m;
}

// Normalised 1D Legendre polynomial sqrt((2n+1)/2) L_n, orthonormal on [-1,1].
static double lhat(int n, double x) { return std::sqrt((2.0 * n + 1.0) / 2.0) * legendre(n, x); }
static double dlhat(int n, double x) { return std::sqrt((2.0 * n + 1.0) / 2.0) * dlegendre(n, x); }

}  // namespace orc

// ---------------------------------------------------------------- C interface
extern "C" {
typedef struct orc_mesh {
  int nx, ny, nz, k;
  int nq;  // Gauss points per direction; 0 selects k+1
  double nu, c, eta;
  const double* xn;  // nx+1 node coordinates along x (periodic box)
  const double* yn;
  const double* zn;
  int wall_y;  // 1: no-slip walls at y = yn[0] and y = yn[ny] (else periodic)
} orc_mesh;
}

namespace orc {

struct Disc {
  int n[3];
  int k, nb, nq;  // degree, modes per variable, Gauss points per direction
  double nu, c, eta;
  std::vector<double> node[3];
  std::vector<Mode> md;
  std::vector<double> gx, gw;
  int ne;
  bool wall_y;
  Disc(const orc_mesh* m) {
    n[0] = m->nx; n[1] = m->ny; n[2] = m->nz;
    k = m->k;
    nu = m->nu; c = m->c; eta = m->eta;
    node[0].assign(m->xn, m->xn + n[0] + 1);
    node[1].assign(m->yn, m->yn + n[1] + 1);
    node[2].assign(m->zn, m->zn + n[2] + 1);
    md = modes(k);
    nb = (int)md.size();
    nq = m->nq > 0 ? m->nq : k + 1;
    gauss(nq, gx, gw);
    ne = n[0] * n[1] * n[2];
    wall_y = m->wall_y != 0;
  }
  void ijk(int e, int* I) const {
    I[0] = e % n[0];
    I[1] = (e / n[0]) % n[1];
    I[2] = e / (n[0] * n[1]);
  }
  int elem(const int* I) const { return I[0] + n[0] * (I[1] + n[1] * I[2]); }
  // neighbour across the face normal to axis d, on the + side (s=+1) or - side (s=-1);
  // -1 across a wall
  int nbr(int e, int d, int s) const {
    int I[3];
    ijk(e, I);
    if (wall_y && d == 1 && (I[1] + s < 0 || I[1] + s >= n[1])) return -1;
    I[d] = (I[d] + s + n[d]) % n[d];
    return elem(I);
  }
  double h(int e, int d) const {
    int I[3];
    ijk(e, I);
    return node[d][I[d] + 1] - node[d][I[d]];
  }
  double center(int e, int d) const {
    int I[3];
    ijk(e, I);
    return 0.5 * (node[d][I[d] + 1] + node[d][I[d]]);
  }
  double vol(int e) const { return h(e, 0) * h(e, 1) * h(e, 2); }
  // physical basis function phi_m of element e at reference point xi, and its
  // physical gradient. phi_m = prod_d sqrt((2n_d+1)/h_d) L_{n_d}(xi_d), which is
  // orthonormal on the box.
  void eval(int e, const double* xi, double* phi, double* dphi) const {
    double s = std::sqrt(vol(e) / 8.0);
    double J[3] = {2.0 / h(e, 0), 2.0 / h(e, 1), 2.0 / h(e, 2)};
    for (int m = 0; m < nb; ++m) {
      double L[3], dL[3];
      for (int d = 0; d < 3; ++d) {
        L[d] = lhat(md[m].e[d], xi[d]);
        dL[d] = dlhat(md[m].e[d], xi[d]);
      }
      phi[m] = L[0] * L[1] * L[2] / s;
      if (dphi) {
        dphi[3 * m + 0] = J[0] * dL[0] * L[1] * L[2] / s;
        dphi[3 * m + 1] = J[1] * L[0] * dL[1] * L[2] / s;
        dphi[3 * m + 2] = J[2] * L[0] * L[1] * dL[2] / s;
      }
    }
  }
};

// --------------------------------------------------- artificial-compressibility
// 1D system along the face normal: p_t + c^2 (u_n)_x = 0, (u_n)_t + (u_n^2+p)_x = 0,
// (u_t)_t + (u_n u_t)_x = 0. Wave speeds u_n -+ sqrt(u_n^2+c^2) (always of
// opposite signs) and u_n (contact), so the interface state is the star state.

// Antiderivatives of the rarefaction slopes: along a 1-wave dp/du = -(u + a),
// along a 3-wave dp/du = a - u, with a = sqrt(u^2 + c^2).
template <class T> static T rar1(T s, double c) {
  T a = sqrt(s * s + c * c);
  return 0.5 * (s * s + s * a + c * c * asinh(s / c));
}
template <class T> static T rar3(T s, double c) {
  T a = sqrt(s * s + c * c);
  return 0.5 * (s * a + c * c * asinh(s / c) - s * s);
}
// Pressure on the 1-wave curve through (uL, pL) as a function of the star velocity u:
// a shock (Rankine-Hugoniot, speed the negative root of s^2 - s(uL+u) - c^2 = 0)
// when u < uL, a rarefaction when u >= uL.
template <class T> static T p_wave1(T u, T uL, T pL, double c) {
  if (val(u) < val(uL)) {
    T sig = uL + u;
    T s = 0.5 * (sig - sqrt(sig * sig + 4.0 * c * c));
    return pL + c * c * (u - uL) / s;
  }
  return pL - (rar1(u, c) - rar1(uL, c));
}
// Pressure on the 3-wave curve through (uR, pR): a shock when u > uR
// (positive root), a rarefaction when u <= uR.
template <class T> static T p_wave3(T u, T uR, T pR, double c) {
  if (val(u) > val(uR)) {
    T sig = u + uR;
    T s = 0.5 * (sig + sqrt(sig * sig + 4.0 * c * c));
    return pR + c * c * (u - uR) / s;
  }
  return pR - (rar3(uR, c) - rar3(u, c));
}
// Ratio u_t(star, left of contact) / u_t,L across the 1-wave: along a
// rarefaction u_t (u + a) is invariant; across a shock s[u_t] = [u_n u_t].
template <class T> static T tang1(T u, T uL, double c) {
  if (val(u) < val(uL)) {
    T sig = uL + u;
    T s = 0.5 * (sig - sqrt(sig * sig + 4.0 * c * c));
    return (s - uL) / (s - u);
  }
  return (uL + sqrt(uL * uL + c * c)) / (u + sqrt(u * u + c * c));
}
// Ratio u_t(star, right of contact) / u_t,R across the 3-wave: along a
// rarefaction u_t / (u + a) is invariant.
template <class T> static T tang3(T u, T uR, double c) {
  if (val(u) > val(uR)) {
    T sig = u + uR;
    T s = 0.5 * (sig + sqrt(sig * sig + 4.0 * c * c));
    return (s - uR) / (s - u);
  }
  return (u + sqrt(u * u + c * c)) / (uR + sqrt(uR * uR + c * c));
}
template <class T> static T star_fun(T u, T uL, T pL, T uR, T pR, double c) {
  return p_wave1(u, uL, pL, c) - p_wave3(u, uR, pR, c);
}

// Star velocity by bisection on the decreasing function p_wave1 - p_wave3.
static double star_bisect(double uL, double pL, double uR, double pR, double c) {
  double scale = std::fabs(uL) + std::fabs(uR) + c;
  double lo = std::fmin(uL, uR) - scale, hi = std::fmax(uL, uR) + scale;
  for (int i = 0; i < 200 && star_fun(lo, uL, pL, uR, pR, c) < 0.0; ++i) lo -= (hi - lo);
  for (int i = 0; i < 200 && star_fun(hi, uL, pL, uR, pR, c) > 0.0; ++i) hi += (hi - lo);
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (star_fun(mid, uL, pL, uR, pR, c) > 0.0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

// Inviscid interface flux along n = e_d: flux[i] = n.(u (x) u + pI) for the three
// momentum equations and flux[3] = u_hat . n for the continuity equation.
// Also returns the star state (u*, p*, and the interface tangential velocity).
template <class T>
static void riemann_flux(const T* uL, T pL, const T* uR, T pR, int d, double c, T* flux, T* ustar_out,
                         T* pstar_out, T* uface_out) {
  double us = star_bisect(val(uL[d]), val(pL), val(uR[d]), val(pR), c);
  // implicit function theorem: u* = u*_0 - phi(u*_0; inputs) / phi'(u*_0)
  Dual dphi = star_fun(Dual(us, 1.0), Dual(val(uL[d])), Dual(val(pL)), Dual(val(uR[d])), Dual(val(pR)), c);
  T phiT = star_fun(T(us), uL[d], pL, uR[d], pR, c);
  T ust = T(us) - phiT / dphi.d;
  T pst = p_wave1(ust, uL[d], pL, c);
  double band = 1e-12 * (std::fabs(val(uL[d])) + std::fabs(val(uR[d])) + c);
  T uf[3];
  for (int i = 0; i < 3; ++i) {
    if (i == d) { uf[i] = ust; continue; }
    if (val(ust) > band) uf[i] = uL[i] * tang1(ust, uL[d], c);
    else if (val(ust) < -band) uf[i] = uR[i] * tang3(ust, uR[d], c);
    else uf[i] = 0.5 * (uL[i] * tang1(ust, uL[d], c) + uR[i] * tang3(ust, uR[d], c));
  }
  for (int i = 0; i < 3; ++i) flux[i] = uf[i] * ust + (i == d ? pst : T(0.0));
  flux[3] = ust;
  if (ustar_out) *ustar_out = ust;
  if (pstar_out) *pstar_out = pst;
  if (uface_out) for (int i = 0; i < 3; ++i) uface_out[i] = uf[i];
}

// ---------------------------------------------------------------- the residual
// f_h(w; z) of Eq. (NSdiscrRes) for every basis test function z = phi_m e_i,
// with w and f laid out [element][variable u,v,w,p][mode].
template <class T> static void residual(const Disc& D, const T* w, T* f) {
  const int nb = D.nb, nq = D.nq, ne = D.ne;
  const double nu = D.nu, eta = D.eta;
  for (size_t i = 0; i < (size_t)ne * 4 * nb; ++i) f[i] = T(0.0);
  auto W = [&](int e, int v, int m) -> const T& { return w[((size_t)e * 4 + v) * nb + m]; };
  auto F = [&](int e, int v, int m) -> T& { return f[((size_t)e * 4 + v) * nb + m]; };

  // 1. local lifting operators r^s([u_a]) of every face s = (K, d), as modal
  //    coefficients on K (side 0) and on K' (side 1); only component d is non-zero.
  std::vector<T> lift((size_t)ne * 3 * 2 * 3 * nb, T(0.0));
  auto LIFT = [&](int e, int d, int side, int a, int m) -> T& {
    return lift[((((size_t)e * 3 + d) * 2 + side) * 3 + a) * nb + m];
  };
  // lifting of the wall face at the - side (y = yn[0]) of K, on K
  std::vector<T> liftb((size_t)ne * 3 * nb, T(0.0));
  auto LIFTB = [&](int e, int a, int m) -> T& { return liftb[((size_t)e * 3 + a) * nb + m]; };
  // (the faces (K, d) of different K write different coefficients: K runs in parallel)
#pragma omp parallel for schedule(static)
  for (int K = 0; K < ne; ++K) {
    std::vector<double> phiK(nb), phiP(nb);
    for (int d = 0; d < 3; ++d) {
      int P = D.nbr(K, d, +1);
      int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      for (int q1 = 0; q1 < nq; ++q1)
        for (int q2 = 0; q2 < nq; ++q2) {
          double xiK[3], xiP[3];
          xiK[d] = 1.0; xiP[d] = -1.0;
          xiK[t1] = xiP[t1] = D.gx[q1];
          xiK[t2] = xiP[t2] = D.gx[q2];
          double wq = D.gw[q1] * D.gw[q2] * 0.25 * D.h(K, t1) * D.h(K, t2);
          D.eval(K, xiK, phiK.data(), nullptr);
          if (P >= 0) D.eval(P, xiP, phiP.data(), nullptr);
          for (int a = 0; a < 3; ++a) {
            T uk = T(0.0), up = T(0.0);
            for (int m = 0; m < nb; ++m) {
              uk += W(K, a, m) * phiK[m];
              if (P >= 0) up += W(P, a, m) * phiP[m];
            }
            T jump = uk - up;  // at a wall: u_K - f with f = 0
            for (int m = 0; m < nb; ++m) {
              if (P >= 0) {
                LIFT(K, d, 0, a, m) += 0.5 * wq * jump * phiK[m];
                LIFT(K, d, 1, a, m) += 0.5 * wq * jump * phiP[m];
              } else {
                LIFT(K, d, 0, a, m) += wq * jump * phiK[m];
              }
            }
          }
        }
      // the wall face below K (K on the + side of the face): [u] = f - u_K
      if (d == 1 && D.nbr(K, 1, -1) < 0)
        for (int q1 = 0; q1 < nq; ++q1)
          for (int q2 = 0; q2 < nq; ++q2) {
            double xiK[3];
            xiK[1] = -1.0;
            xiK[t1] = D.gx[q1];
            xiK[t2] = D.gx[q2];
            double wq = D.gw[q1] * D.gw[q2] * 0.25 * D.h(K, t1) * D.h(K, t2);
            D.eval(K, xiK, phiK.data(), nullptr);
            for (int a = 0; a < 3; ++a) {
              T uk = T(0.0);
              for (int m = 0; m < nb; ++m) uk += W(K, a, m) * phiK[m];
              T jump = -uk;
              for (int m = 0; m < nb; ++m) LIFTB(K, a, m) += wq * jump * phiK[m];
            }
          }
    }

  }

  // 2. volume terms: - int_K Ftilde_{p,i}(w) d_p z_i with the BR2 corrected
  //    gradient grad u - R^K(u), R^K = sum of the liftings of the faces of K
  //    (each K writes only its own residual: K runs in parallel).
#pragma omp parallel for schedule(static)
  for (int K = 0; K < ne; ++K) {
    std::vector<double> phiK(nb), dK(3 * nb);
    double vq = D.vol(K) / 8.0;
    for (int q0 = 0; q0 < nq; ++q0)
      for (int q1 = 0; q1 < nq; ++q1)
        for (int q2 = 0; q2 < nq; ++q2) {
          double xi[3] = {D.gx[q0], D.gx[q1], D.gx[q2]};
          double wq = D.gw[q0] * D.gw[q1] * D.gw[q2] * vq;
          D.eval(K, xi, phiK.data(), dK.data());
          T u[3], p = T(0.0), g[3][3];
          for (int a = 0; a < 3; ++a) {
            u[a] = T(0.0);
            for (int b = 0; b < 3; ++b) g[a][b] = T(0.0);
          }
          for (int m = 0; m < nb; ++m) {
            for (int a = 0; a < 3; ++a) {
              u[a] += W(K, a, m) * phiK[m];
              for (int b = 0; b < 3; ++b) g[a][b] += W(K, a, m) * dK[3 * m + b];
            }
            p += W(K, 3, m) * phiK[m];
          }
          // subtract R^K: face (K,b) has K on side 0, face (K-_b, b) has K on side 1
          for (int b = 0; b < 3; ++b) {
            int Km = D.nbr(K, b, -1);
            for (int a = 0; a < 3; ++a) {
              T r = T(0.0);
              for (int m = 0; m < nb; ++m)
                r += (LIFT(K, b, 0, a, m) + (Km >= 0 ? LIFT(Km, b, 1, a, m) : LIFTB(K, a, m))) * phiK[m];
              g[a][b] -= r;
            }
          }
          T div = g[0][0] + g[1][1] + g[2][2];
          T Ft[3][4];  // Ft[p][i]
          for (int pp = 0; pp < 3; ++pp) {
            for (int i = 0; i < 3; ++i) {
              T fv = nu * (g[i][pp] + g[pp][i]) - (pp == i ? (2.0 / 3.0) * nu * div : T(0.0));
              Ft[pp][i] = u[pp] * u[i] + (pp == i ? p : T(0.0)) - fv;
            }
            Ft[pp][3] = u[pp];
          }
          for (int i = 0; i < 4; ++i)
            for (int m = 0; m < nb; ++m) {
              T s = T(0.0);
              for (int pp = 0; pp < 3; ++pp) s += Ft[pp][i] * dK[3 * m + pp];
              F(K, i, m) -= wq * s;
            }
        }
  }

  // 3. face terms: + int_s n.(Fhat^c - Fhat^nu) [z] with the exact AC Riemann
  //    flux and Fhat^nu = F^nu({grad u - eta r^s([u])}); at a wall the ghost
  //    state (f, p_K) on the missing side and the one-sided Dirichlet flux.
  //    (a) the weighted normal flux w_q n.(Fhat^c - Fhat^nu) at every point of
  //        every face: the faces (K, d) of different K run in parallel;
  //    (b) the integral against the test functions of the two sides, element by
  //        element: + on K (the face's lower side), - on K' (its upper side).
  const size_t nqf = (size_t)nq * nq;
  std::vector<T> fl((size_t)ne * 3 * nqf * 4, T(0.0));   // [K][d][q1 q2][i], face (K, d)
  std::vector<T> flb(D.wall_y ? (size_t)ne * nqf * 4 : 0, T(0.0));  // [K][q1 q2][i], wall face below K
#pragma omp parallel for schedule(dynamic, 4)
  for (int K = 0; K < ne; ++K) {
    std::vector<double> phiK(nb), phiP(nb), dK(3 * nb), dP(3 * nb);
    for (int d = 0; d < 3; ++d) {
      int P = D.nbr(K, d, +1);
      int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      for (int q1 = 0; q1 < nq; ++q1)
        for (int q2 = 0; q2 < nq; ++q2) {
          double xiK[3], xiP[3];
          xiK[d] = 1.0; xiP[d] = -1.0;
          xiK[t1] = xiP[t1] = D.gx[q1];
          xiK[t2] = xiP[t2] = D.gx[q2];
          double wq = D.gw[q1] * D.gw[q2] * 0.25 * D.h(K, t1) * D.h(K, t2);
          D.eval(K, xiK, phiK.data(), dK.data());
          if (P >= 0) D.eval(P, xiP, phiP.data(), dP.data());
          T uk[3], up[3], pk = T(0.0), pp_ = T(0.0), gk[3][3], gp[3][3], rk[3], rp[3];
          for (int a = 0; a < 3; ++a) {
            uk[a] = up[a] = rk[a] = rp[a] = T(0.0);
            for (int b = 0; b < 3; ++b) gk[a][b] = gp[a][b] = T(0.0);
          }
          for (int m = 0; m < nb; ++m) {
            for (int a = 0; a < 3; ++a) {
              uk[a] += W(K, a, m) * phiK[m];
              for (int b = 0; b < 3; ++b) gk[a][b] += W(K, a, m) * dK[3 * m + b];
              rk[a] += LIFT(K, d, 0, a, m) * phiK[m];
              if (P >= 0) {
                up[a] += W(P, a, m) * phiP[m];
                for (int b = 0; b < 3; ++b) gp[a][b] += W(P, a, m) * dP[3 * m + b];
                rp[a] += LIFT(K, d, 1, a, m) * phiP[m];
              }
            }
            pk += W(K, 3, m) * phiK[m];
            if (P >= 0) pp_ += W(P, 3, m) * phiP[m];
          }
          T gh[3][3];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              if (P >= 0) {
                gh[a][b] = 0.5 * (gk[a][b] + gp[a][b]);
                if (b == d) gh[a][b] -= eta * 0.5 * (rk[a] + rp[a]);
              } else {  // wall: one-sided gradient and the full lifting of [u] = u_K - f
                gh[a][b] = gk[a][b];
                if (b == d) gh[a][b] -= eta * rk[a];
              }
            }
          if (P < 0) {  // ghost state (2 f - u_K, p_K), f = 0
            for (int a = 0; a < 3; ++a) up[a] = -uk[a];
            pp_ = pk;
          }
          T divh = gh[0][0] + gh[1][1] + gh[2][2];
          T fc[4];
          riemann_flux<T>(uk, pk, up, pp_, d, D.c, fc, nullptr, nullptr, nullptr);
          T fn[4];
          for (int i = 0; i < 3; ++i) {
            T fv = nu * (gh[i][d] + gh[d][i]) - (i == d ? (2.0 / 3.0) * nu * divh : T(0.0));
            fn[i] = fc[i] - fv;
          }
          fn[3] = fc[3];
          for (int i = 0; i < 4; ++i) fl[(((size_t)K * 3 + d) * nqf + q1 * nq + q2) * 4 + i] = wq * fn[i];
        }
      // the wall face below K: the ghost state on the - side, K on the + side
      if (d == 1 && D.nbr(K, 1, -1) < 0)
        for (int q1 = 0; q1 < nq; ++q1)
          for (int q2 = 0; q2 < nq; ++q2) {
            double xiK[3];
            xiK[1] = -1.0;
            xiK[t1] = D.gx[q1];
            xiK[t2] = D.gx[q2];
            double wq = D.gw[q1] * D.gw[q2] * 0.25 * D.h(K, t1) * D.h(K, t2);
            D.eval(K, xiK, phiK.data(), dK.data());
            T uk[3], ug[3], pk = T(0.0), gk[3][3], rk[3];
            for (int a = 0; a < 3; ++a) {
              uk[a] = ug[a] = rk[a] = T(0.0);
              for (int b = 0; b < 3; ++b) gk[a][b] = T(0.0);
            }
            for (int m = 0; m < nb; ++m) {
              for (int a = 0; a < 3; ++a) {
                uk[a] += W(K, a, m) * phiK[m];
                for (int b = 0; b < 3; ++b) gk[a][b] += W(K, a, m) * dK[3 * m + b];
                rk[a] += LIFTB(K, a, m) * phiK[m];
              }
              pk += W(K, 3, m) * phiK[m];
            }
            for (int a = 0; a < 3; ++a) ug[a] = -uk[a];  // ghost state (2 f - u_K, p_K), f = 0
            T gh[3][3];
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) gh[a][b] = gk[a][b] - (b == 1 ? eta * rk[a] : T(0.0));
            T divh = gh[0][0] + gh[1][1] + gh[2][2];
            T fc[4];
            riemann_flux<T>(ug, pk, uk, pk, 1, D.c, fc, nullptr, nullptr, nullptr);
            T fn[4];
            for (int i = 0; i < 3; ++i) {
              T fv = nu * (gh[i][1] + gh[1][i]) - (i == 1 ? (2.0 / 3.0) * nu * divh : T(0.0));
              fn[i] = fc[i] - fv;
            }
            fn[3] = fc[3];
            for (int i = 0; i < 4; ++i) flb[((size_t)K * nqf + q1 * nq + q2) * 4 + i] = wq * fn[i];
          }
    }
  }
#pragma omp parallel for schedule(static)
  for (int E = 0; E < ne; ++E) {
    std::vector<double> phi(nb);
    for (int d = 0; d < 3; ++d) {
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      const int Km = D.nbr(E, d, -1);  // the element below E's lower face (-1: a wall)
      for (int side = 0; side < 2; ++side) {  // 0: E is K of its face (E, d); 1: E is K' of (Km, d)
        const T* src = side == 0 ? &fl[(size_t)E * 3 * nqf * 4 + (size_t)d * nqf * 4]
                       : Km >= 0 ? &fl[(size_t)Km * 3 * nqf * 4 + (size_t)d * nqf * 4]
                                 : (d == 1 ? &flb[(size_t)E * nqf * 4] : nullptr);
        if (!src) continue;
        const double sgn = side == 0 ? 1.0 : -1.0;
        for (int q1 = 0; q1 < nq; ++q1)
          for (int q2 = 0; q2 < nq; ++q2) {
            double xi[3];
            xi[d] = side == 0 ? 1.0 : -1.0;
            xi[t1] = D.gx[q1];
            xi[t2] = D.gx[q2];
            D.eval(E, xi, phi.data(), nullptr);
            const T* fq = src + (size_t)(q1 * nq + q2) * 4;
            for (int i = 0; i < 4; ++i)
              for (int m = 0; m < nb; ++m) F(E, i, m) += sgn * fq[i] * phi[m];
          }
      }
    }
  }
}

// Taylor-Green initial field on [0,2pi]^3 (U0 = L = 1).
static void tgv(const double* x, double* out) {
  out[0] = std::sin(x[0]) * std::cos(x[1]) * std::cos(x[2]);
  out[1] = -std::cos(x[0]) * std::sin(x[1]) * std::cos(x[2]);
  out[2] = 0.0;
  out[3] = (1.0 / 16.0) * (std::cos(2.0 * x[0]) + std::cos(2.0 * x[1])) * (std::cos(2.0 * x[2]) + 2.0);
}

}  // namespace orc

using namespace orc;

extern "C" {

int orc_nb(int k) { return (int)modes(k).size(); }

// Threads of the OpenMP loops over elements (n > 0 sets them); returns the number in use.
// Every result is the same for any thread count: each loop iteration writes its own entries.
int orc_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
}

void orc_modes(int k, int* out) {
  auto m = modes(k);
  for (size_t i = 0; i < m.size(); ++i)
    for (int d = 0; d < 3; ++d) out[3 * i + d] = m[i].e[d];
}

void orc_gauss(int n, double* x, double* w) {
  std::vector<double> gx, gw;
  gauss(n, gx, gw);
  for (int i = 0; i < n; ++i) { x[i] = gx[i]; w[i] = gw[i]; }
}

void orc_legendre(int n, double x, double* val_out, double* der_out) {
  *val_out = legendre(n, x);
  *der_out = dlegendre(n, x);
}

// Basis functions and gradients of element e at reference points xi[npts][3]:
// phi[npts][nb], dphi[npts][nb][3].
void orc_basis(const orc_mesh* m, int e, int npts, const double* xi, double* phi, double* dphi) {
  Disc D(m);
  std::vector<double> ph(D.nb), dp(3 * D.nb);
  for (int i = 0; i < npts; ++i) {
    D.eval(e, xi + 3 * i, ph.data(), dp.data());
    for (int j = 0; j < D.nb; ++j) {
      phi[(size_t)i * D.nb + j] = ph[j];
      for (int d = 0; d < 3; ++d) dphi[((size_t)i * D.nb + j) * 3 + d] = dp[3 * j + d];
    }
  }
}

// Volume quadrature points and weights of every element: x[ne][nq^3][3], wq[ne][nq^3].
void orc_quad_points(const orc_mesh* m, double* x, double* wq) {
  Disc D(m);
  int nq = D.nq, npt = nq * nq * nq;
  for (int e = 0; e < D.ne; ++e) {
    int i = 0;
    for (int q0 = 0; q0 < nq; ++q0)
      for (int q1 = 0; q1 < nq; ++q1)
        for (int q2 = 0; q2 < nq; ++q2, ++i) {
          double xi[3] = {D.gx[q0], D.gx[q1], D.gx[q2]};
          for (int d = 0; d < 3; ++d) x[((size_t)e * npt + i) * 3 + d] = D.center(e, d) + 0.5 * D.h(e, d) * xi[d];
          wq[(size_t)e * npt + i] = D.gw[q0] * D.gw[q1] * D.gw[q2] * D.vol(e) / 8.0;
        }
  }
}

// L2 projection of point values vals[ne][4][nq^3] (at orc_quad_points) onto the basis.
void orc_project_points(const orc_mesh* m, const double* vals, double* w) {
  Disc D(m);
  int nq = D.nq, npt = nq * nq * nq, nb = D.nb;
  std::vector<double> ph(nb);
  for (size_t i = 0; i < (size_t)D.ne * 4 * nb; ++i) w[i] = 0.0;
  for (int e = 0; e < D.ne; ++e) {
    int i = 0;
    for (int q0 = 0; q0 < nq; ++q0)
      for (int q1 = 0; q1 < nq; ++q1)
        for (int q2 = 0; q2 < nq; ++q2, ++i) {
          double xi[3] = {D.gx[q0], D.gx[q1], D.gx[q2]};
          double wq = D.gw[q0] * D.gw[q1] * D.gw[q2] * D.vol(e) / 8.0;
          D.eval(e, xi, ph.data(), nullptr);
          for (int v = 0; v < 4; ++v)
            for (int j = 0; j < nb; ++j)
              w[((size_t)e * 4 + v) * nb + j] += wq * vals[((size_t)e * 4 + v) * npt + i] * ph[j];
        }
  }
}

// L2 projection of the Taylor-Green field with the Gauss rule.
void orc_project_tgv(const orc_mesh* m, double* w) {
  Disc D(m);
  int nq = D.nq, nb = D.nb;
  std::vector<double> ph(nb);
  for (size_t i = 0; i < (size_t)D.ne * 4 * nb; ++i) w[i] = 0.0;
  for (int e = 0; e < D.ne; ++e)
    for (int q0 = 0; q0 < nq; ++q0)
      for (int q1 = 0; q1 < nq; ++q1)
        for (int q2 = 0; q2 < nq; ++q2) {
          double xi[3] = {D.gx[q0], D.gx[q1], D.gx[q2]};
          double x[3], val4[4];
          for (int d = 0; d < 3; ++d) x[d] = D.center(e, d) + 0.5 * D.h(e, d) * xi[d];
          double wq = D.gw[q0] * D.gw[q1] * D.gw[q2] * D.vol(e) / 8.0;
          D.eval(e, xi, ph.data(), nullptr);
          tgv(x, val4);
          for (int v = 0; v < 4; ++v)
            for (int j = 0; j < nb; ++j) w[((size_t)e * 4 + v) * nb + j] += wq * val4[v] * ph[j];
        }
}

// Evaluate the DG polynomial w at reference points xi of element e: out[npts][4].
void orc_eval_field(const orc_mesh* m, const double* w, int e, int npts, const double* xi, double* out) {
  Disc D(m);
  std::vector<double> ph(D.nb);
  for (int i = 0; i < npts; ++i) {
    D.eval(e, xi + 3 * i, ph.data(), nullptr);
    for (int v = 0; v < 4; ++v) {
      double s = 0.0;
      for (int j = 0; j < D.nb; ++j) s += w[((size_t)e * 4 + v) * D.nb + j] * ph[j];
      out[4 * i + v] = s;
    }
  }
}

// f = f_h(w; phi_m e_i), Eq. (NSdiscrRes).
void orc_residual(const orc_mesh* m, const double* w, double* f) {
  Disc D(m);
  residual<double>(D, w, f);
}

// out = G v = J(w) v + (1/(gamma dt)) M v, with J the exact derivative of the
// residual (Eqs. (jacTrilFnotNU), (jacTrilnu)) and M the velocity-only mass form
// (Eq. (massBil); identity on the velocity modes of an orthonormal basis).
void orc_jvp(const orc_mesh* m, const double* w, const double* v, double inv_gdt, double* out) {
  Disc D(m);
  size_t n = (size_t)D.ne * 4 * D.nb;
  std::vector<Dual> wd(n), fd(n);
  for (size_t i = 0; i < n; ++i) wd[i] = Dual(w[i], v[i]);
  residual<Dual>(D, wd.data(), fd.data());
  for (size_t i = 0; i < n; ++i) {
    int var = (int)((i / D.nb) % 4);
    out[i] = fd[i].d + (var < 3 ? inv_gdt * v[i] : 0.0);
  }
}

// Matrix-free finite-difference action of Eqs. (matrix-free), (epsdef):
// J v ~ (f(w + Delta v) - f(w)) / Delta, Delta = eps sqrt(1 + ||w||) / ||v||,
// plus the mass term. ||.||_{L2(Omega)} is the Euclidean norm of orthonormal
// coefficients.
void orc_jvp_fd(const orc_mesh* m, const double* w, const double* v, double inv_gdt, double eps, double* out) {
  Disc D(m);
  size_t n = (size_t)D.ne * 4 * D.nb;
  double nw = 0.0, nv = 0.0;
  for (size_t i = 0; i < n; ++i) { nw += w[i] * w[i]; nv += v[i] * v[i]; }
  nw = std::sqrt(nw);
  nv = std::sqrt(nv);
  if (nv == 0.0) { for (size_t i = 0; i < n; ++i) out[i] = 0.0; return; }
  double delta = eps * std::sqrt(1.0 + nw) / nv;
  std::vector<double> f0(n), f1(n), wp(n);
  residual<double>(D, w, f0.data());
  for (size_t i = 0; i < n; ++i) wp[i] = w[i] + delta * v[i];
  residual<double>(D, wp.data(), f1.data());
  for (size_t i = 0; i < n; ++i) {
    int var = (int)((i / D.nb) % 4);
    out[i] = (f1[i] - f0[i]) / delta + (var < 3 ? inv_gdt * v[i] : 0.0);
  }
}

// Dense G (row-major, G[row * n + col]) by columns of the exact Jacobian action
// (the columns in parallel; each residual inside runs on its one thread).
void orc_dense_G(const orc_mesh* m, const double* w, double inv_gdt, double* G) {
  Disc D(m);
  long n = (long)D.ne * 4 * D.nb;
  omp_set_max_active_levels(1);
#pragma omp parallel for schedule(dynamic)
  for (long col = 0; col < n; ++col) {
    std::vector<Dual> wd(n), fd(n);
    for (long i = 0; i < n; ++i) wd[i] = Dual(w[i], i == col ? 1.0 : 0.0);
    residual<Dual>(D, wd.data(), fd.data());
    for (long i = 0; i < n; ++i) {
      int var = (int)((i / D.nb) % 4);
      G[i * n + col] = fd[i].d + (i == col && var < 3 ? inv_gdt : 0.0);
    }
  }
}

// Inviscid interface flux for a single state pair along axis d (for unit tests):
// flux[4], star[3] = (u*, p*, 0), uface[3].
void orc_riemann(const double* uL, double pL, const double* uR, double pR, int d, double c, double* flux,
                 double* star, double* uface) {
  double us, ps;
  riemann_flux<double>(uL, pL, uR, pR, d, c, flux, &us, &ps, uface);
  star[0] = us;
  star[1] = ps;
  star[2] = 0.0;
}

// Exact derivative of orc_riemann's flux along the direction (duL, dpL, duR, dpR).
void orc_riemann_tangent(const double* uL, double pL, const double* uR, double pR, const double* duL,
                         double dpL, const double* duR, double dpR, int d, double c, double* dflux) {
  Dual l[3], r[3], fl[4];
  for (int i = 0; i < 3; ++i) { l[i] = Dual(uL[i], duL[i]); r[i] = Dual(uR[i], duR[i]); }
  riemann_flux<Dual>(l, Dual(pL, dpL), r, Dual(pR, dpR), d, c, fl, nullptr, nullptr, nullptr);
  for (int i = 0; i < 4; ++i) dflux[i] = fl[i].d;
}

// Pressure on the 1- and 3-wave curves (for the wave-curve ODE pin).
double orc_p_wave1(double u, double uL, double pL, double c) { return p_wave1<double>(u, uL, pL, c); }
double orc_p_wave3(double u, double uR, double pR, double c) { return p_wave3<double>(u, uR, pR, c); }
double orc_tang1(double u, double uL, double c) { return tang1<double>(u, uL, c); }
double orc_tang3(double u, double uR, double c) { return tang3<double>(u, uR, c); }

}  // extern "C"
