// Matrix-free DG operator on sm_103a: residual f_h (Eq. (NSdiscrRes)), its
// exact linearisation (Eqs. (jacTrilFnotNU), (jacTrilnu)) and the
// finite-difference action (Eqs. (matrix-free), (epsdef)).
//
// GB300 has a narrow FP64 pipe (2 DFMA/clk/SM), so the kernels spend FP64
// operations only where the method needs quadrature and do everything that is
// polynomial exactly in modal space:
//  * face_kernel (one warp per face s = (K, K')): traces of both sides as 2D
//    modal coefficients on the face (collapse over the normal exponent, exact),
//    point values only of the four fields the nonlinear artificial-compressibility
//    Riemann flux needs, the flux (exact star state by safeguarded Newton; in
//    tangent mode its cached Jacobian) projected back onto the 2D modes, the BR2
//    lifting r^s([u]) = a diagonal scaling of the 2D jump coefficients, and the
//    BR2 viscous face flux F^nu({grad u - eta r^s}) built exactly in 2D modal
//    space. Writes per element face slot the 2D-modal face contribution and the
//    scaled jump from which the volume pass expands the lifting.
//  * vol_kernel (one CTA per element): corrected-gradient coefficients
//    grad u - R^K(u) (sparse exact modal derivative minus the six liftings), the
//    viscous and pressure terms and the continuity equation as exact modal
//    derivatives (F^nu is linear, p and u are polynomials of degree k), the
//    convective term u (x) u by sum-factorised interpolation to and projection
//    from the Gauss points, plus the six face contributions and the mass shift.
// All of this equals the quadrature form of the paper's weak form up to
// rounding, because the Gauss rule with k+1 points integrates every
// polynomial product that is done exactly here.
//
// Conventions (also in the C ABI header): orthonormal modal basis
// phi_m = phi_hat_m(xi)/s, s = sqrt(|K|/8); the normal of a face points from K
// (lower index) to K'; [v] = v_K - v_K'; the lifting is defined by
// int r . tau = + int_s [v] {tau} . n so that grad u - R^K is the consistent
// gradient (Sec. 2.1).
#include <algorithm>
#include <mutex>
#include <vector>

#include "dg_internal.h"

namespace dg {

template <int K>
struct Sz {
  static constexpr int NB = nb_of(K), N1 = K + 1, NQ = N1 * N1 * N1, NQF = N1 * N1;
};

// MODE_LINPART: the state-independent linear part of the Jacobian action (viscous and BR2
// terms, pressure gradient, continuity); no convective product, no Riemann flux, no mass.
enum { MODE_RES = 0, MODE_RES_LIN = 1, MODE_TAN = 2, MODE_LINPART = 3 };

template <int K>
struct Sz2 {
  static constexpr int NB = nb_of(K), N1 = K + 1, NQ = N1 * N1 * N1, NQF = N1 * N1, N2 = (K + 1) * (K + 2) / 2;
};

// Real-valued tables in the kernel's precision (the integer tables stay in Tables).
template <class R>
struct RTab {
  const R* L1;
  const R* wvol;
  const R* B2;
  const R* W2;
  const R* pv;
  const R* pd;
  const R* Drow_val;
  const R* Dcol_val;
  const R* D2_val;
};

template <class R>
struct OpArgsT {
  MeshDev M;
  Tables T;
  RTab<R> rt;
  const R* in;
  R* out;
  R* face_out;
  R* face_lift;
  R* ubar;
  R* dFlux;
  double nu, c, eta, inv_gdt;
  unsigned* status;
  int riemann_its;  // iteration cap of the star-state solve
};
using OpArgs = OpArgsT<double>;

// ------------------------------------------------------------------ Riemann
// The rarefaction branches below read a = sqrt(u^2+c^2) and A = asinh(u/c) at the star
// velocity u and aL, AL (aR, AR) at the side's normal velocity. The caller computes each
// once: the side values once per point, the star values once per Newton iterate, and only
// when a rarefaction branch is taken.
//
// Pressure on the 1-wave curve through (uL, pL) at star velocity u, and its
// partial derivatives in u and uL (dp/dpL = 1). Shock (u < uL): Rankine-Hugoniot
// with the negative root s of s^2 - (uL+u)s - c^2 = 0, p = pL + c^2 (u-uL)/s.
// Rarefaction: dp/du = -(u + sqrt(u^2+c^2)) integrated in closed form.
__device__ __forceinline__ void wave1(double u, double a, double A, double uL, double aL, double AL, double pL,
                                      double c, double& p, double& dpdu, double& dpduL) {
  const double c2 = c * c;
  if (u < uL) {
    const double sig = uL + u, Q = sqrt(sig * sig + 4.0 * c2), s = 0.5 * (sig - Q);
    const double ss = -s / Q;  // ds/dsig
    const double du = u - uL, is = 1.0 / s;
    p = pL + c2 * du * is;
    dpdu = c2 * (is - du * ss * is * is);
    dpduL = c2 * (-is - du * ss * is * is);
  } else {
    const double Gu = 0.5 * (u * u + u * a + c2 * A);
    const double GL = 0.5 * (uL * uL + uL * aL + c2 * AL);
    p = pL - (Gu - GL);
    dpdu = -(u + a);
    dpduL = uL + aL;
  }
}
// Pressure on the 3-wave curve through (uR, pR): shock for u > uR (positive root),
// rarefaction dp/du = sqrt(u^2+c^2) - u otherwise. Partials in u and uR (dp/dpR = 1).
__device__ __forceinline__ void wave3(double u, double a, double A, double uR, double aR, double AR, double pR,
                                      double c, double& p, double& dpdu, double& dpduR) {
  const double c2 = c * c;
  if (u > uR) {
    const double sig = u + uR, Q = sqrt(sig * sig + 4.0 * c2), s = 0.5 * (sig + Q);
    const double ss = s / Q;
    const double du = u - uR, is = 1.0 / s;
    p = pR + c2 * du * is;
    dpdu = c2 * (is - du * ss * is * is);
    dpduR = c2 * (-is - du * ss * is * is);
  } else {
    const double Hu = 0.5 * (u * a + c2 * A - u * u);
    const double HR = 0.5 * (uR * aR + c2 * AR - uR * uR);
    p = pR - (HR - Hu);
    dpdu = a - u;
    dpduR = -(aR - uR);
  }
}
// Tangential-velocity ratio across the 1-wave, tau = u_t(star)/u_t(L), with partials
// in u* and uL. Rarefaction: u_t (u + a) invariant; shock: s [u_t] = [u_n u_t].
__device__ __forceinline__ void tang1(double u, double a, double uL, double aL, double c, double& t, double& dtdu,
                                      double& dtduL) {
  const double c2 = c * c;
  if (u < uL) {
    const double sig = uL + u, Q = sqrt(sig * sig + 4.0 * c2), s = 0.5 * (sig - Q), ss = -s / Q;
    const double den = s - u, num = s - uL, id = 1.0 / den;
    t = num * id;
    dtdu = (ss * den - num * (ss - 1.0)) * id * id;
    dtduL = ((ss - 1.0) * den - num * ss) * id * id;
  } else {
    t = (uL + aL) / (u + a);
    dtdu = -t / a;
    dtduL = t / aL;
  }
}
// Ratio across the 3-wave, tau = u_t(star)/u_t(R). Rarefaction: u_t/(u + a) invariant.
__device__ __forceinline__ void tang3(double u, double a, double uR, double aR, double c, double& t, double& dtdu,
                                      double& dtduR) {
  const double c2 = c * c;
  if (u > uR) {
    const double sig = u + uR, Q = sqrt(sig * sig + 4.0 * c2), s = 0.5 * (sig + Q), ss = s / Q;
    const double den = s - u, num = s - uR, id = 1.0 / den;
    t = num * id;
    dtdu = (ss * den - num * (ss - 1.0)) * id * id;
    dtduR = ((ss - 1.0) * den - num * ss) * id * id;
  } else {
    t = (u + a) / (uR + aR);
    dtdu = t / a;
    dtduR = -t / aR;
  }
}

// Exact interface flux of the artificial-compressibility Riemann problem along the face
// normal, in the face's frame (n, t1, t2): inputs the normal and the two tangential velocity
// components and the pressure of each side, outputs F = (n.(u(x)u + pI) along n, t1, t2; u_n*)
// at the interface state, which is the star state, since the two acoustic waves always travel
// in opposite directions. The tangential velocity is taken from the side the contact (speed
// u*) comes from, the two sides averaged when |u*| is within a rounding band of zero. With
// J != nullptr also the Jacobian J[r][c] of F with respect to (un, t1, t2, p) of the left side
// (c = 0..3) and of the right side (c = 4..7). Every index is fixed at compile time, so after
// inlining F and J stay in registers.
__device__ __forceinline__ void ac_riemann(double ul, double t1l, double t2l, double pL, double ur, double t1r,
                                           double t2r, double pR, double c, double (&F)[4], double (*J)[8],
                                           unsigned* status, int max_its) {
  const double c2 = c * c;
  const double al = sqrt(ul * ul + c2), ar = sqrt(ur * ur + c2);
  const double Al = asinh(ul / c), Ar = asinh(ur / c);
  const double scale = fabs(ul) + fabs(ur) + c;
  // sqrt(u^2+c^2) and asinh(u/c) at a star velocity, where a rarefaction branch reads them
  auto at_star = [&](double u, double& as, double& As) {
    if (!(u < ul) || !(u > ur)) {
      as = sqrt(u * u + c2);
      As = asinh(u / c);
    } else {
      as = 0.0;
      As = 0.0;
    }
  };
  // two-rarefaction linearisation as the initial guess
  double us = (pL - pR + ul * (ul + al) + ur * (ar - ur)) / ((ul + al) + (ar - ur));
  double lo = -1e300, hi = 1e300;
  bool ok = false;
  double p1, d1u, d1l, p3, d3u, d3r, as, As;
  for (int it = 0; it < max_its; ++it) {
    at_star(us, as, As);
    wave1(us, as, As, ul, al, Al, pL, c, p1, d1u, d1l);
    wave3(us, as, As, ur, ar, Ar, pR, c, p3, d3u, d3r);
    const double phi = p1 - p3, dphi = d1u - d3u;  // dphi < 0
    if (phi > 0.0) lo = us; else hi = us;
    double nxt = us - phi / dphi;
    const bool newton = nxt > lo && nxt < hi;
    if (!newton) nxt = (lo > -1e299 && hi < 1e299) ? 0.5 * (lo + hi) : nxt;
    const double step = nxt - us;
    us = nxt;
    // After a Newton step of size |step| the error is about K step^2, with K = |phi''| / (2 |phi'|)
    // at the root. The wave curves are C^2 in u. With two rarefactions K = |u*| / (2 (u*^2 + c^2))
    // <= 1 / (4 c); over shocks as well it stays below 0.5 / c (about 0.33 / c at most over seeded
    // states with |u_L|, |u_R| up to 300 c, evaluated in extended precision). A Newton step below
    // 1e-9 c therefore leaves an error below 1e-18 c, and the confirming iteration is skipped.
    if (fabs(step) <= 1e-15 * scale || (newton && fabs(step) <= 1e-9 * c)) { ok = true; break; }
  }
  if (!ok && status) atomicOr(status, (unsigned)DG_STATUS_RIEMANN);
  at_star(us, as, As);
  wave1(us, as, As, ul, al, Al, pL, c, p1, d1u, d1l);
  wave3(us, as, As, ur, ar, Ar, pR, c, p3, d3u, d3r);
  const double ps = p1;
  // tangential ratios
  double tl, tlu, tll, tr, tru, trr;
  tang1(us, as, ul, al, c, tl, tlu, tll);
  tang3(us, as, ur, ar, c, tr, tru, trr);
  const double band = 1e-12 * scale;
  double wl, wr;  // weights of the left / right star tangential values
  if (us > band) { wl = 1.0; wr = 0.0; }
  else if (us < -band) { wl = 0.0; wr = 1.0; }
  else { wl = 0.5; wr = 0.5; }
  const double tL[2] = {t1l, t2l}, tR[2] = {t1r, t2r};
  F[0] = us * us + ps;
  F[3] = us;
#pragma unroll
  for (int t = 0; t < 2; ++t) F[1 + t] = (wl * tL[t] * tl + wr * tR[t] * tr) * us;
  if (J) {
    // implicit-function derivatives of u* and p* with respect to (ul, pL, ur, pR)
    const double iphi = 1.0 / (d1u - d3u);
    const double dus_ul = -d1l * iphi, dus_pl = -iphi, dus_ur = d3r * iphi, dus_pr = iphi;
    const double dps_ul = d1u * dus_ul + d1l, dps_pl = d1u * dus_pl + 1.0;
    const double dps_ur = d1u * dus_ur, dps_pr = d1u * dus_pr;
    const double du[8] = {dus_ul, 0.0, 0.0, dus_pl, dus_ur, 0.0, 0.0, dus_pr};
    const double dp[8] = {dps_ul, 0.0, 0.0, dps_pl, dps_ur, 0.0, 0.0, dps_pr};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      J[3][j] = du[j];
      J[0][j] = 2.0 * us * du[j] + dp[j];
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const double ut = wl * tL[t] * tl + wr * tR[t] * tr;
      // d(ut) = wl (tl dtL + tL (tlu du* + tll dul)) + wr (tr dtR + tR (tru du* + trr dur))
      double dut[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) dut[j] = (wl * tL[t] * tlu + wr * tR[t] * tru) * du[j];
      dut[0] += wl * tL[t] * tll;
      dut[4] += wr * tR[t] * trr;
      dut[1 + t] += wl * tl;
      dut[5 + t] += wr * tr;
#pragma unroll
      for (int j = 0; j < 8; ++j) J[1 + t][j] = us * dut[j] + ut * du[j];
    }
  }
}

// ---------------------------------------------------------------- face pass
// eight consecutive values from 16-byte aligned shared memory (two 16-byte loads for float,
// four for double), and the same from global memory (the cached Riemann Jacobian)
__device__ __forceinline__ void load8(const float* p, float* o) {
  const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void load8(const double* p, double* o) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 v = reinterpret_cast<const double2*>(p)[i];
    o[2 * i] = v.x;
    o[2 * i + 1] = v.y;
  }
}
__device__ __forceinline__ void load8g(const float* p, float* o) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void load8g(const double* p, double* o) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
    o[2 * i] = v.x;
    o[2 * i + 1] = v.y;
  }
}

__device__ __forceinline__ void store8(float* p, const float* v) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void store8(double* p, const double* v) {
#pragma unroll
  for (int i = 0; i < 4; ++i) reinterpret_cast<double2*>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

constexpr int kFaceWarps = 4;  // default faces per CTA, one warp each (the tangent pass's is tunable)

template <int K, class R = double, int FW = kFaceWarps>
struct FaceSmem {
  using S = Sz2<K>;
  // per warp
  static constexpr int C = 0;                           // [2][4][NB] coefficients of K and K'; later the
                                                        // partial sums of the two sum-factorised steps
  static constexpr int T = C + 8 * S::NB;               // [N2][2][4] value traces (a 2D mode's 8 together)
  static constexpr int N = T + 8 * S::N2;               // [2][3][N2] normal-derivative traces of velocity
  static constexpr int F = N + 6 * S::N2;               // [4][NQF] weighted Riemann flux
  static constexpr int P = F + 4 * S::NQF;              // [4][N2] its projection
  static constexpr int WARP = (P + 4 * S::N2 + 3) / 4 * 4;  // 16-byte multiple (vector loads of T)
  // per CTA tables (after the warps)
  static constexpr int B2 = FW * WARP;                  // [NQF][N2] (the FP32 pass's dense 2D tables)
  static constexpr int W2 = B2 + (sizeof(R) == 4 ? S::NQF * S::N2 : 0);  // [NQF]
  static constexpr int PV = W2 + S::NQF;                // [2][K+1]
  static constexpr int PD = PV + 2 * (K + 1);           // [2][K+1]
  static constexpr int D2V = PD + 2 * (K + 1);          // [2][N2][kDw]
  static constexpr int L1 = D2V + 2 * S::N2 * Tables::kDw;  // [K+1][N1] P_hat_a at the 1D Gauss points
  static constexpr int DOUBLES = L1 + (K + 1) * S::N1;
  static_assert(8 * (K + 1) * S::N1 <= 8 * S::NB && 4 * (K + 1) * S::N1 <= 8 * S::NB, "partial sums fit in C");
  // ints after the doubles
  static constexpr int M3 = 0;                          // [3][N2][K+1]
  static constexpr int D2I = M3 + 3 * S::N2 * (K + 1);  // [2][N2][kDw]
  static constexpr int DEG = D2I + 2 * S::N2 * Tables::kDw;  // [N2] total degree of each 2D mode
  static constexpr int INTS = DEG + S::N2;
  static constexpr size_t bytes() { return sizeof(R) * DOUBLES + sizeof(int) * INTS; }
};

template <int K, int MODE, class R, int FW = kFaceWarps>
__global__ void __launch_bounds__(32 * FW) face_kernel(OpArgsT<R> a) {
  using S = Sz2<K>;
  using L = FaceSmem<K, R, FW>;
  constexpr int NB = S::NB, NQF = S::NQF, N2 = S::N2, K1 = K + 1, DW = Tables::kDw;
  extern __shared__ __align__(16) unsigned char smraw_[];
  R* sm = reinterpret_cast<R*>(smraw_);
  R* W2 = sm + L::W2;
  R* PV = sm + L::PV;
  R* PD = sm + L::PD;
  R* D2V = sm + L::D2V;
  R* sL1 = sm + L::L1;
  R* B2 = sm + L::B2;
  // the FP64 pass (bound by GB300's FP64 pipe) takes the face points by sum factorisation, 40 %
  // fewer multiply-adds; the FP32 pass, bound by issue and latency, keeps the dense 2D tables
  constexpr bool kSumFact = sizeof(R) == 8;
  int* ism = reinterpret_cast<int*>(sm + L::DOUBLES);
  int* M3 = ism + L::M3;
  int* D2I = ism + L::D2I;
  int* DEG = ism + L::DEG;
  const int tid = threadIdx.x;
  for (int t = tid; t < N2; t += blockDim.x) DEG[t] = a.T.pab[2 * t] + a.T.pab[2 * t + 1];
  for (int t = tid; t < NQF; t += blockDim.x) W2[t] = a.rt.W2[t];
  for (int t = tid; t < 2 * K1; t += blockDim.x) { PV[t] = a.rt.pv[t]; PD[t] = a.rt.pd[t]; }
  for (int t = tid; t < 2 * N2 * DW; t += blockDim.x) { D2V[t] = a.rt.D2_val[t]; D2I[t] = a.T.D2_idx[t]; }
  for (int t = tid; t < 3 * N2 * K1; t += blockDim.x) M3[t] = a.T.M3[t];
  for (int t = tid; t < K1 * K1; t += blockDim.x) sL1[t] = a.rt.L1[t];
  if constexpr (!kSumFact)
    for (int t = tid; t < NQF * N2; t += blockDim.x) B2[t] = a.rt.B2[t];
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const R nu = R(a.nu), eta = R(a.eta);
  R* W = sm + warp * L::WARP;
  R* sC = W + L::C;
  R* sT = W + L::T;
  R* sN = W + L::N;
  R* sF = W + L::F;
  R* sP = W + L::P;
  const int nint = 3 * a.M.ne, nfaces = nint + a.M.nbf;
  for (int f = blockIdx.x * FW + warp; f < nfaces; f += gridDim.x * FW) {
    // face f: element e0 on its - side, e1 on its + side, normal along d. A wall face has one
    // real element; its other side is the ghost state (2f - u_K, p_K) with f = 0 (wall 1: the
    // ghost on the + side, wall 2: on the - side); both sides then read the real element here.
    int e0, d, e1, wall = 0;
    if (f < nint) {
      e0 = f / 3;
      d = f - 3 * e0;
      e1 = a.M.nbr[e0 * 6 + 2 * d + 1];
      if (e1 < 0) { e1 = e0; wall = 1; }
    } else {
      e1 = a.M.bface[f - nint];
      e0 = e1;
      d = 1;
      wall = 2;
    }
    const R* g0 = geo_row<R>(a.M, e0);
    const R* g1 = geo_row<R>(a.M, e1);
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    // the geometry along the face's axes, read with selects (no run-time indexing), in the
    // kernel's precision: the FP32 pass does no FP64 arithmetic or conversion (GB300's FP64 pipe
    // is 1/64 of the FP32 rate); the FP64 pass reads the same values as before
    auto sel3 = [](const R* v, int i) { return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]); };
    const R J0d = sel3(g0 + 5, d), J1d = sel3(g1 + 5, d);
    const R J0t1 = sel3(g0 + 5, t1), J0t2 = sel3(g0 + 5, t2);
    const R A4 = R(0.25) * sel3(g0, t1) * sel3(g0, t2);
    const R is0 = g0[4], is1 = g1[4];
    for (int t = lane; t < 8 * NB; t += 32) {
      const int side = t / (4 * NB), r = t - side * 4 * NB;
      sC[t] = a.in[(size_t)(side ? e1 : e0) * 4 * NB + r];
    }
    __syncwarp();
    // 2D trace coefficients, one lane per (side, 2D mode j): the values of u, v, w, p and the
    // normal derivatives of u, v, w (2 N2 <= 30 lanes for k <= 4)
    if (lane < 2 * N2) {
      const int side = lane >= N2 ? 1 : 0, j = lane - side * N2;
      const int* mm = M3 + (d * N2 + j) * K1;
      const R* cs = sC + side * 4 * NB;
      const R* pw = PV + side * K1;
      const R* pdw = PD + side * K1;
      R val[4] = {R(0), R(0), R(0), R(0)}, der[3] = {R(0), R(0), R(0)};
#pragma unroll
      for (int e = 0; e < K1; ++e) {
        const int m = mm[e];
        if (m >= 0) {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const R c = cs[v * NB + m];
            val[v] += pw[e] * c;
            if (v < 3) der[v] += pdw[e] * c;
          }
        }
      }
      const R is = side ? is1 : is0;
      const R js = is * (side ? J1d : J0d);
      R* tt = sT + j * 8 + side * 4;
#pragma unroll
      for (int v = 0; v < 4; ++v) tt[v] = val[v] * is;
#pragma unroll
      for (int c = 0; c < 3; ++c) sN[side * 3 * N2 + c * N2 + j] = der[c] * js;
    }
    __syncwarp();
    if (wall && lane < N2) {  // ghost traces: velocity 2f - u_K = -u_K, the real pressure and normal derivatives
      const int rs = wall == 1 ? 0 : 1, gs = 1 - rs, j = lane;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const R x = sT[j * 8 + rs * 4 + v];
        sT[j * 8 + gs * 4 + v] = v < 3 ? -x : x;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) sN[gs * 3 * N2 + c * N2 + j] = sN[rs * 3 * N2 + c * N2 + j];
    }
    __syncwarp();
    // point values by sum factorisation over the face's two axes (the 2D basis at point
    // q = (q1, q2) is P_hat_a(x_q1) P_hat_b(x_q2)): first U[a][q2] = sum_b P_hat_b(x_q2) T[(a, b)], one lane per
    // (a, q2), for the 8 traces of a mode together; the coefficients in C are dead by now
    R* sU = W + L::C;  // [K+1][N1][8]
    if (kSumFact && lane < NQF) {
      const int a0 = lane / K1, q2 = lane - a0 * K1;
      R u[8];
#pragma unroll
      for (int s8 = 0; s8 < 8; ++s8) u[s8] = R(0);
#pragma unroll
      for (int b = 0; b <= K; ++b) {
        if (a0 + b <= K) {
          const int j = (a0 + b) * (a0 + b + 1) / 2 + b;  // graded 2D order: degree, then b
          const R l = sL1[b * K1 + q2];
          R tt[8];
          load8(sT + j * 8, tt);
#pragma unroll
          for (int s8 = 0; s8 < 8; ++s8) u[s8] += l * tt[s8];
        }
      }
      store8(sU + lane * 8, u);
    }
    if constexpr (kSumFact) __syncwarp();
    // one lane per face point q = (q1, q2): the point values of both sides (kept in registers),
    // sum_a P_hat_a(x_q1) U[a][q2], and the Riemann flux, or its linearisation, at that point
    if (lane < NQF) {
      const int q = lane, q1 = q / K1, q2 = q - q1 * K1;
      R pvq[8];
#pragma unroll
      for (int s8 = 0; s8 < 8; ++s8) pvq[s8] = R(0);
      if constexpr (kSumFact) {
#pragma unroll
        for (int a0 = 0; a0 <= K; ++a0) {
          const R l = sL1[a0 * K1 + q1];
          R tt[8];
          load8(sU + (a0 * K1 + q2) * 8, tt);
#pragma unroll
          for (int s8 = 0; s8 < 8; ++s8) pvq[s8] += l * tt[s8];
        }
      } else {
        const R* b = B2 + q * N2;  // dense: sum over the 2D modes
#pragma unroll
        for (int j = 0; j < N2; ++j) {
          const R bj = b[j];
          R tt[8];
          load8(sT + j * 8, tt);
#pragma unroll
          for (int s8 = 0; s8 < 8; ++s8) pvq[s8] += bj * tt[s8];
        }
      }
      R uL[3] = {pvq[0], pvq[1], pvq[2]};
      R uR[3] = {pvq[4], pvq[5], pvq[6]};
      const R pL = pvq[3], pR = pvq[7];
      R Fc[4] = {R(0), R(0), R(0), R(0)};
      if constexpr (MODE == MODE_TAN) {
        const R* Jq = a.dFlux + ((size_t)f * NQF + q) * 32;
        R Jr[32];
#pragma unroll
        for (int i = 0; i < 32; i += 8) load8g(Jq + i, Jr + i);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          R acc = R(0);
#pragma unroll
          for (int j = 0; j < 8; ++j) acc += Jr[i * 8 + j] * pvq[j];
          Fc[i] = acc;
        }
      } else if constexpr (MODE == MODE_RES_LIN || MODE == MODE_RES) {
        // residual modes run in FP64 only. The solve works in the face's frame (n, t1, t2):
        // components d, t1, t2 of the velocities in, the flux and its Jacobian back to x, y, z
        auto comp = [&](const R* u, int i) { return i == 0 ? u[0] : (i == 1 ? u[1] : u[2]); };
        double Fr[4], Jr[4][8];
        ac_riemann(comp(uL, d), comp(uL, t1), comp(uL, t2), pL, comp(uR, d), comp(uR, t1), comp(uR, t2), pR, a.c,
                   Fr, MODE == MODE_RES_LIN ? Jr : nullptr, a.status, a.riemann_its);
        // original component i of a frame row / column r: d, t1, t2, then the pressure (3)
        auto orig = [&](int r) { return r == 0 ? d : (r == 1 ? t1 : (r == 2 ? t2 : 3)); };
#pragma unroll
        for (int i = 0; i < 3; ++i) Fc[i] = i == d ? Fr[0] : (i == t1 ? Fr[1] : Fr[2]);
        Fc[3] = Fr[3];
        if constexpr (MODE == MODE_RES_LIN) {
          R* Jq = a.dFlux + ((size_t)f * NQF + q) * 32;
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) Jq[orig(r) * 8 + (cc >> 2) * 4 + orig(cc & 3)] = Jr[r][cc];
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) sF[i * NQF + q] = Fc[i] * W2[q];
    }
    __syncwarp();
    // projection onto the 2D modes, sum factorised the other way round: S[i][a][q2] =
    // sum_q1 P_hat_a(x_q1) F_i(q1, q2), then P[i][(a, b)] = sum_q2 P_hat_b(x_q2) S[i][a][q2]
    R* sS = W + L::C;  // [4][K+1][N1]; the point-value partial sums are dead by now
    for (int t = lane; kSumFact && t < 4 * NQF; t += 32) {
      const int i = t / NQF, r = t - i * NQF, a0 = r / K1, q2 = r - a0 * K1;
      const R* Fi = sF + i * NQF + q2;
      R acc = R(0);
#pragma unroll
      for (int q1 = 0; q1 < K1; ++q1) acc += sL1[a0 * K1 + q1] * Fi[q1 * K1];
      sS[t] = acc;
    }
    if constexpr (kSumFact) __syncwarp();
    for (int t = lane; t < 4 * N2; t += 32) {
      const int i = t / N2, j = t - i * N2;
      R acc = R(0);
      if constexpr (kSumFact) {
        const int deg = DEG[j], b = j - deg * (deg + 1) / 2, a0 = deg - b;
        const R* Si = sS + (i * K1 + a0) * K1;
#pragma unroll
        for (int q2 = 0; q2 < K1; ++q2) acc += sL1[b * K1 + q2] * Si[q2];
      } else {
        const R* Fi = sF + i * NQF;
#pragma unroll
        for (int q = 0; q < NQF; ++q) acc += B2[q * N2 + j] * Fi[q];
      }
      sP[t] = acc;
    }
    __syncwarp();
    // viscous face flux in 2D modal space, total flux, lifting: two lanes per 2D mode j (lane j
    // and lane j + 16). The first forms the tangential derivatives of the normal component and
    // writes the - side's (element e0's) slot, the second those of the tangential components
    // and writes the + side's; they swap their derivatives by one shuffle. Every lane of the
    // warp takes part in the shuffle; lanes past the last mode compute on mode 0 and store nothing.
    static_assert(N2 <= 16, "two lanes per 2D mode");
    {
      const int half = lane >> 4, j0 = lane & 15;
      const bool act = j0 < N2;
      const int j = act ? j0 : 0;
      // trace of variable v on side s at 2D mode jj
      auto tr = [&](int s2, int v, int jj) { return sT[jj * 8 + s2 * 4 + v]; };
      // {r^s} of the normal gradient component, 2D mode j of total degree bj:
      // (k - bj + 1)^2 / 4 * (1/h_K + 1/h_K') * [u]
      const int bj = DEG[j];
      // at a wall the lifting lives on the real element alone, with the full jump:
      // (k - bj + 1)^2 / 2 * (2/h_K) * [u]
      const R lr = wall ? R(0.5) * R((K - bj + 1) * (K - bj + 1)) * J0d
                        : R(0.125) * R((K - bj + 1) * (K - bj + 1)) * (J0d + J1d);
      R jump[3], Gd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        // [u] = u_K - u_K' inside; at a wall u_K - f (upper) or f - u_K (lower), half the
        // difference of the real and the mirrored ghost traces
        jump[c] = (wall ? R(0.5) : R(1)) * (tr(0, c, j) - tr(1, c, j));
        Gd[c] = R(0.5) * (sN[c * N2 + j] + sN[3 * N2 + c * N2 + j]) - eta * lr * jump[c];  // Ghat[c][d]
      }
      // tangential derivatives (2D modal) of the normal component and of the tangential ones
      auto tder = [&](int s2, int v, int dir) {
        R acc = R(0);
#pragma unroll
        for (int q = 0; q < DW; ++q) {
          const int o = (dir * N2 + j) * DW + q;
          acc += D2V[o] * tr(s2, v, D2I[o]);
        }
        return acc;
      };
      const R it1 = J0t1, it2 = J0t2;
      // tangential derivatives: the average of both sides, or the real side's at a wall; the
      // first lane of a mode: Ghat[d][t1], Ghat[d][t2]; the second: Ghat[t1][t1], Ghat[t2][t2]
      const int A0 = wall == 2 ? 1 : 0;
      const int A1 = wall == 1 ? 0 : 1;
      const int va = half ? t1 : d, vb = half ? t2 : d;
      const R x0 = R(0.5) * (tder(A0, va, 0) + tder(A1, va, 0)) * it1;
      const R x1 = R(0.5) * (tder(A0, vb, 1) + tder(A1, vb, 1)) * it2;
      const R y0 = __shfl_xor_sync(0xffffffffu, x0, 16), y1 = __shfl_xor_sync(0xffffffffu, x1, 16);
      const R Gdt1 = half ? y0 : x0, Gdt2 = half ? y1 : x1;  // Ghat[d][t1], Ghat[d][t2]
      const R Gt1 = half ? x0 : y0, Gt2 = half ? x1 : y1;    // Ghat[t1][t1], Ghat[t2][t2]
      // Ghat[c][d] of the components along d, t1, t2 (selects: no run-time array indexing)
      auto pick = [&](int c) { return c == 0 ? Gd[0] : (c == 1 ? Gd[1] : Gd[2]); };
      const R Gdd = pick(d), Gt1d = pick(t1), Gt2d = pick(t2);
      const R trG = Gdd + Gt1 + Gt2;
      const R Fvd = nu * (R(2) * Gdd - R(2.0 / 3.0) * trG);
      const R Fvt1 = nu * (Gt1d + Gdt1);
      const R Fvt2 = nu * (Gt2d + Gdt2);
      R Fn[4];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R Fv = i == d ? Fvd : (i == t1 ? Fvt1 : Fvt2);
        Fn[i] = A4 * (sP[i * N2 + j] - Fv);
      }
      Fn[3] = A4 * sP[3 * N2 + j];
      const R lw = wall ? R(1) : R(0.5);  // share of the lifting on each real side
      if (act && half == 0 && wall != 2) {
        R* o0 = a.face_out + ((size_t)e0 * 6 + 2 * d + 1) * 4 * N2;
        R* l0 = a.face_lift + ((size_t)e0 * 6 + 2 * d + 1) * 3 * N2;
#pragma unroll
        for (int i = 0; i < 4; ++i) o0[i * N2 + j] = Fn[i] * is0;
#pragma unroll
        for (int c = 0; c < 3; ++c) l0[c * N2 + j] = lw * A4 * is0 * jump[c];
      }
      if (act && half == 1 && wall != 1) {
        R* o1 = a.face_out + ((size_t)e1 * 6 + 2 * d) * 4 * N2;
        R* l1 = a.face_lift + ((size_t)e1 * 6 + 2 * d) * 3 * N2;
#pragma unroll
        for (int i = 0; i < 4; ++i) o1[i * N2 + j] = -Fn[i] * is1;
#pragma unroll
        for (int c = 0; c < 3; ++c) l1[c * N2 + j] = lw * A4 * is1 * jump[c];
      }
    }
    __syncwarp();
  }
}

// -------------------------------------------------------------- volume pass
template <int K, class R = double>
struct VolSmem {
  using S = Sz2<K>;
  static constexpr int NB = S::NB, N1 = S::N1, NQ = S::NQ, N2 = S::N2, K1 = K + 1;
  static constexpr int L1 = 0;                        // [K+1][N1]
  static constexpr int W3 = L1 + K1 * N1;             // [NQ]
  static constexpr int PV = W3 + NQ;                  // [2][K+1]
  static constexpr int C = PV + 2 * K1;               // [4][NB]
  static constexpr int G = C + 4 * NB;                // [9][NB] corrected gradient
  static constexpr int FV = G + 9 * NB;               // [6][NB] viscous flux (symmetric pairs)
  static constexpr int U = FV + 6 * NB;               // [3][NQ] velocity (or its variation) at the points
  static constexpr int T1 = U + 3 * NQ;               // [3][N2][N1] interpolation step 1
  static constexpr int T2 = T1 + 3 * N2 * N1;         // [3][K+1][N1*N1] interpolation step 2
  static constexpr int PR = T2 + 3 * K1 * N1 * N1;    // [6][NQ] weighted products
  static constexpr int S1 = PR + 6 * NQ;              // [6][K+1][N1*N1] projection step 1
  static constexpr int S2 = S1 + 6 * K1 * N1 * N1;    // [6][N2][N1] projection step 2
  static constexpr int CV = S2 + 6 * N2 * N1;         // [6][NB] projections of the products
  static constexpr int DOUBLES = CV + 6 * NB;
  static constexpr int MD3 = 0;                       // [NB][3]
  static constexpr int PIDX = MD3 + 3 * NB;           // [K+1][K+1]
  static constexpr int PAB = PIDX + K1 * K1;          // [N2][2]
  static constexpr int FMAP = PAB + 2 * N2;           // [3][NB]
  static constexpr int FA = FMAP + 3 * NB;            // [3][NB]
  static constexpr int IDX3 = FA + 3 * NB;            // [K+1]^3 3D mode of exponents (a, b, c) or -1
  static constexpr int INTS = IDX3 + K1 * K1 * K1;
  static constexpr size_t bytes() { return sizeof(R) * DOUBLES + sizeof(int) * INTS; }
};

__device__ __forceinline__ int sym_index(int p, int i) { return p == i ? p : (p + i + 2); }  // 01->3 02->4 12->5

template <int K, int MODE, class R>
__global__ void __launch_bounds__(256) vol_kernel(OpArgsT<R> a) {
  using L = VolSmem<K, R>;
  constexpr int NB = L::NB, N1 = L::N1, NQ = L::NQ, N2 = L::N2, K1 = L::K1, DW = Tables::kDw;
  extern __shared__ __align__(16) unsigned char smraw_[];
  R* sm = reinterpret_cast<R*>(smraw_);
  R* L1 = sm + L::L1;
  R* W3 = sm + L::W3;
  R* PV = sm + L::PV;
  R* sC = sm + L::C;
  R* sG = sm + L::G;
  R* sFv = sm + L::FV;
  R* sU = sm + L::U;
  R* sT1 = sm + L::T1;
  R* sT2 = sm + L::T2;
  R* sPr = sm + L::PR;
  R* sS1 = sm + L::S1;
  R* sS2 = sm + L::S2;
  R* sCv = sm + L::CV;
  int* ism = reinterpret_cast<int*>(sm + L::DOUBLES);
  int* MD3 = ism + L::MD3;
  int* PIDX = ism + L::PIDX;
  int* PAB = ism + L::PAB;
  int* FMAP = ism + L::FMAP;
  int* FA = ism + L::FA;
  int* IDX3 = ism + L::IDX3;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < K1 * K1 * K1; t += nt) IDX3[t] = -1;
  __syncthreads();
  for (int m = tid; m < NB; m += nt)
    IDX3[(a.T.md3[3 * m] * K1 + a.T.md3[3 * m + 1]) * K1 + a.T.md3[3 * m + 2]] = m;
  for (int t = tid; t < K1 * N1; t += nt) L1[t] = a.rt.L1[t];
  for (int t = tid; t < NQ; t += nt) W3[t] = a.rt.wvol[t];
  for (int t = tid; t < 2 * K1; t += nt) PV[t] = a.rt.pv[t];
  for (int t = tid; t < 3 * NB; t += nt) { MD3[t] = a.T.md3[t]; FMAP[t] = a.T.fmap[t]; FA[t] = a.T.fa[t]; }
  for (int t = tid; t < K1 * K1; t += nt) PIDX[t] = a.T.pidx[t];
  for (int t = tid; t < 2 * N2; t += nt) PAB[t] = a.T.pab[t];
  __syncthreads();
  // the 1D table P_hat_a(x_q) in registers for the whole kernel: every sum-factorisation step
  // below has a thread compute a pencil of K+1 outputs from values it loads once
  R Lr[K1][N1];
#pragma unroll
  for (int pa = 0; pa < K1; ++pa)
#pragma unroll
    for (int q = 0; q < N1; ++q) Lr[pa][q] = L1[pa * N1 + q];
  bool nonfinite = false;
  for (int e = blockIdx.x; e < a.M.ne; e += gridDim.x) {
    const ElemGeom g = elem_geom(a.M, e);
    const R is = R(g.is);
    const R shift = R(a.inv_gdt * g.sh);  // the mass shift's multiplier (tangent mode)
    const R Jd[3] = {R(g.J[0]), R(g.J[1]), R(g.J[2])};
    for (int t = tid; t < 4 * NB; t += nt) sC[t] = a.in[(size_t)e * 4 * NB + t];
    __syncthreads();
    // (A) corrected gradient coefficients; interpolation step 1 of the velocity
    const R* Lf = a.face_lift + (size_t)e * 6 * 3 * N2;
    if constexpr (sizeof(R) == 4) {  // FP32: one thread per (b, m) for the three components
      for (int t = tid; t < 3 * NB; t += nt) {
        const int b = t / NB, m = t - b * NB;
        int di[DW];
        R dv[DW];
#pragma unroll
        for (int j = 0; j < DW; ++j) {
          const int o = (b * NB + m) * DW + j;
          di[j] = a.T.Drow_idx[o];
          dv[j] = a.rt.Drow_val[o];
        }
        const int j2 = FMAP[b * NB + m], ex = FA[b * NB + m];
        const R p1 = PV[K1 + ex], p0 = PV[ex];
        const R jb = b == 0 ? Jd[0] : (b == 1 ? Jd[1] : Jd[2]);
#pragma unroll
        for (int av = 0; av < 3; ++av) {
          const R* cv = sC + av * NB;
          R acc = R(0);
#pragma unroll
          for (int j = 0; j < DW; ++j) acc += dv[j] * cv[di[j]];
          // R^K_b(u_av): liftings of the faces normal to b, K on side 1 (slot 2b) and side 0 (slot 2b+1)
          const R r = p1 * Lf[(2 * b) * 3 * N2 + av * N2 + j2] + p0 * Lf[(2 * b + 1) * 3 * N2 + av * N2 + j2];
          sG[(av * 3 + b) * NB + m] = acc * jb - r;
        }
      }
    } else {
      for (int t = tid; t < 9 * NB; t += nt) {
        const int ab = t / NB, m = t - ab * NB, av = ab / 3, b = ab - 3 * av;
        const R* cv = sC + av * NB;
        R acc = R(0);
  #pragma unroll
        for (int j = 0; j < DW; ++j) {
          const int o = (b * NB + m) * DW + j;
          acc += a.rt.Drow_val[o] * cv[a.T.Drow_idx[o]];
        }
        // R^K_b(u_av): liftings of the faces normal to b, K on side 1 (slot 2b) and side 0 (slot 2b+1)
        const int j2 = FMAP[b * NB + m], ex = FA[b * NB + m];
        const R r = PV[K1 + ex] * Lf[(2 * b) * 3 * N2 + av * N2 + j2] + PV[ex] * Lf[(2 * b + 1) * 3 * N2 + av * N2 + j2];
        sG[t] = acc * (b == 0 ? Jd[0] : (b == 1 ? Jd[1] : Jd[2])) - r;  // selects: no local memory
      }
    }
    if constexpr (sizeof(R) == 4) {  // FP32: pencils, fewer instructions per output
      for (int t = tid; t < 3 * N2; t += nt) {  // pencil (field, pair (a, b)): all q2
        const int fl = t / N2, pi = t - fl * N2;
        const int pa = PAB[2 * pi], pb = PAB[2 * pi + 1];
        const R* c = sC + fl * NB;
        const int* row = IDX3 + (pa * K1 + pb) * K1;
        R o[N1];
  #pragma unroll
        for (int q = 0; q < N1; ++q) o[q] = R(0);
  #pragma unroll
        for (int cc = 0; cc < K1; ++cc)
          if (cc <= K - pa - pb) {
            const R v = c[row[cc]];
  #pragma unroll
            for (int q = 0; q < N1; ++q) o[q] += v * Lr[cc][q];
          }
  #pragma unroll
        for (int q = 0; q < N1; ++q) sT1[(fl * N2 + pi) * N1 + q] = o[q];
      }
    } else {  // FP64 (pipe-bound): one output per item keeps more threads busy; the field is the
              // fastest index, so a warp's items share the pair (a, b) and the sum's length
      for (int t = tid; t < 3 * N2 * N1; t += nt) {
        const int fl = t % 3, r = t / 3, pi = r / N1, q2 = r - pi * N1;
        const int pa = PAB[2 * pi], pb = PAB[2 * pi + 1];
        const R* c = sC + fl * NB;
        R acc = R(0);
        const int* row = IDX3 + (pa * K1 + pb) * K1;
        for (int cc = 0; cc <= K - pa - pb; ++cc) acc += c[row[cc]] * L1[cc * N1 + q2];
        sT1[(fl * N2 + pi) * N1 + q2] = acc;
      }
    }
    __syncthreads();
    // (B) viscous flux coefficients; interpolation step 2
    // one thread per mode for the six symmetric pairs (p, i): nu (G_ip + G_pi - 2/3 delta_pi tr G)
    for (int m = tid; m < NB; m += nt) {
      const R nu = R(a.nu);
      const R g00 = sG[0 * NB + m], g11 = sG[4 * NB + m], g22 = sG[8 * NB + m];
      const R c23 = R(2.0 / 3.0) * (g00 + g11 + g22);
      sFv[0 * NB + m] = nu * (g00 + g00 - c23);
      sFv[1 * NB + m] = nu * (g11 + g11 - c23);
      sFv[2 * NB + m] = nu * (g22 + g22 - c23);
      sFv[3 * NB + m] = nu * (sG[(1 * 3 + 0) * NB + m] + sG[(0 * 3 + 1) * NB + m]);  // (p, i) = (0, 1)
      sFv[4 * NB + m] = nu * (sG[(2 * 3 + 0) * NB + m] + sG[(0 * 3 + 2) * NB + m]);  // (0, 2)
      sFv[5 * NB + m] = nu * (sG[(2 * 3 + 1) * NB + m] + sG[(1 * 3 + 2) * NB + m]);  // (1, 2)
    }
    if constexpr (sizeof(R) == 4) {  // FP32: pencils, fewer instructions per output
      for (int t = tid; t < 3 * K1 * N1; t += nt) {  // pencil (field, a, q2): all q1
        const int fl = t / (K1 * N1), r = t - fl * K1 * N1, pa = r / N1, q2 = r - pa * N1;
        R o[N1];
  #pragma unroll
        for (int q = 0; q < N1; ++q) o[q] = R(0);
  #pragma unroll
        for (int pb = 0; pb < K1; ++pb)
          if (pb <= K - pa) {
            const R v = sT1[(fl * N2 + PIDX[pa * K1 + pb]) * N1 + q2];
  #pragma unroll
            for (int q1 = 0; q1 < N1; ++q1) o[q1] += v * Lr[pb][q1];
          }
  #pragma unroll
        for (int q1 = 0; q1 < N1; ++q1) sT2[((fl * K1 + pa) * N1 + q1) * N1 + q2] = o[q1];
      }
    } else {  // FP64 (pipe-bound): one output per item keeps more threads busy; the field is the
              // fastest index, so a warp's items share a and the sum's length
      for (int t = tid; t < 3 * K1 * N1 * N1; t += nt) {
        const int fl = t % 3, r = t / 3, pa = r / (N1 * N1), r2 = r - pa * N1 * N1;
        const int q1 = r2 / N1, q2 = r2 - q1 * N1;
        R acc = R(0);
        for (int pb = 0; pb <= K - pa; ++pb) acc += sT1[fl * N2 * N1 + PIDX[pa * K1 + pb] * N1 + q2] * L1[pb * N1 + q1];
        sT2[fl * K1 * N1 * N1 + r] = acc;
      }
    }
    __syncthreads();
    // (C) interpolation step 3: velocity (or its variation) at the Gauss points
    if constexpr (sizeof(R) == 4) {  // FP32: pencils, fewer instructions per output
      for (int t = tid; t < 3 * N1 * N1; t += nt) {  // pencil (field, q1 q2): all q0
        const int fl = t / (N1 * N1), r = t - fl * N1 * N1;
        R o[N1];
  #pragma unroll
        for (int q = 0; q < N1; ++q) o[q] = R(0);
  #pragma unroll
        for (int pa = 0; pa < K1; ++pa) {
          const R v = sT2[(fl * K1 + pa) * N1 * N1 + r];
  #pragma unroll
          for (int q0 = 0; q0 < N1; ++q0) o[q0] += v * Lr[pa][q0];
        }
  #pragma unroll
        for (int q0 = 0; q0 < N1; ++q0) sU[fl * NQ + q0 * N1 * N1 + r] = o[q0] * is;
      }
    } else {  // FP64 (pipe-bound): one output per item keeps more threads busy
      for (int t = tid; t < 3 * NQ; t += nt) {
        const int fl = t / NQ, q = t - fl * NQ, q0 = q / (N1 * N1), r = q - q0 * N1 * N1;
        R acc = R(0);
  #pragma unroll
        for (int pa = 0; pa < K1; ++pa) acc += sT2[(fl * K1 + pa) * N1 * N1 + r] * L1[pa * N1 + q0];
        sU[t] = acc * is;
      }
    }
    __syncthreads();
    // (D) pointwise convective products, weighted
    for (int q = tid; q < NQ; q += nt) {
      const R u[3] = {sU[q], sU[NQ + q], sU[2 * NQ + q]};
      R ub[3];
      if (MODE == MODE_TAN) {
#pragma unroll
        for (int c = 0; c < 3; ++c) ub[c] = a.ubar[((size_t)e * 3 + c) * NQ + q];
      } else if (MODE == MODE_LINPART) {
#pragma unroll
        for (int c = 0; c < 3; ++c) ub[c] = R(0);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) ub[c] = u[c];
        if (MODE == MODE_RES_LIN)
#pragma unroll
          for (int c = 0; c < 3; ++c) a.ubar[((size_t)e * 3 + c) * NQ + q] = u[c];
      }
      // the weight goes on the velocity (or its variation) first: u_w = w_q u
      const R wq = W3[q];
      const R uw[3] = {u[0] * wq, u[1] * wq, u[2] * wq};
#pragma unroll
      for (int sp = 0; sp < 6; ++sp) {
        int p, i;
        if (sp < 3) { p = sp; i = sp; } else if (sp == 3) { p = 0; i = 1; } else if (sp == 4) { p = 0; i = 2; } else { p = 1; i = 2; }
        R v;
        if (MODE == MODE_TAN) {
          if (sp < 3) {
            const R h = uw[p] * ub[p];
            v = h + h;
          } else {
            v = uw[p] * ub[i] + ub[p] * uw[i];
          }
        } else {
          v = (MODE == MODE_LINPART) ? R(0) : uw[p] * u[i];
        }
        sPr[sp * NQ + q] = v;
      }
    }
    __syncthreads();
    // (E) projection step 1: S1[sp][a][q1 q2] = sum_q0 L1[a][q0] Pr[sp][q0 q1 q2]
    if constexpr (sizeof(R) == 4) {  // FP32: pencils, fewer instructions per output
      for (int t = tid; t < 6 * N1 * N1; t += nt) {  // pencil (product, q1 q2): all a
        const int sp = t / (N1 * N1), r2 = t - sp * N1 * N1;
        R v[N1];
  #pragma unroll
        for (int q0 = 0; q0 < N1; ++q0) v[q0] = sPr[sp * NQ + q0 * N1 * N1 + r2];
  #pragma unroll
        for (int pa = 0; pa < K1; ++pa) {
          R acc = R(0);
  #pragma unroll
          for (int q0 = 0; q0 < N1; ++q0) acc += Lr[pa][q0] * v[q0];
          sS1[(sp * K1 + pa) * N1 * N1 + r2] = acc;
        }
      }
    } else {  // FP64 (pipe-bound): one output per item keeps more threads busy
      for (int t = tid; t < 6 * K1 * N1 * N1; t += nt) {
        const int sp = t / (K1 * N1 * N1), r = t - sp * K1 * N1 * N1, pa = r / (N1 * N1), r2 = r - pa * N1 * N1;
        R acc = R(0);
  #pragma unroll
        for (int q0 = 0; q0 < N1; ++q0) acc += L1[pa * N1 + q0] * sPr[sp * NQ + q0 * N1 * N1 + r2];
        sS1[t] = acc;
      }
    }
    __syncthreads();
    // (F) projection step 2: S2[sp][pair(a,b)][q2] = sum_q1 L1[b][q1] S1[sp][a][q1 q2]
    if constexpr (sizeof(R) == 4) {  // FP32: pencils, fewer instructions per output
      for (int t = tid; t < 6 * K1 * N1; t += nt) {  // pencil (product, a, q2): all b <= K - a
        const int sp = t / (K1 * N1), r = t - sp * K1 * N1, pa = r / N1, q2 = r - pa * N1;
        R v[N1];
  #pragma unroll
        for (int q1 = 0; q1 < N1; ++q1) v[q1] = sS1[(sp * K1 + pa) * N1 * N1 + q1 * N1 + q2];
  #pragma unroll
        for (int pb = 0; pb < K1; ++pb)
          if (pb <= K - pa) {
            R acc = R(0);
  #pragma unroll
            for (int q1 = 0; q1 < N1; ++q1) acc += Lr[pb][q1] * v[q1];
            sS2[(sp * N2 + PIDX[pa * K1 + pb]) * N1 + q2] = acc;
          }
      }
    } else {  // FP64 (pipe-bound): one output per item keeps more threads busy
      for (int t = tid; t < 6 * N2 * N1; t += nt) {
        const int sp = t / (N2 * N1), r = t - sp * N2 * N1, pi = r / N1, q2 = r - pi * N1;
        const int pa = PAB[2 * pi], pb = PAB[2 * pi + 1];
        R acc = R(0);
  #pragma unroll
        for (int q1 = 0; q1 < N1; ++q1) acc += L1[pb * N1 + q1] * sS1[(sp * K1 + pa) * N1 * N1 + q1 * N1 + q2];
        sS2[t] = acc;
      }
    }
    __syncthreads();
    // (G) projection step 3: Cv[sp][m] = s * sum_q2 L1[c][q2] S2[sp][pair(a,b)][q2]
    if constexpr (sizeof(R) == 4) {  // FP32: pencils, fewer instructions per output
      for (int t = tid; t < 6 * N2; t += nt) {  // pencil (product, pair (a, b)): all c <= K - a - b
        const int sp = t / N2, pi = t - sp * N2;
        const int pa = PAB[2 * pi], pb = PAB[2 * pi + 1];
        const int* row = IDX3 + (pa * K1 + pb) * K1;
        R v[N1];
  #pragma unroll
        for (int q2 = 0; q2 < N1; ++q2) v[q2] = sS2[(sp * N2 + pi) * N1 + q2];
  #pragma unroll
        for (int pc = 0; pc < K1; ++pc)
          if (pc <= K - pa - pb) {
            R acc = R(0);
  #pragma unroll
            for (int q2 = 0; q2 < N1; ++q2) acc += Lr[pc][q2] * v[q2];
            const int m = row[pc];
            sCv[sp * NB + m] = (sp < 3 ? sFv[sp * NB + m] - sC[3 * NB + m] : sFv[sp * NB + m]) - acc * R(g.s);
          }
      }
    } else {  // FP64 (pipe-bound): one output per item keeps more threads busy
      for (int t = tid; t < 6 * NB; t += nt) {
        const int sp = t / NB, m = t - sp * NB;
        const int pa = MD3[3 * m], pb = MD3[3 * m + 1], pc = MD3[3 * m + 2];
        const R* s2 = sS2 + (sp * N2 + PIDX[pa * K1 + pb]) * N1;
        R acc = R(0);
  #pragma unroll
        for (int q2 = 0; q2 < N1; ++q2) acc += L1[pc * N1 + q2] * s2[q2];
        sCv[t] = (sp < 3 ? sFv[t] - sC[3 * NB + m] : sFv[t]) - acc * R(g.s);
      }
    }
    __syncthreads();
    // (H) assemble: modal derivatives of (F^nu - u(x)u) and p, continuity, face terms, mass shift
    const R* FO = a.face_out + (size_t)e * 6 * 4 * N2;
    if constexpr (sizeof(R) == 4) {  // FP32: one thread per mode m for the four variables
      for (int m = tid; m < NB; m += nt) {
        R acc[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
        for (int pp = 0; pp < 3; ++pp) {
          R s2[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
          for (int j = 0; j < DW; ++j) {
            const int o = (pp * NB + m) * DW + j;
            const int n = a.T.Dcol_idx[o];
            const R dv = a.rt.Dcol_val[o];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const int sp = sym_index(pp, i);
              s2[i] += dv * sCv[sp * NB + n];
            }
            s2[3] += dv * (-sC[pp * NB + n]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] += Jd[pp] * s2[i];
        }
#pragma unroll
        for (int sl = 0; sl < 6; ++sl) {
          const int dd = sl >> 1, side = (sl & 1) ? 0 : 1;
          const R pw = PV[side * K1 + FA[dd * NB + m]];
          const int fm = FMAP[dd * NB + m];
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] += pw * FO[sl * 4 * N2 + i * N2 + fm];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (MODE == MODE_TAN && i < 3) acc[i] += shift * sC[i * NB + m];
          nonfinite |= !isfinite(acc[i]);
          a.out[(size_t)e * 4 * NB + i * NB + m] = acc[i];
        }
      }
    } else {
      for (int t = tid; t < 4 * NB; t += nt) {
        const int i = t / NB, m = t - i * NB;
        R acc = R(0);
  #pragma unroll
        for (int pp = 0; pp < 3; ++pp) {
          R s2 = R(0);
  #pragma unroll
          for (int j = 0; j < DW; ++j) {
            const int o = (pp * NB + m) * DW + j;
            const int n = a.T.Dcol_idx[o];
            const R fld = i < 3 ? sCv[sym_index(pp, i) * NB + n] : -sC[pp * NB + n];
            s2 += a.rt.Dcol_val[o] * fld;
          }
          acc += Jd[pp] * s2;
        }
  #pragma unroll
        for (int sl = 0; sl < 6; ++sl) {
          const int dd = sl >> 1, side = (sl & 1) ? 0 : 1;
          acc += PV[side * K1 + FA[dd * NB + m]] * FO[sl * 4 * N2 + i * N2 + FMAP[dd * NB + m]];
        }
        if (MODE == MODE_TAN && i < 3) acc += shift * sC[t];
        nonfinite |= !isfinite(acc);
        a.out[(size_t)e * 4 * NB + t] = acc;
      }
    }
    __syncthreads();
  }
  // scan of the outputs: a non-finite entry (from a non-finite input or an overflow) sets the
  // status bit, once per thread that wrote one
  if (nonfinite && a.status) atomicOr(a.status, (unsigned)DG_STATUS_NONFINITE);
}

// ------------------------------------------------------- Taylor-Green vortex
template <int K>
__global__ void __launch_bounds__(128) tgv_kernel(MeshDev M, const double* Bvol, const double* wvol,
                                                  const double* xg, double* w) {
  using S = Sz<K>;
  constexpr int NB = S::NB, NQ = S::NQ, N1 = S::N1;
  __shared__ double sF[4 * NQ];
  for (int e = blockIdx.x; e < M.ne; e += gridDim.x) {
    const ElemGeom g = elem_geom(M, e);
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
      const int q0 = q / (N1 * N1), q1 = (q / N1) % N1, q2 = q % N1;
      const double x = g.lo[0] + 0.5 * g.h[0] * (xg[q0] + 1.0);
      const double y = g.lo[1] + 0.5 * g.h[1] * (xg[q1] + 1.0);
      const double z = g.lo[2] + 0.5 * g.h[2] * (xg[q2] + 1.0);
      const double wq = wvol[q];
      sF[0 * NQ + q] = sin(x) * cos(y) * cos(z) * wq;
      sF[1 * NQ + q] = -cos(x) * sin(y) * cos(z) * wq;
      sF[2 * NQ + q] = 0.0;
      sF[3 * NQ + q] = (cos(2.0 * x) + cos(2.0 * y)) * (cos(2.0 * z) + 2.0) * (1.0 / 16.0) * wq;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * NB; t += blockDim.x) {
      const int v = t / NB, m = t - v * NB;
      double acc = 0.0;
      for (int q = 0; q < NQ; ++q) acc += Bvol[q * NB + m] * sF[v * NQ + q];
      w[(size_t)e * 4 * NB + t] = acc * g.s;
    }
    __syncthreads();
  }
}

// ------------------------------------------------ points and projections of given fields
template <int K>
__global__ void __launch_bounds__(128) quad_points_kernel(MeshDev M, const double* xg, double* xyz) {
  constexpr int N1 = K + 1, NQ = N1 * N1 * N1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)M.ne * NQ;
       i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i / NQ), q = (int)(i - (long long)e * NQ);
    const int q0 = q / (N1 * N1), q1 = (q / N1) % N1, q2 = q % N1;
    const ElemGeom g = elem_geom(M, e);
    double* o = xyz + i * 3;
    o[0] = g.lo[0] + 0.5 * g.h[0] * (xg[q0] + 1.0);
    o[1] = g.lo[1] + 0.5 * g.h[1] * (xg[q1] + 1.0);
    o[2] = g.lo[2] + 0.5 * g.h[2] * (xg[q2] + 1.0);
  }
}

// w[e][v][m] = s_e sum_q phi_hat_m(x_q) wvol_q vals[e][v][q]: the Gauss-rule L2 projection onto the
// orthonormal basis phi_m = phi_hat_m / s_e (the |K|/8 of dx and the 1/s of phi_m give s_e)
template <int K>
__global__ void __launch_bounds__(128) project_points_kernel(MeshDev M, const double* Bvol, const double* wvol,
                                                             const double* vals, double* w) {
  using S = Sz<K>;
  constexpr int NB = S::NB, NQ = S::NQ;
  for (int e = blockIdx.x; e < M.ne; e += gridDim.x) {
    const ElemGeom g = elem_geom(M, e);
    const double* ve = vals + (size_t)e * 4 * NQ;
    for (int t = threadIdx.x; t < 4 * NB; t += blockDim.x) {
      const int v = t / NB, m = t - v * NB;
      double acc = 0.0;
      for (int q = 0; q < NQ; ++q) acc += Bvol[q * NB + m] * wvol[q] * ve[v * NQ + q];
      w[(size_t)e * 4 * NB + t] = acc * g.s;
    }
  }
}

// ------------------------------------------------------------- FD helpers
__global__ void fd_perturb_kernel(long long n, const double* w, const double* v, const double* wnorm2,
                                  const double* vnorm2, double* out) {
  const double nv = sqrt(*vnorm2);
  const double delta = nv > 0.0 ? 1e-9 * sqrt(1.0 + sqrt(*wnorm2)) / nv : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = w[i] + delta * v[i];
}
__global__ void fd_finish_kernel(long long n, int nb, const double* f1, const double* f0, const double* v,
                                 const double* wnorm2, const double* vnorm2, double inv_gdt, const double* geo,
                                 double* out) {
  const double nv = sqrt(*vnorm2);
  const double delta = nv > 0.0 ? 1e-9 * sqrt(1.0 + sqrt(*wnorm2)) / nv : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int var = (int)((i / nb) & 3);
    const long long e = i / (4 * nb);
    const double mass = var < 3 ? inv_gdt * geo[e * kGeo + 11] * v[i] : 0.0;
    out[i] = (delta > 0.0 ? (f1[i] - f0[i]) / delta : 0.0) + mass;
  }
}

// ------------------------------------------------------------- launchers
static OpArgs make_args(Handle* h, const double* in, double* out) {
  OpArgs a;
  a.M = mesh_dev(h);
  a.T = h->tab;
  a.rt = RTab<double>{h->tab.L1, h->tab.wvol, h->tab.B2, h->tab.W2, h->tab.pv, h->tab.pd, h->tab.Drow_val,
                     h->tab.Dcol_val, h->tab.D2_val};
  a.in = in;
  a.out = out;
  a.face_out = h->face_out;
  a.face_lift = h->face_lift;
  a.ubar = h->ubar;
  a.dFlux = h->dFlux;
  a.nu = h->p.nu;
  a.c = h->p.ac_c;
  a.eta = h->p.eta;
  a.inv_gdt = h->inv_gdt;
  a.status = h->status;
  a.riemann_its = h->dbg.riemann_its;
  return a;
}

static OpArgsT<float> make_args_f(Handle* h, const float* in, float* out) {
  OpArgsT<float> a;
  const TablesF& F = h->tabf;
  a.M = mesh_dev(h);
  a.T = h->tab;
  a.rt = RTab<float>{F.L1, F.wvol, F.B2, F.W2, F.pv, F.pd, F.Drow_val, F.Dcol_val, F.D2_val};
  a.in = in;
  a.out = out;
  a.face_out = h->face_out_f;
  a.face_lift = h->face_lift_f;
  a.ubar = h->ubar_f;
  a.dFlux = h->dFlux_f;
  a.nu = h->p.nu;
  a.c = h->p.ac_c;
  a.eta = h->p.eta;
  a.inv_gdt = h->inv_gdt;
  a.status = h->status;
  a.riemann_its = h->dbg.riemann_its;
  return a;
}

// CTAs of `kernel` that one SM holds at once (registers, shared memory and threads), cached per
// (kernel, block size): the grids below are one wave of the GPU, so that no SM runs a second,
// thinner wave of a grid-stride loop
template <class Kern>
static int resident_ctas(Kern kernel, int threads, size_t smem) {
  struct Entry {
    const void* fn;
    int threads;
    size_t smem;
    int n;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  const void* fn = reinterpret_cast<const void*>(kernel);
  std::lock_guard<std::mutex> lk(mu);
  for (const Entry& c : cache)
    if (c.fn == fn && c.threads == threads && c.smem == smem) return c.n;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 0;  // unknown: the caller keeps its own bound
  }
  cache.push_back(Entry{fn, threads, smem, n});
  return n;
}

// Launch shapes of the tangent passes (the hot products of the solver): faces per CTA of the face
// pass, threads per CTA of the volume pass, CTAs per SM of each (0: as many as shared memory
// allows, at most 8 / 12). Every output entry is computed by the same arithmetic in the same order
// whatever the shape, so the results do not depend on it.
template <int K, int MODE, class R, int FW>
static int launch_face(Handle* h, const OpArgsT<R>& a, int per_sm_cap, cudaStream_t st) {
  const size_t fs = FaceSmem<K, R, FW>::bytes();
  DG_CUDA(h, cudaFuncSetAttribute(face_kernel<K, MODE, R, FW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs));
  int per_sm = (int)((200 * 1024) / fs);
  per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
  const int res = resident_ctas(face_kernel<K, MODE, R, FW>, 32 * FW, fs);
  if (res > 0 && per_sm > res) per_sm = res;
  if (per_sm_cap > 0 && per_sm > per_sm_cap) per_sm = per_sm_cap;
  const int fblocks = (3 * h->ne + h->nbf + FW - 1) / FW;
  int gf = h->nsm * per_sm;
  if (gf > fblocks) gf = fblocks;
  face_kernel<K, MODE, R, FW><<<gf, 32 * FW, fs, st>>>(a);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

template <int K, int MODE, class R>
static int run_operator(Handle* h, const OpArgsT<R>& a, cudaStream_t st, bool face_only = false) {
  const bool tan = (MODE == MODE_TAN || MODE == MODE_LINPART);
  const OpTune tu = MODE == MODE_TAN ? h->tune[sizeof(R) == 4 ? 1 : 0] : OpTune{};
  const size_t vs = VolSmem<K, R>::bytes();
  DG_CUDA(h, cudaFuncSetAttribute(vol_kernel<K, MODE, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vs));
  int per_sm_v = (int)((200 * 1024) / vs);
  per_sm_v = per_sm_v < 1 ? 1 : (per_sm_v > 12 ? 12 : per_sm_v);
  const int res_v = resident_ctas(vol_kernel<K, MODE, R>, tu.vol_threads, vs);
  if (res_v > 0 && per_sm_v > res_v) per_sm_v = res_v;
  if (tu.vol_per_sm > 0 && per_sm_v > tu.vol_per_sm) per_sm_v = tu.vol_per_sm;
  int gv = h->nsm * per_sm_v;
  if (gv > h->ne) gv = h->ne;
  const int cf = tan ? (sizeof(R) == 4 ? DG_PROF_FACE_TAN32 : DG_PROF_FACE_TAN) : DG_PROF_FACE_RES;
  const int cv = tan ? (sizeof(R) == 4 ? DG_PROF_VOL_TAN32 : DG_PROF_VOL_TAN) : DG_PROF_VOL_RES;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc;
  if ((rc = prof_begin(h, st, &e0))) return rc;
  if constexpr (MODE == MODE_TAN) {
    switch (tu.face_warps) {
      case 2: rc = launch_face<K, MODE, R, 2>(h, a, tu.face_per_sm, st); break;
      case 8: rc = launch_face<K, MODE, R, 8>(h, a, tu.face_per_sm, st); break;
      default: rc = launch_face<K, MODE, R, 4>(h, a, tu.face_per_sm, st); break;
    }
  } else {
    rc = launch_face<K, MODE, R, kFaceWarps>(h, a, 0, st);
  }
  if (rc) return rc;
  if ((rc = prof_end(h, cf, st, e0))) return rc;
  if (face_only) return DG_OK;
  if ((rc = prof_begin(h, st, &e1))) return rc;
  vol_kernel<K, MODE, R><<<gv, tu.vol_threads, vs, st>>>(a);
  DG_LAUNCH_CHECK(h);
  if ((rc = prof_end(h, cv, st, e1))) return rc;
  ++h->op_apps;
  return DG_OK;
}

template <int MODE, class R>
static int dispatch(Handle* h, const OpArgsT<R>& a, cudaStream_t st, bool face_only = false) {
  switch (h->tab.k) {
    case 1: return run_operator<1, MODE, R>(h, a, st, face_only);
    case 2: return run_operator<2, MODE, R>(h, a, st, face_only);
    case 3: return run_operator<3, MODE, R>(h, a, st, face_only);
    case 4: return run_operator<4, MODE, R>(h, a, st, face_only);
  }
  return fail(h, DG_ERR_ARG, "unsupported degree");
}

int op_residual(Handle* h, const double* w, double* f, bool store_lin, cudaStream_t st) {
  OpArgs a = make_args(h, w, f);
  if (store_lin) a.status = h->status + 1;  // the linearisation's own word, read by dg_set_linearization
  return store_lin ? dispatch<MODE_RES_LIN>(h, a, st) : dispatch<MODE_RES>(h, a, st);
}

int op_tangent(Handle* h, const double* v, double* out, cudaStream_t st) {
  OpArgs a = make_args(h, v, out);
  return dispatch<MODE_TAN>(h, a, st);
}

int op_tangent_f32(Handle* h, const float* v, float* out, int tc, cudaStream_t st) {
  OpArgsT<float> a = make_args_f(h, v, out);
  if (!tc) return dispatch<MODE_TAN>(h, a, st);
  // the face pass as usual, then the volume pass with its contractions on the tensor cores
  int rc = dispatch<MODE_TAN>(h, a, st, true);
  if (rc) return rc;
  cudaEvent_t e1 = nullptr;
  if ((rc = prof_begin(h, st, &e1))) return rc;
  if ((rc = tc_volume_tangent(h, v, out, tc, st))) return rc;
  if ((rc = prof_end(h, DG_PROF_VOL_TC32, st, e1))) return rc;
  ++h->op_apps;
  return DG_OK;
}

int op_linear_part(Handle* h, const double* v, double* out, cudaStream_t st) {
  OpArgs a = make_args(h, v, out);
  return dispatch<MODE_LINPART>(h, a, st);
}

int op_fd(Handle* h, const double* v, double* out, cudaStream_t st) {
  const long long n = h->lev[0].n;
  int rc = vec_norm2(h, v, n, h->red_out, st);
  if (rc) return rc;
  const int blocks = h->nsm * 8;
  fd_perturb_kernel<<<blocks, 256, 0, st>>>(n, h->wlin, v, h->wnorm2, h->red_out, h->fd_w);
  DG_LAUNCH_CHECK(h);
  rc = op_residual(h, h->fd_w, h->fd_f, false, st);
  if (rc) return rc;
  fd_finish_kernel<<<blocks, 256, 0, st>>>(n, h->lev[0].nb, h->fd_f, h->flin, v, h->wnorm2, h->red_out,
                                           h->inv_gdt, h->geo, out);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

int op_quad_points(Handle* h, double* xyz, cudaStream_t st) {
  const MeshDev M = mesh_dev(h);
  const int grid = h->nsm * 8;
  switch (h->tab.k) {
    case 1: quad_points_kernel<1><<<grid, 128, 0, st>>>(M, h->tab.xg, xyz); break;
    case 2: quad_points_kernel<2><<<grid, 128, 0, st>>>(M, h->tab.xg, xyz); break;
    case 3: quad_points_kernel<3><<<grid, 128, 0, st>>>(M, h->tab.xg, xyz); break;
    case 4: quad_points_kernel<4><<<grid, 128, 0, st>>>(M, h->tab.xg, xyz); break;
  }
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

int op_project_points(Handle* h, const double* vals, double* w, cudaStream_t st) {
  const MeshDev M = mesh_dev(h);
  const int grid = std::min(h->ne, h->nsm * 8);
  switch (h->tab.k) {
    case 1: project_points_kernel<1><<<grid, 128, 0, st>>>(M, h->tab.Bvol, h->tab.wvol, vals, w); break;
    case 2: project_points_kernel<2><<<grid, 128, 0, st>>>(M, h->tab.Bvol, h->tab.wvol, vals, w); break;
    case 3: project_points_kernel<3><<<grid, 128, 0, st>>>(M, h->tab.Bvol, h->tab.wvol, vals, w); break;
    case 4: project_points_kernel<4><<<grid, 128, 0, st>>>(M, h->tab.Bvol, h->tab.wvol, vals, w); break;
  }
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

int op_project_tgv(Handle* h, double* w, cudaStream_t st) {
  const MeshDev M = mesh_dev(h);
  const int grid = h->ne < h->nsm * 8 ? h->ne : h->nsm * 8;
  switch (h->tab.k) {
    case 1: tgv_kernel<1><<<grid, 128, 0, st>>>(M, h->tab.Bvol, h->tab.wvol, h->tab.xg, w); break;
    case 2: tgv_kernel<2><<<grid, 128, 0, st>>>(M, h->tab.Bvol, h->tab.wvol, h->tab.xg, w); break;
    case 3: tgv_kernel<3><<<grid, 128, 0, st>>>(M, h->tab.Bvol, h->tab.wvol, h->tab.xg, w); break;
    case 4: tgv_kernel<4><<<grid, 128, 0, st>>>(M, h->tab.Bvol, h->tab.wvol, h->tab.xg, w); break;
    default: return fail(h, DG_ERR_ARG, "unsupported degree");
  }
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// ------------------------------------------------- residual without allocation
// Scratch of dg_residual_noalloc: the per-face-slot contributions and lifting
// coefficients of the face pass (N_e * 6 * (4 + 3) * N_2 doubles, N_2 = (k+1)(k+2)/2), in a
// file-scope device array instead of the handle's own buffers. Every GPU that
// loads the library holds it until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[DG_NOALLOC_SCRATCH_DOUBLES];

// Device address of g_noalloc_scratch on the handle's device, looked up once per device with
// that device current (the caller's device must be the handle's). In host code the array's name
// is only a host-side stand-in, never a device address, so it must not be passed to a kernel.
static int noalloc_scratch(Handle* h, double** out) {
  static std::mutex mu;
  static double* addr[64] = {};
  const int dev = h->device;
  int cur = -1;
  DG_CUDA(h, cudaGetDevice(&cur));
  if (cur != dev)
    return fail(h, DG_ERR_ARG, "dg_residual_noalloc: make the handle's device (" + std::to_string(dev) +
                                   ") current; device " + std::to_string(cur) + " is");
  if (dev < 0 || dev >= 64) return fail(h, DG_ERR_ARG, "device index out of range for the static scratch");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    double* p = nullptr;
    DG_CUDA(h, cudaGetSymbolAddress((void**)&p, g_noalloc_scratch));
    if (!p) return fail(h, DG_ERR_CUDA, "cudaGetSymbolAddress returned a null address");
    addr[dev] = p;
  }
  *out = addr[dev];
  return DG_OK;
}

}  // namespace dg

extern "C" int dg_residual_noalloc(dg_handle* hh, const double* w, double* f, void* stream) {
  using namespace dg;
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!w || !f || w == f) return fail(h, DG_ERR_ARG, "w and f must be distinct non-null device pointers");
  const int n2 = h->tab.n2;
  const long long need = (long long)h->ne * 6 * 7 * n2;
  if (need > (long long)DG_NOALLOC_SCRATCH_DOUBLES)
    return fail(h, DG_ERR_ARG,
                "mesh too large for the static scratch of dg_residual_noalloc: it needs N_e*42*N_2 = " +
                    std::to_string(need) + " doubles, the limit is " + std::to_string(DG_NOALLOC_SCRATCH_DOUBLES));
  double* scratch = nullptr;
  int rc = noalloc_scratch(h, &scratch);
  if (rc) return rc;
  OpArgs a = make_args(h, w, f);
  a.face_out = scratch;
  a.face_lift = scratch + (size_t)h->ne * 6 * 4 * n2;
  return dispatch<MODE_RES, double>(h, a, as_stream(stream));
}
