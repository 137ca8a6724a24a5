// Matrix-free DG operator on sm_103a: residual f_h (Eq. (NSdiscrRes)), its
// exact linearisation (Eqs. (jacTrilFnotNU), (jacTrilnu)) and the
// finite-difference action (Eqs. (matrix-free), (epsdef)).
//
// Two kernels per application:
//  * face_kernel: one face s = (K, K') at a time. Traces of the four
//    variables and of the nine velocity gradients on both sides, the BR2 local
//    liftings r^s([u]) (coefficients on K and K'), the artificial-compressibility
//    Riemann flux (exact star state by safeguarded Newton; in tangent mode its
//    cached Jacobian), the BR2 face viscous flux F^nu({grad u - eta r^s}), and
//    the integration against the test functions of both sides. Writes per
//    element face slot: the face-term contribution and the lifting coefficients.
//  * vol_kernel: one element at a time. Corrected-gradient coefficients
//    grad u - R^K(u) (exact modal derivative + the six liftings), values at the
//    Gauss points, pointwise flux F~, its projection onto the basis, and the
//    exact modal derivative of that projection (= integration against grad phi),
//    plus the six face contributions and the mass shift.
//
// Conventions (also in the C ABI header): orthonormal modal basis
// phi_m = phi_hat_m(xi)/s, s = sqrt(|K|/8), Gauss rule with k+1 points per
// axis; the normal of a face points from K (lower index) to K'; [v] = v_K - v_K';
// the lifting is defined by int r . tau = + int_s [v] {tau} . n so that
// grad u - R^K is the consistent gradient (Sec. 2.1).
#include <mutex>

#include "dg_internal.h"

namespace dg {

template <int K>
struct Sz {
  static constexpr int NB = nb_of(K), N1 = K + 1, NQ = N1 * N1 * N1, NQF = N1 * N1;
};

enum { MODE_RES = 0, MODE_RES_LIN = 1, MODE_TAN = 2 };

struct OpArgs {
  MeshDev M;
  const double* Bvol;
  const double* wvol;
  const double* Bface;
  const double* wface;
  const int* Drow_idx;
  const double* Drow_val;
  const int* Dcol_idx;
  const double* Dcol_val;
  const double* in;
  double* out;
  double* face_out;
  double* face_lift;
  double* ubar;
  double* dFlux;
  double nu, c, eta, inv_gdt;
  unsigned* status;
};

// ------------------------------------------------------------------ Riemann
// Pressure on the 1-wave curve through (uL, pL) at star velocity u, and its
// partial derivatives in u and uL (dp/dpL = 1). Shock (u < uL): Rankine-Hugoniot
// with the negative root s of s^2 - (uL+u)s - c^2 = 0, p = pL + c^2 (u-uL)/s.
// Rarefaction: dp/du = -(u + sqrt(u^2+c^2)) integrated in closed form.
__device__ __forceinline__ void wave1(double u, double uL, double pL, double c, double& p, double& dpdu,
                                      double& dpduL) {
  const double c2 = c * c;
  if (u < uL) {
    const double sig = uL + u, Q = sqrt(sig * sig + 4.0 * c2), s = 0.5 * (sig - Q);
    const double ss = -s / Q;  // ds/dsig
    const double du = u - uL, is = 1.0 / s;
    p = pL + c2 * du * is;
    dpdu = c2 * (is - du * ss * is * is);
    dpduL = c2 * (-is - du * ss * is * is);
  } else {
    const double a = sqrt(u * u + c2), aL = sqrt(uL * uL + c2);
    const double Gu = 0.5 * (u * u + u * a + c2 * asinh(u / c));
    const double GL = 0.5 * (uL * uL + uL * aL + c2 * asinh(uL / c));
    p = pL - (Gu - GL);
    dpdu = -(u + a);
    dpduL = uL + aL;
  }
}
// Pressure on the 3-wave curve through (uR, pR): shock for u > uR (positive root),
// rarefaction dp/du = sqrt(u^2+c^2) - u otherwise. Partials in u and uR (dp/dpR = 1).
__device__ __forceinline__ void wave3(double u, double uR, double pR, double c, double& p, double& dpdu,
                                      double& dpduR) {
  const double c2 = c * c;
  if (u > uR) {
    const double sig = u + uR, Q = sqrt(sig * sig + 4.0 * c2), s = 0.5 * (sig + Q);
    const double ss = s / Q;
    const double du = u - uR, is = 1.0 / s;
    p = pR + c2 * du * is;
    dpdu = c2 * (is - du * ss * is * is);
    dpduR = c2 * (-is - du * ss * is * is);
  } else {
    const double a = sqrt(u * u + c2), aR = sqrt(uR * uR + c2);
    const double Hu = 0.5 * (u * a + c2 * asinh(u / c) - u * u);
    const double HR = 0.5 * (uR * aR + c2 * asinh(uR / c) - uR * uR);
    p = pR - (HR - Hu);
    dpdu = a - u;
    dpduR = -(aR - uR);
  }
}
// Tangential-velocity ratio across the 1-wave, tau = u_t(star)/u_t(L), with partials
// in u* and uL. Rarefaction: u_t (u + a) invariant; shock: s [u_t] = [u_n u_t].
__device__ __forceinline__ void tang1(double u, double uL, double c, double& t, double& dtdu, double& dtduL) {
  const double c2 = c * c;
  if (u < uL) {
    const double sig = uL + u, Q = sqrt(sig * sig + 4.0 * c2), s = 0.5 * (sig - Q), ss = -s / Q;
    const double den = s - u, num = s - uL, id = 1.0 / den;
    t = num * id;
    dtdu = (ss * den - num * (ss - 1.0)) * id * id;
    dtduL = ((ss - 1.0) * den - num * ss) * id * id;
  } else {
    const double a = sqrt(u * u + c2), aL = sqrt(uL * uL + c2);
    t = (uL + aL) / (u + a);
    dtdu = -t / a;
    dtduL = t / aL;
  }
}
// Ratio across the 3-wave, tau = u_t(star)/u_t(R). Rarefaction: u_t/(u + a) invariant.
__device__ __forceinline__ void tang3(double u, double uR, double c, double& t, double& dtdu, double& dtduR) {
  const double c2 = c * c;
  if (u > uR) {
    const double sig = u + uR, Q = sqrt(sig * sig + 4.0 * c2), s = 0.5 * (sig + Q), ss = s / Q;
    const double den = s - u, num = s - uR, id = 1.0 / den;
    t = num * id;
    dtdu = (ss * den - num * (ss - 1.0)) * id * id;
    dtduR = ((ss - 1.0) * den - num * ss) * id * id;
  } else {
    const double a = sqrt(u * u + c2), aR = sqrt(uR * uR + c2);
    t = (u + a) / (uR + aR);
    dtdu = t / a;
    dtduR = -t / aR;
  }
}

// Exact interface flux of the artificial-compressibility Riemann problem along
// e_d: F[i] = n.(u(x)u + pI) at the interface state for i < 3, F[3] = u_n*.
// The two acoustic waves always travel in opposite directions, so the interface
// state is the star state; the tangential velocity is taken from the side the
// contact (speed u*) comes from, the two sides averaged when |u*| is within a
// rounding band of zero. With J != nullptr also the Jacobian J[i][j] with respect
// to (uL[0..2], pL, uR[0..2], pR).
__device__ void ac_riemann(const double* uL, double pL, const double* uR, double pR, int d, double c, double* F,
                           double (*J)[8], unsigned* status) {
  const double ul = uL[d], ur = uR[d], c2 = c * c;
  const double al = sqrt(ul * ul + c2), ar = sqrt(ur * ur + c2);
  const double scale = fabs(ul) + fabs(ur) + c;
  // two-rarefaction linearisation as the initial guess
  double us = (pL - pR + ul * (ul + al) + ur * (ar - ur)) / ((ul + al) + (ar - ur));
  double lo = -1e300, hi = 1e300;
  bool ok = false;
  double p1, d1u, d1l, p3, d3u, d3r;
  for (int it = 0; it < 60; ++it) {
    wave1(us, ul, pL, c, p1, d1u, d1l);
    wave3(us, ur, pR, c, p3, d3u, d3r);
    const double phi = p1 - p3, dphi = d1u - d3u;  // dphi < 0
    if (phi > 0.0) lo = us; else hi = us;
    double nxt = us - phi / dphi;
    if (!(nxt > lo && nxt < hi)) nxt = (lo > -1e299 && hi < 1e299) ? 0.5 * (lo + hi) : nxt;
    const double step = nxt - us;
    us = nxt;
    if (fabs(step) <= 1e-15 * scale) { ok = true; break; }
  }
  if (!ok && status) atomicOr(status, (unsigned)DG_STATUS_RIEMANN);
  wave1(us, ul, pL, c, p1, d1u, d1l);
  wave3(us, ur, pR, c, p3, d3u, d3r);
  const double ps = p1;
  // implicit-function derivatives of u* and p* with respect to (ul, pL, ur, pR)
  const double iphi = 1.0 / (d1u - d3u);
  const double dus_ul = -d1l * iphi, dus_pl = -iphi, dus_ur = d3r * iphi, dus_pr = iphi;
  const double dps_ul = d1u * dus_ul + d1l, dps_pl = d1u * dus_pl + 1.0;
  const double dps_ur = d1u * dus_ur, dps_pr = d1u * dus_pr;
  // tangential ratios
  double tl, tlu, tll, tr, tru, trr;
  tang1(us, ul, c, tl, tlu, tll);
  tang3(us, ur, c, tr, tru, trr);
  const double band = 1e-12 * scale;
  double wl, wr;  // weights of the left / right star tangential values
  if (us > band) { wl = 1.0; wr = 0.0; }
  else if (us < -band) { wl = 0.0; wr = 1.0; }
  else { wl = 0.5; wr = 0.5; }
  F[d] = us * us + ps;
  F[3] = us;
  if (J) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 8; ++j) J[i][j] = 0.0;
    // d(u*) row and the normal momentum row
    const double gus[8] = {0, 0, 0, dus_pl, 0, 0, 0, dus_pr};
    double du[8], dp[8];
    for (int j = 0; j < 8; ++j) { du[j] = gus[j]; dp[j] = 0.0; }
    du[d] = dus_ul; du[4 + d] = dus_ur;
    dp[d] = dps_ul; dp[3] = dps_pl; dp[4 + d] = dps_ur; dp[7] = dps_pr;
    for (int j = 0; j < 8; ++j) {
      J[3][j] = du[j];
      J[d][j] = 2.0 * us * du[j] + dp[j];
    }
    for (int t = 1; t < 3; ++t) {
      const int i = (d + t) % 3;
      const double ut = wl * uL[i] * tl + wr * uR[i] * tr;
      F[i] = ut * us;
      // d(ut) = wl (tl duL_i + uL_i (tlu du* + tll dul)) + wr (tr duR_i + uR_i (tru du* + trr dur))
      double dut[8];
      for (int j = 0; j < 8; ++j) dut[j] = (wl * uL[i] * tlu + wr * uR[i] * tru) * du[j];
      dut[d] += wl * uL[i] * tll;
      dut[4 + d] += wr * uR[i] * trr;
      dut[i] += wl * tl;
      dut[4 + i] += wr * tr;
      for (int j = 0; j < 8; ++j) J[i][j] = us * dut[j] + ut * du[j];
    }
  } else {
    for (int t = 1; t < 3; ++t) {
      const int i = (d + t) % 3;
      F[i] = (wl * uL[i] * tl + wr * uR[i] * tr) * us;
    }
  }
}

// ---------------------------------------------------------------- face pass
template <int K, int MODE>
__global__ void __launch_bounds__(128) face_kernel(OpArgs a) {
  using S = Sz<K>;
  constexpr int NB = S::NB, NQF = S::NQF;
  extern __shared__ double sm[];
  double* sBf = sm;                 // [3][2][NQF][NB]
  double* sC = sBf + 6 * NQF * NB;  // [2][4][NB]
  double* sG = sC + 8 * NB;         // [2][9][NB] velocity-gradient coefficients, index a*3+b
  double* sT = sG + 18 * NB;        // [2][13][NQF] traces: 0..3 values, 4 + a*3+b gradients
  double* sR = sT + 26 * NQF;       // [2][3][NB] lifting coefficients
  double* sRq = sR + 6 * NB;        // [2][3][NQF] liftings at the face points
  double* sFn = sRq + 6 * NQF;      // [4][NQF] weighted normal flux
  double* sW = sFn + 4 * NQF;       // [NQF] reference face weights
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < 6 * NQF * NB; t += nt) sBf[t] = a.Bface[t];
  for (int t = tid; t < NQF; t += nt) sW[t] = a.wface[t];
  __syncthreads();
  const int nfaces = 3 * a.M.ne;
  for (int f = blockIdx.x; f < nfaces; f += gridDim.x) {
    const int e0 = f / 3, d = f - 3 * e0;
    const int e1 = a.M.nbr[e0 * 6 + 2 * d + 1];
    const ElemGeom g0 = elem_geom(a.M, e0), g1 = elem_geom(a.M, e1);
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const double A4 = 0.25 * g0.h[t1] * g0.h[t2];
    const double is0 = 1.0 / g0.s, is1 = 1.0 / g1.s;
    for (int t = tid; t < 8 * NB; t += nt) {
      const int side = t / (4 * NB), r = t - side * 4 * NB;
      sC[t] = a.in[(size_t)(side ? e1 : e0) * 4 * NB + r];
    }
    __syncthreads();
    for (int t = tid; t < 18 * NB; t += nt) {
      const int side = t / (9 * NB), r = t - side * 9 * NB, ab = r / NB, m = r - ab * NB;
      const int av = ab / 3, b = ab - 3 * av;
      const double* cv = sC + side * 4 * NB + av * NB;
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < Tables::kDw; ++j) {
        const int o = (b * NB + m) * Tables::kDw + j;
        acc += a.Drow_val[o] * cv[a.Drow_idx[o]];
      }
      sG[t] = acc * (2.0 / (side ? g1.h[b] : g0.h[b]));
    }
    __syncthreads();
    const double* B0 = sBf + (2 * d + 0) * NQF * NB;
    const double* B1 = sBf + (2 * d + 1) * NQF * NB;
    for (int t = tid; t < 26 * NQF; t += nt) {
      const int side = t / (13 * NQF), r = t - side * 13 * NQF, fld = r / NQF, q = r - fld * NQF;
      const double* cf = fld < 4 ? sC + side * 4 * NB + fld * NB : sG + side * 9 * NB + (fld - 4) * NB;
      const double* B = (side ? B1 : B0) + q * NB;
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < NB; ++m) acc += B[m] * cf[m];
      sT[t] = acc * (side ? is1 : is0);
    }
    __syncthreads();
    for (int t = tid; t < 6 * NB; t += nt) {
      const int side = t / (3 * NB), r = t - side * 3 * NB, av = r / NB, m = r - av * NB;
      const double* B = side ? B1 : B0;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NQF; ++q) acc += sW[q] * (sT[av * NQF + q] - sT[13 * NQF + av * NQF + q]) * B[q * NB + m];
      sR[t] = 0.5 * A4 * (side ? is1 : is0) * acc;
    }
    __syncthreads();
    for (int t = tid; t < 6 * NQF; t += nt) {
      const int side = t / (3 * NQF), r = t - side * 3 * NQF, av = r / NQF, q = r - av * NQF;
      const double* B = (side ? B1 : B0) + q * NB;
      const double* rc = sR + side * 3 * NB + av * NB;
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < NB; ++m) acc += B[m] * rc[m];
      sRq[t] = acc * (side ? is1 : is0);
    }
    __syncthreads();
    for (int q = tid; q < NQF; q += nt) {
      const double* T0 = sT;
      const double* T1 = sT + 13 * NQF;
      double uL[3] = {T0[0 * NQF + q], T0[1 * NQF + q], T0[2 * NQF + q]};
      double uR[3] = {T1[0 * NQF + q], T1[1 * NQF + q], T1[2 * NQF + q]};
      const double pL = T0[3 * NQF + q], pR = T1[3 * NQF + q];
      double Fc[4];
      if (MODE == MODE_TAN) {
        const double* Jq = a.dFlux + ((size_t)f * NQF + q) * 32;
        const double ds[8] = {uL[0], uL[1], uL[2], pL, uR[0], uR[1], uR[2], pR};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          double acc = 0.0;
#pragma unroll
          for (int j = 0; j < 8; ++j) acc += Jq[i * 8 + j] * ds[j];
          Fc[i] = acc;
        }
      } else if (MODE == MODE_RES_LIN) {
        double Jm[4][8];
        ac_riemann(uL, pL, uR, pR, d, a.c, Fc, Jm, a.status);
        double* Jq = a.dFlux + ((size_t)f * NQF + q) * 32;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) Jq[i * 8 + j] = Jm[i][j];
      } else {
        ac_riemann(uL, pL, uR, pR, d, a.c, Fc, nullptr, a.status);
      }
      double Gh[3][3];
#pragma unroll
      for (int av = 0; av < 3; ++av)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          Gh[av][b] = 0.5 * (T0[(4 + av * 3 + b) * NQF + q] + T1[(4 + av * 3 + b) * NQF + q]);
          if (b == d) Gh[av][b] -= a.eta * 0.5 * (sRq[av * NQF + q] + sRq[3 * NQF + av * NQF + q]);
        }
      const double trG = Gh[0][0] + Gh[1][1] + Gh[2][2];
      const double wq = sW[q] * A4;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double fv = a.nu * (Gh[i][d] + Gh[d][i]) - (i == d ? (2.0 / 3.0) * a.nu * trG : 0.0);
        sFn[i * NQF + q] = (Fc[i] - fv) * wq;
      }
      sFn[3 * NQF + q] = Fc[3] * wq;
    }
    __syncthreads();
    for (int t = tid; t < 8 * NB; t += nt) {
      const int side = t / (4 * NB), r = t - side * 4 * NB, i = r / NB, m = r - i * NB;
      const double* B = side ? B1 : B0;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NQF; ++q) acc += B[q * NB + m] * sFn[i * NQF + q];
      const int el = side ? e1 : e0, slot = side ? 2 * d : 2 * d + 1;
      a.face_out[((size_t)el * 6 + slot) * 4 * NB + r] = side ? -acc * is1 : acc * is0;
    }
    for (int t = tid; t < 6 * NB; t += nt) {
      const int side = t / (3 * NB), r = t - side * 3 * NB;
      const int el = side ? e1 : e0, slot = side ? 2 * d : 2 * d + 1;
      a.face_lift[((size_t)el * 6 + slot) * 3 * NB + r] = sR[t];
    }
    __syncthreads();
  }
}

// -------------------------------------------------------------- volume pass
template <int K, int MODE>
__global__ void __launch_bounds__(128) vol_kernel(OpArgs a) {
  using S = Sz<K>;
  constexpr int NB = S::NB, NQ = S::NQ;
  extern __shared__ double sm[];
  double* sB = sm;              // [NQ][NB]
  double* sW = sB + NQ * NB;    // [NQ]
  double* sC = sW + NQ;         // [4][NB]
  double* sG = sC + 4 * NB;     // [9][NB]
  double* sV = sG + 9 * NB;     // [13][NQ]
  double* sF = sV + 13 * NQ;    // [12][NQ] weighted flux, index p*4+i
  double* sP = sF + 12 * NQ;    // [12][NB]
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < NQ * NB; t += nt) sB[t] = a.Bvol[t];
  for (int t = tid; t < NQ; t += nt) sW[t] = a.wvol[t];
  __syncthreads();
  for (int e = blockIdx.x; e < a.M.ne; e += gridDim.x) {
    const ElemGeom g = elem_geom(a.M, e);
    const double is = 1.0 / g.s;
    const double Jd[3] = {2.0 / g.h[0], 2.0 / g.h[1], 2.0 / g.h[2]};
    for (int t = tid; t < 4 * NB; t += nt) sC[t] = a.in[(size_t)e * 4 * NB + t];
    __syncthreads();
    // corrected gradient coefficients (grad u - R^K(u))_{ab}, R^K = liftings of the six faces
    for (int t = tid; t < 9 * NB; t += nt) {
      const int ab = t / NB, m = t - ab * NB, av = ab / 3, b = ab - 3 * av;
      const double* cv = sC + av * NB;
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < Tables::kDw; ++j) {
        const int o = (b * NB + m) * Tables::kDw + j;
        acc += a.Drow_val[o] * cv[a.Drow_idx[o]];
      }
      const double* L = a.face_lift + (size_t)e * 6 * 3 * NB;
      sG[t] = acc * Jd[b] - (L[(2 * b) * 3 * NB + av * NB + m] + L[(2 * b + 1) * 3 * NB + av * NB + m]);
    }
    __syncthreads();
    for (int t = tid; t < 13 * NQ; t += nt) {
      const int fld = t / NQ, q = t - fld * NQ;
      const double* cf = fld < 4 ? sC + fld * NB : sG + (fld - 4) * NB;
      const double* B = sB + q * NB;
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < NB; ++m) acc += B[m] * cf[m];
      sV[t] = acc * is;
    }
    __syncthreads();
    for (int q = tid; q < NQ; q += nt) {
      const double u[3] = {sV[0 * NQ + q], sV[1 * NQ + q], sV[2 * NQ + q]};
      const double p = sV[3 * NQ + q];
      double G[3][3];
#pragma unroll
      for (int av = 0; av < 3; ++av)
#pragma unroll
        for (int b = 0; b < 3; ++b) G[av][b] = sV[(4 + av * 3 + b) * NQ + q];
      const double trG = G[0][0] + G[1][1] + G[2][2];
      double ub[3];
      if (MODE == MODE_TAN) {
#pragma unroll
        for (int c = 0; c < 3; ++c) ub[c] = a.ubar[((size_t)e * 3 + c) * NQ + q];
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) ub[c] = u[c];
        if (MODE == MODE_RES_LIN) {
#pragma unroll
          for (int c = 0; c < 3; ++c) a.ubar[((size_t)e * 3 + c) * NQ + q] = u[c];
        }
      }
      const double wq = sW[q];
#pragma unroll
      for (int pp = 0; pp < 3; ++pp) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const double fv = a.nu * (G[i][pp] + G[pp][i]) - (pp == i ? (2.0 / 3.0) * a.nu * trG : 0.0);
          // residual: u_p u_i; tangent: du_p ub_i + ub_p du_i
          const double conv = (MODE == MODE_TAN) ? (u[pp] * ub[i] + ub[pp] * u[i]) : u[pp] * u[i];
          sF[(pp * 4 + i) * NQ + q] = (conv + (pp == i ? p : 0.0) - fv) * wq;
        }
        sF[(pp * 4 + 3) * NQ + q] = u[pp] * wq;
      }
    }
    __syncthreads();
    for (int t = tid; t < 12 * NB; t += nt) {
      const int j = t / NB, n = t - j * NB;
      const double* F = sF + j * NQ;
      double acc = 0.0;
#pragma unroll 5
      for (int q = 0; q < NQ; ++q) acc += sB[q * NB + n] * F[q];
      sP[t] = acc * g.s;
    }
    __syncthreads();
    for (int t = tid; t < 4 * NB; t += nt) {
      const int i = t / NB, m = t - i * NB;
      double acc = 0.0;
#pragma unroll
      for (int pp = 0; pp < 3; ++pp) {
        double s2 = 0.0;
#pragma unroll
        for (int j = 0; j < Tables::kDw; ++j) {
          const int o = (pp * NB + m) * Tables::kDw + j;
          s2 += a.Dcol_val[o] * sP[(pp * 4 + i) * NB + a.Dcol_idx[o]];
        }
        acc += Jd[pp] * s2;
      }
      const double* FO = a.face_out + (size_t)e * 6 * 4 * NB + i * NB + m;
      double v = -acc;
#pragma unroll
      for (int s = 0; s < 6; ++s) v += FO[s * 4 * NB];
      if (MODE == MODE_TAN && i < 3) v += a.inv_gdt * sC[t];
      a.out[(size_t)e * 4 * NB + t] = v;
    }
    __syncthreads();
  }
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

// ------------------------------------------------------------- FD helpers
__global__ void fd_perturb_kernel(long long n, const double* w, const double* v, const double* wnorm2,
                                  const double* vnorm2, double* out) {
  const double nv = sqrt(*vnorm2);
  const double delta = nv > 0.0 ? 1e-9 * sqrt(1.0 + sqrt(*wnorm2)) / nv : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = w[i] + delta * v[i];
}
__global__ void fd_finish_kernel(long long n, int nb, const double* f1, const double* f0, const double* v,
                                 const double* wnorm2, const double* vnorm2, double inv_gdt, double* out) {
  const double nv = sqrt(*vnorm2);
  const double delta = nv > 0.0 ? 1e-9 * sqrt(1.0 + sqrt(*wnorm2)) / nv : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int var = (int)((i / nb) & 3);
    const double mass = var < 3 ? inv_gdt * v[i] : 0.0;
    out[i] = (delta > 0.0 ? (f1[i] - f0[i]) / delta : 0.0) + mass;
  }
}

// ------------------------------------------------------------- launchers
template <int K>
static size_t face_smem() {
  using S = Sz<K>;
  return sizeof(double) * (6 * S::NQF * S::NB + 8 * S::NB + 18 * S::NB + 26 * S::NQF + 6 * S::NB + 6 * S::NQF +
                           4 * S::NQF + S::NQF);
}
template <int K>
static size_t vol_smem() {
  using S = Sz<K>;
  return sizeof(double) * (S::NQ * S::NB + S::NQ + 4 * S::NB + 9 * S::NB + 13 * S::NQ + 12 * S::NQ + 12 * S::NB);
}

static OpArgs make_args(Handle* h, const double* in, double* out) {
  OpArgs a;
  a.M = mesh_dev(h);
  a.Bvol = h->tab.Bvol;
  a.wvol = h->tab.wvol;
  a.Bface = h->tab.Bface;
  a.wface = h->tab.wface;
  a.Drow_idx = h->tab.Drow_idx;
  a.Drow_val = h->tab.Drow_val;
  a.Dcol_idx = h->tab.Dcol_idx;
  a.Dcol_val = h->tab.Dcol_val;
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
  return a;
}

template <int K, int MODE>
static int run_operator(Handle* h, const OpArgs& a, cudaStream_t st) {
  const size_t fs = face_smem<K>(), vs = vol_smem<K>();
  DG_CUDA(h, cudaFuncSetAttribute(face_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs));
  DG_CUDA(h, cudaFuncSetAttribute(vol_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vs));
  const int nfaces = 3 * h->ne;
  const int per_sm_f = (int)(200 * 1024 / fs) < 8 ? (int)(200 * 1024 / fs) : 8;
  const int per_sm_v = (int)(200 * 1024 / vs) < 8 ? (int)(200 * 1024 / vs) : 8;
  int gf = h->nsm * (per_sm_f > 0 ? per_sm_f : 1);
  int gv = h->nsm * (per_sm_v > 0 ? per_sm_v : 1);
  if (gf > nfaces) gf = nfaces;
  if (gv > h->ne) gv = h->ne;
  const int cf = MODE == MODE_TAN ? DG_PROF_FACE_TAN : DG_PROF_FACE_RES;
  const int cv = MODE == MODE_TAN ? DG_PROF_VOL_TAN : DG_PROF_VOL_RES;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc;
  if ((rc = prof_begin(h, st, &e0))) return rc;
  face_kernel<K, MODE><<<gf, 128, fs, st>>>(a);
  DG_LAUNCH_CHECK(h);
  if ((rc = prof_end(h, cf, st, e0))) return rc;
  if ((rc = prof_begin(h, st, &e1))) return rc;
  vol_kernel<K, MODE><<<gv, 128, vs, st>>>(a);
  DG_LAUNCH_CHECK(h);
  if ((rc = prof_end(h, cv, st, e1))) return rc;
  ++h->op_apps;
  return DG_OK;
}

template <int MODE>
static int dispatch(Handle* h, const OpArgs& a, cudaStream_t st) {
  switch (h->tab.k) {
    case 1: return run_operator<1, MODE>(h, a, st);
    case 2: return run_operator<2, MODE>(h, a, st);
    case 3: return run_operator<3, MODE>(h, a, st);
    case 4: return run_operator<4, MODE>(h, a, st);
  }
  return fail(h, DG_ERR_ARG, "unsupported degree");
}

int op_residual(Handle* h, const double* w, double* f, bool store_lin, cudaStream_t st) {
  OpArgs a = make_args(h, w, f);
  return store_lin ? dispatch<MODE_RES_LIN>(h, a, st) : dispatch<MODE_RES>(h, a, st);
}

int op_tangent(Handle* h, const double* v, double* out, cudaStream_t st) {
  OpArgs a = make_args(h, v, out);
  return dispatch<MODE_TAN>(h, a, st);
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
                                           h->inv_gdt, out);
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
// coefficients of the face pass (N_e * 6 * (4 + 3) * N_b doubles), in a
// file-scope device array instead of the handle's own buffers. Every GPU that
// loads the library holds it until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[DG_NOALLOC_SCRATCH_DOUBLES];

// Device address of g_noalloc_scratch on the current device, looked up once per
// device. In host code the array's name is only a host-side stand-in, never a
// device address, so it must not be passed to a kernel.
static int noalloc_scratch(Handle* h, double** out) {
  static std::mutex mu;
  static double* addr[64] = {};
  int dev = 0;
  DG_CUDA(h, cudaGetDevice(&dev));
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
  const int nb = h->lev[0].nb;
  const long long need = (long long)h->ne * 6 * 7 * nb;
  if (need > (long long)DG_NOALLOC_SCRATCH_DOUBLES)
    return fail(h, DG_ERR_ARG,
                "mesh too large for the static scratch of dg_residual_noalloc: it needs N_e*42*N_b = " +
                    std::to_string(need) + " doubles, the limit is " + std::to_string(DG_NOALLOC_SCRATCH_DOUBLES));
  double* scratch = nullptr;
  int rc = noalloc_scratch(h, &scratch);
  if (rc) return rc;
  OpArgs a = make_args(h, w, f);
  a.face_out = scratch;
  a.face_lift = scratch + (size_t)h->ne * 6 * 4 * nb;
  return dispatch<MODE_RES>(h, a, as_stream(stream));
}
