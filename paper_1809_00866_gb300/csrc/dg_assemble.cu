// Preconditioner assembly at the current linearisation (Sec. 2.3-2.4):
//  * the state-independent linear part of J (viscous and BR2 terms, pressure
//    gradient, continuity) is probed once per handle with unit vectors on the
//    elements of one colour: a distance-1 colouring (no two face neighbours share
//    a colour) for the element diagonal blocks, a distance-2 colouring (no element
//    has two face neighbours of one colour) for the off-diagonal blocks at the
//    degree of level 1 (Sec. 2.4.3: coarse off-diagonal blocks are built at the
//    coarse degree);
//  * the state-dependent part (convective volume term, Riemann face terms) and
//    the mass shift are assembled directly per element at every call;
//  * inherited operators of every coarser level by sub-block extraction
//    (Eq. (GalProj) with a hierarchical orthonormal basis);
//  * LU factors with partial pivoting of all diagonal blocks (element-wise block
//    Jacobi), one block per CTA in shared memory.
// Blocks are stored column-major: block[c * b + r] = G[row r][col c].
#include <algorithm>
#include <vector>

#include "dg_internal.h"

namespace dg {

// ------------------------------------------------ direct state-dependent assembly
// J = J_lin + J_state. J_lin (viscous and BR2 terms, pressure gradient, continuity)
// depends on the mesh only; its blocks are probed once per handle (MODE_LINPART).
// J_state is assembled here per element from the cached linearisation:
//  * convective volume term: -int (u_p u_i)' d_p phi_m with weighted mass matrices
//    U_c[n'][n] = sum_q w_q ubar_c(q) phi_hat_n'(q) phi_hat_n(q) (|K|/8 / s^2 = 1):
//    A[i,m; j,n] = -J_j (D_j^T U_i)[m][n] - delta_ij sum_p J_p (D_p^T U_p)[m][n];
//  * Riemann face terms: with the cached flux Jacobian dF_i/ds_j at the face points
//    and phi_m on a face = P_hat_a(+-1) B2[q][n2(m)] / s, each face adds
//    sign * A4/(s s') P_hat_a(side) P_hat_a'(side') E_ij[n2(m)][n2(n)],
//    E_ij = sum_q w2_q dF_i/ds_j(q) B2[q][n2] B2[q][n2'].
// Diagonal blocks use the own side's columns of the Jacobian; the level-1 off-diagonal
// blocks the other side's, restricted to the coarse modes.
template <int K, class R = double>
struct AsmSmem {
  static constexpr int NB = nb_of(K), N1 = K + 1, NQ = N1 * N1 * N1, NQF = N1 * N1, N2 = (K + 1) * (K + 2) / 2;
  static constexpr int N2C = K * (K + 1) / 2;   // 2D modes of a coarser level (degree <= K - 1)
  static constexpr int B = 0;                   // [NQ][NB]
  static constexpr int UB = B + NQ * NB;        // [3][NQ] w_q ubar_c(q)
  static constexpr int U = UB + 3 * NQ;         // [3][NB][NB]
  static constexpr int E = U + 3 * NB * NB;     // [4 j][6 slot][N2][N2] face matrices of one row variable i
  static constexpr int JQ = E + 24 * N2 * N2;   // [2 buffers][2 own/other][6 slot][NQF][4 j] weighted Jacobian entries
  static constexpr int B2 = JQ + 2 * 2 * 6 * NQF * 4;  // [NQF][N2]
  static constexpr int W2 = B2 + NQF * N2;      // [NQF]
  static constexpr int PVN = W2 + NQF;          // [6 slot][NB] P_hat_a(side) of mode n's exponent along the slot's axis
  static constexpr int SLOT = PVN + 6 * NB;     // [6] scale of the slot's off-diagonal block
  // last, sized for the coarse degree of the handle (n2c 2D modes): [6 slot][4 j][n2c][n2c] the
  // face matrices with the other side's columns; the ints follow it
  static constexpr int EO = SLOT + 6;
  __host__ __device__ static constexpr int doubles(int n2c) { return EO + 24 * n2c * n2c; }
  static constexpr int FMN = 0;                 // [6 slot][NB] 2D mode of mode n on the slot's face
  static constexpr int PVO = FMN + 6 * NB;      // [6 slot][NB] index of P_hat_a(other side) of mode n (into pv)
  static constexpr int SINFO = PVO + 6 * NB;    // [6][3] face index, neighbour, target slot
  static constexpr int INTS = SINFO + 18;
  __host__ __device__ static constexpr size_t bytes(int n2c) { return sizeof(R) * doubles(n2c) + sizeof(int) * INTS; }
};

template <class R>
struct AsmArgs {
  MeshDev M;
  Tables T;
  const R* Bvol;       // tables in the assembly precision
  const R* wvol;
  const R* B2;
  const R* W2;
  const R* pv;
  const R* Dcol_val;
  const R* ubar;       // linearisation cache in the assembly precision
  const R* dFlux;
  const double* Dlin;  // level 0 linear-part diagonal blocks (FP64, probed once)
  R* D;                // level 0 diagonal blocks (output)
  const double* Blin;  // level 1 linear-part off-diagonal blocks (FP64)
  R* Bsr;              // level 1 block rows (output, slots 1..6)
  int nb1;             // modes per variable on level 1 (0: no coarse level)
  double inv_gdt;
};

template <int K, class R>
__global__ void __launch_bounds__(256) assemble_state_kernel(AsmArgs<R> a) {
  using L = AsmSmem<K, R>;
  constexpr int NB = L::NB, NQ = L::NQ, NQF = L::NQF, N2 = L::N2, K1 = K + 1, BS = 4 * NB, DW = Tables::kDw;
  constexpr int NDT = 4 * NB;  // diagonal-block tasks (j, m) of one row variable
  extern __shared__ __align__(16) unsigned char smraw_[];
  R* sm = reinterpret_cast<R*>(smraw_);
  R* sB = sm + L::B;
  R* sUb = sm + L::UB;
  R* sU = sm + L::U;
  R* sE = sm + L::E;
  R* sEo = sm + L::EO;
  R* sJ = sm + L::JQ;
  R* sB2 = sm + L::B2;
  R* sW2 = sm + L::W2;
  R* PVN = sm + L::PVN;
  R* sScl = sm + L::SLOT;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nb1 = a.nb1, b1 = 4 * nb1;
  // coarse 2D modes: the graded 2D ordering lists the modes of degree <= k_1 first
  int k1 = 0;
  while (nb1 > 0 && nb_of(k1) < nb1) ++k1;
  const int N2c = nb1 > 0 ? (k1 + 1) * (k1 + 2) / 2 : 0;  // <= L::N2C: the coarse degree is below K
  int* ism = reinterpret_cast<int*>(sm + L::doubles(N2c));
  int* FMN = ism + L::FMN;
  int* PVO = ism + L::PVO;
  int* SI = ism + L::SINFO;  // per slot: face index, neighbour (-1 at a wall), target block slot
  for (int t = tid; t < NQ * NB; t += nt) sB[t] = a.Bvol[t];
  for (int t = tid; t < NQF * N2; t += nt) sB2[t] = a.B2[t];
  for (int t = tid; t < NQF; t += nt) sW2[t] = a.W2[t];
  // per slot sl (face normal d = sl / 2, the element on side 1 of slot 2d and side 0 of slot 2d+1)
  // and mode n: P_hat of n's exponent along d on the element's side, its 2D face mode, and the
  // index of P_hat on the other side
  for (int t = tid; t < 6 * NB; t += nt) {
    const int sl = t / NB, n = t - sl * NB, d = sl >> 1, side = (sl & 1) ? 0 : 1;
    PVN[t] = a.pv[side * K1 + a.T.fa[d * NB + n]];
    PVO[t] = (1 - side) * K1 + a.T.fa[d * NB + n];
    FMN[t] = a.T.fmap[d * NB + n];
  }
  __syncthreads();
  for (int e = blockIdx.x; e < a.M.ne; e += gridDim.x) {
    const ElemGeom g = elem_geom(a.M, e);
    const R Jd[3] = {R(g.J[0]), R(g.J[1]), R(g.J[2])};
    // Jd at a run-time index through selects (no local-memory copy of the array)
    auto jd = [&](int c) { return c == 0 ? Jd[0] : (c == 1 ? Jd[1] : Jd[2]); };
    // the weighted Jacobian entries (i, j) of the six face slots at the face points: the own
    // side's columns (diagonal block) and the other side's (off-diagonal block); buffer i & 1
    auto load_jac = [&](int i) {
      R* dst = sJ + (i & 1) * 2 * 6 * NQF * 4;
      for (int t = tid; t < 2 * 6 * NQF * 4; t += nt) {
        const int oth = t / (6 * NQF * 4), r = t - oth * 6 * NQF * 4, sl = r / (NQF * 4), r2 = r - sl * NQF * 4;
        const int q = r2 >> 2, j = r2 & 3, d = sl >> 1, side = (sl & 1) ? 0 : 1;
        const int nb_ = a.M.nbr[e * 6 + sl];
        R v = R(0);
        if (!oth) {
          const int f = side == 0 ? 3 * e + d : (nb_ >= 0 ? 3 * nb_ + d : 3 * a.M.ne + a.M.bslot[e]);
          const R* Jq = a.dFlux + ((size_t)f * NQF + q) * 32 + i * 8;
          v = Jq[(side == 0 ? 0 : 4) + j];
          // at a wall the ghost state (-u_K, p_K) is the element's own: its columns add with
          // sign -1 (velocity) and +1 (pressure)
          if (nb_ < 0) v += (j == 3 ? R(1) : -R(1)) * Jq[(side == 0 ? 4 : 0) + j];
        } else if (nb_ >= 0 && nb1 > 0) {
          const int f = side == 0 ? 3 * e + d : 3 * nb_ + d;
          v = a.dFlux[((size_t)f * NQF + q) * 32 + i * 8 + (side == 0 ? 4 : 0) + j];
        }
        dst[t] = v * sW2[q];
      }
    };
    for (int t = tid; t < 3 * NQ; t += nt) {
      const int q = t % NQ;
      sUb[t] = a.wvol[q] * a.ubar[(size_t)e * 3 * NQ + t];
    }
    if (tid < 6) {
      const int sl = tid, d = sl >> 1, side = (sl & 1) ? 0 : 1;
      const int p = a.M.nbr[e * 6 + sl];
      int tgt = sl;
      for (int s2 = 0; s2 < sl; ++s2)
        if (a.M.nbr[e * 6 + s2] == p) { tgt = s2; break; }
      SI[3 * sl + 0] = side == 0 ? 3 * e + d : (p >= 0 ? 3 * p + d : -1);
      SI[3 * sl + 1] = p;
      SI[3 * sl + 2] = tgt;
      R sc = R(0);
      if (p >= 0) {
        const ElemGeom gp = elem_geom(a.M, p);
        const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        auto h3 = [&](int c) { return c == 0 ? g.h[0] : (c == 1 ? g.h[1] : g.h[2]); };  // no local memory
        sc = R((side == 0 ? 1.0 : -1.0) * 0.25 * h3(t1) * h3(t2) * g.is * gp.is);
      }
      sScl[sl] = sc;
    }
    load_jac(0);
    __syncthreads();
    // weighted mass matrices U_c (symmetric): one thread per mode pair n1 <= n computes all three
    // c, so the two basis values of a point are loaded once
    for (int t = tid; t < NB * (NB + 1) / 2; t += nt) {
      int n1 = 0, r = t;
      while (r >= NB - n1) { r -= NB - n1; ++n1; }
      const int n = n1 + r;
      R acc[3] = {R(0), R(0), R(0)};
      for (int q = 0; q < NQ; ++q) {
        const R bb = sB[q * NB + n1] * sB[q * NB + n];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] += sUb[c * NQ + q] * bb;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sU[(c * NB + n1) * NB + n] = acc[c];
        sU[(c * NB + n) * NB + n1] = acc[c];
      }
    }
    for (int i = 0; i < 4; ++i) {
      // face matrices of row variable i: E[j][sl] = sum_q w_q dF_ij(q) B2[q][j1] B2[q][j2], symmetric
      // in (j1, j2): threads [0, ntE) take one 2D mode pair j1 <= j2 each (all 4 j and 6 slots;
      // the four j of a point are one vector) and write both halves; the threads after them
      // form the other side's matrices for the coarse 2D modes, symmetric as well
      const R* Jo = sJ + (i & 1) * 2 * 6 * NQF * 4;  // own columns [6][NQF][4]
      const R* Jx = Jo + 6 * NQF * 4;                 // other side's columns
      constexpr int NPE = N2 * (N2 + 1) / 2;
      const int ntE = NPE < nt - 32 ? NPE : nt - 32;
      const int NPc = N2c * (N2c + 1) / 2;
      if (tid < ntE) {
        for (int t = tid; t < NPE; t += ntE) {
          int j1 = 0, r = t;
          while (r >= N2 - j1) { r -= N2 - j1; ++j1; }
          const int j2 = j1 + r;
          R acc[4][6];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int sl = 0; sl < 6; ++sl) acc[j][sl] = R(0);
#pragma unroll 5
          for (int q = 0; q < NQF; ++q) {
            const R bb = sB2[q * N2 + j1] * sB2[q * N2 + j2];
#pragma unroll
            for (int sl = 0; sl < 6; ++sl) {
              const R* jv = Jo + (sl * NQF + q) * 4;
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[j][sl] += jv[j] * bb;
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int sl = 0; sl < 6; ++sl) {
              R* Ejs = sE + (j * 6 + sl) * N2 * N2;
              Ejs[j1 * N2 + j2] = acc[j][sl];
              Ejs[j2 * N2 + j1] = acc[j][sl];
            }
        }
      } else {
        for (int t = tid - ntE; t < 6 * 4 * NPc; t += nt - ntE) {
          const int sl = t / (4 * NPc), r0 = t - sl * 4 * NPc, j = r0 / NPc;
          int j1 = 0, r = r0 - j * NPc;
          while (r >= N2c - j1) { r -= N2c - j1; ++j1; }
          const int j2 = j1 + r;
          R acc = R(0);
#pragma unroll 5
          for (int q = 0; q < NQF; ++q) acc += Jx[(sl * NQF + q) * 4 + j] * (sB2[q * N2 + j1] * sB2[q * N2 + j2]);
          R* Eo = sEo + (sl * 4 + j) * N2c * N2c;
          Eo[j1 * N2c + j2] = acc;
          Eo[j2 * N2c + j1] = acc;
        }
      }
      __syncthreads();
      if (i < 3) load_jac(i + 1);  // the other buffer, read after the next barrier
      if constexpr (sizeof(R) == 4) {
        // FP32: one thread per (j, n, m) over the whole CTA, so that many loads of the probed
        // linear part are in flight (the FP32 assembly waits on memory, not on its arithmetic)
        R* Dout = a.D + (size_t)e * BS * BS;
        const double* Dl = a.Dlin + (size_t)e * BS * BS;
#pragma unroll 4
        for (int t = tid; t < 4 * NB * NB; t += nt) {
          const int j = t / (NB * NB), r = t - j * NB * NB, n = r / NB, m = r - n * NB;
          R v = R(__ldg(Dl + (size_t)(j * NB + n) * BS + i * NB + m));
          if (i == j && i < 3 && m == n) v += R(a.inv_gdt * g.sh);
          if (i < 3 && j < 3) {
            // -J_j (D_j^T U_i)[m][n] - delta_ij sum_p J_p (D_p^T U_p)[m][n]
            R cv = R(0);
#pragma unroll
            for (int q = 0; q < DW; ++q) {
              const int o = (j * NB + m) * DW + q;
              cv += a.Dcol_val[o] * sU[(i * NB + a.T.Dcol_idx[o]) * NB + n];
            }
            v -= jd(j) * cv;
            if (i == j) {
#pragma unroll
              for (int pp = 0; pp < 3; ++pp) {
                R c2 = R(0);
#pragma unroll
                for (int q = 0; q < DW; ++q) {
                  const int o = (pp * NB + m) * DW + q;
                  c2 += a.Dcol_val[o] * sU[(pp * NB + a.T.Dcol_idx[o]) * NB + n];
                }
                v -= Jd[pp] * c2;
              }
            }
          }
#pragma unroll
          for (int sl = 0; sl < 6; ++sl) {
            const int d = sl >> 1;
            const R scale = ((sl & 1) ? R(1) : -R(1)) * Jd[d];  // A4 / s^2 = 2 / h_d, sign of the side
            v += scale * PVN[sl * NB + m] * PVN[sl * NB + n] *
                 sE[((j * 6 + sl) * N2 + FMN[sl * NB + m]) * N2 + FMN[sl * NB + n]];
          }
          Dout[(size_t)(j * NB + n) * BS + i * NB + m] = v;
        }
        if (nb1 > 0)
          for (int t = tid; t < 6 * 4 * nb1 * nb1; t += nt) {
            const int so = t / (4 * nb1 * nb1), r = t - so * 4 * nb1 * nb1, j = r / (nb1 * nb1), r2 = r - j * nb1 * nb1;
            const int n = r2 / nb1, m = r2 - n * nb1;
            const size_t o = (size_t)(j * nb1 + n) * b1 + i * nb1 + m;
            R* blk = a.Bsr + ((size_t)e * 7 + 1 + so) * b1 * b1;
            if (SI[3 * so + 1] < 0 || SI[3 * so + 2] != so) {
              blk[o] = R(0);
              continue;
            }
            R v = R(a.Blin[((size_t)e * 7 + 1 + so) * b1 * b1 + o]);
            for (int sl = so; sl < 6; ++sl) {
              if (SI[3 * sl + 1] < 0 || SI[3 * sl + 2] != so) continue;
              v += sScl[sl] * PVN[sl * NB + m] * a.pv[PVO[sl * NB + n]] *
                   sEo[((sl * 4 + j) * N2c + FMN[sl * NB + m]) * N2c + FMN[sl * NB + n]];
            }
            blk[o] = v;
          }
      } else if (tid < NDT) {
        // the diagonal block's rows of variable i: one thread per (j, m), all columns n
        const int j = tid / NB, m = tid - j * NB;
        R* Dout = a.D + (size_t)e * BS * BS + i * NB + m;
        const double* Dl = a.Dlin + (size_t)e * BS * BS + i * NB + m;
        R pm[6];
        int fm[6];
#pragma unroll
        for (int sl = 0; sl < 6; ++sl) {
          const int d = sl >> 1, side = (sl & 1) ? 0 : 1;
          pm[sl] = (side == 0 ? R(1) : -R(1)) * Jd[d] * PVN[sl * NB + m];  // A4 / s^2 = 2 / h_d
          fm[sl] = ((j * 6 + sl) * N2 + FMN[sl * NB + m]) * N2;
        }
        // -J_j (D_j^T U_i)[m][n] - delta_ij sum_p J_p (D_p^T U_p)[m][n]: rows of U the sparse
        // derivative picks for (j, m) and, on the diagonal pair, for every p
        const bool vol = i < 3 && j < 3;
        int ui[4][DW];
        R uv[4][DW];
#pragma unroll
        for (int pp = 0; pp < 4; ++pp)
#pragma unroll
          for (int q = 0; q < DW; ++q) {
            const int dj = pp < 3 ? pp : j;  // slot 3: the off-diagonal term -J_j (D_j^T U_i)
            const int ci = pp < 3 ? pp : i;
            const int o = (dj * NB + m) * DW + q;
            const bool use = vol && (pp == 3 || i == j);
            ui[pp][q] = use ? (ci * NB + a.T.Dcol_idx[o]) * NB : 0;
            uv[pp][q] = use ? -a.Dcol_val[o] * (pp < 3 ? jd(pp) : jd(j)) : R(0);
          }
        const R shift = R(a.inv_gdt * g.sh);
#pragma unroll 5
        for (int n = 0; n < NB; ++n) {
          R v = R(__ldg(Dl + (size_t)(j * NB + n) * BS));
          if (i == j && i < 3 && m == n) v += shift;
          if (vol) {
            R cv = R(0);
#pragma unroll
            for (int q = 0; q < DW; ++q) cv += uv[3][q] * sU[ui[3][q] + n];
            v += cv;
            if (i == j) {
#pragma unroll
              for (int pp = 0; pp < 3; ++pp) {
                R c2 = R(0);
#pragma unroll
                for (int q = 0; q < DW; ++q) c2 += uv[pp][q] * sU[ui[pp][q] + n];
                v += c2;
              }
            }
          }
#pragma unroll
          for (int sl = 0; sl < 6; ++sl) v += pm[sl] * PVN[sl * NB + n] * sE[fm[sl] + FMN[sl * NB + n]];
          Dout[(size_t)(j * NB + n) * BS] = v;
        }
      } else if (nb1 > 0) {
        // level-1 off-diagonal blocks, rows of variable i, coarse modes only: the linear part of
        // the slot plus the Riemann terms of every slot facing the same neighbour, in slot order
        // (a neighbour met on two faces keeps its block at the first slot; the other is zero; a
        // wall slot is zero)
        for (int t = tid - NDT; t < 6 * 4 * nb1 * nb1; t += nt - NDT) {
          const int so = t / (4 * nb1 * nb1), r = t - so * 4 * nb1 * nb1, j = r / (nb1 * nb1), r2 = r - j * nb1 * nb1;
          const int n = r2 / nb1, m = r2 - n * nb1;
          const size_t o = (size_t)(j * nb1 + n) * b1 + i * nb1 + m;
          R* blk = a.Bsr + ((size_t)e * 7 + 1 + so) * b1 * b1;
          if (SI[3 * so + 1] < 0 || SI[3 * so + 2] != so) {
            blk[o] = R(0);
            continue;
          }
          R v = R(a.Blin[((size_t)e * 7 + 1 + so) * b1 * b1 + o]);
          for (int sl = so; sl < 6; ++sl) {
            if (SI[3 * sl + 1] < 0 || SI[3 * sl + 2] != so) continue;
            v += sScl[sl] * PVN[sl * NB + m] * a.pv[PVO[sl * NB + n]] *
                 sEo[((sl * 4 + j) * N2c + FMN[sl * NB + m]) * N2c + FMN[sl * NB + n]];
          }
          blk[o] = v;
        }
      }
      __syncthreads();
    }
  }
}

template <int K, class R>
static int launch_assemble_state(Handle* h, const AsmArgs<R>& a, cudaStream_t st) {
  // the coarse face matrices are sized for the handle's level-1 degree
  const int n2c = a.nb1 > 0 ? (h->lev[1].k + 1) * (h->lev[1].k + 2) / 2 : 0;
  const size_t smem = AsmSmem<K, R>::bytes(n2c);
  DG_CUDA(h, cudaFuncSetAttribute(assemble_state_kernel<K, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = (int)((227 * 1024) / (smem + 1024));  // 1 KB of each CTA's shared memory is reserved
  int res = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, assemble_state_kernel<K, R>, 256, smem) == cudaSuccess &&
      res > 0 && res < per_sm)
    per_sm = res;
  per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
  int grid = h->nsm * per_sm;
  if (grid > h->ne) grid = h->ne;
  assemble_state_kernel<K, R><<<grid, 256, smem, st>>>(a);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

static std::vector<int> greedy_colouring(const Handle* h, int dist) {
  const int ne = h->ne;
  const std::vector<int>& nb6 = h->nbr_host;
  std::vector<int> col(ne, -1);
  if (dist == 2 && h->nprob == 1 && h->n[0] % 8 == 0 && h->n[1] % 8 == 0 && h->n[2] % 8 == 0) {
    // (i + 2j + 3k) mod 8: the six neighbour offsets +-1, +-2, +-3 are distinct and non-zero mod 8,
    // so no element shares a colour with a neighbour or with a neighbour's neighbour
    for (int e = 0; e < ne; ++e) {
      const int i = e % h->n[0], j = (e / h->n[0]) % h->n[1], k = e / (h->n[0] * h->n[1]);
      col[e] = (i + 2 * j + 3 * k) % 8;
    }
    return col;
  }
  std::vector<int> mark(64, -1);
  for (int e = 0; e < ne; ++e) {
    std::vector<int> around;
    for (int f = 0; f < 6; ++f) {
      const int p = nb6[e * 6 + f];
      if (p < 0) continue;  // a wall
      around.push_back(p);
      if (dist >= 2)
        for (int g = 0; g < 6; ++g)
          if (nb6[p * 6 + g] >= 0) around.push_back(nb6[p * 6 + g]);
    }
    for (int p : around)
      if (p != e && col[p] >= 0) mark[col[p]] = e;
    int c = 0;
    while (mark[c] == e) ++c;
    col[e] = c;
  }
  return col;
}

__global__ void probe_kernel(long long n, int b, const int* colour, int c, int j, double* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / b;
    const int r = (int)(i - e * b);
    v[i] = (colour[e] == c && r == j) ? 1.0 : 0.0;
  }
}

// Dblk[e][j][r] = out[e][r] for elements of colour c.
__global__ void scatter_diag_kernel(int ne, int b, const int* colour, int c, int j, const double* out, double* D) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)ne * b;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / b;
    const int r = (int)(i - e * b);
    if (colour[e] == c) D[(e * b + j) * b + r] = out[e * b + r];
  }
}

// For every element p and face slot f whose neighbour e = nbr[p][f] has colour c
// (and f is the first slot of p facing e): Bsr1[p][1+f][jc][rc] = out[p][fine row of rc].
__global__ void scatter_offdiag_kernel(int ne, int nb0, int nb1, const int* nbr, const int* colour, int c, int jc,
                                       const double* out, double* Bsr) {
  const int b1 = 4 * nb1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)ne * 6 * b1;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / (6 * b1);
    const int rem = (int)(i - p * 6 * b1), f = rem / b1, rc = rem - f * b1;
    const int e = nbr[p * 6 + f];
    if (e < 0 || colour[e] != c) continue;
    bool first = true;
    for (int g = 0; g < f; ++g)
      if (nbr[p * 6 + g] == e) first = false;
    if (!first) continue;
    const int var = rc / nb1, m = rc - var * nb1;
    Bsr[(((p * 7 + 1 + f) * (long long)b1) + jc) * b1 + rc] = out[(p * 4 + var) * nb0 + m];
  }
}

// Row-block probing: for every element p, slot 0 (p itself, when p has colour c) and each face
// slot f whose neighbour e = nbr[p][f] has colour c (first slot facing e only):
// A[p][slot][jc][rc] += sign * out[p][fine row of rc] (level-1 modes nb1 of nb0).
__global__ void scatter_rows_kernel(int ne, int nb0, int nb1, const int* nbr, const int* colour, int c, int jc,
                                    const double* out, double sign, double* A) {
  const int b1 = 4 * nb1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)ne * 7 * b1;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / (7 * b1);
    const int rem = (int)(i - p * 7 * b1), s = rem / b1, rc = rem - s * b1;
    const int e = s == 0 ? (int)p : nbr[p * 6 + s - 1];
    if (e < 0 || colour[e] != c) continue;
    if (s > 0) {
      bool first = true;
      for (int g = 0; g < s - 1; ++g)
        if (nbr[p * 6 + g] == e) first = false;
      if (!first || e == (int)p) continue;
    }
    const int var = rc / nb1, m = rc - var * nb1;
    A[(((p * 7 + s) * (long long)b1) + jc) * b1 + rc] += sign * out[(p * 4 + var) * nb0 + m];
  }
}

// Inherited coarse blocks (Eq. (GalProj) with a hierarchical orthonormal basis: the leading
// sub-block of every variable pair), with the rescaling of Appendix A: for the slots
// s = blockIdx.y of every element block, dst = sub(src) [+ coef * sub(stb)], where stb holds the
// level-1 stabilisation blocks (nb1 modes per variable) and src the finer blocks (nbs modes);
// dst2, if given, receives a second copy. src and dst may be the same blocks (an in-place add).
// One CTA row per slot, 32-bit index arithmetic within a block, arithmetic in R.
template <class R>
__global__ void inherit_kernel(int nblocks, int nbs, const R* src, long long src_blk, long long src_slot, int nbd,
                               R* dst, long long dst_blk, long long dst_slot, R* dst2, long long dst2_blk,
                               const R* __restrict__ stb, long long stb_blk, long long stb_slot, int nb1, R coef) {
  const int bs = 4 * nbs, bd = 4 * nbd, b1 = 4 * nb1, sl = blockIdx.y;
  for (int blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
    const R* sb = src + blk * src_blk + sl * src_slot;
    const R* tb = stb ? stb + blk * stb_blk + sl * stb_slot : nullptr;
    R* db = dst + blk * dst_blk + sl * dst_slot;
    R* d2 = dst2 ? dst2 + blk * dst2_blk : nullptr;
    for (int t = threadIdx.x; t < bd * bd; t += blockDim.x) {
      const int c = t / bd, r = t - c * bd;
      const int cv = c / nbd, cm = c - cv * nbd, rv = r / nbd, rm = r - rv * nbd;
      R v = sb[(cv * nbs + cm) * bs + rv * nbs + rm];
      if (tb) v += coef * tb[(cv * nb1 + cm) * b1 + rv * nb1 + rm];
      db[t] = v;
      if (d2) d2[t] = v;
    }
  }
}

// In-place LU factorisation with partial (row) pivoting of one b x b block per CTA in
// shared memory (row-major, padded leading dimension). Output, column-major per block:
// the unit-lower L below the diagonal, U above it, and 1/U_kk on the diagonal; and the
// row permutation pi (row i of P A is row pi[i] of A).
template <class R>
__global__ void __launch_bounds__(256) lu_factor_kernel(int nblk, int b, const R* in, R* out, int* perm,
                                                       unsigned* status) {
  extern __shared__ __align__(16) unsigned char smraw_[];
  R* sm = reinterpret_cast<R*>(smraw_);
  const int LD = b + 1;
  R* A = sm;                               // [b][LD]
  int* piv = reinterpret_cast<int*>(A + b * LD);  // [b] row swapped with k at step k
  __shared__ int s_piv;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const R* src = in + (size_t)blk * b * b;
    for (int t = tid; t < b * b; t += nt) {
      const int c = t / b, r = t - c * b;
      A[r * LD + c] = src[t];
    }
    __syncthreads();
    for (int k = 0; k < b; ++k) {
      if (warp == 0) {
        R best = R(-1);
        int bi = k;
        for (int i = k + lane; i < b; i += 32) {
          const R v = fabs(A[i * LD + k]);
          if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const R ov = __shfl_down_sync(0xffffffffu, best, off);
          const int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) {
          s_piv = bi;
          piv[k] = bi;
          if (!(best > R(0)) && status) atomicOr(status, (unsigned)DG_STATUS_NONFINITE);
        }
      }
      __syncthreads();
      const int p = s_piv;
      if (p != k)
        for (int j = tid; j < b; j += nt) {
          const R t = A[k * LD + j];
          A[k * LD + j] = A[p * LD + j];
          A[p * LD + j] = t;
        }
      __syncthreads();
      const R rk = R(1) / A[k * LD + k];
      for (int i = k + 1 + tid; i < b; i += nt) A[i * LD + k] *= rk;
      __syncthreads();
      // trailing update: warp w takes rows k+1+w, k+1+w+nw, ...; lanes take the columns
      for (int i = k + 1 + warp; i < b; i += nw) {
        const R l = A[i * LD + k];
        R* Ai = A + i * LD;
        const R* Ak = A + k * LD;
        for (int j = k + 1 + lane; j < b; j += 32) Ai[j] = fma(-l, Ak[j], Ai[j]);
      }
      if (tid == 0) A[k * LD + k] = rk;
      __syncthreads();
    }
    R* dst = out + (size_t)blk * b * b;
    for (int t = tid; t < b * b; t += nt) {
      const int c = t / b, r = t - c * b;
      dst[t] = A[r * LD + c];
    }
    if (tid == 0) {
      // compose the swaps into pi: apply them in order to the identity
      int* pi = perm + (size_t)blk * b;
      for (int i = 0; i < b; ++i) pi[i] = i;
      for (int kk = 0; kk < b; ++kk) {
        const int q = piv[kk];
        const int t = pi[kk];
        pi[kk] = pi[q];
        pi[q] = t;
      }
    }
    __syncthreads();
  }
}

template <class R>
static int factor_blocks(Handle* h, int nblk, int b, const R* in, R* out, int* perm, cudaStream_t st) {
  const size_t smem = sizeof(R) * (size_t)b * (b + 1) + sizeof(int) * b;
  DG_CUDA(h, cudaFuncSetAttribute(lu_factor_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = (int)((220 * 1024) / smem);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  int grid = h->nsm * per_sm;
  if (grid > nblk) grid = nblk;
  lu_factor_kernel<R><<<grid, 256, smem, st>>>(nblk, b, in, out, perm, h->status + 2);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// Blocks of the state-independent linear part of J (viscous and BR2 terms, pressure
// gradient, continuity), probed once per handle: element diagonal blocks on level 0 and
// the level-1 off-diagonal blocks.
static int probe_linear_part(Handle* h, cudaStream_t st) {
  const int ne = h->ne;
  Level& L0 = h->lev[0];
  const int b0 = L0.b;
  const int grid = h->nsm * 8;
  int rc;
  if (!h->colour) DG_CUDA(h, cudaMalloc((void**)&h->colour, sizeof(int) * ne));
  int* dcol = h->colour;
  double* probe = L0.t0;
  double* out = L0.t1;
  const std::vector<int> c1 = greedy_colouring(h, 1);
  const int nc1 = *std::max_element(c1.begin(), c1.end()) + 1;
  DG_CUDA(h, cudaMemcpyAsync(dcol, c1.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, st));
  for (int c = 0; c < nc1; ++c)
    for (int j = 0; j < b0; ++j) {
      probe_kernel<<<grid, 256, 0, st>>>(L0.n, b0, dcol, c, j, probe);
      DG_LAUNCH_CHECK(h);
      if ((rc = op_linear_part(h, probe, out, st))) return rc;
      scatter_diag_kernel<<<grid, 256, 0, st>>>(ne, b0, dcol, c, j, out, L0.Dlin);
      DG_LAUNCH_CHECK(h);
    }
  if (h->nlev > 1) {
    Level& L1 = h->lev[1];
    const int b1 = L1.b;
    DG_CUDA(h, cudaMemsetAsync(L1.Blin, 0, sizeof(double) * (size_t)b1 * b1 * 7 * ne, st));
    const std::vector<int> c2 = greedy_colouring(h, 2);
    const int nc2 = *std::max_element(c2.begin(), c2.end()) + 1;
    DG_CUDA(h, cudaMemcpyAsync(dcol, c2.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, st));
    for (int c = 0; c < nc2; ++c)
      for (int jc = 0; jc < b1; ++jc) {
        const int jf = (jc / L1.nb) * L0.nb + jc % L1.nb;
        probe_kernel<<<grid, 256, 0, st>>>(L0.n, b0, dcol, c, jf, probe);
        DG_LAUNCH_CHECK(h);
        if ((rc = op_linear_part(h, probe, out, st))) return rc;
        scatter_offdiag_kernel<<<grid, 256, 0, st>>>(ne, L0.nb, L1.nb, h->nbr, dcol, c, jc, out, L1.Blin);
        DG_LAUNCH_CHECK(h);
      }
  }
  return DG_OK;
}

// The stabilisation part of the level-1 block rows, G(eta) - G(0) probed with the linear part
// (the eta term is linear and state independent), distance-2 colouring.
static int probe_stb(Handle* h, cudaStream_t st) {
  const int ne = h->ne;
  Level& L0 = h->lev[0];
  Level& L1 = h->lev[1];
  const int b0 = L0.b, b1 = L1.b;
  const int grid = h->nsm * 8;
  int rc;
  if (!h->stb1) DG_CUDA(h, cudaMalloc((void**)&h->stb1, sizeof(double) * (size_t)b1 * b1 * 7 * ne));
  DG_CUDA(h, cudaMemsetAsync(h->stb1, 0, sizeof(double) * (size_t)b1 * b1 * 7 * ne, st));
  if (!h->colour) DG_CUDA(h, cudaMalloc((void**)&h->colour, sizeof(int) * ne));
  int* dcol = h->colour;
  double* probe = L0.t0;
  double* out = L0.t1;
  const std::vector<int> c2 = greedy_colouring(h, 2);
  const int nc2 = *std::max_element(c2.begin(), c2.end()) + 1;
  DG_CUDA(h, cudaMemcpyAsync(dcol, c2.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, st));
  const double eta = h->p.eta;
  for (int pass = 0; pass < 2; ++pass) {
    h->p.eta = pass == 0 ? eta : 0.0;
    for (int c = 0; c < nc2; ++c)
      for (int jc = 0; jc < b1; ++jc) {
        const int jf = (jc / L1.nb) * L0.nb + jc % L1.nb;
        probe_kernel<<<grid, 256, 0, st>>>(L0.n, b0, dcol, c, jf, probe);
        DG_LAUNCH_CHECK(h);
        if ((rc = op_linear_part(h, probe, out, st))) { h->p.eta = eta; return rc; }
        scatter_rows_kernel<<<grid, 256, 0, st>>>(ne, L0.nb, L1.nb, h->nbr, dcol, c, jc, out,
                                                  pass == 0 ? 1.0 : -1.0, h->stb1);
        DG_LAUNCH_CHECK(h);
      }
  }
  h->p.eta = eta;
  return DG_OK;
}

static int alloc_fp32_levels(Handle* h) {
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->lev[l];
    const size_t nbb = (size_t)h->ne * L.b * L.b;
    if (!L.LUf) DG_CUDA(h, cudaMalloc((void**)&L.LUf, sizeof(float) * nbb));
    if (!L.t0f) DG_CUDA(h, cudaMalloc((void**)&L.t0f, sizeof(float) * L.n));
    if (!L.t1f) DG_CUDA(h, cudaMalloc((void**)&L.t1f, sizeof(float) * L.n));
    if (!L.t2f) DG_CUDA(h, cudaMalloc((void**)&L.t2f, sizeof(float) * L.n));
    if (l >= 1 && !L.Bsrf) DG_CUDA(h, cudaMalloc((void**)&L.Bsrf, sizeof(float) * nbb * 7));
    if (!L.perm) DG_CUDA(h, cudaMalloc((void**)&L.perm, sizeof(int) * (size_t)h->ne * L.b));
  }
  return DG_OK;
}

template <class R>
static int assemble_levels(Handle* h, const AsmArgs<R>& a, R* const* Dlev, R* const* Bsrlev, const R* stb,
                           cudaStream_t st) {
  const int ne = h->ne;
  const int grid = h->nsm * 8;
  int rc;
  switch (h->tab.k) {
    case 1: rc = launch_assemble_state<1, R>(h, a, st); break;
    case 2: rc = launch_assemble_state<2, R>(h, a, st); break;
    case 3: rc = launch_assemble_state<3, R>(h, a, st); break;
    case 4: rc = launch_assemble_state<4, R>(h, a, st); break;
    default: rc = fail(h, DG_ERR_ARG, "unsupported degree");
  }
  if (rc) return rc;
  const Level& L0 = h->lev[0];
  const int b0 = L0.b;
  // coarse levels: inherited sub-blocks (taken before the fine blocks are factored in place);
  // with the rescaling of Appendix A, the stabilisation part of level l is weighted by S_0^l
  const int k0 = L0.k, nb1 = h->nlev > 1 ? h->lev[1].nb : 0, b1 = 4 * nb1;
  const R* sb = h->stb_rescale ? stb : nullptr;
  const long long s1 = (long long)b1 * b1;
  double s_prev = 1.0;
  for (int l = 1; l < h->nlev; ++l) {
    Level& L = h->lev[l];
    const long long bb = (long long)L.b * L.b;
    const double S = (double)(L.k * (L.k + 3)) / (double)(k0 * (k0 + 3));
    // diagonal: sub(D_0) [+ (S - 1) sub(stabilisation slot 0)], also slot 0 of the block row
    inherit_kernel<R><<<dim3(grid, 1), 256, 0, st>>>(ne, L0.nb, Dlev[0], (long long)b0 * b0, 0, L.nb, Dlev[l], bb, 0,
                                                   Bsrlev[l], bb * 7, sb, s1 * 7, s1, nb1, R(S - 1.0));
    DG_LAUNCH_CHECK(h);
    // off-diagonal slots: level 1's come from the state assembly (the add is in place), level
    // l >= 2 inherits level l - 1's; level 1 carries S - 1, level l >= 2 adds S - s_prev
    if (l >= 2 || sb) {
      const Level& P = h->lev[l == 1 ? 1 : l - 1];
      const long long pbb = (long long)P.b * P.b;
      inherit_kernel<R><<<dim3(grid, 6), 256, 0, st>>>(ne, P.nb, Bsrlev[l == 1 ? 1 : l - 1] + pbb, pbb * 7, pbb,
                                                     L.nb, Bsrlev[l] + bb, bb * 7, bb, nullptr, 0,
                                                     sb ? sb + s1 : nullptr, s1 * 7, s1, nb1,
                                                     R(l == 1 ? S - 1.0 : S - s_prev));
      DG_LAUNCH_CHECK(h);
    }
    s_prev = S;
  }
  return DG_OK;
}

__global__ void narrow_f32_kernel(long long n, const double* __restrict__ x, float* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void or_bits_kernel(unsigned* status, unsigned bits) { atomicOr(status, bits); }

int assemble_all(Handle* h, int precision, cudaStream_t st) {
  const int ne = h->ne;
  Level& L0 = h->lev[0];
  int rc;
  DG_CUDA(h, cudaMemsetAsync(h->status + 2, 0, sizeof(unsigned), st));  // this assembly's own status word
  // the linear part (FP64, mesh only) and the FP64 fine diagonal-block buffer it lives next to
  if (!L0.Dlin) DG_CUDA(h, cudaMalloc((void**)&L0.Dlin, sizeof(double) * (size_t)L0.b * L0.b * ne));
  if (h->nlev > 1 && !h->lev[1].Blin) {
    const size_t nbl = sizeof(double) * (size_t)h->lev[1].b * h->lev[1].b * 7 * ne;
    DG_CUDA(h, cudaMalloc((void**)&h->lev[1].Blin, nbl));
    DG_CUDA(h, cudaMemsetAsync(h->lev[1].Blin, 0, nbl, st));  // slots across a wall stay zero
  }
  if (!h->linpart_ready) {
    if ((rc = probe_linear_part(h, st))) return rc;
    h->linpart_ready = true;
  }
  if (h->stb_rescale && !h->stb_ready) {
    if ((rc = probe_stb(h, st))) return rc;
    h->stb_ready = true;
  }
  if (precision == DG_PRECOND_FP64) {
    for (int l = 0; l < h->nlev; ++l) {
      Level& L = h->lev[l];
      const size_t bb = (size_t)L.b * L.b;
      if (!L.Dblk) DG_CUDA(h, cudaMalloc((void**)&L.Dblk, sizeof(double) * bb * ne));
      if (!L.Dinv) DG_CUDA(h, cudaMalloc((void**)&L.Dinv, sizeof(double) * bb * ne));
      if (l >= 1 && !L.Bsr) DG_CUDA(h, cudaMalloc((void**)&L.Bsr, sizeof(double) * bb * 7 * ne));
      if (!L.perm) DG_CUDA(h, cudaMalloc((void**)&L.perm, sizeof(int) * (size_t)ne * L.b));
    }
    AsmArgs<double> a;
    a.M = mesh_dev(h);
    a.T = h->tab;
    a.Bvol = h->tab.Bvol; a.wvol = h->tab.wvol; a.B2 = h->tab.B2; a.W2 = h->tab.W2; a.pv = h->tab.pv;
    a.Dcol_val = h->tab.Dcol_val;
    a.ubar = h->ubar;
    a.dFlux = h->dFlux;
    a.Dlin = L0.Dlin;
    a.D = L0.Dblk;
    a.Blin = h->nlev > 1 ? h->lev[1].Blin : nullptr;
    a.Bsr = h->nlev > 1 ? h->lev[1].Bsr : nullptr;
    a.nb1 = h->nlev > 1 ? h->lev[1].nb : 0;
    a.inv_gdt = h->inv_gdt;
    double* Dl[DG_MAX_LEVELS];
    double* Bl[DG_MAX_LEVELS];
    for (int l = 0; l < h->nlev; ++l) { Dl[l] = h->lev[l].Dblk; Bl[l] = h->lev[l].Bsr; }
    if ((rc = assemble_levels<double>(h, a, Dl, Bl, h->stb1, st))) return rc;
    for (int l = 0; l < h->nlev; ++l) {
      Level& L = h->lev[l];
      if ((rc = factor_blocks<double>(h, ne, L.b, L.Dblk, L.Dinv, L.perm, st))) return rc;
    }
  } else {
    if ((rc = alloc_fp32_levels(h))) return rc;
    if ((rc = prepare_lin_fp32(h, st))) return rc;
    AsmArgs<float> a;
    const TablesF& F = h->tabf;
    a.M = mesh_dev(h);
    a.T = h->tab;
    a.Bvol = F.Bvol; a.wvol = F.wvol; a.B2 = F.B2; a.W2 = F.W2; a.pv = F.pv; a.Dcol_val = F.Dcol_val;
    a.ubar = h->ubar_f;
    a.dFlux = h->dFlux_f;
    a.Dlin = L0.Dlin;
    a.D = L0.LUf;
    a.Blin = h->nlev > 1 ? h->lev[1].Blin : nullptr;
    a.Bsr = h->nlev > 1 ? h->lev[1].Bsrf : nullptr;
    a.nb1 = h->nlev > 1 ? h->lev[1].nb : 0;
    a.inv_gdt = h->inv_gdt;
    float* Dl[DG_MAX_LEVELS];
    float* Bl[DG_MAX_LEVELS];
    for (int l = 0; l < h->nlev; ++l) { Dl[l] = h->lev[l].LUf; Bl[l] = h->lev[l].Bsrf; }
    if (h->stb_rescale && !h->stb1f) {  // an FP32 copy of the stabilisation blocks (fixed per handle)
      const long long n = 7ll * h->lev[1].b * h->lev[1].b * ne;
      DG_CUDA(h, cudaMalloc((void**)&h->stb1f, sizeof(float) * n));
      narrow_f32_kernel<<<h->nsm * 8, 256, 0, st>>>(n, h->stb1, h->stb1f);
      DG_LAUNCH_CHECK(h);
    }
    if ((rc = assemble_levels<float>(h, a, Dl, Bl, h->stb1f, st))) return rc;
    if ((rc = invert_levels_f32(h, st, h->status + 2))) return rc;  // the FP32 smoother applies explicit inverses
  }
  // the verdict on this assembly's own status word (flags of earlier calls do not count); its
  // bits also go to the handle's word, which dg_get_status reads
  DG_CUDA(h, cudaStreamSynchronize(st));
  unsigned s = 0;
  DG_CUDA(h, cudaMemcpy(&s, h->status + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (s) {
    or_bits_kernel<<<1, 1, 0, st>>>(h->status, s);
    DG_LAUNCH_CHECK(h);
  }
  if (s & DG_STATUS_NONFINITE) return fail(h, DG_ERR_NONFINITE, "singular or non-finite element block");
  return DG_OK;
}

}  // namespace dg
