// Tensor-core volume pass of the FP32 preconditioner cycle's Jacobian action (sm_103a).
//
// The convective volume term of the linearised residual (Eq. (jacTrilFnotNU): the quadrature of
// d(u (x) u)[du] : grad phi_j in Eq. (NSdiscrRes)) needs the velocity variation at the Gauss
// points and the integral of the weighted products against the basis. Here both contractions run
// as dense per-element GEMMs on the 5th-generation tensor cores (tcgen05.mma, kind::f16: FP16 or
// BF16 operands, FP32 accumulation in tensor memory), 21 elements per tile:
//
//   interpolation  D1[q][(e,f)] = sum_m phi_hat_m(x_q) * sigma_e c_{e,f,m}
//                  M = 128 Gauss points (125 used), N = 64 (63 = 21 x 3 velocity components),
//                  K = 48 modes (35 used);
//   integration    D2[(e,s)][m] = sum_q P_{e,s}(x_q) * phi_hat_m(x_q)
//                  M = 128 (126 = 21 x 6 symmetric products), N = 48 modes, K = 128 points,
//
// with P_{e,s}(x_q) = w_q (u_p ub_i + ub_p u_i) scaled by sigma_e tau_e s_e. The scales are powers
// of two per element: sigma_e from the largest velocity coefficient of the tile's input and tau_e
// from the largest linearisation velocity at the element's points (computed once per
// linearisation), so that every 16-bit operand lies near unit size whatever the magnitude of the
// Krylov vector the cycle is applied to. Power-of-two scales are exact, and the FP32 results are
// unscaled exactly.
//
// Everything else of the volume pass is the CUDA-core FP32 arithmetic of vol_kernel: corrected
// gradients with the BR2 liftings, the viscous flux, the pressure and continuity terms as exact
// sparse modal derivatives, the six face contributions and the mass shift (Eqs. (vflux),
// (massBil)).
//
// Operand layout in shared memory (K-major, no swizzle): cores of 8 rows x 16 bytes; the shared
// memory descriptor's leading byte offset is the distance of K-adjacent cores, the stride byte
// offset that of row-adjacent 8-row groups. The 16-bit basis tables (D1's A operand, D2's B
// operand) are built on the host once per handle. The products' operand uses a K-core distance
// of 144 bytes, so that the 2-byte stores of 32 consecutive points hit 32 distinct banks.
//
// One elected thread issues the MMAs and commits them to an mbarrier; every wait is bounded
// (DG_STATUS_WAIT, then a second bounded wait for the MMAs in flight before the tensor memory is
// released).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <vector>

#include "dg_async.h"
#include "dg_internal.h"

namespace dg {
namespace {

constexpr int kTcE = 21;                // elements per tile (6 x 21 = 126 <= 128 rows of D2)
constexpr int kTcThreads = 256;         // warps w and w + 4 read TMEM lane quarter w % 4
constexpr unsigned kTcCols = 128;       // TMEM columns per CTA: D1 at 0..63, D2 at 64..111
constexpr unsigned kTcD2 = 64;
constexpr int kQP = 128;                // padded Gauss points
constexpr int kMP = 48;                 // padded modes
constexpr int kN1 = 64;                 // N of the interpolation
// shared-memory byte offsets of the operands
constexpr unsigned kTA1 = 0;            // [128 q][48 m]
constexpr unsigned kTB2 = 12288;        // [48 m][128 q]
constexpr unsigned kB1 = 24576;         // [64 (e,f)][48 m]
constexpr unsigned kA2 = 30720;         // [128 (e,s)][128 q], K-cores 144 B apart
constexpr unsigned kA2Bytes = 16 * 16 * 144;
constexpr unsigned kTabBytes = 24576;   // TA1 + TB2
constexpr unsigned kKc = 128, kKcA2 = 144;  // K-core distances
constexpr unsigned kRgTA1 = 6 * 128, kRgTB2 = 16 * 128, kRgB1 = 6 * 128, kRgA2 = 16 * 144;  // row-group distances

template <int K>
struct TcSz {
  static constexpr int NB = nb_of(K), N1 = K + 1, NQ = N1 * N1 * N1, N2 = (K + 1) * (K + 2) / 2, K1 = K + 1;
  static constexpr unsigned SC = kA2 + kA2Bytes;                                  // [E][4][NB] f32
  static constexpr unsigned FV = SC + ((kTcE * 4 * NB * 4 + 127) / 128) * 128;   // [E][6][NB] f32
  static constexpr unsigned BYTES = FV + ((kTcE * 6 * NB * 4 + 127) / 128) * 128;
  static_assert(NQ <= kQP && NB <= kMP, "tile sizes");
  static_assert(kTcE * 9 * NB * 4 <= (int)kA2Bytes, "corrected gradients fit the products' buffer");
};

// byte offset of element (r, k) in a K-major no-swizzle operand
__host__ __device__ constexpr unsigned core_off(int r, int k, unsigned kcore, unsigned rgroup) {
  return (unsigned)(r / 8) * rgroup + (unsigned)(k / 8) * kcore + (unsigned)(r % 8) * 16 + (unsigned)(k % 8) * 2;
}

// ---------------------------------------------------------------- tcgen05 wrappers
__device__ __forceinline__ uint64_t umma_smem_desc(unsigned addr, unsigned kcore, unsigned rgroup) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((kcore >> 4) & 0x3FFF) << 16;   // leading byte offset: K-adjacent cores
  d |= (uint64_t)((rgroup >> 4) & 0x3FFF) << 32;  // stride byte offset: row-adjacent 8-row groups
  d |= (uint64_t)1 << 46;                         // descriptor version (fixed 0b001 at bits 46-48)
  return d;                                       // base offset 0, relative offsets, no swizzle
}
// kind::f16 instruction descriptor: D in FP32, A and B both FP16 (bf = 0) or both BF16 (bf = 1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr unsigned umma_idesc(int bf, int m, int n) {
  return (1u << 4) | ((unsigned)bf << 7) | ((unsigned)bf << 10) | ((unsigned)(n >> 3) << 17) |
         ((unsigned)(m >> 4) << 24);
}
__device__ __forceinline__ void umma(unsigned dtmem, uint64_t a, uint64_t b, unsigned idesc, unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define DG_TMEM_R8(i) "=r"(r[i + 0]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), "=r"(r[i + 4]), "=r"(r[i + 5]), \
                      "=r"(r[i + 6]), "=r"(r[i + 7])
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : DG_TMEM_R8(0), DG_TMEM_R8(8), DG_TMEM_R8(16), DG_TMEM_R8(24)
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(unsigned taddr, unsigned (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : DG_TMEM_R8(0), DG_TMEM_R8(8)
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld2(unsigned taddr, unsigned (&r)[2]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr) : "memory");
}
#undef DG_TMEM_R8
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int BF>
__device__ __forceinline__ unsigned short to16(float x) {
  if constexpr (BF) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<const unsigned short*>(&h);
  } else {
    const __half h = __float2half_rn(x);
    return *reinterpret_cast<const unsigned short*>(&h);
  }
}

__device__ __forceinline__ float pow2_scale(float mx) {  // 2^-ceil(log2 mx): brings mx into (1/2, 1]
  if (!(mx > 0.0f) || !isfinite(mx)) return 1.0f;
  int ex;
  frexpf(mx, &ex);  // mx = f 2^ex, f in [1/2, 1)
  return ldexpf(1.0f, -ex);
}

struct TcVolArgs {
  MeshDev M;
  const int* Drow_idx;
  const int* Dcol_idx;
  const int* fmap;
  const int* fa;
  const float* Drow_val;
  const float* Dcol_val;
  const float* pv;
  const float* wvol;
  const float* in;
  float* out;
  const float* face_out;
  const float* face_lift;
  const float* ubar;
  const float* ubar_scale;
  const uint4* tab;  // TA1 then TB2, 16-bit, in the operand layout (kTabBytes)
  float nu;
  double inv_gdt;
  unsigned* status;
  unsigned wait_polls;
};

__device__ __forceinline__ int sym_pair(int sp, int& i) {  // sp -> (p, i): 0,1,2 diagonal; 3 = 01, 4 = 02, 5 = 12
  int p;
  if (sp < 3) { p = sp; i = sp; } else if (sp == 3) { p = 0; i = 1; } else if (sp == 4) { p = 0; i = 2; } else { p = 1; i = 2; }
  return p;
}
__device__ __forceinline__ int sym_idx(int p, int i) { return p == i ? p : (p + i + 2); }

// Pointwise products of the elements EL0 .. EL0 + NEL - 1 at this thread's Gauss point q: their
// interpolated (scaled) velocity variation sits in TMEM columns 3 el + f, loaded here from column
// COL0 on (NC = 32 or 34 columns).
template <int K, int BF, int EL0, int NEL, int COL0, int NC>
__device__ __forceinline__ void tc_pointwise(const TcVolArgs& a, unsigned tmem_lane, int q, int e0, int cnt,
                                             const float* sSig, const float* sTau, float wq, unsigned char* sm) {
  using Z = TcSz<K>;
  unsigned r[NC];
  {
    unsigned r32[32];
    tmem_ld32(tmem_lane + COL0, r32);
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = r32[j];
    if constexpr (NC == 34) {
      unsigned r2[2];
      tmem_ld2(tmem_lane + COL0 + 32, r2);
      r[32] = r2[0];
      r[33] = r2[1];
    }
  }
  tmem_wait_ld();
  const bool qv = q < Z::NQ;
  float ub[NEL][3];
#pragma unroll
  for (int j = 0; j < NEL; ++j) {
    const int el = EL0 + j;
    const bool ok = qv && el < cnt;
#pragma unroll
    for (int c = 0; c < 3; ++c) ub[j][c] = ok ? a.ubar[((size_t)(e0 + el) * 3 + c) * Z::NQ + q] : 0.0f;
  }
  unsigned char* A2 = sm + kA2;
#pragma unroll
  for (int j = 0; j < NEL; ++j) {
    const int el = EL0 + j;
    const float tau = sTau[el];
    float u[3], b[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      u[f] = __uint_as_float(r[3 * el + f - COL0]);
      b[f] = tau * ub[j][f];
    }
    const bool ok = qv && el < cnt;
#pragma unroll
    for (int sp = 0; sp < 6; ++sp) {
      int i;
      const int p = sym_pair(sp, i);
      const float v = ok ? wq * (u[p] * b[i] + b[p] * u[i]) : 0.0f;
      *reinterpret_cast<unsigned short*>(A2 + core_off(6 * el + sp, q, kKcA2, kRgA2)) = to16<BF>(v);
    }
  }
  (void)sSig;
}

template <int K, int BF>
__global__ void __launch_bounds__(kTcThreads) tc_vol_kernel(TcVolArgs a) {
  using Z = TcSz<K>;
  constexpr int NB = Z::NB, NQ = Z::NQ, N2 = Z::N2, K1 = Z::K1, DW = Tables::kDw;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ unsigned tslot;
  __shared__ float sSig[kTcE], sTau[kTcE], sJ[kTcE][3], sShift[kTcE];
  __shared__ float PV[2 * K1];
  __shared__ int FMAP[3 * NB], FA[3 * NB];
  float* sC = reinterpret_cast<float*>(sm + Z::SC);    // [E][4][NB]
  float* sFv = reinterpret_cast<float*>(sm + Z::FV);   // [E][6][NB]
  float* sG = reinterpret_cast<float*>(sm + kA2);      // [E][9][NB], while the products' buffer is idle
  float* sCv = reinterpret_cast<float*>(sm + kA2);     // [E][6][NB], after the integration MMA
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x;
  const int ne = a.M.ne, ntiles = (ne + kTcE - 1) / kTcE;

  if (tid == 0) mbar_init(&bar, 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the basis tables (16-bit operands), zeroed interpolation operand (its K padding stays zero)
  {
    uint4* s4 = reinterpret_cast<uint4*>(sm);
    for (int i = tid; i < (int)(kTabBytes / 16); i += nt) s4[i] = a.tab[i];
    for (int i = tid; i < (int)((kA2 - kB1) / 16); i += nt) s4[kB1 / 16 + i] = make_uint4(0, 0, 0, 0);
  }
  for (int t = tid; t < 2 * K1; t += nt) PV[t] = a.pv[t];
  for (int t = tid; t < 3 * NB; t += nt) { FMAP[t] = a.fmap[t]; FA[t] = a.fa[t]; }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tslot;
  const unsigned lane_base = (unsigned)(32 * (warp & 3)) << 16;
  const unsigned sbase = smem_u32(sm);
  const int q = 32 * (warp & 3) + lane;
  const float wq = q < NQ ? a.wvol[q] : 0.0f;
  unsigned phase = 0;
  bool nonfinite = false;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int e0 = tile * kTcE;
    const int cnt = min(kTcE, ne - e0);
    if (tid == 0 && tile + (int)gridDim.x < ntiles) {
      // the next tile's contiguous inputs into L2 while this tile is computed
      const int n0 = (tile + gridDim.x) * kTcE, n1 = min(ne, n0 + kTcE);
      prefetch_l2(a.in + (size_t)n0 * 4 * NB, a.in + (size_t)n1 * 4 * NB);
      prefetch_l2(a.face_lift + (size_t)n0 * 6 * 3 * N2, a.face_lift + (size_t)n1 * 6 * 3 * N2);
      prefetch_l2(a.ubar + (size_t)n0 * 3 * NQ, a.ubar + (size_t)n1 * 3 * NQ);
      prefetch_l2(a.face_out + (size_t)n0 * 6 * 4 * N2, a.face_out + (size_t)n1 * 6 * 4 * N2);
    }
    // 1. input coefficients (FP32, contiguous), element geometry
    for (int t = tid; t < kTcE * 4 * NB; t += nt)
      sC[t] = t < cnt * 4 * NB ? a.in[(size_t)e0 * 4 * NB + t] : 0.0f;
    for (int t = tid; t < kTcE; t += nt) {
      const bool ok = t < cnt;
      const double* G = a.M.geo + (size_t)(e0 + (ok ? t : 0)) * kGeo;
      sJ[t][0] = (float)G[5];
      sJ[t][1] = (float)G[6];
      sJ[t][2] = (float)G[7];
      sShift[t] = (float)(a.inv_gdt * G[11]);
      sTau[t] = ok ? a.ubar_scale[e0 + t] : 1.0f;
    }
    __syncthreads();
    // 2. per-element scale of the velocity coefficients (warp per element)
    for (int el = warp; el < kTcE; el += nt / 32) {
      float mx = 0.0f;
      for (int t = lane; t < 3 * NB; t += 32) mx = fmaxf(mx, fabsf(sC[el * 4 * NB + t]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) sSig[el] = pow2_scale(mx);
    }
    __syncthreads();
    // 3. the interpolation's B operand: rows (e, f), K = modes
    for (int t = tid; t < kTcE * 3 * NB; t += nt) {
      const int r = t / NB, m = t - r * NB, el = r / 3, f = r - 3 * el;
      *reinterpret_cast<unsigned short*>(sm + kB1 + core_off(r, m, kKc, kRgB1)) =
          to16<BF>(sSig[el] * sC[(el * 4 + f) * NB + m]);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      constexpr unsigned id1 = umma_idesc(BF, 128, kN1);
#pragma unroll
      for (int kk = 0; kk < kMP / 16; ++kk)
        umma(tmem, umma_smem_desc(sbase + kTA1 + kk * 2 * kKc, kKc, kRgTA1),
             umma_smem_desc(sbase + kB1 + kk * 2 * kKc, kKc, kRgB1), id1, kk > 0);
      umma_commit(&bar);
    }
    // 4. while the MMA runs: corrected gradients grad u - R^K (into the idle products' buffer)
    for (int t = tid; t < kTcE * 3 * NB; t += nt) {
      const int el = t / (3 * NB), r = t - el * 3 * NB, b = r / NB, m = r - b * NB;
      if (el >= cnt) continue;
      int di[DW];
      float dv[DW];
#pragma unroll
      for (int j = 0; j < DW; ++j) {
        const int o = (b * NB + m) * DW + j;
        di[j] = a.Drow_idx[o];
        dv[j] = a.Drow_val[o];
      }
      const int j2 = FMAP[b * NB + m], ex = FA[b * NB + m];
      const float p1 = PV[K1 + ex], p0 = PV[ex], jb = sJ[el][b];
      const float* Lf = a.face_lift + (size_t)(e0 + el) * 6 * 3 * N2;
      const float* cv0 = sC + el * 4 * NB;
#pragma unroll
      for (int av = 0; av < 3; ++av) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < DW; ++j) acc += dv[j] * cv0[av * NB + di[j]];
        const float rl = p1 * Lf[(2 * b) * 3 * N2 + av * N2 + j2] + p0 * Lf[(2 * b + 1) * 3 * N2 + av * N2 + j2];
        sG[(el * 9 + av * 3 + b) * NB + m] = acc * jb - rl;
      }
    }
    __syncthreads();
    // viscous flux coefficients F^nu(grad u - R^K) (symmetric pairs)
    for (int t = tid; t < kTcE * 6 * NB; t += nt) {
      const int el = t / (6 * NB), r = t - el * 6 * NB, sp = r / NB, m = r - sp * NB;
      if (el >= cnt) continue;
      int i;
      const int p = sym_pair(sp, i);
      const float* G = sG + el * 9 * NB;
      const float trG = G[0 * NB + m] + G[4 * NB + m] + G[8 * NB + m];
      sFv[t] = a.nu * (G[(i * 3 + p) * NB + m] + G[(p * 3 + i) * NB + m] - (p == i ? (2.0f / 3.0f) * trG : 0.0f));
    }
    // 5. the interpolated velocity variation: wait for the MMA
    bool ok = mbar_wait(&bar, phase & 1, a.wait_polls);
    ++phase;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(a.status, (unsigned)DG_STATUS_WAIT);
        mbar_wait(&bar, (phase - 1) & 1);  // the MMA in flight lands before the tensor memory is freed
      }
      break;
    }
    tc_fence_after();
    // 6. pointwise products into the integration's A operand (sG is no longer needed)
    if (warp < 4)
      tc_pointwise<K, BF, 0, 11, 0, 34>(a, tmem + lane_base, q, e0, cnt, sSig, sTau, wq, sm);
    else
      tc_pointwise<K, BF, 11, kTcE - 11, 32, 32>(a, tmem + lane_base, q, e0, cnt, sSig, sTau, wq, sm);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      constexpr unsigned id2 = umma_idesc(BF, 128, kMP);
#pragma unroll
      for (int kk = 0; kk < kQP / 16; ++kk)
        umma(tmem + kTcD2, umma_smem_desc(sbase + kA2 + kk * 2 * kKcA2, kKcA2, kRgA2),
             umma_smem_desc(sbase + kTB2 + kk * 2 * kKc, kKc, kRgTB2), id2, kk > 0);
      umma_commit(&bar);
    }
    ok = mbar_wait(&bar, phase & 1, a.wait_polls);
    ++phase;
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicOr(a.status, (unsigned)DG_STATUS_WAIT);
        mbar_wait(&bar, (phase - 1) & 1);
      }
      break;
    }
    tc_fence_after();
    // 7. projections of the products onto the basis, unscaled: Cv = D2 / (sigma tau)
    {
      const int rr = 32 * (warp & 3) + lane, el = rr / 6, sp = rr - 6 * el;
      const bool rv = el < cnt;
      const float inv = rv ? 1.0f / (sSig[el] * sTau[el]) : 0.0f;
      if (warp < 4) {
        unsigned r32[32];
        tmem_ld32(tmem + lane_base + kTcD2, r32);
        tmem_wait_ld();
        if (rv)
#pragma unroll
          for (int m = 0; m < 32; ++m)
            if (m < NB) sCv[(el * 6 + sp) * NB + m] = __uint_as_float(r32[m]) * inv;
      } else {
        unsigned r16[16];
        tmem_ld16(tmem + lane_base + kTcD2 + 32, r16);
        tmem_wait_ld();
        if (rv)
#pragma unroll
          for (int m = 0; m < 16; ++m)
            if (32 + m < NB) sCv[(el * 6 + sp) * NB + 32 + m] = __uint_as_float(r16[m]) * inv;
      }
    }
    tc_fence_before();
    __syncthreads();
    // 8. assemble: modal derivatives of (F^nu - u (x) u) and p, continuity, face terms, mass shift
    for (int t = tid; t < kTcE * NB; t += nt) {
      const int el = t / NB, m = t - el * NB;
      if (el >= cnt) continue;
      const int e = e0 + el;
      const float* cE = sC + el * 4 * NB;
      const float* fE = sFv + el * 6 * NB;
      const float* vE = sCv + el * 6 * NB;
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int pp = 0; pp < 3; ++pp) {
        float s2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < DW; ++j) {
          const int o = (pp * NB + m) * DW + j;
          const int n = a.Dcol_idx[o];
          const float dv = a.Dcol_val[o];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const int sp = sym_idx(pp, i);
            s2[i] += dv * (fE[sp * NB + n] - vE[sp * NB + n] - (pp == i ? cE[3 * NB + n] : 0.0f));
          }
          s2[3] += dv * (-cE[pp * NB + n]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += sJ[el][pp] * s2[i];
      }
      const float* FO = a.face_out + (size_t)e * 6 * 4 * N2;
#pragma unroll
      for (int sl = 0; sl < 6; ++sl) {
        const int dd = sl >> 1, side = (sl & 1) ? 0 : 1;
        const float pw = PV[side * K1 + FA[dd * NB + m]];
        const int fm = FMAP[dd * NB + m];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] += pw * FO[sl * 4 * N2 + i * N2 + fm];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (i < 3) acc[i] += sShift[el] * cE[i * NB + m];
        nonfinite |= !isfinite(acc[i]);
        a.out[(size_t)e * 4 * NB + i * NB + m] = acc[i];
      }
    }
    __syncthreads();  // sC, sFv and sCv are rewritten by the next tile
  }
  if (nonfinite && a.status) atomicOr(a.status, (unsigned)DG_STATUS_NONFINITE);
  tc_fence_before();
  __syncthreads();
  if (warp == 0)  // always released: a CTA must not exit holding tensor memory
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
}

// one warp per element: tau_e = 2^-ceil(log2 max |ub|) over the element's linearisation velocity
__global__ void ubar_scale_kernel(int ne, int n3q, const float* __restrict__ ubar, float* __restrict__ scale) {
  const int lane = threadIdx.x & 31;
  for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < ne; e += (gridDim.x * blockDim.x) >> 5) {
    float mx = 0.0f;
    for (int t = lane; t < n3q; t += 32) mx = fmaxf(mx, fabsf(ubar[(size_t)e * n3q + t]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) scale[e] = pow2_scale(mx);
  }
}

template <int K, int BF>
int launch_tc(Handle* h, const TcVolArgs& a, cudaStream_t st) {
  const size_t smem = TcSz<K>::BYTES;
  DG_CUDA(h, cudaFuncSetAttribute(tc_vol_kernel<K, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int ntiles = (h->ne + kTcE - 1) / kTcE;
  const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(2, (227 * 1024) / (smem + 2048)));
  const int grid = std::min(ntiles, h->nsm * per_sm);
  tc_vol_kernel<K, BF><<<grid, kTcThreads, smem, st>>>(a);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

}  // namespace

// The 16-bit basis tables of the tensor-core volume pass (FP16 and BF16), from the FP64 table
// phi_hat_m(x_q): interpolation A operand [128 q][48 m] and integration B operand [48 m][128 q],
// zero outside q < N_q, m < N_b. Once per handle; allocates, so it runs before any capture.
int tc_prepare_tables(Handle* h) {
  if (h->tc_tab[0] && h->tc_tab[1]) return DG_OK;
  const int nq = h->tab.nq, nb = h->tab.nb;
  if (nq > kQP || nb > kMP) return fail(h, DG_ERR_ARG, "degree unsuited to the tensor-core volume pass");
  std::vector<double> B((size_t)nq * nb);
  DG_CUDA(h, cudaMemcpy(B.data(), h->tab.Bvol, sizeof(double) * B.size(), cudaMemcpyDeviceToHost));
  for (int bf = 0; bf < 2; ++bf) {
    std::vector<unsigned short> T(kTabBytes / 2, 0);
    auto put = [&](unsigned byte_off, double v) {
      unsigned short u;
      if (bf) {
        const __nv_bfloat16 x = __float2bfloat16_rn((float)v);
        u = *reinterpret_cast<const unsigned short*>(&x);
      } else {
        const __half x = __float2half_rn((float)v);
        u = *reinterpret_cast<const unsigned short*>(&x);
      }
      T[byte_off / 2] = u;
    };
    for (int qq = 0; qq < nq; ++qq)
      for (int m = 0; m < nb; ++m) {
        const double v = B[(size_t)qq * nb + m];
        put(kTA1 + core_off(qq, m, kKc, kRgTA1), v);
        put(kTB2 + core_off(m, qq, kKc, kRgTB2), v);
      }
    DG_CUDA(h, cudaMalloc(&h->tc_tab[bf], kTabBytes));
    DG_CUDA(h, cudaMemcpy(h->tc_tab[bf], T.data(), kTabBytes, cudaMemcpyHostToDevice));
  }
  return DG_OK;
}

// per-element scale of the FP32 linearisation velocity (after prepare_lin_fp32 refreshed it)
int tc_prepare_lin(Handle* h, cudaStream_t st) {
  if (!h->ubar_scale) DG_CUDA(h, cudaMalloc(&h->ubar_scale, sizeof(float) * (size_t)h->ne));
  const int n3q = 3 * h->tab.nq;
  const int grid = std::min(h->nsm * 8, (h->ne * 32 + 255) / 256);
  ubar_scale_kernel<<<grid, 256, 0, st>>>(h->ne, n3q, h->ubar_f, h->ubar_scale);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// Volume pass of the FP32 Jacobian action on the tensor cores; the face pass (face_out_f,
// face_lift_f) has run. tc = 1: FP16 operands, tc = 2: BF16 operands.
int tc_volume_tangent(Handle* h, const float* in, float* out, int tc, cudaStream_t st) {
  if (!h->tc_tab[0] || !h->ubar_scale) return fail(h, DG_ERR_STATE, "tensor-core tables not prepared");
  const Tables& T = h->tab;
  const TablesF& F = h->tabf;
  const int bf = tc == 2 ? 1 : 0;
  TcVolArgs a;
  a.M = mesh_dev(h);
  a.Drow_idx = T.Drow_idx;
  a.Dcol_idx = T.Dcol_idx;
  a.fmap = T.fmap;
  a.fa = T.fa;
  a.Drow_val = F.Drow_val;
  a.Dcol_val = F.Dcol_val;
  a.pv = F.pv;
  a.wvol = F.wvol;
  a.in = in;
  a.out = out;
  a.face_out = h->face_out_f;
  a.face_lift = h->face_lift_f;
  a.ubar = h->ubar_f;
  a.ubar_scale = h->ubar_scale;
  a.tab = static_cast<const uint4*>(h->tc_tab[bf]);
  a.nu = (float)h->p.nu;
  a.inv_gdt = h->inv_gdt;
  a.status = h->status;
  a.wait_polls = h->dbg.wait_polls > 0 ? (unsigned)h->dbg.wait_polls : kBulkWaitLimit;
  switch (T.k) {
    case 1: return bf ? launch_tc<1, 1>(h, a, st) : launch_tc<1, 0>(h, a, st);
    case 2: return bf ? launch_tc<2, 1>(h, a, st) : launch_tc<2, 0>(h, a, st);
    case 3: return bf ? launch_tc<3, 1>(h, a, st) : launch_tc<3, 0>(h, a, st);
    case 4: return bf ? launch_tc<4, 1>(h, a, st) : launch_tc<4, 0>(h, a, st);
  }
  return fail(h, DG_ERR_ARG, "unsupported degree");
}

}  // namespace dg
