// Preconditioner assembly at the current linearisation (Sec. 2.3-2.4):
//  * element diagonal blocks of G on the fine level, by probing the exact
//    Jacobian action with unit vectors on the elements of one colour of a
//    distance-1 colouring (no two face neighbours share a colour);
//  * off-diagonal blocks at the degree of level 1 only (Sec. 2.4.3: coarse
//    off-diagonal blocks are built at the coarse degree), by probing the coarse
//    modes on the elements of one colour of a distance-2 colouring (no element
//    has two face neighbours of one colour);
//  * inherited operators of every coarser level by sub-block extraction
//    (Eq. (GalProj) with a hierarchical orthonormal basis);
//  * inverses of all diagonal blocks (element-wise block Jacobi) by in-place
//    Gauss-Jordan elimination with partial pivoting, one block per CTA in
//    shared memory.
// Blocks are stored column-major: block[c * b + r] = G[row r][col c].
#include <algorithm>
#include <vector>

#include "dg_internal.h"

namespace dg {

static std::vector<int> greedy_colouring(const Handle* h, int dist) {
  const int ne = h->ne;
  std::vector<int> nb6((size_t)ne * 6);
  for (int e = 0; e < ne; ++e) {
    const int i = e % h->n[0], j = (e / h->n[0]) % h->n[1], k = e / (h->n[0] * h->n[1]);
    auto id = [&](int a, int b, int c) {
      a = (a + h->n[0]) % h->n[0]; b = (b + h->n[1]) % h->n[1]; c = (c + h->n[2]) % h->n[2];
      return a + h->n[0] * (b + h->n[1] * c);
    };
    nb6[e * 6 + 0] = id(i - 1, j, k); nb6[e * 6 + 1] = id(i + 1, j, k);
    nb6[e * 6 + 2] = id(i, j - 1, k); nb6[e * 6 + 3] = id(i, j + 1, k);
    nb6[e * 6 + 4] = id(i, j, k - 1); nb6[e * 6 + 5] = id(i, j, k + 1);
  }
  std::vector<int> col(ne, -1);
  std::vector<int> mark(64, -1);
  for (int e = 0; e < ne; ++e) {
    std::vector<int> around;
    for (int f = 0; f < 6; ++f) {
      const int p = nb6[e * 6 + f];
      around.push_back(p);
      if (dist >= 2)
        for (int g = 0; g < 6; ++g) around.push_back(nb6[p * 6 + g]);
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
    if (colour[e] != c) continue;
    bool first = true;
    for (int g = 0; g < f; ++g)
      if (nbr[p * 6 + g] == e) first = false;
    if (!first) continue;
    const int var = rc / nb1, m = rc - var * nb1;
    Bsr[(((p * 7 + 1 + f) * (long long)b1) + jc) * b1 + rc] = out[(p * 4 + var) * nb0 + m];
  }
}

// dst block (size bd, nbd modes/variable) = leading sub-block of src block (bs, nbs).
__global__ void subblock_kernel(long long nblocks, int nbs, int nbd, const double* src, long long src_stride,
                                double* dst, long long dst_stride) {
  const int bs = 4 * nbs, bd = 4 * nbd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nblocks * bd * bd;
       i += (long long)gridDim.x * blockDim.x) {
    const long long blk = i / ((long long)bd * bd);
    const int rem = (int)(i - blk * bd * bd), c = rem / bd, r = rem - c * bd;
    const int cs = (c / nbd) * nbs + c % nbd, rs = (r / nbd) * nbs + r % nbd;
    dst[blk * dst_stride + (long long)c * bd + r] = src[blk * src_stride + (long long)cs * bs + rs];
  }
}

// In-place Gauss-Jordan inversion with partial (row) pivoting of one b x b block per
// CTA in shared memory (row-major with a padded leading dimension).
__global__ void __launch_bounds__(256) gj_inverse_kernel(int nblk, int b, const double* in, double* out,
                                                         unsigned* status) {
  extern __shared__ double sm[];
  const int LD = b + 1;
  double* A = sm;             // [b][LD]
  double* col = A + b * LD;   // [b]
  int* perm = reinterpret_cast<int*>(col + b);  // [b]
  __shared__ int s_piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const double* src = in + (size_t)blk * b * b;
    for (int t = tid; t < b * b; t += nt) {
      const int c = t / b, r = t - c * b;
      A[r * LD + c] = src[t];
    }
    __syncthreads();
    for (int k = 0; k < b; ++k) {
      if (tid < 32) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < b; i += 32) {
          const double v = fabs(A[i * LD + k]);
          if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const double ov = __shfl_down_sync(0xffffffffu, best, off);
          const int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (tid == 0) {
          s_piv = bi;
          perm[k] = bi;
          if (!(best > 0.0) && status) atomicOr(status, (unsigned)DG_STATUS_NONFINITE);
        }
      }
      __syncthreads();
      const int p = s_piv;
      if (p != k)
        for (int j = tid; j < b; j += nt) {
          const double t = A[k * LD + j];
          A[k * LD + j] = A[p * LD + j];
          A[p * LD + j] = t;
        }
      __syncthreads();
      for (int i = tid; i < b; i += nt) col[i] = A[i * LD + k];
      __syncthreads();
      const double ipiv = 1.0 / col[k];
      for (int j = tid; j < b; j += nt) A[k * LD + j] = (j == k ? 1.0 : A[k * LD + j]) * ipiv;
      __syncthreads();
      for (int t = tid; t < b * b; t += nt) {
        const int i = t / b, j = t - i * b;
        if (i == k) continue;
        const double f = col[i];
        A[i * LD + j] = (j == k) ? -f * A[k * LD + k] : A[i * LD + j] - f * A[k * LD + j];
      }
      __syncthreads();
    }
    for (int k = b - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k)
        for (int i = tid; i < b; i += nt) {
          const double t = A[i * LD + k];
          A[i * LD + k] = A[i * LD + p];
          A[i * LD + p] = t;
        }
      __syncthreads();
    }
    double* dst = out + (size_t)blk * b * b;
    for (int t = tid; t < b * b; t += nt) {
      const int c = t / b, r = t - c * b;
      dst[t] = A[r * LD + c];
    }
    __syncthreads();
  }
}

static int invert_blocks(Handle* h, int nblk, int b, const double* in, double* out, cudaStream_t st) {
  const size_t smem = sizeof(double) * ((size_t)b * (b + 1) + b) + sizeof(int) * b;
  DG_CUDA(h, cudaFuncSetAttribute(gj_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = (int)((220 * 1024) / smem);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  int grid = h->nsm * per_sm;
  if (grid > nblk) grid = nblk;
  gj_inverse_kernel<<<grid, 256, smem, st>>>(nblk, b, in, out, h->status);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

int assemble_all(Handle* h, cudaStream_t st) {
  const int ne = h->ne;
  Level& L0 = h->lev[0];
  const int b0 = L0.b;
  const int grid = h->nsm * 8;
  int rc;
  // allocate on first use
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->lev[l];
    const size_t bb = (size_t)L.b * L.b;
    if (!L.Dblk) DG_CUDA(h, cudaMalloc((void**)&L.Dblk, sizeof(double) * bb * ne));
    if (!L.Dinv) DG_CUDA(h, cudaMalloc((void**)&L.Dinv, sizeof(double) * bb * ne));
    if (l >= 1 && !L.Bsr) DG_CUDA(h, cudaMalloc((void**)&L.Bsr, sizeof(double) * bb * 7 * ne));
  }
  // --- fine diagonal blocks
  const std::vector<int> c1 = greedy_colouring(h, 1);
  const int nc1 = *std::max_element(c1.begin(), c1.end()) + 1;
  if (!h->colour) DG_CUDA(h, cudaMalloc((void**)&h->colour, sizeof(int) * ne));
  int* dcol = h->colour;
  DG_CUDA(h, cudaMemcpyAsync(dcol, c1.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, st));
  double* probe = L0.t0;
  double* out = L0.t1;
  for (int c = 0; c < nc1; ++c)
    for (int j = 0; j < b0; ++j) {
      probe_kernel<<<grid, 256, 0, st>>>(L0.n, b0, dcol, c, j, probe);
      DG_LAUNCH_CHECK(h);
      if ((rc = op_tangent(h, probe, out, st))) return rc;
      scatter_diag_kernel<<<grid, 256, 0, st>>>(ne, b0, dcol, c, j, out, L0.Dblk);
      DG_LAUNCH_CHECK(h);
    }
  // --- coarse levels
  if (h->nlev > 1) {
    Level& L1 = h->lev[1];
    const int b1 = L1.b;
    DG_CUDA(h, cudaMemsetAsync(L1.Bsr, 0, sizeof(double) * (size_t)b1 * b1 * 7 * ne, st));
    const std::vector<int> c2 = greedy_colouring(h, 2);
    const int nc2 = *std::max_element(c2.begin(), c2.end()) + 1;
    DG_CUDA(h, cudaMemcpyAsync(dcol, c2.data(), sizeof(int) * ne, cudaMemcpyHostToDevice, st));
    for (int c = 0; c < nc2; ++c)
      for (int jc = 0; jc < b1; ++jc) {
        const int jf = (jc / L1.nb) * L0.nb + jc % L1.nb;
        probe_kernel<<<grid, 256, 0, st>>>(L0.n, b0, dcol, c, jf, probe);
        DG_LAUNCH_CHECK(h);
        if ((rc = op_tangent(h, probe, out, st))) return rc;
        scatter_offdiag_kernel<<<grid, 256, 0, st>>>(ne, L0.nb, L1.nb, h->nbr, dcol, c, jc, out, L1.Bsr);
        DG_LAUNCH_CHECK(h);
      }
    for (int l = 1; l < h->nlev; ++l) {
      Level& L = h->lev[l];
      const size_t bb = (size_t)L.b * L.b;
      // diagonal: leading sub-block of the fine diagonal block
      subblock_kernel<<<grid, 256, 0, st>>>(ne, L0.nb, L.nb, L0.Dblk, (long long)b0 * b0, L.Dblk, (long long)bb);
      DG_LAUNCH_CHECK(h);
      subblock_kernel<<<grid, 256, 0, st>>>(ne, L.nb, L.nb, L.Dblk, (long long)bb, L.Bsr, (long long)bb * 7);
      DG_LAUNCH_CHECK(h);
      if (l >= 2) {
        const Level& P = h->lev[l - 1];
        for (int s = 1; s < 7; ++s) {
          subblock_kernel<<<grid, 256, 0, st>>>(ne, P.nb, L.nb, P.Bsr + (size_t)s * P.b * P.b,
                                                (long long)P.b * P.b * 7, L.Bsr + (size_t)s * bb, (long long)bb * 7);
          DG_LAUNCH_CHECK(h);
        }
      }
    }
  }
  // --- inverses
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->lev[l];
    if ((rc = invert_blocks(h, ne, L.b, L.Dblk, L.Dinv, st))) return rc;
  }
  DG_CUDA(h, cudaStreamSynchronize(st));
  unsigned s = 0;
  DG_CUDA(h, cudaMemcpy(&s, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (s & DG_STATUS_NONFINITE) return fail(h, DG_ERR_NONFINITE, "singular or non-finite element block");
  return DG_OK;
}

}  // namespace dg
