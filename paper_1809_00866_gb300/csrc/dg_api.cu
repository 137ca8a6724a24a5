// Handle management, basis/quadrature tables and the operator entry points of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "dg_internal.h"

namespace dg {

static thread_local std::string g_create_error;

int fail(Handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

// ----------------------------------------------------- host basis tables
// Legendre polynomial P_n(x) and derivative via P'_n = n (x P_n - P_{n-1}) / (x^2 - 1)
// (interior points only; the face tables evaluate values only).
static void legendre_pair(int n, double x, double* p, double* dp) {
  double pm1 = 1.0, pn = x;
  if (n == 0) { *p = 1.0; if (dp) *dp = 0.0; return; }
  for (int j = 2; j <= n; ++j) {
    const double pj = ((2 * j - 1) * x * pn - (j - 1) * pm1) / j;
    pm1 = pn;
    pn = pj;
  }
  *p = pn;
  if (dp) *dp = n * (x * pn - pm1) / (x * x - 1.0);
}

// Gauss-Legendre rule on [-1,1] (ascending nodes): Newton from Chebyshev-like guesses.
static void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double t = -std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    double p, dp;
    for (int it = 0; it < 60; ++it) {
      legendre_pair(n, t, &p, &dp);
      const double step = p / dp;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    legendre_pair(n, t, &p, &dp);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

static double phat1(int n, double x) {
  double p;
  legendre_pair(n, x, &p, nullptr);
  return std::sqrt((2.0 * n + 1.0) * 0.5) * p;
}

// Hierarchical ordering of the total-degree modes: degree 0, 1, ..., k; within a
// degree the x exponent descending, then the y exponent descending.
static std::vector<int> mode_list(int k) {
  std::vector<int> m;
  for (int t = 0; t <= k; ++t)
    for (int a = t; a >= 0; --a)
      for (int b = t - a; b >= 0; --b) {
        m.push_back(a);
        m.push_back(b);
        m.push_back(t - a - b);
      }
  return m;
}

template <class T>
static int upload(Handle* h, T** dst, const std::vector<T>& src) {
  DG_CUDA(h, cudaMalloc((void**)dst, sizeof(T) * (src.empty() ? 1 : src.size())));
  if (!src.empty()) DG_CUDA(h, cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return DG_OK;
}

static int build_tables(Handle* h, int k) {
  Tables& T = h->tab;
  T.k = k;
  T.nb = nb_of(k);
  T.n1 = k + 1;
  T.nq = T.n1 * T.n1 * T.n1;
  T.nqf = T.n1 * T.n1;
  const int nb = T.nb, n1 = T.n1;
  std::vector<double> xg, wg;
  gauss_rule(n1, xg, wg);
  const std::vector<int> md = mode_list(k);
  std::vector<double> Bv((size_t)T.nq * nb), wv(T.nq);
  for (int q0 = 0; q0 < n1; ++q0)
    for (int q1 = 0; q1 < n1; ++q1)
      for (int q2 = 0; q2 < n1; ++q2) {
        const int q = (q0 * n1 + q1) * n1 + q2;
        wv[q] = wg[q0] * wg[q1] * wg[q2];
        const double xi[3] = {xg[q0], xg[q1], xg[q2]};
        for (int m = 0; m < nb; ++m)
          Bv[(size_t)q * nb + m] = phat1(md[3 * m], xi[0]) * phat1(md[3 * m + 1], xi[1]) * phat1(md[3 * m + 2], xi[2]);
      }
  // d/dxi P_hat_a = sum_{a' < a, a - a' odd} sqrt((2a+1)(2a'+1)) P_hat_a'
  const int W = Tables::kDw;
  std::vector<int> ri((size_t)3 * nb * W, 0), ci((size_t)3 * nb * W, 0);
  std::vector<double> rv((size_t)3 * nb * W, 0.0), cv((size_t)3 * nb * W, 0.0);
  std::vector<int> rc((size_t)3 * nb, 0), cc((size_t)3 * nb, 0);
  for (int b = 0; b < 3; ++b)
    for (int n = 0; n < nb; ++n)
      for (int m = 0; m < nb; ++m) {
        bool same = true;
        for (int t = 0; t < 3; ++t)
          if (t != b && md[3 * m + t] != md[3 * n + t]) same = false;
        const int an = md[3 * n + b], am = md[3 * m + b];
        if (!same || am >= an || ((an - am) & 1) == 0) continue;
        const double val = std::sqrt((2.0 * an + 1.0) * (2.0 * am + 1.0));
        int& r = rc[b * nb + m];
        int& c = cc[b * nb + n];
        if (r >= W || c >= W) return fail(h, DG_ERR_ARG, "derivative table width exceeded");
        ri[((size_t)b * nb + m) * W + r] = n;
        rv[((size_t)b * nb + m) * W + r] = val;
        ++r;
        ci[((size_t)b * nb + n) * W + c] = m;
        cv[((size_t)b * nb + n) * W + c] = val;
        ++c;
      }
  // 1D values, 2D trace modes and the maps between 3D and face modes
  const int k1 = k + 1;
  T.n2 = k1 * (k + 2) / 2;
  const int n2 = T.n2;
  std::vector<double> L1((size_t)k1 * n1), pvv(2 * k1), pdv(2 * k1);
  for (int a = 0; a <= k; ++a) {
    for (int q = 0; q < n1; ++q) L1[(size_t)a * n1 + q] = phat1(a, xg[q]);
    const double na = std::sqrt((2.0 * a + 1.0) * 0.5);
    const double der = na * a * (a + 1) * 0.5;  // P_a'(1) = a(a+1)/2
    pvv[a] = na;
    pvv[k1 + a] = (a & 1) ? -na : na;
    pdv[a] = der;
    pdv[k1 + a] = (a & 1) ? der : -der;  // P_a'(-1) = (-1)^(a+1) a(a+1)/2
  }
  std::vector<int> pab, pidx((size_t)k1 * k1, -1);
  for (int t = 0; t <= k; ++t)
    for (int a = t; a >= 0; --a) {
      pidx[a * k1 + (t - a)] = (int)(pab.size() / 2);
      pab.push_back(a);
      pab.push_back(t - a);
    }
  std::vector<double> B2((size_t)T.nqf * n2), W2(T.nqf);
  for (int q1 = 0; q1 < n1; ++q1)
    for (int q2 = 0; q2 < n1; ++q2) {
      const int q = q1 * n1 + q2;
      W2[q] = wg[q1] * wg[q2];
      for (int j = 0; j < n2; ++j) B2[(size_t)q * n2 + j] = phat1(pab[2 * j], xg[q1]) * phat1(pab[2 * j + 1], xg[q2]);
    }
  std::vector<int> M3((size_t)3 * n2 * k1, -1), fmap((size_t)3 * nb), fa((size_t)3 * nb), md3((size_t)nb * 3);
  for (int m = 0; m < nb; ++m)
    for (int t = 0; t < 3; ++t) md3[3 * m + t] = md[3 * m + t];
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < nb; ++m) {
      const int a = md[3 * m + d], b = md[3 * m + (d + 1) % 3], c = md[3 * m + (d + 2) % 3];
      const int j = pidx[b * k1 + c];
      fmap[(size_t)d * nb + m] = j;
      fa[(size_t)d * nb + m] = a;
      M3[((size_t)d * n2 + j) * k1 + a] = m;
    }
  std::vector<int> d2i((size_t)2 * n2 * W, 0), d2c((size_t)2 * n2, 0);
  std::vector<double> d2v((size_t)2 * n2 * W, 0.0);
  for (int dir = 0; dir < 2; ++dir)
    for (int jo = 0; jo < n2; ++jo)
      for (int ji = 0; ji < n2; ++ji) {
        const int bo = pab[2 * jo + dir], co = pab[2 * jo + 1 - dir];
        const int bi = pab[2 * ji + dir], ci2 = pab[2 * ji + 1 - dir];
        if (co != ci2 || bo >= bi || ((bi - bo) & 1) == 0) continue;
        int& r = d2c[dir * n2 + jo];
        if (r >= W) return fail(h, DG_ERR_ARG, "2D derivative table width exceeded");
        d2i[((size_t)dir * n2 + jo) * W + r] = ji;
        d2v[((size_t)dir * n2 + jo) * W + r] = std::sqrt((2.0 * bi + 1.0) * (2.0 * bo + 1.0));
        ++r;
      }
  int rcode;
  if ((rcode = upload(h, &T.Bvol, Bv)) || (rcode = upload(h, &T.wvol, wv)) || (rcode = upload(h, &T.xg, xg)) ||
      (rcode = upload(h, &T.Drow_idx, ri)) || (rcode = upload(h, &T.Drow_val, rv)) ||
      (rcode = upload(h, &T.Dcol_idx, ci)) || (rcode = upload(h, &T.Dcol_val, cv)) ||
      (rcode = upload(h, &T.L1, L1)) || (rcode = upload(h, &T.B2, B2)) || (rcode = upload(h, &T.W2, W2)) ||
      (rcode = upload(h, &T.pv, pvv)) || (rcode = upload(h, &T.pd, pdv)) || (rcode = upload(h, &T.M3, M3)) ||
      (rcode = upload(h, &T.fmap, fmap)) || (rcode = upload(h, &T.fa, fa)) || (rcode = upload(h, &T.md3, md3)) ||
      (rcode = upload(h, &T.pidx, pidx)) || (rcode = upload(h, &T.pab, pab)) || (rcode = upload(h, &T.D2_idx, d2i)) ||
      (rcode = upload(h, &T.D2_val, d2v)))
    return rcode;
  auto tof = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
  TablesF& TF = h->tabf;
  if ((rcode = upload(h, &TF.Bvol, tof(Bv))) || (rcode = upload(h, &TF.L1, tof(L1))) || (rcode = upload(h, &TF.wvol, tof(wv))) ||
      (rcode = upload(h, &TF.B2, tof(B2))) || (rcode = upload(h, &TF.W2, tof(W2))) ||
      (rcode = upload(h, &TF.pv, tof(pvv))) || (rcode = upload(h, &TF.pd, tof(pdv))) ||
      (rcode = upload(h, &TF.Drow_val, tof(rv))) || (rcode = upload(h, &TF.Dcol_val, tof(cv))) ||
      (rcode = upload(h, &TF.D2_val, tof(d2v))))
    return rcode;
  return DG_OK;
}

__global__ void or_status_kernel(unsigned* status, unsigned bits) { atomicOr(status, bits); }

template <class T>
static int dalloc(Handle* h, T** p, size_t count) {
  DG_CUDA(h, cudaMalloc((void**)p, sizeof(T) * (count ? count : 1)));
  DG_CUDA(h, cudaMemset(*p, 0, sizeof(T) * (count ? count : 1)));
  return DG_OK;
}

cudaEvent_t prof_event(Handle* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int prof_begin(Handle* h, cudaStream_t st, cudaEvent_t* a) {
  *a = nullptr;
  if (!h->prof) return DG_OK;
  *a = prof_event(h);
  if (!*a) return fail(h, DG_ERR_CUDA, "cudaEventCreate failed");
  DG_CUDA(h, cudaEventRecord(*a, st));
  return DG_OK;
}

int prof_end(Handle* h, int cls, cudaStream_t st, cudaEvent_t a, double bytes) {
  if (!h->prof || !a) return DG_OK;
  cudaEvent_t b = prof_event(h);
  if (!b) return fail(h, DG_ERR_CUDA, "cudaEventCreate failed");
  DG_CUDA(h, cudaEventRecord(b, st));
  h->prof_pending.push_back(Handle::ProfEv{cls, a, b, bytes});
  return DG_OK;
}

static void free_all(Handle* h) {
  for (auto& p : h->prof_pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  h->prof_pending.clear();
  h->ev_pool.clear();
  auto F = [](void* p) { if (p) cudaFree(p); };
  Tables& T = h->tab;
  F(T.Bvol); F(T.wvol); F(T.xg); F(T.Drow_idx); F(T.Drow_val); F(T.Dcol_idx); F(T.Dcol_val);
  F(T.L1); F(T.B2); F(T.W2); F(T.pv); F(T.pd); F(T.M3); F(T.fmap); F(T.fa); F(T.md3); F(T.pidx); F(T.pab);
  F(T.D2_idx); F(T.D2_val);
  TablesF& TF = h->tabf;
  F(TF.Bvol); F(TF.L1); F(TF.wvol); F(TF.B2); F(TF.W2); F(TF.pv); F(TF.pd); F(TF.Drow_val); F(TF.Dcol_val); F(TF.D2_val);
  F(h->face_out_f); F(h->face_lift_f); F(h->ubar_f); F(h->dFlux_f);
  F(h->tc_tab[0]); F(h->tc_tab[1]); F(h->ubar_scale);
  for (int d = 0; d < 3; ++d) F(h->dnode[d]);
  F(h->geo);
  F(h->geof);
  F(h->nbr);
  F(h->elem_prob); F(h->dshift); F(h->chunk); F(h->chunk_prob); F(h->pchunk0); F(h->bface); F(h->bslot);
  F(h->colour);
  for (int l = 0; l < DG_MAX_LEVELS; ++l) {
    F(h->lev[l].Dblk); F(h->lev[l].Dinv); F(h->lev[l].Bsr); F(h->lev[l].t0); F(h->lev[l].t1); F(h->lev[l].t2);
    F(h->lev[l].Dlin); F(h->lev[l].Blin); F(h->lev[l].perm);
    F(h->lev[l].LUf); F(h->lev[l].Bsrf); F(h->lev[l].t0f); F(h->lev[l].t1f); F(h->lev[l].t2f);
    F(h->lev[l].LU16); F(h->lev[l].Bsr16);
  }
  F(h->face_out); F(h->face_lift); F(h->wlin); F(h->flin); F(h->ubar); F(h->dFlux); F(h->wnorm2);
  F(h->fd_w); F(h->fd_f); F(h->red); F(h->red_out); F(h->status); F(h->V); F(h->Z); F(h->hcol);
  if (h->hcol_host) cudaFreeHost(h->hcol_host);
  for (int l = 0; l < DG_MAX_LEVELS; ++l) F(h->smV[l]);
  F(h->smSmall);
  F(h->stb1);
  F(h->stb1f);
  F(h->net);
}

__global__ void write_shifts_kernel(int ne, const int* elem_prob, const double* shift, double* geo, float* geof) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    geo[(size_t)e * kGeo + 11] = shift[elem_prob[e]];
    geof[(size_t)e * kGeo + 11] = (float)shift[elem_prob[e]];
  }
}

static int write_shifts(Handle* h, cudaStream_t st) {
  write_shifts_kernel<<<(h->ne + 255) / 256, 256, 0, st>>>(h->ne, h->elem_prob, h->dshift, h->geo, h->geof);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// One periodic box of a handle: cells per axis and host node coordinates per axis.
struct Box {
  int n[3];
  const double* node[3];
};

// Reduction chunks of about kChunkDoubles level-0 entries, never across two problems.
constexpr int kChunkDoubles = 2048;

static int create(const dg_params* p, const std::vector<Box>& boxes, Handle* h) {
  if (!p) return fail(h, DG_ERR_ARG, "null params");
  if (boxes.empty()) return fail(h, DG_ERR_ARG, "no problem");
  long long ne = 0;
  for (const Box& bx : boxes) {
    for (int d = 0; d < 3; ++d) {
      if (bx.n[d] < 2) return fail(h, DG_ERR_ARG, "every axis needs at least 2 cells");
      if (!bx.node[d]) return fail(h, DG_ERR_ARG, "null node array");
      for (int i = 0; i < bx.n[d]; ++i)
        if (!(bx.node[d][i + 1] > bx.node[d][i])) return fail(h, DG_ERR_ARG, "node coordinates must increase");
    }
    ne += (long long)bx.n[0] * bx.n[1] * bx.n[2];
    if (ne > (1LL << 28)) return fail(h, DG_ERR_ARG, "mesh too large");
  }
  if (p->nlevels < 1 || p->nlevels > DG_MAX_LEVELS) return fail(h, DG_ERR_ARG, "nlevels out of range");
  for (int l = 0; l < p->nlevels; ++l) {
    if (p->k[l] < 1 || p->k[l] > kMaxK) return fail(h, DG_ERR_ARG, "degree out of range 1..4");
    if (l > 0 && p->k[l] >= p->k[l - 1]) return fail(h, DG_ERR_ARG, "degrees must decrease with the level");
  }
  if (!(p->nu > 0.0) || !(p->ac_c > 0.0) || !(p->eta > 0.0)) return fail(h, DG_ERR_ARG, "nu, ac_c, eta must be > 0");
  if (p->walls != DG_WALLS_NONE && p->walls != DG_WALLS_Y) return fail(h, DG_ERR_ARG, "unknown walls flag");
  const bool walls = p->walls == DG_WALLS_Y;
  for (const Box& bx : boxes)
    if (walls && bx.n[1] < 2) return fail(h, DG_ERR_ARG, "walls need at least 2 cells across the channel");
  h->p = *p;
  h->p.xn = h->p.yn = h->p.zn = nullptr;
  h->nprob = (int)boxes.size();
  for (int d = 0; d < 3; ++d) h->n[d] = h->nprob == 1 ? boxes[0].n[d] : 0;  // structured sizes: single box only
  h->ne = (int)ne;
  h->nlev = p->nlevels;
  int dev = 0;
  DG_CUDA(h, cudaGetDevice(&dev));
  h->device = dev;
  DG_CUDA(h, cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
  int rc;
  if (h->nprob == 1)
    for (int d = 0; d < 3; ++d) h->node[d].assign(boxes[0].node[d], boxes[0].node[d] + boxes[0].n[d] + 1);
  // elements problem by problem, x fastest within a box; periodic neighbours within the box
  h->pe0.assign(h->nprob + 1, 0);
  std::vector<int>& nbr = h->nbr_host;
  nbr.assign((size_t)ne * 6, 0);
  std::vector<int> eprob((size_t)ne);
  std::vector<int> bface, bslot((size_t)ne, -1);
  std::vector<double> geo((size_t)ne * kGeo, 0.0);
  for (int q = 0; q < h->nprob; ++q) {
    const Box& bx = boxes[q];
    const int* nn = bx.n;
    const long long e0 = h->pe0[q], nq = (long long)nn[0] * nn[1] * nn[2];
    h->pe0[q + 1] = (int)(e0 + nq);
    for (long long el = 0; el < nq; ++el) {
      const long long e = e0 + el;
      const int I[3] = {(int)(el % nn[0]), (int)((el / nn[0]) % nn[1]), (int)(el / ((long long)nn[0] * nn[1]))};
      auto id = [&](int a, int b, int c) {
        a = (a + nn[0]) % nn[0]; b = (b + nn[1]) % nn[1]; c = (c + nn[2]) % nn[2];
        return (int)(e0 + a + nn[0] * (b + nn[1] * c));
      };
      nbr[e * 6 + 0] = id(I[0] - 1, I[1], I[2]); nbr[e * 6 + 1] = id(I[0] + 1, I[1], I[2]);
      nbr[e * 6 + 2] = id(I[0], I[1] - 1, I[2]); nbr[e * 6 + 3] = id(I[0], I[1] + 1, I[2]);
      nbr[e * 6 + 4] = id(I[0], I[1], I[2] - 1); nbr[e * 6 + 5] = id(I[0], I[1], I[2] + 1);
      if (walls && I[1] == 0) {  // the wall below: no neighbour, one extra face
        nbr[e * 6 + 2] = -1;
        bslot[e] = (int)bface.size();
        bface.push_back((int)e);
      }
      if (walls && I[1] == nn[1] - 1) nbr[e * 6 + 3] = -1;
      eprob[e] = q;
      double* G = &geo[(size_t)e * kGeo];
      for (int d = 0; d < 3; ++d) {
        G[d] = bx.node[d][I[d] + 1] - bx.node[d][I[d]];
        G[5 + d] = 2.0 / G[d];
        G[8 + d] = bx.node[d][I[d]];
      }
      G[3] = std::sqrt(G[0] * G[1] * G[2] * 0.125);
      G[4] = 1.0 / G[3];
      G[11] = 1.0;
    }
  }
  if ((rc = upload(h, &h->nbr, nbr))) return rc;
  h->nbf = (int)bface.size();
  if ((rc = upload(h, &h->bface, bface)) || (rc = upload(h, &h->bslot, bslot))) return rc;
  if ((rc = upload(h, &h->elem_prob, eprob))) return rc;
  if ((rc = upload(h, &h->dshift, std::vector<double>(h->nprob, 1.0)))) return rc;
  {
    const int b0 = 4 * nb_of(p->k[0]);
    const int ce = std::max(1, kChunkDoubles / b0);
    std::vector<int2> ch;
    std::vector<int> cp, pc0(h->nprob + 1, 0);
    for (int q = 0; q < h->nprob; ++q) {
      pc0[q] = (int)ch.size();
      for (int e = h->pe0[q]; e < h->pe0[q + 1]; e += ce) {
        ch.push_back(make_int2(e, std::min(e + ce, h->pe0[q + 1])));
        cp.push_back(q);
      }
    }
    pc0[h->nprob] = (int)ch.size();
    h->nchunk = (int)ch.size();
    if ((rc = upload(h, &h->chunk, ch)) || (rc = upload(h, &h->chunk_prob, cp)) || (rc = upload(h, &h->pchunk0, pc0)))
      return rc;
  }
  if ((rc = upload(h, &h->geo, geo))) return rc;
  {
    const std::vector<float> geof(geo.begin(), geo.end());
    if ((rc = upload(h, &h->geof, geof))) return rc;
  }
  if ((rc = build_tables(h, p->k[0]))) return rc;
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->lev[l];
    L.k = p->k[l];
    L.nb = nb_of(L.k);
    L.b = 4 * L.nb;
    L.n = ne * L.b;
    if ((rc = dalloc(h, &L.t0, L.n)) || (rc = dalloc(h, &L.t1, L.n)) || (rc = dalloc(h, &L.t2, L.n))) return rc;
  }
  const long long n0 = h->lev[0].n;
  const int n2f = h->tab.n2;
  if ((rc = dalloc(h, &h->face_out, (size_t)ne * 6 * 4 * n2f)) || (rc = dalloc(h, &h->face_lift, (size_t)ne * 6 * 3 * n2f)) ||
      (rc = dalloc(h, &h->wlin, n0)) || (rc = dalloc(h, &h->flin, n0)) || (rc = dalloc(h, &h->fd_w, n0)) ||
      (rc = dalloc(h, &h->fd_f, n0)) || (rc = dalloc(h, &h->ubar, (size_t)ne * 3 * h->tab.nq)) ||
      (rc = dalloc(h, &h->dFlux, (size_t)(3 * ne + h->nbf) * h->tab.nqf * 32)) || (rc = dalloc(h, &h->wnorm2, 1)) ||
      (rc = dalloc(h, &h->red, 4096)) || (rc = dalloc(h, &h->red_out, 8)) || (rc = dalloc(h, &h->status, 3)))
    return rc;
  if ((rc = dalloc(h, &h->face_out_f, (size_t)ne * 6 * 4 * n2f)) ||
      (rc = dalloc(h, &h->face_lift_f, (size_t)ne * 6 * 3 * n2f)) ||
      (rc = dalloc(h, &h->ubar_f, (size_t)ne * 3 * h->tab.nq)) ||
      (rc = dalloc(h, &h->dFlux_f, (size_t)(3 * ne + h->nbf) * h->tab.nqf * 32)))
    return rc;
  DG_CUDA(h, cudaDeviceSynchronize());
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" {

int dg_create(const dg_params* p, dg_handle** out) {
  if (!out) return fail(nullptr, DG_ERR_ARG, "null output handle pointer");
  *out = nullptr;
  Handle* h = new (std::nothrow) Handle();
  if (!h) return fail(nullptr, DG_ERR_ARG, "out of host memory");
  std::vector<Box> boxes;
  if (p) boxes.push_back(Box{{p->nx, p->ny, p->nz}, {p->xn, p->yn, p->zn}});
  const int rc = create(p, boxes, h);
  if (rc != DG_OK) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return rc;
  }
  *out = reinterpret_cast<dg_handle*>(h);
  return DG_OK;
}

int dg_create_batch(const dg_params* p, int nprob, const int* dims, const double* nodes, dg_handle** out) {
  if (!out) return fail(nullptr, DG_ERR_ARG, "null output handle pointer");
  *out = nullptr;
  if (!p || nprob < 1 || !dims || !nodes) return fail(nullptr, DG_ERR_ARG, "null argument or nprob < 1");
  std::vector<Box> boxes((size_t)nprob);
  size_t off = 0;
  for (int q = 0; q < nprob; ++q)
    for (int d = 0; d < 3; ++d) {
      boxes[q].n[d] = dims[3 * q + d];
      if (boxes[q].n[d] < 2) return fail(nullptr, DG_ERR_ARG, "every axis needs at least 2 cells");
      boxes[q].node[d] = nodes + off;
      off += (size_t)boxes[q].n[d] + 1;
    }
  Handle* h = new (std::nothrow) Handle();
  if (!h) return fail(nullptr, DG_ERR_ARG, "out of host memory");
  const int rc = create(p, boxes, h);
  if (rc != DG_OK) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return rc;
  }
  *out = reinterpret_cast<dg_handle*>(h);
  return DG_OK;
}

int dg_problems(const dg_handle* hh, int* nprob, int* elem_start) {
  const Handle* h = reinterpret_cast<const Handle*>(hh);
  if (!h || !nprob) return DG_ERR_ARG;
  *nprob = h->nprob;
  if (elem_start)
    for (int q = 0; q <= h->nprob; ++q) elem_start[q] = h->pe0[q];
  return DG_OK;
}

int dg_set_problem_shifts(dg_handle* hh, const double* mult, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!mult) return fail(h, DG_ERR_ARG, "null multipliers");
  for (int q = 0; q < h->nprob; ++q)
    if (!(mult[q] >= 0.0) || !std::isfinite(mult[q])) return fail(h, DG_ERR_ARG, "multipliers must be finite and >= 0");
  cudaStream_t st = as_stream(stream);
  DG_CUDA(h, cudaMemcpyAsync(h->dshift, mult, sizeof(double) * h->nprob, cudaMemcpyHostToDevice, st));
  if (int rc = write_shifts(h, st)) return rc;
  DG_CUDA(h, cudaStreamSynchronize(st));
  h->assembled = h->asm64_ready = h->asm_f_ready = false;  // the blocks hold the shift
  h->asm16 = 0;
  return DG_OK;
}

int dg_destroy(dg_handle* hh) {
  if (!hh) return DG_OK;
  Handle* h = reinterpret_cast<Handle*>(hh);
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return DG_OK;
}

int dg_set_stb_rescaling(dg_handle* hh, int enable) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (enable && h->nlev < 2) return fail(h, DG_ERR_ARG, "the rescaling acts on coarse levels: needs two or more");
  h->stb_rescale = enable != 0;
  h->assembled = h->asm64_ready = h->asm_f_ready = false;  // the coarse operators change
  h->asm16 = 0;
  return DG_OK;
}

int dg_reuse_assembly(dg_handle* hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!h->asm64_ready && !h->asm_f_ready) return fail(h, DG_ERR_STATE, "no assembled preconditioner to reuse");
  if (!h->linearized) return fail(h, DG_ERR_STATE, "dg_reuse_assembly needs dg_set_linearization first");
  h->assembled = true;
  return DG_OK;
}

const char* dg_last_error(const dg_handle* hh) {
  if (!hh) return g_create_error.c_str();
  return reinterpret_cast<const Handle*>(hh)->err.c_str();
}

int dg_level_size(const dg_handle* hh, int lvl, int* nb, long long* n) {
  const Handle* h = reinterpret_cast<const Handle*>(hh);
  if (!h || lvl < 0 || lvl >= h->nlev) return DG_ERR_ARG;
  if (nb) *nb = h->lev[lvl].nb;
  if (n) *n = h->lev[lvl].n;
  return DG_OK;
}

int dg_set_test_knob(dg_handle* hh, int knob, long long value) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  switch (knob) {
    case DG_KNOB_RIEMANN_ITS:
      if (value < 0 || value > 1000) return fail(h, DG_ERR_ARG, "Riemann iteration cap: 0..1000");
      h->dbg.riemann_its = (int)value;
      return DG_OK;
    case DG_KNOB_WAIT_POLLS:
      if (value < 0 || value > (1ll << 30)) return fail(h, DG_ERR_ARG, "wait polls: 0..2^30");
      h->dbg.wait_polls = (int)value;
      return DG_OK;
    case DG_KNOB_WITHHOLD_COPY:
      h->dbg.withhold_copy = value != 0;
      return DG_OK;
  }
  return fail(h, DG_ERR_ARG, "unknown test knob");
}

int dg_get_status(dg_handle* hh, unsigned* status, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !status) return DG_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  DG_CUDA(h, cudaMemcpyAsync(status, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  DG_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned), st));
  DG_CUDA(h, cudaStreamSynchronize(st));
  return DG_OK;
}

int dg_project_tgv(dg_handle* hh, double* w, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !w) return h ? fail(h, DG_ERR_ARG, "null pointer") : DG_ERR_ARG;
  return op_project_tgv(h, w, as_stream(stream));
}

int dg_quad_points(dg_handle* hh, double* xyz, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !xyz) return h ? fail(h, DG_ERR_ARG, "null pointer") : DG_ERR_ARG;
  return op_quad_points(h, xyz, as_stream(stream));
}

int dg_project_points(dg_handle* hh, const double* vals, double* w, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !vals || !w) return h ? fail(h, DG_ERR_ARG, "null pointer") : DG_ERR_ARG;
  return op_project_points(h, vals, w, as_stream(stream));
}

int dg_residual(dg_handle* hh, const double* w, double* f, void* stream) {
  const dg::NvtxRange nvtx_range_("dg_residual");
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!w || !f || w == f) return fail(h, DG_ERR_ARG, "w and f must be distinct non-null device pointers");
  return op_residual(h, w, f, false, as_stream(stream));
}

int dg_set_linearization(dg_handle* hh, const double* w, double inv_gamma_dt, void* stream) {
  const dg::NvtxRange nvtx_range_("dg_set_linearization");
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!w || !(inv_gamma_dt >= 0.0)) return fail(h, DG_ERR_ARG, "null state or negative 1/(gamma dt)");
  cudaStream_t st = as_stream(stream);
  const long long n0 = h->lev[0].n;
  DG_CUDA(h, cudaMemcpyAsync(h->wlin, w, sizeof(double) * n0, cudaMemcpyDeviceToDevice, st));
  h->inv_gdt = inv_gamma_dt;
  h->linearized = false;
  DG_CUDA(h, cudaMemsetAsync(h->status + 1, 0, sizeof(unsigned), st));
  int rc = op_residual(h, h->wlin, h->flin, true, st);  // records its conditions in status[1]
  if (rc) return rc;
  if ((rc = vec_norm2(h, h->wlin, n0, h->wnorm2, st))) return rc;
  unsigned s = 0;
  double wn2 = 0.0;
  DG_CUDA(h, cudaMemcpyAsync(&s, h->status + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  DG_CUDA(h, cudaMemcpyAsync(&wn2, h->wnorm2, sizeof(double), cudaMemcpyDeviceToHost, st));
  DG_CUDA(h, cudaStreamSynchronize(st));
  if (!std::isfinite(wn2)) s |= DG_STATUS_NONFINITE;
  if (s) {  // keep the conditions for dg_get_status as well
    or_status_kernel<<<1, 1, 0, st>>>(h->status, s);
    DG_LAUNCH_CHECK(h);
  }
  h->assembled = false;
  h->lin_f_ready = false;
  if (s & DG_STATUS_NONFINITE) return fail(h, DG_ERR_NONFINITE, "non-finite state or residual at the linearisation");
  if (s & DG_STATUS_RIEMANN)
    return fail(h, DG_ERR_RIEMANN, "the star-state iteration of the Riemann solver did not converge on some face");
  h->linearized = true;
  return DG_OK;
}

int dg_set_linearization_rhs(dg_handle* hh, const double* w, double inv_gamma_dt, double* g, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!g || g == w) return fail(h, DG_ERR_ARG, "g must be a non-null device pointer distinct from w");
  int rc = dg_set_linearization(hh, w, inv_gamma_dt, stream);
  if (rc) return rc;
  return launch_axpby(h, h->lev[0].n, -1.0, h->flin, 0.0, g, as_stream(stream));  // g = -f_h(w)
}

int dg_stage_update(dg_handle* hh, double* w, const double* dw, double b, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!w || !dw || w == dw) return fail(h, DG_ERR_ARG, "w and dw must be distinct non-null device pointers");
  return launch_axpby(h, h->lev[0].n, b, dw, 1.0, w, as_stream(stream));  // w = b dw + w
}

int dg_jvp(dg_handle* hh, const double* v, double* out, int mode, void* stream) {
  const dg::NvtxRange nvtx_range_("dg_jvp");
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!v || !out || v == out) return fail(h, DG_ERR_ARG, "v and out must be distinct non-null device pointers");
  if (!h->linearized) return fail(h, DG_ERR_STATE, "dg_jvp needs dg_set_linearization first");
  if (mode == DG_JVP_TANGENT) return op_tangent(h, v, out, as_stream(stream));
  if (mode == DG_JVP_FD) {
    if (h->nprob > 1) return fail(h, DG_ERR_ARG, "the FD step size is global: one problem per handle only");
    return op_fd(h, v, out, as_stream(stream));
  }
  return fail(h, DG_ERR_ARG, "unknown jvp mode");
}

int dg_assemble_precision(dg_handle* hh, int precision, void* stream) {
  const dg::NvtxRange nvtx_range_("dg_assemble");
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!h->linearized) return fail(h, DG_ERR_STATE, "dg_assemble needs dg_set_linearization first");
  if (precision == DG_PRECOND_FP32_H16 || precision == DG_PRECOND_FP32_BF16 || precision == DG_PRECOND_FP32_H16_TC ||
      precision == DG_PRECOND_FP32_BF16_TC)
    precision = DG_PRECOND_FP32;  // the 16-bit copies are rounded from the FP32 assembly at first use
  if (precision != DG_PRECOND_FP64 && precision != DG_PRECOND_FP32) return fail(h, DG_ERR_ARG, "unknown precision");
  h->assembled = h->asm64_ready = h->asm_f_ready = false;
  h->asm16 = 0;
  const int rc = assemble_all(h, precision, as_stream(stream));
  if (rc == DG_OK) {
    h->assembled = true;
    h->asm64_ready = precision == DG_PRECOND_FP64;
    h->asm_f_ready = precision == DG_PRECOND_FP32;
  }
  return rc;
}

int dg_assemble(dg_handle* hh, void* stream) { return dg_assemble_precision(hh, DG_PRECOND_FP64, stream); }

int dg_counters(const dg_handle* hh, long long* kernel_launches, long long* operator_applications) {
  const Handle* h = reinterpret_cast<const Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (kernel_launches) *kernel_launches = h->launches;
  if (operator_applications) *operator_applications = h->op_apps;
  return DG_OK;
}

int dg_profile(dg_handle* hh, int enable) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  h->prof = enable != 0;
  return DG_OK;
}

int dg_profile_read(dg_handle* hh, double* ms, long long* counts) {
  return dg_profile_read_bytes(hh, ms, counts, nullptr);
}

int dg_profile_read_bytes(dg_handle* hh, double* ms, long long* counts, double* bytes) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || !ms || !counts) return h ? fail(h, DG_ERR_ARG, "null output") : DG_ERR_ARG;
  DG_CUDA(h, cudaDeviceSynchronize());
  for (auto& p : h->prof_pending) {
    float t = 0.f;
    DG_CUDA(h, cudaEventElapsedTime(&t, p.a, p.b));
    h->prof_ms[p.cls] += t;
    h->prof_cnt[p.cls] += 1;
    h->prof_bytes[p.cls] += p.bytes;
    h->ev_pool.push_back(p.a);
    h->ev_pool.push_back(p.b);
  }
  h->prof_pending.clear();
  for (int i = 0; i < DG_PROF_N; ++i) {
    ms[i] = h->prof_ms[i];
    counts[i] = h->prof_cnt[i];
    if (bytes) bytes[i] = h->prof_bytes[i];
    h->prof_ms[i] = 0.0;
    h->prof_cnt[i] = 0;
    h->prof_bytes[i] = 0.0;
  }
  return DG_OK;
}

}  // extern "C"
