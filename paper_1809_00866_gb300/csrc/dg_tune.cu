// Launch-shape tuning of the hot kernels per (degree k, quadrature size N_q): the faces per CTA
// of the face pass, the threads per CTA of the volume pass, the CTAs per SM of both, and the
// element blocks staged per bulk copy of the FP32 block-Jacobi apply. The paper's CPU code has no
// counterpart; on a GPU the best shapes depend on k (the shared-memory footprint of a face or an
// element grows with N_b and N_q) and on the mesh size (grid fill), so they are measured on the
// handle itself: every candidate runs the real kernels on the handle's current linearisation and
// the fastest per kernel is kept. Results are cached per (precision, k, N_q, SM count, log2 N_e)
// for the process, so handles of the same shape (a batch of boxes) tune once.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "dg_internal.h"

namespace dg {

template <class R>
__global__ void tune_fill_kernel(long long n, R* x, double phase) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = R(sin(0.37 * (double)i + phase) * 0.01);
}

using TuneKey = std::tuple<int, int, int, int, int, int>;  // precision, k, N_q, SMs, log2 N_e, block storage
static std::map<TuneKey, OpTune> g_tune_cache;
static std::mutex g_tune_mu;

static int ilog2(long long v) {
  int r = 0;
  while (v > 1) { v >>= 1; ++r; }
  return r;
}

static int valid(const dg_tuning* t) {
  return t && (t->face_warps == 2 || t->face_warps == 4 || t->face_warps == 8) &&
         (t->vol_threads == 64 || t->vol_threads == 128 || t->vol_threads == 160 || t->vol_threads == 192 ||
          t->vol_threads == 256) && t->face_ctas_per_sm >= 0 &&
         t->face_ctas_per_sm <= 32 && t->vol_ctas_per_sm >= 0 && t->vol_ctas_per_sm <= 32 &&
         t->jacobi_stage_kb >= 8 && t->jacobi_stage_kb <= 224 && t->jacobi_max_ctas >= 0 &&
         t->jacobi_max_ctas <= 4096;
}

static OpTune from_abi(const dg_tuning& t) {
  OpTune o;
  o.face_warps = t.face_warps;
  o.vol_threads = t.vol_threads;
  o.face_per_sm = t.face_ctas_per_sm;
  o.vol_per_sm = t.vol_ctas_per_sm;
  o.jacobi_stage_kb = t.jacobi_stage_kb;
  o.jacobi_max_ctas = t.jacobi_max_ctas;
  return o;
}

static dg_tuning to_abi(const OpTune& o) {
  dg_tuning t;
  t.face_warps = o.face_warps;
  t.vol_threads = o.vol_threads;
  t.face_ctas_per_sm = o.face_per_sm;
  t.vol_ctas_per_sm = o.vol_per_sm;
  t.jacobi_stage_kb = o.jacobi_stage_kb;
  t.jacobi_max_ctas = o.jacobi_max_ctas;
  return t;
}

// device milliseconds per launch of the profiled classes over `reps` calls of fn
template <class F>
static int time_classes(Handle* hh, F fn, int reps, double* ms, cudaStream_t st) {
  dg_handle* h = reinterpret_cast<dg_handle*>(hh);
  double acc[DG_PROF_N];
  long long cnt[DG_PROF_N];
  int rc;
  for (int w = 0; w < 2; ++w)
    if ((rc = fn())) return rc;
  if ((rc = dg_profile_read(h, acc, cnt))) return rc;  // drop the warm-up launches
  for (int r = 0; r < reps; ++r)
    if ((rc = fn())) return rc;
  DG_CUDA(hh, cudaStreamSynchronize(st));
  if ((rc = dg_profile_read(h, acc, cnt))) return rc;
  for (int c = 0; c < DG_PROF_N; ++c) ms[c] = cnt[c] ? acc[c] / cnt[c] : 0.0;
  return DG_OK;
}

static int autotune(Handle* h, int which, bool use_cache, double* report, cudaStream_t st) {
  const bool f32 = which == DG_TUNE_FP32;
  const int storage = f32 ? (h->asm16 ? h->asm16 : (h->asm_f_ready ? DG_PRECOND_FP32 : 0)) : 0;
  const TuneKey key{which, h->tab.k, h->tab.nq, h->nsm, ilog2(h->ne), storage};
  if (use_cache) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      h->tune[which] = it->second;
      if (report)
        for (int i = 0; i < 6; ++i) report[i] = 0.0;
      return DG_OK;
    }
  }
  if (!h->linearized) return fail(h, DG_ERR_STATE, "dg_autotune needs dg_set_linearization first");
  int rc;
  const long long n0 = h->lev[0].n;
  Level& L0 = h->lev[0];
  float *xf = nullptr, *yf = nullptr, *zf = nullptr;
  // keep the caller's profile: flush what it holds now, restore it at the end
  double saved_ms[DG_PROF_N], saved_bytes[DG_PROF_N];
  long long saved_cnt[DG_PROF_N];
  dg_handle* hh = reinterpret_cast<dg_handle*>(h);
  const bool prof_was = h->prof;
  if ((rc = dg_profile_read_bytes(hh, saved_ms, saved_cnt, saved_bytes))) return rc;
  const OpTune base = h->tune[which];
  OpTune best = base;
  double best_f = 1e30, best_v = 1e30, def_f = 0.0, def_v = 0.0, def_j = 0.0, best_j = 0.0;
  auto measure = [&]() -> int {
    int r;
    if (f32) {
      if ((r = prepare_lin_fp32(h, st))) return r;
      DG_CUDA(h, cudaMalloc((void**)&xf, sizeof(float) * n0));
      DG_CUDA(h, cudaMalloc((void**)&yf, sizeof(float) * n0));
      DG_CUDA(h, cudaMalloc((void**)&zf, sizeof(float) * n0));
      DG_CUDA(h, cudaMemsetAsync(zf, 0, sizeof(float) * n0, st));
      tune_fill_kernel<float><<<h->nsm * 4, 256, 0, st>>>(n0, xf, 0.1);
    } else {
      tune_fill_kernel<double><<<h->nsm * 4, 256, 0, st>>>(n0, L0.t0, 0.1);
    }
    DG_LAUNCH_CHECK(h);
    h->prof = true;
    auto op = [&]() -> int { return f32 ? op_tangent_f32(h, xf, yf, 0, st) : op_tangent(h, L0.t0, L0.t1, st); };
    const int cf = f32 ? DG_PROF_FACE_TAN32 : DG_PROF_FACE_TAN, cv = f32 ? DG_PROF_VOL_TAN32 : DG_PROF_VOL_TAN;
    const int face_w[3] = {2, 4, 8};
    // 160 threads: one pass over the 4 N_b outputs of the last volume phase at P4 (140)
    const int vol_t[5] = {64, 128, 160, 192, 256};
    const int vol_cap[2] = {0, 4};
    double ms[DG_PROF_N];
    // ten operator configurations: face shape i % 3 (timed for i < 3), volume shape i
    for (int i = 0; i < 10; ++i) {
      OpTune t = base;
      t.face_warps = face_w[i % 3];
      t.face_per_sm = 0;
      t.vol_threads = vol_t[i % 5];
      t.vol_per_sm = vol_cap[i / 5];
      h->tune[which] = t;
      if ((r = time_classes(h, op, 5, ms, st))) return r;
      if (i < 3 && ms[cf] < best_f) { best_f = ms[cf]; best.face_warps = t.face_warps; best.face_per_sm = 0; }
      if (ms[cv] < best_v) { best_v = ms[cv]; best.vol_threads = t.vol_threads; best.vol_per_sm = t.vol_per_sm; }
      if (t.face_warps == 4 && i < 3) def_f = ms[cf];
      if (t.vol_threads == 128 && t.vol_per_sm == 0) def_v = ms[cv];
    }
    // the FP32 block-Jacobi apply on the fine level, with the blocks the cycle will use
    if (f32 && storage) {
      const int kb[4] = {48, 96, 144, 200};
      double bj = 1e30;
      tune_fill_kernel<float><<<h->nsm * 4, 256, 0, st>>>(n0, yf, 0.2);
      DG_LAUNCH_CHECK(h);
      for (int i = 0; i < 4; ++i) {
        h->tune[which] = best;
        h->tune[which].jacobi_stage_kb = kb[i];
        auto sweep = [&]() -> int {
          const int q = staged_jacobi_f(h, 0, xf, yf, 0.9f, false, zf, storage, st);
          return q < 0 ? fail(h, DG_ERR_ARG, "element block unsuited to the staged apply") : q;
        };
        if ((r = time_classes(h, sweep, 5, ms, st))) return r;
        if (kb[i] == base.jacobi_stage_kb) def_j = ms[DG_PROF_BJ32];
        if (ms[DG_PROF_BJ32] < bj) { bj = ms[DG_PROF_BJ32]; best.jacobi_stage_kb = kb[i]; }
      }
      best_j = bj;
    }
    return DG_OK;
  };
  rc = measure();
  h->tune[which] = rc == DG_OK ? best : base;
  {  // restore the caller's profile
    double tmp_ms[DG_PROF_N], tmp_b[DG_PROF_N];
    long long tmp_c[DG_PROF_N];
    dg_profile_read_bytes(hh, tmp_ms, tmp_c, tmp_b);
    for (int c = 0; c < DG_PROF_N; ++c) {
      h->prof_ms[c] = saved_ms[c];
      h->prof_cnt[c] = saved_cnt[c];
      h->prof_bytes[c] = saved_bytes[c];
    }
    h->prof = prof_was;
  }
  if (xf) cudaFree(xf);
  if (yf) cudaFree(yf);
  if (zf) cudaFree(zf);
  if (rc) return rc;
  if (report) {
    report[0] = def_f; report[1] = best_f; report[2] = def_v; report[3] = best_v;
    report[4] = def_j; report[5] = best_j;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" {

int dg_get_tuning(const dg_handle* hh, int which, dg_tuning* t) {
  const Handle* h = reinterpret_cast<const Handle*>(hh);
  if (!h || !t || (which != DG_TUNE_FP64 && which != DG_TUNE_FP32)) return DG_ERR_ARG;
  *t = to_abi(h->tune[which]);
  return DG_OK;
}

int dg_set_tuning(dg_handle* hh, int which, const dg_tuning* t) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (which != DG_TUNE_FP64 && which != DG_TUNE_FP32) return fail(h, DG_ERR_ARG, "which: DG_TUNE_FP64 or DG_TUNE_FP32");
  if (!valid(t)) return fail(h, DG_ERR_ARG, "launch shape out of the supported set");
  h->tune[which] = from_abi(*t);
  return DG_OK;
}

int dg_autotune(dg_handle* hh, int which, int use_cache, double* report, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (which != DG_TUNE_FP64 && which != DG_TUNE_FP32) return fail(h, DG_ERR_ARG, "which: DG_TUNE_FP64 or DG_TUNE_FP32");
  return autotune(h, which, use_cache != 0, report, as_stream(stream));
}

}  // extern "C"
