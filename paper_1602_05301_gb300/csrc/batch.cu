// Batched evaluation of independent problems through one CUDA graph, and the
// measured plan selection (autotuner) used to pick direct or FMM evaluation
// per problem.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qbx_internal.h"

namespace {

bool is_dev(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

typedef std::tuple<int, int, int, int, int, int, int> TuneKey;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune_cache;

}  // namespace

struct qbx_batch {
  std::vector<qbx_handle*> h;
  std::vector<int64_t> soff, toff;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> evs;
  cudaStream_t main = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
  DevBuf<cd> sS, sD, out;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int cap_prec = -1;
  bool cap_S = false, cap_D = false;
  std::vector<double> cap_c;
  ~qbx_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto s : streams) cudaStreamDestroy(s);
    for (auto e : evs) cudaEventDestroy(e);
    if (main) cudaStreamDestroy(main);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_fork) cudaEventDestroy(ev_fork);
  }
};

extern "C" qbx_status qbx_batch_create(int32_t n, qbx_handle* const* handles, int32_t n_streams,
                                       qbx_batch** out) {
  set_error("%s", "");
  if (!out || !handles || n <= 0) {
    set_error("qbx_batch_create: bad arguments");
    return QBX_ERR_ARG;
  }
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!handles[i] || !handles[i]->planned) {
      set_error("qbx_batch_create: handle %d is NULL or has no plan (call qbx_tree_build)", i);
      return QBX_ERR_STATE;
    }
  qbx_batch* b = new qbx_batch();
  b->h.assign(handles, handles + n);
  for (int i = 0; i < n; ++i) handles[i]->batched = true;
  b->soff.assign(n + 1, 0);
  b->toff.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    b->soff[i + 1] = b->soff[i] + handles[i]->n_density();
    b->toff[i + 1] = b->toff[i] + handles[i]->n_tgt;
  }
  const int ns = std::max(1, std::min<int>(n_streams > 0 ? n_streams : 16, n));
  auto fail = [&](cudaError_t e) {
    set_error("qbx_batch_create: %s", cudaGetErrorString(e));
    delete b;
    return e == cudaErrorMemoryAllocation ? QBX_ERR_OOM : QBX_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  if ((e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  for (int j = 0; j < ns; ++j) {
    cudaStream_t s;
    cudaEvent_t ev;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    b->streams.push_back(s);
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    b->evs.push_back(ev);
  }
  if ((e = b->sS.alloc(std::max<int64_t>(1, b->soff[n]))) != cudaSuccess) return fail(e);
  if ((e = b->sD.alloc(std::max<int64_t>(1, b->soff[n]))) != cudaSuccess) return fail(e);
  if ((e = b->out.alloc(std::max<int64_t>(1, b->toff[n]))) != cudaSuccess) return fail(e);
  *out = b;
  return QBX_OK;
}

extern "C" void qbx_batch_destroy(qbx_batch* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  for (qbx_handle* h : b->h) h->batched = false;
  delete b;
}

namespace {

qbx_status capture(qbx_batch* b, const double* cS, bool S, const double* cD, bool D, int prec) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  const int n = (int)b->h.size(), ns = (int)b->streams.size();
  QBX_CUDA_TRY(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeRelaxed));
  qbx_status st = QBX_OK;
  cudaEventRecord(b->ev_fork, b->main);
  for (int j = 0; j < ns; ++j) cudaStreamWaitEvent(b->streams[j], b->ev_fork, 0);
  for (int i = 0; i < n && st == QBX_OK; ++i) {
    qbx_handle* h = b->h[i];
    const bool timing = h->timing;
    h->timing = false;
    st = qbx_layer_potential_eval(
        h, S ? cS[2 * i] : 0.0, S ? cS[2 * i + 1] : 0.0,
        S ? (const double*)(b->sS.ptr + b->soff[i]) : nullptr, D ? cD[2 * i] : 0.0,
        D ? cD[2 * i + 1] : 0.0, D ? (const double*)(b->sD.ptr + b->soff[i]) : nullptr,
        (double*)(b->out.ptr + b->toff[i]), nullptr, prec, b->streams[i % ns]);
    h->timing = timing;
  }
  for (int j = 0; j < ns; ++j) {
    cudaEventRecord(b->evs[j], b->streams[j]);
    cudaStreamWaitEvent(b->main, b->evs[j], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->main, &g);
  if (st != QBX_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    set_error("batch graph capture failed: %s", cudaGetErrorString(e));
    if (g) cudaGraphDestroy(g);
    return QBX_ERR_CUDA;
  }
  b->graph = g;
  QBX_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
  b->cap_prec = prec;
  b->cap_S = S;
  b->cap_D = D;
  b->cap_c.assign(4 * n, 0.0);
  for (int i = 0; i < n; ++i) {
    if (S) { b->cap_c[4 * i] = cS[2 * i]; b->cap_c[4 * i + 1] = cS[2 * i + 1]; }
    if (D) { b->cap_c[4 * i + 2] = cD[2 * i]; b->cap_c[4 * i + 3] = cD[2 * i + 1]; }
  }
  return QBX_OK;
}

}  // namespace

extern "C" qbx_status qbx_batch_eval(qbx_batch* b, const double* cS, const double* sigma_S,
                                     const double* cD, const double* sigma_D, double* out,
                                     int32_t precision, void* cuda_stream) {
  set_error("%s", "");
  if (!b || !out) { set_error("qbx_batch_eval: NULL batch or output"); return QBX_ERR_ARG; }
  const bool S = sigma_S != nullptr, D = sigma_D != nullptr;
  if ((S && !cS) || (D && !cD) || (!S && !D)) {
    set_error("qbx_batch_eval: each present layer needs its coefficients; one layer at least");
    return QBX_ERR_ARG;
  }
  if (precision != QBX_FP64 && precision != QBX_MIXED) {
    set_error("qbx_batch_eval: unknown precision %d", precision);
    return QBX_ERR_ARG;
  }
  const int n = (int)b->h.size();
  for (int i = 0; i < n; ++i)
    if (!b->h[i]->planned) {
      set_error("qbx_batch_eval: handle %d lost its plan", i);
      return QBX_ERR_STATE;
    }
  cudaStream_t us = (cudaStream_t)cuda_stream;
  const int64_t ns_src = b->soff[n], ns_tgt = b->toff[n];
  // stage inputs on the batch's main stream, after the caller's stream
  QBX_CUDA_TRY(cudaEventRecord(b->ev_in, us));
  QBX_CUDA_TRY(cudaStreamWaitEvent(b->main, b->ev_in, 0));
  bool host = !is_dev(out);
  if (S) {
    host = host || !is_dev(sigma_S);
    QBX_CUDA_TRY(cudaMemcpyAsync(b->sS.ptr, sigma_S, ns_src * sizeof(cd), cudaMemcpyDefault, b->main));
  }
  if (D) {
    host = host || !is_dev(sigma_D);
    QBX_CUDA_TRY(cudaMemcpyAsync(b->sD.ptr, sigma_D, ns_src * sizeof(cd), cudaMemcpyDefault, b->main));
  }
  bool same = b->exec && b->cap_prec == precision && b->cap_S == S && b->cap_D == D;
  for (int i = 0; i < n && same; ++i) {
    if (S) same = same && b->cap_c[4 * i] == cS[2 * i] && b->cap_c[4 * i + 1] == cS[2 * i + 1];
    if (D) same = same && b->cap_c[4 * i + 2] == cD[2 * i] && b->cap_c[4 * i + 3] == cD[2 * i + 1];
  }
  if (!same) {
    // the capture must not overlap the staging copies: order them first
    QBX_CUDA_TRY(cudaStreamSynchronize(b->main));
    const qbx_status st = capture(b, cS, S, cD, D, precision);
    if (st != QBX_OK) return st;
  }
  QBX_CUDA_TRY(cudaGraphLaunch(b->exec, b->main));
  QBX_CUDA_TRY(cudaMemcpyAsync(out, b->out.ptr, ns_tgt * sizeof(cd), cudaMemcpyDefault, b->main));
  QBX_CUDA_TRY(cudaEventRecord(b->ev_out, b->main));
  QBX_CUDA_TRY(cudaStreamWaitEvent(us, b->ev_out, 0));
  if (host) QBX_CUDA_TRY(cudaStreamSynchronize(b->main));
  return QBX_OK;
}

// ---------------------------------------------------------------- autotuner
extern "C" qbx_status qbx_autotune(qbx_handle* h, const qbx_tree_desc* desc, int32_t precision,
                                   int32_t has_S, int32_t has_D, int32_t reps, double* times_ms,
                                   int32_t* chosen) {
  set_error("%s", "");
  if (!h || !desc || (!has_S && !has_D)) {
    set_error("qbx_autotune: bad arguments");
    return QBX_ERR_ARG;
  }
  reps = std::max(1, std::min(reps, 20));
  const int modes[4] = {QBX_DIRECT, QBX_FMM, QBX_FMM, QBX_FMM};
  const int nmax[4] = {0, 32, 64, 128};
  double hmean = 0.0;
  {
    std::vector<double> hh(h->n_panels);
    QBX_CUDA_TRY(cudaMemcpy(hh.data(), h->panel_h.ptr, hh.size() * sizeof(double),
                            cudaMemcpyDeviceToHost));
    for (double v : hh) hmean += v;
    hmean /= (double)std::max<int64_t>(1, h->n_panels);
  }
  const TuneKey key((int)std::lround(std::log2((double)std::max<int64_t>(1, h->n_src))),
                    (int)std::lround(8.0 * h->k * hmean), h->p, precision, h->sides, has_S,
                    has_D);
  int best = -1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) best = it->second;
  }
  double t[4] = {0, 0, 0, 0};
  if (best < 0) {
    // random unit densities (deterministic)
    std::vector<cd> hs(std::max<int64_t>(1, h->n_src));
    uint64_t st = 0x9e3779b97f4a7c15ull;
    for (auto& v : hs) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      const double a = (double)(st >> 11) * (1.0 / 9007199254740992.0) * 6.283185307179586;
      v = mk(std::cos(a), std::sin(a));
    }
    DevBuf<cd> sig, out;
    QBX_CUDA_TRY(sig.alloc(hs.size()));
    // the targets of the plans being timed (the handle may not hold a plan yet)
    QBX_CUDA_TRY(out.alloc(std::max<int64_t>(1, desc->n_targets)));
    QBX_CUDA_TRY(cudaMemcpy(sig.ptr, hs.data(), hs.size() * sizeof(cd), cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double bt = 1e300;
    for (int c = 0; c < 4; ++c) {
      if (modes[c] == QBX_FMM && h->n_src < 512) continue;
      qbx_tree_desc d = *desc;
      d.mode = modes[c];
      d.n_max = nmax[c];
      qbx_status s = qbx_tree_build(h, &d);
      if (s != QBX_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return s;
      }
      std::vector<float> ms;
      for (int r = 0; r <= reps; ++r) {
        cudaEventRecord(e0, 0);
        s = qbx_layer_potential_eval(h, 1.0, 0.0, has_S ? (const double*)sig.ptr : nullptr, 1.0,
                                     0.0, has_D ? (const double*)sig.ptr : nullptr,
                                     (double*)out.ptr, nullptr, precision, nullptr);
        cudaEventRecord(e1, 0);
        if (s != QBX_OK) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return s;
        }
        const cudaError_t se = cudaEventSynchronize(e1);
        if (se != cudaSuccess) {
          set_error("qbx_autotune: evaluation of candidate %d failed: %s", c,
                    cudaGetErrorString(se));
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return QBX_ERR_CUDA;
        }
        float v = 0.f;
        cudaEventElapsedTime(&v, e0, e1);
        if (r > 0) ms.push_back(v);  // the first run is a warm-up
      }
      std::sort(ms.begin(), ms.end());
      t[c] = ms[ms.size() / 2];
      if (t[c] < bt) {
        bt = t[c];
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
  }
  qbx_tree_desc d = *desc;
  d.mode = modes[best];
  d.n_max = nmax[best];
  const qbx_status s = qbx_tree_build(h, &d);
  if (s != QBX_OK) return s;
  if (times_ms)
    for (int c = 0; c < 4; ++c) times_ms[c] = t[c];
  if (chosen) *chosen = best;
  return QBX_OK;
}

// ---------------------------------------------------------------- accuracy-aware autotuner
namespace {

struct TolKey {
  int lg_n, kh8, p, prec, sides, S, D, lg_tol;
  bool operator<(const TolKey& o) const {
    return std::tie(lg_n, kh8, p, prec, sides, S, D, lg_tol) <
           std::tie(o.lg_n, o.kh8, o.p, o.prec, o.sides, o.S, o.D, o.lg_tol);
  }
};
struct TolPlan {
  int mode, n_max, p_fmm, engine, g;
};
std::mutex g_tol_mu;
std::map<TolKey, TolPlan> g_tol_cache;

}  // namespace

extern "C" qbx_status qbx_autotune_tol(qbx_handle* h, const qbx_tree_desc* desc,
                                       int32_t precision, int32_t has_S, int32_t has_D,
                                       double tol, int32_t reps, int32_t* plan_out,
                                       double* report) {
  set_error("%s", "");
  if (!h || !desc || (!has_S && !has_D) || !(tol > 0.0) || desc->p_fmm < 1) {
    set_error("qbx_autotune_tol: bad arguments");
    return QBX_ERR_ARG;
  }
  reps = std::max(1, std::min(reps, 20));
  double hmean = 0.0;
  {
    std::vector<double> hh(h->n_panels);
    QBX_CUDA_TRY(cudaMemcpy(hh.data(), h->panel_h.ptr, hh.size() * sizeof(double),
                            cudaMemcpyDeviceToHost));
    for (double v : hh) hmean += v;
    hmean /= (double)std::max<int64_t>(1, h->n_panels);
  }
  const TolKey key{(int)std::lround(std::log2((double)std::max<int64_t>(1, h->n_src))),
                   (int)std::lround(8.0 * h->k * hmean), h->p, precision, h->sides, has_S, has_D,
                   (int)std::lround(std::log10(tol))};
  TolPlan best{-1, 0, 0, 0, 0};
  {
    std::lock_guard<std::mutex> lock(g_tol_mu);
    auto it = g_tol_cache.find(key);
    if (it != g_tol_cache.end()) best = it->second;
  }
  const int64_t nt = std::max<int64_t>(1, desc->n_targets);
  DevBuf<cd> sig, out, ref;
  QBX_CUDA_TRY(sig.alloc(std::max<int64_t>(1, h->n_density())));
  QBX_CUDA_TRY(out.alloc(nt));
  QBX_CUDA_TRY(ref.alloc(nt));
  {  // random unit densities (deterministic)
    std::vector<cd> hs(sig.n);
    uint64_t st = 0x2545f4914f6cdd1dull;
    for (auto& v : hs) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      const double a = (double)(st >> 11) * (1.0 / 9007199254740992.0) * 6.283185307179586;
      v = mk(std::cos(a), std::sin(a));
    }
    QBX_CUDA_TRY(cudaMemcpy(sig.ptr, hs.data(), hs.size() * sizeof(cd), cudaMemcpyHostToDevice));
  }
  const double* sS = has_S ? (const double*)sig.ptr : nullptr;
  const double* sD = has_D ? (const double*)sig.ptr : nullptr;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto finish = [&](qbx_status st) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  };
  auto build = [&](const TolPlan& c) -> qbx_status {
    qbx_tree_desc d = *desc;
    d.mode = c.mode;
    d.n_max = c.n_max;
    d.p_fmm = c.p_fmm > 0 ? c.p_fmm : desc->p_fmm;
    d.m2l_engine = c.engine;
    h->l2qbxl_g = c.g;
    return qbx_tree_build(h, &d);
  };
  // median time of reps evaluations (after one warm-up) in precision pr into o
  auto timed = [&](int pr, cd* o, double& ms) -> qbx_status {
    std::vector<float> v;
    for (int r = 0; r <= reps; ++r) {
      cudaEventRecord(e0, 0);
      const qbx_status s = qbx_layer_potential_eval(h, 1.0, 0.0, sS, 1.0, 0.0, sD, (double*)o,
                                                    nullptr, pr, nullptr);
      cudaEventRecord(e1, 0);
      if (s != QBX_OK) return s;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        set_error("qbx_autotune_tol: a candidate evaluation failed");
        return QBX_ERR_CUDA;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0) v.push_back(t);
    }
    std::sort(v.begin(), v.end());
    ms = v[v.size() / 2];
    return QBX_OK;
  };
  // relative l2 distance of out from ref (host side: small vectors)
  auto error = [&]() -> double {
    std::vector<cd> a(nt), b(nt);
    cudaMemcpy(a.data(), out.ptr, nt * sizeof(cd), cudaMemcpyDeviceToHost);
    cudaMemcpy(b.data(), ref.ptr, nt * sizeof(cd), cudaMemcpyDeviceToHost);
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < nt; ++i) {
      num += (a[i].x - b[i].x) * (a[i].x - b[i].x) + (a[i].y - b[i].y) * (a[i].y - b[i].y);
      den += b[i].x * b[i].x + b[i].y * b[i].y;
    }
    return den > 0.0 ? std::sqrt(num / den) : std::sqrt(num);
  };
  double best_ms = 0.0, best_err = 0.0;
  int tried = 0;
  if (best.mode < 0) {
    // the reference: the most accurate plan (direct QBX for small problems,
    // else FMM at the requested orders), FP64
    const bool small = h->n_src < 512;
    TolPlan refp{small ? QBX_DIRECT : QBX_FMM, 64, desc->p_fmm, 0, 0};
    qbx_status s = build(refp);
    if (s != QBX_OK) return finish(s);
    double ms;
    if ((s = timed(QBX_FP64, ref.ptr, ms)) != QBX_OK) return finish(s);
    double bt = 1e300;
    auto consider = [&](const TolPlan& c) -> qbx_status {
      qbx_status st = build(c);
      if (st != QBX_OK) return st;
      double t;
      if ((st = timed(precision, out.ptr, t)) != QBX_OK) return st;
      const double err = error();
      ++tried;
      if (err <= tol && t < bt) {
        bt = t;
        best = c;
        best_ms = t;
        best_err = err;
      }
      return QBX_OK;
    };
    // 1. plan kind and leaf size at the requested orders
    if ((s = consider({QBX_DIRECT, 0, desc->p_fmm, 0, 0})) != QBX_OK) return finish(s);
    if (!small)
      for (int nm : {16, 32, 64, 128})
        if ((s = consider({QBX_FMM, nm, desc->p_fmm, 0, 0})) != QBX_OK) return finish(s);
    if (best.mode == QBX_FMM) {
      // 2. lower box orders while the result stays within tol
      for (int pf = desc->p_fmm - 4; pf >= 4; pf -= 4) {
        const double before = bt;
        if ((s = consider({QBX_FMM, best.n_max, pf, 0, 0})) != QBX_OK) return finish(s);
        if (bt == before) break;
      }
      // 3. the M2L engine, 4. centres per L2QBXL warp
      for (int e : {1, 2})
        if ((s = consider({QBX_FMM, best.n_max, best.p_fmm, e, 0})) != QBX_OK) return finish(s);
      for (int g : {4, 8, 16, 32})
        if ((s = consider({QBX_FMM, best.n_max, best.p_fmm, best.engine, g})) != QBX_OK)
          return finish(s);
    }
    if (best.mode < 0) {
      set_error("qbx_autotune_tol: no candidate met tol = %g", tol);
      return finish(QBX_ERR_CONDITION);
    }
    std::lock_guard<std::mutex> lock(g_tol_mu);
    g_tol_cache[key] = best;
  }
  const qbx_status s = build(best);
  if (s != QBX_OK) return finish(s);
  if (plan_out) {
    plan_out[0] = best.mode;
    plan_out[1] = best.n_max;
    plan_out[2] = best.p_fmm;
    plan_out[3] = best.engine;
    plan_out[4] = best.g;
  }
  if (report) {
    report[0] = best_ms;
    report[1] = best_err;
    report[2] = tried;
  }
  return finish(QBX_OK);
}