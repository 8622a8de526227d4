// C ABI of the library (declared in include/qbx.h): handle life cycle, argument
// checking, host/device staging and the order of the evaluation stages.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <algorithm>
#include <new>
#include <vector>

#include "qbx_internal.h"

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* qbx_last_error(void) { return g_err; }

namespace {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
qbx_status copy_in(DevBuf<T>& dst, const T* src, size_t n) {
  QBX_CUDA_TRY(dst.alloc(n));
  if (n) QBX_CUDA_TRY(cudaMemcpy(dst.ptr, src, n * sizeof(T), cudaMemcpyDefault));
  return QBX_OK;
}

template <typename T>
std::vector<T> to_host(const T* src, size_t n) {
  std::vector<T> v(n);
  if (n) cudaMemcpy(v.data(), src, n * sizeof(T), cudaMemcpyDefault);
  return v;
}

#define QBX_TRY(expr)                    \
  do {                                   \
    qbx_status st_ = (expr);             \
    if (st_ != QBX_OK) return st_;       \
  } while (0)

}  // namespace

// QBX_DEBUG_SYNC=1 in the environment: synchronise around every stage and
// report the first stage whose kernels failed (a debugging aid; off by default).
int debug_sync() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("QBX_DEBUG_SYNC");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v;
}

static void debug_check(qbx_handle* h, int stage, cudaStream_t s, bool end) {
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && h->dbg_err == cudaSuccess) {
    h->dbg_err = e;
    h->dbg_stage = stage;
    h->dbg_end = end;
  }
}

void stage_begin(qbx_handle* h, int stage, cudaStream_t s) {
  if (debug_sync()) debug_check(h, stage, s, false);
  if (!h->timing) return;
  cudaEventRecord(h->ev[2 * stage], s);
  h->ev_used[stage] = true;
}

void stage_end(qbx_handle* h, int stage, cudaStream_t s) {
  if (debug_sync()) debug_check(h, stage, s, true);
  if (!h->timing) return;
  cudaEventRecord(h->ev[2 * stage + 1], s);
}

extern "C" qbx_status qbx_geometry_create(const qbx_geometry_desc* d, qbx_handle** out) {
  g_err[0] = 0;
  if (!d || !out) { set_error("qbx_geometry_create: NULL argument"); return QBX_ERR_ARG; }
  *out = nullptr;
  if (d->n_panels <= 0 || d->q <= 0 || !d->node_xy || !d->normal_xy || !d->panel_h) {
    set_error("qbx_geometry_create: empty geometry or missing node/normal/panel arrays");
    return QBX_ERR_ARG;
  }
  if (d->p_qbx < 0 || d->p_qbx > QBX_MAX_P) {
    set_error("qbx_geometry_create: p_qbx=%d outside [0, %d]", d->p_qbx, QBX_MAX_P);
    return QBX_ERR_ARG;
  }
  if (d->center_sides != 1 && d->center_sides != 2) {
    set_error("qbx_geometry_create: center_sides must be 1 or 2");
    return QBX_ERR_ARG;
  }
  if (!(d->k > 0.0)) { set_error("qbx_geometry_create: k must be > 0"); return QBX_ERR_ARG; }
  const bool own_src = d->q_src > 0 && d->src_xy != nullptr;
  const bool upsample = d->q_src > 0 && d->src_xy == nullptr;
  if (own_src && (!d->src_normal_xy || !d->src_weight)) {
    set_error("qbx_geometry_create: a source grid needs src_xy, src_normal_xy, src_weight");
    return QBX_ERR_ARG;
  }
  if (upsample && (d->src_normal_xy || d->src_weight || d->q_src > 256)) {
    set_error("qbx_geometry_create: q_src > 0 without src_xy asks the library to make the "
              "source grid (q_src <= 256); src_normal_xy and src_weight must then be NULL");
    return QBX_ERR_ARG;
  }
  if (!own_src && !upsample && !d->weight) {
    set_error("qbx_geometry_create: weight is required when the density grid is the source grid");
    return QBX_ERR_ARG;
  }
  const int64_t n_nodes = d->n_panels * d->q;
  if (n_nodes * d->center_sides > INT32_MAX) {
    set_error("qbx_geometry_create: too many centres for 32-bit association indices");
    return QBX_ERR_ARG;
  }
  // Condition 4 (Sec. 3.2): k * max_k h_k <= 5
  std::vector<double> hh = to_host(d->panel_h, (size_t)d->n_panels);
  double hmax = 0.0;
  for (double v : hh) {
    if (!(v > 0.0)) { set_error("qbx_geometry_create: panel length <= 0"); return QBX_ERR_ARG; }
    hmax = std::max(hmax, v);
  }
  if (d->k * hmax > 5.0 && !d->defer_conditions) {
    set_error("Condition 4 violated: k * max h = %.4g > 5; refine the panels", d->k * hmax);
    return QBX_ERR_CONDITION;
  }
  // curves: consecutive panel ranges (one curve when none are given)
  std::vector<long long> coff;
  if (d->n_curves > 1 || (d->n_curves == 1 && d->curve_panel_offset)) {
    if (!d->curve_panel_offset) {
      set_error("qbx_geometry_create: n_curves > 1 needs curve_panel_offset");
      return QBX_ERR_ARG;
    }
    std::vector<int64_t> co = to_host(d->curve_panel_offset, (size_t)d->n_curves + 1);
    if (co[0] != 0 || co[d->n_curves] != d->n_panels) {
      set_error("qbx_geometry_create: curve_panel_offset must run from 0 to n_panels");
      return QBX_ERR_ARG;
    }
    for (int c = 0; c < d->n_curves; ++c)
      if (co[c + 1] <= co[c]) {
        set_error("qbx_geometry_create: curve %d has no panels", c);
        return QBX_ERR_ARG;
      }
    coff.assign(co.begin(), co.end());
  } else if (d->n_curves < 0) {
    set_error("qbx_geometry_create: n_curves < 0");
    return QBX_ERR_ARG;
  } else {
    coff = {0, (long long)d->n_panels};
  }
  qbx_handle* h = new (std::nothrow) qbx_handle();
  if (!h) { set_error("out of host memory"); return QBX_ERR_OOM; }
  auto fail = [&](qbx_status st) { qbx_destroy(h); return st; };
  h->n_panels = d->n_panels;
  h->q = d->q;
  h->n_nodes = n_nodes;
  h->k = d->k;
  h->h_max = hmax;
  h->p = d->p_qbx;
  h->sides = d->center_sides;
  h->upsample = upsample;
  h->own_src = own_src;
  h->defer_conditions = d->defer_conditions != 0;
  h->curve_off = coff;
  h->panel_origin.resize(d->n_panels);
  for (int64_t k = 0; k < d->n_panels; ++k) h->panel_origin[k] = k;
  h->panel_interval.assign(d->n_panels, make_double2(-1.0, 1.0));
  h->q_src = (own_src || upsample) ? d->q_src : d->q;
  h->n_src = d->n_panels * h->q_src;
  h->n_ctr = n_nodes * h->sides;
  qbx_status st;
  if ((st = copy_in(h->node_xy, d->node_xy, 2 * n_nodes)) != QBX_OK) return fail(st);
  if ((st = copy_in(h->node_nrm, d->normal_xy, 2 * n_nodes)) != QBX_OK) return fail(st);
  if ((st = copy_in(h->panel_h, d->panel_h, d->n_panels)) != QBX_OK) return fail(st);
  if (d->weight) {
    if ((st = copy_in(h->node_w, d->weight, n_nodes)) != QBX_OK) return fail(st);
  } else if ((st = density_weights(h)) != QBX_OK) {
    return fail(st);
  }
  if (upsample) {
    if ((st = upsample_geometry(h)) != QBX_OK) return fail(st);
  } else if (own_src) {
    if ((st = copy_in(h->src_xy, d->src_xy, 2 * h->n_src)) != QBX_OK) return fail(st);
    if ((st = copy_in(h->src_nrm, d->src_normal_xy, 2 * h->n_src)) != QBX_OK) return fail(st);
    if ((st = copy_in(h->src_w, d->src_weight, h->n_src)) != QBX_OK) return fail(st);
  } else {
    if ((st = copy_in(h->src_xy, d->node_xy, 2 * h->n_src)) != QBX_OK) return fail(st);
    if ((st = copy_in(h->src_nrm, d->normal_xy, 2 * h->n_src)) != QBX_OK) return fail(st);
    if ((st = copy_in(h->src_w, d->weight, h->n_src)) != QBX_OK) return fail(st);
  }
  cudaError_t e;
  if ((e = h->ctr_xy.alloc(2 * h->n_ctr)) != cudaSuccess ||
      (e = h->ctr_r.alloc(h->n_ctr)) != cudaSuccess ||
      (e = h->q_str.alloc(h->n_src)) != cudaSuccess ||
      (e = h->d_str.alloc(h->n_src)) != cudaSuccess ||
      (e = h->alpha.alloc(h->n_ctr * (2 * h->p + 1))) != cudaSuccess ||
      (e = h->counters.alloc(16)) != cudaSuccess) {
    set_error("device allocation failed: %s", cudaGetErrorString(e));
    return fail(QBX_ERR_OOM);
  }
  if ((st = launch_place_centres(h, 0)) != QBX_OK) return fail(st);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    set_error("geometry set-up failed: %s", cudaGetErrorString(e));
    return fail(QBX_ERR_CUDA);
  }
  for (int i = 0; i < 2 * QBX_STAGE_COUNT; ++i) cudaEventCreate(&h->ev[i]);
  h->stats[0] = h->n_src;
  h->stats[1] = h->n_ctr;
  *out = h;
  return QBX_OK;
}

extern "C" qbx_status qbx_tree_build(qbx_handle* h, const qbx_tree_desc* d) {
  g_err[0] = 0;
  if (!h || !d) { set_error("qbx_tree_build: NULL argument"); return QBX_ERR_ARG; }
  if (d->n_targets < 0 || (d->n_targets > 0 && !d->target_xy)) {
    set_error("qbx_tree_build: invalid targets");
    return QBX_ERR_ARG;
  }
  if (d->n_targets > INT32_MAX) { set_error("qbx_tree_build: too many targets"); return QBX_ERR_ARG; }
  if (d->mode != QBX_DIRECT && d->mode != QBX_FMM) {
    set_error("qbx_tree_build: unknown mode %d", d->mode);
    return QBX_ERR_ARG;
  }
  if (d->m2l_engine < 0 || d->m2l_engine > 2) {
    set_error("qbx_tree_build: unknown m2l_engine %d", d->m2l_engine);
    return QBX_ERR_ARG;
  }
  h->m2l_engine = d->m2l_engine;
  h->planned = false;
  if (h->k * h->h_max > 5.0) {  // a geometry accepted with defer_conditions, not yet refined
    set_error("Condition 4 violated: k * max h = %.4g > 5; call qbx_refine", h->k * h->h_max);
    return QBX_ERR_CONDITION;
  }
  const double eps = d->eps_assoc > 0.0 ? d->eps_assoc : 0.1;
  h->n_tgt = d->n_targets;
  std::vector<int64_t> on_node;
  std::vector<int8_t> on_side;
  if (d->on_surface_node) {
    on_node = to_host(d->on_surface_node, (size_t)h->n_tgt);
    if (d->on_surface_side) on_side = to_host(d->on_surface_side, (size_t)h->n_tgt);
    for (int64_t t = 0; t < h->n_tgt; ++t) {
      if (on_node[t] >= h->n_nodes) {
        set_error("qbx_tree_build: on_surface_node[%lld] = %lld out of range", (long long)t,
                  (long long)on_node[t]);
        return QBX_ERR_ARG;
      }
      if (on_node[t] >= 0 && !on_side.empty() && on_side[t] <= 0 && h->sides < 2) {
        set_error("qbx_tree_build: target %lld asks for the interior side or the two-sided "
                  "value but the geometry has exterior centres only", (long long)t);
        return QBX_ERR_ARG;
      }
    }
  }
  // side 0: the on-surface value, the mean of both one-sided limits
  h->has_avg = false;
  h->avg.release();
  if (!on_side.empty()) {
    std::vector<int8_t> avg(h->n_tgt, 0);
    for (int64_t t = 0; t < h->n_tgt; ++t)
      if (on_node[t] >= 0 && on_side[t] == 0) avg[t] = 1, h->has_avg = true;
    if (h->has_avg) QBX_TRY(copy_in(h->avg, avg.data(), avg.size()));
  }
  QBX_TRY(copy_in(h->tgt_xy, d->target_xy, 2 * h->n_tgt));
  QBX_CUDA_TRY(h->assoc.alloc(h->n_tgt));
  DevBuf<int64_t> dn;
  DevBuf<int8_t> ds;
  if (!on_node.empty()) QBX_TRY(copy_in(dn, on_node.data(), on_node.size()));
  if (!on_side.empty()) QBX_TRY(copy_in(ds, on_side.data(), on_side.size()));
  const int32_t init[2] = {0, INT32_MAX};
  QBX_CUDA_TRY(cudaMemcpy(h->counters.ptr, init, sizeof(init), cudaMemcpyHostToDevice));
  h->mode = d->mode;
  if (d->mode == QBX_FMM) {
    QBX_TRY(fmm_plan_build(h, d, dn.ptr, ds.ptr, eps));  // tree, lists, association, orders
  } else {
    QBX_TRY(launch_associate_direct(h, dn.ptr, ds.ptr, eps, 0));
  }
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  int32_t ctr[2];
  QBX_CUDA_TRY(cudaMemcpy(ctr, h->counters.ptr, sizeof(ctr), cudaMemcpyDeviceToHost));
  std::vector<int32_t> assoc = to_host(h->assoc.ptr, (size_t)h->n_tgt);
  if (d->assoc_out) {
    std::vector<int32_t> ao(assoc);
    for (auto& a : ao) a = a < -1 ? -1 : a;
    QBX_CUDA_TRY(cudaMemcpy(d->assoc_out, ao.data(), ao.size() * sizeof(int32_t),
                            cudaMemcpyDefault));
  }
  if (ctr[0] > 0) {
    set_error("target association failed for %d target(s); first failing target %d lies within "
              "h/4 of the curve but in no expansion disk (increase eps_assoc or refine)",
              ctr[0], ctr[1]);
    return QBX_ERR_ASSOCIATION;
  }
  // target lists in index order
  std::vector<int32_t> ql, dl;
  ql.reserve(assoc.size());
  dl.reserve(assoc.size());
  for (int64_t t = 0; t < h->n_tgt; ++t) (assoc[t] >= 0 ? ql : dl).push_back((int32_t)t);
  h->n_qbx_tgt = (int64_t)ql.size();
  h->n_direct_tgt = (int64_t)dl.size();
  QBX_TRY(copy_in(h->qbx_tgt_list, ql.data(), ql.size()));
  QBX_TRY(copy_in(h->direct_tgt_list, dl.data(), dl.size()));
  QBX_CUDA_TRY(h->out_dev.alloc(h->n_tgt));
  h->stats[2] = h->n_tgt;
  h->stats[3] = h->n_qbx_tgt;
  if (d->mode == QBX_DIRECT) {
    h->stats[12] = h->n_src * h->n_ctr;
    h->stats[13] = h->n_src * h->n_direct_tgt;
  }
  h->planned = true;
  return QBX_OK;
}

extern "C" qbx_status qbx_layer_potential_eval(qbx_handle* h, double cS_re, double cS_im,
                                               const double* sigma_S, double cD_re,
                                               double cD_im, const double* sigma_D, double* out,
                                               double* alpha_out, int32_t precision,
                                               void* cuda_stream) {
  g_err[0] = 0;
  if (!h || !out) { set_error("qbx_layer_potential_eval: NULL handle or output"); return QBX_ERR_ARG; }
  if (!h->planned) { set_error("qbx_layer_potential_eval: call qbx_tree_build first"); return QBX_ERR_STATE; }
  if (precision != QBX_FP64 && precision != QBX_MIXED) {
    set_error("qbx_layer_potential_eval: unknown precision %d", precision);
    return QBX_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (int i = 0; i < QBX_STAGE_COUNT; ++i) h->ev_used[i] = false;
  const bool has_S = sigma_S != nullptr, has_D = sigma_D != nullptr;
  const cd* sS = nullptr;
  const cd* sD = nullptr;
  bool host_io = false;
  if (has_S) {
    if (is_device_ptr(sigma_S)) sS = (const cd*)sigma_S;
    else {
      host_io = true;
      if (h->sigS_dev.n < (size_t)h->n_density()) QBX_CUDA_TRY(h->sigS_dev.alloc(h->n_density()));
      QBX_CUDA_TRY(cudaMemcpyAsync(h->sigS_dev.ptr, sigma_S, h->n_density() * sizeof(cd),
                                   cudaMemcpyDefault, s));
      sS = h->sigS_dev.ptr;
    }
  }
  if (has_D) {
    if (is_device_ptr(sigma_D)) sD = (const cd*)sigma_D;
    else {
      host_io = true;
      if (h->sigD_dev.n < (size_t)h->n_density()) QBX_CUDA_TRY(h->sigD_dev.alloc(h->n_density()));
      QBX_CUDA_TRY(cudaMemcpyAsync(h->sigD_dev.ptr, sigma_D, h->n_density() * sizeof(cd),
                                   cudaMemcpyDefault, s));
      sD = h->sigD_dev.ptr;
    }
  }
  const bool out_dev = is_device_ptr(out);
  cd* o = out_dev ? (cd*)out : h->out_dev.ptr;
  host_io = host_io || !out_dev;
  const bool alpha_dev = alpha_out && is_device_ptr(alpha_out);
  if (alpha_out && !alpha_dev) host_io = true;

  h->launches = 0;
  h->dbg_err = cudaSuccess;
  stage_begin(h, QBX_STAGE_STRENGTHS, s);
  if (h->upsample)
    QBX_TRY(launch_strengths_upsampled(h, mk(cS_re, cS_im), sS, mk(cD_re, cD_im), sD, s));
  else
    QBX_TRY(launch_strengths(h, mk(cS_re, cS_im), sS, mk(cD_re, cD_im), sD, s));
  stage_end(h, QBX_STAGE_STRENGTHS, s);
  if (h->mode == QBX_FMM) {
    QBX_TRY(fmm_eval(h, has_S, has_D, o, precision, alpha_out != nullptr, s));
  } else {
    stage_begin(h, QBX_STAGE_P2QBXL, s);
    QBX_TRY(launch_p2qbxl_direct(h, has_S, has_D, precision, s));
    stage_end(h, QBX_STAGE_P2QBXL, s);
    stage_begin(h, QBX_STAGE_P2P, s);
    QBX_TRY(launch_p2p_direct(h, has_S, has_D, o, precision, s));
    stage_end(h, QBX_STAGE_P2P, s);
  }
  stage_begin(h, QBX_STAGE_QBXL2P, s);
  QBX_TRY(launch_qbxl2p(h, o, s));
  stage_end(h, QBX_STAGE_QBXL2P, s);
  h->stats[16] = h->launches;
  if (h->dbg_err != cudaSuccess) {
    set_error("debug sync: stage %d (%s) failed: %s", h->dbg_stage, h->dbg_end ? "end" : "begin",
              cudaGetErrorString(h->dbg_err));
    return QBX_ERR_CUDA;
  }
  if (!out_dev)
    QBX_CUDA_TRY(cudaMemcpyAsync(out, o, h->n_tgt * sizeof(cd), cudaMemcpyDefault, s));
  if (alpha_out)
    QBX_CUDA_TRY(cudaMemcpyAsync(alpha_out, h->alpha.ptr,
                                 h->n_ctr * (2 * h->p + 1) * sizeof(cd), cudaMemcpyDefault, s));
  if (host_io) {
    QBX_CUDA_TRY(cudaStreamSynchronize(s));
    return read_wait_flag(h);
  }
  return QBX_OK;
}

extern "C" qbx_status qbx_sync(qbx_handle* h) {
  set_error("%s", "");
  if (!h) { set_error("qbx_sync: NULL handle"); return QBX_ERR_ARG; }
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  return read_wait_flag(h);
}

namespace {
template <typename T>
void take(DevBuf<T>& dst, DevBuf<T>& src) {
  dst.release();
  dst.ptr = src.ptr;
  dst.n = src.n;
  src.ptr = nullptr;
  src.n = 0;
}
}  // namespace

qbx_status replace_geometry(qbx_handle* h, int64_t n_panels, DevBuf<double>& node_xy,
                            DevBuf<double>& node_nrm, DevBuf<double>& node_w,
                            const std::vector<double>& panel_h) {
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  if (h->fmm) fmm_plan_free(h->fmm);
  h->fmm = nullptr;
  h->planned = false;
  h->n_panels = n_panels;
  h->n_nodes = n_panels * h->q;
  take(h->node_xy, node_xy);
  take(h->node_nrm, node_nrm);
  take(h->node_w, node_w);
  QBX_TRY(copy_in(h->panel_h, panel_h.data(), panel_h.size()));
  h->h_max = 0.0;
  for (double v : panel_h) h->h_max = std::max(h->h_max, v);
  h->n_src = n_panels * h->q_src;
  h->n_ctr = h->n_nodes * h->sides;
  if (h->n_ctr * (2 * h->p + 1) > ((int64_t)1 << 40) || h->n_ctr > INT32_MAX) {
    set_error("refined geometry too large");
    return QBX_ERR_ARG;
  }
  if (h->upsample) {
    QBX_TRY(upsample_geometry(h));
  } else {
    QBX_TRY(copy_in(h->src_xy, h->node_xy.ptr, 2 * h->n_src));
    QBX_TRY(copy_in(h->src_nrm, h->node_nrm.ptr, 2 * h->n_src));
    QBX_TRY(copy_in(h->src_w, h->node_w.ptr, h->n_src));
  }
  cudaError_t e;
  if ((e = h->ctr_xy.alloc(2 * h->n_ctr)) != cudaSuccess ||
      (e = h->ctr_r.alloc(h->n_ctr)) != cudaSuccess ||
      (e = h->q_str.alloc(h->n_src)) != cudaSuccess ||
      (e = h->d_str.alloc(h->n_src)) != cudaSuccess ||
      (e = h->alpha.alloc(h->n_ctr * (2 * h->p + 1))) != cudaSuccess) {
    set_error("device allocation failed: %s", cudaGetErrorString(e));
    return QBX_ERR_OOM;
  }
  QBX_TRY(launch_place_centres(h, 0));
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  h->stats[0] = h->n_src;
  h->stats[1] = h->n_ctr;
  return QBX_OK;
}

extern "C" void qbx_destroy(qbx_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  if (h->fmm) fmm_plan_free(h->fmm);
  h->fmm = nullptr;
  for (int i = 0; i < 2 * QBX_STAGE_COUNT; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  delete h;
}

extern "C" qbx_status qbx_get_stats(const qbx_handle* h, int64_t* stats, int32_t n) {
  if (!h || !stats || n < 20) { set_error("qbx_get_stats: bad arguments"); return QBX_ERR_ARG; }
  for (int i = 0; i < 20; ++i) stats[i] = h->stats[i];
  return QBX_OK;
}

extern "C" qbx_status qbx_set_timing(qbx_handle* h, int32_t enable) {
  if (!h) { set_error("qbx_set_timing: NULL handle"); return QBX_ERR_ARG; }
  h->timing = enable != 0;
  return QBX_OK;
}

extern "C" int32_t qbx_get_stage_times(qbx_handle* h, double* t, int32_t n) {
  if (!h || !t) return 0;
  int32_t m = n < QBX_STAGE_COUNT ? n : QBX_STAGE_COUNT;
  for (int i = 0; i < m; ++i) {
    t[i] = 0.0;
    if (!h->ev_used[i]) continue;
    float ms = 0.f;
    if (cudaEventSynchronize(h->ev[2 * i + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess)
      t[i] = ms;
  }
  return m;
}
