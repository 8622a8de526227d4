// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qbx.h"

// ---------------------------------------------------------------- complex helpers
struct __align__(16) cd {  // complex double, interleaved like the ABI
  double x, y;
};

__host__ __device__ __forceinline__ cd mk(double a, double b) { cd r; r.x = a; r.y = b; return r; }
__host__ __device__ __forceinline__ cd cadd(cd a, cd b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cd csub(cd a, cd b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cd cmul(cd a, cd b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cd cconj(cd a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ cd cscale(cd a, double s) { return mk(a.x * s, a.y * s); }
// a += b * c
__host__ __device__ __forceinline__ void cfma(cd& a, cd b, cd c) {
  a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}

// ---------------------------------------------------------------- error handling
void set_error(const char* fmt, ...);
#define QBX_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                __LINE__);                                                        \
      return e_ == cudaErrorMemoryAllocation ? QBX_ERR_OOM : QBX_ERR_CUDA;        \
    }                                                                             \
  } while (0)

// ---------------------------------------------------------------- device buffers
template <typename T>
struct DevBuf {
  T* ptr = nullptr;
  size_t n = 0;
  cudaError_t alloc(size_t count) {
    release();
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)&ptr, count * sizeof(T));
    if (e == cudaSuccess) n = count; else ptr = nullptr;
    return e;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    n = 0;
  }
  ~DevBuf() { release(); }
};

// ---------------------------------------------------------------- geometry / plan
struct FmmPlan;  // fmm.cu
// Largest box expansion order (coarse boxes spanning many wavelengths need
// orders of about k * side; beyond this the plan is refused).
constexpr int kMaxBoxOrder = 1200;

struct qbx_handle {
  // geometry (device)
  int64_t n_panels = 0, n_nodes = 0, n_src = 0, n_ctr = 0;
  int q = 0, q_src = 0, p = 0, sides = 1;
  double k = 0;
  double h_max = 0;                         // longest panel
  DevBuf<double> node_xy, node_nrm, panel_h;
  DevBuf<double> node_w;                    // density-grid weights
  bool own_src = false;                     // the caller supplied the source grid
  bool defer_conditions = false;            // Condition 4 is checked at tree build instead
  std::vector<long long> curve_off;         // [n_curves + 1] first panel of every curve
  std::vector<long long> panel_origin;      // original panel of every panel (refinement)
  std::vector<double2> panel_interval;      // its part of the original panel, in u
  DevBuf<double> src_xy, src_nrm, src_w;
  DevBuf<double> ctr_xy, ctr_r;
  // Set when the library made the source grid itself (q_src nodes per panel
  // by polynomial interpolation of the density grid): densities passed to
  // eval then live on the density grid and are interpolated the same way.
  bool upsample = false;
  DevBuf<double> up_L;                      // [q_src][q] Lagrange interpolation matrix
  int64_t n_density() const { return upsample ? n_nodes : n_src; }
  // targets / association (device)
  int64_t n_tgt = 0, n_qbx_tgt = 0, n_direct_tgt = 0;
  bool planned = false;
  int mode = QBX_DIRECT;
  // Set while the handle belongs to a batch: many problems then run at once,
  // so an evaluation favours throughput (one stream, 32 centres per L2QBXL
  // warp, wide tiles) over the latency of a single problem.
  bool batched = false;
  // plan choices an autotuner may set (0: automatic): the M2L engine of the
  // next plan (0: FP64 on tensor cores where exact, mixed on the FP32 CUDA-core
  // GEMM; 1: tensor cores for both; 2: CUDA cores for both) and the centres
  // per warp of L2QBXL
  int m2l_engine = 0;
  int l2qbxl_g = 0;
  DevBuf<double> tgt_xy;
  DevBuf<int32_t> assoc;                    // [n_tgt] centre or -1
  DevBuf<int32_t> qbx_tgt_list, direct_tgt_list;
  // on-surface targets that ask for the on-surface value (side 0): the mean of
  // the two one-sided QBX limits, from the node's exterior centre (assoc) and
  // its interior centre (assoc + n_nodes)
  DevBuf<int8_t> avg;                       // [n_tgt] 1 = two-sided mean (or empty)
  bool has_avg = false;
  // evaluation scratch
  DevBuf<cd> q_str, d_str;                  // per-source charge / dipole strengths
  DevBuf<cd> sigS_dev, sigD_dev, out_dev;   // staging for host buffers
  DevBuf<cd> alpha;                         // [n_ctr][2p+1]
  DevBuf<int32_t> counters;                 // small device counters
  FmmPlan* fmm = nullptr;
  int64_t stats[20] = {0};
  int64_t launches = 0;                     // kernel launches of the current eval
  // stage timing
  bool timing = false;
  cudaEvent_t ev[2 * QBX_STAGE_COUNT] = {};
  bool ev_used[QBX_STAGE_COUNT] = {};
  cudaError_t dbg_err = cudaSuccess;        // QBX_DEBUG_SYNC bookkeeping
  int dbg_stage = -1;
  bool dbg_end = false;
};

// ---------------------------------------------------------------- kernels entry points
// direct.cu
qbx_status launch_strengths(qbx_handle* h, cd cS, const cd* sigS, cd cD, const cd* sigD,
                            cudaStream_t s);
qbx_status launch_p2qbxl_direct(qbx_handle* h, bool has_S, bool has_D, int precision,
                                cudaStream_t s);
qbx_status launch_p2p_direct(qbx_handle* h, bool has_S, bool has_D, cd* out, int precision,
                             cudaStream_t s);
qbx_status launch_qbxl2p(qbx_handle* h, cd* out, cudaStream_t s);
qbx_status launch_associate_direct(qbx_handle* h, const int64_t* on_node, const int8_t* on_side,
                                   double eps, cudaStream_t s);
qbx_status launch_place_centres(qbx_handle* h, cudaStream_t s);
// surface.cu
void gl_nodes(int n, std::vector<double>& x, std::vector<double>& w);
qbx_status upsample_geometry(qbx_handle* h);
// conditions.cu
qbx_status density_weights(qbx_handle* h);
// api.cu: QBX_ERR_TIMEOUT (and clears the flag) if a bounded device wait gave up
qbx_status read_wait_flag(qbx_handle* h);
// api.cu: replace a handle's density geometry (after refinement); drops any plan
qbx_status replace_geometry(qbx_handle* h, int64_t n_panels, DevBuf<double>& node_xy,
                            DevBuf<double>& node_nrm, DevBuf<double>& node_w,
                            const std::vector<double>& panel_h);
qbx_status launch_strengths_upsampled(qbx_handle* h, cd cS, const cd* sigS, cd cD, const cd* sigD,
                                      cudaStream_t s);
// fmm.cu
qbx_status fmm_plan_build(qbx_handle* h, const qbx_tree_desc* d, const int64_t* on_node_dev,
                          const int8_t* on_side_dev, double eps);
qbx_status fmm_eval(qbx_handle* h, bool has_S, bool has_D, cd* out, int precision,
                    bool all_centres, cudaStream_t s);
void fmm_plan_free(FmmPlan* f);

// stage timing helpers (api.cu)
void stage_begin(qbx_handle* h, int stage, cudaStream_t s);
void stage_end(qbx_handle* h, int stage, cudaStream_t s);
// QBX_DEBUG_SYNC=1: synchronise after every kernel and name the one that failed
int debug_sync();
#define QBX_KCHECK(name, stream)                                                      \
  do {                                                                                \
    if (debug_sync()) {                                                               \
      const cudaError_t e_ = cudaStreamSynchronize(stream);                           \
      if (e_ != cudaSuccess) {                                                        \
        set_error("kernel %s failed: %s", name, cudaGetErrorString(e_));              \
        return QBX_ERR_CUDA;                                                          \
      }                                                                               \
    }                                                                                 \
  } while (0)
