// Quadtree, interaction lists and FMM plan (Sec. 4 and Sec. 7 of the paper).
#pragma once
#include "qbx_internal.h"

// particle classes held by the tree
enum { PT_SRC = 0, PT_CTR = 1, PT_TGT = 2, PT_NODE = 3, PT_COUNT = 4 };

constexpr int kMortonBits = 24;   // levels 0..24
constexpr int kMaxLevels = 24;

struct BoxArrays {
  DevBuf<int> level, parent, child;     // child: [n][4], -1 = none
  DevBuf<int2> ij;                      // integer position at own level
  DevBuf<unsigned long long> key;       // Morton key of (ij) at own level
  DevBuf<double2> centre;
  DevBuf<int2> rng[PT_COUNT];           // [start, end) in each sorted particle array
};

struct Csr {
  DevBuf<int> off, idx;
  int64_t nnz = 0;
};

struct CentreSet {
  DevBuf<int> clist, wp_ctr, wp_box, wp_off;
  int n = 0, n_pairs = 0;
  int wp_pbmax = 0;  // largest box order among the M2QBXL pairs' boxes
};

// An opaque TMA tensor map (CUtensorMap: 128 bytes, 64-byte aligned)
struct alignas(64) TmapBlob {
  unsigned char b[128];
};

// One parent level of the FP64 M2M or L2L on the tensor cores: four groups
// (the child quadrants), the bf16 matrix slices of their sigma-normalised
// operators, the source vectors' slices, and the rows (one per child).
struct TcLevelOp {
  bool use = false;
  int S = 0, beta = 0, K = 0, Np = 0, Q = 0;  // slices, digit bits, input width, output rows, outputs
  int n_rows = 0, n_src = 0, n_items = 0, n_par = 0;
  DevBuf<int4> gp, items;
  DevBuf<long long> gaoff, gfoff, xoff, yoff;
  DevBuf<uint16_t> A, X;
  DevBuf<int> fexp, xexp, src, rowsrc, rowdst, prow;
};

struct FmmPlan {
  // concurrency of the near-field stages (see fmm_eval)
  cudaStream_t near_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_p2l = nullptr, ev_m2m = nullptr,
              ev_out = nullptr;
  ~FmmPlan() {
    if (near_stream) cudaStreamDestroy(near_stream);
    for (cudaEvent_t ev : {ev_fork, ev_join, ev_p2l, ev_m2m, ev_out})
      if (ev) cudaEventDestroy(ev);
  }
  // tree
  double x0 = 0, y0 = 0, side = 0;      // root square [x0, x0+side] x [y0, y0+side]
  int n_levels = 0, n_boxes = 0;
  std::vector<int> level_off;           // [n_levels + 1]
  BoxArrays box;
  std::vector<int> h_level_off;
  // sorted particles: perm[type][i] = original index of the i-th particle in tree order
  DevBuf<unsigned long long> keys[PT_COUNT];
  DevBuf<int> perm[PT_COUNT];
  int64_t count[PT_COUNT] = {0, 0, 0, 0};
  // lists
  Csr U, V, W, X;
  DevBuf<int> V_cls;                    // offset class of every V entry (0..48)
  DevBuf<int> leaves;                   // leaf box ids
  int n_leaves = 0;
  DevBuf<int> nonleaf;                  // all non-leaf boxes ordered by level
  std::vector<int> nonleaf_off;         // [n_levels + 1] offsets into nonleaf
  DevBuf<int> xbox;                     // boxes with non-empty X list
  int n_xbox = 0;
  // P2L work items (box, first position in p2l_src, sources), their partial
  // coefficient rows (offsets p2l_poff) and each X box's first item
  DevBuf<int4> p2l_items;
  DevBuf<int> p2l_src, p2l_boff;
  DevBuf<long long> p2l_poff;
  DevBuf<cd> p2l_part;
  int n_p2l_items = 0;
  size_t p2l_sm = 0;
  DevBuf<int> vbox;                     // boxes with non-empty V list
  int n_vbox = 0;
  // orders and scales: box order pb_l per level (0 on levels 0 and 1, which
  // carry no expansions), Q_l = 2 pb_l + 1 coefficients per box
  std::vector<int> h_pb;                // [n_levels]
  int pb_max = 0, pb_fine = 0;          // largest order; order at the finest level
  DevBuf<int> lpb;                      // [n_levels]
  DevBuf<long long> eoff;               // [n_boxes] first coefficient of each box
  int64_t n_coef = 0;                   // coefficients per expansion array
  DevBuf<double> scale;                 // per level s_l = min(1, k * side_l)
  DevBuf<double> pw, ipw;               // per level powers s^j, s^-j
  DevBuf<int> src_leaves;               // leaves holding sources (levels >= 2)
  int n_src_leaves = 0;
  // P2M items over segments of the source leaves (first segment, segments,
  // first packed source, sources); per segment its leaf, rows in its item and
  // partial-row offset; per source leaf its first segment; per packed source
  // its index and leaf
  DevBuf<int4> p2m_items;
  DevBuf<int> p2m_segleaf, p2m_lseg, p2m_src, p2m_srcleaf;
  DevBuf<int2> p2m_segrow;
  DevBuf<long long> p2m_segpoff;
  DevBuf<cd> p2m_part;
  int n_p2m_items = 0;
  size_t p2m_sm = 0;
  // xbox and vbox are ordered by level; [n_levels + 1] offsets
  std::vector<int> xbox_off, vbox_off;
  int q_leaf = 1, q_w = 1;              // largest Q_l among leaves / W-list boxes
  DevBuf<int> cleaf;                    // [n_centres] leaf of each sorted centre
  int cleaf_pb_max = 0;                 // largest order of a leaf holding centres
  DevBuf<int> tleaf;                    // [n_targets] leaf of each sorted target
  DevBuf<int> dtgt, utgt, wtgt;         // direct targets (sorted indices): all, with
  int n_dtgt = 0, n_utgt = 0, n_wtgt = 0;  // U-list sources, with a W list
  DevBuf<int> m2p_tgt, m2p_box, m2p_off;   // M2P (target, W box) pairs, CSR by wtgt position
  DevBuf<cd> m2p_part;                   // [pairs] partial values
  int n_m2p_pairs = 0;
  DevBuf<int> m2p_wbox;                  // boxes M2P reads (mixed path converts them)
  int n_m2p_wbox = 0;
  DevBuf<float2> m2p_mu;                 // [n_coef] their sigma-normalised FP32 multipoles
  DevBuf<double2> m2p_rec;               // [n_levels][pbmax + 2] sigma-scaled Hankel recurrence
  DevBuf<int> m2p_t;                     // [n_levels][pbmax + 2] round(log2 sig_m)
  DevBuf<double2> sigr;                  // [n_levels][pbmax + 2] (sig_{m-1}/sig_m, sig_{m+1}/sig_m)
  DevBuf<int> m2p_scaled;                // [n_levels] 1: the unscaled recurrence could overflow
  // Centre sets: [0] every centre, [1] the centres some target uses. Each
  // lists sorted centre indices (clist) and its M2QBXL work items, the
  // (sorted centre, W-list box) pairs grouped by list position (CSR wp_off).
  CentreSet cset[2];
  int n_wpairs = 0;                     // pairs over all centres (statistics)
  DevBuf<cd> wpart;                     // [max pairs][2p+1] partial coefficients
  // mixed-precision M2QBXL and L2QBXL: coefficients in split form (FP32
  // mantissa, exponent; the multipoles while M2QBXL runs, then the leaf locals
  // for L2QBXL, which starts after it) and the powers s^j (|j| <= p) of every
  // level
  DevBuf<float2> sp_m;
  DevBuf<int> sp_e, sf_e;
  DevBuf<float> sf_m;
  DevBuf<int> wd_off, wd_box;           // per centre: W-list boxes summed directly (CSR)
  DevBuf<cd> t_m2l;                     // [n_levels][49][4 pb_max + 1] scaled Hankel vectors
  DevBuf<cd> t_m2m;                     // [n_levels][4][4 pb_max + 1] conj(V_m(d)) child->parent
  DevBuf<cd> t_l2l;                     // [n_levels][4][4 pb_max + 1] (-1)^m V_m(d) parent->child
  // sorted particle data used by the eval kernels
  DevBuf<double2> s_xy, s_nrm, c_xy, t_xy;
  DevBuf<double> c_r;                   // sorted centre radii
  DevBuf<int> t_assoc;                  // association of sorted targets (centre id or -1)
  // expansions
  DevBuf<cd> mpole, local;              // [n_coef], box b at eoff[b]
  DevBuf<cd> lpq;                       // [n_coef], leaf L2P coefficients in cos/sin form
  DevBuf<cd> qs, ds;                    // sorted strengths
  DevBuf<float2> q32;                   // their FP32 charges and dipole factors (mixed path)
  DevBuf<float4> ab32;
  DevBuf<int> err;                      // device error flags
  // mixed precision (sigma-normalised FP32 M2L)
  DevBuf<double> lsig, conv;            // [n_levels][pb_max+1] log sig_j, s^j / sig_j
  DevBuf<double> isig;                  // [n_levels][pb_max+2] 1 / sig_min(j, pb) (mixed P2M)
  DevBuf<float2> tm_f32;                // per level l >= 2: [49][Q_l][Q_l] M2L matrices
  std::vector<long long> h_tm_off;      // [n_levels] offset of level l's matrices
  // M2L as batched GEMMs: V entries grouped by (level, offset class) into
  // rows; work items over tiles of rows, row offsets into the result
  // buffers, and the result row of every V entry
  DevBuf<long long> m2l_goff;           // [n_levels * 49] matrix offset per (level, class)
  DevBuf<int4> m2l_items32, m2l_items64;  // (first row, rows, first output order, group)
  int n_m2l_items32 = 0, n_m2l_items64 = 0;
  DevBuf<long long> m2l_eyoff;          // result-row offset of every V entry
  DevBuf<long long> m2l_rowoff;         // coefficient offset of each row's source box
  DevBuf<long long> m2l_yoff;
  DevBuf<float2> m2l_y;
  DevBuf<cd> tm_f64;                    // FP64 M2L matrices (same offsets as the FP32 ones)
  DevBuf<cd> m2l_y64;                   // FP64 result rows of the FP64 M2L GEMM
  DevBuf<int> m2l_vsrc;                 // boxes that are V-list sources
  int n_vsrc = 0;
  DevBuf<float2> mu32;                  // [n_coef] their sigma-normalised FP32 multipoles
  DevBuf<float2> tl_f32;                // per parent level l: [4][Q_l][Q_{l+1}] L2L matrices
  std::vector<long long> h_tl_off;
  DevBuf<float2> tmm_f32;               // per parent level l: [4][Q_{l+1}][Q_l] M2M matrices
  std::vector<long long> h_tmm_off;
  // tensor-core M2L of the FP64 path (m2l_tc.cu)
  std::vector<int> h_row_src;           // source box of every M2L row
  std::vector<int64_t> h_gcount;        // [n_levels * 49 + 1] first row of every group
  std::vector<int4> h_items64;          // the FP64 GEMM items (host copy)
  DevBuf<int4> m2l_items64_rest;        // FP64 GEMM items of the levels left to it
  int n_m2l_items64_rest = 0;
  std::vector<int4> h_tc_lvl;           // per level (use, beta, S, padded 2Q)
  DevBuf<int4> tc_lvl;
  DevBuf<int4> tc_gp;                   // per group (K, Q, beta, Np) of the tile product
  std::vector<TcLevelOp> tc_m2m, tc_l2l;  // per parent level (FP64 path)
  // FP64 M2L through TMA: the rows' source slices copied into row order per
  // group ([S][rows][K] at x2off), and the tensor maps of those copies and of
  // the matrix slices, per group
  bool tc_tma = false;
  int n_tc_rows = 0;
  DevBuf<uint16_t> tc_X2;
  DevBuf<long long> tc_x2src, tc_x2dst, tc_x2ts, tc_gstart;
  DevBuf<int2> tc_x2sk;
  DevBuf<TmapBlob> tc_mapA, tc_mapX;
  DevBuf<cd> tc_mml_y;                  // their result rows (one level at a time)
  bool tc_any = false;
  DevBuf<uint16_t> tc_A;                // bf16 matrix slices [S][Kp][Kp] per group
  DevBuf<int> tc_fexp;                  // row exponents [Kp] per group
  DevBuf<long long> tc_gaoff, tc_gfoff; // [n_levels * 49] offsets of a group's slices / exponents
  DevBuf<int> tc_src;                   // V-list sources on tensor-core levels
  int n_tc_src = 0;
  DevBuf<long long> tc_xoff;            // their bf16 vector slices [S][Kp]
  DevBuf<int> tc_xexp;                  // and exponents
  DevBuf<uint16_t> tc_X;
  DevBuf<int> tc_rowsrc;                // per M2L row: position of its source in tc_src
  DevBuf<int4> tc_items[3];             // (first row, rows, first output, group) for S = 6, 7, 8
  int n_tc_items[3] = {0, 0, 0};
};

qbx_status mixed_plan_build(qbx_handle* h, FmmPlan* f);
qbx_status configure_mixed_kernels(int smem_optin);
qbx_status launch_m2l_f32(qbx_handle* h, FmmPlan* f, cudaStream_t s);
qbx_status launch_l2l_f32(qbx_handle* h, FmmPlan* f, cudaStream_t s);
qbx_status launch_m2m_f32(qbx_handle* h, FmmPlan* f, cudaStream_t s);
qbx_status launch_m2l_f64(qbx_handle* h, FmmPlan* f, cudaStream_t s);
qbx_status launch_m2l_f64_gemm_rest(qbx_handle* h, FmmPlan* f, cudaStream_t s);
// m2l_tc.cu
qbx_status configure_tc_kernels(int smem_optin);
qbx_status tc_plan_build(qbx_handle* h, FmmPlan* f);
qbx_status tc_mml_plan_build(qbx_handle* h, FmmPlan* f);
// FP64 M2M (kind 0) or L2L (kind 1) of parent level l on the tensor cores;
// *done = false when the level stays on the CUDA-core kernel
qbx_status launch_mml_tc(qbx_handle* h, FmmPlan* f, int kind, int l, bool* done, cudaStream_t s);
qbx_status launch_m2l_tc(qbx_handle* h, FmmPlan* f, bool mixed, cudaStream_t s);
// shared memory of one M2M / L2L tile-GEMM block at box order pb
size_t gemm_smem_bytes(int pb);

qbx_status tree_build(qbx_handle* h, FmmPlan* f, int n_max, double kappa);
qbx_status tree_lists(qbx_handle* h, FmmPlan* f);
qbx_status gather_sorted(qbx_handle* h, FmmPlan* f);
qbx_status tree_associate(qbx_handle* h, FmmPlan* f, const int64_t* on_node, const int8_t* on_side,
                          double eps);
