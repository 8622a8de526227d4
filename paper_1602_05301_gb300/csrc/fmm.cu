// FMM-accelerated Global QBX (Sec. 7.2, Stages 2-8), FP64.
//
// Expansions about box centres, with per-level scale s = min(1, k * side):
//   multipole  phi(x) = sum_n  mh_n s^|n| W_n(x - m)            (H-expansion)
//   local      psi(x) = sum_n  lh_n s^-|n| conj(V_n(x - m))      (J-expansion)
// where W_n(z) = H_n(k|z|) e^{i n arg z} and V_n(z) = J_n(k|z|) e^{i n arg z}.
// Storing mh = a / s^|n| and lh = gamma s^|n| keeps the stored numbers of
// order one although H_n grows and J_n decays factorially with n for small
// k*side. The operators come from Graf's addition theorem (DLMF 10.23.7):
//   W_n(A - B) = sum_l W_{n+l}(A) conj(V_l(B))   (|B| < |A|),
//   V_n(A - B) = sum_l V_{n+l}(A) conj(V_l(B))   (all A, B),
// giving, in unscaled form (d the translation vector),
//   P2M   a_n     = sum_j q_j conj(V_n(y_j - m))                   (Stage 2)
//   M2M   a_s     = sum_n a'_n conj(V_{s-n}(m' - m))               (Stage 2)
//   M2L   gamma_l = (-1)^l sum_n a_n W_{n+l}(m_b - m_c)            (Stage 4)
//   P2L   gamma_l = sum_j q_j W_l(y_j - m)                         (Stage 6)
//   L2L   gamma'_s = sum_n gamma_n (-1)^{s-n} V_{s-n}(m' - m)      (Stage 7)
// and the QBX steps marked "New" in the paper: P2QBXL (Stage 3), M2QBXL
// (Stage 5) and L2QBXL (Stage 8) are P2L, M2L and L2L with a QBX centre as the
// target and order p. A double-layer source contributes
// (k/2)(nu Z_{n-1} - conj(nu) Z_{n+1}) for Z = W, and the conjugate form for
// conj(V), with nu = n_x + i n_y its normal (normal derivative of the Graf
// kernel in the source).
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <set>
#include <vector>

#include "special.cuh"
#include "tree.cuh"

namespace {

constexpr int kThreads = 128;
// CTA size of the per-leaf kernels (threads over the centres or targets of one
// leaf). Leaves that hold centres are kept at least kLeafOverRadius disk radii
// wide, so they carry many centres (about 65 on the starfish workloads) and few
// leaves hold any: one warp per leaf left most SMs idle (measured 2x slower).
constexpr int kLeafThreads = 128;
// Sources per shared-memory chunk in P2M / P2L. Their rows (one FP64 recurrence
// per source) are built by threads 0..kChunk-1, a full warp: the SM's FP64
// rate is shared by its warps and a warp instruction costs the same with few
// lanes active, so partly filled warps waste it (measured).
constexpr int kChunk = 32;
// Leaves holding a centre are at least this many expansion radii wide.
constexpr double kLeafOverRadius = 4.0;
// A W-list box c is translated to a centre z (M2QBXL) only if
// (R_c + r_z) <= kW * |z - m_c| (R_c: half-diagonal of c, r_z: disk radius);
// otherwise its sources are summed directly into the coefficients.
constexpr double kW = 0.6;

inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }
// opt-in shared memory per block of the current device (set by configure_kernels)
int g_smem_optin = 48 * 1024;
#define TRY_MIXED(x)                    \
  do {                                  \
    qbx_status s_ = (x);                \
    if (s_ != QBX_OK) return s_;        \
  } while (0)

struct Fmm {
  // boxes
  const int* level;
  const int* child;
  const double2* centre;
  const int2* rsrc;
  const int2* rctr;
  const int2* rtgt;
  // lists
  const int *uoff, *uidx, *voff, *vidx, *vcls, *woff, *widx, *xoff, *xidx;
  // sorted particles
  const double2* sxy;
  const double2* snrm;
  const cd* qs;
  const cd* ds;
  const float2* q32;     // FP32 charges (mixed path)
  const float4* ab32;    // FP32 dipole factors (A, B) (mixed path)
  const double2* cxy;
  const double* crad;    // sorted centre radii
  const int* cid;
  const double2* txy;
  const int* tid;
  const int* tassoc;
  // orders and tables (box order pb_l per level; Q_l = 2 pb_l + 1 coefficients)
  const int* lpb;        // [n_levels]
  const long long* eoff; // [n_boxes] first coefficient of each box in mpole / local
  const double* scale;   // [n_levels]
  const double* pw;      // [n_levels][2 pbmax + 3] s^j
  const double* ipw;     // [n_levels][pbmax + 2]  s^-j
  const cd* t_m2l;       // [n_levels][49][4 pbmax + 1], order m stored at m + 2 pbmax
  const cd* t_m2m;       // [n_levels][4][4 pbmax + 1]
  const cd* t_l2l;       // [n_levels][4][4 pbmax + 1]
  cd* mpole;
  cd* local;
  cd* lpq;               // [n_coef] leaf cos/sin coefficients of L2P (see unscale_leaf_locals_kernel)
  const double* conv;    // [n_levels][pbmax + 1] s^j / sig_j (mixed path)
  const double* lsig;    // [n_levels][pbmax + 1] log sig_j
  const double* isig;    // [n_levels][pbmax + 2] 1 / sig_min(j, pb) (mixed P2M)
  const double2* sigr;   // [n_levels][pbmax + 2] (sig_{j-1} / sig_j, sig_{j+1} / sig_j)
  double k, ik, side;    // wavenumber, 1 / k, root box side
  int pbmax, p, n_levels, has_S, has_D;
};

__device__ __forceinline__ const double* pw_row(const Fmm& F, int l) { return F.pw + (size_t)l * (2 * F.pbmax + 3); }
__device__ __forceinline__ const double* ipw_row(const Fmm& F, int l) { return F.ipw + (size_t)l * (F.pbmax + 2); }
// Centred translation table of (level l, item): entry m at [m].
__device__ __forceinline__ const cd* table(const Fmm& F, const cd* t, int items, int l, int item) {
  return t + ((size_t)l * items + item) * (4 * F.pbmax + 1) + 2 * F.pbmax;
}

// Unnormalised Miller recurrence for J_0..J_M of x into row[0..M]; returns the
// normalisation (divide by it). Rescales the stored part when values grow.
__device__ double miller_row(double x, int M, double* row, int stride) {
  if (x < 1e-8) {
    double t = 1.0;
    for (int i = 0; i <= M; ++i) {
      row[i * stride] = t;
      t *= 0.5 * x / (double)(i + 1);
    }
    return 1.0;
  }
  const double inv = 2.0 / x;
  const int N = miller_start(M, x);  // > M + 1: every row entry is written
  double fn1 = 0.0, fn = 0x1p-600, sum = 0.0, dn = (double)N;
  for (int n = N; n >= 1; --n) {
    const double fm = fma(dn * inv, fn, -fn1);  // f_{n-1} = (2n/x) f_n - f_{n+1}
    dn -= 1.0;
    if ((n & 1) == 0) sum += fn;
    if (n - 1 <= M) row[(n - 1) * stride] = fm;
    fn1 = fn;
    fn = fm;
    // rescale by 2^-332 (exact) once |f| reaches 2^332: an integer test on the
    // exponent field
    if ((__double2hiint(fn) & 0x7FFFFFFF) >= (1355 << 20)) {
      const double sc = 0x1p-332;
      fn *= sc;
      fn1 *= sc;
      sum *= sc;
      for (int i = n - 1; i <= M; ++i) row[i * stride] *= sc;
    }
  }
  return fn + 2.0 * sum;
}

// ---------------------------------------------------------------- translation tables
// One thread per (level, item): items 0..48 M2L offset classes, 49..52 M2M
// quadrants, 53..56 L2L quadrants. Rows have stride 4 pbmax + 1 with order m
// at m + 2 pbmax; only the orders a level's translations read are written:
// |m| <= 2 pb_l for M2L, |m| <= pb_l + pb_{l+1} for M2M / L2L. Levels 0 and 1
// carry no expansions.
__global__ void tables_kernel(int n_levels, double side, double k, int pbmax,
                              const int* __restrict__ lpb, const double* __restrict__ scale,
                              cd* __restrict__ t_m2l, cd* __restrict__ t_m2m,
                              cd* __restrict__ t_l2l, double* __restrict__ jwork) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_levels * 57) return;
  const int l = g / 57, item = g % 57;
  const int TS = 4 * pbmax + 1, C = 2 * pbmax;
  const int pb = lpb[l];
  if (l < 2 || pb == 0) return;
  const double sl = side / (double)(1 << l);
  if (item < 49) {
    cd* out = t_m2l + ((size_t)l * 49 + item) * TS + C;
    const int dx = item / 7 - 3, dy = item % 7 - 3;  // (ix_b - ix_c, iy_b - iy_c)
    if (max(abs(dx), abs(dy)) < 2) return;          // not a V-list offset
    const int M = 2 * pb;
    const double s = scale[l];
    const double Dx = dx * sl, Dy = dy * sl, r = sqrt(Dx * Dx + Dy * Dy), x = k * r;
    const cd e1 = mk(Dx / r, Dy / r);
    cd h0, h1;
    hankel01(x, h0, h1);
    cd hm1 = h0, hm = cscale(h1, s);  // scaled H_m s^m
    cd e = mk(1.0, 0.0);
    out[0] = h0;
    for (int m = 1; m <= M; ++m) {
      e = cmul(e, e1);
      out[m] = cmul(hm, e);
      const double sg = (m & 1) ? -1.0 : 1.0;
      out[-m] = cscale(cmul(hm, cconj(e)), sg);
      // next: H_{m+1} s^{m+1} = (2m/x) s H_m s^m - s^2 H_{m-1} s^{m-1}
      const cd hn = csub(cscale(hm, 2.0 * m * s / x), cscale(hm1, s * s));
      hm1 = hm;
      hm = hn;
    }
    return;
  }
  if (l + 1 >= n_levels) return;
  const bool m2m = item < 53;
  const int c = m2m ? item - 49 : item - 53;
  cd* out = (m2m ? t_m2m : t_l2l) + ((size_t)l * 4 + c) * TS + C;
  const int M = pb + lpb[l + 1];
  // child centre minus parent centre, child side = sl/2
  const double cs = 0.5 * sl;
  const double dx = ((c & 1) - 0.5) * cs, dy = ((c >> 1) - 0.5) * cs;
  const double r = sqrt(dx * dx + dy * dy), x = k * r;
  double* J = jwork + (size_t)g * (2 * pbmax + 1);
  const double norm = miller_row(x, M, J, 1);
  const cd e1 = mk(dx / r, dy / r);
  cd e = mk(1.0, 0.0);
  for (int m = 0; m <= M; ++m) {
    const double j = J[m] / norm;
    const double sg = (m & 1) ? -1.0 : 1.0;
    if (m2m) {  // conj(V_m) = J_m e^{-im th}; conj(V_{-m}) = (-1)^m J_m e^{im th}
      out[m] = cscale(cconj(e), j);
      out[-m] = cscale(e, sg * j);
    } else {    // (-1)^m V_m = (-1)^m J_m e^{im th}; (-1)^m V_{-m} = J_m e^{-im th}
      out[m] = cscale(e, sg * j);
      out[-m] = cscale(cconj(e), j);
    }
    e = cmul(e, e1);
  }
}

// Per level: pw[j] = s^j for j <= 2 pb_l + 2, ipw[j] = s^-j for j <= pb_l + 1 (rest 0).
__global__ void powers_kernel(int n_levels, int pbmax, const int* __restrict__ lpb,
                              const double* __restrict__ scale, double* __restrict__ pw,
                              double* __restrict__ ipw) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_levels) return;
  const double s = scale[l];
  const int pb = lpb[l];
  double a = 1.0;
  for (int j = 0; j < 2 * pbmax + 3; ++j) {
    pw[(size_t)l * (2 * pbmax + 3) + j] = j <= 2 * pb + 2 ? a : 0.0;
    a *= s;
  }
  a = 1.0;
  for (int j = 0; j < pbmax + 2; ++j) {
    ipw[(size_t)l * (pbmax + 2) + j] = j <= pb + 1 ? a : 0.0;
    if (j <= pb + 1) a /= s;
  }
}

// ---------------------------------------------------------------- strengths
// Sorted strengths; for the mixed path also their FP32 forms, with the dipole
// factors A = d (k/2) nu and B = d (k/2) conj(nu) (nu = n_x + i n_y) formed
// once per source instead of once per (source, centre) pair.
__global__ void gather_strengths_kernel(int64_t n, const int* __restrict__ perm,
                                        const cd* __restrict__ q, const cd* __restrict__ d,
                                        const double2* __restrict__ snrm, double k,
                                        cd* __restrict__ qs, cd* __restrict__ ds,
                                        float2* __restrict__ q32, float4* __restrict__ ab32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cd qi = q[perm[i]], di = d[perm[i]];
  qs[i] = qi;
  ds[i] = di;
  if (q32) {
    const cd dk = cscale(di, 0.5 * k);
    const cd nu = mk(snrm[i].x, snrm[i].y);
    const cd A = cmul(dk, nu), B = cmul(dk, cconj(nu));
    q32[i] = make_float2((float)qi.x, (float)qi.y);
    ab32[i] = make_float4((float)A.x, (float)A.y, (float)B.x, (float)B.y);
  }
}

// ---------------------------------------------------------------- P2M (Stage 2)
// Shared memory of the source-row kernels (P2M, P2L): an accumulator per output
// order, then up to kChunk rows of 2 pb + 3 table values and three strengths.
__host__ __device__ inline size_t rows_smem(int pb, int chunk) {
  return ((size_t)(2 * pb + 1) + (size_t)chunk * (2 * pb + 6)) * sizeof(cd);
}
__host__ __device__ inline int rows_chunk(int pb, size_t sm_bytes) {
  const size_t per = (size_t)(2 * pb + 6) * sizeof(cd);
  const size_t avail = sm_bytes - (size_t)(2 * pb + 1) * sizeof(cd);
  const size_t c = avail / per;
  return (int)(c < (size_t)kChunk ? c : (size_t)kChunk);
}

// Row of source i for the multipole of a box with centre m, order pb and
// scale s: row[t] = conj(V_t(y_i - m)) / s^|t|, |t| <= pb + 1 (row points at
// t = 0), and the source's charge and dipole factors in sq, sa, sb.
__device__ __forceinline__ void p2m_fill_row(const Fmm& F, int i, double2 m, double is, int pb,
                                             cd* row, cd& sq, cd& sa, cd& sb) {
  const double dx = F.sxy[i].x - m.x, dy = F.sxy[i].y - m.y;
  const double rr = sqrt(dx * dx + dy * dy);
  // J_0..J_{pb+1} (unnormalised) into the real parts of row[0..pb+1]
  const double norm = miller_row(F.k * rr, pb + 1, (double*)row, 2);
  const cd em = rr > 0.0 ? mk(dx / rr, -dy / rr) : mk(1.0, 0.0);  // e^{-i th}
  cd e = mk(1.0, 0.0);
  double f = 1.0 / norm;
  for (int j = 0; j <= pb + 1; ++j) {
    const double v = row[j].x * f;                // J_j / s^j
    const cd c = cscale(e, v);                    // conj(V_j) / s^j
    row[j] = c;
    if (j > 0) row[-j] = (j & 1) ? mk(-c.x, c.y) : mk(c.x, -c.y);  // (-1)^j conj(c)
    e = cmul(e, em);
    f *= is;
  }
  const cd dk = cscale(F.ds[i], 0.5 * F.k);
  const cd nu = mk(F.snrm[i].x, F.snrm[i].y);
  sq = F.qs[i];
  sa = cmul(dk, cconj(nu));
  sb = cmul(dk, nu);
}

// Order n of a box's multipole from rows j0..j1 of the staged rows:
// a_n = sum_j [q_j row_j[n] + s^{|n-1| - |n|} A_j row_j[n-1] - s^{|n+1| - |n|} B_j row_j[n+1]]
// (charge and dipole terms in separate sums, each scaled once).
__device__ __forceinline__ cd p2m_order(const Fmm& F, const cd* rows, int RW, const cd* sq,
                                        const cd* sa, const cd* sb, int j0, int j1, int n,
                                        double s, double is) {
  const int an = abs(n);
  // conj(V_{n-+1})/s^|n| = row[n-+1] s^{|n-+1| - |n|}
  const double fm = (abs(n - 1) > an) ? s : is;
  const double fp = (abs(n + 1) > an) ? s : is;
  cd aq = mk(0.0, 0.0), aa = mk(0.0, 0.0), ab = mk(0.0, 0.0);
  for (int j = j0; j < j1; ++j) {
    const cd* row = rows + j * RW;
    if (F.has_S) cfma(aq, sq[j], row[n]);
    if (F.has_D) {
      cfma(aa, sa[j], row[n - 1]);
      cfma(ab, sb[j], row[n + 1]);
    }
  }
  return cadd(aq, csub(cscale(aa, fm), cscale(ab, fp)));
}

// P2M work: every source leaf's sources are cut into segments of at most a
// row chunk; segments of one level are packed into items of up to a chunk of
// sources (item = (first segment, segments, first packed source, sources)),
// so small leaves share a CTA and large ones spread over several. One warp
// fills the item's rows with full lanes; then the threads run over
// (segment, order) pairs and write each segment's part of its leaf's multipole
// to partial[seg_poff[segment] + n + pb]; p2m_sum_kernel adds a leaf's
// segments in order.
__global__ void __launch_bounds__(kThreads) p2m_item_kernel(Fmm F, const int4* __restrict__ items,
                                                            const int* __restrict__ seg_leaf,
                                                            const int2* __restrict__ seg_row,
                                                            const long long* __restrict__ seg_poff,
                                                            const int* __restrict__ src,
                                                            const int* __restrict__ src_leaf,
                                                            cd* __restrict__ partial,
                                                            unsigned sm_bytes) {
  extern __shared__ cd smem[];
  const int4 it = items[blockIdx.x];
  const int l = F.level[seg_leaf[it.x]];
  const int pb = F.lpb[l], Q = 2 * pb + 1, RW = 2 * pb + 3;
  const int chunk = rows_chunk(pb, sm_bytes);  // >= it.w
  cd* rows = smem;                        // [chunk][RW]
  cd* sq = rows + chunk * RW;             // [chunk]
  cd* sa = sq + chunk;                    // [chunk]
  cd* sb = sa + chunk;                    // [chunk]
  const double s = F.scale[l], is = 1.0 / s;
  if ((int)threadIdx.x < it.w) {
    const int j = threadIdx.x;
    p2m_fill_row(F, src[it.z + j], F.centre[src_leaf[it.z + j]], is, pb, rows + j * RW + (pb + 1),
                 sq[j], sa[j], sb[j]);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < it.y * Q; idx += kThreads) {
    const int u = idx / Q, n = idx % Q - pb;
    const int2 rr = seg_row[it.x + u];
    partial[seg_poff[it.x + u] + n + pb] =
        p2m_order(F, rows + (pb + 1), RW, sq, sa, sb, rr.x, rr.x + rr.y, n, s, is);
  }
}

// mpole(leaves[t]) = sum of its segments' partial multipoles, in order
// (segments lseg[t]..lseg[t+1]).
__global__ void __launch_bounds__(kThreads) p2m_sum_kernel(Fmm F, const int* __restrict__ leaves,
                                                           const int* __restrict__ lseg,
                                                           const long long* __restrict__ seg_poff,
                                                           const cd* __restrict__ partial) {
  const int t = blockIdx.x, b = leaves[t];
  const int Q = 2 * F.lpb[F.level[b]] + 1;
  cd* dst = F.mpole + F.eoff[b];
  for (int n = threadIdx.x; n < Q; n += kThreads) {
    cd sum = mk(0.0, 0.0);
    for (int g = lseg[t]; g < lseg[t + 1]; ++g) sum = cadd(sum, partial[seg_poff[g] + n]);
    dst[n] = sum;
  }
}

// ---------------------------------------------------------------- M2M (Stage 2)
// CTA per parent (level l, order pp) over its children (level l+1, order pc):
// a_s = sum_{|n| <= pc} a'_n conj(V_{s-n}), |s| <= pp.
__host__ __device__ inline size_t m2m_smem(int pp, int pc) {
  return ((size_t)(2 * pc + 1) + (size_t)(2 * (pp + pc) + 1) + (size_t)(2 * pp + 1)) * sizeof(cd);
}

__global__ void __launch_bounds__(kThreads) m2m_kernel(Fmm F, const int* __restrict__ boxes) {
  extern __shared__ cd smem[];
  const int b = boxes[blockIdx.x];
  const int l = F.level[b];
  const int pp = F.lpb[l], pc = F.lpb[l + 1];
  const int Qp = 2 * pp + 1, Qc = 2 * pc + 1, M = pp + pc, T = 2 * M + 1;
  cd* a = smem;        // [Qc]
  cd* t = a + Qc;      // [T]  t[m + M] = conj(V_m)
  cd* acc = t + T;     // [Qp]
  const double* pwc = pw_row(F, l + 1);
  const double* ipp = ipw_row(F, l);
  for (int i = threadIdx.x; i < Qp; i += kThreads) acc[i] = mk(0.0, 0.0);
  for (int c = 0; c < 4; ++c) {
    const int d = F.child[4 * b + c];
    if (d < 0) continue;
    const cd* mp = F.mpole + F.eoff[d];
    for (int i = threadIdx.x; i < Qc; i += kThreads) a[i] = cscale(mp[i], pwc[abs(i - pc)]);
    const cd* tab = table(F, F.t_m2m, 4, l, c);
    for (int i = threadIdx.x; i < T; i += kThreads) t[i] = tab[i - M];
    __syncthreads();
    for (int s = (int)threadIdx.x - pp; s <= pp; s += kThreads) {
      cd sum = mk(0.0, 0.0);
      for (int n = -pc; n <= pc; ++n) cfma(sum, t[s - n + M], a[n + pc]);
      acc[s + pp] = cadd(acc[s + pp], sum);
    }
    __syncthreads();
  }
  cd* dst = F.mpole + F.eoff[b];
  for (int i = threadIdx.x; i < Qp; i += kThreads) dst[i] = cscale(acc[i], ipp[abs(i - pp)]);
}

// ---------------------------------------------------------------- M2L (Stage 4)
// lh_l += (-1)^l sum_n What_{n+l} mh_n c(l,n), What_m = s^|m| W_m(m_b - m_c),
// c(l,n) = s^{2 min(|l|,|n|)} when l and n have opposite signs, else 1: both
// precisions run it as tile GEMMs over dense per-(level, offset class)
// matrices (mixed.cu).

// ---------------------------------------------------------------- P2L (Stage 6)
// lh_n += s^|n| sum_j [q_j W_n + d_j (k/2)(nu_j W_{n-1} - conj(nu_j) W_{n+1})](y_j - m_b)
// over the sources of the boxes in b's X list. Work items: up to one row chunk
// of an X box's sources (its X list's leaves, concatenated in list order), so
// that a box's work spreads over several CTAs and every chunk is full. One
// warp fills a row per source with Wh_t = s^|t| W_t, |t| <= pb + 1; then all
// threads form the item's part of lh_n (the charge and the two dipole terms in
// separate sums, scaled once) into partial[poff[item] + n + pb], and
// p2l_sum_kernel adds each box's items in order.
__global__ void __launch_bounds__(kThreads) p2l_item_kernel(Fmm F, const int4* __restrict__ items,
                                                            const int* __restrict__ src,
                                                            const long long* __restrict__ poff,
                                                            cd* __restrict__ partial,
                                                            unsigned sm_bytes) {
  extern __shared__ cd smem[];
  const int4 it = items[blockIdx.x];  // (box, first position in src, sources, -)
  const int b = it.x, cnt = it.z;
  const int l = F.level[b];
  const int pb = F.lpb[l], RW = 2 * pb + 3;  // row: Wh_t, |t| <= pb+1
  const int chunk = rows_chunk(pb, sm_bytes);  // >= cnt (items are cut to fit)
  cd* rows = smem;                        // [chunk][RW]
  cd* sq = rows + chunk * RW;             // [chunk]
  cd* sa = sq + chunk;                    // [chunk]  A = d (k/2) nu
  cd* sb = sa + chunk;                    // [chunk]  B = d (k/2) conj(nu)
  const double s = F.scale[l], is = 1.0 / s;
  const double2 m = F.centre[b];
  const double hk = 0.5 * F.k;
  if ((int)threadIdx.x < cnt) {
    const int i = src[it.y + threadIdx.x];
    const double dx = F.sxy[i].x - m.x, dy = F.sxy[i].y - m.y;
    const double rr = sqrt(dx * dx + dy * dy), irr = 1.0 / rr;
    const double x = F.k * rr, ix = 1.0 / x;
    const cd e1 = mk(dx * irr, dy * irr);
    cd h0, h1;
    hankel01(x, ix, h0, h1);
    const double c1 = 2.0 * s * ix, s2 = s * s;  // Wh_{j+1} = j c1 Wh_j - s2 Wh_{j-1}
    cd* row = rows + threadIdx.x * RW + (pb + 1);   // row[t], t = -(pb+1)..pb+1
    cd hm1 = h0, hm = cscale(h1, s), ee = mk(1.0, 0.0);
    row[0] = h0;
    for (int j = 1; j <= pb + 1; ++j) {
      ee = cmul(ee, e1);
      const double ac = hm.x * ee.x, bd = hm.y * ee.y, ad = hm.x * ee.y, bc = hm.y * ee.x;
      row[j] = mk(ac - bd, ad + bc);                                       // s^j W_j
      row[-j] = (j & 1) ? mk(-(ac + bd), ad - bc) : mk(ac + bd, bc - ad);  // s^j W_{-j}
      const cd hn = csub(cscale(hm, j * c1), cscale(hm1, s2));
      hm1 = hm;
      hm = hn;
    }
    const cd dk = cscale(F.ds[i], hk);
    const cd nu = mk(F.snrm[i].x, F.snrm[i].y);
    sq[threadIdx.x] = F.qs[i];
    sa[threadIdx.x] = cmul(dk, nu);
    sb[threadIdx.x] = cmul(dk, cconj(nu));
  }
  __syncthreads();
  cd* dst = partial + poff[blockIdx.x] + pb;
  for (int n = (int)threadIdx.x - pb; n <= pb; n += kThreads) {
    const int an = abs(n);
    // s^|n| W_{n-1} = Wh_{n-1} s^{|n| - |n-1|}, s^|n| W_{n+1} = Wh_{n+1} s^{|n| - |n+1|}
    const double fm = (abs(n - 1) > an) ? is : s;
    const double fp = (abs(n + 1) > an) ? is : s;
    cd aq = mk(0.0, 0.0), aa = mk(0.0, 0.0), ab = mk(0.0, 0.0);
    for (int j = 0; j < cnt; ++j) {
      const cd* row = rows + j * RW + (pb + 1);
      if (F.has_S) cfma(aq, sq[j], row[n]);
      if (F.has_D) {
        cfma(aa, sa[j], row[n - 1]);
        cfma(ab, sb[j], row[n + 1]);
      }
    }
    dst[n] = cadd(aq, csub(cscale(aa, fm), cscale(ab, fp)));
  }
}

// lh(xbox[t]) += its items' partial coefficients, in item order.
__global__ void __launch_bounds__(kThreads) p2l_sum_kernel(Fmm F, const int* __restrict__ xbox,
                                                           const int* __restrict__ boff,
                                                           const long long* __restrict__ poff,
                                                           const cd* __restrict__ partial) {
  const int t = blockIdx.x, b = xbox[t];
  const int pb = F.lpb[F.level[b]], Q = 2 * pb + 1;
  cd* dst = F.local + F.eoff[b];
  for (int n = threadIdx.x; n < Q; n += kThreads) {
    cd sum = mk(0.0, 0.0);
    for (int it = boff[t]; it < boff[t + 1]; ++it) sum = cadd(sum, partial[poff[it] + n]);
    dst[n] = cadd(dst[n], sum);
  }
}

// ---------------------------------------------------------------- L2L (Stage 7)
// CTA per parent (level l, order pp) into its children (order pc):
// gamma'_s = sum_{|n| <= pp} gamma_n (-1)^{s-n} V_{s-n}, |s| <= pc.
__host__ __device__ inline size_t l2l_smem(int pp, int pc) {
  return ((size_t)(2 * pp + 1) + (size_t)(2 * (pp + pc) + 1)) * sizeof(cd);
}

__global__ void __launch_bounds__(kThreads) l2l_kernel(Fmm F, const int* __restrict__ boxes) {
  extern __shared__ cd smem[];
  const int b = boxes[blockIdx.x];
  const int l = F.level[b];
  const int pp = F.lpb[l], pc = F.lpb[l + 1];
  const int Qp = 2 * pp + 1, M = pp + pc, T = 2 * M + 1;
  cd* g = smem;   // true local coefficients gamma_n
  cd* t = g + Qp;
  const double* ipp = ipw_row(F, l);
  const double* pwc = pw_row(F, l + 1);
  const cd* lp = F.local + F.eoff[b];
  for (int i = threadIdx.x; i < Qp; i += kThreads) g[i] = cscale(lp[i], ipp[abs(i - pp)]);
  for (int c = 0; c < 4; ++c) {
    const int d = F.child[4 * b + c];
    if (d < 0) continue;
    const cd* tab = table(F, F.t_l2l, 4, l, c);
    for (int i = threadIdx.x; i < T; i += kThreads) t[i] = tab[i - M];
    __syncthreads();
    cd* dl = F.local + F.eoff[d];
    for (int s = (int)threadIdx.x - pc; s <= pc; s += kThreads) {
      cd sum = mk(0.0, 0.0);
      for (int n = -pp; n <= pp; ++n) cfma(sum, t[s - n + M], g[n + pp]);
      dl[s + pc] = cadd(dl[s + pc], cscale(sum, pwc[abs(s)]));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- targets (Stages 3, 5, 8)
// CTA per leaf; one thread per target of the leaf (strided). Only targets that
// are not associated with a QBX centre are evaluated.
// L2P writes out[t], M2P and P2P add to it.
// Sources of a list of boxes, concatenated: the boxes of leaf b's U list
// (U.idx[uoff[b]..uoff[b+1])) followed by the boxes xidx[x0..x1) (the W-list
// boxes summed directly for one centre; empty for targets). Lane `lane` takes
// the sources t = lane, lane + 32, ... of the concatenation (a cursor per lane
// walks the boxes), so a warp runs ceil(total / 32) iterations.
struct SourceCursor {
  const int* uidx;   // the U-list index array
  const int2* rsrc;  // source range of every box
  int u0, nu, x0, nx;
  const int* xidx;
  __device__ int box(int e) const { return e < nu ? uidx[u0 + e] : xidx[x0 + e - nu]; }
  __device__ int total() const {
    int t = 0;
    for (int e = 0; e < nu + nx; ++e) {
      const int2 r = rsrc[box(e)];
      t += r.y - r.x;
    }
    return t;
  }
};

template <typename Fn>
__device__ __forceinline__ void deal_sources(const SourceCursor& sc, int lane, Fn&& fn) {
  const int tot = sc.total();
  int e = 0, base = 0;
  int2 r = sc.nu + sc.nx > 0 ? sc.rsrc[sc.box(0)] : make_int2(0, 0);
  for (int t = lane; t < tot; t += 32) {
    while (t >= base + (r.y - r.x)) {  // advance to the box holding source t
      base += r.y - r.x;
      r = sc.rsrc[sc.box(++e)];
    }
    fn(r.x + (t - base));
  }
}

// L2P: one thread per direct target (sorted index list), from the local
// coefficients of its leaf in cosine/sine form (P_m, Q_m); adds to out. The
// backward recurrence yields f_m for descending m, and Clenshaw's recurrences
// for the cosine and sine sums run in the same loop (two FMAs per real
// component and order, no complex products).
__global__ void __launch_bounds__(kThreads) l2p_kernel(Fmm F, const int* __restrict__ dtgt,
                                                       const int* __restrict__ tleaf, int n,
                                                       cd* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = dtgt[t];
  const int b = tleaf[i];
  const int pb = F.lpb[F.level[b]];
  const cd* g = F.local + F.eoff[b];
  const double2 m = F.centre[b];
  const double dx = F.txy[i].x - m.x, dy = F.txy[i].y - m.y;
  const double d2 = dx * dx + dy * dy;
  const bool at_centre = (__double2hiint(d2) | __double2loint(d2)) == 0;
  const double ir = at_centre ? 0.0 : rsqrt(d2), x = F.k * (d2 * ir);
  const cd e1 = at_centre ? mk(1.0, 0.0) : mk(dx * ir, dy * ir);
  // psi = sum_m f_m [g_m e^{-im th} + (m>0) (-1)^m g_{-m} e^{im th}] / norm
  cd acc;
  double norm;
  if (x < 1e-8) {
    // J_m(x) = (x/2)^m / m! to relative O(x^2); the terms vanish after a few
    // orders (a target a rounding distance from the leaf centre still needs
    // the m = 1 term: it is O(x) of the result, not O(x^2))
    acc = mk(0.0, 0.0);
    norm = 1.0;
    double t = 1.0;
    cd e = mk(1.0, 0.0);  // e^{i m th}
    for (int mm = 0; mm <= pb && t != 0.0; ++mm) {
      acc = cadd(acc, cscale(cmul(g[pb + mm], cconj(e)), t));
      if (mm > 0) acc = cadd(acc, cscale(cmul(g[pb - mm], e), (mm & 1) ? -t : t));
      t *= 0.5 * x / (double)(mm + 1);
      e = cmul(e, e1);
    }
  } else {
    // Miller's backward recurrence for f_m ~ J_m(x) (unnormalised), fused with
    // Clenshaw's recurrences for sum_m f_m P_m cos(m th) (u: b_{m+1}, b_{m+2})
    // and sum_m f_m Q_m sin(m th) (v), both run from m = pb down:
    //   b_m = f_m c_m + 2 cos(th) b_{m+1} - b_{m+2},
    //   sum c_m cos(m th) = b_0 - cos(th) b_1,  sum_{m>=1} c_m sin(m th) = sin(th) b_1.
    const cd* pq = F.lpq + F.eoff[b];
    const double c = e1.x, c2 = 2.0 * c;
    const double inv = 2.0 / x;
    const int N = miller_start(pb, x);
    double fn1 = 0.0, fn = 0x1p-600, sum = 0.0, dn = (double)N;
    // f_{n-1} = (2n/x) f_n - f_{n+1}; the sum of the even orders normalises
    // (J_0 + 2 sum J_{2k} = 1); a power of two rescales everything kept when
    // f grows past 2^332 (an integer test on the exponent field)
    auto step = [&]() {
      const double fm = fma(dn * inv, fn, -fn1);
      fn1 = fn;
      fn = fm;
      dn -= 1.0;
    };
    int nn = N;
    for (; nn >= pb + 2; --nn) {  // orders above pb: the recurrence alone
      if ((nn & 1) == 0) sum += fn;
      step();
      if ((__double2hiint(fn) & 0x7FFFFFFF) >= (1355 << 20)) {
        fn *= 0x1p-332; fn1 *= 0x1p-332; sum *= 0x1p-332;
      }
    }
    cd u1 = mk(0.0, 0.0), u2 = u1, v1 = u1, v2 = u1;
    for (; nn >= 1; --nn) {
      if ((nn & 1) == 0) sum += fn;
      step();
      const int mm = nn - 1;  // fn = f_mm
      const cd P = pq[mm];
      const cd u0 = mk(fma(fn, P.x, fma(c2, u1.x, -u2.x)), fma(fn, P.y, fma(c2, u1.y, -u2.y)));
      u2 = u1;
      u1 = u0;
      if (mm >= 1) {
        const cd Qm = pq[pb + mm];
        const cd v0 = mk(fma(fn, Qm.x, fma(c2, v1.x, -v2.x)), fma(fn, Qm.y, fma(c2, v1.y, -v2.y)));
        v2 = v1;
        v1 = v0;
      }
      if ((__double2hiint(fn) & 0x7FFFFFFF) >= (1355 << 20)) {
        const double sc = 0x1p-332;
        fn *= sc; fn1 *= sc; sum *= sc;
        u1 = cscale(u1, sc); u2 = cscale(u2, sc); v1 = cscale(v1, sc); v2 = cscale(v2, sc);
      }
    }
    acc = mk(fma(-c, u2.x, u1.x) + e1.y * v1.x, fma(-c, u2.y, u1.y) + e1.y * v1.y);
    norm = fn + 2.0 * sum;
  }
  cd* dst = out + F.tid[i];
  *dst = cadd(*dst, cscale(acc, 1.0 / norm));
}

// M2P: one thread per (direct target, W-list box of its leaf) pair, in
// target order; writes the pair's value to partial[pair]. m2p_sum_kernel adds
// each target's pairs in order.
__global__ void __launch_bounds__(kThreads) m2p_pair_kernel(Fmm F, const int* __restrict__ pt,
                                                            const int* __restrict__ pbx, int n,
                                                            cd* __restrict__ partial) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = pt[t], c = pbx[t];
  const int lc = F.level[c];
  const int pb = F.lpb[lc];
  const cd* a = F.mpole + F.eoff[c];
  const double s = F.scale[lc];
  const double2 mc = F.centre[c];
  const double dx = F.txy[i].x - mc.x, dy = F.txy[i].y - mc.y;
  // one reciprocal square root gives r, 1/r and 1/x: no division
  const double d2 = dx * dx + dy * dy;
  const double ir = rsqrt(d2), x = F.k * (d2 * ir), ix = ir * F.ik;
  const cd e1 = mk(dx * ir, dy * ir);
  cd h0, h1;
  hankel01(x, ix, h0, h1);
  // Wh_m = s^m H_m: Wh_{m+1} = m c1 Wh_m - s^2 Wh_{m-1}, c1 = 2 s / x
  const double c1 = 2.0 * s * ix, s2 = s * s;
  cd hm1 = h0, hm = cscale(h1, s), ee = mk(1.0, 0.0);
  cd sum = cmul(a[pb], h0);
  double dm = 0.0;
  for (int m = 1; m <= pb; ++m) {
    ee = cmul(ee, e1);
    // Wh_m e^{i m th} and Wh_m e^{-i m th} from the same four products
    const double rr_ = hm.x * ee.x, ii_ = hm.y * ee.y, ri_ = hm.x * ee.y, ir_ = hm.y * ee.x;
    cfma(sum, a[pb + m], mk(rr_ - ii_, ri_ + ir_));
    const cd v = mk(rr_ + ii_, ir_ - ri_);
    cfma(sum, a[pb - m], (m & 1) ? mk(-v.x, -v.y) : v);
    dm += 1.0;
    const double cm = dm * c1;
    const cd hn = mk(fma(cm, hm.x, -s2 * hm1.x), fma(cm, hm.y, -s2 * hm1.y));
    hm1 = hm;
    hm = hn;
  }
  partial[t] = sum;
}

// out[target] += sum of its M2P pairs, in pair order (targets wtgt[0..n)).
__global__ void m2p_sum_kernel(int n, const int* __restrict__ wtgt, const int* __restrict__ off,
                               const cd* __restrict__ partial, const int* __restrict__ tid,
                               cd* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  cd sum = mk(0.0, 0.0);
  for (int e = off[t]; e < off[t + 1]; ++e) sum = cadd(sum, partial[e]);
  cd* dst = out + tid[wtgt[t]];
  *dst = cadd(*dst, sum);
}

// P2P over the U list: one warp per direct target whose leaf's U list holds
// sources; lanes deal the sources round-robin, a shuffle tree adds them. WIDE:
// the mixed path's Hankel tables (relative error below 1e-13 instead of 1e-15;
// the sum stays FP64).
template <bool HS, bool HD, bool WIDE>
__global__ void __launch_bounds__(kThreads) p2p_warp_kernel(Fmm F, const int* __restrict__ utgt,
                                                            const int* __restrict__ tleaf, int n,
                                                            cd* __restrict__ out) {
  const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const int i = utgt[t];
  const int b = tleaf[i];
  const double k = F.k, ik = 1.0 / k;
  const double tx = F.txy[i].x, ty = F.txy[i].y;
  cd acc = mk(0.0, 0.0);
  const SourceCursor sc{F.uidx, F.rsrc, F.uoff[b], F.uoff[b + 1] - F.uoff[b], 0, 0, nullptr};
  deal_sources(sc, lane, [&](int j) {
    const double dx = tx - F.sxy[j].x, dy = ty - F.sxy[j].y;
    const double r2 = dx * dx + dy * dy;
    if (r2 == 0.0) return;
    const double ir = rsqrt(r2), x = k * r2 * ir;
    cd h0, h1;
    hankel01_any<WIDE, HS, HD>(x, ik * ir, h0, h1);
    if (HS) cfma(acc, F.qs[j], h0);
    if (HD) {
      const double2 nv = F.snrm[j];
      cfma(acc, F.ds[j], cscale(h1, k * (nv.x * dx + nv.y * dy) * ir));
    }
  });
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if (lane == 0) {
    cd* dst = out + F.tid[i];
    *dst = cadd(*dst, acc);
  }
}

// ---------------------------------------------------------------- centres (Stages 3, 5, 8 "New")
// L2QBXL: alpha_s += sum_n gamma_n (-1)^{s-n} V_{s-n}(z - m_b), |s| <= p, from
// the true local coefficients gamma of the centre's leaf (leaf locals are
// unscaled in place once the downward pass is complete). A warp takes G
// centres. First each of G lanes fills its centre's row V_m = J_m(k r) e^{i m th},
// 0 <= m <= M = pb + p, in shared memory (one backward recurrence per centre);
// then the lanes take the warp's (centre, output order s) pairs and form
// alpha_s = sum_n gamma_n t_{s-n} over ascending n, with t_m = (-1)^m V_m for
// m >= 0 and t_m = (-1)^m V_m = conj(V_{-m}) for m < 0 (signs set on the bits,
// off the FP64 pipe). The result does not depend on G or on the launch.
__global__ void __launch_bounds__(32) l2qbxl_kernel(Fmm F, const int* __restrict__ cleaf,
                                                    const int* __restrict__ clist, int n_ctr,
                                                    int G, int TW, cd* __restrict__ alpha) {
  extern __shared__ cd trow[];  // [G][TW], TW > max M
  const int lane = threadIdx.x;
  const int c0 = blockIdx.x * G;
  const int p = F.p, P = 2 * p + 1;
  if (lane < G && c0 + lane < n_ctr) {
    const int i = clist[c0 + lane];
    const int b = cleaf[i];
    const int M = F.lpb[F.level[b]] + p;
    const double2 mb = F.centre[b];
    const double dx = F.cxy[i].x - mb.x, dy = F.cxy[i].y - mb.y;
    const double rr = sqrt(dx * dx + dy * dy);
    cd* row = trow + (size_t)lane * TW;
    // J_0..J_M (unnormalised) into the real parts of row[0..M]
    const double in = 1.0 / miller_row(F.k * rr, M, (double*)row, 2);
    const cd e1 = rr > 0.0 ? mk(dx / rr, dy / rr) : mk(1.0, 0.0);
    cd e = mk(1.0, 0.0);
    for (int m = 0; m <= M; ++m) {
      row[m] = cscale(e, row[m].x * in);
      e = cmul(e, e1);
    }
  }
  __syncwarp();
  constexpr unsigned long long kSign = 0x8000000000000000ull;
  const int nG = min(G, n_ctr - c0);
  for (int o = lane; o < nG * P; o += 32) {
    const int u = o / P, so = o % P - p;
    const int i = clist[c0 + u];
    const int b = cleaf[i];
    const int pb = F.lpb[F.level[b]];
    const cd* row = trow + (size_t)u * TW;
    const cd* g = F.local + F.eoff[b] + pb;
    cd a = mk(0.0, 0.0);
    for (int n = -pb; n <= pb; ++n) {
      const int m = so - n;
      const cd v = row[abs(m)];
      const unsigned long long fx = (m >= 0 && (m & 1)) ? kSign : 0ull;
      const unsigned long long fy = (m < 0) ? kSign : fx;
      const cd t = mk(__longlong_as_double(__double_as_longlong(v.x) ^ fx),
                      __longlong_as_double(__double_as_longlong(v.y) ^ fy));
      cfma(a, g[n], t);
    }
    cd* dst = alpha + (size_t)F.cid[i] * P + p + so;
    *dst = cadd(*dst, a);
  }
}


// Leaf local coefficients lh_n = gamma_n s^|n| -> gamma_n, in place, once the
// downward pass (M2L, P2L, L2L) is complete; L2P and L2QBXL read gamma. The
// same pass writes the leaf's L2P coefficients in cosine/sine form: with
// s_m = (-1)^m, the term of order m of the local expansion at (r, th) is
//   J_m(k r) [gamma_m e^{-i m th} + s_m gamma_{-m} e^{i m th}]
//     = J_m(k r) [P_m cos(m th) + Q_m sin(m th)],
//   P_m = gamma_m + s_m gamma_{-m},  Q_m = i (s_m gamma_{-m} - gamma_m),  P_0 = gamma_0,
// stored as lpq[eoff + m] = P_m (m = 0..pb), lpq[eoff + pb + m] = Q_m (m = 1..pb).
__global__ void __launch_bounds__(kThreads) unscale_leaf_locals_kernel(Fmm F,
                                                                       const int* __restrict__ leaves) {
  const int b = leaves[blockIdx.x];
  const int l = F.level[b];
  const int pb = F.lpb[l];
  const double* ipp = ipw_row(F, l);
  cd* lp = F.local + F.eoff[b];
  cd* pq = F.lpq + F.eoff[b];
  for (int m = threadIdx.x; m <= pb; m += kThreads) {
    const cd gp = cscale(lp[pb + m], ipp[m]);
    lp[pb + m] = gp;
    if (m == 0) {
      pq[0] = gp;
      continue;
    }
    const cd gn = cscale(lp[pb - m], ipp[m]);
    lp[pb - m] = gn;
    const cd sg = (m & 1) ? mk(-gn.x, -gn.y) : gn;
    pq[m] = cadd(gp, sg);
    const cd d = csub(sg, gp);
    pq[pb + m] = mk(-d.y, d.x);
  }
}


// One source's contribution to the QBX coefficients of a centre (P2QBXL):
// alpha_l += q W_l + d (k/2) (nu W_{l-1} - conj(nu) W_{l+1}),  W_l = H_l(k r) e^{i l th},
// (r, th) the polar coordinates of source - centre; upward Hankel recurrence.
template <int PM, bool HS, bool HD>
__device__ __forceinline__ void p2qbxl_pair(cd (&acc)[2 * PM + 1], double dx, double dy, cd q,
                                            cd A, cd B, double k, double ik, int p) {
  // A = d (k/2) nu, B = d (k/2) conj(nu): alpha_l += q W_l + A W_{l-1} - B W_{l+1}.
  // W_m and W_{-m} are kept in sliding windows so each is formed once. One
  // reciprocal square root gives r, 1/r and 1/x (ik = 1/k): no division.
  const double r2 = dx * dx + dy * dy;
  if (r2 == 0.0) return;
  const double ir = rsqrt(r2), rr = r2 * ir, x = k * rr, ix = ik * ir, ix2 = 2.0 * ix;
  const cd e1 = mk(dx * ir, dy * ir);
  cd h0, h1;
  hankel01(x, ix, h0, h1);
  const cd w1 = cmul(h1, e1);
  const cd wm1 = cscale(cmul(h1, cconj(e1)), -1.0);
  if (HS) cfma(acc[PM], q, h0);
  if (HD) {
    cfma(acc[PM], A, wm1);
    cfma(acc[PM], mk(-B.x, -B.y), w1);
  }
  cd hprev = h0, hcur = h1, ecur = e1;
  cd wp_prev = h0, wp_cur = w1;   // W_{m-1}, W_m
  cd wn_prev = h0, wn_cur = wm1;  // W_{-(m-1)}, W_{-m}
  const cd mB = mk(-B.x, -B.y);
  // H_{m+1} = (2m/x) H_m - H_{m-1} (two FMAs per component; 2m/x = dm ix2 with
  // dm counted exactly); W_{m+1} = H_{m+1} e^{i(m+1)th} and
  // W_{-(m+1)} = (-1)^{m+1} H_{m+1} e^{-i(m+1)th} from the same four products
  double dm = 0.0;
  auto step = [&](int m, cd& hnext, cd& enext, cd& wp, cd& wn) {
    dm += 1.0;
    const double cm = dm * ix2;
    hnext = mk(fma(cm, hcur.x, -hprev.x), fma(cm, hcur.y, -hprev.y));
    enext = cmul(ecur, e1);
    const double rr_ = hnext.x * enext.x, ii_ = hnext.y * enext.y;
    const double ri_ = hnext.x * enext.y, ir_ = hnext.y * enext.x;
    wp = mk(rr_ - ii_, ri_ + ir_);
    wn = (m & 1) ? mk(rr_ + ii_, ir_ - ri_) : mk(-(rr_ + ii_), ri_ - ir_);
  };
#pragma unroll
  for (int m = 1; m <= PM; ++m) {
    if (m > p) break;
    if (HS) {
      cfma(acc[PM + m], q, wp_cur);
      cfma(acc[PM - m], q, wn_cur);
    }
    if (HD) {
      cd hnext, enext, wp_next, wn_next;
      step(m, hnext, enext, wp_next, wn_next);
      cfma(acc[PM + m], A, wp_prev);
      cfma(acc[PM + m], mB, wp_next);
      cfma(acc[PM - m], A, wn_next);
      cfma(acc[PM - m], mB, wn_prev);
      hprev = hcur;
      hcur = hnext;
      ecur = enext;
      wp_prev = wp_cur;
      wp_cur = wp_next;
      wn_prev = wn_cur;
      wn_cur = wn_next;
    } else if (m < p) {
      cd hnext, enext;
      step(m, hnext, enext, wp_cur, wn_cur);
      hprev = hcur;
      hcur = hnext;
      ecur = enext;
    }
  }
}

// M2QBXL: alpha_l += (-1)^l sum_n mh_n Wh_{n+l} s^{|n| - |n+l|},  Wh_m = s^|m| W_m(z - m_c),
// for the (centre, W-list box) pairs whose box is far enough from the centre's
// disk for the multipole series to converge on it ((R_c + r_z) <= kW |z - m_c|;
// the others are summed source by source with the U list in P2QBXL). Each pair
// is split over ceil((2p+1) / kM2qbxlOrders) threads, each with kM2qbxlOrders
// consecutive output orders; each writes its orders of partial[pair][2p+1],
// and m2qbxl_sum_kernel adds each centre's pairs in order. Threads walk
// m = |n + l| upwards with the Hankel recurrence; once m > p every term of
// output l has the same power factor (s^-l for n + l = m, s^l for n + l = -m),
// so those terms go to two plain sums scaled once at the end. One warp per
// block spreads the pairs over all SMs (the FP64 pipe is per SM).
constexpr int kM2qbxlOrders = 4;
constexpr int kM2qbxlBlock = 32;
// shared memory of the L2QBXL rows of one warp. FP64: 16 centres per warp at
// order 16 on 41-order leaves (the dot products keep the FP64 pipe busy);
// mixed: small enough for a dozen or more warps per SM, which hide the latency
// of the split coefficients' loads (8 centres per warp: L2QBXL 1.29 -> 1.02
// ms on ellipses-200; 4 was slower again)
constexpr size_t kL2qbxlSmem = 24 * 1024, kL2qbxlMixedSmem = 12 * 1024;
// shared memory of the split rows of one mixed-precision M2QBXL warp, and the
// pairs per warp: at most 8, so that a dozen or more warps share an SM (8 on
// ellipses-200: M2QBXL 1.08 -> 0.69 ms against 32)
constexpr size_t kM2qbxlMixedSmem = 48 * 1024;
constexpr int kM2qbxlMixedPairs = 8;
template <int PM, bool HS, bool HD>
__global__ void __launch_bounds__(kThreads) m2qbxl_pair_kernel(Fmm F, const int* __restrict__ pair_ctr,
                                                               const int* __restrict__ pair_box,
                                                               int n_pairs, cd* __restrict__ partial) {
  constexpr int LC = kM2qbxlOrders;
  const int p = F.p, P = 2 * p + 1;
  const int nparts = (P + LC - 1) / LC;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = g / nparts, part = g % nparts;
  if (t >= n_pairs) return;
  const int i = pair_ctr[t], c = pair_box[t];
  const int lo0 = -p + part * LC;  // first output order of this thread (<= p)
  const double k = F.k;
  const int lc = F.level[c];
  const double s = F.scale[lc];
  const int pb = F.lpb[lc], M = pb + p;
  const cd* a = F.mpole + F.eoff[c];
  const double* pwl = pw_row(F, lc);
  const double* ipl = ipw_row(F, lc);
  const double2 z = F.cxy[i];
  const double2 mc = F.centre[c];
  const double dx = z.x - mc.x, dy = z.y - mc.y;
  const double rr = sqrt(dx * dx + dy * dy);
  const double x = k * rr, ix = 1.0 / x;
  const cd e1 = mk(dx / rr, dy / rr);
  cd h0, h1;
  hankel01(x, ix, h0, h1);
  const double c1 = 2.0 * s * ix, s2 = s * s;  // Wh_{m+1} = m c1 Wh_m - s2 Wh_{m-1}
  cd acc[LC], accp[LC], accq[LC];
#pragma unroll
  for (int j = 0; j < LC; ++j) acc[j] = accp[j] = accq[j] = mk(0.0, 0.0);
  cd hm1 = h0, hm = h0, ee = mk(1.0, 0.0);
  for (int mm = 0; mm <= M; ++mm) {
    if (mm == 1) { hm1 = h0; hm = cscale(h1, s); }
    if (mm >= 1) ee = cmul(ee, e1);
    // Wh_m = hm ee and Wh_{-m} = (-1)^m hm conj(ee) from the same four products
    const double ac = hm.x * ee.x, bd = hm.y * ee.y, ad = hm.x * ee.y, bc = hm.y * ee.x;
    const cd wp = mk(ac - bd, ad + bc);
    const double sm = (mm & 1) ? -1.0 : 1.0;
    const cd wq = mk(sm * (ac + bd), sm * (bc - ad));
    if (mm <= p) {  // |n| - |n + l| depends on n: per-term factors
#pragma unroll
      for (int j = 0; j < LC; ++j) {
        const int lo = lo0 + j;
        const int n1 = mm - lo;  // n + l = m
        if (lo <= p && n1 >= -pb && n1 <= pb) {
          const int ex = abs(n1) - mm;
          cfma(acc[j], cscale(a[n1 + pb], ex >= 0 ? pwl[ex] : ipl[-ex]), wp);
        }
        const int n2 = -mm - lo;  // n + l = -m
        if (mm > 0 && lo <= p && n2 >= -pb && n2 <= pb) {
          const int ex = abs(n2) - mm;
          cfma(acc[j], cscale(a[n2 + pb], ex >= 0 ? pwl[ex] : ipl[-ex]), wq);
        }
      }
    } else {  // n + l = m > 0 has n > 0, n + l = -m has n < 0: factors s^-l, s^l
#pragma unroll
      for (int j = 0; j < LC; ++j) {
        const int lo = lo0 + j;
        const int n1 = mm - lo, n2 = -mm - lo;
        const cd av = (n1 >= -pb && n1 <= pb) ? a[n1 + pb] : mk(0.0, 0.0);
        const cd aq = (n2 >= -pb && n2 <= pb) ? a[n2 + pb] : mk(0.0, 0.0);
        cfma(accp[j], av, wp);
        cfma(accq[j], aq, wq);
      }
    }
    if (mm >= 1) {
      const cd hn = csub(cscale(hm, mm * c1), cscale(hm1, s2));
      hm1 = hm;
      hm = hn;
    }
  }
  cd* dst = partial + (size_t)t * P;
#pragma unroll
  for (int j = 0; j < LC; ++j) {
    const int lo = lo0 + j;
    if (lo > p) break;
    const double fp = lo <= 0 ? pwl[-lo] : ipl[lo];  // s^-l
    const double fq = lo >= 0 ? pwl[lo] : ipl[-lo];  // s^l
    cd v = cadd(acc[j], cadd(cscale(accp[j], fp), cscale(accq[j], fq)));
    if (lo & 1) v = mk(-v.x, -v.y);
    dst[lo + p] = v;
  }
}

// alpha[centre] += sum of its pairs' partial coefficients, in pair order
// (centres clist[0..n), pairs of position t at cpo[t]..cpo[t+1]).
__global__ void m2qbxl_sum_kernel(int n, int P, const int* __restrict__ cpo,
                                  const cd* __restrict__ partial, const int* __restrict__ cid,
                                  const int* __restrict__ clist, cd* __restrict__ alpha) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= (int64_t)n * P) return;
  const int t = (int)(g / P), l = (int)(g % P);
  const int t0 = cpo[t], t1 = cpo[t + 1];
  if (t1 == t0) return;
  cd sum = mk(0.0, 0.0);
  for (int e = t0; e < t1; ++e) sum = cadd(sum, partial[(size_t)e * P + l]);
  cd* dst = alpha + (size_t)cid[clist[t]] * P + l;
  *dst = cadd(*dst, sum);
}

// ---------------------------------------------------------------- mixed precision P2QBXL
// H_0, H_1 and the Hankel recurrence stay FP64; the terms sigma^|l| W_l
// (sigma = 2^s near rho = k r_c, which keeps them of moderate size) are
// rounded to FP32, multiplied by the FP32 strengths and added with Kahan
// compensation into ah_l = alpha_l sigma^|l|; alpha_l = ah_l sigma^-|l| is
// formed in FP64 at the end.
__device__ __forceinline__ void kahan2(float2& s, float2& c, float2 v) {
  float y = v.x - c.x, t = s.x + y;
  c.x = (t - s.x) - y;
  s.x = t;
  y = v.y - c.y;
  t = s.y + y;
  c.y = (t - s.y) - y;
  s.y = t;
}
__device__ __forceinline__ float2 fmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 fsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2(cd a) { return make_float2(f32_from_f64(a.x), f32_from_f64(a.y)); }

template <int PM, bool HS, bool HD>
__device__ __forceinline__ void p2qbxl_pair_mixed(float2 (&S)[2 * PM + 1], float2 (&C)[2 * PM + 1],
                                                  double dx, double dy, float2 q, float2 A,
                                                  float2 B, double k, double ik, int s, float fr,
                                                  float fi, int p) {
  // one reciprocal square root gives r, 1/r and 1/x (ik = 1/k): no division
  const double d2 = dx * dx + dy * dy;
  if ((__double2hiint(d2) | __double2loint(d2)) == 0) return;  // d2 == 0 (integer test)
  const double irr = rsqrt(d2), rr = d2 * irr, x = k * rr, ix = ik * irr;
  cd h0, h1;
  hankel01_wide(x, ix, h0, h1);
  // The FP64 recurrence runs on H_m itself, H_{m+1} = (2m/x) H_m - H_{m-1}
  // (two FMAs per order); the terms are sigma^|l| W_l with sigma = 2^s close
  // to rho = k r_c (fr = sigma, fi = 1/sigma), so H_m sigma^m is formed by an
  // exponent offset while H_m is rounded to FP32, which keeps the terms of
  // moderate size.
  const double c2 = 2.0 * ix;
  cd hprev = h0, hcur = h1;
  // angular factors e^{i m th} in FP32 (unit modulus; rounding grows like m eps_32),
  // from the FP32 roundings of dx, dy and 1/r
  const float irf = f32_from_f64(irr);
  const float2 e1f = make_float2(f32_from_f64(dx) * irf, f32_from_f64(dy) * irf);
  float2 ecur = e1f;
  // W^s_m = sigma^|m| W_m for m = -1, 0, 1, the products in FP32 as for every
  // other order
  const float2 h1s = make_float2(f32_from_f64_sh(h1.x, s), f32_from_f64_sh(h1.y, s));
  const float2 t1 = fmul(h1s, make_float2(e1f.x, -e1f.y));
  float2 wm1 = make_float2(-t1.x, -t1.y);  // W^s_{-1}
  float2 w0 = f2(h0);
  float2 w1 = fmul(h1s, e1f);
  // l = 0: q W_0 + A W_{-1} - B W_1, with W_{-1} = W^s_{-1} / sigma, W_1 = W^s_1 / sigma
  {
    float2 v = make_float2(0.f, 0.f);
    if (HS) v = fmul(q, w0);
    if (HD) {
      const float2 t = fsub(fmul(A, wm1), fmul(B, w1));
      v = make_float2(v.x + fi * t.x, v.y + fi * t.y);
    }
    kahan2(S[PM], C[PM], v);
  }
  float2 wp_prev = w0, wp_cur = w1;   // W^s_{m-1}, W^s_m (positive side)
  float2 wn_prev = w0, wn_cur = wm1;  // W^s_{-(m-1)}, W^s_{-m}
  double cm = 0.0;                    // 2m/x, kept by addition
#pragma unroll
  for (int m = 1; m <= PM; ++m) {
    if (m > p) break;
    cm += c2;
    const cd hnext = mk(fma(cm, hcur.x, -hprev.x), fma(cm, hcur.y, -hprev.y));
    const float2 enext = fmul(ecur, e1f);
    const int sh = (m + 1) * s;
    const float2 hn32 = make_float2(f32_from_f64_sh(hnext.x, sh), f32_from_f64_sh(hnext.y, sh));
    const float2 wp_next = fmul(hn32, enext);                                // W^s_{m+1}
    const float2 wq = fmul(hn32, make_float2(enext.x, -enext.y));
    // W^s_{-(m+1)} = (-1)^{m+1} conj-angle term
    const float2 wn_next = (m & 1) ? wq : make_float2(-wq.x, -wq.y);
    // sigma^m W_{m-1} = sigma W^s_{m-1},  sigma^m W_{m+1} = W^s_{m+1} / sigma (same for -m)
    float2 vp = make_float2(0.f, 0.f), vn = make_float2(0.f, 0.f);
    if (HS) {
      vp = fmul(q, wp_cur);
      vn = fmul(q, wn_cur);
    }
    if (HD) {
      const float2 ap = fmul(A, wp_prev), bp = fmul(B, wp_next);
      vp.x += fr * ap.x - fi * bp.x;
      vp.y += fr * ap.y - fi * bp.y;
      const float2 an = fmul(A, wn_next), bn = fmul(B, wn_prev);
      vn.x += fi * an.x - fr * bn.x;
      vn.y += fi * an.y - fr * bn.y;
    }
    kahan2(S[PM + m], C[PM + m], vp);
    kahan2(S[PM - m], C[PM - m], vn);
    hprev = hcur;
    hcur = hnext;
    ecur = enext;
    wp_prev = wp_cur;
    wp_cur = wp_next;
    wn_prev = wn_cur;
    wn_cur = wn_next;
  }
}

// ---------------------------------------------------------------- M2QBXL in mixed precision
// The same translation as m2qbxl_pair_kernel,
//   alpha_l += (-1)^l sum_n mh_n Wh_{n+l} s^{|n| - |n+l|},
// with the Hankel recurrence and the angular factors in FP64 and the Q x P
// products in FP32. The factors span far more than FP32's range (Wh_m grows
// and mh_n falls by many decades with m, n), so each is held in split form,
// FP32 mantissa times 2^e (split_pair): the product of three split factors is
// an FP32 mantissa product and an integer exponent sum, exact apart from the
// FP32 rounding of the mantissas. Every output sums its terms relative to its
// largest one (2^Emax), FP32 with Kahan compensation, and is formed in FP64.
//
// A warp takes PW pairs: lane j runs pair j's recurrence and writes the split
// rows Wp_m = Wh_m e^{i m th}, Wq_m = (-1)^m Wh_m e^{-i m th}, m <= pb + p,
// to shared memory; then the lanes take the warp's (pair, output order)
// items. Inputs: the split multipoles (split_coef_kernel) and the split powers
// s^j, |j| <= p, per level (sf).

// coefficients (multipoles or locals) of every box in split form, same layout
__global__ void split_coef_kernel(const cd* __restrict__ mpole, long long n, float2* __restrict__ mm,
                                int* __restrict__ me) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float2 m;
  int e;
  split_one(mpole[i], m, e);
  mm[i] = m;
  me[i] = e;
}

// s_l^j, j = -p..p, of every level in split form: [n_levels][2p+1]
__global__ void sf_split_kernel(Fmm F, float* __restrict__ sfm, int* __restrict__ sfe) {
  const int l = blockIdx.x, P = 2 * F.p + 1;
  const double* pwl = pw_row(F, l);
  const double* ipl = ipw_row(F, l);
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    const int jj = j - F.p;
    const double v = jj >= 0 ? pwl[jj] : ipl[-jj];
    float2 m;
    int e;
    split_one(mk(v, 0.0), m, e);
    sfm[(size_t)l * P + j] = m.x;
    sfe[(size_t)l * P + j] = e;
  }
}

__global__ void __launch_bounds__(32) m2qbxl_mixed_kernel(
    Fmm F, const int* __restrict__ pair_ctr, const int* __restrict__ pair_box, int n_pairs,
    int PW, int TW, const float2* __restrict__ mm, const int* __restrict__ me,
    const float* __restrict__ sfm, const int* __restrict__ sfe, cd* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char m2q_smem[];
  float2* wp = reinterpret_cast<float2*>(m2q_smem);  // [PW][TW]
  float2* wq = wp + (size_t)PW * TW;                 // [PW][TW]
  int* we = reinterpret_cast<int*>(wq + (size_t)PW * TW);  // [PW][TW]
  const int lane = threadIdx.x;
  const int t0 = blockIdx.x * PW;
  const int p = F.p, P = 2 * p + 1;
  const int npw = min(PW, n_pairs - t0);
  if (lane < npw) {
    const int t = t0 + lane;
    const int i = pair_ctr[t], c = pair_box[t];
    const int lc = F.level[c];
    const double s = F.scale[lc];
    const int M = F.lpb[lc] + p;
    const double2 z = F.cxy[i];
    const double2 mc = F.centre[c];
    const double dx = z.x - mc.x, dy = z.y - mc.y;
    const double d2 = dx * dx + dy * dy;
    const double irr = rsqrt(d2), rr = d2 * irr, x = F.k * rr, ix = irr * F.ik;
    const cd e1 = mk(dx * irr, dy * irr);
    cd h0, h1;
    hankel01_wide(x, ix, h0, h1);
    const double c1 = 2.0 * s * ix, s2 = s * s;
    cd hm1 = h0, hm = cscale(h1, s), ee = mk(1.0, 0.0);
    float2* rp = wp + (size_t)lane * TW;
    float2* rq = wq + (size_t)lane * TW;
    int* re = we + (size_t)lane * TW;
    split_pair(h0, h0, rp[0], rq[0], re[0]);
    for (int m = 1; m <= M; ++m) {
      ee = cmul(ee, e1);
      const double ac = hm.x * ee.x, bd = hm.y * ee.y, ad = hm.x * ee.y, bc = hm.y * ee.x;
      const double sm = (m & 1) ? -1.0 : 1.0;
      split_pair(mk(ac - bd, ad + bc), mk(sm * (ac + bd), sm * (bc - ad)), rp[m], rq[m], re[m]);
      const cd hn = mk(fma((double)m * c1, hm.x, -s2 * hm1.x), fma((double)m * c1, hm.y, -s2 * hm1.y));
      hm1 = hm;
      hm = hn;
    }
  }
  __syncwarp();
  for (int o = lane; o < npw * P; o += 32) {
    const int u = o / P, lo = o % P - p;
    const int t = t0 + u;
    const int c = pair_box[t];
    const int lc = F.level[c];
    const int pb = F.lpb[lc];
    const long long off = F.eoff[c] + pb;
    const float2* rp = wp + (size_t)u * TW;
    const float2* rq = wq + (size_t)u * TW;
    const int* re = we + (size_t)u * TW;
    const float* fm = sfm + (size_t)lc * P + p;
    const int* fe = sfe + (size_t)lc * P + p;
    // one pass: the sums are kept relative to the largest exponent seen so
    // far and rescaled (by a power of two) when a larger one appears
    int emax = 2 * kZeroExp;
    float2 S = make_float2(0.f, 0.f), C = make_float2(0.f, 0.f);
    for (int n = -pb; n <= pb; ++n) {
      const int m = n + lo, am = abs(m);
      const int j = abs(n) - am;
      const int e = me[off + n] + re[am] + fe[j];
      if (e > emax) {
        const float r = pow2f(emax - e);
        S = make_float2(S.x * r, S.y * r);
        C = make_float2(C.x * r, C.y * r);
        emax = e;
      }
      const int d = e - emax;
      if (d < -126) continue;
      const float f = fm[j] * pow2f(d);
      const float2 w = m >= 0 ? rp[am] : rq[am];
      const float2 v = fmul(mm[off + n], w);
      kahan2(S, C, make_float2(v.x * f, v.y * f));
    }
    const double sc = (lo & 1) ? -pow2d(emax) : pow2d(emax);
    partial[(size_t)t * P + lo + p] =
        mk(((double)S.x - (double)C.x) * sc, ((double)S.y - (double)C.y) * sc);
  }
}

// ---------------------------------------------------------------- L2QBXL in mixed precision
// The translation of l2qbxl_kernel, alpha_s += sum_n gamma_n t_{s-n}, with the
// Miller recurrence (J_m) and the angular factors in FP64 and the products in
// FP32 on split factors (as in m2qbxl_mixed_kernel): the leaf's local
// coefficients gamma_n (large for large |n|) and the row V_m = J_m e^{i m th}
// (small for large m) as FP32 mantissas with integer exponents; each output
// sums relative to its largest term with Kahan compensation. A warp takes G
// centres; lane j fills centre j's row in FP64 and converts it in place to
// split form (FP32 mantissa pair and exponent in the 16 bytes of each entry).
__global__ void __launch_bounds__(32) l2qbxl_mixed_kernel(Fmm F, const int* __restrict__ cleaf,
                                                          const int* __restrict__ clist, int n_ctr,
                                                          int G, int TW,
                                                          const float2* __restrict__ gm,
                                                          const int* __restrict__ ge,
                                                          cd* __restrict__ alpha) {
  extern __shared__ cd trow[];  // [G][TW]
  const int lane = threadIdx.x;
  const int c0 = blockIdx.x * G;
  const int p = F.p, P = 2 * p + 1;
  if (lane < G && c0 + lane < n_ctr) {
    const int i = clist[c0 + lane];
    const int b = cleaf[i];
    const int M = F.lpb[F.level[b]] + p;
    const double2 mb = F.centre[b];
    const double dx = F.cxy[i].x - mb.x, dy = F.cxy[i].y - mb.y;
    const double rr = sqrt(dx * dx + dy * dy);
    cd* row = trow + (size_t)lane * TW;
    const double in = 1.0 / miller_row(F.k * rr, M, (double*)row, 2);
    const cd e1 = rr > 0.0 ? mk(dx / rr, dy / rr) : mk(1.0, 0.0);
    cd e = mk(1.0, 0.0);
    for (int m = 0; m <= M; ++m) {
      float2 mv;
      int ev;
      split_one(cscale(e, row[m].x * in), mv, ev);
      float4* slot = reinterpret_cast<float4*>(row + m);
      *slot = make_float4(mv.x, mv.y, __int_as_float(ev), 0.f);
      e = cmul(e, e1);
    }
  }
  __syncwarp();
  const int nG = min(G, n_ctr - c0);
  for (int o = lane; o < nG * P; o += 32) {
    const int u = o / P, so = o % P - p;
    const int i = clist[c0 + u];
    const int b = cleaf[i];
    const int pb = F.lpb[F.level[b]];
    const float4* row = reinterpret_cast<const float4*>(trow + (size_t)u * TW);
    const long long off = F.eoff[b] + pb;
    // one pass: the sums are kept relative to the largest exponent seen so
    // far and rescaled (by a power of two) when a larger one appears
    int emax = 2 * kZeroExp;
    float2 S = make_float2(0.f, 0.f), C = make_float2(0.f, 0.f);
    for (int n = -pb; n <= pb; ++n) {
      const int m = so - n;
      const float4 v = row[abs(m)];
      const int e = ge[off + n] + __float_as_int(v.z);
      if (e > emax) {
        const float r = pow2f(emax - e);
        S = make_float2(S.x * r, S.y * r);
        C = make_float2(C.x * r, C.y * r);
        emax = e;
      }
      const int d = e - emax;
      if (d < -126) continue;
      // t_m = (-1)^m V_m (m >= 0), conj(V_-m) (m < 0): signs on the bits
      const unsigned fx = (m >= 0 && (m & 1)) ? 0x80000000u : 0u;
      const unsigned fy = m < 0 ? 0x80000000u : fx;
      const float2 t = make_float2(__uint_as_float(__float_as_uint(v.x) ^ fx),
                                   __uint_as_float(__float_as_uint(v.y) ^ fy));
      const float f = pow2f(d);
      const float2 w = fmul(gm[off + n], t);
      kahan2(S, C, make_float2(w.x * f, w.y * f));
    }
    const double sc = pow2d(emax);
    cd* dst = alpha + (size_t)F.cid[i] * P + p + so;
    *dst = cadd(*dst, mk(((double)S.x - (double)C.x) * sc, ((double)S.y - (double)C.y) * sc));
  }
}

// ---------------------------------------------------------------- M2P in mixed precision
// The FP32 multipoles that M2P reads. On levels where the unscaled Hankel
// recurrence stays in range (scaled[l] == 0): mu'_n = a_n 2^-t_|n|, a_n = mh_n
// s^|n| the true coefficient and t_m = round(log2 sig_m), so that mu' is of
// order one; otherwise the sigma-normalised mu_n = mh_n conv_|n| (conv = s^j /
// sig_j).
__global__ void __launch_bounds__(kThreads) mpole_f32_list_kernel(
    Fmm F, const int* __restrict__ boxes, const double* __restrict__ conv,
    const int* __restrict__ tpow, const int* __restrict__ scaled, float2* __restrict__ mu) {
  const int b = boxes[blockIdx.x];
  const int l = F.level[b];
  const int pb = F.lpb[l];
  const double* cv = conv + (size_t)l * (F.pbmax + 1);
  const double* pwl = pw_row(F, l);
  const int* tl = tpow + (size_t)l * (F.pbmax + 2);
  const bool sc = scaled[l] != 0;
  const cd* a = F.mpole + F.eoff[b];
  float2* dst = mu + F.eoff[b];
  for (int n = threadIdx.x; n <= 2 * pb; n += kThreads) {
    const int m = abs(n - pb);
    const double f = sc ? cv[m] : pwl[m] * pow2d(-tl[m]);
    dst[n] = make_float2((float)(a[n].x * f), (float)(a[n].y * f));
  }
}

// M2P with the Hankel recurrence in FP64 and the rest in FP32: the multipole
// sum_m a_m H_m(kr) e^{imth}, each term formed as an FP32 product of order-one
// factors:
//  * unscaled levels: H_{m+1} = (2m/x) H_m - H_{m-1} (two FMAs per order), H_m
//    rounded to FP32 with the exponent offset t_m (H_m 2^t_m, t_m = round(log2
//    sig_m)) against mu'_m = a_m 2^-t_m;
//  * levels where H_pb could leave the FP64 range: G_m = sig_m H_m by
//      G_{m+1} = (2m/x)(sig_{m+1}/sig_m) G_m - (sig_{m+1}/sig_{m-1}) G_{m-1}
//    (rec[l][m] = (2m sig_{m+1}/sig_m, sig_{m+1}/sig_{m-1}), rec[l][0].x =
//    sig_1) against mu_m = a_m / sig_m.
// Angular factors, products and the compensated (Kahan) sum are FP32;
// H_{-m} = (-1)^m H_m.
__global__ void __launch_bounds__(kThreads) m2p_pair_mixed_kernel(
    Fmm F, const int* __restrict__ pt, const int* __restrict__ pbx, int n,
    const float2* __restrict__ mu, const double2* __restrict__ rec, const int* __restrict__ tpow,
    const int* __restrict__ scaled, cd* __restrict__ partial) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = pt[t], c = pbx[t];
  const int lc = F.level[c];
  const int pb = F.lpb[lc];
  const float2* a = mu + F.eoff[c] + pb;  // a[m], |m| <= pb
  const double2 mc = F.centre[c];
  const double dx = F.txy[i].x - mc.x, dy = F.txy[i].y - mc.y;
  const double d2 = dx * dx + dy * dy;
  const double irr = rsqrt(d2), rr = d2 * irr, x = F.k * rr, ix = irr * F.ik;
  cd h0, h1;
  hankel01_wide(x, ix, h0, h1);
  const float irf = f32_from_f64(irr);
  const float2 e1 = make_float2(f32_from_f64(dx) * irf, f32_from_f64(dy) * irf);
  float2 ee = e1;
  float2 S = fmul(a[0], f2(h0)), C = make_float2(0.f, 0.f);
  if (!scaled[lc]) {
    const int* tl = tpow + (size_t)lc * (F.pbmax + 2);
    const double c2 = 2.0 * ix;
    double cm = 0.0;  // 2m/x
    cd hprev = h0, hcur = h1;
    for (int m = 1; m <= pb; ++m) {
      const int sh = tl[m];
      const float2 g = make_float2(f32_from_f64_sh(hcur.x, sh), f32_from_f64_sh(hcur.y, sh));
      const float2 wp = fmul(g, ee);                                // H_m 2^t e^{im th}
      float2 wn = fmul(g, make_float2(ee.x, -ee.y));                // H_m 2^t e^{-im th}
      if (m & 1) wn = make_float2(-wn.x, -wn.y);                    // (-1)^m
      const float2 vp = fmul(a[m], wp), vn = fmul(a[-m], wn);
      kahan2(S, C, make_float2(vp.x + vn.x, vp.y + vn.y));
      if (m < pb) {
        cm += c2;
        const cd hn = mk(fma(cm, hcur.x, -hprev.x), fma(cm, hcur.y, -hprev.y));
        hprev = hcur;
        hcur = hn;
        ee = fmul(ee, e1);
      }
    }
  } else {
    const double2* R = rec + (size_t)lc * (F.pbmax + 2);
    cd gprev = h0, gcur = cscale(h1, R[0].x);
    for (int m = 1; m <= pb; ++m) {
      const float2 g = f2(gcur);
      const float2 wp = fmul(g, ee);                                // G_m e^{im th}
      float2 wn = fmul(g, make_float2(ee.x, -ee.y));                // G_m e^{-im th}
      if (m & 1) wn = make_float2(-wn.x, -wn.y);                    // (-1)^m
      const float2 vp = fmul(a[m], wp), vn = fmul(a[-m], wn);
      kahan2(S, C, make_float2(vp.x + vn.x, vp.y + vn.y));
      if (m < pb) {
        const double c1 = R[m].x * ix, c2 = R[m].y;
        const cd gn = mk(fma(c1, gcur.x, -c2 * gprev.x), fma(c1, gcur.y, -c2 * gprev.y));
        gprev = gcur;
        gcur = gn;
        ee = fmul(ee, e1);
      }
    }
  }
  partial[t] = mk((double)S.x - (double)C.x, (double)S.y - (double)C.y);
}

// ---------------------------------------------------------------- P2M in mixed precision
// The item structure of p2m_item_kernel with the sums in FP32: the rows
// R_t = conj(V_t) / sig_|t| (the FP64 Miller recurrence, FP32 from the
// normalisation on; stored in the first half of each 16-byte row slot) and,
// over the item's sources with Kahan compensation,
//   mu_n = sum_j [q_j R_n + A_j R_{n-1} sig_|n-1| / sig_|n| - B_j R_{n+1} sig_|n+1| / sig_|n|],
// A = d (k/2) conj(nu), B = d (k/2) nu; mu_n = a_n / sig_|n|, of order one.
// p2m_sum_mixed_kernel adds a leaf's segments in FP64 and forms mh_n = mu_n /
// conv_|n| (conv = s^j / sig_j).
__device__ __forceinline__ void p2m_fill_row_mixed(const Fmm& F, int i, double2 m, int l, int pb,
                                                   cd* row, cd& sq, cd& sa, cd& sb) {
  const double dx = F.sxy[i].x - m.x, dy = F.sxy[i].y - m.y;
  const double d2 = dx * dx + dy * dy;
  const bool at_centre = (__double2hiint(d2) | __double2loint(d2)) == 0;
  const double ir = at_centre ? 0.0 : rsqrt(d2);
  const double norm = miller_row(F.k * (d2 * ir), pb + 1, (double*)row, 2);
  // R_j = J_j / sig_j e^{-i j th} = row_j / (norm sig_j) e^{-i j th}: row_j / sig_j
  // in FP64 (one product), the factor 2^-e of norm = mn 2^e as an exponent offset
  // in the FP32 rounding, 1 / mn and the angular factor in FP32
  const double* isg = F.isig + (size_t)l * (F.pbmax + 2);
  const int en = (int)((__double2hiint(norm) >> 20) & 0x7FF) - 1023;
  const float imn = 1.0f / f32_from_f64_sh(norm, -en);
  // e^{-i j th}: FP64 anchors every eighth order (e^{-8 i th} by three
  // squarings), FP32 products in between
  const cd em = at_centre ? mk(1.0, 0.0) : mk(dx * ir, -dy * ir);
  cd e8 = cmul(em, em);
  e8 = cmul(e8, e8);
  e8 = cmul(e8, e8);
  const float2 emf = f2(em);
  cd E = mk(1.0, 0.0);
  float2 ef = make_float2(1.f, 0.f);
  for (int j = 0; j <= pb + 1; ++j) {
    if ((j & 7) == 0) {
      ef = f2(E);
      E = cmul(E, e8);
    } else {
      ef = fmul(ef, emf);
    }
    const float v = f32_from_f64_sh(row[j].x * isg[j], -en) * imn;
    const float2 c = make_float2(ef.x * v, ef.y * v);  // R_j
    reinterpret_cast<float2*>(row + j)[0] = c;
    if (j > 0) reinterpret_cast<float2*>(row - j)[0] = (j & 1) ? make_float2(-c.x, c.y)
                                                                : make_float2(c.x, -c.y);
  }
  const float4 ab = F.ab32[i];
  reinterpret_cast<float2*>(&sq)[0] = F.q32[i];
  reinterpret_cast<float2*>(&sa)[0] = make_float2(ab.z, ab.w);  // d (k/2) conj(nu)
  reinterpret_cast<float2*>(&sb)[0] = make_float2(ab.x, ab.y);  // d (k/2) nu
}

__global__ void __launch_bounds__(kThreads) p2m_item_mixed_kernel(
    Fmm F, const int4* __restrict__ items, const int* __restrict__ seg_leaf,
    const int2* __restrict__ seg_row, const long long* __restrict__ seg_poff,
    const int* __restrict__ src, const int* __restrict__ src_leaf, cd* __restrict__ partial,
    unsigned sm_bytes) {
  extern __shared__ cd smem[];
  const int4 it = items[blockIdx.x];
  const int l = F.level[seg_leaf[it.x]];
  const int pb = F.lpb[l], Q = 2 * pb + 1, RW = 2 * pb + 3;
  const int chunk = rows_chunk(pb, sm_bytes);  // >= it.w
  cd* rows = smem;                        // [chunk][RW]
  cd* sq = rows + chunk * RW;             // [chunk]
  cd* sa = sq + chunk;                    // [chunk]
  cd* sb = sa + chunk;                    // [chunk]
  if ((int)threadIdx.x < it.w) {
    const int j = threadIdx.x;
    p2m_fill_row_mixed(F, src[it.z + j], F.centre[src_leaf[it.z + j]], l, pb,
                       rows + j * RW + (pb + 1), sq[j], sa[j], sb[j]);
  }
  __syncthreads();
  const double2* sr = F.sigr + (size_t)l * (F.pbmax + 2);
  for (int idx = threadIdx.x; idx < it.y * Q; idx += kThreads) {
    const int u = idx / Q, n = idx % Q - pb;
    const int2 rg = seg_row[it.x + u];
    float2 Sq = make_float2(0.f, 0.f), Cq = Sq, Sa = Sq, Ca = Sq, Sb = Sq, Cb = Sq;
    for (int j = rg.x; j < rg.x + rg.y; ++j) {
      const float2* r = reinterpret_cast<const float2*>(rows + j * RW + (pb + 1));
      if (F.has_S) kahan2(Sq, Cq, fmul(reinterpret_cast<const float2*>(sq + j)[0], r[2 * n]));
      if (F.has_D) {
        kahan2(Sa, Ca, fmul(reinterpret_cast<const float2*>(sa + j)[0], r[2 * (n - 1)]));
        kahan2(Sb, Cb, fmul(reinterpret_cast<const float2*>(sb + j)[0], r[2 * (n + 1)]));
      }
    }
    // sig_|n-1| / sig_|n| and sig_|n+1| / sig_|n| (1 beyond order pb)
    const int an = abs(n);
    const double2 rt = sr[an];  // (sig_{an-1} / sig_an, sig_{an+1} / sig_an)
    const double fm = n > 0 ? rt.x : rt.y, fp = n < 0 ? rt.x : rt.y;
    const double re = ((double)Sq.x - (double)Cq.x) + fm * ((double)Sa.x - (double)Ca.x) -
                      fp * ((double)Sb.x - (double)Cb.x);
    const double im = ((double)Sq.y - (double)Cq.y) + fm * ((double)Sa.y - (double)Ca.y) -
                      fp * ((double)Sb.y - (double)Cb.y);
    partial[seg_poff[it.x + u] + n + pb] = mk(re, im);
  }
}

__global__ void __launch_bounds__(kThreads) p2m_sum_mixed_kernel(
    Fmm F, const int* __restrict__ leaves, const int* __restrict__ lseg,
    const long long* __restrict__ seg_poff, const cd* __restrict__ partial) {
  const int t = blockIdx.x, b = leaves[t];
  const int l = F.level[b];
  const int pb = F.lpb[l], Q = 2 * pb + 1;
  const double* cv = F.conv + (size_t)l * (F.pbmax + 1);
  cd* dst = F.mpole + F.eoff[b];
  for (int n = threadIdx.x; n < Q; n += kThreads) {
    cd sum = mk(0.0, 0.0);
    for (int g = lseg[t]; g < lseg[t + 1]; ++g) sum = cadd(sum, partial[seg_poff[g] + n]);
    dst[n] = cscale(sum, 1.0 / cv[abs(n - pb)]);
  }
}

// P2L in mixed precision: the item structure of p2l_item_kernel with FP32
// rows and sums. Row j of a source holds G_j e^{i j th} (j >= 0) and
// (-1)^j G_j e^{-i j th} (j < 0), G_j = sig_j H_j(k r) by the FP64 recurrence
// G_{j+1} = rec[j].x (1/x) G_j - rec[j].y G_{j-1} (sig of the box's level,
// sig_{pb+1} taken as sig_pb); X-list sources lie at least 1.5 box sides from
// the centre, so G_j is of order one or smaller. The angular factors are FP32
// between FP64 anchors every eighth order. Per output order n the charge and
// the two dipole sums are FP32 with Kahan compensation over the item's
// sources; lambda_n = sig_n gamma_n = Sq + (sig_n / sig_|n-1|) Sa -
// (sig_n / sig_|n+1|) Sb and lh_n = lambda_n conv_|n| are formed in FP64.
__global__ void __launch_bounds__(kThreads) p2l_item_mixed_kernel(
    Fmm F, const int4* __restrict__ items, const int* __restrict__ src,
    const long long* __restrict__ poff, cd* __restrict__ partial, unsigned sm_bytes,
    const double2* __restrict__ rec) {
  extern __shared__ cd smem[];
  const int4 it = items[blockIdx.x];  // (box, first position in src, sources, -)
  const int b = it.x, cnt = it.z;
  const int l = F.level[b];
  const int pb = F.lpb[l], RW = 2 * pb + 3;  // row: |t| <= pb+1
  const int chunk = rows_chunk(pb, sm_bytes);
  cd* rows = smem;                        // [chunk][RW], FP32 entries in the first half of each slot
  cd* sq = rows + chunk * RW;             // [chunk]
  cd* sa = sq + chunk;                    // [chunk]  A = d (k/2) nu
  cd* sb = sa + chunk;                    // [chunk]  B = d (k/2) conj(nu)
  const double2 m = F.centre[b];
  if ((int)threadIdx.x < cnt) {
    const int i = src[it.y + threadIdx.x];
    const double dx = F.sxy[i].x - m.x, dy = F.sxy[i].y - m.y;
    const double d2 = dx * dx + dy * dy;
    const double ir = rsqrt(d2), x = F.k * (d2 * ir), ix = ir * F.ik;
    cd h0, h1;
    hankel01_wide(x, ix, h0, h1);
    const double2* R = rec + (size_t)l * (F.pbmax + 2);
    const cd e1 = mk(dx * ir, dy * ir);
    cd e8 = cmul(e1, e1);
    e8 = cmul(e8, e8);
    e8 = cmul(e8, e8);
    const float2 e1f = f2(e1);
    float2* row = reinterpret_cast<float2*>(rows + threadIdx.x * RW + (pb + 1));
    cd gprev = h0, gcur = cscale(h1, R[0].x);  // G_0, G_1
    cd E = mk(1.0, 0.0);
    float2 ef = make_float2(1.f, 0.f);
    row[0] = f2(h0);
    for (int j = 1; j <= pb + 1; ++j) {
      if ((j & 7) == 0) {  // e^{i j th}: an FP64 anchor every eighth order
        E = cmul(E, e8);
        ef = f2(E);
      } else {
        ef = fmul(ef, e1f);
      }
      const float2 g = f2(gcur);
      const float2 wp = fmul(g, ef);
      const float2 wq = fmul(g, make_float2(ef.x, -ef.y));
      row[2 * j] = wp;
      row[-2 * j] = (j & 1) ? make_float2(-wq.x, -wq.y) : wq;
      if (j <= pb) {
        const double c1 = R[j].x * ix, c2 = R[j].y;
        const cd gn = mk(fma(c1, gcur.x, -c2 * gprev.x), fma(c1, gcur.y, -c2 * gprev.y));
        gprev = gcur;
        gcur = gn;
      }
    }
    const float4 ab = F.ab32[i];
    reinterpret_cast<float2*>(sq + threadIdx.x)[0] = F.q32[i];
    reinterpret_cast<float2*>(sa + threadIdx.x)[0] = make_float2(ab.x, ab.y);  // d (k/2) nu
    reinterpret_cast<float2*>(sb + threadIdx.x)[0] = make_float2(ab.z, ab.w);  // d (k/2) conj(nu)
  }
  __syncthreads();
  const double2* sr = F.sigr + (size_t)l * (F.pbmax + 2);
  const double* cv = F.conv + (size_t)l * (F.pbmax + 1);
  cd* dst = partial + poff[blockIdx.x] + pb;
  for (int n = (int)threadIdx.x - pb; n <= pb; n += kThreads) {
    float2 Sq = make_float2(0.f, 0.f), Cq = Sq, Sa = Sq, Ca = Sq, Sb = Sq, Cb = Sq;
    for (int j = 0; j < cnt; ++j) {
      const float2* r = reinterpret_cast<const float2*>(rows + j * RW + (pb + 1));
      if (F.has_S) kahan2(Sq, Cq, fmul(reinterpret_cast<const float2*>(sq + j)[0], r[2 * n]));
      if (F.has_D) {
        kahan2(Sa, Ca, fmul(reinterpret_cast<const float2*>(sa + j)[0], r[2 * (n - 1)]));
        kahan2(Sb, Cb, fmul(reinterpret_cast<const float2*>(sb + j)[0], r[2 * (n + 1)]));
      }
    }
    // sig_|n| / sig_|n-1| and sig_|n| / sig_|n+1| from the ratio table (which
    // holds sig_|n-1| / sig_|n| and sig_|n+1| / sig_|n|, 1 beyond order pb)
    const int an = abs(n);
    const double2 rt = sr[an];
    const double fm = 1.0 / (n > 0 ? rt.x : rt.y), fp = 1.0 / (n < 0 ? rt.x : rt.y);
    const double c = cv[an];
    const double re = ((double)Sq.x - (double)Cq.x) + fm * ((double)Sa.x - (double)Ca.x) -
                      fp * ((double)Sb.x - (double)Cb.x);
    const double im = ((double)Sq.y - (double)Cq.y) + fm * ((double)Sa.y - (double)Ca.y) -
                      fp * ((double)Sb.y - (double)Cb.y);
    dst[n] = mk(re * c, im * c);
  }
}

// Lift the 48 KB default of dynamic shared memory to the device's opt-in
// maximum for every kernel that uses it (once per device); the size given at
// each launch still decides the occupancy.

qbx_status configure_kernels() {
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  QBX_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(dev)) return QBX_OK;
  int optin = 0;
  QBX_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const void* k[] = {(const void*)p2m_item_kernel, (const void*)p2m_item_mixed_kernel,
                     (const void*)m2m_kernel,
                     (const void*)p2l_item_kernel, (const void*)p2l_item_mixed_kernel,
                     (const void*)l2l_kernel};
  for (const void* f : k)
    QBX_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  TRY_MIXED(configure_mixed_kernels(optin));
  TRY_MIXED(configure_tc_kernels(optin));
  g_smem_optin = optin;
  done.insert(dev);
  return QBX_OK;
}

// ---------------------------------------------------------------- P2QBXL, one warp per centre
// Lanes stride over the concatenated sources of the centre's U-list boxes (so
// the load is balanced to within one source), each lane keeps partial
// coefficients, and a reduce-scatter of shuffles adds them: after it, lane L
// holds coefficient indices K L .. K L + K - 1 of the 32 K padded ones
// (K = 1 for p <= 15, 2 for p = 16). Padding indices hold zeros.
template <int NC>
__device__ __forceinline__ void warp_reduce_scatter(cd (&acc)[NC], int lane) {
  constexpr int NP = 32 * ((NC + 31) / 32);
#pragma unroll
  for (int h = NP / 2, off = 16; off >= 1; h >>= 1, off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const cd lo = i < NC ? acc[i] : mk(0.0, 0.0);
      const cd hi = i + h < NC ? acc[i + h] : mk(0.0, 0.0);
      const cd send = upper ? lo : hi;
      cd keep = upper ? hi : lo;
      keep.x += __shfl_xor_sync(0xffffffffu, send.x, off);
      keep.y += __shfl_xor_sync(0xffffffffu, send.y, off);
      if (i < NC) acc[i] = keep;
    }
  }
}

template <int PM, bool HS, bool HD>
__global__ void __launch_bounds__(kThreads) p2qbxl_warp_kernel(Fmm F, const int* __restrict__ cleaf,
                                                               const int* __restrict__ wdoff,
                                                               const int* __restrict__ wdbox,
                                                               const int* __restrict__ clist,
                                                               int n_ctr, cd* __restrict__ alpha) {
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);  // position in clist  // sorted centre
  const int lane = threadIdx.x & 31;
  if (w >= n_ctr) return;  // whole warps leave together
  const int i = clist[w];  // sorted centre
  const int b = cleaf[i];
  const double k = F.k, ik = 1.0 / k;
  const int p = F.p, P = 2 * p + 1;
  const double2 c = F.cxy[i];
  cd acc[2 * PM + 1];
#pragma unroll
  for (int j = 0; j <= 2 * PM; ++j) acc[j] = mk(0.0, 0.0);
  auto one = [&](int j) {
    const double2 y = F.sxy[j];
    cd A = mk(0.0, 0.0), B = mk(0.0, 0.0);
    if (HD) {
      const cd dk = cscale(F.ds[j], 0.5 * k);
      const cd nu = mk(F.snrm[j].x, F.snrm[j].y);
      A = cmul(dk, nu);
      B = cmul(dk, cconj(nu));
    }
    p2qbxl_pair<PM, HS, HD>(acc, y.x - c.x, y.y - c.y, HS ? F.qs[j] : mk(0.0, 0.0), A, B, k, ik, p);
  };
  // U-list boxes of the leaf, then the W-list boxes summed directly for this centre
  const SourceCursor sc{F.uidx, F.rsrc, F.uoff[b], F.uoff[b + 1] - F.uoff[b], wdoff[i],
                        wdoff[i + 1] - wdoff[i], wdbox};
  deal_sources(sc, lane, one);
  warp_reduce_scatter<2 * PM + 1>(acc, lane);
  constexpr int K = (2 * PM + 1 + 31) / 32;
  cd* dst = alpha + (size_t)F.cid[i] * P;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int lo = K * lane + j - PM;
    if (lo >= -p && lo <= p) dst[lo + p] = cadd(dst[lo + p], acc[j]);
  }
}

template <int PM, bool HS, bool HD>
__global__ void __launch_bounds__(kThreads) p2qbxl_warp_mixed_kernel(Fmm F, const int* __restrict__ cleaf,
                                                                     const int* __restrict__ wdoff,
                                                                     const int* __restrict__ wdbox,
                                                                     const int* __restrict__ clist,
                                                                     int n_ctr, cd* __restrict__ alpha) {
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);  // position in clist
  const int lane = threadIdx.x & 31;
  if (w >= n_ctr) return;
  const int i = clist[w];
  const int b = cleaf[i];
  const double k = F.k, ik = 1.0 / k;
  const int p = F.p, P = 2 * p + 1;
  const double2 c = F.cxy[i];
  // sigma = 2^s within a factor sqrt 2 of rho = k r_c: the power that scales
  // the lane sums (ah_l = alpha_l sigma^|l|)
  const int s = ilogb(k * F.crad[i] * 1.4142135623730951);
  const float fr = pow2f(s), fi = pow2f(-s);
  float2 S[2 * PM + 1], C[2 * PM + 1];
#pragma unroll
  for (int j = 0; j <= 2 * PM; ++j) S[j] = C[j] = make_float2(0.f, 0.f);
  auto one = [&](int j) {
    const double2 y = F.sxy[j];
    float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
    if (HD) {  // A = d (k/2) nu, B = d (k/2) conj(nu), formed once per source
      const float4 ab = F.ab32[j];
      A = make_float2(ab.x, ab.y);
      B = make_float2(ab.z, ab.w);
    }
    p2qbxl_pair_mixed<PM, HS, HD>(S, C, y.x - c.x, y.y - c.y,
                                  HS ? F.q32[j] : make_float2(0.f, 0.f), A, B, k, ik, s, fr, fi,
                                  p);
  };
  const SourceCursor sc{F.uidx, F.rsrc, F.uoff[b], F.uoff[b + 1] - F.uoff[b], wdoff[i],
                        wdoff[i + 1] - wdoff[i], wdbox};
  deal_sources(sc, lane, one);
  // lane partial sums (compensation removed) in FP64, then the warp sum
  cd acc[2 * PM + 1];
#pragma unroll
  for (int j = 0; j <= 2 * PM; ++j)
    acc[j] = mk((double)S[j].x - (double)C[j].x, (double)S[j].y - (double)C[j].y);
  warp_reduce_scatter<2 * PM + 1>(acc, lane);
  constexpr int K = (2 * PM + 1 + 31) / 32;
  cd* dst = alpha + (size_t)F.cid[i] * P;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int lo = K * lane + j - PM;
    if (lo >= -p && lo <= p) {
      const double ip = pow2d(-s * abs(lo));  // sigma^-|lo|: ah_l = alpha_l sigma^|l|
      dst[lo + p] = cadd(dst[lo + p], cscale(acc[j], ip));
    }
  }
}

}  // namespace

#define TRY(x)                          \
  do {                                  \
    qbx_status s_ = (x);                \
    if (s_ != QBX_OK) return s_;        \
  } while (0)

// Shared memory of a source-row kernel (P2M, P2L) at box order pb: a full
// warp's chunk of rows while that keeps the block within kRowsSmemTarget
// (several blocks per SM), else half a warp's; never above the opt-in limit.
constexpr size_t kRowsSmemTarget = 60 * 1024;
size_t rows_launch_smem(int pb) {
  const size_t full = rows_smem(pb, kChunk);
  const size_t sm = full <= kRowsSmemTarget ? full : rows_smem(pb, kChunk / 2);
  return std::min(sm, (size_t)g_smem_optin);
}

// Largest box order among the levels l with off[l+1] > off[l] (boxes of a
// level-ordered list); the single launch over the list sizes its shared memory
// for it. The lists are ordered coarse to fine, so the CTAs with the most work
// (highest orders) start first.
int max_order(const std::vector<int>& pb, const std::vector<int>& off) {
  int m = 0;
  for (size_t l = 0; l + 1 < off.size(); ++l)
    if (off[l + 1] > off[l]) m = std::max(m, pb[l]);
  return m;
}

qbx_status fmm_plan_build(qbx_handle* h, const qbx_tree_desc* d, const int64_t* on_node_dev,
                          const int8_t* on_side_dev, double eps) {
  if (h->fmm) fmm_plan_free(h->fmm);
  FmmPlan* f = new FmmPlan();
  h->fmm = f;
  const int n_max = d->n_max > 0 ? d->n_max : 64;
  TRY(tree_build(h, f, n_max, kLeafOverRadius));
  TRY(tree_lists(h, f));
  TRY(tree_associate(h, f, on_node_dev, on_side_dev, eps));
  TRY(gather_sorted(h, f));
  const int p_add = d->p_add >= 0 ? d->p_add : qbx_default_p_add(h->p);
  if (f->n_levels > kMaxLevels + 1) {
    set_error("tree has %d levels (at most %d)", f->n_levels, kMaxLevels + 1);
    return QBX_ERR_ARG;
  }
  // box order per level (Sec. 7.1): p_fmm on the finest level, more on coarse
  // levels whose boxes span wavelengths, plus p_add
  f->h_pb.assign(f->n_levels, 0);
  TRY(qbx_fmm_level_orders(h->k, f->side, f->n_levels, std::max(1, d->p_fmm), p_add,
                           f->h_pb.data()));
  f->pb_max = 1;
  for (int l = 0; l < f->n_levels; ++l) f->pb_max = std::max(f->pb_max, f->h_pb[l]);
  f->pb_fine = f->h_pb[f->n_levels - 1];
  // scales, powers, translation tables
  std::vector<double> sc(f->n_levels);
  for (int l = 0; l < f->n_levels; ++l) {
    sc[l] = std::min(1.0, h->k * f->side / (double)(1 << l));
    if (l >= 2 && std::pow(sc[l], f->h_pb[l] + 1) < 1e-250) {
      set_error("tree level %d too fine for the box order %d (k*side = %.3g)", l, f->h_pb[l],
                sc[l]);
      return QBX_ERR_ARG;
    }
  }
  // coefficient offsets: boxes of level l are [level_off[l], level_off[l+1])
  {
    std::vector<long long> eo(f->n_boxes);
    long long off = 0;
    for (int l = 0; l < f->n_levels; ++l)
      for (int b = f->level_off[l]; b < f->level_off[l + 1]; ++b) {
        eo[b] = off;
        off += 2 * f->h_pb[l] + 1;
      }
    f->n_coef = off;
    QBX_CUDA_TRY(f->eoff.alloc(std::max(1, f->n_boxes)));
    if (f->n_boxes)
      QBX_CUDA_TRY(cudaMemcpy(f->eoff.ptr, eo.data(), eo.size() * sizeof(long long),
                              cudaMemcpyHostToDevice));
  }
  QBX_CUDA_TRY(f->lpb.alloc(f->n_levels));
  QBX_CUDA_TRY(cudaMemcpy(f->lpb.ptr, f->h_pb.data(), f->n_levels * sizeof(int),
                          cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(f->scale.alloc(f->n_levels));
  QBX_CUDA_TRY(cudaMemcpy(f->scale.ptr, sc.data(), sc.size() * sizeof(double),
                          cudaMemcpyHostToDevice));
  const int pbm = f->pb_max, TS = 4 * pbm + 1;
  QBX_CUDA_TRY(f->t_m2l.alloc((size_t)f->n_levels * 49 * TS));
  QBX_CUDA_TRY(f->t_m2m.alloc((size_t)f->n_levels * 4 * TS));
  QBX_CUDA_TRY(f->t_l2l.alloc((size_t)f->n_levels * 4 * TS));
  QBX_CUDA_TRY(f->pw.alloc((size_t)f->n_levels * (2 * pbm + 3)));
  QBX_CUDA_TRY(f->ipw.alloc((size_t)f->n_levels * (pbm + 2)));
  DevBuf<double> jwork;
  QBX_CUDA_TRY(jwork.alloc((size_t)f->n_levels * 57 * (2 * pbm + 1)));
  tables_kernel<<<nblk(f->n_levels * 57, 64), 64>>>(f->n_levels, f->side, h->k, pbm, f->lpb.ptr,
                                                    f->scale.ptr, f->t_m2l.ptr, f->t_m2m.ptr,
                                                    f->t_l2l.ptr, jwork.ptr);
  powers_kernel<<<1, 64>>>(f->n_levels, pbm, f->lpb.ptr, f->scale.ptr, f->pw.ptr, f->ipw.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(f->mpole.alloc(std::max<int64_t>(1, f->n_coef)));
  QBX_CUDA_TRY(f->local.alloc(std::max<int64_t>(1, f->n_coef)));
  QBX_CUDA_TRY(f->lpq.alloc(std::max<int64_t>(1, f->n_coef)));
  QBX_CUDA_TRY(f->sp_m.alloc(std::max<int64_t>(1, f->n_coef)));
  QBX_CUDA_TRY(f->sp_e.alloc(std::max<int64_t>(1, f->n_coef)));
  TRY(configure_kernels());
  // side stream and events for the concurrent near-field stages (created here,
  // outside any stream capture; owned by the plan)
  QBX_CUDA_TRY(cudaStreamCreateWithFlags(&f->near_stream, cudaStreamNonBlocking));
  for (cudaEvent_t* ev : {&f->ev_fork, &f->ev_join, &f->ev_p2l, &f->ev_m2m, &f->ev_out})
    QBX_CUDA_TRY(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  // the largest per-block footprint (the M2M / L2L GEMMs at the largest
  // order) bounds all others
  const size_t smem_need = gemm_smem_bytes(f->pb_max);
  if (smem_need > (size_t)g_smem_optin) {
    set_error("box order %d needs %zu bytes of shared memory per block (device: %d)", f->pb_max,
              smem_need, g_smem_optin);
    return QBX_ERR_ARG;
  }
  TRY(mixed_plan_build(h, f));
  TRY(tc_plan_build(h, f));
  TRY(tc_mml_plan_build(h, f));
  QBX_CUDA_TRY(f->qs.alloc(std::max<int64_t>(1, h->n_src)));
  QBX_CUDA_TRY(f->ds.alloc(std::max<int64_t>(1, h->n_src)));
  QBX_CUDA_TRY(f->q32.alloc(std::max<int64_t>(1, h->n_src)));
  QBX_CUDA_TRY(f->ab32.alloc(std::max<int64_t>(1, h->n_src)));
  // leaves holding sources (P2M)
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  // stats
  std::vector<int> uoff(f->n_boxes + 1), woff(f->n_boxes + 1), xoff(f->n_boxes + 1);
  std::vector<int2> rs(f->n_boxes), rc(f->n_boxes), rt(f->n_boxes);
  std::vector<int> uidx(std::max<int64_t>(1, f->U.nnz)), widx(std::max<int64_t>(1, f->W.nnz)),
      xidx(std::max<int64_t>(1, f->X.nnz));
  QBX_CUDA_TRY(cudaMemcpy(uoff.data(), f->U.off.ptr, uoff.size() * 4, cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(woff.data(), f->W.off.ptr, woff.size() * 4, cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(xoff.data(), f->X.off.ptr, xoff.size() * 4, cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(rs.data(), f->box.rng[PT_SRC].ptr, rs.size() * 8, cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(rc.data(), f->box.rng[PT_CTR].ptr, rc.size() * 8, cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(rt.data(), f->box.rng[PT_TGT].ptr, rt.size() * 8, cudaMemcpyDeviceToHost));
  if (f->U.nnz) QBX_CUDA_TRY(cudaMemcpy(uidx.data(), f->U.idx.ptr, f->U.nnz * 4, cudaMemcpyDeviceToHost));
  if (f->W.nnz) QBX_CUDA_TRY(cudaMemcpy(widx.data(), f->W.idx.ptr, f->W.nnz * 4, cudaMemcpyDeviceToHost));
  if (f->X.nnz) QBX_CUDA_TRY(cudaMemcpy(xidx.data(), f->X.idx.ptr, f->X.nnz * 4, cudaMemcpyDeviceToHost));
  std::vector<int> assoc_s(std::max<int64_t>(1, h->n_tgt));
  if (h->n_tgt)
    QBX_CUDA_TRY(cudaMemcpy(assoc_s.data(), f->t_assoc.ptr, h->n_tgt * 4, cudaMemcpyDeviceToHost));
  std::vector<int> leaves(f->n_leaves), blev(f->n_boxes);
  QBX_CUDA_TRY(cudaMemcpy(leaves.data(), f->leaves.ptr, leaves.size() * 4, cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(blev.data(), f->box.level.ptr, blev.size() * 4, cudaMemcpyDeviceToHost));
  int64_t p2qbxl = 0, p2p = 0, m2qbxl = 0, m2p = 0, p2l = 0;
  std::vector<int> src_leaves;
  for (int b : leaves) {
    int64_t us = 0;
    for (int e = uoff[b]; e < uoff[b + 1]; ++e) us += rs[uidx[e]].y - rs[uidx[e]].x;
    int64_t nd = 0;
    for (int i = rt[b].x; i < rt[b].y; ++i) nd += assoc_s[i] < 0 ? 1 : 0;
    p2qbxl += us * (rc[b].y - rc[b].x);
    p2p += us * nd;
    m2qbxl += (int64_t)(woff[b + 1] - woff[b]) * (rc[b].y - rc[b].x);
    m2p += (int64_t)(woff[b + 1] - woff[b]) * nd;
    if (rs[b].y > rs[b].x && blev[b] >= 2) src_leaves.push_back(b);
    f->q_leaf = std::max(f->q_leaf, 2 * f->h_pb[blev[b]] + 1);
    for (int e = woff[b]; e < woff[b + 1]; ++e)
      f->q_w = std::max(f->q_w, 2 * f->h_pb[blev[widx[e]]] + 1);
  }
  // leaf of every sorted target; direct targets, and those among them whose
  // leaf has U-list sources (P2P) or a W list (M2P)
  {
    std::vector<int> tl(std::max<int64_t>(1, h->n_tgt), 0), dt, ut, wt;
    for (int b : leaves)
      for (int i = rt[b].x; i < rt[b].y; ++i) tl[i] = b;
    std::vector<int64_t> usrc(f->n_boxes, 0);
    for (int b : leaves)
      for (int e = uoff[b]; e < uoff[b + 1]; ++e) usrc[b] += rs[uidx[e]].y - rs[uidx[e]].x;
    for (int64_t i = 0; i < h->n_tgt; ++i) {
      if (assoc_s[i] >= 0) continue;
      const int b = tl[i];
      dt.push_back((int)i);
      if (usrc[b] > 0) ut.push_back((int)i);
      if (woff[b + 1] > woff[b]) wt.push_back((int)i);
    }
    auto up = [](DevBuf<int>& d, const std::vector<int>& v) -> qbx_status {
      QBX_CUDA_TRY(d.alloc(std::max<size_t>(1, v.size())));
      if (!v.empty())
        QBX_CUDA_TRY(cudaMemcpy(d.ptr, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
      return QBX_OK;
    };
    // M2P work items: (target, W box) pairs in wtgt order, CSR by position
    std::vector<int> mt, mbx, moff(wt.size() + 1, 0);
    for (size_t t = 0; t < wt.size(); ++t) {
      const int b = tl[wt[t]];
      for (int e = woff[b]; e < woff[b + 1]; ++e) {
        mt.push_back(wt[t]);
        mbx.push_back(widx[e]);
      }
      moff[t + 1] = (int)mt.size();
    }
    TRY(up(f->tleaf, tl));
    TRY(up(f->dtgt, dt));
    TRY(up(f->utgt, ut));
    TRY(up(f->wtgt, wt));
    TRY(up(f->m2p_tgt, mt));
    TRY(up(f->m2p_box, mbx));
    TRY(up(f->m2p_off, moff));
    QBX_CUDA_TRY(f->m2p_part.alloc(std::max<size_t>(1, mt.size())));
    {  // the boxes M2P reads, and FP32 room for their normalised multipoles
      std::vector<int> wb(mbx);
      std::sort(wb.begin(), wb.end());
      wb.erase(std::unique(wb.begin(), wb.end()), wb.end());
      TRY(up(f->m2p_wbox, wb));
      f->n_m2p_wbox = (int)wb.size();
      QBX_CUDA_TRY(f->m2p_mu.alloc(wb.empty() ? 1 : std::max<int64_t>(1, f->n_coef)));
    }
    f->n_dtgt = (int)dt.size();
    f->n_utgt = (int)ut.size();
    f->n_wtgt = (int)wt.size();
    f->n_m2p_pairs = (int)mt.size();
  }
  // leaf of every centre (sorted order)
  std::vector<int> cl(std::max<int64_t>(1, h->n_ctr), 0);
  for (int b : leaves)
    for (int i = rc[b].x; i < rc[b].y; ++i) cl[i] = b;
  f->cleaf_pb_max = 0;
  for (int b : leaves)
    if (rc[b].y > rc[b].x) f->cleaf_pb_max = std::max(f->cleaf_pb_max, f->h_pb[blev[b]]);
  QBX_CUDA_TRY(f->cleaf.alloc(cl.size()));
  QBX_CUDA_TRY(cudaMemcpy(f->cleaf.ptr, cl.data(), cl.size() * sizeof(int),
                          cudaMemcpyHostToDevice));
  // W-list boxes per centre: those far enough from the centre's disk for
  // M2QBXL ((R_c + r_z) <= kW |z - m_c|), and the rest, summed directly in
  // P2QBXL (wd_off / wd_box, CSR by sorted centre)
  std::vector<std::vector<int>> wtrans(std::max<int64_t>(1, h->n_ctr));
  int64_t w_direct_src = 0;
  {
    std::vector<double2> cxy(std::max<int64_t>(1, h->n_ctr)), bctr(f->n_boxes);
    std::vector<double> crad(std::max<int64_t>(1, h->n_ctr));
    if (h->n_ctr) {
      QBX_CUDA_TRY(cudaMemcpy(cxy.data(), f->c_xy.ptr, h->n_ctr * sizeof(double2), cudaMemcpyDeviceToHost));
      QBX_CUDA_TRY(cudaMemcpy(crad.data(), f->c_r.ptr, h->n_ctr * sizeof(double), cudaMemcpyDeviceToHost));
    }
    QBX_CUDA_TRY(cudaMemcpy(bctr.data(), f->box.centre.ptr, f->n_boxes * sizeof(double2), cudaMemcpyDeviceToHost));
    std::vector<int> dbx, doff(std::max<int64_t>(1, h->n_ctr) + 1, 0);
    for (int64_t i = 0; i < h->n_ctr; ++i) {
      const int b = cl[i];
      for (int e = woff[b]; e < woff[b + 1]; ++e) {
        const int c = widx[e];
        const double dx = cxy[i].x - bctr[c].x, dy = cxy[i].y - bctr[c].y;
        const double Rc = 0.70710678118654752 * f->side / (double)(1 << blev[c]);
        if (Rc + crad[i] > kW * std::sqrt(dx * dx + dy * dy)) {
          dbx.push_back(c);
          w_direct_src += rs[c].y - rs[c].x;
        } else {
          wtrans[i].push_back(c);
        }
      }
      doff[i + 1] = (int)dbx.size();
    }
    QBX_CUDA_TRY(f->wd_box.alloc(std::max<size_t>(1, dbx.size())));
    QBX_CUDA_TRY(f->wd_off.alloc(doff.size()));
    if (!dbx.empty())
      QBX_CUDA_TRY(cudaMemcpy(f->wd_box.ptr, dbx.data(), dbx.size() * 4, cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(f->wd_off.ptr, doff.data(), doff.size() * 4, cudaMemcpyHostToDevice));
  }
  // Centre sets: every centre (set 0), and the centres some target is
  // associated with (set 1; alpha is only read there). Each set lists sorted
  // centre indices and its M2QBXL (centre, W box) pairs, CSR by list position.
  {
    std::vector<int> all(std::max<int64_t>(0, h->n_ctr)), used;
    for (int64_t i = 0; i < h->n_ctr; ++i) all[i] = (int)i;
    if (h->n_ctr) {
      std::vector<int> cperm(h->n_ctr), inv(h->n_ctr), ta(std::max<int64_t>(1, h->n_tgt));
      std::vector<char> mark(h->n_ctr, 0);
      QBX_CUDA_TRY(cudaMemcpy(cperm.data(), f->perm[PT_CTR].ptr, h->n_ctr * 4, cudaMemcpyDeviceToHost));
      if (h->n_tgt)
        QBX_CUDA_TRY(cudaMemcpy(ta.data(), h->assoc.ptr, h->n_tgt * 4, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < h->n_ctr; ++i) inv[cperm[i]] = (int)i;
      for (int64_t t = 0; t < h->n_tgt; ++t)
        if (ta[t] >= 0) mark[inv[ta[t]]] = 1;
      if (h->has_avg) {  // two-sided targets also read their node's interior centre
        std::vector<int8_t> av(h->n_tgt);
        QBX_CUDA_TRY(cudaMemcpy(av.data(), h->avg.ptr, h->n_tgt, cudaMemcpyDeviceToHost));
        for (int64_t t = 0; t < h->n_tgt; ++t)
          if (av[t] && ta[t] >= 0) mark[inv[ta[t] + h->n_nodes]] = 1;
      }
      for (int64_t i = 0; i < h->n_ctr; ++i)
        if (mark[i]) used.push_back((int)i);
    }
    size_t max_pairs = 1;
    for (int k = 0; k < 2; ++k) {
      const std::vector<int>& list = k == 0 ? all : used;
      CentreSet& S = f->cset[k];
      std::vector<int> pc, pbx, off(list.size() + 1, 0);
      for (size_t t = 0; t < list.size(); ++t) {
        for (int c : wtrans[list[t]]) {
          pc.push_back(list[t]);
          pbx.push_back(c);
        }
        off[t + 1] = (int)pc.size();
      }
      S.n = (int)list.size();
      S.n_pairs = (int)pc.size();
      S.wp_pbmax = 0;
      for (int c : pbx) S.wp_pbmax = std::max(S.wp_pbmax, f->h_pb[blev[c]]);
      max_pairs = std::max(max_pairs, pc.size());
      auto up = [](DevBuf<int>& d, const std::vector<int>& v) -> qbx_status {
        QBX_CUDA_TRY(d.alloc(std::max<size_t>(1, v.size())));
        if (!v.empty())
          QBX_CUDA_TRY(cudaMemcpy(d.ptr, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
        return QBX_OK;
      };
      TRY(up(S.clist, list));
      TRY(up(S.wp_ctr, pc));
      TRY(up(S.wp_box, pbx));
      TRY(up(S.wp_off, off));
    }
    QBX_CUDA_TRY(f->wpart.alloc(max_pairs * (size_t)(2 * h->p + 1)));
    f->n_wpairs = f->cset[0].n_pairs;
    QBX_CUDA_TRY(f->sf_m.alloc((size_t)f->n_levels * (2 * h->p + 1)));
    QBX_CUDA_TRY(f->sf_e.alloc((size_t)f->n_levels * (2 * h->p + 1)));
  }
  // P2M work items over segments of the source leaves (see p2m_item_kernel)
  {
    int pbs = 0;  // largest order over the source leaves
    for (int b : src_leaves) pbs = std::max(pbs, f->h_pb[blev[b]]);
    f->p2m_sm = rows_launch_smem(pbs);
    const int chunk = rows_chunk(pbs, f->p2m_sm);  // the least capacity over the leaf levels
    std::vector<int> sleaf, psrc, psleaf, lseg(src_leaves.size() + 1, 0);
    std::vector<int2> srow;
    std::vector<long long> spoff;
    std::vector<int4> items;
    long long ptot = 0;
    int cur_lev = -1;
    for (size_t t = 0; t < src_leaves.size(); ++t) {
      const int b = src_leaves[t];
      const int Q = 2 * f->h_pb[blev[b]] + 1;
      lseg[t] = (int)sleaf.size();
      for (int i0 = rs[b].x; i0 < rs[b].y;) {
        if (items.empty() || cur_lev != blev[b] || items.back().w == chunk) {
          items.push_back(make_int4((int)sleaf.size(), 0, (int)psrc.size(), 0));
          cur_lev = blev[b];
        }
        int4& it = items.back();
        const int cnt = std::min(chunk - it.w, rs[b].y - i0);
        srow.push_back(make_int2(it.w, cnt));
        sleaf.push_back(b);
        spoff.push_back(ptot);
        ptot += Q;
        for (int i = i0; i < i0 + cnt; ++i) {
          psrc.push_back(i);
          psleaf.push_back(b);
        }
        it.y += 1;
        it.w += cnt;
        i0 += cnt;
      }
    }
    lseg[src_leaves.size()] = (int)sleaf.size();
    f->n_p2m_items = (int)items.size();
    QBX_CUDA_TRY(f->p2m_items.alloc(std::max<size_t>(1, items.size())));
    QBX_CUDA_TRY(f->p2m_segleaf.alloc(std::max<size_t>(1, sleaf.size())));
    QBX_CUDA_TRY(f->p2m_segrow.alloc(std::max<size_t>(1, srow.size())));
    QBX_CUDA_TRY(f->p2m_segpoff.alloc(std::max<size_t>(1, spoff.size())));
    QBX_CUDA_TRY(f->p2m_lseg.alloc(lseg.size()));
    QBX_CUDA_TRY(f->p2m_src.alloc(std::max<size_t>(1, psrc.size())));
    QBX_CUDA_TRY(f->p2m_srcleaf.alloc(std::max<size_t>(1, psleaf.size())));
    QBX_CUDA_TRY(f->p2m_part.alloc(std::max<long long>(1, ptot)));
    if (!items.empty()) {
      QBX_CUDA_TRY(cudaMemcpy(f->p2m_items.ptr, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(cudaMemcpy(f->p2m_segleaf.ptr, sleaf.data(), sleaf.size() * sizeof(int), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(cudaMemcpy(f->p2m_segrow.ptr, srow.data(), srow.size() * sizeof(int2), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(cudaMemcpy(f->p2m_segpoff.ptr, spoff.data(), spoff.size() * sizeof(long long), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(cudaMemcpy(f->p2m_src.ptr, psrc.data(), psrc.size() * sizeof(int), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(cudaMemcpy(f->p2m_srcleaf.ptr, psleaf.data(), psleaf.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    QBX_CUDA_TRY(cudaMemcpy(f->p2m_lseg.ptr, lseg.data(), lseg.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  for (int b = 0; b < f->n_boxes; ++b)
    for (int e = xoff[b]; e < xoff[b + 1]; ++e) p2l += rs[xidx[e]].y - rs[xidx[e]].x;
  {  // P2L work items: each X box's sources, cut into pieces of one row chunk
    std::vector<int> xb(std::max(1, f->n_xbox));
    if (f->n_xbox)
      QBX_CUDA_TRY(cudaMemcpy(xb.data(), f->xbox.ptr, f->n_xbox * sizeof(int), cudaMemcpyDeviceToHost));
    const int pbx = max_order(f->h_pb, f->xbox_off);
    f->p2l_sm = rows_launch_smem(pbx);
    const int chunk = rows_chunk(pbx, f->p2l_sm);  // the least capacity over the X levels
    std::vector<int> src, boff(f->n_xbox + 1, 0);
    std::vector<int4> items;
    std::vector<long long> poff;
    long long ptot = 0;
    for (int t = 0; t < f->n_xbox; ++t) {
      const int b = xb[t];
      const int Q = 2 * f->h_pb[blev[b]] + 1;
      const int s0 = (int)src.size();
      for (int e = xoff[b]; e < xoff[b + 1]; ++e)
        for (int i = rs[xidx[e]].x; i < rs[xidx[e]].y; ++i) src.push_back(i);
      boff[t] = (int)items.size();
      for (int a = s0; a < (int)src.size(); a += chunk) {
        items.push_back(make_int4(b, a, std::min(chunk, (int)src.size() - a), 0));
        poff.push_back(ptot);
        ptot += Q;
      }
    }
    boff[f->n_xbox] = (int)items.size();
    f->n_p2l_items = (int)items.size();
    QBX_CUDA_TRY(f->p2l_items.alloc(std::max<size_t>(1, items.size())));
    QBX_CUDA_TRY(f->p2l_poff.alloc(std::max<size_t>(1, poff.size())));
    QBX_CUDA_TRY(f->p2l_src.alloc(std::max<size_t>(1, src.size())));
    QBX_CUDA_TRY(f->p2l_boff.alloc(boff.size()));
    QBX_CUDA_TRY(f->p2l_part.alloc(std::max<long long>(1, ptot)));
    if (!items.empty()) {
      QBX_CUDA_TRY(cudaMemcpy(f->p2l_items.ptr, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(cudaMemcpy(f->p2l_poff.ptr, poff.data(), poff.size() * sizeof(long long), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(cudaMemcpy(f->p2l_src.ptr, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    QBX_CUDA_TRY(cudaMemcpy(f->p2l_boff.ptr, boff.data(), boff.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  QBX_CUDA_TRY(f->src_leaves.alloc(std::max<size_t>(1, src_leaves.size())));
  if (!src_leaves.empty())
    QBX_CUDA_TRY(cudaMemcpy(f->src_leaves.ptr, src_leaves.data(), src_leaves.size() * 4,
                            cudaMemcpyHostToDevice));
  f->n_src_leaves = (int)src_leaves.size();
  h->stats[4] = f->n_boxes;
  h->stats[5] = f->n_leaves;
  h->stats[6] = f->n_levels - 1;
  h->stats[7] = f->pb_fine;
  h->stats[19] = f->pb_max;
  h->stats[8] = f->U.nnz;
  h->stats[9] = f->V.nnz;
  h->stats[10] = f->W.nnz;
  h->stats[11] = f->X.nnz;
  h->stats[12] = p2qbxl + w_direct_src;  // over all centres
  h->stats[13] = p2p;
  h->stats[14] = f->n_wpairs;
  h->stats[15] = m2p;
  h->stats[17] = p2l;
  {
    int64_t mm = 0;  // M2M and L2L translations (parents on levels >= 2)
    for (int b = 0; b < f->n_boxes; ++b)
      if (blev[b] >= 3) mm += 2;
    h->stats[18] = mm;
  }
  return QBX_OK;
}

namespace {

Fmm make_view(qbx_handle* h, FmmPlan* f, bool S, bool D) {
  Fmm F;
  F.level = f->box.level.ptr;
  F.child = f->box.child.ptr;
  F.centre = f->box.centre.ptr;
  F.rsrc = f->box.rng[PT_SRC].ptr;
  F.rctr = f->box.rng[PT_CTR].ptr;
  F.rtgt = f->box.rng[PT_TGT].ptr;
  F.uoff = f->U.off.ptr; F.uidx = f->U.idx.ptr;
  F.voff = f->V.off.ptr; F.vidx = f->V.idx.ptr; F.vcls = f->V_cls.ptr;
  F.woff = f->W.off.ptr; F.widx = f->W.idx.ptr;
  F.xoff = f->X.off.ptr; F.xidx = f->X.idx.ptr;
  F.sxy = f->s_xy.ptr; F.snrm = f->s_nrm.ptr; F.qs = f->qs.ptr; F.ds = f->ds.ptr;
  F.q32 = f->q32.ptr; F.ab32 = f->ab32.ptr;
  F.cxy = f->c_xy.ptr; F.crad = f->c_r.ptr; F.cid = f->perm[PT_CTR].ptr;
  F.txy = f->t_xy.ptr; F.tid = f->perm[PT_TGT].ptr; F.tassoc = f->t_assoc.ptr;
  F.lpb = f->lpb.ptr; F.eoff = f->eoff.ptr;
  F.scale = f->scale.ptr; F.pw = f->pw.ptr; F.ipw = f->ipw.ptr;
  F.t_m2l = f->t_m2l.ptr; F.t_m2m = f->t_m2m.ptr; F.t_l2l = f->t_l2l.ptr;
  F.mpole = f->mpole.ptr; F.local = f->local.ptr; F.lpq = f->lpq.ptr;
  F.conv = f->conv.ptr; F.lsig = f->lsig.ptr; F.isig = f->isig.ptr; F.sigr = f->sigr.ptr;
  F.k = h->k; F.ik = 1.0 / h->k; F.side = f->side; F.pbmax = f->pb_max; F.p = h->p; F.n_levels = f->n_levels;
  F.has_S = S ? 1 : 0; F.has_D = D ? 1 : 0;
  return F;
}

// L2QBXL at the centres of set C (adds to alpha).
qbx_status launch_l2qbxl(const Fmm& F, FmmPlan* f, qbx_handle* h, const CentreSet& C, cd* alpha,
                         bool mixed, cudaStream_t s) {
  if (C.n == 0) return QBX_OK;
  stage_begin(h, QBX_STAGE_L2QBXL, s);
  // a warp per G centres. G: up to 32 (every lane fills a row), but no more
  // than keeps about two warps per SM for a handle evaluated alone (the dot
  // products keep the FP64 pipe busy from one warp; batched handles share the
  // GPU), within the shared memory of the rows.
  {
    const int TW = f->cleaf_pb_max + h->p + 1;
    int G = 32;
    if (h->l2qbxl_g > 0) G = h->l2qbxl_g;  // set by an autotuner
    else
      while (!h->batched && G > 1 && (C.n + G - 1) / G < 152 * 2) G /= 2;
    // (batched handles share the SMs with other curves' stages and keep the
    // larger rows)
    const size_t lim = (mixed && !h->batched) ? kL2qbxlMixedSmem : kL2qbxlSmem;
    while (G > 1 && (size_t)G * TW * sizeof(cd) > lim) G /= 2;
    const size_t sm = (size_t)G * TW * sizeof(cd);
    if (mixed) {
      split_coef_kernel<<<nblk(f->n_coef, 256), 256, 0, s>>>(f->local.ptr, f->n_coef, f->sp_m.ptr,
                                                             f->sp_e.ptr);
      l2qbxl_mixed_kernel<<<nblk(C.n, G), 32, sm, s>>>(F, f->cleaf.ptr, C.clist.ptr, C.n, G, TW,
                                                      f->sp_m.ptr, f->sp_e.ptr, alpha);
      h->launches += 1;
    } else {
      l2qbxl_kernel<<<nblk(C.n, G), 32, sm, s>>>(F, f->cleaf.ptr, C.clist.ptr, C.n, G, TW, alpha);
    }
  }
  QBX_KCHECK("l2qbxl", s);
  stage_end(h, QBX_STAGE_L2QBXL, s);
  h->launches += 1;
  return QBX_OK;
}

// M2QBXL at the centres of set C (adds to alpha).
template <int PM>
qbx_status launch_m2qbxl(const Fmm& F, FmmPlan* f, qbx_handle* h, bool S, bool D,
                         const CentreSet& C, cd* alpha, bool mixed, cudaStream_t s) {
  if (C.n == 0) return QBX_OK;
  stage_begin(h, QBX_STAGE_M2QBXL, s);
  if (C.n_pairs > 0 && (S || D)) {
    const int np = C.n_pairs;
    cd* part = f->wpart.ptr;
    // mixed: pairs per warp PW (at most kM2qbxlMixedPairs for a handle
    // evaluated alone, 32 for batched handles, which share the SMs with other
    // curves' stages) so that a warp's split rows (20 B per order) take at most
    // kM2qbxlMixedSmem, and, for a handle evaluated alone, fewer while that
    // leaves under two warps per SM (few pairs: spread the sequential
    // recurrences over all SMs)
    const int TW = C.wp_pbmax + h->p + 1;
    int PW = h->batched ? 32 : kM2qbxlMixedPairs;
    while (PW > 1 && (size_t)PW * TW * 20 > kM2qbxlMixedSmem) PW /= 2;
    while (!h->batched && PW > 1 && (np + PW - 1) / PW < 152 * 2) PW /= 2;
    if (mixed && (size_t)PW * TW * 20 <= kM2qbxlMixedSmem) {
      const long long ncoef = f->n_coef;
      split_coef_kernel<<<nblk(ncoef, 256), 256, 0, s>>>(f->mpole.ptr, ncoef, f->sp_m.ptr,
                                                        f->sp_e.ptr);
      sf_split_kernel<<<f->n_levels, 64, 0, s>>>(F, f->sf_m.ptr, f->sf_e.ptr);
      m2qbxl_mixed_kernel<<<nblk(np, PW), 32, (size_t)PW * TW * 20, s>>>(
          F, C.wp_ctr.ptr, C.wp_box.ptr, np, PW, TW, f->sp_m.ptr, f->sp_e.ptr, f->sf_m.ptr,
          f->sf_e.ptr, part);
      h->launches += 2;
    } else {
      const int nparts = (2 * h->p + 1 + kM2qbxlOrders - 1) / kM2qbxlOrders;
      const unsigned gb = nblk((int64_t)np * nparts, kM2qbxlBlock);
      constexpr int B = kM2qbxlBlock;
      if (S && D) m2qbxl_pair_kernel<PM, true, true><<<gb, B, 0, s>>>(F, C.wp_ctr.ptr, C.wp_box.ptr, np, part);
      else if (S) m2qbxl_pair_kernel<PM, true, false><<<gb, B, 0, s>>>(F, C.wp_ctr.ptr, C.wp_box.ptr, np, part);
      else m2qbxl_pair_kernel<PM, false, true><<<gb, B, 0, s>>>(F, C.wp_ctr.ptr, C.wp_box.ptr, np, part);
    }
    QBX_KCHECK("m2qbxl", s);
    const int P = 2 * h->p + 1;
    m2qbxl_sum_kernel<<<nblk((int64_t)C.n * P, 256), 256, 0, s>>>(C.n, P, C.wp_off.ptr, part,
                                                                 f->perm[PT_CTR].ptr, C.clist.ptr,
                                                                 alpha);
    QBX_KCHECK("m2qbxl_sum", s);
    h->launches += 2;
  }
  stage_end(h, QBX_STAGE_M2QBXL, s);
  return QBX_OK;
}

// P2QBXL (U list and directly summed W boxes): one warp per centre, adds to alpha.
template <int PM>
qbx_status launch_centre_near(const Fmm& F, FmmPlan* f, qbx_handle* h, bool S, bool D,
                              const CentreSet& C, cd* alpha, bool mixed, cudaStream_t s) {
  if (!(S || D) || C.n == 0) return QBX_OK;
  stage_begin(h, QBX_STAGE_P2QBXL, s);
  const int nc = C.n;
  const unsigned gw = nblk(nc, kThreads / 32);  // one warp per centre
  const int* wo = f->wd_off.ptr;
  const int* wb = f->wd_box.ptr;
  const int* cl = C.clist.ptr;
  if (mixed) {
    if (S && D) p2qbxl_warp_mixed_kernel<PM, true, true><<<gw, kThreads, 0, s>>>(F, f->cleaf.ptr, wo, wb, cl, nc, alpha);
    else if (S) p2qbxl_warp_mixed_kernel<PM, true, false><<<gw, kThreads, 0, s>>>(F, f->cleaf.ptr, wo, wb, cl, nc, alpha);
    else p2qbxl_warp_mixed_kernel<PM, false, true><<<gw, kThreads, 0, s>>>(F, f->cleaf.ptr, wo, wb, cl, nc, alpha);
  } else {
    if (S && D) p2qbxl_warp_kernel<PM, true, true><<<gw, kThreads, 0, s>>>(F, f->cleaf.ptr, wo, wb, cl, nc, alpha);
    else if (S) p2qbxl_warp_kernel<PM, true, false><<<gw, kThreads, 0, s>>>(F, f->cleaf.ptr, wo, wb, cl, nc, alpha);
    else p2qbxl_warp_kernel<PM, false, true><<<gw, kThreads, 0, s>>>(F, f->cleaf.ptr, wo, wb, cl, nc, alpha);
  }
  QBX_KCHECK("p2qbxl", s);
  stage_end(h, QBX_STAGE_P2QBXL, s);
  h->launches += 1;
  return QBX_OK;
}


}  // namespace

namespace {

template <int PM>
qbx_status centre_near_dispatch(const Fmm& F, FmmPlan* f, qbx_handle* h, bool S, bool D,
                                const CentreSet& C, bool mixed, cudaStream_t s) {
  return launch_centre_near<PM>(F, f, h, S, D, C, h->alpha.ptr, mixed, s);
}

}  // namespace

// Stream organisation. Two streams: the caller's (main) and the plan's side
// stream. Every stage adds into zeroed outputs, and each output array is
// written by one stream at a time:
//   main: P2M, M2M | M2L (after P2L) | L2L, unscale | L2P (after M2P) |
//         L2QBXL (after the side stream)
//   side: zero alpha, out; P2L; P2QBXL; P2P | M2QBXL, M2P (after M2M)
// P2L needs only the strengths and adds into the locals before M2L does; the
// centre coefficients alpha are written by P2QBXL and M2QBXL (side) before
// L2QBXL (main); out is written by P2P and M2P (side) before L2P (main).
// L2QBXL follows L2P instead of running beside it: run concurrently, the two
// took longer than one after the other (2.62 against 2.10 ms for the whole
// step of the starfish k = 10 workload). With per-stage timing on, everything
// runs on the main stream in the same order, so that stage times do not
// overlap.
qbx_status fmm_eval(qbx_handle* h, bool S, bool D, cd* out, int precision, bool all_centres,
                    cudaStream_t s) {
  FmmPlan* f = h->fmm;
  if (!f) { set_error("FMM plan missing"); return QBX_ERR_STATE; }
  // alpha is formed at every centre when the caller asks for it, else only at
  // the centres some target is associated with (the only ones QBXL2P reads)
  const CentreSet& C = f->cset[all_centres ? 0 : 1];
  const std::vector<int>& pb = f->h_pb;
  const bool mixed = precision == QBX_MIXED;
  if (h->n_src > 0) {
    gather_strengths_kernel<<<nblk(h->n_src, 256), 256, 0, s>>>(
        h->n_src, f->perm[PT_SRC].ptr, h->q_str.ptr, h->d_str.ptr, f->s_nrm.ptr, h->k,
        f->qs.ptr, f->ds.ptr, mixed ? f->q32.ptr : nullptr, mixed ? f->ab32.ptr : nullptr);
    QBX_KCHECK("gather_strengths", s);
    h->launches += 1;
  }
  Fmm F = make_view(h, f, S, D);
  QBX_CUDA_TRY(cudaMemsetAsync(f->mpole.ptr, 0, (size_t)f->n_coef * sizeof(cd), s));
  QBX_CUDA_TRY(cudaMemsetAsync(f->local.ptr, 0, (size_t)f->n_coef * sizeof(cd), s));
  const bool fork = !h->timing && !debug_sync() && !h->batched && f->near_stream != nullptr;
  cudaStream_t s2 = fork ? f->near_stream : s;
  auto signal = [&](cudaEvent_t ev, cudaStream_t from) -> qbx_status {
    if (fork) QBX_CUDA_TRY(cudaEventRecord(ev, from));
    return QBX_OK;
  };
  auto wait = [&](cudaStream_t on, cudaEvent_t ev) -> qbx_status {
    if (fork) QBX_CUDA_TRY(cudaStreamWaitEvent(on, ev, 0));
    return QBX_OK;
  };
  TRY(signal(f->ev_fork, s));
  TRY(wait(s2, f->ev_fork));
  const int P = 2 * h->p + 1;
  // ---- side: zero the outputs, P2L, then the near field
  if (h->n_ctr > 0) QBX_CUDA_TRY(cudaMemsetAsync(h->alpha.ptr, 0, (size_t)h->n_ctr * P * sizeof(cd), s2));
  if (h->n_tgt > 0) QBX_CUDA_TRY(cudaMemsetAsync(out, 0, (size_t)h->n_tgt * sizeof(cd), s2));
  stage_begin(h, QBX_STAGE_P2L, s2);
  if ((S || D) && f->n_p2l_items > 0) {  // X lists without sources add nothing
    if (mixed)
      p2l_item_mixed_kernel<<<f->n_p2l_items, kThreads, f->p2l_sm, s2>>>(
          F, f->p2l_items.ptr, f->p2l_src.ptr, f->p2l_poff.ptr, f->p2l_part.ptr,
          (unsigned)f->p2l_sm, f->m2p_rec.ptr);
    else
      p2l_item_kernel<<<f->n_p2l_items, kThreads, f->p2l_sm, s2>>>(
          F, f->p2l_items.ptr, f->p2l_src.ptr, f->p2l_poff.ptr, f->p2l_part.ptr, (unsigned)f->p2l_sm);
    QBX_KCHECK("p2l", s2);
    p2l_sum_kernel<<<f->n_xbox, kThreads, 0, s2>>>(F, f->xbox.ptr, f->p2l_boff.ptr, f->p2l_poff.ptr,
                                                  f->p2l_part.ptr);
    QBX_KCHECK("p2l_sum", s2);
    h->launches += 2;
  }
  stage_end(h, QBX_STAGE_P2L, s2);
  TRY(signal(f->ev_p2l, s2));
  if (h->n_ctr > 0) {
    if (h->p <= 4) TRY(centre_near_dispatch<4>(F, f, h, S, D, C, mixed, s2));
    else if (h->p <= 8) TRY(centre_near_dispatch<8>(F, f, h, S, D, C, mixed, s2));
    else if (h->p <= 12) TRY(centre_near_dispatch<12>(F, f, h, S, D, C, mixed, s2));
    else TRY(centre_near_dispatch<16>(F, f, h, S, D, C, mixed, s2));
  }
  stage_begin(h, QBX_STAGE_P2P, s2);
  if (f->n_utgt > 0 && (S || D)) {
    const unsigned gw = nblk(f->n_utgt, kThreads / 32);  // one warp per target
#define P2P_LAUNCH(A, B)                                                                      \
    do {                                                                                       \
      if (mixed)                                                                               \
        p2p_warp_kernel<A, B, true><<<gw, kThreads, 0, s2>>>(F, f->utgt.ptr, f->tleaf.ptr,     \
                                                             f->n_utgt, out);                  \
      else                                                                                     \
        p2p_warp_kernel<A, B, false><<<gw, kThreads, 0, s2>>>(F, f->utgt.ptr, f->tleaf.ptr,    \
                                                              f->n_utgt, out);                 \
    } while (0)
    if (S && D) P2P_LAUNCH(true, true);
    else if (S) P2P_LAUNCH(true, false);
    else P2P_LAUNCH(false, true);
#undef P2P_LAUNCH
    QBX_KCHECK("p2p", s2);
    h->launches += 1;
  }
  stage_end(h, QBX_STAGE_P2P, s2);
  // ---- main: upward pass
  stage_begin(h, QBX_STAGE_P2M, s);
  if ((S || D) && f->n_p2m_items > 0) {
    if (mixed) {
      p2m_item_mixed_kernel<<<f->n_p2m_items, kThreads, f->p2m_sm, s>>>(
          F, f->p2m_items.ptr, f->p2m_segleaf.ptr, f->p2m_segrow.ptr, f->p2m_segpoff.ptr,
          f->p2m_src.ptr, f->p2m_srcleaf.ptr, f->p2m_part.ptr, (unsigned)f->p2m_sm);
      QBX_KCHECK("p2m", s);
      p2m_sum_mixed_kernel<<<f->n_src_leaves, kThreads, 0, s>>>(
          F, f->src_leaves.ptr, f->p2m_lseg.ptr, f->p2m_segpoff.ptr, f->p2m_part.ptr);
    } else {
      p2m_item_kernel<<<f->n_p2m_items, kThreads, f->p2m_sm, s>>>(
          F, f->p2m_items.ptr, f->p2m_segleaf.ptr, f->p2m_segrow.ptr, f->p2m_segpoff.ptr,
          f->p2m_src.ptr, f->p2m_srcleaf.ptr, f->p2m_part.ptr, (unsigned)f->p2m_sm);
      QBX_KCHECK("p2m", s);
      p2m_sum_kernel<<<f->n_src_leaves, kThreads, 0, s>>>(F, f->src_leaves.ptr, f->p2m_lseg.ptr,
                                                         f->p2m_segpoff.ptr, f->p2m_part.ptr);
    }
    QBX_KCHECK("p2m_sum", s);
    h->launches += 2;
  }
  stage_end(h, QBX_STAGE_P2M, s);
  stage_begin(h, QBX_STAGE_M2M, s);
  if (mixed) {
    TRY(launch_m2m_f32(h, f, s));
  } else {
    for (int l = f->n_levels - 2; l >= 2; --l) {
      const int nb = f->nonleaf_off[l + 1] - f->nonleaf_off[l];
      if (nb == 0) continue;
      bool done = false;  // tensor cores where the level's split is exact
      TRY(launch_mml_tc(h, f, 0, l, &done, s));
      if (done) {
        QBX_KCHECK("m2m_tc", s);
        continue;
      }
      m2m_kernel<<<nb, kThreads, m2m_smem(pb[l], pb[l + 1]), s>>>(F, f->nonleaf.ptr + f->nonleaf_off[l]);
      QBX_KCHECK("m2m", s);
      h->launches += 1;
    }
  }
  stage_end(h, QBX_STAGE_M2M, s);
  TRY(signal(f->ev_m2m, s));
  // ---- side: W-list stages (need the multipoles)
  TRY(wait(s2, f->ev_m2m));
  if (h->n_ctr > 0) {
    cd* alpha = h->alpha.ptr;
    if (h->p <= 4) TRY(launch_m2qbxl<4>(F, f, h, S, D, C, alpha, mixed, s2));
    else if (h->p <= 8) TRY(launch_m2qbxl<8>(F, f, h, S, D, C, alpha, mixed, s2));
    else if (h->p <= 12) TRY(launch_m2qbxl<12>(F, f, h, S, D, C, alpha, mixed, s2));
    else TRY(launch_m2qbxl<16>(F, f, h, S, D, C, alpha, mixed, s2));
  }
  stage_begin(h, QBX_STAGE_M2P, s2);
  if (f->n_wtgt > 0 && f->n_m2p_pairs > 0) {
    if (mixed) {
      mpole_f32_list_kernel<<<f->n_m2p_wbox, kThreads, 0, s2>>>(
          F, f->m2p_wbox.ptr, f->conv.ptr, f->m2p_t.ptr, f->m2p_scaled.ptr, f->m2p_mu.ptr);
      QBX_KCHECK("m2p_mu", s2);
      m2p_pair_mixed_kernel<<<nblk(f->n_m2p_pairs, kThreads), kThreads, 0, s2>>>(
          F, f->m2p_tgt.ptr, f->m2p_box.ptr, f->n_m2p_pairs, f->m2p_mu.ptr, f->m2p_rec.ptr,
          f->m2p_t.ptr, f->m2p_scaled.ptr, f->m2p_part.ptr);
      h->launches += 1;
    } else {
      m2p_pair_kernel<<<nblk(f->n_m2p_pairs, kThreads), kThreads, 0, s2>>>(
          F, f->m2p_tgt.ptr, f->m2p_box.ptr, f->n_m2p_pairs, f->m2p_part.ptr);
    }
    QBX_KCHECK("m2p", s2);
    m2p_sum_kernel<<<nblk(f->n_wtgt, kThreads), kThreads, 0, s2>>>(
        f->n_wtgt, f->wtgt.ptr, f->m2p_off.ptr, f->m2p_part.ptr, f->perm[PT_TGT].ptr, out);
    QBX_KCHECK("m2p_sum", s2);
    h->launches += 2;
  }
  stage_end(h, QBX_STAGE_M2P, s2);
  TRY(signal(f->ev_out, s2));
  // ---- main: downward pass (M2L after P2L has added into the locals)
  TRY(wait(s, f->ev_p2l));
  stage_begin(h, QBX_STAGE_M2L, s);
  // tensor cores for the FP64 path; the mixed path keeps the FP32 CUDA-core
  // tile GEMM (faster on every measured workload) unless engine 1 asks for them
  if (f->tc_any && (!mixed || h->m2l_engine == 1)) {
    TRY(launch_m2l_tc(h, f, mixed, s));
  } else if (mixed) {
    TRY(launch_m2l_f32(h, f, s));
  } else {
    TRY(launch_m2l_f64(h, f, s));
  }
  stage_end(h, QBX_STAGE_M2L, s);
  stage_begin(h, QBX_STAGE_L2L, s);
  if (mixed) {
    TRY(launch_l2l_f32(h, f, s));
  } else {
    for (int l = 2; l + 1 < f->n_levels; ++l) {
      const int nb = f->nonleaf_off[l + 1] - f->nonleaf_off[l];
      if (nb == 0) continue;
      bool done = false;  // tensor cores where the level's split is exact
      TRY(launch_mml_tc(h, f, 1, l, &done, s));
      if (done) {
        QBX_KCHECK("l2l_tc", s);
        continue;
      }
      l2l_kernel<<<nb, kThreads, l2l_smem(pb[l], pb[l + 1]), s>>>(F, f->nonleaf.ptr + f->nonleaf_off[l]);
      QBX_KCHECK("l2l", s);
      h->launches += 1;
    }
  }
  if (f->n_leaves > 0) {
    unscale_leaf_locals_kernel<<<f->n_leaves, kThreads, 0, s>>>(F, f->leaves.ptr);
    QBX_KCHECK("unscale_leaf_locals", s);
    h->launches += 1;
  }
  stage_end(h, QBX_STAGE_L2L, s);
  // ---- main: L2P (out, after M2P), then L2QBXL (alpha, after the side stream)
  TRY(signal(f->ev_join, s2));
  TRY(wait(s, f->ev_out));
  if (f->n_dtgt > 0) {
    stage_begin(h, QBX_STAGE_L2P, s);
    l2p_kernel<<<nblk(f->n_dtgt, kThreads), kThreads, 0, s>>>(F, f->dtgt.ptr, f->tleaf.ptr, f->n_dtgt, out);
    QBX_KCHECK("l2p", s);
    stage_end(h, QBX_STAGE_L2P, s);
    h->launches += 1;
  }
  TRY(wait(s, f->ev_join));
  if (h->n_ctr > 0) {
    cd* alpha = h->alpha.ptr;
    TRY(launch_l2qbxl(F, f, h, C, alpha, mixed, s));
  }
  QBX_CUDA_TRY(cudaGetLastError());
  return QBX_OK;
}

void fmm_plan_free(FmmPlan* f) { delete f; }

extern "C" qbx_status qbx_export_tree(const qbx_handle* h, int64_t* info, double* root,
                                      int32_t* box_level, int32_t* box_ij, int32_t* box_child,
                                      int32_t* box_range, int32_t* lists_off,
                                      int32_t* lists_idx, int32_t* perm_src, int32_t* perm_ctr,
                                      int32_t* perm_tgt) {
  if (!h) { set_error("qbx_export_tree: NULL handle"); return QBX_ERR_ARG; }
  const FmmPlan* f = h->fmm;
  if (!f || !h->planned || h->mode != QBX_FMM) {
    set_error("qbx_export_tree: no FMM plan (call qbx_tree_build with QBX_FMM)");
    return QBX_ERR_STATE;
  }
  const int nb = f->n_boxes;
  if (info) {
    info[0] = nb; info[1] = f->n_levels; info[2] = f->U.nnz; info[3] = f->V.nnz;
    info[4] = f->W.nnz; info[5] = f->X.nnz; info[6] = f->pb_fine; info[7] = f->n_leaves;
  }
  if (root) { root[0] = f->x0; root[1] = f->y0; root[2] = f->side; }
  if (box_level) QBX_CUDA_TRY(cudaMemcpy(box_level, f->box.level.ptr, nb * 4, cudaMemcpyDeviceToHost));
  if (box_ij) QBX_CUDA_TRY(cudaMemcpy(box_ij, f->box.ij.ptr, nb * 8, cudaMemcpyDeviceToHost));
  if (box_child) QBX_CUDA_TRY(cudaMemcpy(box_child, f->box.child.ptr, (size_t)nb * 16, cudaMemcpyDeviceToHost));
  if (box_range) {
    std::vector<int2> r(nb);
    for (int t = 0; t < PT_COUNT; ++t) {
      QBX_CUDA_TRY(cudaMemcpy(r.data(), f->box.rng[t].ptr, (size_t)nb * 8, cudaMemcpyDeviceToHost));
      for (int b = 0; b < nb; ++b) {
        box_range[(size_t)b * 8 + 2 * t] = r[b].x;
        box_range[(size_t)b * 8 + 2 * t + 1] = r[b].y;
      }
    }
  }
  const Csr* L[4] = {&f->U, &f->V, &f->W, &f->X};
  size_t pos = 0;
  for (int i = 0; i < 4; ++i) {
    if (lists_off)
      QBX_CUDA_TRY(cudaMemcpy(lists_off + (size_t)i * (nb + 1), L[i]->off.ptr, (nb + 1) * 4,
                              cudaMemcpyDeviceToHost));
    if (lists_idx && L[i]->nnz)
      QBX_CUDA_TRY(cudaMemcpy(lists_idx + pos, L[i]->idx.ptr, L[i]->nnz * 4, cudaMemcpyDeviceToHost));
    pos += L[i]->nnz;
  }
  if (perm_src && h->n_src) QBX_CUDA_TRY(cudaMemcpy(perm_src, f->perm[PT_SRC].ptr, h->n_src * 4, cudaMemcpyDeviceToHost));
  if (perm_ctr && h->n_ctr) QBX_CUDA_TRY(cudaMemcpy(perm_ctr, f->perm[PT_CTR].ptr, h->n_ctr * 4, cudaMemcpyDeviceToHost));
  if (perm_tgt && h->n_tgt) QBX_CUDA_TRY(cudaMemcpy(perm_tgt, f->perm[PT_TGT].ptr, h->n_tgt * 4, cudaMemcpyDeviceToHost));
  return QBX_OK;
}

extern "C" qbx_status qbx_get_box_orders(const qbx_handle* h, int32_t* pb_out, int32_t n) {
  if (!h || !pb_out || n < 0) { set_error("qbx_get_box_orders: bad arguments"); return QBX_ERR_ARG; }
  const FmmPlan* f = h->fmm;
  if (!f || !h->planned || h->mode != QBX_FMM) {
    set_error("qbx_get_box_orders: no FMM plan (call qbx_tree_build with QBX_FMM)");
    return QBX_ERR_STATE;
  }
  for (int l = 0; l < n; ++l) pb_out[l] = l < f->n_levels ? f->h_pb[l] : 0;
  return QBX_OK;
}
