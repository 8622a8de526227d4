// Mixed-precision kernels (QBX_MIXED): the M2M translation of Stage 2, the M2L
// translation of Stage 4 and the L2L translation of Stage 7 in complex FP32
// with compensated (Kahan) accumulation.
//
// FP32 cannot hold the power-scaled expansions of the FP64 path (their
// translation entries still grow like a factorial), so the FP32 operators act
// on sigma-normalised coefficients
//     mu_n = a_n / sig_|n|,   lam_l = gamma_l sig_|l|,
//     sig_j = min(1, (x/2)^j / j!),  x = k * side  (the size of J_j at a box),
// for which every M2L entry sig_l sig_n (-1)^l W_{n+l}(D) is of order one or
// smaller, and so is every L2L entry (sig'_s / sig_n) (-1)^{s-n} V_{s-n}(d)
// (sig' of the child level) and M2M entry (sig_n / sig'_s) conj(V_{s-n}(d))
// (sig' of the parent level): the scale ratios are binomial-sized while
// J_{s-n}(k d) decays factorially. The entries are computed in FP64 (through logarithms
// of the scale factors) and stored as FP32 matrices, one per (level, offset
// class) for M2L and per (level, quadrant) for L2L; the coefficient
// conversions between the two normalisations are FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tree.cuh"
#include "m2l_entry.cuh"

namespace {

constexpr int kT = 128;

inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

// per level: lsig[j] = log sig_j, conv[j] = s^j / sig_j  (j = 0..pb_l; stride
// pbmax + 1), isig[j] = 1 / sig_min(j, pb_l) (j = 0..pb_l + 1; stride pbmax + 2)
__global__ void sigma_tables_kernel(int n_levels, int pbmax, const int* __restrict__ lpb,
                                    double k, double side, const double* __restrict__ scale,
                                    double* __restrict__ lsig, double* __restrict__ conv,
                                    double* __restrict__ isig) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_levels) return;
  const double x = k * side / (double)(1 << l);
  const double ls = log(scale[l]);
  double v = 0.0;
  for (int j = 0; j <= lpb[l]; ++j) {
    v = fmin(0.0, j * log(0.5 * x) - lgamma((double)j + 1.0));
    lsig[(size_t)l * (pbmax + 1) + j] = v;
    conv[(size_t)l * (pbmax + 1) + j] = exp(j * ls - v);
    isig[(size_t)l * (pbmax + 2) + j] = exp(-v);
  }
  isig[(size_t)l * (pbmax + 2) + lpb[l] + 1] = exp(-v);
}

// Recurrence factors of G_m = sig_m H_m on level l (mixed M2P and P2L):
// rec[m] = (2m sig_{m+1} / sig_m, sig_{m+1} / sig_{m-1}) for 1 <= m < pb_l,
// rec[0] = (sig_1, 0), and rec[pb_l] with sig_{pb+1} taken as sig_pb.
__global__ void m2p_rec_kernel(int n_levels, int pbmax, const int* __restrict__ lpb,
                               const double* __restrict__ lsig, double2* __restrict__ rec) {
  const int l = blockIdx.x;
  if (l >= n_levels) return;
  const double* sg = lsig + (size_t)l * (pbmax + 1);
  double2* r = rec + (size_t)l * (pbmax + 2);
  const int pb = lpb[l];
  for (int m = threadIdx.x; m <= pbmax + 1; m += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (m == 0 && pb >= 1) v.x = exp(sg[1]);
    if (m >= 1 && m < pb)
      v = make_double2(2.0 * m * exp(sg[m + 1] - sg[m]), exp(sg[m + 1] - sg[m - 1]));
    // one order beyond pb, normalised by sig_pb (mixed P2L's dipole terms)
    if (m == pb && pb >= 1) v = make_double2(2.0 * m, exp(sg[m] - sg[m - 1]));
    r[m] = v;
  }
}

// t[l][m] = round(log2 sig_m) of level l: the power of two that M2P moves from
// the multipole to the Hankel value (exponent offsets, no arithmetic)
__global__ void m2p_t_kernel(int n_levels, int pbmax, const int* __restrict__ lpb,
                             const double* __restrict__ lsig, int* __restrict__ t) {
  const int l = blockIdx.x;
  if (l >= n_levels) return;
  const double* sg = lsig + (size_t)l * (pbmax + 1);
  for (int m = threadIdx.x; m <= pbmax + 1; m += blockDim.x)
    t[(size_t)l * (pbmax + 2) + m] = m <= lpb[l] ? (int)lrint(sg[m] * 1.4426950408889634) : 0;
}

// r[l][m] = (sig_{m-1} / sig_m, sig_{m+1} / sig_m) of level l, 1 where the
// neighbour order is outside 0..pb (the mixed P2M's dipole terms)
__global__ void sig_ratio_kernel(int n_levels, int pbmax, const int* __restrict__ lpb,
                                 const double* __restrict__ lsig, double2* __restrict__ r) {
  const int l = blockIdx.x;
  if (l >= n_levels) return;
  const double* sg = lsig + (size_t)l * (pbmax + 1);
  const int pb = lpb[l];
  for (int m = threadIdx.x; m <= pbmax + 1; m += blockDim.x) {
    double2 v = make_double2(1.0, 1.0);
    if (m <= pb) {
      if (m >= 1) v.x = exp(sg[m - 1] - sg[m]);
      else v.x = exp(sg[1 <= pb ? 1 : 0] - sg[0]);  // |0 - 1| = 1
      if (m + 1 <= pb) v.y = exp(sg[m + 1] - sg[m]);
    }
    r[(size_t)l * (pbmax + 2) + m] = v;
  }
}

// Level l's matrices Tm[cls][n][lo] = sig_lo sig_n (-1)^lo W_{n+lo}(D) (orders
// up to pb = pb_l; M2lNorm), stored in FP32. Grid: (cls, n), threads over lo.
__global__ void m2l_f32_matrix_kernel(int l, int pb, int pbmax, const cd* __restrict__ t_m2l,
                                      const double* __restrict__ scale,
                                      const double* __restrict__ lsig, float2* __restrict__ Tm) {
  const int cls = blockIdx.x;
  const int n = (int)blockIdx.y - pb;
  const int Q = 2 * pb + 1;
  const M2lNorm nm(t_m2l, scale, lsig, l, cls, pbmax);
  float2* dst = Tm + ((size_t)cls * Q + (n + pb)) * Q;
  for (int lo = (int)threadIdx.x - pb; lo <= pb; lo += blockDim.x) {
    const cd v = nm.entry(n, lo);
    dst[lo + pb] = make_float2((float)v.x, (float)v.y);
  }
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// M2L as batched complex GEMMs. The V-list pairs (target box b, source box c)
// are grouped by (level, offset class) at plan time; all pairs of a group use
// the same matrix Tm[cls]. A CTA takes kGemmRows pairs of one group: their
// sigma-normalised source coefficients mu (FP32) go to shared memory ([n][row],
// n-major), and each thread computes one output order lo for all the rows,
// streaming matrix row n once for all of them (so the matrix is read once per
// kGemmRows pairs instead of once per pair). Sums: plain FP32 FMAs over blocks
// of kGemmBlock terms, blocks added with Kahan compensation. Each pair's result
// goes to its row of Y (FP32); m2l_f32_reduce_kernel adds each target box's
// rows in its V-list order with Kahan compensation (deterministic).
constexpr int kGemmRows = 16;
constexpr int kGemmBlock = 8;
// M2M / L2L levels with fewer parents than kWideLevel use tiles of kNarrowRows
// parents, so that the launch still spreads over the SMs.
constexpr int kNarrowRows = 4;
constexpr int kWideLevel = kGemmRows * 2 * 152;

// Staged rows: x[n * stage_stride(R) + r]. Two float2 of padding per n keep
// the row pairs 16-byte aligned and spread the staging stores over the banks.
__host__ __device__ constexpr int stage_stride(int R) { return R + 2; }

// One block of nj (1 <= nj <= kGemmBlock) terms of a tile product column:
// (tr, ti)[r] = sum_{j < nj} tb[j] * x[j * RS + r], started from the first term.
template <int R>
__device__ __forceinline__ void gemm_block(const float2 (&tb)[kGemmBlock], int nj,
                                           const float2* __restrict__ x, float (&tr)[R],
                                           float (&ti)[R]) {
  static_assert(R % 2 == 0, "rows are read in pairs");
  constexpr int RS = stage_stride(R);
#pragma unroll
  for (int j = 0; j < kGemmBlock; ++j) {
    if (j < nj) {
      const float2 t = tb[j];
      const float4* m = reinterpret_cast<const float4*>(x + j * RS);
#pragma unroll
      for (int r2 = 0; r2 < R / 2; ++r2) {
        const float4 v = m[r2];  // rows 2 r2 (x, y) and 2 r2 + 1 (z, w)
        if (j == 0) {
          tr[2 * r2] = fmaf(t.x, v.x, -t.y * v.y);
          ti[2 * r2] = fmaf(t.x, v.y, t.y * v.x);
          tr[2 * r2 + 1] = fmaf(t.x, v.z, -t.y * v.w);
          ti[2 * r2 + 1] = fmaf(t.x, v.w, t.y * v.z);
        } else {
          tr[2 * r2] = fmaf(t.x, v.x, fmaf(-t.y, v.y, tr[2 * r2]));
          ti[2 * r2] = fmaf(t.x, v.y, fmaf(t.y, v.x, ti[2 * r2]));
          tr[2 * r2 + 1] = fmaf(t.x, v.z, fmaf(-t.y, v.w, tr[2 * r2 + 1]));
          ti[2 * r2 + 1] = fmaf(t.x, v.w, fmaf(t.y, v.z, ti[2 * r2 + 1]));
        }
      }
    }
  }
}

template <int R>
__device__ __forceinline__ void gemm_block_add(const float2 (&tb)[kGemmBlock], int nj,
                                               const float2* __restrict__ x, float (&sr)[R],
                                               float (&si)[R], float (&cr)[R], float (&ci)[R]) {
  float tr[R], ti[R];
  gemm_block<R>(tb, nj, x, tr, ti);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    kahan_add(sr[r], cr[r], tr[r]);
    kahan_add(si[r], ci[r], ti[r]);
  }
}

// One output column lo of a tile product: for every row r < R,
// (sr, si)[r] += sum_{n < N} M[n * ld + lo] * x[n * RS + r], with x in
// shared memory (16-byte aligned, RS = stage_stride(R)). Plain FP32 FMAs over
// blocks of kGemmBlock terms (whose matrix entries are loaded one block ahead,
// into two alternating register sets), the blocks added with Kahan
// compensation (cr, ci). Threads with act == false read column 0 and their
// sums are not used.
template <int R = kGemmRows>
__device__ __forceinline__ void tile_gemm_column(const float2* __restrict__ M, size_t ld, int N,
                                                 const float2* __restrict__ x, int lo, bool act,
                                                 float (&sr)[R], float (&si)[R], float (&cr)[R],
                                                 float (&ci)[R]) {
  constexpr int RS = stage_stride(R);
  const float2* Mc = M + (act ? lo : 0);
  const int nfull = N - N % kGemmBlock;
  float2 ba[kGemmBlock], bb[kGemmBlock];
  if (nfull > 0) {
#pragma unroll
    for (int j = 0; j < kGemmBlock; ++j) ba[j] = Mc[(size_t)j * ld];
  }
  for (int n0 = 0; n0 < nfull; n0 += 2 * kGemmBlock) {
    const int n1 = n0 + kGemmBlock;
    if (n1 < nfull) {
#pragma unroll
      for (int j = 0; j < kGemmBlock; ++j) bb[j] = Mc[(size_t)(n1 + j) * ld];
    }
    gemm_block_add<R>(ba, kGemmBlock, x + n0 * RS, sr, si, cr, ci);
    if (n1 >= nfull) break;
    if (n1 + kGemmBlock < nfull) {
#pragma unroll
      for (int j = 0; j < kGemmBlock; ++j) ba[j] = Mc[(size_t)(n1 + kGemmBlock + j) * ld];
    }
    gemm_block_add<R>(bb, kGemmBlock, x + n1 * RS, sr, si, cr, ci);
  }
  if (nfull < N) {  // the last, partial block
    const int nj = N - nfull;
#pragma unroll
    for (int j = 0; j < kGemmBlock; ++j)
      ba[j] = j < nj ? Mc[(size_t)(nfull + j) * ld] : make_float2(0.f, 0.f);
    gemm_block_add<R>(ba, nj, x + nfull * RS, sr, si, cr, ci);
  }
}

// mu32 = mh * conv (sigma-normalised multipoles in FP32), once per box that
// is a V-list source; the GEMM tiles gather these rows.
__global__ void __launch_bounds__(kT) mpole_to_f32_kernel(
    int pbmax, const int* __restrict__ boxes, const int* __restrict__ level,
    const int* __restrict__ lpb, const long long* __restrict__ eoff,
    const double* __restrict__ conv, const cd* __restrict__ mpole, float2* __restrict__ mu32) {
  const int b = boxes[blockIdx.x];
  const int l = level[b];
  const int pb = lpb[l], Q = 2 * pb + 1;
  const double* cv = conv + (size_t)l * (pbmax + 1);
  const cd* a = mpole + eoff[b];
  float2* dst = mu32 + eoff[b];
  for (int n = threadIdx.x; n < Q; n += kT) {
    const double f = cv[abs(n - pb)];
    dst[n] = make_float2((float)(a[n].x * f), (float)(a[n].y * f));
  }
}

// M2L work items: (first row, rows, first output order, group) over the tiles
// of kGemmRows rows of one group. Each CTA computes kT consecutive output
// orders (one per thread) of its rows and
// stages the source rows through shared memory kChunkK orders at a time, so
// its footprint does not grow with the box order. kChunkK is a multiple of
// kGemmBlock: the compensated blocks, and so the result bits, do not depend on
// the staging.
constexpr int kChunkK = 128;
static_assert(kChunkK % kGemmBlock == 0, "staging must keep the summation blocks");

// (four CTAs per SM: 128 registers, a few spilled; 2 % faster than three)
__global__ void __launch_bounds__(kT, 4) m2l_f32_gemm_kernel(
    const int4* __restrict__ items, const int* __restrict__ lpb,
    const long long* __restrict__ goff, const long long* __restrict__ row_off,
    const float2* __restrict__ mu32, const float2* __restrict__ tm,
    const long long* __restrict__ yoff, float2* __restrict__ Y) {
  constexpr int RS = stage_stride(kGemmRows);
  __shared__ __align__(16) float2 mu[kChunkK * RS];  // [n][row]
  const int4 I = items[blockIdx.x];  // (first row, rows, first output order, group)
  const int row0 = I.x, nr = I.y;
  const int Q = 2 * lpb[I.w / 49] + 1;
  const int lo = I.z + (int)threadIdx.x;
  const bool act = lo < Q;
  // warps past the last output order only help stage the sources: an FMA
  // costs its warp the same however few lanes are active
  const bool warp_act = I.z + (int)(threadIdx.x & ~31u) < Q;
  const float2* M = tm + goff[I.w];
  float sr[kGemmRows], si[kGemmRows], cr[kGemmRows], ci[kGemmRows];
#pragma unroll
  for (int r = 0; r < kGemmRows; ++r) sr[r] = si[r] = cr[r] = ci[r] = 0.f;
  for (int n0 = 0; n0 < Q; n0 += kChunkK) {
    const int nk = min(kChunkK, Q - n0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nk * (kGemmRows / 2); idx += kT) {
      const int r = 2 * (idx / nk), n = idx % nk;  // coalesced reads along each source row
      const float2 a = r < nr ? mu32[row_off[row0 + r] + n0 + n] : make_float2(0.f, 0.f);
      const float2 b = r + 1 < nr ? mu32[row_off[row0 + r + 1] + n0 + n] : make_float2(0.f, 0.f);
      *reinterpret_cast<float4*>(mu + n * RS + r) = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    if (warp_act) tile_gemm_column(M + (size_t)n0 * Q, Q, nk, mu, lo, act, sr, si, cr, ci);
  }
  if (act) {
#pragma unroll
    for (int r = 0; r < kGemmRows; ++r)
      if (r < nr) Y[yoff[row0 + r] + lo] = make_float2(sr[r] - cr[r], si[r] - ci[r]);
  }
}

// lh_lo(b) += conv_lo * sum over b's V entries e (in list order) of Y[row(e)][lo]:
// FP32 sums with Kahan compensation (FP32 arithmetic is cheap on this GPU, a
// conversion to FP64 per element is not), converted and scaled once in FP64.
__global__ void __launch_bounds__(kT) m2l_f32_reduce_kernel(
    int pbmax, const int* __restrict__ boxes, const int* __restrict__ level,
    const int* __restrict__ lpb, const int* __restrict__ voff, const long long* __restrict__ eyoff,
    const float2* __restrict__ Y, const double* __restrict__ conv,
    const long long* __restrict__ eoff, cd* __restrict__ local) {
  const int b = boxes[blockIdx.x];
  const int l = level[b];
  const int pb = lpb[l], Q = 2 * pb + 1;
  const double* cv = conv + (size_t)l * (pbmax + 1);
  cd* dst = local + eoff[b];
  for (int lo = threadIdx.x; lo < Q; lo += kT) {
    float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
    const int e1 = voff[b + 1];
    int e = voff[b];
    for (; e + 4 <= e1; e += 4) {  // four loads in flight, added in list order
      float2 y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) y[u] = Y[eyoff[e + u] + lo];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        kahan_add(sr, cr, y[u].x);
        kahan_add(si, ci, y[u].y);
      }
    }
    for (; e < e1; ++e) {
      const float2 y = Y[eyoff[e] + lo];
      kahan_add(sr, cr, y.x);
      kahan_add(si, ci, y.y);
    }
    const double f = cv[abs(lo - pb)];
    dst[lo] = cadd(dst[lo], mk(((double)sr - (double)cr) * f, ((double)si - (double)ci) * f));
  }
}

// ---------------------------------------------------------------- FP64 M2L as tile GEMMs
// The FP64 path's M2L, lh_l += (-1)^l sum_n What_{n+l} c(l, n) mh_n with
// What_m = s^|m| W_m(D) and c(l, n) = s^{2 min(|l|,|n|)} when l and n have
// opposite signs (else 1), written as dense matrices per (level, offset
// class): T64[cls][n][l] = (-1)^l What_{n+l} c(l, n) (FP64; the same tiles and
// ordered reduction as the FP32 M2L, without normalisation or compensation).
__global__ void m2l_f64_matrix_kernel(int l, int pb, int pbmax, const cd* __restrict__ t_m2l,
                                      const double* __restrict__ pw, cd* __restrict__ Tm) {
  const int cls = blockIdx.x;
  const int n = (int)blockIdx.y - pb;
  const int Q = 2 * pb + 1;
  const cd* w = t_m2l + ((size_t)l * 49 + cls) * (4 * pbmax + 1) + 2 * pbmax;
  const double* p2 = pw + (size_t)l * (2 * pbmax + 3);  // s^j
  cd* dst = Tm + ((size_t)cls * Q + (n + pb)) * Q;
  const int dx = cls / 7 - 3, dy = cls % 7 - 3;
  const bool used = max(abs(dx), abs(dy)) >= 2;  // V-list offsets only
  for (int lo = (int)threadIdx.x - pb; lo <= pb; lo += blockDim.x) {
    cd v = mk(0.0, 0.0);
    if (used) {
      v = w[n + lo];
      if ((n < 0 && lo > 0) || (n > 0 && lo < 0)) v = cscale(v, p2[2 * min(abs(n), abs(lo))]);
      if (lo & 1) v = mk(-v.x, -v.y);
    }
    dst[lo + pb] = v;
  }
}

// FP64 work items take kF64Rows rows of a tile (the accumulators of 16 FP64
// rows would not fit in registers), kT output orders and the same staging as
// the FP32 items. Results go to the FP64 rows of Y64, added per target box by
// m2l_f64_reduce_kernel in V-list order.
constexpr int kF64Rows = 8;
__global__ void __launch_bounds__(kT) m2l_f64_gemm_kernel(
    const int4* __restrict__ items, const int* __restrict__ lpb,
    const long long* __restrict__ goff, const long long* __restrict__ row_off,
    const cd* __restrict__ mpole, const cd* __restrict__ tm,
    const long long* __restrict__ yoff, cd* __restrict__ Y) {
  __shared__ __align__(16) cd xs[kChunkK * kF64Rows];  // [n][row]
  const int4 I = items[blockIdx.x];  // (first row, rows <= kF64Rows, first output order, group)
  const int row0 = I.x, nr = I.y;
  const int Q = 2 * lpb[I.w / 49] + 1;
  const int lo = I.z + (int)threadIdx.x;
  const bool act = lo < Q;
  const bool warp_act = I.z + (int)(threadIdx.x & ~31u) < Q;  // as in the FP32 items
  const cd* M = tm + goff[I.w];
  cd acc[kF64Rows];
#pragma unroll
  for (int r = 0; r < kF64Rows; ++r) acc[r] = mk(0.0, 0.0);
  for (int n0 = 0; n0 < Q; n0 += kChunkK) {
    const int nk = min(kChunkK, Q - n0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nk * kF64Rows; idx += kT) {
      const int r = idx / nk, n = idx % nk;
      xs[n * kF64Rows + r] = r < nr ? mpole[row_off[row0 + r] + n0 + n] : mk(0.0, 0.0);
    }
    __syncthreads();
    if (!warp_act) continue;
    for (int j0 = 0; j0 < nk; j0 += kGemmBlock) {
      cd tb[kGemmBlock];
#pragma unroll
      for (int j = 0; j < kGemmBlock; ++j)
        tb[j] = (act && j0 + j < nk) ? M[(size_t)(n0 + j0 + j) * Q + lo] : mk(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < kGemmBlock; ++j) {
        if (j0 + j >= nk) break;
        const cd* x = xs + (j0 + j) * kF64Rows;
#pragma unroll
        for (int r = 0; r < kF64Rows; ++r) cfma(acc[r], tb[j], x[r]);
      }
    }
  }
  if (act) {
#pragma unroll
    for (int r = 0; r < kF64Rows; ++r)
      if (r < nr) Y[yoff[row0 + r] + lo] = acc[r];
  }
}

// lh_lo(b) += sum over b's V entries e (in list order) of Y64[row(e)][lo].
__global__ void __launch_bounds__(kT) m2l_f64_reduce_kernel(
    const int* __restrict__ boxes, const int* __restrict__ level, const int* __restrict__ lpb,
    const int* __restrict__ voff, const long long* __restrict__ eyoff, const cd* __restrict__ Y,
    const long long* __restrict__ eoff, cd* __restrict__ local) {
  const int b = boxes[blockIdx.x];
  const int Q = 2 * lpb[level[b]] + 1;
  cd* dst = local + eoff[b];
  for (int lo = threadIdx.x; lo < Q; lo += kT) {
    cd sum = mk(0.0, 0.0);
    const int e1 = voff[b + 1];
    int e = voff[b];
    for (; e + 4 <= e1; e += 4) {  // four loads in flight, added in list order
      cd y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) y[u] = Y[eyoff[e + u] + lo];
#pragma unroll
      for (int u = 0; u < 4; ++u) sum = cadd(sum, y[u]);
    }
    for (; e < e1; ++e) sum = cadd(sum, Y[eyoff[e] + lo]);
    dst[lo] = cadd(dst[lo], sum);
  }
}

// L2L matrices of parent level l (order pp) and quadrant c, child order pc:
// Tl[c][n][s] = (sig'_s / sig_n) (-1)^{s-n} V_{s-n}(d), sig' on level l+1,
// sig on level l, from the FP64 table of (-1)^m V_m(d) (row stride
// 4 pbmax + 1, order m at m + 2 pbmax). Grid: (quadrant, n), threads over s.
__global__ void l2l_f32_matrix_kernel(int l, int pp, int pc, int pbmax, const cd* __restrict__ t_l2l,
                                      const double* __restrict__ lsig, float2* __restrict__ Tl) {
  const int c = blockIdx.x;
  const int n = (int)blockIdx.y - pp;
  const int Qp = 2 * pp + 1, Qc = 2 * pc + 1;
  const cd* v = t_l2l + ((size_t)l * 4 + c) * (4 * pbmax + 1) + 2 * pbmax;
  const double* sp = lsig + (size_t)l * (pbmax + 1);
  const double* sc = lsig + (size_t)(l + 1) * (pbmax + 1);
  float2* dst = Tl + ((size_t)c * Qp + (n + pp)) * Qc;
  for (int so = (int)threadIdx.x - pc; so <= pc; so += blockDim.x) {
    const cd e = v[so - n];
    const double mag = hypot(e.x, e.y);
    float2 out = make_float2(0.f, 0.f);
    if (mag > 0.0) {
      const double lf = sc[abs(so)] - sp[abs(n)] + log(mag);
      const double f = lf < -700.0 ? 0.0 : exp(lf) / mag;
      out = make_float2((float)(e.x * f), (float)(e.y * f));
    }
    dst[so + pc] = out;
  }
}

// L2L on level l as tile GEMMs: a CTA takes R parents, one child quadrant
// c = blockIdx.y and kT child orders (chunk blockIdx.z), stages the parents' sigma-normalised locals
// lambda_n = lh_n / conv_n (FP32) in shared memory, and computes
// lambda'_s = sum_n Tl[c][n][s] lambda_n for all of them at once (threads over
// s); the quadrant-c children get lh'_s += lambda'_s conv'_s in FP64.
template <int R>
__global__ void __launch_bounds__(kT) l2l_f32_kernel(
    int l, int pp, int pc, int pbmax, const int* __restrict__ parents, int nb,
    const int* __restrict__ child, const long long* __restrict__ eoff,
    const float2* __restrict__ Tl, const double* __restrict__ conv, cd* __restrict__ local) {
  extern __shared__ __align__(16) float2 lam[];  // [Qp][stage_stride(R)]
  const int Qp = 2 * pp + 1, Qc = 2 * pc + 1;
  const int p0 = blockIdx.x * R, nr = min(R, nb - p0);
  const double* cvp = conv + (size_t)l * (pbmax + 1);
  const double* cvc = conv + (size_t)(l + 1) * (pbmax + 1);
  for (int idx = threadIdx.x; idx < Qp * R; idx += kT) {
    const int r = idx / Qp, n = idx % Qp;
    float2 v = make_float2(0.f, 0.f);
    if (r < nr) {
      const cd g = local[eoff[parents[p0 + r]] + n];
      const double f = 1.0 / cvp[abs(n - pp)];
      v = make_float2((float)(g.x * f), (float)(g.y * f));
    }
    lam[n * stage_stride(R) + r] = v;
  }
  __syncthreads();
  {
    const int c = blockIdx.y;
    const float2* M = Tl + (size_t)c * Qp * Qc;
    {
      const int so = (int)blockIdx.z * kT + threadIdx.x;  // output chunk blockIdx.z
      const bool act = so < Qc;
      float sr[R], si[R], cr[R], ci[R];
#pragma unroll
      for (int r = 0; r < R; ++r) sr[r] = si[r] = cr[r] = ci[r] = 0.f;
      tile_gemm_column<R>(M, Qc, Qp, lam, so, act, sr, si, cr, ci);
      if (act) {
        const double f = cvc[abs(so - pc)];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r >= nr) break;
          const int d = child[4 * parents[p0 + r] + c];
          if (d < 0) continue;
          cd* dl = local + eoff[d] + so;
          dl->x += ((double)sr[r] - (double)cr[r]) * f;
          dl->y += ((double)si[r] - (double)ci[r]) * f;
        }
      }
    }
  }
}

// M2M matrices of parent level l (order pp) and quadrant c, child order pc:
// Tm2m[c][n][s] = (sig_n / sig'_s) conj(V_{s-n}(d)), sig on the child level
// l+1, sig' on level l, from the FP64 table of conj(V_m(d)). Grid: (quadrant,
// n), threads over s.
__global__ void m2m_f32_matrix_kernel(int l, int pp, int pc, int pbmax, const cd* __restrict__ t_m2m,
                                      const double* __restrict__ lsig, float2* __restrict__ Tmm) {
  const int c = blockIdx.x;
  const int n = (int)blockIdx.y - pc;
  const int Qp = 2 * pp + 1, Qc = 2 * pc + 1;
  const cd* v = t_m2m + ((size_t)l * 4 + c) * (4 * pbmax + 1) + 2 * pbmax;
  const double* sp = lsig + (size_t)l * (pbmax + 1);
  const double* sc = lsig + (size_t)(l + 1) * (pbmax + 1);
  float2* dst = Tmm + ((size_t)c * Qc + (n + pc)) * Qp;
  for (int so = (int)threadIdx.x - pp; so <= pp; so += blockDim.x) {
    const cd e = v[so - n];
    const double mag = hypot(e.x, e.y);
    float2 out = make_float2(0.f, 0.f);
    if (mag > 0.0) {
      const double lf = sc[abs(n)] - sp[abs(so)] + log(mag);
      const double f = lf < -700.0 ? 0.0 : exp(lf) / mag;
      out = make_float2((float)(e.x * f), (float)(e.y * f));
    }
    dst[so + pp] = out;
  }
}

// M2M on level l as tile GEMMs: a CTA takes R parents and kT output orders
// (chunk blockIdx.y, so that the few wide boxes of coarse levels spread over
// many CTAs); for each quadrant it stages the children's sigma-normalised
// multipoles mu_n = mh_n conv_n (FP32) and adds sum_n Tm2m[c][n][s] mu_n to the
// parents' compensated sums (threads over s); mh'_s = mu'_s / conv'_s in FP64.
template <int R>
__global__ void __launch_bounds__(kT) m2m_f32_kernel(
    int l, int pp, int pc, int pbmax, const int* __restrict__ parents, int nb,
    const int* __restrict__ child, const long long* __restrict__ eoff,
    const float2* __restrict__ Tmm, const double* __restrict__ conv, cd* __restrict__ mpole) {
  extern __shared__ __align__(16) float2 mus[];  // [Qc][stage_stride(R)]
  __shared__ long long coff[4][R], poff[R];       // children's (-1: none) and parents' offsets
  const int Qp = 2 * pp + 1, Qc = 2 * pc + 1;
  const int p0 = blockIdx.x * R, nr = min(R, nb - p0);
  const double* cvp = conv + (size_t)l * (pbmax + 1);
  const double* cvc = conv + (size_t)(l + 1) * (pbmax + 1);
  for (int idx = threadIdx.x; idx < 5 * R; idx += kT) {
    const int r = idx % R, c = idx / R;
    long long o = -1;
    if (r < nr) {
      if (c == 4) {
        o = eoff[parents[p0 + r]];
      } else {
        const int d = child[4 * parents[p0 + r] + c];
        if (d >= 0) o = eoff[d];
      }
    }
    if (c == 4) poff[r] = o; else coff[c][r] = o;
  }
  {
    const int so = (int)blockIdx.y * kT + threadIdx.x;  // output chunk blockIdx.y
    const bool act = so < Qp;
    float sr[R], si[R], cr[R], ci[R];
#pragma unroll
    for (int r = 0; r < R; ++r) sr[r] = si[r] = cr[r] = ci[r] = 0.f;
    for (int c = 0; c < 4; ++c) {
      __syncthreads();
      for (int idx = threadIdx.x; idx < Qc * R; idx += kT) {
        const int r = idx / Qc, n = idx % Qc;
        float2 v = make_float2(0.f, 0.f);
        const long long o = coff[c][r];
        if (o >= 0) {
          const cd a = mpole[o + n];
          const double f = cvc[abs(n - pc)];
          v = make_float2((float)(a.x * f), (float)(a.y * f));
        }
        mus[n * stage_stride(R) + r] = v;
      }
      __syncthreads();
      tile_gemm_column<R>(Tmm + (size_t)c * Qc * Qp, Qp, Qc, mus, so, act, sr, si, cr, ci);
    }
    if (act) {
      const double f = 1.0 / cvp[abs(so - pp)];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r >= nr) break;
        cd* dst = mpole + poff[r] + so;
        dst->x = ((double)sr[r] - (double)cr[r]) * f;
        dst->y = ((double)si[r] - (double)ci[r]) * f;
      }
    }
  }
}

// Coarse levels (few parents, high orders) as split-K tile GEMMs: the two
// kernels above give each thread one output column and the whole K range, so
// a level of a few dozen boxes runs a few CTAs with K-long dependent chains.
// Here a CTA of kT threads takes R parents and 32 output orders (chunk
// blockIdx.y or blockIdx.z); warp w sums its quarter of K (M2M: child quadrant
// w; L2L: the w-th quarter of the parent's orders) for the 32 orders, and the
// four partial sums are added in FP64 in warp order (deterministic).
constexpr int kSplitCols = 32, kSplitWarps = kT / 32;

template <int R>
__device__ __forceinline__ void split_reduce(float (&sr)[R], float (&si)[R], float (&cr)[R],
                                             float (&ci)[R], float2* red, int warp, int lane,
                                             double (&outr)[R], double (&outi)[R]) {
  // red: [kSplitWarps][R][32]
#pragma unroll
  for (int r = 0; r < R; ++r)
    red[(warp * R + r) * 32 + lane] = make_float2(sr[r] - cr[r], si[r] - ci[r]);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kSplitWarps; ++w) {
      const float2 v = red[(w * R + r) * 32 + lane];
      a += (double)v.x;
      b += (double)v.y;
    }
    outr[r] = a;
    outi[r] = b;
  }
}

template <int R>
__global__ void __launch_bounds__(kT) m2m_f32_split_kernel(
    int l, int pp, int pc, int pbmax, const int* __restrict__ parents, int nb,
    const int* __restrict__ child, const long long* __restrict__ eoff,
    const float2* __restrict__ Tmm, const double* __restrict__ conv, cd* __restrict__ mpole) {
  extern __shared__ __align__(16) float2 mus4[];  // [4][Qc][stage_stride(R)], then red
  __shared__ long long coff[4][R], poff[R];
  const int Qp = 2 * pp + 1, Qc = 2 * pc + 1;
  const int RS = stage_stride(R);
  const int p0 = blockIdx.x * R, nr = min(R, nb - p0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* cvp = conv + (size_t)l * (pbmax + 1);
  const double* cvc = conv + (size_t)(l + 1) * (pbmax + 1);
  for (int idx = threadIdx.x; idx < 5 * R; idx += kT) {
    const int r = idx % R, c = idx / R;
    long long o = -1;
    if (r < nr) {
      if (c == 4) {
        o = eoff[parents[p0 + r]];
      } else {
        const int d = child[4 * parents[p0 + r] + c];
        if (d >= 0) o = eoff[d];
      }
    }
    if (c == 4) poff[r] = o; else coff[c][r] = o;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 4 * Qc * R; idx += kT) {
    const int c = idx / (Qc * R), rem = idx % (Qc * R), r = rem / Qc, n = rem % Qc;
    float2 v = make_float2(0.f, 0.f);
    const long long o = coff[c][r];
    if (o >= 0) {
      const cd a = mpole[o + n];
      const double f = cvc[abs(n - pc)];
      v = make_float2((float)(a.x * f), (float)(a.y * f));
    }
    mus4[((size_t)c * Qc + n) * RS + r] = v;
  }
  __syncthreads();
  const int so = (int)blockIdx.y * kSplitCols + lane;
  const bool act = so < Qp;
  float sr[R], si[R], cr[R], ci[R];
#pragma unroll
  for (int r = 0; r < R; ++r) sr[r] = si[r] = cr[r] = ci[r] = 0.f;
  tile_gemm_column<R>(Tmm + (size_t)warp * Qc * Qp, Qp, Qc, mus4 + (size_t)warp * Qc * RS, so,
                      act, sr, si, cr, ci);
  __syncthreads();  // the staged rows are dead: the reduction reuses the space
  double outr[R], outi[R];
  split_reduce<R>(sr, si, cr, ci, mus4, warp, lane, outr, outi);
  if (warp == 0 && act) {
    const double f = 1.0 / cvp[abs(so - pp)];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r >= nr) break;
      cd* dst = mpole + poff[r] + so;
      dst->x = outr[r] * f;
      dst->y = outi[r] * f;
    }
  }
}

template <int R>
__global__ void __launch_bounds__(kT) l2l_f32_split_kernel(
    int l, int pp, int pc, int pbmax, const int* __restrict__ parents, int nb,
    const int* __restrict__ child, const long long* __restrict__ eoff,
    const float2* __restrict__ Tl, const double* __restrict__ conv, cd* __restrict__ local) {
  extern __shared__ __align__(16) float2 lam2[];  // [Qp][stage_stride(R)], then red
  const int Qp = 2 * pp + 1, Qc = 2 * pc + 1;
  const int RS = stage_stride(R);
  const int p0 = blockIdx.x * R, nr = min(R, nb - p0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* cvp = conv + (size_t)l * (pbmax + 1);
  const double* cvc = conv + (size_t)(l + 1) * (pbmax + 1);
  for (int idx = threadIdx.x; idx < Qp * R; idx += kT) {
    const int r = idx / Qp, n = idx % Qp;
    float2 v = make_float2(0.f, 0.f);
    if (r < nr) {
      const cd g = local[eoff[parents[p0 + r]] + n];
      const double f = 1.0 / cvp[abs(n - pp)];
      v = make_float2((float)(g.x * f), (float)(g.y * f));
    }
    lam2[n * RS + r] = v;
  }
  __syncthreads();
  const int c = blockIdx.y;
  const int so = (int)blockIdx.z * kSplitCols + lane;
  const bool act = so < Qc;
  // warp w: parent orders [n0, n1)
  const int per = (Qp + kSplitWarps - 1) / kSplitWarps;
  const int n0 = min(Qp, warp * per), n1 = min(Qp, n0 + per);
  float sr[R], si[R], cr[R], ci[R];
#pragma unroll
  for (int r = 0; r < R; ++r) sr[r] = si[r] = cr[r] = ci[r] = 0.f;
  if (n1 > n0)
    tile_gemm_column<R>(Tl + (size_t)c * Qp * Qc + (size_t)n0 * Qc, Qc, n1 - n0, lam2 + n0 * RS,
                        so, act, sr, si, cr, ci);
  __syncthreads();
  double outr[R], outi[R];
  split_reduce<R>(sr, si, cr, ci, lam2, warp, lane, outr, outi);
  if (warp == 0 && act) {
    const double f = cvc[abs(so - pc)];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r >= nr) break;
      const int d = child[4 * parents[p0 + r] + c];
      if (d < 0) continue;
      cd* dl = local + eoff[d] + so;
      dl->x += outr[r] * f;
      dl->y += outi[r] * f;
    }
  }
}

// out[i] = eoff[idx[i]]: the coefficient offset of each M2L source row
__global__ void gather_offsets_kernel(const int* __restrict__ idx, const long long* __restrict__ eoff,
                                      long long* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = eoff[idx[i]];
}

}  // namespace

static int g_mixed_smem_optin = 48 * 1024;  // the device's opt-in limit once configured

qbx_status configure_mixed_kernels(int smem_optin) {
  g_mixed_smem_optin = smem_optin;
  const void* k[] = {(const void*)l2l_f32_kernel<kGemmRows>, (const void*)l2l_f32_kernel<kNarrowRows>,
                     (const void*)m2m_f32_kernel<kGemmRows>, (const void*)m2m_f32_kernel<kNarrowRows>,
                     (const void*)m2m_f32_split_kernel<kNarrowRows>,
                     (const void*)l2l_f32_split_kernel<kNarrowRows>};
  for (const void* fn : k) {
    cudaFuncAttributes a;
    QBX_CUDA_TRY(cudaFuncGetAttributes(&a, fn));  // dynamic + static must fit the opt-in size
    QBX_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      smem_optin - (int)a.sharedSizeBytes));
  }
  return QBX_OK;
}

qbx_status mixed_plan_build(qbx_handle* h, FmmPlan* f) {
  const int pbm = f->pb_max;
  QBX_CUDA_TRY(f->lsig.alloc((size_t)f->n_levels * (pbm + 1)));
  QBX_CUDA_TRY(f->conv.alloc((size_t)f->n_levels * (pbm + 1)));
  QBX_CUDA_TRY(f->isig.alloc((size_t)f->n_levels * (pbm + 2)));
  sigma_tables_kernel<<<1, 64>>>(f->n_levels, pbm, f->lpb.ptr, h->k, f->side, f->scale.ptr,
                                 f->lsig.ptr, f->conv.ptr, f->isig.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(f->m2p_rec.alloc((size_t)f->n_levels * (pbm + 2)));
  m2p_rec_kernel<<<f->n_levels, 128>>>(f->n_levels, pbm, f->lpb.ptr, f->lsig.ptr, f->m2p_rec.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(f->sigr.alloc((size_t)f->n_levels * (pbm + 2)));
  sig_ratio_kernel<<<f->n_levels, 128>>>(f->n_levels, pbm, f->lpb.ptr, f->lsig.ptr, f->sigr.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(f->m2p_t.alloc((size_t)f->n_levels * (pbm + 2)));
  m2p_t_kernel<<<f->n_levels, 128>>>(f->n_levels, pbm, f->lpb.ptr, f->lsig.ptr, f->m2p_t.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  {  // levels where H_pb(x) could leave the FP64 range: x = k |t - m_c| >= 1.5 k
     // side for a W-list box (taken as 0.5 k side), |H_m(x)| <~ (m-1)! (2/x)^m
    std::vector<int> scaled(f->n_levels, 0);
    for (int l = 0; l < f->n_levels; ++l) {
      const int pb = f->h_pb[l];
      if (pb < 1) continue;
      const double x_lo = 0.5 * h->k * f->side / (double)(1LL << std::min(l, 62));
      const double ln_h = std::lgamma((double)pb) + pb * std::log(2.0 / x_lo);
      scaled[l] = ln_h > 650.0 ? 1 : 0;
    }
    QBX_CUDA_TRY(f->m2p_scaled.alloc(f->n_levels));
    QBX_CUDA_TRY(cudaMemcpy(f->m2p_scaled.ptr, scaled.data(), f->n_levels * sizeof(int),
                            cudaMemcpyHostToDevice));
  }
  // matrices for the levels that have V lists
  std::vector<long long> off(f->n_levels, 0);
  long long tot = 0;
  for (int l = 0; l < f->n_levels; ++l) {
    off[l] = tot;
    if (f->vbox_off[l + 1] > f->vbox_off[l]) {
      const long long Q = 2 * f->h_pb[l] + 1;
      tot += 49 * Q * Q;
    }
  }
  QBX_CUDA_TRY(f->tm_f32.alloc(std::max<long long>(1, tot)));
  f->h_tm_off = off;
  for (int l = 2; l < f->n_levels; ++l) {
    if (f->vbox_off[l + 1] == f->vbox_off[l]) continue;
    const int pb = f->h_pb[l];
    dim3 grid(49, 2 * pb + 1);
    m2l_f32_matrix_kernel<<<grid, kT>>>(l, pb, pbm, f->t_m2l.ptr, f->scale.ptr, f->lsig.ptr,
                                        f->tm_f32.ptr + off[l]);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  // M2L work: V-list pairs grouped by (level, offset class), cut into tiles
  // of kGemmRows rows; the row of V entry e is vrow[e], its output at yoff[row]
  {
    const int nb = f->n_boxes;
    const int64_t nv = f->V.nnz;
    std::vector<int> voff(nb + 1), vidx(std::max<int64_t>(1, nv)), vcls(std::max<int64_t>(1, nv)),
        blev(nb);
    QBX_CUDA_TRY(cudaMemcpy(voff.data(), f->V.off.ptr, (nb + 1) * sizeof(int), cudaMemcpyDeviceToHost));
    if (nv) {
      QBX_CUDA_TRY(cudaMemcpy(vidx.data(), f->V.idx.ptr, nv * sizeof(int), cudaMemcpyDeviceToHost));
      QBX_CUDA_TRY(cudaMemcpy(vcls.data(), f->V_cls.ptr, nv * sizeof(int), cudaMemcpyDeviceToHost));
    }
    QBX_CUDA_TRY(cudaMemcpy(blev.data(), f->box.level.ptr, nb * sizeof(int), cudaMemcpyDeviceToHost));
    const int ng = f->n_levels * 49;
    std::vector<int64_t> gcount(ng + 1, 0);
    std::vector<int> egroup(std::max<int64_t>(1, nv));
    for (int b = 0; b < nb; ++b)
      for (int e = voff[b]; e < voff[b + 1]; ++e) {
        egroup[e] = blev[b] * 49 + vcls[e];
        gcount[egroup[e] + 1] += 1;
      }
    for (int g = 0; g < ng; ++g) gcount[g + 1] += gcount[g];
    std::vector<int> vrow(std::max<int64_t>(1, nv)), row_src(std::max<int64_t>(1, nv));
    std::vector<long long> yoff(std::max<int64_t>(1, nv));
    std::vector<int64_t> fill(gcount.begin(), gcount.end() - 1);
    for (int b = 0; b < nb; ++b)
      for (int e = voff[b]; e < voff[b + 1]; ++e) {
        const int row = (int)fill[egroup[e]]++;
        vrow[e] = row;
        row_src[row] = vidx[e];
      }
    f->h_row_src = row_src;
    f->h_row_src.resize(gcount[ng]);
    f->h_gcount.assign(gcount.begin(), gcount.end());
    long long ytot = 0;
    std::vector<int4> tiles;
    for (int g = 0; g < ng; ++g) {
      const int l = g / 49, Q = 2 * f->h_pb[l] + 1;
      for (int64_t r = gcount[g]; r < gcount[g + 1]; ++r) {
        yoff[r] = ytot;
        ytot += Q;
      }
      for (int64_t r = gcount[g]; r < gcount[g + 1]; r += kGemmRows)
        tiles.push_back(make_int4(g, (int)r, (int)std::min<int64_t>(kGemmRows, gcount[g + 1] - r), l));
    }
    // coarse levels (largest orders) first; work items (first row, rows,
    // first output order, group) per tile: chunks of kT output orders, and
    // for FP64 also groups of kF64Rows rows
    std::vector<int4> it32, it64;
    for (const int4& t : tiles) {
      const int Q = 2 * f->h_pb[t.w] + 1;
      for (int c0 = 0; c0 < Q; c0 += kT) {
        it32.push_back(make_int4(t.y, t.z, c0, t.x));
        for (int r0 = 0; r0 < t.z; r0 += kF64Rows)
          it64.push_back(make_int4(t.y + r0, std::min(kF64Rows, t.z - r0), c0, t.x));
      }
    }
    // matrix offset of each group (level l, class c): level offset + c Q_l^2
    std::vector<long long> goff(ng, 0);
    for (int g = 0; g < ng; ++g) {
      const long long Q = 2 * f->h_pb[g / 49] + 1;
      goff[g] = off[g / 49] + (long long)(g % 49) * Q * Q;
    }
    QBX_CUDA_TRY(f->m2l_goff.alloc(ng));
    QBX_CUDA_TRY(cudaMemcpy(f->m2l_goff.ptr, goff.data(), ng * sizeof(long long), cudaMemcpyHostToDevice));
    f->n_m2l_items32 = (int)it32.size();
    f->n_m2l_items64 = (int)it64.size();
    f->h_items64 = it64;
    QBX_CUDA_TRY(f->m2l_items32.alloc(std::max<size_t>(1, it32.size())));
    QBX_CUDA_TRY(f->m2l_items64.alloc(std::max<size_t>(1, it64.size())));
    if (!it32.empty()) {
      QBX_CUDA_TRY(cudaMemcpy(f->m2l_items32.ptr, it32.data(), it32.size() * sizeof(int4), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(cudaMemcpy(f->m2l_items64.ptr, it64.data(), it64.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
    QBX_CUDA_TRY(f->m2l_eyoff.alloc(vrow.size()));
    QBX_CUDA_TRY(f->m2l_yoff.alloc(yoff.size()));
    QBX_CUDA_TRY(f->m2l_y.alloc(std::max<long long>(1, ytot)));
    // the boxes that are V-list sources, and FP32 room for their multipoles
    std::vector<char> is_src(nb, 0);
    for (int64_t e = 0; e < nv; ++e) is_src[vidx[e]] = 1;
    std::vector<int> vsrc;
    for (int b = 0; b < nb; ++b)
      if (is_src[b]) vsrc.push_back(b);
    f->n_vsrc = (int)vsrc.size();
    QBX_CUDA_TRY(f->m2l_vsrc.alloc(std::max<size_t>(1, vsrc.size())));
    if (!vsrc.empty())
      QBX_CUDA_TRY(cudaMemcpy(f->m2l_vsrc.ptr, vsrc.data(), vsrc.size() * sizeof(int), cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(f->mu32.alloc(std::max<int64_t>(1, f->n_coef)));
    {  // result-row offset of every V entry
      std::vector<long long> eyoff(vrow.size(), 0);
      for (int64_t e = 0; e < nv; ++e) eyoff[e] = yoff[vrow[e]];
      QBX_CUDA_TRY(cudaMemcpy(f->m2l_eyoff.ptr, eyoff.data(), eyoff.size() * sizeof(long long),
                              cudaMemcpyHostToDevice));
    }
    {  // coefficient offset of each row's source box
      DevBuf<int> rs;
      QBX_CUDA_TRY(rs.alloc(row_src.size()));
      QBX_CUDA_TRY(cudaMemcpy(rs.ptr, row_src.data(), row_src.size() * sizeof(int), cudaMemcpyHostToDevice));
      QBX_CUDA_TRY(f->m2l_rowoff.alloc(row_src.size()));
      gather_offsets_kernel<<<nblk((int64_t)row_src.size(), 256), 256>>>(rs.ptr, f->eoff.ptr,
                                                                          f->m2l_rowoff.ptr, (int64_t)row_src.size());
      QBX_CUDA_TRY(cudaGetLastError());
      QBX_CUDA_TRY(cudaDeviceSynchronize());  // before rs is freed
    }
    QBX_CUDA_TRY(cudaMemcpy(f->m2l_yoff.ptr, yoff.data(), yoff.size() * sizeof(long long), cudaMemcpyHostToDevice));
  }
  // FP64 M2L matrices (same offsets as the FP32 ones) and result rows
  QBX_CUDA_TRY(f->tm_f64.alloc(std::max<long long>(1, tot)));
  for (int l = 2; l < f->n_levels; ++l) {
    if (f->vbox_off[l + 1] == f->vbox_off[l]) continue;
    const int pb = f->h_pb[l];
    dim3 grid(49, 2 * pb + 1);
    m2l_f64_matrix_kernel<<<grid, kT>>>(l, pb, pbm, f->t_m2l.ptr, f->pw.ptr, f->tm_f64.ptr + off[l]);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  QBX_CUDA_TRY(f->m2l_y64.alloc(std::max<size_t>(1, f->m2l_y.n)));
  // M2M matrices for parents on levels 2 .. n_levels - 2
  {
    std::vector<long long> moff(f->n_levels, 0);
    long long mtot = 0;
    for (int l = 2; l + 1 < f->n_levels; ++l) {
      moff[l] = mtot;
      mtot += 4LL * (2 * f->h_pb[l] + 1) * (2 * f->h_pb[l + 1] + 1);
    }
    QBX_CUDA_TRY(f->tmm_f32.alloc(std::max<long long>(1, mtot)));
    f->h_tmm_off = moff;
    for (int l = 2; l + 1 < f->n_levels; ++l) {
      const int pp = f->h_pb[l], pc = f->h_pb[l + 1];
      dim3 grid(4, 2 * pc + 1);
      m2m_f32_matrix_kernel<<<grid, kT>>>(l, pp, pc, pbm, f->t_m2m.ptr, f->lsig.ptr,
                                          f->tmm_f32.ptr + moff[l]);
      QBX_CUDA_TRY(cudaGetLastError());
    }
  }
  // L2L matrices for parents on levels 2 .. n_levels - 2
  std::vector<long long> loff(f->n_levels, 0);
  long long ltot = 0;
  for (int l = 2; l + 1 < f->n_levels; ++l) {
    loff[l] = ltot;
    ltot += 4LL * (2 * f->h_pb[l] + 1) * (2 * f->h_pb[l + 1] + 1);
  }
  QBX_CUDA_TRY(f->tl_f32.alloc(std::max<long long>(1, ltot)));
  f->h_tl_off = loff;
  for (int l = 2; l + 1 < f->n_levels; ++l) {
    const int pp = f->h_pb[l], pc = f->h_pb[l + 1];
    dim3 grid(4, 2 * pp + 1);
    l2l_f32_matrix_kernel<<<grid, kT>>>(l, pp, pc, pbm, f->t_l2l.ptr, f->lsig.ptr,
                                        f->tl_f32.ptr + loff[l]);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  return QBX_OK;
}

size_t gemm_smem_bytes(int pb) {
  return (size_t)(2 * pb + 1) * stage_stride(kGemmRows) * sizeof(float2) +
         5 * kGemmRows * sizeof(long long);
}

qbx_status launch_m2l_f64(qbx_handle* h, FmmPlan* f, cudaStream_t s) {
  if (f->n_vbox == 0 || f->n_m2l_items64 == 0) return QBX_OK;
  m2l_f64_gemm_kernel<<<f->n_m2l_items64, kT, 0, s>>>(
      f->m2l_items64.ptr, f->lpb.ptr, f->m2l_goff.ptr, f->m2l_rowoff.ptr, f->mpole.ptr,
      f->tm_f64.ptr, f->m2l_yoff.ptr, f->m2l_y64.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  m2l_f64_reduce_kernel<<<f->n_vbox, kT, 0, s>>>(
      f->vbox.ptr, f->box.level.ptr, f->lpb.ptr, f->V.off.ptr, f->m2l_eyoff.ptr,
      f->m2l_y64.ptr, f->eoff.ptr, f->local.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 2;
  return QBX_OK;
}

// The FP64 tile GEMM over the items of the levels that the tensor-core M2L
// does not take (their result rows, FP64, are added by the tensor-core path's
// reduction).
qbx_status launch_m2l_f64_gemm_rest(qbx_handle* h, FmmPlan* f, cudaStream_t s) {
  if (f->n_m2l_items64_rest == 0) return QBX_OK;
  m2l_f64_gemm_kernel<<<f->n_m2l_items64_rest, kT, 0, s>>>(
      f->m2l_items64_rest.ptr, f->lpb.ptr, f->m2l_goff.ptr, f->m2l_rowoff.ptr, f->mpole.ptr,
      f->tm_f64.ptr, f->m2l_yoff.ptr, f->m2l_y64.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}

// Dynamic shared memory of a split-K M2M / L2L CTA staging `rows` coefficient
// rows of kNarrowRows boxes (the reduction reuses the space); split_fits: within
// the opt-in limit with room for the kernels' static shared memory.
static size_t split_smem(int rows) {
  const size_t stage = (size_t)rows * stage_stride(kNarrowRows) * sizeof(float2);
  const size_t red = (size_t)kSplitWarps * kNarrowRows * 32 * sizeof(float2);
  return std::max(stage, red);
}
static bool split_fits(int rows) { return split_smem(rows) + 1024 <= (size_t)g_mixed_smem_optin; }
// The split kernels serve levels whose one-column-per-thread grid would have
// fewer than four CTAs per SM (GB300: 152 SMs); wider levels keep the others.
constexpr long long kSplitBelow = 4 * 152;

qbx_status launch_m2m_f32(qbx_handle* h, FmmPlan* f, cudaStream_t s) {
  for (int l = f->n_levels - 2; l >= 2; --l) {
    const int nb = f->nonleaf_off[l + 1] - f->nonleaf_off[l];
    if (nb == 0) continue;
    const int pp = f->h_pb[l], pc = f->h_pb[l + 1];
    const int* par = f->nonleaf.ptr + f->nonleaf_off[l];
    const float2* T = f->tmm_f32.ptr + f->h_tmm_off[l];
    if (nb >= kWideLevel || h->batched)
      m2m_f32_kernel<kGemmRows><<<dim3(nblk(nb, kGemmRows), nblk(2 * pp + 1, kT)), kT, (size_t)(2 * pc + 1) * stage_stride(kGemmRows) * sizeof(float2), s>>>(
          l, pp, pc, f->pb_max, par, nb, f->box.child.ptr, f->eoff.ptr, T, f->conv.ptr, f->mpole.ptr);
    else if ((long long)nblk(nb, kNarrowRows) * nblk(2 * pp + 1, kT) < kSplitBelow &&
             split_fits(4 * (2 * pc + 1)))
      m2m_f32_split_kernel<kNarrowRows><<<dim3(nblk(nb, kNarrowRows), nblk(2 * pp + 1, kSplitCols)), kT, split_smem(4 * (2 * pc + 1)), s>>>(
          l, pp, pc, f->pb_max, par, nb, f->box.child.ptr, f->eoff.ptr, T, f->conv.ptr, f->mpole.ptr);
    else
      m2m_f32_kernel<kNarrowRows><<<dim3(nblk(nb, kNarrowRows), nblk(2 * pp + 1, kT)), kT, (size_t)(2 * pc + 1) * stage_stride(kNarrowRows) * sizeof(float2), s>>>(
          l, pp, pc, f->pb_max, par, nb, f->box.child.ptr, f->eoff.ptr, T, f->conv.ptr, f->mpole.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    h->launches += 1;
  }
  return QBX_OK;
}

qbx_status launch_l2l_f32(qbx_handle* h, FmmPlan* f, cudaStream_t s) {
  for (int l = 2; l + 1 < f->n_levels; ++l) {
    const int nb = f->nonleaf_off[l + 1] - f->nonleaf_off[l];
    if (nb == 0) continue;
    const int pp = f->h_pb[l], pc = f->h_pb[l + 1];
    const int* par = f->nonleaf.ptr + f->nonleaf_off[l];
    const float2* T = f->tl_f32.ptr + f->h_tl_off[l];
    if (nb >= kWideLevel || h->batched)
      l2l_f32_kernel<kGemmRows><<<dim3(nblk(nb, kGemmRows), 4, nblk(2 * pc + 1, kT)), kT, (size_t)(2 * pp + 1) * stage_stride(kGemmRows) * sizeof(float2), s>>>(
          l, pp, pc, f->pb_max, par, nb, f->box.child.ptr, f->eoff.ptr, T, f->conv.ptr, f->local.ptr);
    else if ((long long)nblk(nb, kNarrowRows) * 4 * nblk(2 * pc + 1, kT) < kSplitBelow &&
             split_fits(2 * pp + 1))
      l2l_f32_split_kernel<kNarrowRows><<<dim3(nblk(nb, kNarrowRows), 4, nblk(2 * pc + 1, kSplitCols)), kT, split_smem(2 * pp + 1), s>>>(
          l, pp, pc, f->pb_max, par, nb, f->box.child.ptr, f->eoff.ptr, T, f->conv.ptr, f->local.ptr);
    else
      l2l_f32_kernel<kNarrowRows><<<dim3(nblk(nb, kNarrowRows), 4, nblk(2 * pc + 1, kT)), kT, (size_t)(2 * pp + 1) * stage_stride(kNarrowRows) * sizeof(float2), s>>>(
          l, pp, pc, f->pb_max, par, nb, f->box.child.ptr, f->eoff.ptr, T, f->conv.ptr, f->local.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    h->launches += 1;
  }
  return QBX_OK;
}

qbx_status launch_m2l_f32(qbx_handle* h, FmmPlan* f, cudaStream_t s) {
  if (f->n_vbox == 0 || f->n_m2l_items32 == 0) return QBX_OK;
  if (f->n_vsrc > 0) {
    mpole_to_f32_kernel<<<f->n_vsrc, kT, 0, s>>>(f->pb_max, f->m2l_vsrc.ptr, f->box.level.ptr,
                                                 f->lpb.ptr, f->eoff.ptr, f->conv.ptr,
                                                 f->mpole.ptr, f->mu32.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    h->launches += 1;
  }
  m2l_f32_gemm_kernel<<<f->n_m2l_items32, kT, 0, s>>>(
      f->m2l_items32.ptr, f->lpb.ptr, f->m2l_goff.ptr, f->m2l_rowoff.ptr, f->mu32.ptr,
      f->tm_f32.ptr, f->m2l_yoff.ptr, f->m2l_y.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  m2l_f32_reduce_kernel<<<f->n_vbox, kT, 0, s>>>(
      f->pb_max, f->vbox.ptr, f->box.level.ptr, f->lpb.ptr, f->V.off.ptr, f->m2l_eyoff.ptr,
      f->m2l_y.ptr, f->conv.ptr, f->eoff.ptr, f->local.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 2;
  return QBX_OK;
}
