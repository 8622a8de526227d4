// Quadtree construction (Sec. 4, Sec. 7 Stage 1), the U/V/W/X interaction lists
// (Sec. 7.2) and target association through the tree (Sec. 6.1), all on the GPU.
//
// Tree: the root is the smallest axis-aligned square holding every particle
// (sources, centres, targets and density nodes). Every particle class is sorted
// by its Morton key at the finest level (24 bits per axis); a box at level l is
// a key prefix, so the particles of a box are a contiguous range of each sorted
// array, found by binary search. Levels are built one after the other: a box is
// split when it holds more than n_max sources + centres + targets; empty
// children are pruned. Boxes of a level are stored in Morton order, so a box
// is found from its integer position by binary search in its level.
#include <cub/cub.cuh>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "special.cuh"
#include "tree.cuh"

namespace {

typedef unsigned long long u64;

__host__ __device__ __forceinline__ u64 spread_bits(unsigned v) {
  u64 x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
__host__ __device__ __forceinline__ u64 morton(int ix, int iy) {
  return spread_bits((unsigned)ix) | (spread_bits((unsigned)iy) << 1);
}

__device__ __forceinline__ long long ordered(double v) {
  long long i = __double_as_longlong(v);
  return i ^ ((i >> 63) & 0x7fffffffffffffffLL);
}
__host__ __forceinline__ double unordered(long long i) {
  i ^= (i >> 63) & 0x7fffffffffffffffLL;
  double v;
  memcpy(&v, &i, sizeof(v));
  return v;
}

// bbox[0..3] = ordered(min x), ordered(min y), ordered(max x), ordered(max y)
__global__ void bbox_kernel(int64_t n, const double* __restrict__ xy, long long* bbox) {
  __shared__ long long red[4][256];
  long long mnx = LLONG_MAX, mny = LLONG_MAX, mxx = LLONG_MIN, mxy = LLONG_MIN;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    long long a = ordered(xy[2 * i]), b = ordered(xy[2 * i + 1]);
    mnx = min(mnx, a); mny = min(mny, b); mxx = max(mxx, a); mxy = max(mxy, b);
  }
  red[0][threadIdx.x] = mnx; red[1][threadIdx.x] = mny;
  red[2][threadIdx.x] = mxx; red[3][threadIdx.x] = mxy;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] = min(red[0][threadIdx.x], red[0][threadIdx.x + s]);
      red[1][threadIdx.x] = min(red[1][threadIdx.x], red[1][threadIdx.x + s]);
      red[2][threadIdx.x] = max(red[2][threadIdx.x], red[2][threadIdx.x + s]);
      red[3][threadIdx.x] = max(red[3][threadIdx.x], red[3][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicMin(&bbox[0], red[0][0]);
    atomicMin(&bbox[1], red[1][0]);
    atomicMax(&bbox[2], red[2][0]);
    atomicMax(&bbox[3], red[3][0]);
  }
}

__global__ void morton_kernel(int64_t n, const double* __restrict__ xy, double x0, double y0,
                              double inv_cell, u64* __restrict__ keys, int* __restrict__ vals) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lim = (1 << kMortonBits) - 1;
  int ix = (int)floor((xy[2 * i] - x0) * inv_cell);
  int iy = (int)floor((xy[2 * i + 1] - y0) * inv_cell);
  ix = min(max(ix, 0), lim);
  iy = min(max(iy, 0), lim);
  keys[i] = morton(ix, iy);
  vals[i] = (int)i;
}

__device__ __forceinline__ int lower_bound(const u64* __restrict__ a, int lo, int hi, u64 v) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct KeySet {
  const u64* k[PT_COUNT];
};

// child c of a box: its range of particle class t
__device__ __forceinline__ int2 child_range(const KeySet& ks, int t, int2 r, u64 prefix, int level,
                                            int c) {
  const int sh = 2 * (kMortonBits - level - 1);
  u64 cp = (prefix << 2) | (u64)c;
  int a = lower_bound(ks.k[t], r.x, r.y, cp << sh);
  int b = lower_bound(ks.k[t], a, r.y, (cp + 1) << sh);
  return make_int2(a, b);
}

// A box is split when it holds more than n_max sources + centres + targets,
// unless its children would be narrower than kappa times the expansion radius
// of a centre it holds: every QBX disk then stays well inside the region where
// the local expansion of its leaf converges.
__global__ void split_count_kernel(int nb, int off, int level, int n_max, KeySet ks,
                                   const u64* __restrict__ bkey, const int2* __restrict__ r0,
                                   const int2* __restrict__ r1, const int2* __restrict__ r2,
                                   const int2* __restrict__ r3, const double* __restrict__ crad,
                                   double child_side, double kappa,
                                   int* __restrict__ nchild) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int b = off + i;
  const int2 r[PT_COUNT] = {r0[b], r1[b], r2[b], r3[b]};
  int total = (r[0].y - r[0].x) + (r[1].y - r[1].x) + (r[2].y - r[2].x);
  bool wide = true;
  for (int j = r[PT_CTR].x; j < r[PT_CTR].y && wide; ++j) wide = kappa * crad[j] <= child_side;
  int cnt = 0;
  if (total > n_max && level < kMaxLevels && wide) {
    for (int c = 0; c < 4; ++c) {
      bool ne = false;
      for (int t = 0; t < PT_COUNT && !ne; ++t) {
        int2 cr = child_range(ks, t, r[t], bkey[b], level, c);
        ne = cr.y > cr.x;
      }
      cnt += ne ? 1 : 0;
    }
  }
  nchild[i] = cnt;
}

__global__ void split_fill_kernel(int nb, int off, int level, int next_off, KeySet ks,
                                  const int* __restrict__ nchild, const int* __restrict__ choff,
                                  double x0, double y0, double side, int* __restrict__ blevel,
                                  int* __restrict__ bparent, int* __restrict__ bchild,
                                  int2* __restrict__ bij, u64* __restrict__ bkey,
                                  double2* __restrict__ bcentre, int2* r0, int2* r1, int2* r2,
                                  int2* r3) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int b = off + i;
  if (nchild[i] == 0) return;
  int2* rr[PT_COUNT] = {r0, r1, r2, r3};
  const int2 r[PT_COUNT] = {r0[b], r1[b], r2[b], r3[b]};
  int slot = next_off + choff[i];
  const int2 pij = bij[b];
  const double cs = side / (double)(1 << (level + 1));
  for (int c = 0; c < 4; ++c) {
    int2 cr[PT_COUNT];
    bool ne = false;
    for (int t = 0; t < PT_COUNT; ++t) {
      cr[t] = child_range(ks, t, r[t], bkey[b], level, c);
      ne = ne || cr[t].y > cr[t].x;
    }
    if (!ne) continue;
    const int d = slot++;
    const int ix = 2 * pij.x + (c & 1), iy = 2 * pij.y + (c >> 1);
    blevel[d] = level + 1;
    bparent[d] = b;
    bij[d] = make_int2(ix, iy);
    bkey[d] = morton(ix, iy);
    bcentre[d] = make_double2(x0 + (ix + 0.5) * cs, y0 + (iy + 0.5) * cs);
    for (int t = 0; t < PT_COUNT; ++t) rr[t][d] = cr[t];
    for (int q = 0; q < 4; ++q) bchild[4 * d + q] = -1;
    bchild[4 * b + c] = d;
  }
}

template <typename T>
__global__ void gather_kernel(int64_t n, const int* __restrict__ perm, const T* __restrict__ src,
                              T* __restrict__ dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}

// ---------------------------------------------------------------- lists
struct TreeView {
  const int* level;
  const int* parent;
  const int* child;
  const int2* ij;
  const u64* key;
  const int* level_off;
  int n_levels;
};

__device__ __forceinline__ int find_box(const TreeView& T, int lev, int ix, int iy) {
  if (lev < 0 || lev >= T.n_levels) return -1;
  const int lim = 1 << lev;
  if (ix < 0 || iy < 0 || ix >= lim || iy >= lim) return -1;
  const u64 v = morton(ix, iy);
  int lo = T.level_off[lev], hi = T.level_off[lev + 1];
  int p = lower_bound(T.key, lo, hi, v);
  return (p < hi && T.key[p] == v) ? p : -1;
}

__device__ __forceinline__ bool is_leaf(const TreeView& T, int b) {
  const int* c = T.child + 4 * b;
  return c[0] < 0 && c[1] < 0 && c[2] < 0 && c[3] < 0;
}

// closed squares of b (level lb) and d (level ld >= lb) touch
__device__ __forceinline__ bool adjacent(int2 bij, int lb, int2 dij, int ld) {
  const int sh = ld - lb;
  const long long lox = (long long)bij.x << sh, hix = (((long long)bij.x + 1) << sh) - 1;
  const long long loy = (long long)bij.y << sh, hiy = (((long long)bij.y + 1) << sh) - 1;
  return dij.x >= lox - 1 && dij.x <= hix + 1 && dij.y >= loy - 1 && dij.y <= hiy + 1;
}

constexpr int kStack = 256;

template <bool FILL>
__global__ void lists_kernel(int nb, TreeView T, int* __restrict__ ucnt, int* __restrict__ vcnt,
                             int* __restrict__ wcnt, const int* __restrict__ uoff,
                             const int* __restrict__ voff, const int* __restrict__ woff,
                             int* __restrict__ uidx, int* __restrict__ vidx,
                             int* __restrict__ vcls, int* __restrict__ widx,
                             int* __restrict__ err) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int lb = T.level[b];
  const int2 bij = T.ij[b];
  int nu = 0, nv = 0, nw = 0;
  // V list: children of the parent's colleagues that are not adjacent to b
  if (lb >= 2) {
    const int P = T.parent[b];
    const int2 pij = T.ij[P];
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int C = find_box(T, lb - 1, pij.x + dx, pij.y + dy);
        if (C < 0) continue;
        for (int c = 0; c < 4; ++c) {
          const int d = T.child[4 * C + c];
          if (d < 0) continue;
          const int2 dij = T.ij[d];
          const int ax = dij.x - bij.x, ay = dij.y - bij.y;
          if (max(abs(ax), abs(ay)) >= 2) {
            if (FILL) {
              vidx[voff[b] + nv] = d;
              vcls[voff[b] + nv] = (bij.x - dij.x + 3) * 7 + (bij.y - dij.y + 3);
            }
            ++nv;
          }
        }
      }
  }
  if (is_leaf(T, b)) {
    int stack[kStack];
    int sp = 0;
    if (FILL) uidx[uoff[b] + nu] = b;
    ++nu;
    int coarse[8];
    int nco = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0) continue;
        const int lim = 1 << lb;
        const int nx = bij.x + dx, ny = bij.y + dy;
        if (nx < 0 || ny < 0 || nx >= lim || ny >= lim) continue;
        const int C = find_box(T, lb, nx, ny);
        if (C >= 0) {
          if (is_leaf(T, C)) {
            if (FILL) uidx[uoff[b] + nu] = C;
            ++nu;
          } else if (sp < kStack) {
            stack[sp++] = C;
          } else {
            atomicOr(err, 1);
          }
          continue;
        }
        // no box at this level there: the deepest coarser box holding that cell
        for (int l = lb - 1; l >= 0; --l) {
          const int B = find_box(T, l, nx >> (lb - l), ny >> (lb - l));
          if (B < 0) continue;
          if (is_leaf(T, B)) {
            bool dup = false;
            for (int i = 0; i < nco; ++i) dup = dup || coarse[i] == B;
            if (!dup) {
              coarse[nco++] = B;
              if (FILL) uidx[uoff[b] + nu] = B;
              ++nu;
            }
          }
          break;
        }
      }
    // finer descendants of colleagues: adjacent leaves -> U, non-adjacent -> W
    while (sp > 0) {
      const int B = stack[--sp];
      for (int c = 0; c < 4; ++c) {
        const int d = T.child[4 * B + c];
        if (d < 0) continue;
        if (adjacent(bij, lb, T.ij[d], T.level[d])) {
          if (is_leaf(T, d)) {
            if (FILL) uidx[uoff[b] + nu] = d;
            ++nu;
          } else if (sp < kStack) {
            stack[sp++] = d;
          } else {
            atomicOr(err, 1);
          }
        } else {
          if (FILL) widx[woff[b] + nw] = d;
          ++nw;
        }
      }
    }
  }
  if (!FILL) {
    ucnt[b] = nu;
    vcnt[b] = nv;
    wcnt[b] = nw;
  }
}

__global__ void xcount_kernel(int nb, const int* __restrict__ woff, const int* __restrict__ widx,
                              int* __restrict__ xcnt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  for (int i = woff[b]; i < woff[b + 1]; ++i) atomicAdd(&xcnt[widx[i]], 1);
}

__global__ void xfill_kernel(int nb, const int* __restrict__ woff, const int* __restrict__ widx,
                             int* __restrict__ cursor, int* __restrict__ xidx) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  for (int i = woff[b]; i < woff[b + 1]; ++i) {
    const int pos = atomicAdd(&cursor[widx[i]], 1);
    xidx[pos] = b;
  }
}

__global__ void sort_lists_kernel(int nb, const int* __restrict__ off, int* __restrict__ idx) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  for (int i = off[b] + 1; i < off[b + 1]; ++i) {
    int v = idx[i], j = i - 1;
    while (j >= off[b] && idx[j] > v) {
      idx[j + 1] = idx[j];
      --j;
    }
    idx[j + 1] = v;
  }
}

// ---------------------------------------------------------------- association
__global__ void associate_tree_kernel(
    int64_t n_tgt, const double* __restrict__ tgt_xy, const int64_t* __restrict__ on_node,
    const int8_t* __restrict__ on_side, int64_t n_nodes, const double* __restrict__ node_xy,
    const double* __restrict__ panel_h, int q, const double* __restrict__ ctr_xy,
    const double* __restrict__ ctr_r, double eps, double rq_ctr, double rq_node, TreeView T,
    const double2* __restrict__ bcentre, double side, const int2* __restrict__ rctr,
    const int2* __restrict__ rnode, const int* __restrict__ perm_ctr,
    const int* __restrict__ perm_node, int32_t* __restrict__ assoc, int32_t* __restrict__ ctrs,
    int* __restrict__ err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_tgt) return;
  if (on_node && on_node[t] >= 0) {
    const int64_t j = on_node[t];
    const int side_ = on_side ? on_side[t] : 1;
    assoc[t] = (int32_t)(side_ >= 0 ? j : n_nodes + j);
    return;
  }
  const double tx = tgt_xy[2 * t], ty = tgt_xy[2 * t + 1];
  const double one_eps = __dadd_rn(1.0, eps);
  int stack[kStack];
  // pass 1: nearest eligible centre
  long long best = -1;
  double best_d2 = 1.0 / 0.0;
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const int b = stack[--sp];
    const double half = 0.5 * side / (double)(1 << T.level[b]);
    const double2 c = bcentre[b];
    const double reach = (half + rq_ctr) * (1.0 + 1e-12) + 1e-300;
    if (fabs(tx - c.x) > reach || fabs(ty - c.y) > reach) continue;
    if (is_leaf(T, b)) {
      const int2 r = rctr[b];
      for (int i = r.x; i < r.y; ++i) {
        const int ci = perm_ctr[i];
        const double dx = __dsub_rn(tx, ctr_xy[2 * ci]);
        const double dy = __dsub_rn(ty, ctr_xy[2 * ci + 1]);
        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        const double lim = __dmul_rn(one_eps, ctr_r[ci]);
        if (d2 <= __dmul_rn(lim, lim) && (d2 < best_d2 || (d2 == best_d2 && ci < best))) {
          best = ci;
          best_d2 = d2;
        }
      }
    } else {
      for (int k = 0; k < 4; ++k) {
        const int d = T.child[4 * b + k];
        if (d < 0) continue;
        if (sp < kStack) stack[sp++] = d; else atomicOr(err, 2);
      }
    }
  }
  if (best >= 0) {
    assoc[t] = (int32_t)best;
    return;
  }
  // pass 2: is the target within h/4 of a density node (Gamma_near)?
  sp = 0;
  stack[sp++] = 0;
  bool near = false;
  while (sp > 0 && !near) {
    const int b = stack[--sp];
    const double half = 0.5 * side / (double)(1 << T.level[b]);
    const double2 c = bcentre[b];
    const double reach = (half + rq_node) * (1.0 + 1e-12) + 1e-300;
    if (fabs(tx - c.x) > reach || fabs(ty - c.y) > reach) continue;
    if (is_leaf(T, b)) {
      const int2 r = rnode[b];
      for (int i = r.x; i < r.y && !near; ++i) {
        const int j = perm_node[i];
        const double dx = __dsub_rn(tx, node_xy[2 * j]);
        const double dy = __dsub_rn(ty, node_xy[2 * j + 1]);
        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        const double qh = __dmul_rn(0.25, panel_h[j / q]);
        near = d2 <= __dmul_rn(qh, qh);
      }
    } else {
      for (int k = 0; k < 4; ++k) {
        const int d = T.child[4 * b + k];
        if (d < 0) continue;
        if (sp < kStack) stack[sp++] = d; else atomicOr(err, 2);
      }
    }
  }
  if (near) {
    assoc[t] = -2;
    atomicAdd(&ctrs[0], 1);
    atomicMin(&ctrs[1], (int32_t)t);
  } else {
    assoc[t] = -1;
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

template <typename T>
qbx_status grow(DevBuf<T>& b, size_t need, size_t keep) {
  if (b.n >= need) return QBX_OK;
  DevBuf<T> nb;
  QBX_CUDA_TRY(nb.alloc(std::max(need, 2 * b.n)));
  if (keep) QBX_CUDA_TRY(cudaMemcpy(nb.ptr, b.ptr, keep * sizeof(T), cudaMemcpyDeviceToDevice));
  std::swap(b.ptr, nb.ptr);
  std::swap(b.n, nb.n);
  return QBX_OK;
}

TreeView view(FmmPlan* f, const DevBuf<int>& level_off_dev) {
  TreeView T;
  T.level = f->box.level.ptr;
  T.parent = f->box.parent.ptr;
  T.child = f->box.child.ptr;
  T.ij = f->box.ij.ptr;
  T.key = f->box.key.ptr;
  T.level_off = level_off_dev.ptr;
  T.n_levels = f->n_levels;
  return T;
}

qbx_status scan(const int* in, int* out, int n) {
  size_t bytes = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, n);
  DevBuf<unsigned char> tmp;
  QBX_CUDA_TRY(tmp.alloc(bytes + 1));
  QBX_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp.ptr, bytes, in, out, n));
  return QBX_OK;
}

// offsets [n+1] from counts [n]; returns total
qbx_status counts_to_offsets(const int* cnt, DevBuf<int>& off, int n, int64_t* total) {
  QBX_CUDA_TRY(off.alloc(n + 1));
  if (n > 0) {
    qbx_status st = scan(cnt, off.ptr, n);
    if (st != QBX_OK) return st;
  }
  int last_off = 0, last_cnt = 0;
  if (n > 0) {
    QBX_CUDA_TRY(cudaMemcpy(&last_off, off.ptr + n - 1, sizeof(int), cudaMemcpyDeviceToHost));
    QBX_CUDA_TRY(cudaMemcpy(&last_cnt, cnt + n - 1, sizeof(int), cudaMemcpyDeviceToHost));
  }
  const int tot = last_off + last_cnt;
  QBX_CUDA_TRY(cudaMemcpy(off.ptr + n, &tot, sizeof(int), cudaMemcpyHostToDevice));
  *total = tot;
  return QBX_OK;
}

}  // namespace

#define TRY(x)                          \
  do {                                  \
    qbx_status s_ = (x);                \
    if (s_ != QBX_OK) return s_;        \
  } while (0)

qbx_status tree_build(qbx_handle* h, FmmPlan* f, int n_max, double kappa) {
  const double* xy[PT_COUNT] = {h->src_xy.ptr, h->ctr_xy.ptr, h->tgt_xy.ptr, h->node_xy.ptr};
  const int64_t n[PT_COUNT] = {h->n_src, h->n_ctr, h->n_tgt, h->n_nodes};
  for (int t = 0; t < PT_COUNT; ++t) f->count[t] = n[t];
  // bounding square
  DevBuf<long long> bb;
  QBX_CUDA_TRY(bb.alloc(4));
  long long init[4] = {LLONG_MAX, LLONG_MAX, LLONG_MIN, LLONG_MIN};
  QBX_CUDA_TRY(cudaMemcpy(bb.ptr, init, sizeof(init), cudaMemcpyHostToDevice));
  for (int t = 0; t < PT_COUNT; ++t)
    if (n[t] > 0) bbox_kernel<<<std::min<unsigned>(nblk(n[t], 256), 1024), 256>>>(n[t], xy[t], bb.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  long long hb[4];
  QBX_CUDA_TRY(cudaMemcpy(hb, bb.ptr, sizeof(hb), cudaMemcpyDeviceToHost));
  const double xmin = unordered(hb[0]), ymin = unordered(hb[1]);
  const double xmax = unordered(hb[2]), ymax = unordered(hb[3]);
  double side = std::max(xmax - xmin, ymax - ymin);
  side = side * (1.0 + 1e-9) + 1e-300;
  const double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax);
  f->x0 = cx - 0.5 * side;
  f->y0 = cy - 0.5 * side;
  f->side = side;
  const double inv_cell = (double)(1 << kMortonBits) / side;
  // Morton keys, sorted per class
  for (int t = 0; t < PT_COUNT; ++t) {
    const int64_t m = n[t];
    QBX_CUDA_TRY(f->keys[t].alloc(std::max<int64_t>(m, 1)));
    QBX_CUDA_TRY(f->perm[t].alloc(std::max<int64_t>(m, 1)));
    if (m == 0) continue;
    DevBuf<u64> k0;
    DevBuf<int> v0;
    QBX_CUDA_TRY(k0.alloc(m));
    QBX_CUDA_TRY(v0.alloc(m));
    morton_kernel<<<nblk(m, 256), 256>>>(m, xy[t], f->x0, f->y0, inv_cell, k0.ptr, v0.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    size_t bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, bytes, k0.ptr, f->keys[t].ptr, v0.ptr,
                                    f->perm[t].ptr, (int)m, 0, 2 * kMortonBits);
    DevBuf<unsigned char> tmp;
    QBX_CUDA_TRY(tmp.alloc(bytes + 1));
    QBX_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.ptr, bytes, k0.ptr, f->keys[t].ptr, v0.ptr,
                                                 f->perm[t].ptr, (int)m, 0, 2 * kMortonBits));
  }
  // centre radii in Morton order (for the split rule)
  DevBuf<double> crad_sorted;
  QBX_CUDA_TRY(crad_sorted.alloc(std::max<int64_t>(1, n[PT_CTR])));
  if (n[PT_CTR] > 0) {
    gather_kernel<double><<<nblk(n[PT_CTR], 256), 256>>>(n[PT_CTR], f->perm[PT_CTR].ptr,
                                                         h->ctr_r.ptr, crad_sorted.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  // levels
  size_t cap = 1024;
  BoxArrays& B = f->box;
  QBX_CUDA_TRY(B.level.alloc(cap));
  QBX_CUDA_TRY(B.parent.alloc(cap));
  QBX_CUDA_TRY(B.child.alloc(4 * cap));
  QBX_CUDA_TRY(B.ij.alloc(cap));
  QBX_CUDA_TRY(B.key.alloc(cap));
  QBX_CUDA_TRY(B.centre.alloc(cap));
  for (int t = 0; t < PT_COUNT; ++t) QBX_CUDA_TRY(B.rng[t].alloc(cap));
  {
    int lv = 0, par = -1, ch[4] = {-1, -1, -1, -1};
    int2 ij = make_int2(0, 0);
    u64 key = 0;
    double2 c = make_double2(cx, cy);
    QBX_CUDA_TRY(cudaMemcpy(B.level.ptr, &lv, sizeof(int), cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(B.parent.ptr, &par, sizeof(int), cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(B.child.ptr, ch, sizeof(ch), cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(B.ij.ptr, &ij, sizeof(ij), cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(B.key.ptr, &key, sizeof(key), cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(B.centre.ptr, &c, sizeof(c), cudaMemcpyHostToDevice));
    for (int t = 0; t < PT_COUNT; ++t) {
      int2 r = make_int2(0, (int)n[t]);
      QBX_CUDA_TRY(cudaMemcpy(B.rng[t].ptr, &r, sizeof(r), cudaMemcpyHostToDevice));
    }
  }
  KeySet ks;
  for (int t = 0; t < PT_COUNT; ++t) ks.k[t] = f->keys[t].ptr;
  std::vector<int> loff = {0, 1};
  int level = 0;
  while (true) {
    const int off = loff[level], nb = loff[level + 1] - loff[level];
    DevBuf<int> nch, choff;
    QBX_CUDA_TRY(nch.alloc(nb));
    QBX_CUDA_TRY(choff.alloc(nb));
    split_count_kernel<<<nblk(nb, 128), 128>>>(nb, off, level, n_max, ks, B.key.ptr,
                                               B.rng[0].ptr, B.rng[1].ptr, B.rng[2].ptr,
                                               B.rng[3].ptr, crad_sorted.ptr,
                                               side / (double)(1 << (level + 1)), kappa, nch.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    TRY(scan(nch.ptr, choff.ptr, nb));
    int last_off = 0, last_cnt = 0;
    QBX_CUDA_TRY(cudaMemcpy(&last_off, choff.ptr + nb - 1, sizeof(int), cudaMemcpyDeviceToHost));
    QBX_CUDA_TRY(cudaMemcpy(&last_cnt, nch.ptr + nb - 1, sizeof(int), cudaMemcpyDeviceToHost));
    const int nnext = last_off + last_cnt;
    if (nnext == 0) break;
    const int next_off = loff[level + 1];
    const size_t need = (size_t)next_off + nnext;
    if (need > B.level.n) {
      const size_t keep = next_off;
      TRY(grow(B.level, need, keep));
      TRY(grow(B.parent, need, keep));
      TRY(grow(B.ij, need, keep));
      TRY(grow(B.key, need, keep));
      TRY(grow(B.centre, need, keep));
      for (int t = 0; t < PT_COUNT; ++t) TRY(grow(B.rng[t], need, keep));
      TRY(grow(B.child, 4 * B.level.n, 4 * keep));
    }
    split_fill_kernel<<<nblk(nb, 128), 128>>>(nb, off, level, next_off, ks, nch.ptr, choff.ptr,
                                              f->x0, f->y0, side, B.level.ptr, B.parent.ptr,
                                              B.child.ptr, B.ij.ptr, B.key.ptr, B.centre.ptr,
                                              B.rng[0].ptr, B.rng[1].ptr, B.rng[2].ptr,
                                              B.rng[3].ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    loff.push_back(next_off + nnext);
    ++level;
  }
  f->level_off = loff;
  f->h_level_off = loff;
  f->n_levels = (int)loff.size() - 1;
  f->n_boxes = loff.back();
  return QBX_OK;
}

qbx_status tree_lists(qbx_handle* h, FmmPlan* f) {
  (void)h;
  const int nb = f->n_boxes;
  DevBuf<int> loff;
  QBX_CUDA_TRY(loff.alloc(f->level_off.size()));
  QBX_CUDA_TRY(cudaMemcpy(loff.ptr, f->level_off.data(), f->level_off.size() * sizeof(int),
                          cudaMemcpyHostToDevice));
  TreeView T = view(f, loff);
  DevBuf<int> uc, vc, wc;
  QBX_CUDA_TRY(uc.alloc(nb));
  QBX_CUDA_TRY(vc.alloc(nb));
  QBX_CUDA_TRY(wc.alloc(nb));
  QBX_CUDA_TRY(f->err.alloc(4));
  QBX_CUDA_TRY(cudaMemset(f->err.ptr, 0, 4 * sizeof(int)));
  lists_kernel<false><<<nblk(nb, 128), 128>>>(nb, T, uc.ptr, vc.ptr, wc.ptr, nullptr, nullptr,
                                              nullptr, nullptr, nullptr, nullptr, nullptr,
                                              f->err.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  TRY(counts_to_offsets(uc.ptr, f->U.off, nb, &f->U.nnz));
  TRY(counts_to_offsets(vc.ptr, f->V.off, nb, &f->V.nnz));
  TRY(counts_to_offsets(wc.ptr, f->W.off, nb, &f->W.nnz));
  QBX_CUDA_TRY(f->U.idx.alloc(std::max<int64_t>(1, f->U.nnz)));
  QBX_CUDA_TRY(f->V.idx.alloc(std::max<int64_t>(1, f->V.nnz)));
  QBX_CUDA_TRY(f->V_cls.alloc(std::max<int64_t>(1, f->V.nnz)));
  QBX_CUDA_TRY(f->W.idx.alloc(std::max<int64_t>(1, f->W.nnz)));
  lists_kernel<true><<<nblk(nb, 128), 128>>>(nb, T, nullptr, nullptr, nullptr, f->U.off.ptr,
                                             f->V.off.ptr, f->W.off.ptr, f->U.idx.ptr,
                                             f->V.idx.ptr, f->V_cls.ptr, f->W.idx.ptr,
                                             f->err.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  // X = transpose of W
  DevBuf<int> xc;
  QBX_CUDA_TRY(xc.alloc(nb));
  QBX_CUDA_TRY(cudaMemset(xc.ptr, 0, nb * sizeof(int)));
  xcount_kernel<<<nblk(nb, 128), 128>>>(nb, f->W.off.ptr, f->W.idx.ptr, xc.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  TRY(counts_to_offsets(xc.ptr, f->X.off, nb, &f->X.nnz));
  QBX_CUDA_TRY(f->X.idx.alloc(std::max<int64_t>(1, f->X.nnz)));
  DevBuf<int> cur;
  QBX_CUDA_TRY(cur.alloc(nb + 1));
  QBX_CUDA_TRY(cudaMemcpy(cur.ptr, f->X.off.ptr, nb * sizeof(int), cudaMemcpyDeviceToDevice));
  xfill_kernel<<<nblk(nb, 128), 128>>>(nb, f->W.off.ptr, f->W.idx.ptr, cur.ptr, f->X.idx.ptr);
  sort_lists_kernel<<<nblk(nb, 128), 128>>>(nb, f->X.off.ptr, f->X.idx.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  int herr = 0;
  QBX_CUDA_TRY(cudaMemcpy(&herr, f->err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) {
    set_error("interaction lists: traversal stack overflow (tree too deep/unbalanced)");
    return QBX_ERR_ARG;
  }
  // host-side bookkeeping of box classes (leaves, parents per level, V and X boxes)
  std::vector<int> child(4 * (size_t)nb), voff(nb + 1), xoff(nb + 1);
  QBX_CUDA_TRY(cudaMemcpy(child.data(), f->box.child.ptr, child.size() * sizeof(int),
                          cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(voff.data(), f->V.off.ptr, voff.size() * sizeof(int),
                          cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(xoff.data(), f->X.off.ptr, xoff.size() * sizeof(int),
                          cudaMemcpyDeviceToHost));
  std::vector<int> leaves, nonleaf, vbox, xbox;
  f->nonleaf_off.assign(f->n_levels + 1, 0);
  f->vbox_off.assign(f->n_levels + 1, 0);
  f->xbox_off.assign(f->n_levels + 1, 0);
  for (int l = 0; l < f->n_levels; ++l) {
    f->nonleaf_off[l] = (int)nonleaf.size();
    f->vbox_off[l] = (int)vbox.size();
    f->xbox_off[l] = (int)xbox.size();
    for (int b = f->level_off[l]; b < f->level_off[l + 1]; ++b) {
      bool leaf = child[4 * b] < 0 && child[4 * b + 1] < 0 && child[4 * b + 2] < 0 &&
                  child[4 * b + 3] < 0;
      (leaf ? leaves : nonleaf).push_back(b);
      if (voff[b + 1] > voff[b]) vbox.push_back(b);
      if (xoff[b + 1] > xoff[b]) xbox.push_back(b);
    }
  }
  f->nonleaf_off[f->n_levels] = (int)nonleaf.size();
  f->vbox_off[f->n_levels] = (int)vbox.size();
  f->xbox_off[f->n_levels] = (int)xbox.size();
  f->n_leaves = (int)leaves.size();
  f->n_vbox = (int)vbox.size();
  f->n_xbox = (int)xbox.size();
  auto up = [](DevBuf<int>& d, const std::vector<int>& v) -> qbx_status {
    QBX_CUDA_TRY(d.alloc(std::max<size_t>(1, v.size())));
    if (!v.empty())
      QBX_CUDA_TRY(cudaMemcpy(d.ptr, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
    return QBX_OK;
  };
  TRY(up(f->leaves, leaves));
  TRY(up(f->nonleaf, nonleaf));
  TRY(up(f->vbox, vbox));
  TRY(up(f->xbox, xbox));
  return QBX_OK;
}

qbx_status tree_associate(qbx_handle* h, FmmPlan* f, const int64_t* on_node, const int8_t* on_side,
                          double eps) {
  if (h->n_tgt == 0) return QBX_OK;
  DevBuf<int> loff;
  QBX_CUDA_TRY(loff.alloc(f->level_off.size()));
  QBX_CUDA_TRY(cudaMemcpy(loff.ptr, f->level_off.data(), f->level_off.size() * sizeof(int),
                          cudaMemcpyHostToDevice));
  TreeView T = view(f, loff);
  const double rq_ctr = (1.0 + eps) * 0.5 * h->h_max;
  const double rq_node = 0.25 * h->h_max;
  associate_tree_kernel<<<nblk(h->n_tgt, 128), 128>>>(
      h->n_tgt, h->tgt_xy.ptr, on_node, on_side, h->n_nodes, h->node_xy.ptr, h->panel_h.ptr, h->q,
      h->ctr_xy.ptr, h->ctr_r.ptr, eps, rq_ctr, rq_node, T, f->box.centre.ptr, f->side,
      f->box.rng[PT_CTR].ptr, f->box.rng[PT_NODE].ptr, f->perm[PT_CTR].ptr, f->perm[PT_NODE].ptr,
      h->assoc.ptr, h->counters.ptr, f->err.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  int herr = 0;
  QBX_CUDA_TRY(cudaMemcpy(&herr, f->err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr & 2) {
    set_error("target association: traversal stack overflow");
    return QBX_ERR_ARG;
  }
  return QBX_OK;
}

// gathers used by the plan (sorted copies of particle data)
qbx_status gather_sorted(qbx_handle* h, FmmPlan* f) {
  auto g2 = [](DevBuf<double2>& dst, const double* src, const DevBuf<int>& perm,
               int64_t n) -> qbx_status {
    QBX_CUDA_TRY(dst.alloc(std::max<int64_t>(1, n)));
    if (n) {
      gather_kernel<double2><<<nblk(n, 256), 256>>>(n, perm.ptr, (const double2*)src, dst.ptr);
      QBX_CUDA_TRY(cudaGetLastError());
    }
    return QBX_OK;
  };
  TRY(g2(f->s_xy, h->src_xy.ptr, f->perm[PT_SRC], h->n_src));
  TRY(g2(f->s_nrm, h->src_nrm.ptr, f->perm[PT_SRC], h->n_src));
  TRY(g2(f->c_xy, h->ctr_xy.ptr, f->perm[PT_CTR], h->n_ctr));
  TRY(g2(f->t_xy, h->tgt_xy.ptr, f->perm[PT_TGT], h->n_tgt));
  QBX_CUDA_TRY(f->c_r.alloc(std::max<int64_t>(1, h->n_ctr)));
  if (h->n_ctr) {
    gather_kernel<double><<<nblk(h->n_ctr, 256), 256>>>(h->n_ctr, f->perm[PT_CTR].ptr,
                                                        h->ctr_r.ptr, f->c_r.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  QBX_CUDA_TRY(f->t_assoc.alloc(std::max<int64_t>(1, h->n_tgt)));
  if (h->n_tgt) {
    gather_kernel<int><<<nblk(h->n_tgt, 256), 256>>>(h->n_tgt, f->perm[PT_TGT].ptr,
                                                     (const int*)h->assoc.ptr, f->t_assoc.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
  }
  return QBX_OK;
}
