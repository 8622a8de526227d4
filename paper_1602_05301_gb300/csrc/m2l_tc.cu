// M2L of the FP64 path (Sec. 7.2, Stage 4) on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory).
//
// The translation of one (level, offset class) is a dense complex Q x Q matrix
// applied to the multipoles of every V-list source of that class. It is done
// on the sigma-normalised operators of the mixed path (entries of order one
// or smaller, so that a bound relative to the largest entry of a row is also a
// relative one), written as a real 2Q x 2Q matrix A acting on the real vector
// x = (Re mu, Im mu). FP64 accuracy comes from an error-free split into bf16
// slices (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59 (2012)):
//
//  * every matrix row j is scaled by 2^-f_j and every vector by 2^-e so that
//    its largest entry lies in [1/4, 1/2); the scaled value times 2^(beta S) is
//    rounded to an integer Z and written in S signed base-2^beta digits,
//    Z = sum_i d_i 2^(beta (S - i)), |d_i| <= 2^(beta-1): each digit is a bf16
//    integer, exact;
//  * the products of digit slices (i, j) with i + j = s carry the same weight
//    2^(-beta s); for each s = 2 .. S + 1 one TMEM accumulator sums all of them
//    over k. Every partial sum is an integer of magnitude at most
//    S K 2^(2 beta - 2) <= 2^24, so the FP32 accumulation is exact;
//  * the S group sums are combined in float-float (two FP32 words, 48 bits),
//    scaled by 2^(e + f_j), added over each target box's V list in
//    float-float, and converted to FP64 once per coefficient.
// Slice pairs with i + j > S + 1 are dropped: the truncation error is about
// S 2^(-beta S) of the largest term, 2^-46 or below for the (beta, S) used
// (beta S >= 48).
//
// Work mapping: a CTA takes 128 V pairs of one group (the MMA's M) and 64 real
// output orders (N = 64). Operand tiles of 32 input orders (two MMAs of K = 16)
// are staged through shared memory in the no-swizzle K-major layout (8 x 16-byte
// core matrices), double-buffered; one thread issues the MMAs, an mbarrier
// tracks their completion (tcgen05.commit), and all waits are bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "tree.cuh"
#include "m2l_entry.cuh"

#define TRY_TC(x)               \
  do {                          \
    const qbx_status s_ = (x);  \
    if (s_ != QBX_OK) return s_; \
  } while (0)

namespace {
template <typename T>
qbx_status upload(DevBuf<T>& d, const std::vector<T>& v) {
  QBX_CUDA_TRY(d.alloc(std::max<size_t>(1, v.size())));
  if (!v.empty())
    QBX_CUDA_TRY(cudaMemcpy(d.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return QBX_OK;
}
}  // namespace

namespace {

constexpr int kRows = 128;      // V pairs per CTA (MMA M)
constexpr int kNC = 64;         // real outputs per CTA (MMA N)
constexpr int kKC = 32;         // real inputs per staging chunk
constexpr int kPad = 64;        // 2Q is padded to a multiple of this (K and N)
constexpr int kThr = 128;
// Every mbarrier wait is bounded twice: by a deadline on the global timer
// (kWaitNs; each try_wait itself returns after a system-dependent suspension
// limit) and by an iteration count.
constexpr long long kSpin = 1LL << 26;
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s

inline unsigned nblk(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance of
// core matrices adjacent in K, sbo = of core matrices adjacent in M/N
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: bf16 A and B (K-major), f32 D, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t id,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(id), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar)));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the given phase parity of an mbarrier; false when the
// deadline (limit_ns from the first call) or the iteration bound ran out
// sleep_ns > 0: a waiter off the critical path (a whole warp waiting for the
// next accumulators, a producer ahead of the MMAs) sleeps between tries and
// leaves its scheduler's issue slots to the warps that work
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs,
                                          unsigned sleep_ns = 0) {
  const unsigned long long t0 = global_ns();
  for (long long it = 0; it < kSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
    if (sleep_ns) __nanosleep(sleep_ns);
  }
  return false;
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without the wait: several loads in flight, one
// tcgen05.wait::ld, then reg_fence16 on each destination so that nothing
// reads the registers before the wait
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;"); }
__device__ __forceinline__ void reg_fence16(uint32_t (&r)[16]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]));
}
// 2^e as an FP32 for -126 <= e <= 127 (0 outside: callers fall back to ldexpf)
__device__ __forceinline__ float exp2i(int e) {
  return (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : 0.f;
}

// ---------------------------------------------------------------- float-float
// s + e = a + b exactly (Knuth's TwoSum; additions only, so no contraction)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (hi, lo) += (bh, bl), renormalised
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e += lo + bl;
  hi = s + e;
  lo = e - (hi - s);
}

// ---------------------------------------------------------------- slicing
// The S signed base-2^beta digits of rint(x 2^(beta S - e)) (|x| 2^-e < 1/2),
// most significant first, as bf16 (exact: |d| <= 2^(beta - 1) <= 128): the
// lower S - 1 digits in [-2^(beta-1), 2^(beta-1)), the top one whatever is left,
// which is at most 2^(beta - 1) in magnitude since |rint(x 2^(beta S - e))| <=
// 2^(beta S - 1).
__device__ __forceinline__ void split_digits(double x, int e, int beta, int S,
                                             __nv_bfloat16* __restrict__ out, size_t stride) {
  long long Z = __double2ll_rn(ldexp(x, beta * S - e));
  const long long half = 1LL << (beta - 1), mask = (1LL << beta) - 1;
  for (int i = S - 1; i >= 1; --i) {
    long long d = Z & mask;
    if (d >= half) d -= mask + 1;
    Z = (Z - d) >> beta;
    out[(size_t)i * stride] = __float2bfloat16_rn((float)d);
  }
  // the top digit takes the rest, |Z| <= 2^(beta - 1) (no carry is dropped)
  out[0] = __float2bfloat16_rn((float)Z);
}
// exponent e with max_abs 2^-e in [1/4, 1/2) (0 for max_abs == 0)
__device__ __forceinline__ int scale_exponent(double max_abs) {
  if (!(max_abs > 0.0)) return 0;
  int E;
  frexp(max_abs, &E);  // max_abs = m 2^E, m in [1/2, 1)
  return E + 1;
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  __syncthreads();
  return m;
}

// Matrix slices of one group (level l, class cls), row j of the real form:
//   A[j][k] = Re T[n][lo] (j < Q, k < Q), -Im T[n][lo] (j < Q, k >= Q),
//             Im T[n][lo] (j >= Q, k < Q), Re T[n][lo] (j >= Q, k >= Q),
// lo = j mod Q, n = k mod Q, T the sigma-normalised M2L matrix; zero padding.
// Grid (used groups, Np), threads over k. Slices [S][Np][Kp] at aoff.
__global__ void __launch_bounds__(kThr) tc_matrix_kernel(
    const int* __restrict__ groups, const long long* __restrict__ aoff,
    const long long* __restrict__ foff, const int4* __restrict__ lvl, const int* __restrict__ lpb,
    int pbmax, const cd* __restrict__ t_m2l, const double* __restrict__ scale,
    const double* __restrict__ lsig, __nv_bfloat16* __restrict__ A, int* __restrict__ fexp) {
  __shared__ double red[kThr / 32];
  const int g = groups[blockIdx.x];
  const int l = g / 49, cls = g % 49;
  const int4 P = lvl[l];  // (use, beta, S, Kp)
  const int Kp = P.w, beta = P.y, S = P.z;
  const int pb = lpb[l], Q = 2 * pb + 1;
  const int j = blockIdx.y;
  if (j >= Kp) return;
  const int lo = (j < Q ? j : j - Q) - pb;
  const bool im_out = j >= Q;
  const M2lNorm nm(t_m2l, scale, lsig, l, cls, pbmax);
  double vals[16];  // k = threadIdx.x + 128 t, Kp <= 2048
  double m = 0.0;
  for (int t = 0; t < 16; ++t) {
    const int k = threadIdx.x + kThr * t;
    double v = 0.0;
    if (j < 2 * Q && k < 2 * Q) {
      const int n = (k < Q ? k : k - Q) - pb;
      const cd T = nm.entry(n, lo);
      const bool im_in = k >= Q;
      v = im_out ? (im_in ? T.x : T.y) : (im_in ? -T.y : T.x);
    }
    vals[t] = v;
    m = fmax(m, fabs(v));
  }
  m = block_max(m, red);
  const int e = scale_exponent(m);
  if (threadIdx.x == 0) fexp[foff[blockIdx.x] + j] = e;
  __nv_bfloat16* dst = A + aoff[blockIdx.x] + (size_t)j * Kp;
  for (int t = 0; t < 16; ++t) {
    const int k = threadIdx.x + kThr * t;
    if (k < Kp) split_digits(vals[t], e, beta, S, dst + k, (size_t)Kp * Kp);
  }
}

// Vector slices of the V-list sources: mu_n = mh_n conv_|n| (FP64), x = (Re mu,
// Im mu) padded to Kp, one exponent per box. One block per box.
__global__ void __launch_bounds__(kThr) tc_mu_kernel(
    const int* __restrict__ boxes, const int* __restrict__ level, const int* __restrict__ lpb,
    const long long* __restrict__ eoff, const double* __restrict__ conv, int pbmax,
    const int4* __restrict__ lvl, const cd* __restrict__ mpole, const long long* __restrict__ xoff,
    __nv_bfloat16* __restrict__ X, int* __restrict__ xexp) {
  __shared__ double red[kThr / 32];
  const int b = boxes[blockIdx.x];
  const int l = level[b];
  const int4 P = lvl[l];
  const int Kp = P.w, beta = P.y, S = P.z;
  const int pb = lpb[l], Q = 2 * pb + 1;
  const double* cv = conv + (size_t)l * (pbmax + 1);
  const cd* a = mpole + eoff[b];
  double vals[16];  // Kp <= 2048
  double m = 0.0;
  for (int t = 0; t < 16; ++t) {
    const int k = threadIdx.x + kThr * t;
    double v = 0.0;
    if (k < 2 * Q) {
      const int n = k < Q ? k : k - Q;
      const cd c = a[n];
      v = (k < Q ? c.x : c.y) * cv[abs(n - pb)];
    }
    vals[t] = v;
    m = fmax(m, fabs(v));
  }
  m = block_max(m, red);
  const int e = scale_exponent(m);
  if (threadIdx.x == 0) xexp[blockIdx.x] = e;
  __nv_bfloat16* dst = X + xoff[blockIdx.x];
  for (int t = 0; t < 16; ++t) {
    const int k = threadIdx.x + kThr * t;
    if (k < Kp) split_digits(vals[t], e, beta, S, dst + k, (size_t)Kp);
  }
}

// Matrix slices of the four quadrant groups of one parent level l of M2M
// (kind 0: child orders in, parent orders out) or L2L (kind 1: parent orders
// in, child orders out), from the FP64 tables of conj(V_m) (M2M) and
// (-1)^m V_m (L2L) of the quadrant's shift, sigma-normalised:
//   M2M  T[so][n] = (sig_{l+1,|n|} / sig_{l,|so|}) conj(V_{so-n}),
//   L2L  T[so][n] = (sig_{l+1,|so|} / sig_{l,|n|}) (-1)^{so-n} V_{so-n},
// in the real form of tc_matrix_kernel. Grid (4, Np), threads over k < K.
// Slices [quadrant][S][Np][K], row exponents [quadrant][Np].
__global__ void __launch_bounds__(kThr) tc_mml_matrix_kernel(
    int kind, int l, int pp, int pc, int pbmax, const cd* __restrict__ tab,
    const double* __restrict__ lsig, int K, int Np, int beta, int S, __nv_bfloat16* __restrict__ A,
    int* __restrict__ fexp) {
  __shared__ double red[kThr / 32];
  const int c = blockIdx.x, j = blockIdx.y;
  const int pin = kind == 0 ? pc : pp, pout = kind == 0 ? pp : pc;
  const int Qin = 2 * pin + 1, Qout = 2 * pout + 1;
  const cd* v = tab + ((size_t)l * 4 + c) * (4 * pbmax + 1) + 2 * pbmax;
  const double* sp = lsig + (size_t)l * (pbmax + 1);        // parent level
  const double* sc = lsig + (size_t)(l + 1) * (pbmax + 1);  // child level
  const int so = (j < Qout ? j : j - Qout) - pout;
  const bool im_out = j >= Qout;
  double vals[16];  // k = threadIdx.x + 128 t, K <= 2048
  double m = 0.0;
  for (int t = 0; t < 16; ++t) {
    const int k = threadIdx.x + kThr * t;
    double val = 0.0;
    if (j < 2 * Qout && k < 2 * Qin) {
      const int n = (k < Qin ? k : k - Qin) - pin;
      const cd e = v[so - n];
      const double mag = hypot(e.x, e.y);
      cd T = mk(0.0, 0.0);
      if (mag > 0.0) {
        const double lf = (kind == 0 ? sc[abs(n)] - sp[abs(so)] : sc[abs(so)] - sp[abs(n)]) + log(mag);
        const double f = lf < -700.0 ? 0.0 : exp(lf) / mag;
        T = mk(e.x * f, e.y * f);
      }
      const bool im_in = k >= Qin;
      val = im_out ? (im_in ? T.x : T.y) : (im_in ? -T.y : T.x);
    }
    vals[t] = val;
    m = fmax(m, fabs(val));
  }
  m = block_max(m, red);
  const int e = scale_exponent(m);
  if (threadIdx.x == 0) fexp[(size_t)c * Np + j] = e;
  __nv_bfloat16* dst = A + (size_t)c * S * Np * K + (size_t)j * K;
  for (int t = 0; t < 16; ++t) {
    const int k = threadIdx.x + kThr * t;
    if (k < K) split_digits(vals[t], e, beta, S, dst + k, (size_t)Np * K);
  }
}

// Vector slices of the source boxes of one M2M / L2L level: M2M the children's
// multipoles mu_n = mh_n conv_|n| (level l+1), L2L the parents' locals
// lambda_n = lh_n / conv_|n| (level l); x = (Re, Im) padded to K, one exponent
// per box, slices [S][K] at xoff[i]. One block per source box.
__global__ void __launch_bounds__(kThr) tc_mml_vec_kernel(
    int kind, const int* __restrict__ boxes, const cd* __restrict__ coef, int lsrc, int pb, int K,
    int beta, int S, const double* __restrict__ conv, int pbmax, const long long* __restrict__ eoff,
    const long long* __restrict__ xoff, __nv_bfloat16* __restrict__ X, int* __restrict__ xexp) {
  __shared__ double red[kThr / 32];
  const int b = boxes[blockIdx.x];
  const int Q = 2 * pb + 1;
  const double* cv = conv + (size_t)lsrc * (pbmax + 1);
  const cd* a = coef + eoff[b];
  double vals[16];  // K <= 2048
  double m = 0.0;
  for (int t = 0; t < 16; ++t) {
    const int k = threadIdx.x + kThr * t;
    double v = 0.0;
    if (k < 2 * Q) {
      const int n = k < Q ? k : k - Q;
      const double f = kind == 0 ? cv[abs(n - pb)] : 1.0 / cv[abs(n - pb)];
      v = (k < Q ? a[n].x : a[n].y) * f;
    }
    vals[t] = v;
    m = fmax(m, fabs(v));
  }
  m = block_max(m, red);
  const int e = scale_exponent(m);
  if (threadIdx.x == 0) xexp[blockIdx.x] = e;
  __nv_bfloat16* dst = X + xoff[blockIdx.x];
  for (int t = 0; t < 16; ++t) {
    const int k = threadIdx.x + kThr * t;
    if (k < K) split_digits(vals[t], e, beta, S, dst + k, (size_t)K);
  }
}

// M2M: mh_p[so] = (sum over the parent's child rows, quadrant order, float-float)
// / conv_l[|so|]. prow[i][c]: the row of parent i's quadrant-c child (-1: none).
__global__ void __launch_bounds__(kThr) tc_m2m_reduce_kernel(
    const int* __restrict__ parents, const int* __restrict__ prow, int pp, int l, int pbmax,
    const double* __restrict__ conv, const cd* __restrict__ Y, const long long* __restrict__ eoff,
    cd* __restrict__ mpole) {
  const int i = blockIdx.x;
  const int Q = 2 * pp + 1;
  const double* cv = conv + (size_t)l * (pbmax + 1);
  cd* dst = mpole + eoff[parents[i]];
  for (int lo = threadIdx.x; lo < Q; lo += kThr) {
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int c = 0; c < 4; ++c) {
      const int r = prow[4 * i + c];
      if (r < 0) continue;
      const float4 y = reinterpret_cast<const float4*>(Y)[(size_t)r * Q + lo];
      ff_add(rh, rl, y.x, y.y);
      ff_add(ih, il, y.z, y.w);
    }
    const double f = 1.0 / cv[abs(lo - pp)];
    dst[lo] = mk(((double)rh + (double)rl) * f, ((double)ih + (double)il) * f);
  }
}

// L2L: lh_child[so] += row value * conv_{l+1}[|so|]. One block per row (child).
__global__ void __launch_bounds__(kThr) tc_l2l_apply_kernel(
    const int* __restrict__ rowdst, int pc, int lc, int pbmax, const double* __restrict__ conv,
    const cd* __restrict__ Y, const long long* __restrict__ eoff, cd* __restrict__ local) {
  const int r = blockIdx.x;
  const int Q = 2 * pc + 1;
  const double* cv = conv + (size_t)lc * (pbmax + 1);
  cd* dst = local + eoff[rowdst[r]];
  for (int lo = threadIdx.x; lo < Q; lo += kThr) {
    const float4 y = reinterpret_cast<const float4*>(Y)[(size_t)r * Q + lo];
    const double f = cv[abs(lo - pc)];
    dst[lo] = cadd(dst[lo], mk(((double)y.x + (double)y.y) * f, ((double)y.z + (double)y.w) * f));
  }
}

// 16-byte asynchronous copy global -> shared (zero fill when bytes == 0)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

// Stages of the shared-memory ring for SU slices in use: as many as fit in
// 220 KB, at most 4.
__host__ __device__ constexpr int tc_stages(int SU) {
  return (220 * 1024) / (SU * (kRows + kNC) * kKC * 2) >= 4
             ? 4
             : (220 * 1024) / (SU * (kRows + kNC) * kKC * 2);
}

// The tile product. A group is one operator: a (level, offset class) of M2L
// or a (level, quadrant) of M2M / L2L, with gp[group] = (K, Q, beta, Np): the
// padded input width (slice stride of X, row stride of A), Q complex outputs
// (2Q real rows of A, padded to Np), the digit bits. Item (first row, rows,
// first output, group). SD slices are
// stored per operand (the level's split), the first SU of them are used: SU =
// SD for the FP64 path, fewer for the mixed path (the leading digits are a
// 24- to 28-bit approximation). Y receives, for each pair row and complex
// output lo, (Re hi, Re lo, Im hi, Im lo) as float4 at yoff[row] + lo: the
// float-float value of (A x)_j 2^(e + f_j).
//
// Pipeline: NS shared-memory stages filled by cp.async (every thread copies
// 16-byte pieces; rows past the tile's end are zero-filled); chunk c is
// consumed when its copy group has landed (cp.async.wait_group), after a proxy
// fence and a barrier; one thread issues its MMAs and commits them to the
// stage's mbarrier; then, with those MMAs queued behind the previous chunk's,
// the threads wait for chunk c - 1's MMAs and refill that stage with chunk
// c + NS - 1.
template <int SD, int SU>
__global__ void __launch_bounds__(kThr, 1) m2l_tc_kernel(
    const int4* __restrict__ items, const int4* __restrict__ gp,
    const long long* __restrict__ gaoff, const long long* __restrict__ gfoff,
    const __nv_bfloat16* __restrict__ A, const int* __restrict__ fexp,
    const int* __restrict__ rowsrc, const long long* __restrict__ xoff,
    const int* __restrict__ xexp, const __nv_bfloat16* __restrict__ X,
    const long long* __restrict__ yoff, cd* __restrict__ Y, int* __restrict__ err) {
  constexpr int NS = tc_stages(SU);
  static_assert(NS >= 2, "at least two stages");
  constexpr int XT = kRows * kKC;             // elements of one X slice tile
  constexpr int AT = kNC * kKC;               // elements of one A slice tile
  constexpr int STAGE = SU * (XT + AT);       // elements of one stage
  constexpr uint32_t LBO = 128;               // core matrices adjacent in K: contiguous
  constexpr uint32_t SBO = (kKC / 8) * 128;   // next 8-row group
  constexpr uint32_t ID = idesc_bf16(kRows, kNC);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __shared__ __align__(8) uint64_t mbar[NS + 1];  // a stage's MMAs; [NS]: all MMAs
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ long long s_xrow[kRows];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 I = items[blockIdx.x];
  const int row0 = I.x, nr = I.y, n0 = I.z, g = I.w;
  // group: K (padded input width; slice stride of X and of an A row), Q
  // complex outputs, digit bits, Np (padded output rows of A)
  const int4 G = gp[g];
  const int Kp = G.x, Q = G.y, beta = G.z, Np = G.w;
  const __nv_bfloat16* Ag = A + gaoff[g];
  const int* fg = fexp + gfoff[g];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    for (int b = 0; b <= NS; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[b])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int nchunks = Kp / kKC;
  // slice offset of every row's source (-1 past the tile's end), read once
  for (int m = tid; m < kRows; m += kThr) s_xrow[m] = m < nr ? xoff[rowsrc[row0 + m]] : -1;
  __syncthreads();
  // 16-byte pieces: a warp's 32 pieces fill four whole 128-byte core matrices
  // (8 rows x 4 k-groups), so its shared-memory writes are free of conflicts
  auto load_chunk = [&](int c) {
    __nv_bfloat16* xs = stg + (size_t)(c % NS) * STAGE;
    __nv_bfloat16* as = xs + SU * XT;
    const int k0 = c * kKC;
    for (int i = tid; i < kRows * SU * 4; i += kThr) {
      const int r = i >> 5, t = r % SU, m = (r / SU) * 8 + (i & 7), q = (i >> 3) & 3;
      const long long xo = s_xrow[m];
      const __nv_bfloat16* src = xo >= 0 ? X + xo + (size_t)t * Kp + k0 + q * 8 : X;
      cp_async16(reinterpret_cast<char*>(xs + t * XT) + (m >> 3) * SBO + q * LBO + (m & 7) * 16,
                 src, xo >= 0 ? 16 : 0);
    }
    for (int i = tid; i < kNC * SU * 4; i += kThr) {
      const int r = i >> 5, t = r % SU, j = (r / SU) * 8 + (i & 7), q = (i >> 3) & 3;
      cp_async16(reinterpret_cast<char*>(as + t * AT) + (j >> 3) * SBO + q * LBO + (j & 7) * 16,
                 Ag + ((size_t)t * Np + (n0 + j)) * Kp + k0 + q * 8, 16);
    }
  };
  for (int c = 0; c < NS - 1; ++c) {  // prologue: NS - 1 groups (empty past the end)
    if (c < nchunks) load_chunk(c);
    cp_async_commit();
  }
  uint32_t acc_started = 0;  // accumulators written at least once (issuing thread)
  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    cp_async_wait<NS - 2>();  // chunk c's group has landed (this thread's copies)
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      const __nv_bfloat16* xs = stg + (size_t)(c % NS) * STAGE;
      const __nv_bfloat16* as = xs + SU * XT;
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int ti = 0; ti < SU; ++ti) {
#pragma unroll
        for (int tj = 0; tj < SU - ti; ++tj) {
          const int a = ti + tj;  // weight 2^(-beta (a + 2))
#pragma unroll
          for (int kk = 0; kk < kKC; kk += 16) {
            const uint64_t da = smem_desc(smem_u32(xs + ti * XT) + (kk / 8) * LBO, LBO, SBO);
            const uint64_t db = smem_desc(smem_u32(as + tj * AT) + (kk / 8) * LBO, LBO, SBO);
            mma_bf16(tmem + a * kNC, da, db, ID, (acc_started >> a) & 1u);
            acc_started |= 1u << a;
          }
        }
      }
      mma_commit(&mbar[c % NS]);
    }
    // refill the stage of chunk c - 1 once its MMAs are done
    const int cn = c + NS - 1;
    if (cn < nchunks) {
      if (c >= 1 && !mbar_wait(&mbar[(c - 1) % NS], ((c - 1) / NS) & 1)) atomicExch(&s_fail, 1);
      __syncthreads();
      if (s_fail) { ok = false; break; }
      load_chunk(cn);
    }
    cp_async_commit();
  }
  cp_async_wait<0>();
  // all MMAs complete: the last chunk's commit covers every earlier one; wait
  // for the earlier stages' last commits too so that no arrival is pending
  if (ok) {
    for (int c = std::max(0, nchunks - NS); c < nchunks; ++c)
      if (!mbar_wait(&mbar[c % NS], (c / NS) & 1)) atomicExch(&s_fail, 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  if (s_fail) {
    // a wait ran out: flag it, then give the MMAs issued so far a bounded
    // wait (one commit tracks them all) before the tensor memory is freed
    if (tid == 0) {
      atomicExch(err, 1);
      mma_commit(&mbar[NS]);
    }
    mbar_wait(&mbar[NS], 0);
  } else {
    // epilogue: warp w holds rows 32w .. 32w + 31 (TMEM lanes)
    const int m = warp * 32 + lane;
    const bool row_ok = m < nr;
    const int e_row = row_ok ? xexp[rowsrc[row0 + m]] : 0;
    const long long yo = row_ok ? yoff[row0 + m] : 0;
    for (int j0 = 0; j0 < kNC; j0 += 16) {
      float hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0.f;
#pragma unroll
      for (int a = SU - 1; a >= 0; --a) {  // smallest weight first
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + a * kNC + j0, v);
        const int sh = -beta * (a + 2);
#pragma unroll
        for (int c = 0; c < 16; ++c) ff_add(hi[c], lo[c], ldexpf(v[c], sh), 0.f);
      }
      if (row_ok) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = n0 + j0 + c;
          if (j >= 2 * Q) break;
          const int sc = e_row + fg[j];
          const float2 w = make_float2(ldexpf(hi[c], sc), ldexpf(lo[c], sc));
          float2* dst = reinterpret_cast<float2*>(Y + yo + (j < Q ? j : j - Q)) + (j < Q ? 0 : 1);
          *dst = w;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// The same tile product as a persistent, warp-specialised kernel: one CTA per
// SM walks items c, c + G, c + 2G, ... (G CTAs), with
//  * warps 0-2, the producers: fill the shared-memory ring stage by stage with
//    cp.async across item boundaries (they run ahead of the MMAs of the
//    current item into the next one); once a stage's copies have landed each
//    lane fences them for the async proxy and arrives on the stage's full
//    barrier (three warps: one warp could not issue the 16-byte copies of a
//    stage as fast as the MMAs consume it);
//  * warp 3, the MMA warp: allocates the tensor memory; one lane waits for a
//    stage, issues its MMAs and commits them to the stage's empty barrier
//    (the producer's refill waits on it), and after an item's last stage
//    commits to the accumulator-full barrier; before an item's first MMA it
//    waits until the epilogue has read the previous item's accumulators;
//  * warps 4-7, the epilogue: TMEM lanes 32 (w mod 4) .. + 31 (the rows),
//    the float-float combination and the stores of tc's epilogue, then an
//    arrival on the accumulator-empty barrier.
// Every wait is bounded (mbar_wait); a wait that runs out sets the CTA's fail
// flag and the global flag, the roles leave their loops, the issued MMAs are
// drained with one more bounded wait, and the tensor memory is freed.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int kWsProd = 3;                       // producer warps
constexpr int kWsThr = 32 * (kWsProd + 1 + 4);   // producers, MMA warp, four epilogue warps

template <int SD, int SU>
__global__ void __launch_bounds__(kWsThr, 1) tc_gemm_ws_kernel(
    const int4* __restrict__ items, int n_items, const int4* __restrict__ gp,
    const long long* __restrict__ gaoff, const long long* __restrict__ gfoff,
    const __nv_bfloat16* __restrict__ A, const int* __restrict__ fexp,
    const int* __restrict__ rowsrc, const long long* __restrict__ xoff,
    const int* __restrict__ xexp, const __nv_bfloat16* __restrict__ X,
    const long long* __restrict__ yoff, cd* __restrict__ Y, int* __restrict__ err) {
  constexpr int NS = tc_stages(SU);
  static_assert(NS >= 2, "at least two stages");
  constexpr int XT = kRows * kKC, AT = kNC * kKC, STAGE = SU * (XT + AT);
  constexpr uint32_t LBO = 128, SBO = (kKC / 8) * 128;
  constexpr uint32_t ID = idesc_bf16(kRows, kNC);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull, tempty, mfin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ long long s_xrow[kWsProd][kRows];  // each producer warp's copy
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  if (warp == kWsProd) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    for (int b = 0; b < NS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[b])),
                   "r"(32 * kWsProd));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&tempty)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mfin)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  auto fail = [&]() {
    atomicExch(&s_fail, 1);
    atomicExch(err, 1);
  };
  auto failed = [&]() { return *(volatile int*)&s_fail != 0; };

  if (warp < kWsProd) {
    // ---------------- producers (warp w takes every kWsProd-th 16-byte piece)
    long long* xrow = s_xrow[warp];
    const int pt = warp * 32 + lane;
    int q = 0;  // stages filled so far (over all items)
    for (int it = blockIdx.x; it < n_items && !failed(); it += G) {
      const int4 I = items[it];
      const int row0 = I.x, nr = I.y, n0 = I.z;
      const int4 P = gp[I.w];
      const int Kp = P.x, Np = P.w;
      const __nv_bfloat16* Ag = A + gaoff[I.w];
      for (int m = lane; m < kRows; m += 32) xrow[m] = m < nr ? xoff[rowsrc[row0 + m]] : -1;
      __syncwarp();
      const int nchunks = Kp / kKC;
      for (int c = 0; c < nchunks; ++c, ++q) {
        const int slot = q % NS;
        if (q >= NS && !mbar_wait(&empty[slot], ((q / NS) - 1) & 1)) {
          fail();
          break;
        }
        __nv_bfloat16* xs = stg + (size_t)slot * STAGE;
        __nv_bfloat16* as = xs + SU * XT;
        const int k0 = c * kKC;
        for (int i = pt; i < kRows * SU * 4; i += 32 * kWsProd) {
          const int r = i >> 5, t = r % SU, m = (r / SU) * 8 + (i & 7), qq = (i >> 3) & 3;
          const long long xo = xrow[m];
          const __nv_bfloat16* src = xo >= 0 ? X + xo + (size_t)t * Kp + k0 + qq * 8 : X;
          cp_async16(reinterpret_cast<char*>(xs + t * XT) + (m >> 3) * SBO + qq * LBO + (m & 7) * 16,
                     src, xo >= 0 ? 16 : 0);
        }
        for (int i = pt; i < kNC * SU * 4; i += 32 * kWsProd) {
          const int r = i >> 5, t = r % SU, j = (r / SU) * 8 + (i & 7), qq = (i >> 3) & 3;
          cp_async16(reinterpret_cast<char*>(as + t * AT) + (j >> 3) * SBO + qq * LBO + (j & 7) * 16,
                     Ag + ((size_t)t * Np + (n0 + j)) * Kp + k0 + qq * 8, 16);
        }
        cp_async_commit();
        // the stage filled NS - 2 steps ago has landed: hand it to the MMAs
        cp_async_wait<NS - 2>();
        asm volatile("fence.proxy.async.shared::cta;");
        if (q - (NS - 2) >= 0) mbar_arrive(&full[(q - (NS - 2)) % NS]);
      }
      __syncwarp();  // xrow is rewritten for the next item
    }
    // the last NS - 2 stages
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;");
    for (int r = std::max(0, q - (NS - 2)); r < q; ++r) mbar_arrive(&full[r % NS]);
  } else if (warp == kWsProd) {
    // ---------------- MMA issue (lane 0)
    if (lane == 0) {
      int q = 0, k = 0;  // stages consumed, items done
      for (int it = blockIdx.x; it < n_items && !failed(); it += G, ++k) {
        const int4 P = gp[items[it].w];
        const int nchunks = P.x / kKC;
        if (k >= 1 && !mbar_wait(&tempty, (k - 1) & 1)) {  // epilogue has read the last item
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        bool ok = true;
        for (int c = 0; c < nchunks; ++c, ++q) {
          const int slot = q % NS;
          if (!mbar_wait(&full[slot], (q / NS) & 1)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const __nv_bfloat16* xs = stg + (size_t)slot * STAGE;
          const __nv_bfloat16* as = xs + SU * XT;
          // descriptors of the stage's first core matrices; the others differ
          // by a constant in the address field (shared-memory addresses stay
          // below 2^18 bytes, so the 14-bit field cannot carry)
          const uint64_t dx0 = smem_desc(smem_u32(xs), LBO, SBO);
          const uint64_t da0 = smem_desc(smem_u32(as), LBO, SBO);
#pragma unroll
          for (int ti = 0; ti < SU; ++ti) {
#pragma unroll
            for (int tj = 0; tj < SU - ti; ++tj) {
              const int a = ti + tj;
#pragma unroll
              for (int kk = 0; kk < kKC; kk += 16) {
                const uint64_t da = dx0 + (uint64_t)((ti * XT * 2 + (kk / 8) * LBO) >> 4);
                const uint64_t db = da0 + (uint64_t)((tj * AT * 2 + (kk / 8) * LBO) >> 4);
                // an accumulator's first product of an item (ti = 0, kk = 0 of its
                // first stage) overwrites, every later one adds
                mma_bf16(tmem + a * kNC, da, db, ID, (c > 0 || ti > 0 || kk > 0) ? 1u : 0u);
              }
            }
          }
          mma_commit(&empty[slot]);
        }
        if (!ok) {
          fail();
          break;
        }
        mma_commit(&tfull);
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: rows (warp mod 4) * 32 + lane
    const int m = (warp & 3) * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    int k = 0;
    for (int it = blockIdx.x; it < n_items && !failed(); it += G, ++k) {
      const int4 I = items[it];
      const int row0 = I.x, nr = I.y, n0 = I.z, g = I.w;
      const int4 P = gp[g];
      const int Q = P.y, beta = P.z;
      const int* fg = fexp + gfoff[g];
      if (!mbar_wait(&tfull, k & 1)) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const bool row_ok = m < nr;
      const int e_row = row_ok ? xexp[rowsrc[row0 + m]] : 0;
      const long long yo = row_ok ? yoff[row0 + m] : 0;
      for (int j0 = 0; j0 < kNC; j0 += 16) {
        // the SU accumulators of these 16 columns: all loads in flight, one wait
        uint32_t r[SU][16];
#pragma unroll
        for (int a = 0; a < SU; ++a) tmem_ld16_async(tl + a * kNC + j0, r[a]);
        tmem_wait_ld();
#pragma unroll
        for (int a = 0; a < SU; ++a) reg_fence16(r[a]);
        float hi[16], lo[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0.f;
#pragma unroll
        for (int a = SU - 1; a >= 0; --a) {
          const float sa = exp2i(-beta * (a + 2));  // exact: -beta (a + 2) >= -80
#pragma unroll
          for (int c = 0; c < 16; ++c) ff_add(hi[c], lo[c], __uint_as_float(r[a][c]) * sa, 0.f);
        }
        if (j0 + 16 >= kNC) {  // every accumulator read: the MMAs may reuse TMEM
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(&tempty);
        }
        if (row_ok) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int j = n0 + j0 + c;
            if (j >= 2 * Q) break;
            const int sc = e_row + fg[j];
            const float f = exp2i(sc);
            const float2 w = f != 0.f ? make_float2(hi[c] * f, lo[c] * f)
                                      : make_float2(ldexpf(hi[c], sc), ldexpf(lo[c], sc));
            float2* dst = reinterpret_cast<float2*>(Y + yo + (j < Q ? j : j - Q)) + (j < Q ? 0 : 1);
            *dst = w;
          }
        }
      }
    }
  }
  __syncthreads();
  if (s_fail) {  // drain whatever MMAs were issued before the tensor memory goes
    if (warp == kWsProd && lane == 0) mma_commit(&mfin);
    mbar_wait(&mfin, 0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == kWsProd)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// The FP64 M2L's tile product fed by TMA. The source slices of the rows are
// first copied into row order per group (tc_x2_fill_kernel: [S][rows][K], a
// TMA-tileable 2D array); then a single producer lane loads a stage as 4 S
// boxes of 128 rows x 16 bytes (rows) and 4 S boxes of 64 rows x 16 bytes
// (matrix), one per slice and 8-wide k-group, with one expect-tx arrival on
// the stage's full barrier. Shared-memory layout of a slice: k-group kg's
// 128 x 16 B at kg * 2 KB (rows; 1 KB for the matrix's 64), i.e. core matrices
// adjacent in M 128 B apart and in K 2 KB (1 KB) apart. The MMA warp and the
// epilogue warps are those of tc_gemm_ws_kernel.
__global__ void tc_x2_fill_kernel(int n_rows, const long long* __restrict__ src,
                                  const long long* __restrict__ dst,
                                  const long long* __restrict__ tstride,
                                  const int2* __restrict__ sk, const uint16_t* __restrict__ X,
                                  uint16_t* __restrict__ X2) {
  const int r = blockIdx.x;
  if (r >= n_rows) return;
  const int S = sk[r].x, K = sk[r].y, V = K / 8;  // 16-byte vectors per slice row
  const uint4* in = reinterpret_cast<const uint4*>(X + src[r]);
  for (int i = threadIdx.x; i < S * V; i += blockDim.x) {
    const int t = i / V, v = i % V;
    *reinterpret_cast<uint4*>(X2 + dst[r] + (size_t)t * tstride[r] + (size_t)v * 8) = in[(size_t)t * V + v];
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

constexpr int kTmaThr = 32 * 6;  // producer warp (one lane), MMA warp, four epilogue warps

template <int SD, int SU>
__global__ void __launch_bounds__(kTmaThr, 1) tc_gemm_tma_kernel(
    const int4* __restrict__ items, int n_items, const int4* __restrict__ gp,
    const TmapBlob* __restrict__ mapA, const TmapBlob* __restrict__ mapX,
    const long long* __restrict__ gstart, const long long* __restrict__ gfoff,
    const int* __restrict__ fexp, const int* __restrict__ rowsrc, const int* __restrict__ xexp,
    const long long* __restrict__ yoff, cd* __restrict__ Y, int* __restrict__ err) {
  constexpr int NS = tc_stages(SU);
  static_assert(NS >= 2, "at least two stages");
  constexpr int XT = kRows * kKC, AT = kNC * kKC, STAGE = SU * (XT + AT);
  constexpr uint32_t LBOX = kRows * 16, LBOA = kNC * 16, SBO = 128;
  constexpr uint32_t ID = idesc_bf16(kRows, kNC);
  constexpr uint32_t kStageBytes = (uint32_t)SU * (kKC / 8) * (kRows + kNC) * 16;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __shared__ __align__(8) uint64_t full[NS], empty[NS], tfull, tempty, mfin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    s_fail = 0;
    for (int b = 0; b < NS; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&tempty)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mfin)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  auto fail = [&]() {
    atomicExch(&s_fail, 1);
    atomicExch(err, 1);
  };
  auto failed = [&]() { return *(volatile int*)&s_fail != 0; };

  if (warp == 0) {
    // ---------------- producer (lane 0): TMA boxes, one expect-tx per stage
    if (lane == 0) {
      int q = 0;
      for (int it = blockIdx.x; it < n_items && !failed(); it += G) {
        const int4 I = items[it];
        const int g = I.w;
        const int4 P = gp[g];
        const int Kp = P.x, Np = P.w;
        const int rows_g = (int)(gstart[g + 1] - gstart[g]);
        const int rl = (int)(I.x - gstart[g]);
        const void* mx = mapX + g;
        const void* ma = mapA + g;
        const int nchunks = Kp / kKC;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c, ++q) {
          const int slot = q % NS;
          if (q >= NS && !mbar_wait(&empty[slot], ((q / NS) - 1) & 1, kWaitNs, 32)) {
            ok = false;
            break;
          }
          __nv_bfloat16* xs = stg + (size_t)slot * STAGE;
          __nv_bfloat16* as = xs + SU * XT;
          mbar_expect_tx(&full[slot], kStageBytes);
          for (int t = 0; t < SU; ++t)
            for (int kg = 0; kg < kKC / 8; ++kg) {
              const int x = c * kKC + kg * 8;
              tma_load_2d(xs + t * XT + kg * (kRows * 8), mx, x, t * rows_g + rl, &full[slot]);
              tma_load_2d(as + t * AT + kg * (kNC * 8), ma, x, t * Np + I.z, &full[slot]);
            }
        }
        if (!ok) {
          fail();
          break;
        }
      }
      // no TMA write may outlive the CTA: the last stages' loads have landed
      // (immediately true when the MMAs consumed them)
      for (int r = q > NS ? q - NS : 0; r < q; ++r) mbar_wait(&full[r % NS], (r / NS) & 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issue (lane 0)
    if (lane == 0) {
      int q = 0, k = 0;
      for (int it = blockIdx.x; it < n_items && !failed(); it += G, ++k) {
        const int4 P = gp[items[it].w];
        const int nchunks = P.x / kKC;
        if (k >= 1 && !mbar_wait(&tempty, (k - 1) & 1)) {
          fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        bool ok = true;
        for (int c = 0; c < nchunks; ++c, ++q) {
          const int slot = q % NS;
          if (!mbar_wait(&full[slot], (q / NS) & 1)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const __nv_bfloat16* xs = stg + (size_t)slot * STAGE;
          const __nv_bfloat16* as = xs + SU * XT;
          const uint64_t dx0 = smem_desc(smem_u32(xs), LBOX, SBO);
          const uint64_t da0 = smem_desc(smem_u32(as), LBOA, SBO);
#pragma unroll
          for (int ti = 0; ti < SU; ++ti) {
#pragma unroll
            for (int tj = 0; tj < SU - ti; ++tj) {
              const int a = ti + tj;
#pragma unroll
              for (int kk = 0; kk < kKC; kk += 16) {
                const uint64_t da = dx0 + (uint64_t)((ti * XT * 2 + (kk / 8) * LBOX) >> 4);
                const uint64_t db = da0 + (uint64_t)((tj * AT * 2 + (kk / 8) * LBOA) >> 4);
                mma_bf16(tmem + a * kNC, da, db, ID, (c > 0 || ti > 0 || kk > 0) ? 1u : 0u);
              }
            }
          }
          mma_commit(&empty[slot]);
        }
        if (!ok) {
          fail();
          break;
        }
        mma_commit(&tfull);
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: rows (warp mod 4) * 32 + lane
    const int m = (warp & 3) * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    int k = 0;
    for (int it = blockIdx.x; it < n_items && !failed(); it += G, ++k) {
      const int4 I = items[it];
      const int row0 = I.x, nr = I.y, n0 = I.z, g = I.w;
      const int4 P = gp[g];
      const int Q = P.y, beta = P.z;
      const int* fg = fexp + gfoff[g];
      if (!mbar_wait(&tfull, k & 1, kWaitNs, 64)) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const bool row_ok = m < nr;
      const int e_row = row_ok ? xexp[rowsrc[row0 + m]] : 0;
      const long long yo = row_ok ? yoff[row0 + m] : 0;
      for (int j0 = 0; j0 < kNC; j0 += 16) {
        // the SU accumulators of these 16 columns: all loads in flight, one wait
        uint32_t r[SU][16];
#pragma unroll
        for (int a = 0; a < SU; ++a) tmem_ld16_async(tl + a * kNC + j0, r[a]);
        tmem_wait_ld();
#pragma unroll
        for (int a = 0; a < SU; ++a) reg_fence16(r[a]);
        float hi[16], lo[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) hi[c] = lo[c] = 0.f;
#pragma unroll
        for (int a = SU - 1; a >= 0; --a) {
          const float sa = exp2i(-beta * (a + 2));  // exact: -beta (a + 2) >= -80
#pragma unroll
          for (int c = 0; c < 16; ++c) ff_add(hi[c], lo[c], __uint_as_float(r[a][c]) * sa, 0.f);
        }
        if (j0 + 16 >= kNC) {
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(&tempty);
        }
        if (row_ok) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int j = n0 + j0 + c;
            if (j >= 2 * Q) break;
            const int sc = e_row + fg[j];
            const float f = exp2i(sc);
            const float2 w = f != 0.f ? make_float2(hi[c] * f, lo[c] * f)
                                      : make_float2(ldexpf(hi[c], sc), ldexpf(lo[c], sc));
            float2* dst = reinterpret_cast<float2*>(Y + yo + (j < Q ? j : j - Q)) + (j < Q ? 0 : 1);
            *dst = w;
          }
        }
      }
    }
  }
  __syncthreads();
  if (s_fail) {
    if (warp == 1 && lane == 0) mma_commit(&mfin);
    mbar_wait(&mfin, 0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// lh_lo(b) += conv_lo * sum over b's V entries of the row values: float-float
// sums (tensor-core levels) or FP64 sums (the others), in V-list order.
__global__ void __launch_bounds__(kThr) m2l_tc_reduce_kernel(
    int pbmax, const int* __restrict__ boxes, const int* __restrict__ level,
    const int* __restrict__ lpb, const int4* __restrict__ lvl, const int* __restrict__ voff,
    const long long* __restrict__ eyoff, const cd* __restrict__ Y,
    const double* __restrict__ conv, const long long* __restrict__ eoff, cd* __restrict__ local) {
  const int b = boxes[blockIdx.x];
  const int l = level[b];
  const int pb = lpb[l], Q = 2 * pb + 1;
  cd* dst = local + eoff[b];
  const int e0 = voff[b], e1 = voff[b + 1];
  if (lvl[l].x) {
    const double* cv = conv + (size_t)l * (pbmax + 1);
    for (int lo = threadIdx.x; lo < Q; lo += kThr) {
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      for (int e = e0; e < e1; ++e) {
        const float4 y = reinterpret_cast<const float4*>(Y)[eyoff[e] + lo];
        ff_add(rh, rl, y.x, y.y);
        ff_add(ih, il, y.z, y.w);
      }
      const double f = cv[abs(lo - pb)];
      dst[lo] = cadd(dst[lo], mk(((double)rh + (double)rl) * f, ((double)ih + (double)il) * f));
    }
  } else {
    for (int lo = threadIdx.x; lo < Q; lo += kThr) {
      cd sum = mk(0.0, 0.0);
      for (int e = e0; e < e1; ++e) sum = cadd(sum, Y[eyoff[e] + lo]);
      dst[lo] = cadd(dst[lo], sum);
    }
  }
}

template <int SU>
size_t tc_smem_bytes() {
  return (size_t)tc_stages(SU) * SU * (kRows * kKC + kNC * kKC) * sizeof(__nv_bfloat16);
}

// slices used by the mixed path for a level split into SD slices of beta bits:
// at least 24 bits (SU beta >= 24)
__host__ __device__ constexpr int mixed_slices(int SD) { return SD == 6 ? 3 : 4; }

// (beta, S) for a padded width Kp: the most bits per digit for which
// S Kp 2^(2 beta - 2) <= 2^24 (exact FP32 sums) with beta S >= 48; 0 if none.
int2 tc_params(int Kp) {
  if (Kp <= 128) return make_int2(8, 6);
  if (Kp <= 576) return make_int2(7, 7);
  if (Kp <= 2048) return make_int2(6, 8);
  return make_int2(0, 0);
}

}  // namespace

int g_tc_sms = 152;  // persistent grid: one CTA per SM (set at configuration)

qbx_status configure_tc_kernels(int smem_optin) {
  {
    int dev = 0;
    QBX_CUDA_TRY(cudaGetDevice(&dev));
    QBX_CUDA_TRY(cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev));
    const void* w[] = {(const void*)tc_gemm_ws_kernel<6, 6>, (const void*)tc_gemm_ws_kernel<7, 7>,
                       (const void*)tc_gemm_ws_kernel<8, 8>, (const void*)tc_gemm_tma_kernel<6, 6>,
                       (const void*)tc_gemm_tma_kernel<7, 7>, (const void*)tc_gemm_tma_kernel<8, 8>};
    const size_t wn[] = {tc_smem_bytes<6>(), tc_smem_bytes<7>(), tc_smem_bytes<8>(),
                         tc_smem_bytes<6>(), tc_smem_bytes<7>(), tc_smem_bytes<8>()};
    for (int i = 0; i < 6; ++i)
      QBX_CUDA_TRY(cudaFuncSetAttribute(w[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)wn[i]));
  }
  const void* k[] = {(const void*)m2l_tc_kernel<6, 6>, (const void*)m2l_tc_kernel<7, 7>,
                     (const void*)m2l_tc_kernel<8, 8>, (const void*)m2l_tc_kernel<6, 3>,
                     (const void*)m2l_tc_kernel<7, 4>, (const void*)m2l_tc_kernel<8, 4>};
  const size_t need[] = {tc_smem_bytes<6>(), tc_smem_bytes<7>(), tc_smem_bytes<8>(),
                         tc_smem_bytes<3>(), tc_smem_bytes<4>(), tc_smem_bytes<4>()};
  for (int i = 0; i < 6; ++i) {
    if (need[i] + 2048 > (size_t)smem_optin) {
      set_error("tensor-core M2L needs %zu bytes of shared memory (device: %d)", need[i],
                smem_optin);
      return QBX_ERR_ARG;
    }
    QBX_CUDA_TRY(cudaFuncSetAttribute(k[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)need[i]));
  }
  return QBX_OK;
}

// Plan-time part: per-level (use, beta, S, Kp), the matrix slices of every
// group with V pairs on a tensor-core level, the vector-slice room of every
// V-list source there, and the work items. Levels whose 2Q is too wide for
// exact FP32 sums keep the FP64 CUDA-core GEMM (its items are filtered here).
namespace {
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to
// the driver library); null when the driver does not provide it
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}
// 2D bf16 tensor [outer][inner] at base, boxes of 8 (16 bytes) x box_rows
bool encode_map(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* base, uint64_t inner,
                uint64_t outer, uint32_t box_rows, TmapBlob* out) {
  static_assert(sizeof(CUtensorMap) == sizeof(TmapBlob), "tensor map size");
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {inner * 2};
  const cuuint32_t box[2] = {8, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
             const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

// TMA layout of the FP64 M2L: every tensor-core group's rows get their source
// slices in row order ([S][rows][K] at x2off), and each group a tensor map of
// that copy and one of its matrix slices ([S][K][K]). QBX_TC_TMA=0 in the
// environment keeps the cp.async kernel (for comparisons).
qbx_status tc_tma_plan_build(qbx_handle* h, FmmPlan* f, const std::vector<int>& groups,
                             const std::vector<int4>& lv, const std::vector<long long>& aoff,
                             const std::vector<int>& rowsrc, const std::vector<long long>& xoff) {
  (void)h;
  f->tc_tma = false;
  const char* env = getenv("QBX_TC_TMA");
  if (env && env[0] == '0') return QBX_OK;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || groups.empty()) return QBX_OK;
  const int ng = f->n_levels * 49;
  std::vector<long long> gstart(ng + 1, 0), x2off(ng, 0);
  for (int g = 0; g <= ng; ++g) gstart[g] = f->h_gcount[g];
  std::vector<long long> src, dst, ts;
  std::vector<int2> sk;
  long long tot = 0;
  for (int g : groups) {
    const int l = g / 49, S = lv[l].z, K = lv[l].w;
    const long long rows = gstart[g + 1] - gstart[g];
    x2off[g] = tot;
    for (long long r = gstart[g]; r < gstart[g + 1]; ++r) {
      src.push_back(xoff[rowsrc[r]]);
      dst.push_back(tot + (r - gstart[g]) * K);
      ts.push_back(rows * K);
      sk.push_back(make_int2(S, K));
    }
    tot += (long long)S * rows * K;
  }
  QBX_CUDA_TRY(f->tc_X2.alloc(std::max<long long>(1, tot)));
  std::vector<TmapBlob> ma(ng), mx(ng);
  std::memset(ma.data(), 0, ng * sizeof(TmapBlob));
  std::memset(mx.data(), 0, ng * sizeof(TmapBlob));
  for (int g : groups) {
    const int l = g / 49, S = lv[l].z, K = lv[l].w;
    const long long rows = gstart[g + 1] - gstart[g];
    if (!encode_map(enc, reinterpret_cast<const uint16_t*>(f->tc_A.ptr) + aoff[g], K,
                    (uint64_t)S * K, kNC, &ma[g]) ||
        !encode_map(enc, f->tc_X2.ptr + x2off[g], K, (uint64_t)S * rows, kRows, &mx[g]))
      return QBX_OK;  // no TMA maps: the cp.async kernel serves
  }
  f->n_tc_rows = (int)src.size();
  TRY_TC(upload(f->tc_x2src, src));
  TRY_TC(upload(f->tc_x2dst, dst));
  TRY_TC(upload(f->tc_x2ts, ts));
  TRY_TC(upload(f->tc_x2sk, sk));
  TRY_TC(upload(f->tc_gstart, gstart));
  TRY_TC(upload(f->tc_mapA, ma));
  TRY_TC(upload(f->tc_mapX, mx));
  f->tc_tma = true;
  return QBX_OK;
}

qbx_status tc_plan_build(qbx_handle* h, FmmPlan* f) {
  const int nl = f->n_levels, ng = nl * 49;
  std::vector<int4> lv(nl, make_int4(0, 0, 0, 0));
  for (int l = 2; l < nl; ++l) {
    if (f->vbox_off[l + 1] == f->vbox_off[l]) continue;
    const int Q = 2 * f->h_pb[l] + 1;
    const int Kp = (2 * Q + kPad - 1) / kPad * kPad;
    const int2 bs = tc_params(Kp);
    if (bs.x > 0) lv[l] = make_int4(1, bs.x, bs.y, Kp);
  }
  // QBX_M2L_TENSOR=0 in the environment keeps every level on the FP64
  // CUDA-core GEMM (for comparisons); the default is the tensor-core path
  {
    const char* env = getenv("QBX_M2L_TENSOR");
    if ((env && env[0] == '0') || h->m2l_engine == 2)
      for (auto& v : lv) v = make_int4(0, 0, 0, 0);
  }
  f->h_tc_lvl = lv;
  {  // FP64 GEMM items of the levels left to the CUDA-core path
    std::vector<int4> rest;
    for (const int4& it : f->h_items64)
      if (!lv[it.w / 49].x) rest.push_back(it);
    f->n_m2l_items64_rest = (int)rest.size();
    QBX_CUDA_TRY(f->m2l_items64_rest.alloc(std::max<size_t>(1, rest.size())));
    if (!rest.empty())
      QBX_CUDA_TRY(cudaMemcpy(f->m2l_items64_rest.ptr, rest.data(), rest.size() * sizeof(int4),
                              cudaMemcpyHostToDevice));
  }
  QBX_CUDA_TRY(f->tc_lvl.alloc(nl));
  QBX_CUDA_TRY(cudaMemcpy(f->tc_lvl.ptr, lv.data(), nl * sizeof(int4), cudaMemcpyHostToDevice));
  {  // per-group parameters of the tile product: (K, Q, beta, Np) of the level
    std::vector<int4> gp(ng);
    for (int g = 0; g < ng; ++g) {
      const int l = g / 49;
      gp[g] = make_int4(lv[l].w, 2 * f->h_pb[l] + 1, lv[l].y, lv[l].w);
    }
    QBX_CUDA_TRY(f->tc_gp.alloc(ng));
    QBX_CUDA_TRY(cudaMemcpy(f->tc_gp.ptr, gp.data(), ng * sizeof(int4), cudaMemcpyHostToDevice));
  }
  // groups with rows on tensor-core levels
  std::vector<int> groups;
  std::vector<long long> aoff(ng, 0), foff(ng, 0), g_aoff, g_foff;
  long long atot = 0, ftot = 0;
  for (int g = 0; g < ng; ++g) {
    const int l = g / 49;
    if (!lv[l].x || f->h_gcount[g + 1] == f->h_gcount[g]) continue;
    const long long Kp = lv[l].w, S = lv[l].z;
    groups.push_back(g);
    aoff[g] = atot;
    foff[g] = ftot;
    g_aoff.push_back(atot);
    g_foff.push_back(ftot);
    atot += S * Kp * Kp;
    ftot += Kp;
  }
  f->tc_any = !groups.empty();
  if (!f->tc_any) return QBX_OK;
  QBX_CUDA_TRY(f->tc_A.alloc(atot));
  QBX_CUDA_TRY(f->tc_fexp.alloc(ftot));
  QBX_CUDA_TRY(f->tc_gaoff.alloc(ng));
  QBX_CUDA_TRY(f->tc_gfoff.alloc(ng));
  QBX_CUDA_TRY(cudaMemcpy(f->tc_gaoff.ptr, aoff.data(), ng * 8, cudaMemcpyHostToDevice));
  QBX_CUDA_TRY(cudaMemcpy(f->tc_gfoff.ptr, foff.data(), ng * 8, cudaMemcpyHostToDevice));
  {
    DevBuf<int> dg;
    DevBuf<long long> da, df;
    QBX_CUDA_TRY(dg.alloc(groups.size()));
    QBX_CUDA_TRY(da.alloc(groups.size()));
    QBX_CUDA_TRY(df.alloc(groups.size()));
    QBX_CUDA_TRY(cudaMemcpy(dg.ptr, groups.data(), groups.size() * 4, cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(da.ptr, g_aoff.data(), groups.size() * 8, cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(df.ptr, g_foff.data(), groups.size() * 8, cudaMemcpyHostToDevice));
    int kpmax = 0;  // <= 2048 = 16 entries per thread (tc_params)
    for (int l = 0; l < nl; ++l) kpmax = std::max(kpmax, lv[l].w);
    dim3 grid((unsigned)groups.size(), (unsigned)kpmax);
    tc_matrix_kernel<<<grid, kThr>>>(dg.ptr, da.ptr, df.ptr, f->tc_lvl.ptr, f->lpb.ptr,
                                     f->pb_max, f->t_m2l.ptr, f->scale.ptr, f->lsig.ptr,
                                     reinterpret_cast<__nv_bfloat16*>(f->tc_A.ptr),
                                     f->tc_fexp.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    QBX_CUDA_TRY(cudaDeviceSynchronize());
  }
  // vector-slice room per V-list source on a tensor-core level
  std::vector<int> vsrc(std::max(1, f->n_vsrc)), blev(f->n_boxes);
  if (f->n_vsrc)
    QBX_CUDA_TRY(cudaMemcpy(vsrc.data(), f->m2l_vsrc.ptr, f->n_vsrc * 4, cudaMemcpyDeviceToHost));
  QBX_CUDA_TRY(cudaMemcpy(blev.data(), f->box.level.ptr, f->n_boxes * 4, cudaMemcpyDeviceToHost));
  std::vector<int> tbox, pos_of(f->n_boxes, -1);
  std::vector<long long> xoff;
  long long xtot = 0;
  for (int i = 0; i < f->n_vsrc; ++i) {
    const int b = vsrc[i], l = blev[b];
    if (!lv[l].x) continue;
    pos_of[b] = (int)tbox.size();
    tbox.push_back(b);
    xoff.push_back(xtot);
    xtot += (long long)lv[l].z * lv[l].w;
  }
  f->n_tc_src = (int)tbox.size();
  QBX_CUDA_TRY(f->tc_src.alloc(std::max<size_t>(1, tbox.size())));
  QBX_CUDA_TRY(f->tc_xoff.alloc(std::max<size_t>(1, xoff.size())));
  QBX_CUDA_TRY(f->tc_xexp.alloc(std::max<size_t>(1, tbox.size())));
  QBX_CUDA_TRY(f->tc_X.alloc(std::max<long long>(1, xtot)));
  if (!tbox.empty()) {
    QBX_CUDA_TRY(cudaMemcpy(f->tc_src.ptr, tbox.data(), tbox.size() * 4, cudaMemcpyHostToDevice));
    QBX_CUDA_TRY(cudaMemcpy(f->tc_xoff.ptr, xoff.data(), xoff.size() * 8, cudaMemcpyHostToDevice));
  }
  // rows: position of their source among the tensor-core sources; items
  const size_t nrows = f->h_row_src.size();
  std::vector<int> rowsrc(std::max<size_t>(1, nrows), -1);
  for (size_t r = 0; r < nrows; ++r) rowsrc[r] = pos_of[f->h_row_src[r]];
  QBX_CUDA_TRY(f->tc_rowsrc.alloc(rowsrc.size()));
  QBX_CUDA_TRY(cudaMemcpy(f->tc_rowsrc.ptr, rowsrc.data(), rowsrc.size() * 4, cudaMemcpyHostToDevice));
  std::vector<int4> items[3];  // by S = 6, 7, 8
  for (int g : groups) {
    const int l = g / 49, S = lv[l].z, Kp = lv[l].w;
    const int Q = 2 * f->h_pb[l] + 1;
    for (int64_t r = f->h_gcount[g]; r < f->h_gcount[g + 1]; r += kRows)
      for (int n0 = 0; n0 < 2 * Q && n0 < Kp; n0 += kNC)
        items[S - 6].push_back(make_int4((int)r, (int)std::min<int64_t>(kRows, f->h_gcount[g + 1] - r),
                                         n0, g));
  }
  for (int s = 0; s < 3; ++s) {
    f->n_tc_items[s] = (int)items[s].size();
    QBX_CUDA_TRY(f->tc_items[s].alloc(std::max<size_t>(1, items[s].size())));
    if (!items[s].empty())
      QBX_CUDA_TRY(cudaMemcpy(f->tc_items[s].ptr, items[s].data(), items[s].size() * sizeof(int4),
                              cudaMemcpyHostToDevice));
  }
  return tc_tma_plan_build(h, f, groups, lv, aoff, rowsrc, xoff);
}



// Plan of the FP64 M2M and L2L on the tensor cores: for every parent level l
// whose contraction width K (2 Q of the child level for M2M, of level l for
// L2L, padded to 64) admits an exact split, the matrix slices of the four
// quadrant operators, the rows (one per child: quadrant-major, parents in
// level order), the source boxes and the work items. Levels without one keep
// the CUDA-core kernels; so do all levels with m2l_engine == 2 or
// QBX_M2L_TENSOR=0.
qbx_status tc_mml_plan_build(qbx_handle* h, FmmPlan* f) {
  const int nl = f->n_levels;
  f->tc_m2m.clear();
  f->tc_l2l.clear();
  f->tc_m2m.resize(nl);
  f->tc_l2l.resize(nl);
  {
    const char* env = getenv("QBX_M2L_TENSOR");
    if ((env && env[0] == '0') || h->m2l_engine == 2) return QBX_OK;
  }
  std::vector<int> child((size_t)4 * f->n_boxes), nonleaf(std::max(1, f->nonleaf_off[nl]));
  QBX_CUDA_TRY(cudaMemcpy(child.data(), f->box.child.ptr, child.size() * sizeof(int),
                          cudaMemcpyDeviceToHost));
  if (f->nonleaf_off[nl] > 0)
    QBX_CUDA_TRY(cudaMemcpy(nonleaf.data(), f->nonleaf.ptr, f->nonleaf_off[nl] * sizeof(int),
                            cudaMemcpyDeviceToHost));
  size_t ymax = 1;
  for (int kind = 0; kind < 2; ++kind) {
    for (int l = 2; l + 1 < nl; ++l) {
      // the level's parents, in the order of the device list (the reduce
      // kernel walks that list)
      const std::vector<int> par(nonleaf.begin() + f->nonleaf_off[l],
                                 nonleaf.begin() + f->nonleaf_off[l + 1]);
      if (par.empty()) continue;
      TcLevelOp& op = kind == 0 ? f->tc_m2m[l] : f->tc_l2l[l];
      const int pp = f->h_pb[l], pc = f->h_pb[l + 1];
      const int qin = kind == 0 ? 2 * pc + 1 : 2 * pp + 1;
      const int qout = kind == 0 ? 2 * pp + 1 : 2 * pc + 1;
      const int K = (2 * qin + kPad - 1) / kPad * kPad;
      const int Np = (2 * qout + kPad - 1) / kPad * kPad;
      const int2 bs = tc_params(K);
      if (bs.x == 0) continue;
      op.use = true;
      op.beta = bs.x;
      op.S = bs.y;
      op.K = K;
      op.Np = Np;
      op.Q = qout;
      op.n_par = (int)par.size();
      // rows: quadrant-major, parents in level order; sources
      std::vector<int> rowsrc, rowdst, prow((size_t)4 * par.size(), -1), src;
      std::vector<int64_t> gcount(5, 0);
      for (int c = 0; c < 4; ++c) {
        gcount[c] = (int64_t)rowdst.size();
        for (size_t i = 0; i < par.size(); ++i) {
          const int d = child[4 * (size_t)par[i] + c];
          if (d < 0) continue;
          prow[4 * i + c] = (int)rowdst.size();
          if (kind == 0) {  // M2M: the row's source is the child
            rowsrc.push_back((int)src.size());
            src.push_back(d);
            rowdst.push_back(par[i]);
          } else {          // L2L: the parent (one source per parent)
            rowsrc.push_back((int)i);
            rowdst.push_back(d);
          }
        }
      }
      gcount[4] = (int64_t)rowdst.size();
      if (kind == 1) src = par;
      op.n_rows = (int)rowdst.size();
      op.n_src = (int)src.size();
      ymax = std::max(ymax, (size_t)op.n_rows * qout);
      std::vector<int4> gp(4, make_int4(K, qout, bs.x, Np));
      std::vector<long long> gaoff(4), gfoff(4), xoff(src.size()), yoff(rowdst.size());
      for (int c = 0; c < 4; ++c) {
        gaoff[c] = (long long)c * bs.y * Np * K;
        gfoff[c] = (long long)c * Np;
      }
      for (size_t i = 0; i < src.size(); ++i) xoff[i] = (long long)i * bs.y * K;
      for (size_t r = 0; r < rowdst.size(); ++r) yoff[r] = (long long)r * qout;
      std::vector<int4> items;
      for (int c = 0; c < 4; ++c)
        for (int64_t r = gcount[c]; r < gcount[c + 1]; r += kRows)
          for (int n0 = 0; n0 < 2 * qout; n0 += kNC)
            items.push_back(make_int4((int)r, (int)std::min<int64_t>(kRows, gcount[c + 1] - r), n0, c));
      op.n_items = (int)items.size();
      TRY_TC(upload(op.gp, gp));
      TRY_TC(upload(op.items, items));
      TRY_TC(upload(op.gaoff, gaoff));
      TRY_TC(upload(op.gfoff, gfoff));
      TRY_TC(upload(op.xoff, xoff));
      TRY_TC(upload(op.yoff, yoff));
      TRY_TC(upload(op.src, src));
      TRY_TC(upload(op.rowsrc, rowsrc));
      TRY_TC(upload(op.rowdst, rowdst));
      TRY_TC(upload(op.prow, prow));
      QBX_CUDA_TRY(op.A.alloc((size_t)4 * bs.y * Np * K));
      QBX_CUDA_TRY(op.fexp.alloc((size_t)4 * Np));
      QBX_CUDA_TRY(op.X.alloc(std::max<size_t>(1, src.size() * (size_t)bs.y * K)));
      QBX_CUDA_TRY(op.xexp.alloc(std::max<size_t>(1, src.size())));
      tc_mml_matrix_kernel<<<dim3(4, Np), kThr>>>(
          kind, l, pp, pc, f->pb_max, kind == 0 ? f->t_m2m.ptr : f->t_l2l.ptr, f->lsig.ptr, K, Np,
          bs.x, bs.y, reinterpret_cast<__nv_bfloat16*>(op.A.ptr), op.fexp.ptr);
      QBX_CUDA_TRY(cudaGetLastError());
    }
  }
  QBX_CUDA_TRY(f->tc_mml_y.alloc(ymax));
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  return QBX_OK;
}

qbx_status launch_mml_tc(qbx_handle* h, FmmPlan* f, int kind, int l, bool* done, cudaStream_t s) {
  *done = false;
  if (l >= (int)f->tc_m2m.size()) return QBX_OK;
  TcLevelOp& op = kind == 0 ? f->tc_m2m[l] : f->tc_l2l[l];
  if (!op.use) return QBX_OK;
  const int pp = f->h_pb[l], pc = f->h_pb[l + 1];
  if (op.n_src > 0) {
    tc_mml_vec_kernel<<<op.n_src, kThr, 0, s>>>(
        kind, op.src.ptr, kind == 0 ? f->mpole.ptr : f->local.ptr, kind == 0 ? l + 1 : l,
        kind == 0 ? pc : pp, op.K, op.beta, op.S, f->conv.ptr, f->pb_max, f->eoff.ptr,
        op.xoff.ptr, reinterpret_cast<__nv_bfloat16*>(op.X.ptr), op.xexp.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
  }
#define TC_MML(S_)                                                                              \
  tc_gemm_ws_kernel<S_, S_><<<std::min(op.n_items, g_tc_sms), kWsThr, tc_smem_bytes<S_>(), s>>>(  \
      op.items.ptr, op.n_items, op.gp.ptr, op.gaoff.ptr, op.gfoff.ptr,                          \
      reinterpret_cast<const __nv_bfloat16*>(op.A.ptr), op.fexp.ptr, op.rowsrc.ptr, op.xoff.ptr, \
      op.xexp.ptr, reinterpret_cast<const __nv_bfloat16*>(op.X.ptr), op.yoff.ptr,               \
      f->tc_mml_y.ptr, f->err.ptr + 1)
  if (op.n_items > 0) {
    if (op.S == 6) TC_MML(6);
    else if (op.S == 7) TC_MML(7);
    else TC_MML(8);
    QBX_CUDA_TRY(cudaGetLastError());
  }
#undef TC_MML
  if (kind == 0)
    tc_m2m_reduce_kernel<<<op.n_par, kThr, 0, s>>>(f->nonleaf.ptr + f->nonleaf_off[l], op.prow.ptr,
                                                   pp, l, f->pb_max, f->conv.ptr, f->tc_mml_y.ptr,
                                                   f->eoff.ptr, f->mpole.ptr);
  else if (op.n_rows > 0)
    tc_l2l_apply_kernel<<<op.n_rows, kThr, 0, s>>>(op.rowdst.ptr, pc, l + 1, f->pb_max, f->conv.ptr,
                                                   f->tc_mml_y.ptr, f->eoff.ptr, f->local.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 3;
  *done = true;
  return QBX_OK;
}

qbx_status launch_m2l_tc(qbx_handle* h, FmmPlan* f, bool mixed, cudaStream_t s) {
  if (f->n_vbox == 0) return QBX_OK;
  if (f->n_tc_src > 0) {
    tc_mu_kernel<<<f->n_tc_src, kThr, 0, s>>>(f->tc_src.ptr, f->box.level.ptr, f->lpb.ptr,
                                              f->eoff.ptr, f->conv.ptr, f->pb_max, f->tc_lvl.ptr,
                                              f->mpole.ptr, f->tc_xoff.ptr,
                                              reinterpret_cast<__nv_bfloat16*>(f->tc_X.ptr),
                                              f->tc_xexp.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    h->launches += 1;
  }
#define TC_LAUNCH(SD, SU)                                                                      \
  if (f->n_tc_items[SD - 6] > 0) {                                                              \
    m2l_tc_kernel<SD, SU><<<f->n_tc_items[SD - 6], kThr, tc_smem_bytes<SU>(), s>>>(             \
        f->tc_items[SD - 6].ptr, f->tc_gp.ptr, f->tc_gaoff.ptr, f->tc_gfoff.ptr,               \
        reinterpret_cast<const __nv_bfloat16*>(f->tc_A.ptr), f->tc_fexp.ptr, f->tc_rowsrc.ptr,   \
        f->tc_xoff.ptr, f->tc_xexp.ptr, reinterpret_cast<const __nv_bfloat16*>(f->tc_X.ptr),     \
        f->m2l_yoff.ptr, f->m2l_y64.ptr, f->err.ptr + 1);                                      \
    QBX_CUDA_TRY(cudaGetLastError());                                                           \
    h->launches += 1;                                                                           \
  }
#define TC_LAUNCH_WS(S_)                                                                        \
  if (f->n_tc_items[S_ - 6] > 0) {                                                              \
    tc_gemm_ws_kernel<S_, S_><<<std::min(f->n_tc_items[S_ - 6], g_tc_sms), kWsThr,              \
                                tc_smem_bytes<S_>(), s>>>(                                       \
        f->tc_items[S_ - 6].ptr, f->n_tc_items[S_ - 6], f->tc_gp.ptr, f->tc_gaoff.ptr,          \
        f->tc_gfoff.ptr, reinterpret_cast<const __nv_bfloat16*>(f->tc_A.ptr), f->tc_fexp.ptr,    \
        f->tc_rowsrc.ptr, f->tc_xoff.ptr, f->tc_xexp.ptr,                                       \
        reinterpret_cast<const __nv_bfloat16*>(f->tc_X.ptr), f->m2l_yoff.ptr, f->m2l_y64.ptr,    \
        f->err.ptr + 1);                                                                        \
    QBX_CUDA_TRY(cudaGetLastError());                                                           \
    h->launches += 1;                                                                           \
  }
  if (mixed) {
    TC_LAUNCH(6, 3)
    TC_LAUNCH(7, 4)
    TC_LAUNCH(8, 4)
  } else if (f->tc_tma) {  // TMA-fed: the rows' slices in row order first
    tc_x2_fill_kernel<<<f->n_tc_rows, 128, 0, s>>>(f->n_tc_rows, f->tc_x2src.ptr, f->tc_x2dst.ptr,
                                                  f->tc_x2ts.ptr, f->tc_x2sk.ptr, f->tc_X.ptr,
                                                  f->tc_X2.ptr);
    QBX_CUDA_TRY(cudaGetLastError());
    h->launches += 1;
#define TC_LAUNCH_TMA(S_)                                                                       \
    if (f->n_tc_items[S_ - 6] > 0) {                                                            \
      tc_gemm_tma_kernel<S_, S_><<<std::min(f->n_tc_items[S_ - 6], g_tc_sms), kTmaThr,          \
                                  tc_smem_bytes<S_>(), s>>>(                                     \
          f->tc_items[S_ - 6].ptr, f->n_tc_items[S_ - 6], f->tc_gp.ptr, f->tc_mapA.ptr,         \
          f->tc_mapX.ptr, f->tc_gstart.ptr, f->tc_gfoff.ptr, f->tc_fexp.ptr, f->tc_rowsrc.ptr,  \
          f->tc_xexp.ptr, f->m2l_yoff.ptr, f->m2l_y64.ptr, f->err.ptr + 1);                      \
      QBX_CUDA_TRY(cudaGetLastError());                                                         \
      h->launches += 1;                                                                         \
    }
    TC_LAUNCH_TMA(6)
    TC_LAUNCH_TMA(7)
    TC_LAUNCH_TMA(8)
#undef TC_LAUNCH_TMA
  } else {  // the persistent warp-specialised kernel on cp.async
    TC_LAUNCH_WS(6)
    TC_LAUNCH_WS(7)
    TC_LAUNCH_WS(8)
  }
#undef TC_LAUNCH
#undef TC_LAUNCH_WS
  {
    const qbx_status st = launch_m2l_f64_gemm_rest(h, f, s);
    if (st != QBX_OK) return st;
  }
  m2l_tc_reduce_kernel<<<f->n_vbox, kThr, 0, s>>>(f->pb_max, f->vbox.ptr, f->box.level.ptr,
                                                  f->lpb.ptr, f->tc_lvl.ptr, f->V.off.ptr,
                                                  f->m2l_eyoff.ptr, f->m2l_y64.ptr, f->conv.ptr,
                                                  f->eoff.ptr, f->local.ptr);
  QBX_CUDA_TRY(cudaGetLastError());
  h->launches += 1;
  return QBX_OK;
}

namespace {
// One warp waits on an mbarrier that nothing arrives at, with the bounded
// wait of the tensor-core kernels (deadline limit_ns), and sets the flag
// those kernels set when a wait runs out.
__global__ void wait_selftest_kernel(int* __restrict__ err, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncwarp();
  const bool done = mbar_wait(&bar, 0, limit_ns);
  if (!done && threadIdx.x == 0) atomicExch(err, 1);
}
}  // namespace

// The flag the tensor-core M2L kernels set when one of their bounded waits
// ran out (the result of that evaluation is then wrong): read after the
// device work, then cleared.
qbx_status read_wait_flag(qbx_handle* h) {
  if (!h->fmm) return QBX_OK;
  int flag = 0;
  QBX_CUDA_TRY(cudaMemcpy(&flag, h->fmm->err.ptr + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (!flag) return QBX_OK;
  QBX_CUDA_TRY(cudaMemset(h->fmm->err.ptr + 1, 0, sizeof(int)));
  set_error("a bounded device-side wait gave up (tensor-core M2L); the results of the "
            "evaluations since the last check are invalid");
  return QBX_ERR_TIMEOUT;
}

extern "C" qbx_status qbx_selftest_wait_timeout(qbx_handle* h, int32_t limit_us) {
  set_error("%s", "");
  if (!h || limit_us < 1 || limit_us > 1000000) {
    set_error("qbx_selftest_wait_timeout: NULL handle or limit_us outside 1..1e6");
    return QBX_ERR_ARG;
  }
  if (!h->planned || !h->fmm) {
    set_error("qbx_selftest_wait_timeout: needs a handle with an FMM plan");
    return QBX_ERR_STATE;
  }
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  wait_selftest_kernel<<<1, 32>>>(h->fmm->err.ptr + 1, 1000ull * (unsigned long long)limit_us);
  QBX_CUDA_TRY(cudaGetLastError());
  QBX_CUDA_TRY(cudaDeviceSynchronize());
  return QBX_OK;
}
