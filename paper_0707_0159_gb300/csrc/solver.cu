// Ground-state solvers on the GPU: FP64 Lanczos and the mixed-precision outer loop.
//
// The paper obtains the superblock ground state by repeated H·v ("HMED",
// discussion of Fig. 5) without naming the eigensolver; this file uses
//   * Lanczos with full reorthogonalisation (classical Gram-Schmidt twice), the
//     tridiagonal eigenproblem solved on the GPU (Sturm bisection + inverse
//     iteration), explicit restart with the Ritz vector when the basis is full;
//   * mixed precision: Lanczos with low-precision H·v gives a start vector; an
//     FP64 outer loop then keeps a small subspace U with H U computed in FP64,
//     takes the Rayleigh-Ritz pair (theta, x) and its FP64 residual r, and adds a
//     correction t from a few conjugate-gradient steps on
//         (I - x x^T)(H~ - theta)(I - x x^T) t = -r
//     with H~ the low-precision H·v.  Only the FP64 residual decides convergence.
// All vectors are FP64 in device memory; reductions use a fixed grid and a fixed
// summation order, so results are bitwise reproducible run to run.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.h"

namespace dmrg2d {

namespace {

constexpr int VT = 256;        // threads per vector-kernel block
constexpr int RED_BLOCKS = 1216;  // 8 x 152 SMs; partial sums per reduction
constexpr int MD_CHUNK = 8;    // basis vectors per multi-dot block

int vgrid(int64_t n) {
  int64_t g = (n + VT - 1) / VT;
  return (int)(g < RED_BLOCKS ? (g < 1 ? 1 : g) : RED_BLOCKS);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double ws[VT / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < VT / 32 ? ws[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                              double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT)
    s += a[i] * b[i];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[i] = op(sum_b part[i*np + b]); one block per i.  op: 0 sum, 1 sqrt(sum)
__global__ void k_reduce(const double* __restrict__ part, int np, double* __restrict__ out, int op) {
  const double* p = part + (size_t)blockIdx.x * np;
  double s = 0.0;
  for (int b = threadIdx.x; b < np; b += VT) s += p[b];
  s = block_sum(s);
  if (threadIdx.x == 0) out[blockIdx.x] = op == 1 ? sqrt(s) : s;
}

// part[(i0+c)*gridDim.x + blk] = partial of Q_{i0+c} . w
__global__ void k_multidot_partial(const double* __restrict__ Q, int64_t stride, int k,
                                   const double* __restrict__ w, int64_t n, double* __restrict__ part) {
  const int i0 = blockIdx.y * MD_CHUNK;
  double acc[MD_CHUNK];
#pragma unroll
  for (int c = 0; c < MD_CHUNK; ++c) acc[c] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    const double we = w[e];
#pragma unroll
    for (int c = 0; c < MD_CHUNK; ++c)
      if (i0 + c < k) acc[c] += Q[(int64_t)(i0 + c) * stride + e] * we;
  }
#pragma unroll
  for (int c = 0; c < MD_CHUNK; ++c) {
    double s = block_sum(acc[c]);
    if (threadIdx.x == 0 && i0 + c < k) part[(size_t)(i0 + c) * gridDim.x + blockIdx.x] = s;
  }
}

// w -= sum_i h[i] Q_i   (sign = -1)  or  x = sum_i h[i] Q_i  (sign = 0)
__global__ void k_combo(double* __restrict__ out, const double* __restrict__ Q, int64_t stride, int k,
                        const double* __restrict__ h, int64_t n, int sign) {
  extern __shared__ double hs[];
  for (int i = threadIdx.x; i < k; i += VT) hs[i] = h[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += hs[i] * Q[(int64_t)i * stride + e];
    out[e] = sign ? out[e] - s : s;
  }
}

// w -= alpha[j] q_j + beta[j-1] q_{j-1}
__global__ void k_lz_axpy2(double* __restrict__ w, const double* __restrict__ qj,
                           const double* __restrict__ qjm1, const double* __restrict__ alpha_j,
                           const double* __restrict__ beta_jm1, int64_t n) {
  const double a = *alpha_j;
  const double b = beta_jm1 ? *beta_jm1 : 0.0;
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    double r = w[e] - a * qj[e];
    if (qjm1) r -= b * qjm1[e];
    w[e] = r;
  }
}

// out = in / *nrm   (zero when the norm is zero)
__global__ void k_scale_inv(double* __restrict__ out, const double* __restrict__ in,
                            const double* __restrict__ nrm, int64_t n) {
  const double s = *nrm;
  const double f = s > 0.0 ? 1.0 / s : 0.0;
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT)
    out[e] = in[e] * f;
}

// y = a*x + b*y with host scalars
__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b,
                        int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT)
    y[e] = a * x[e] + b * y[e];
}

__global__ void k_f64_to_f32(const double* __restrict__ x, float* __restrict__ o, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT)
    o[e] = (float)x[e];
}

__global__ void k_f64_to_bf16(const double* __restrict__ x, __nv_bfloat16* __restrict__ o, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT)
    o[e] = __float2bfloat16_rn((float)x[e]);
}

// the BF16X3 input: hi = bf16(x) at e, lo = bf16(x - hi) at n + e
__global__ void k_f64_to_bf16x3(const double* __restrict__ x, __nv_bfloat16* __restrict__ o,
                                int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x[e]);
    o[e] = h;
    o[n + e] = __float2bfloat16_rn((float)(x[e] - (double)__bfloat162float(h)));
  }
}

__global__ void k_f64_to_tf32(const double* __restrict__ x, float* __restrict__ o, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"((float)x[e]));
    o[e] = __uint_as_float(u);
  }
}

__global__ void k_f32_to_f64(const float* __restrict__ x, double* __restrict__ o, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT)
    o[e] = (double)x[e];
}

// ---- FP32-vector kernels of the mixed solver's low-precision phases -----------------
// Vectors that only ever meet the low-precision H~ (the Lanczos start basis, the vectors
// of the inner CG on the correction equation) are stored in FP32: their own rounding
// (6e-8) is far below H~'s, and it halves their HBM traffic.  Their arithmetic also stays
// on the FP32 pipes: GB300 runs FP64 at 1/64 of the FP32 rate, so a single FP64 operation
// per element already costs more time than the element's HBM traffic.  Dot products keep
// ~48 bits per thread with a compensated FP32 sum (exact products by fmaf, Knuth's
// two-sum), and the per-thread partials are reduced in FP64.

struct acc2 {
  float s = 0.f, c = 0.f;  // value s + c; c collects the rounding errors
};
// a += x, the rounding error of the sum kept in c (two-sum; __fadd_rn is never contracted)
__device__ __forceinline__ void acc_add(acc2& a, float x) {
  const float t = __fadd_rn(a.s, x);
  const float bp = __fsub_rn(t, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  a.s = t;
  a.c = __fadd_rn(a.c, err);
}
// a += x y with the product's rounding error fmaf(x, y, -xy) added to c
__device__ __forceinline__ void acc_fma(acc2& a, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float e = fmaf(x, y, -p);
  acc_add(a, p);
  a.c = __fadd_rn(a.c, e);
}
__device__ __forceinline__ double acc_val(const acc2& a) { return (double)a.s + (double)a.c; }

__device__ __forceinline__ float to_tf32(float f) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(f));
  return __uint_as_float(u);
}

// lo[e] = f in the H~ input format (BF16, TF32 rounded to nearest, FP32, or the BF16X3
// pair: hi at e, lo at n + e)
__device__ __forceinline__ void put_lo(void* lo, int precision, int64_t e, float f, int64_t n) {
  if (precision == DMRG2D_BF16X3) {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    ((__nv_bfloat16*)lo)[e] = h;
    ((__nv_bfloat16*)lo)[n + e] = __float2bfloat16_rn(f - __bfloat162float(h));
  } else if (precision == DMRG2D_BF16)
    ((__nv_bfloat16*)lo)[e] = __float2bfloat16_rn(f);
  else if (precision == DMRG2D_TF32)
    ((float*)lo)[e] = to_tf32(f);
  else
    ((float*)lo)[e] = f;
}

__global__ void k_dot_partial32(const float* __restrict__ a, const float* __restrict__ b,
                                int64_t n, double* __restrict__ part) {
  acc2 s;
#pragma unroll 4
  for (int64_t i = (int64_t)blockIdx.x * VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT)
    acc_fma(s, a[i], b[i]);
  const double v = block_sum(acc_val(s));
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// part[(i0+c)*gridDim.x + blk] = partial of Q_{i0+c} . w   (FP32 basis and vector)
__global__ void k_multidot_partial32(const float* __restrict__ Q, int64_t stride, int k,
                                     const float* __restrict__ w, int64_t n,
                                     double* __restrict__ part) {
  const int i0 = blockIdx.y * MD_CHUNK;
  acc2 acc[MD_CHUNK];
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    const float we = w[e];
#pragma unroll
    for (int c = 0; c < MD_CHUNK; ++c)
      if (i0 + c < k) acc_fma(acc[c], Q[(int64_t)(i0 + c) * stride + e], we);
  }
#pragma unroll
  for (int c = 0; c < MD_CHUNK; ++c) {
    double s = block_sum(acc_val(acc[c]));
    if (threadIdx.x == 0 && i0 + c < k) part[(size_t)(i0 + c) * gridDim.x + blockIdx.x] = s;
  }
}

// out -= sum_i h[i] Q_i (sign = -1) or out = sum_i h[i] Q_i (sign = 0), FP32 arithmetic
template <typename TO>
__global__ void k_combo32(TO* __restrict__ out, const float* __restrict__ Q, int64_t stride, int k,
                          const double* __restrict__ h, int64_t n, int sign) {
  extern __shared__ float hf[];
  for (int i = threadIdx.x; i < k; i += VT) hf[i] = (float)h[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    float s = 0.f;
    for (int i = 0; i < k; ++i) s = fmaf(hf[i], Q[(int64_t)i * stride + e], s);
    out[e] = sign ? (TO)((float)out[e] - s) : (TO)s;
  }
}

// w -= alpha[j] q_j + beta[j-1] q_{j-1}; part[b] = partial w.w of the result
__global__ void k_lz_axpy2_nrm32(float* __restrict__ w, const float* __restrict__ qj,
                                 const float* __restrict__ qjm1, const double* __restrict__ alpha_j,
                                 const double* __restrict__ beta_jm1, int64_t n,
                                 double* __restrict__ part) {
  const float a = (float)*alpha_j;
  const float b = beta_jm1 ? (float)*beta_jm1 : 0.f;
  acc2 s;
#pragma unroll 4
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    float r = fmaf(-a, qj[e], w[e]);
    if (qjm1) r = fmaf(-b, qjm1[e], r);
    w[e] = r;
    acc_fma(s, r, r);
  }
  const double v = block_sum(acc_val(s));
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// q = in / *nrm (zero when the norm is zero) in FP32, and its copy lo in the H~ format
template <typename TI>
__global__ void k_scale_to32(float* __restrict__ q, const TI* __restrict__ in,
                             const double* __restrict__ nrm, void* __restrict__ lo, int precision,
                             int64_t n) {
  const double s = *nrm;
  const float f = s > 0.0 ? (float)(1.0 / s) : 0.f;
#pragma unroll 4
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    const float v = (float)in[e] * f;
    q[e] = v;
    put_lo(lo, precision, e, v, n);
  }
}

// ---- fused conjugate-gradient steps of the mixed solver's inner loop ----------------
// The CG runs on (I - x x^T)(H~ - theta)(I - x x^T) t = -r.  With y = H~ p (FP32, straight
// from the low-precision H·v) the projected operator applied to p is
//   q = y - theta p - (x.q') x,   q' = y - theta p,
// and one step needs x.q', p.q (= p.q' since p is orthogonal to x), then
//   t += a p,  r -= a q,  rr' = r.r,  p = r + (rr'/rr) p.
// Three passes over FP32 vectors (x32 is x rounded to FP32; the correction is
// re-orthogonalised in FP64 afterwards); scalars stay on the device.
enum { CG_XQ = 40, CG_PQ, CG_A, CG_RR, CG_RR1, CG_BETA, CG_THETA };

// CG start: r32 = r, x32 = x, t32 = 0, p32 = r32 and its H~ copy; part[b] = partial r32.r32
__global__ void k_cg_start32(const double* __restrict__ r, const double* __restrict__ x,
                             float* __restrict__ r32, float* __restrict__ x32,
                             float* __restrict__ t32, float* __restrict__ p32,
                             void* __restrict__ lo, int precision, int64_t n,
                             double* __restrict__ part) {
  acc2 s;
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    const float re = (float)r[e];
    r32[e] = re;
    p32[e] = re;
    x32[e] = (float)x[e];
    t32[e] = 0.f;
    put_lo(lo, precision, e, re, n);
    acc_fma(s, re, re);
  }
  const double v = block_sum(acc_val(s));
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// part[b] = partial x.q', part[g + b] = partial p.q'
__global__ void k_cg_dots(const float* __restrict__ y, const float* __restrict__ p,
                          const float* __restrict__ x, const double* __restrict__ scal,
                          int64_t n, double* __restrict__ part) {
  const float theta = (float)scal[CG_THETA];
  acc2 sx, sp;
#pragma unroll 4
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    const float pe = p[e];
    const float q = fmaf(-theta, pe, y[e]);
    acc_fma(sx, x[e], q);
    acc_fma(sp, pe, q);
  }
  const double vx = block_sum(acc_val(sx));
  const double vp = block_sum(acc_val(sp));
  if (threadIdx.x == 0) {
    part[blockIdx.x] = vx;
    part[gridDim.x + blockIdx.x] = vp;
  }
}

// scal[CG_XQ], scal[CG_PQ] from the partials; a = rr / pq (0 when pq <= 0: no update)
__global__ void k_cg_alpha(const double* __restrict__ part, int np, double* __restrict__ scal) {
  double sx = 0.0, sp = 0.0;
  for (int b = threadIdx.x; b < np; b += VT) {
    sx += part[b];
    sp += part[np + b];
  }
  sx = block_sum(sx);
  sp = block_sum(sp);
  if (threadIdx.x == 0) {
    scal[CG_XQ] = sx;
    scal[CG_PQ] = sp;
    scal[CG_A] = sp > 0.0 ? scal[CG_RR] / sp : 0.0;
  }
}

// t += a p, r -= a (y - theta p - xq x); part[b] = partial r.r (of the updated r)
__global__ void k_cg_update(const float* __restrict__ y, const float* __restrict__ p,
                            const float* __restrict__ x, float* __restrict__ t,
                            float* __restrict__ r, const double* __restrict__ scal, int64_t n,
                            double* __restrict__ part) {
  const float a = (float)scal[CG_A], xq = (float)scal[CG_XQ], theta = (float)scal[CG_THETA];
  const bool upd = scal[CG_A] != 0.0;
  acc2 s;
#pragma unroll 4
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    float re = r[e];
    if (upd) {
      const float pe = p[e];
      const float q = fmaf(-xq, x[e], fmaf(-theta, pe, y[e]));
      t[e] = fmaf(a, pe, t[e]);
      re = fmaf(-a, q, re);
      r[e] = re;
    }
    acc_fma(s, re, re);
  }
  const double v = block_sum(acc_val(s));
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// scal[CG_RR1] = sum of partials; beta = rr1 / rr; rr <- rr1
__global__ void k_cg_beta(const double* __restrict__ part, int np, double* __restrict__ scal) {
  double s = 0.0;
  for (int b = threadIdx.x; b < np; b += VT) s += part[b];
  s = block_sum(s);
  if (threadIdx.x == 0) {
    const double rr = scal[CG_RR];
    scal[CG_RR1] = s;
    scal[CG_BETA] = rr > 0.0 ? s / rr : 0.0;
    scal[CG_RR] = s;
  }
}

// p = r + beta p, and the low-precision copy of p that the next H~ p reads
__global__ void k_cg_direction(float* __restrict__ p, const float* __restrict__ r,
                               const double* __restrict__ scal, void* __restrict__ lo,
                               int precision, int64_t n) {
  const float beta = (float)scal[CG_BETA];
#pragma unroll 4
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    const float pe = fmaf(beta, p[e], r[e]);
    p[e] = pe;
    put_lo(lo, precision, e, pe, n);
  }
}

// ---- lowest eigenpair of the Lanczos tridiagonal T_k (diag alpha, off-diag beta) ----
// One block.  The eigenvalue by multisection: every thread evaluates the Sturm count
// (the number of negative pivots of the LDL^T factorisation of T - x, Sylvester's law of
// inertia) at its own point of the current interval, which shrinks 257-fold per round.
// The eigenvector by the twisted factorisation of T - theta (Dhillon and Parlett): the
// top-down LDL^T (thread 0) and bottom-up UDU^T (thread 32) pivots give the twist
// index r with the smallest |gamma_r|, and z solves (T - theta) z = gamma_r e_r with
// z_r = 1 by two product recurrences.  If z is not finite, inverse iteration with
// partial pivoting on one thread is the fallback.
// out[0] = theta, out[1] = |beta_{k-1} s_{k-1}| (the Ritz residual), out[2] = status
// (0 ok, 1 NaN).  k <= TD_MAX.  scratch (fallback only): 5*k doubles.
constexpr int TD_THREADS = 256;
constexpr int TD_MAX = 512;
constexpr int TR_KEEP_MAX = 32;  // Ritz vectors kept at a thick restart

// Negative pivots of LDL^T(T - x) = eigenvalues of T below x; b2 = squared off-diagonal.
// A pivot smaller than pivmin in magnitude is replaced by -pivmin.
__device__ int sturm_count(const double* a, const double* b2, int k, double x, double pivmin) {
  int cnt = 0;
  double q = a[0] - x;
  for (int i = 1;; ++i) {
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
    if (i >= k) break;
    q = (a[i] - x) - b2[i - 1] / q;
  }
  return cnt;
}

// Fallback eigenvector: three steps of inverse iteration, (T - theta) z = s, tridiagonal
// LU with partial pivoting (gtsv style), on one thread.  scr: 5*k doubles.
__device__ bool inverse_iteration(const double* alpha, const double* beta, int k, double theta,
                                  double tiny, double* s, double* scr) {
  double* dl = scr;
  double* dd = scr + k;
  double* du = scr + 2 * k;
  double* du2 = scr + 3 * k;
  double* z = scr + 4 * k;
  for (int i = 0; i < k; ++i) s[i] = 1.0 / sqrt((double)k);
  for (int rep = 0; rep < 3; ++rep) {
    for (int i = 0; i < k; ++i) {
      dd[i] = alpha[i] - theta;
      du[i] = i + 1 < k ? beta[i] : 0.0;
      dl[i] = i + 1 < k ? beta[i] : 0.0;
      du2[i] = 0.0;
      z[i] = s[i];
    }
    for (int i = 0; i + 1 < k; ++i) {
      if (fabs(dd[i]) >= fabs(dl[i])) {
        if (dd[i] == 0.0) dd[i] = tiny;
        const double f = dl[i] / dd[i];
        dd[i + 1] -= f * du[i];
        z[i + 1] -= f * z[i];
        dl[i] = 0.0;
      } else {
        const double f = dd[i] / dl[i];
        dd[i] = dl[i];
        double t = dd[i + 1];
        dd[i + 1] = du[i] - f * t;
        du[i] = t;
        if (i + 2 < k) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
        t = z[i];
        z[i] = z[i + 1];
        z[i + 1] = t - f * z[i + 1];
      }
    }
    if (dd[k - 1] == 0.0) dd[k - 1] = tiny;
    z[k - 1] /= dd[k - 1];
    if (k > 1) z[k - 2] = (z[k - 2] - du[k - 2] * z[k - 1]) / dd[k - 2];
    for (int i = k - 3; i >= 0; --i) z[i] = (z[i] - du[i] * z[i + 1] - du2[i] * z[i + 2]) / dd[i];
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += z[i] * z[i];
    nrm = sqrt(nrm);
    if (!(nrm > 0.0) || !isfinite(nrm)) return false;
    for (int i = 0; i < k; ++i) s[i] = z[i] / nrm;
  }
  return true;
}

// Twisted-factorisation eigenvector of the tridiagonal (a, b) for the eigenvalue theta,
// on one thread: z (unnormalised, z_r = 1).  Dp, Dm, Lf, Ub: k doubles each.
__device__ void twisted_vector(const double* a, const double* b, int k, double theta, double tiny,
                               double* Dp, double* Dm, double* Lf, double* Ub, double* z) {
  double d = a[0] - theta;
  for (int i = 0; i + 1 < k; ++i) {
    if (fabs(d) < tiny) d = d < 0 ? -tiny : tiny;
    Dp[i] = d;
    Lf[i] = b[i] / d;
    d = (a[i + 1] - theta) - Lf[i] * b[i];
  }
  Dp[k - 1] = d;
  d = a[k - 1] - theta;
  for (int i = k - 2; i >= 0; --i) {
    if (fabs(d) < tiny) d = d < 0 ? -tiny : tiny;
    Dm[i + 1] = d;
    Ub[i] = b[i] / d;
    d = (a[i] - theta) - Ub[i] * b[i];
  }
  Dm[0] = d;
  int r = 0;
  double g = INFINITY;
  for (int i = 0; i < k; ++i) {
    const double gi = fabs(Dp[i] + Dm[i] - (a[i] - theta));
    if (gi < g) {
      g = gi;
      r = i;
    }
  }
  z[r] = 1.0;
  for (int i = r - 1; i >= 0; --i) z[i] = -Lf[i] * z[i + 1];
  for (int i = r; i + 1 < k; ++i) z[i + 1] = -Ub[i] * z[i];
}

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Shared set-up of the tridiagonal kernels: a, bb (off-diagonal, bb[k-1] = 0), b2 = bb^2
// in shared memory; Gershgorin interval and pivmin (by thread 0 into *lo, *hi, *pivmin);
// returns false (uniformly) if an entry of alpha[0..k) or beta[0..k) is not finite.
__device__ bool td_setup(const double* __restrict__ alpha, const double* __restrict__ beta, int k,
                         double* a, double* bb, double* b2, double* lo, double* hi,
                         double* pivmin) {
  __shared__ double r_lo[TD_THREADS / 32], r_hi[TD_THREADS / 32], r_b[TD_THREADS / 32];
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  bool mybad = false;
  for (int i = tid; i < k; i += TD_THREADS) {
    const double ai = alpha[i], bi = beta[i];
    if (!isfinite(ai) || !isfinite(bi)) mybad = true;
    a[i] = ai;
    bb[i] = i + 1 < k ? bi : 0.0;
    b2[i] = bb[i] * bb[i];
  }
  if (mybad) atomicOr(&bad, 1);
  __syncthreads();
  double l = 1e300, h = -1e300, bm = 0.0;
  for (int i = tid; i < k; i += TD_THREADS) {
    const double r = (i > 0 ? fabs(bb[i - 1]) : 0.0) + fabs(bb[i]);
    l = fmin(l, a[i] - r);
    h = fmax(h, a[i] + r);
    bm = fmax(bm, b2[i]);
  }
  l = warp_min(l);
  h = warp_max(h);
  bm = warp_max(bm);
  if (lane == 0) {
    r_lo[w] = l;
    r_hi[w] = h;
    r_b[w] = bm;
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 1; i < TD_THREADS / 32; ++i) {
      l = fmin(l, r_lo[i]);
      h = fmax(h, r_hi[i]);
      bm = fmax(bm, r_b[i]);
    }
    *lo = l;
    *hi = h;
    *pivmin = 2.2250738585072014e-308 * fmax(1.0, bm);
  }
  __syncthreads();
  return bad == 0;
}

__global__ void __launch_bounds__(TD_THREADS)
k_tridiag_ground(const double* __restrict__ alpha, const double* __restrict__ beta, int k,
                 double* __restrict__ s, double* __restrict__ out, double* __restrict__ scr) {
  __shared__ double a[TD_MAX], bb[TD_MAX], b2[TD_MAX];
  __shared__ double Dp[TD_MAX], Dm[TD_MAX], Lf[TD_MAX], Ub[TD_MAX], z[TD_MAX];
  __shared__ double sh_lo, sh_hi, sh_piv, sh_red[TD_THREADS / 32];
  __shared__ int sh_first, sh_r[TD_THREADS / 32];
  __shared__ double sh_g[TD_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (!td_setup(alpha, beta, k, a, bb, b2, &sh_lo, &sh_hi, &sh_piv)) {
    if (tid == 0) {
      out[0] = nan("");
      out[1] = nan("");
      out[2] = 1.0;
    }
    return;
  }
  const double pivmin = sh_piv;
  // ---- multisection for the lowest eigenvalue ----
  for (int it = 0; it < 16; ++it) {
    const double L = sh_lo, H = sh_hi;
    if (!(H - L > 4.4e-16 * fmax(fabs(L), fabs(H)) + 1e-300)) break;
    const double x = L + (H - L) * (double)(tid + 1) / (double)(TD_THREADS + 1);
    const bool below = sturm_count(a, b2, k, x, pivmin) >= 1;
    if (tid == 0) sh_first = TD_THREADS;
    __syncthreads();
    if (below) atomicMin(&sh_first, tid);
    __syncthreads();
    if (tid == 0) {
      const int f = sh_first;
      sh_lo = f == 0 ? L : L + (H - L) * (double)f / (double)(TD_THREADS + 1);
      sh_hi = f == TD_THREADS ? H : L + (H - L) * (double)(f + 1) / (double)(TD_THREADS + 1);
    }
    __syncthreads();
  }
  const double theta = 0.5 * (sh_lo + sh_hi);
  const double tiny = 1e-14 * fmax(fabs(sh_lo), fabs(sh_hi)) + 1e-300;
  // ---- twisted factorisation of T - theta ----
  if (tid == 0) {  // top-down LDL^T
    double d = a[0] - theta;
    for (int i = 0; i + 1 < k; ++i) {
      if (fabs(d) < tiny) d = d < 0 ? -tiny : tiny;
      Dp[i] = d;
      Lf[i] = bb[i] / d;
      d = (a[i + 1] - theta) - Lf[i] * bb[i];
    }
    Dp[k - 1] = d;
  } else if (tid == 32) {  // bottom-up UDU^T
    double d = a[k - 1] - theta;
    for (int i = k - 2; i >= 0; --i) {
      if (fabs(d) < tiny) d = d < 0 ? -tiny : tiny;
      Dm[i + 1] = d;
      Ub[i] = bb[i] / d;
      d = (a[i] - theta) - Ub[i] * bb[i];
    }
    Dm[0] = d;
  }
  __syncthreads();
  double g = INFINITY;  // twist index: smallest |gamma_r|, ties to the smaller r
  int r = k;
  for (int i = tid; i < k; i += TD_THREADS) {
    const double gi = fabs(Dp[i] + Dm[i] - (a[i] - theta));
    if (gi < g) {
      g = gi;
      r = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double og = __shfl_down_sync(0xffffffffu, g, o);
    const int orr = __shfl_down_sync(0xffffffffu, r, o);
    if (og < g || (og == g && orr < r)) {
      g = og;
      r = orr;
    }
  }
  if (lane == 0) {
    sh_g[w] = g;
    sh_r[w] = r;
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 1; i < TD_THREADS / 32; ++i)
      if (sh_g[i] < g || (sh_g[i] == g && sh_r[i] < r)) {
        g = sh_g[i];
        r = sh_r[i];
      }
    sh_first = r;
  }
  __syncthreads();
  r = sh_first;
  if (r < k) {
    if (tid == 0) {
      double v = 1.0;
      z[r] = 1.0;
      for (int i = r - 1; i >= 0; --i) {
        v = -Lf[i] * v;
        z[i] = v;
      }
    } else if (tid == 32) {
      double v = 1.0;
      for (int i = r; i + 1 < k; ++i) {
        v = -Ub[i] * v;
        z[i + 1] = v;
      }
    }
  }
  __syncthreads();
  double nn = 0.0;
  if (r < k)
    for (int i = tid; i < k; i += TD_THREADS) nn += z[i] * z[i];
  nn = warp_sum(nn);
  if (lane == 0) sh_red[w] = nn;
  __syncthreads();
  if (tid == 0) {
    for (int i = 1; i < TD_THREADS / 32; ++i) nn += sh_red[i];
    sh_red[0] = (r < k && isfinite(nn) && nn > 0.0) ? sqrt(nn) : -1.0;
  }
  __syncthreads();
  const double nrm = sh_red[0];
  if (nrm < 0.0) {  // fallback: inverse iteration on one thread
    if (tid == 0) {
      const bool ok = inverse_iteration(alpha, beta, k, theta, tiny, s, scr);
      double sg = 1.0;
      for (int i = 0; i < k; ++i)
        if (s[i] != 0.0) {
          sg = s[i] > 0 ? 1.0 : -1.0;
          break;
        }
      for (int i = 0; i < k; ++i) s[i] *= sg;
      out[0] = theta;
      out[1] = fabs(beta[k - 1] * s[k - 1]);
      out[2] = ok ? 0.0 : 1.0;
    }
    return;
  }
  // sign: the first nonzero component positive (deterministic Ritz vector)
  if (tid == 0) sh_first = k;
  __syncthreads();
  for (int i = tid; i < k; i += TD_THREADS)
    if (z[i] != 0.0) {
      atomicMin(&sh_first, i);
      break;
    }
  __syncthreads();
  const double f = (sh_first < k && z[sh_first] < 0.0 ? -1.0 : 1.0) / nrm;
  for (int i = tid; i < k; i += TD_THREADS) s[i] = z[i] * f;
  if (tid == 0) {
    out[0] = theta;
    out[1] = fabs(beta[k - 1] * z[k - 1] * f);
    out[2] = 0.0;
  }
}

// ---- thick restart (Wu and Simon's thick-restart Lanczos) -----------------------------
// At a full basis of k vectors: keep the space of the p lowest Ritz vectors plus the next
// Lanczos vector q_k.  The kept space is re-tridiagonalised so that the recurrence goes on
// unchanged: with S (k x p, orthonormalised) the Ritz coefficient vectors, P = S^T T S and
// the couplings c = beta_{k-1} S[k-1, :] to q_k, a Lanczos process on P started from
// c / |c| gives W (p x p) with W^T P W tridiagonal and W^T c = |c| e_0.  The new basis
// is Z = Q S W in reverse order (z_{p-1}, ..., z_0), then q_k: its projected matrix is
// tridiagonal, with |c| coupling z_0 to q_k.
// Writes M (k x p', column-major, ld k: new vector i = Q M[:, i]), the new alpha[0..p'),
// beta[0..p') (beta[p'-1] = |c|) and out[0] = p' (p' < p if the small Lanczos process
// breaks down or the Ritz vectors are numerically dependent; 0: no restart possible).
// scr: p * (6 k + p) doubles.
__global__ void __launch_bounds__(TD_THREADS)
k_thick_restart(double* __restrict__ alpha, double* __restrict__ beta, int k, int p,
                double* __restrict__ M, double* __restrict__ scr, double* __restrict__ out) {
  __shared__ double a[TD_MAX], bb[TD_MAX], b2[TD_MAX];
  __shared__ double sh_lo, sh_hi, sh_piv, sh_bk, sh_red[TD_THREADS / 32];
  __shared__ double th[TR_KEEP_MAX], P[TR_KEEP_MAX][TR_KEEP_MAX + 1],
      W[TR_KEEP_MAX][TR_KEEP_MAX + 1], cvec[TR_KEEP_MAX], al[TR_KEEP_MAX], be[TR_KEEP_MAX];
  __shared__ int sh_p, sh_pp;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) sh_bk = beta[k - 1];
  if (!td_setup(alpha, beta, k, a, bb, b2, &sh_lo, &sh_hi, &sh_piv) || p < 1 || k < 2) {
    if (tid == 0) out[0] = 0.0;
    return;
  }
  if (p > TR_KEEP_MAX) p = TR_KEEP_MAX;
  if (p > k - 1) p = k - 1;
  const double pivmin = sh_piv;
  // 1. the p lowest eigenvalues, one warp each (32-section, 33-fold per round)
  for (int i = w; i < p; i += TD_THREADS / 32) {
    double L = sh_lo, H = sh_hi;
    for (int it = 0; it < 40; ++it) {
      if (!(H - L > 4.4e-16 * fmax(fabs(L), fabs(H)) + 1e-300)) break;
      const double x = L + (H - L) * (double)(lane + 1) / 33.0;
      const unsigned m = __ballot_sync(0xffffffffu, sturm_count(a, b2, k, x, pivmin) >= i + 1);
      const int f = m ? __ffs(m) - 1 : 32;
      const double nL = f == 0 ? L : L + (H - L) * (double)f / 33.0;
      const double nH = f == 32 ? H : L + (H - L) * (double)(f + 1) / 33.0;
      L = nL;
      H = nH;
    }
    if (lane == 0) th[i] = 0.5 * (L + H);
  }
  __syncthreads();
  // 2. their eigenvectors (twisted factorisation, one thread each) into S (k x p)
  double* S = scr;
  double* TS = scr + (size_t)p * k;
  const double tiny = 1e-14 * fmax(fabs(sh_lo), fabs(sh_hi)) + 1e-300;
  if (tid < p) {
    double* base = scr + 2 * (size_t)p * k + 4 * (size_t)k * tid;
    twisted_vector(a, bb, k, th[tid], tiny, base, base + k, base + 2 * k, base + 3 * k,
                   S + (size_t)tid * k);
  }
  __syncthreads();
  // 3. orthonormalise the columns (Gram-Schmidt twice); stop at a dependent column
  auto block_dot = [&](const double* x, const double* y) -> double {
    double v = 0.0;
    for (int i = tid; i < k; i += TD_THREADS) v += x[i] * y[i];
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh_red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < TD_THREADS / 32; ++i) t += sh_red[i];
    return t;
  };
  if (tid == 0) sh_p = p;
  __syncthreads();
  for (int c = 0; c < p; ++c) {
    double* sc = S + (size_t)c * k;
    const double n0 = sqrt(block_dot(sc, sc));
    if (!(n0 > 0.0) || !isfinite(n0)) {
      if (tid == 0) sh_p = c;
      break;
    }
    for (int i = tid; i < k; i += TD_THREADS) sc[i] /= n0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass)
      for (int c2 = 0; c2 < c; ++c2) {
        const double* s2 = S + (size_t)c2 * k;
        const double dv = block_dot(s2, sc);
        for (int i = tid; i < k; i += TD_THREADS) sc[i] -= dv * s2[i];
        __syncthreads();
      }
    const double n1 = sqrt(block_dot(sc, sc));
    if (!(n1 > 1e-8)) {
      if (tid == 0) sh_p = c;
      break;
    }
    for (int i = tid; i < k; i += TD_THREADS) sc[i] /= n1;
    __syncthreads();
  }
  __syncthreads();
  p = sh_p;
  if (p < 1) {
    if (tid == 0) out[0] = 0.0;
    return;
  }
  // 4. TS = T S, P = S^T T S, c = beta_{k-1} S[k-1, :]
  for (int e = tid; e < p * k; e += TD_THREADS) {
    const int c = e / k, r = e - c * k;
    const double* sc = S + (size_t)c * k;
    double v = a[r] * sc[r];
    if (r > 0) v += bb[r - 1] * sc[r - 1];
    if (r + 1 < k) v += bb[r] * sc[r + 1];
    TS[e] = v;
  }
  __syncthreads();
  for (int e = tid; e < p * p; e += TD_THREADS) {
    const int i = e / p, j = e - i * p;
    const double* si = S + (size_t)i * k;
    const double* tj = TS + (size_t)j * k;
    double v = 0.0;
    for (int r = 0; r < k; ++r) v += si[r] * tj[r];
    P[i][j] = v;
  }
  for (int i = tid; i < p; i += TD_THREADS) cvec[i] = sh_bk * S[(size_t)i * k + k - 1];
  __syncthreads();
  // 5. Lanczos on the symmetrised P from c / |c| (full reorthogonalisation), one thread
  if (tid == 0) {
    double cn = 0.0, pn = 0.0;
    for (int i = 0; i < p; ++i) cn += cvec[i] * cvec[i];
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) pn = fmax(pn, fabs(P[i][j]));
    cn = sqrt(cn);
    int pp = 0;
    if (cn > 0.0 && isfinite(cn)) {
      for (int i = 0; i < p; ++i) W[i][0] = cvec[i] / cn;
      pp = p;
      double u[TR_KEEP_MAX];
      for (int l = 0; l < p; ++l) {
        for (int i = 0; i < p; ++i) {
          double v = 0.0;
          for (int j = 0; j < p; ++j) v += 0.5 * (P[i][j] + P[j][i]) * W[j][l];
          u[i] = v;
        }
        double av = 0.0;
        for (int i = 0; i < p; ++i) av += W[i][l] * u[i];
        al[l] = av;
        if (l + 1 == p) break;
        for (int pass = 0; pass < 2; ++pass)
          for (int l2 = 0; l2 <= l; ++l2) {
            double dv = 0.0;
            for (int i = 0; i < p; ++i) dv += W[i][l2] * u[i];
            for (int i = 0; i < p; ++i) u[i] -= dv * W[i][l2];
          }
        double bn = 0.0;
        for (int i = 0; i < p; ++i) bn += u[i] * u[i];
        bn = sqrt(bn);
        if (!(bn > 1e-12 * pn)) {
          pp = l + 1;
          break;
        }
        be[l] = bn;
        for (int i = 0; i < p; ++i) W[i][l + 1] = u[i] / bn;
      }
    }
    sh_pp = pp;
    sh_red[0] = cn;
  }
  __syncthreads();
  const int pp = sh_pp;
  // 6. M[:, i] = S W[:, pp-1-i]; the new recurrence coefficients
  for (int e = tid; e < pp * k; e += TD_THREADS) {
    const int i = e / k, r = e - i * k;
    const int l = pp - 1 - i;
    double v = 0.0;
    for (int c = 0; c < p; ++c) v += S[(size_t)c * k + r] * W[c][l];
    M[(size_t)i * k + r] = v;
  }
  if (tid < pp) {
    alpha[tid] = al[pp - 1 - tid];
    beta[tid] = tid + 1 < pp ? be[pp - 2 - tid] : sh_red[0];
  }
  if (tid == 0) out[0] = (double)pp;
}

// In place: Q_c[e] = sum_{l<k} M[l + k c] Q_l[e] for c < p <= TR_KEEP_MAX.  Each element's
// k old values are read before its p new ones are written, so the update is safe in place.
__global__ void k_combo_multi(double* __restrict__ Q, int64_t stride, int k,
                              const double* __restrict__ M, int p, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    double acc[TR_KEEP_MAX];
#pragma unroll
    for (int c = 0; c < TR_KEEP_MAX; ++c) acc[c] = 0.0;
    for (int l = 0; l < k; ++l) {
      const double q = Q[(int64_t)l * stride + e];
#pragma unroll
      for (int c = 0; c < TR_KEEP_MAX; ++c)
        if (c < p) acc[c] = fma(M[l + (int64_t)k * c], q, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < TR_KEEP_MAX; ++c)
      if (c < p) Q[(int64_t)c * stride + e] = acc[c];
  }
}

// lowest eigenpair of a small symmetric matrix G (n x n, leading dim ldg) by cyclic Jacobi
// Lowest eigenpair of the symmetrised n x n matrix G (n <= 48): cyclic Jacobi with the
// round-robin ordering, one block: in each round the N/2 disjoint pairs (p, q) of a
// tournament schedule (N = n rounded up to even, a padded index never rotates) get their
// rotations from the same A, then all column and all row updates run in parallel.  A and
// the rotation product V live in shared memory.  out[0] = eigenvalue, c = eigenvector
// (sign: first component >= 0).  scr is unused (kept for the call signature).
constexpr int SE_MAX = 48;
constexpr int SE_THREADS = 256;
__global__ void __launch_bounds__(SE_THREADS)
k_small_eigh(const double* __restrict__ G, int n, int ldg, double* __restrict__ out,
             double* __restrict__ c, double* __restrict__ scr) {
  __shared__ double A[SE_MAX][SE_MAX + 1];
  __shared__ double V[SE_MAX][SE_MAX + 1];
  __shared__ double rc[SE_MAX / 2], rs[SE_MAX / 2];
  __shared__ int rp[SE_MAX / 2], rq[SE_MAX / 2];
  __shared__ double red[SE_THREADS];
  __shared__ int stop;
  const int tid = threadIdx.x;
  const int N = n + (n & 1), half = N / 2;
  for (int e = tid; e < n * n; e += SE_THREADS) {
    const int i = e / n, j = e % n;
    A[i][j] = 0.5 * (G[i * ldg + j] + G[j * ldg + i]);
    V[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < n * n; e += SE_THREADS) {
      const int i = e / n, j = e % n;
      const double v = A[i][j] * A[i][j];
      tot += v;
      if (i != j) off += v;
    }
    red[tid] = off;
    __syncthreads();
    for (int w = SE_THREADS / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    const double off_sum = red[0];
    __syncthreads();
    red[tid] = tot;
    __syncthreads();
    for (int w = SE_THREADS / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) stop = off_sum <= 1e-32 * red[0] + 1e-300;
    __syncthreads();
    if (stop) break;
    for (int round = 0; round < N - 1; ++round) {
      if (tid < half) {  // pair tid of this round: (N-1, round) and a circle around it
        int p, q;
        if (tid == 0) {
          p = round;
          q = N - 1;
        } else {
          p = (round + tid) % (N - 1);
          q = (round + N - 1 - tid) % (N - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double cs = 1.0, sn = 0.0;
        if (q < n) {
          const double apq = A[p][q];
          if (apq != 0.0) {
            const double th = (A[q][q] - A[p][p]) / (2.0 * apq);
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            cs = 1.0 / sqrt(t * t + 1.0);
            sn = t * cs;
          }
        }
        rp[tid] = p;
        rq[tid] = q;
        rc[tid] = cs;
        rs[tid] = sn;
      }
      __syncthreads();
      for (int e = tid; e < half * n; e += SE_THREADS) {  // A <- A J, V <- V J (columns)
        const int k = e / n, r = e % n;
        const int p = rp[k], q = rq[k];
        if (q >= n || rs[k] == 0.0) continue;
        const double cs = rc[k], sn = rs[k];
        const double arp = A[r][p], arq = A[r][q];
        A[r][p] = cs * arp - sn * arq;
        A[r][q] = sn * arp + cs * arq;
        const double vrp = V[r][p], vrq = V[r][q];
        V[r][p] = cs * vrp - sn * vrq;
        V[r][q] = sn * vrp + cs * vrq;
      }
      __syncthreads();
      for (int e = tid; e < half * n; e += SE_THREADS) {  // A <- J^T A (rows)
        const int k = e / n, r = e % n;
        const int p = rp[k], q = rq[k];
        if (q >= n || rs[k] == 0.0) continue;
        const double cs = rc[k], sn = rs[k];
        const double apr = A[p][r], aqr = A[q][r];
        A[p][r] = cs * apr - sn * aqr;
        A[q][r] = sn * apr + cs * aqr;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    int best = 0;
    for (int i = 1; i < n; ++i)
      if (A[i][i] < A[best][best]) best = i;
    const double sg = V[0][best] >= 0 ? 1.0 : -1.0;
    for (int i = 0; i < n; ++i) c[i] = sg * V[i][best];
    out[0] = A[best][best];
  }
}

// ---- host-side helpers ---------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

struct Ctx {
  const dmrg2d_ops* ops;
  cudaStream_t s;
  int64_t n;
  double* part = nullptr;    // RED_BLOCKS * max_k partial sums
  double* scal = nullptr;    // small device scalars
  double* hscal = nullptr;   // pinned host mirror
  void* lo = nullptr;        // low-precision copy of the H·v input
  float* y32 = nullptr;      // low-precision H·v output
  dmrg2d_solver_stats* st = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t ev_used = 0;
  bool timing = true;

  int hv(int prec, const double* x, double* y) {
    cudaEvent_t a = nullptr, b = nullptr;
    D2_TRY(next_events(&a, &b));
    if (prec == DMRG2D_FP64 || prec == DMRG2D_FP64X) {  // the refinement-precision H·v
      if (a) D2_CUDA(cudaEventRecord(a, s));
      if (prec == DMRG2D_FP64X)
        D2_TRY(launch_hv_simt_ff64(ops, x, y, s));
      else
        D2_TRY(launch_hv_simt_f64(ops, x, y, s));
      if (b) D2_CUDA(cudaEventRecord(b, s));
      if (st) st->n_hv_fp64++;
      return DMRG2D_OK;
    }
    D2_TRY(convert_f64_to(x, lo, prec, n, s));
    D2_TRY(hv_lo(prec, a, b));
    k_f32_to_f64<<<vgrid(n), VT, 0, s>>>(y32, y, n);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  }

  // y32 = H~ lo: the low-precision H·v on the already converted input
  int hv_lo(int prec, cudaEvent_t a, cudaEvent_t b, bool count = true) {
    if (a) D2_CUDA(cudaEventRecord(a, s));
    if (prec == DMRG2D_FP32) {
      D2_TRY(launch_hv_simt_f32(ops, (const float*)lo, y32, s));
    } else {
      D2_TRY(launch_hv_tc(ops, lo, y32, prec, s));
    }
    if (b) D2_CUDA(cudaEventRecord(b, s));
    if (st && count) st->n_hv_low++;
    return DMRG2D_OK;
  }
  int hv_lo(int prec) {
    cudaEvent_t a = nullptr, b = nullptr;
    D2_TRY(next_events(&a, &b));
    return hv_lo(prec, a, b);
  }
  int next_events(cudaEvent_t* a, cudaEvent_t* b) {
    if (!timing) return DMRG2D_OK;
    if (ev_used == ev.size()) {
      cudaEvent_t e0, e1;
      D2_CUDA(cudaEventCreate(&e0));
      D2_CUDA(cudaEventCreate(&e1));
      ev.push_back({e0, e1});
    }
    *a = ev[ev_used].first;
    *b = ev[ev_used].second;
    ++ev_used;
    return DMRG2D_OK;
  }

  double hv_ms() {
    double tot = 0.0;
    for (size_t i = 0; i < ev_used; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i].first, ev[i].second) == cudaSuccess) tot += ms;
    }
    return tot;
  }

  ~Ctx() {
    for (auto& e : ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  }

  // *out (device) = a . b
  int dot(const double* a, const double* b, double* out) {
    const int g = vgrid(n);
    k_dot_partial<<<g, VT, 0, s>>>(a, b, n, part);
    k_reduce<<<1, VT, 0, s>>>(part, g, out, 0);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  }
  int nrm(const double* a, double* out) {
    const int g = vgrid(n);
    k_dot_partial<<<g, VT, 0, s>>>(a, a, n, part);
    k_reduce<<<1, VT, 0, s>>>(part, g, out, 1);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  }
  // h[0..k) = Q[0..k) . w
  int multidot(const double* Q, int64_t stride, int k, const double* w, double* h) {
    const int g = vgrid(n);
    dim3 grid(g, (k + MD_CHUNK - 1) / MD_CHUNK);
    k_multidot_partial<<<grid, VT, 0, s>>>(Q, stride, k, w, n, part);
    k_reduce<<<k, VT, 0, s>>>(part, g, h, 0);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  }
  int combo(double* out, const double* Q, int64_t stride, int k, const double* h, int sign) {
    k_combo<<<vgrid(n), VT, k * sizeof(double), s>>>(out, Q, stride, k, h, n, sign);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  }
  int axpby(double* y, const double* x, double a, double b) {
    k_axpby<<<vgrid(n), VT, 0, s>>>(y, x, a, b, n);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  }
  int scale_inv(double* out, const double* in, const double* nrm_dev) {
    k_scale_inv<<<vgrid(n), VT, 0, s>>>(out, in, nrm_dev, n);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  }
  // read k device doubles into the pinned mirror and wait
  int fetch(const double* dsrc, int k) {
    D2_CUDA(cudaMemcpyAsync(hscal, dsrc, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    D2_CUDA(cudaStreamSynchronize(s));
    return DMRG2D_OK;
  }
};

int dmalloc(DevBuf& b, size_t bytes) {
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return set_error(DMRG2D_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  return DMRG2D_OK;
}

// Lanczos from x (FP64, any norm); on return x holds the normalised Ritz vector.
// scal layout: [0] theta, [1] resid, [2] status, [3..] scratch scalars
int lanczos(Ctx& C, int prec, double* x, int max_iter, int kdim, double tol, int fixed,
            int check_every, double* theta_out, double* resid_out, int* iters_out,
            int gs_passes = 2, int thick_keep = 0) {
  const int64_t n = C.n;
  if (kdim < 2) kdim = 2;
  if (kdim > max_iter + 1) kdim = max_iter + 1;
  if (thick_keep > TR_KEEP_MAX) thick_keep = TR_KEEP_MAX;
  if (thick_keep > kdim - 1) thick_keep = kdim - 1;
  DevBuf Qb, wb, ab, bb, hb, sb, tb, Mb, rb;
  if (thick_keep > 0) {
    D2_TRY(dmalloc(Mb, sizeof(double) * (size_t)(kdim + 1) * thick_keep));
    D2_TRY(dmalloc(rb, sizeof(double) * (size_t)thick_keep * (6 * (kdim + 1) + thick_keep)));
  }
  D2_TRY(dmalloc(Qb, sizeof(double) * (size_t)(kdim + 1) * n));
  D2_TRY(dmalloc(wb, sizeof(double) * n));
  D2_TRY(dmalloc(ab, sizeof(double) * (kdim + 1)));
  D2_TRY(dmalloc(bb, sizeof(double) * (kdim + 1)));
  D2_TRY(dmalloc(hb, sizeof(double) * (kdim + 1)));
  D2_TRY(dmalloc(sb, sizeof(double) * (kdim + 1)));
  D2_TRY(dmalloc(tb, sizeof(double) * 6 * (kdim + 1)));
  double* Q = (double*)Qb.p;
  double* w = (double*)wb.p;
  double* alpha = (double*)ab.p;
  double* beta = (double*)bb.p;
  double* h = (double*)hb.p;
  double* sv = (double*)sb.p;
  double* scr = (double*)tb.p;
  double* out3 = C.scal;

  D2_TRY(C.nrm(x, C.scal + 3));
  D2_TRY(C.scale_inv(Q, x, C.scal + 3));
  int j = 0, total = 0;
  double theta = 0.0, resid = INFINITY;
  int status = DMRG2D_ENOCONV;
  if (check_every < 1) check_every = 1;
  while (true) {
    double* qj = Q + (int64_t)j * n;
    D2_TRY(C.hv(prec, qj, w));
    D2_TRY(C.dot(qj, w, alpha + j));
    k_lz_axpy2<<<vgrid(n), VT, 0, C.s>>>(w, qj, j > 0 ? qj - n : nullptr, alpha + j,
                                        j > 0 ? beta + j - 1 : nullptr, n);
    D2_CUDA(cudaGetLastError());
    for (int pass = 0; pass < gs_passes; ++pass) {  // CGS2 (or fewer) against q_0..q_j
      D2_TRY(C.multidot(Q, n, j + 1, w, h));
      D2_TRY(C.combo(w, Q, n, j + 1, h, -1));
    }
    D2_TRY(C.nrm(w, beta + j));
    ++j;
    ++total;
    const bool last = total >= max_iter;
    const bool full = j >= kdim;
    if (last || full || (!fixed && total % check_every == 0)) {
      k_tridiag_ground<<<1, TD_THREADS, 0, C.s>>>(alpha, beta, j, sv, out3, scr);
      D2_CUDA(cudaGetLastError());
      D2_TRY(C.fetch(out3, 3));
      theta = C.hscal[0];
      resid = C.hscal[1];
      if (C.hscal[2] != 0.0 || !std::isfinite(theta)) {
        status = set_error(DMRG2D_ENAN, "NaN/Inf in the Lanczos recurrence");
        break;
      }
      const bool conv = !fixed && resid <= tol * fabs(theta);
      if (full && !conv && !last && thick_keep > 0) {
        // thick restart: q_j = w / beta_{j-1} joins the re-tridiagonalised Ritz space
        D2_TRY(C.scale_inv(Q + (int64_t)j * n, w, beta + j - 1));
        k_thick_restart<<<1, TD_THREADS, 0, C.s>>>(alpha, beta, j, thick_keep, (double*)Mb.p,
                                                   (double*)rb.p, C.scal + 7);
        D2_CUDA(cudaGetLastError());
        D2_TRY(C.fetch(C.scal + 7, 1));
        const int pk = (int)C.hscal[0];
        if (pk >= 1) {
          k_combo_multi<<<vgrid(n), VT, 0, C.s>>>(Q, n, j, (const double*)Mb.p, pk, n);
          D2_CUDA(cudaGetLastError());
          D2_CUDA(cudaMemcpyAsync(Q + (int64_t)pk * n, Q + (int64_t)j * n, sizeof(double) * n,
                                  cudaMemcpyDeviceToDevice, C.s));
          j = pk;
          continue;
        }
      }
      if (conv || last || full) {
        D2_TRY(C.combo(x, Q, n, j, sv, 0));  // Ritz vector
        if (conv) {
          status = DMRG2D_OK;
          break;
        }
        if (last) {
          status = fixed ? DMRG2D_OK : DMRG2D_ENOCONV;
          if (!fixed) set_error(DMRG2D_ENOCONV, "Lanczos: %d steps, residual %.3e", total, resid);
          break;
        }
        // explicit restart from the Ritz vector
        D2_TRY(C.nrm(x, C.scal + 3));
        D2_TRY(C.scale_inv(Q, x, C.scal + 3));
        j = 0;
        continue;
      }
    }
    D2_TRY(C.scale_inv(Q + (int64_t)j * n, w, beta + j - 1));
  }
  D2_TRY(C.nrm(x, C.scal + 3));
  D2_TRY(C.scale_inv(x, x, C.scal + 3));
  *theta_out = theta;
  *resid_out = resid;
  *iters_out = total;
  return status;
}

// Low-precision Lanczos for the mixed solver's start vector: H~ with an FP32 basis (the
// three-term recurrence plus gs_passes classical Gram-Schmidt passes), explicit restarts
// from the Ritz vector every kdim steps.  x (FP64): the start vector in, the normalised
// Ritz vector out.  Per step: H~ q_j into y32, alpha = q_j.w, w -= alpha q_j + beta q_{j-1}
// with |w| in the same pass, q_{j+1} = w / beta with its H~ copy in the same pass.
int lanczos_lo(Ctx& C, int prec, double* x, int max_iter, int kdim, double tol, int check_every,
               double* theta_out, double* resid_out, int* iters_out, int gs_passes) {
  const int64_t n = C.n;
  if (kdim < 2) kdim = 2;
  if (kdim > max_iter + 1) kdim = max_iter + 1;
  DevBuf Qb, ab, bb, hb, sb, tb;
  D2_TRY(dmalloc(Qb, sizeof(float) * (size_t)(kdim + 1) * n));
  D2_TRY(dmalloc(ab, sizeof(double) * (kdim + 1)));
  D2_TRY(dmalloc(bb, sizeof(double) * (kdim + 1)));
  D2_TRY(dmalloc(hb, sizeof(double) * (kdim + 1)));
  D2_TRY(dmalloc(sb, sizeof(double) * (kdim + 1)));
  D2_TRY(dmalloc(tb, sizeof(double) * 6 * (kdim + 1)));
  float* Q = (float*)Qb.p;
  float* w = C.y32;  // H~ q_j lands here and is orthogonalised in place
  double* alpha = (double*)ab.p;
  double* beta = (double*)bb.p;
  double* h = (double*)hb.p;
  double* sv = (double*)sb.p;
  double* scr = (double*)tb.p;
  double* out3 = C.scal;
  const int g = vgrid(n);
  auto start_from_x = [&]() -> int {
    D2_TRY(C.nrm(x, C.scal + 3));
    k_scale_to32<double><<<g, VT, 0, C.s>>>(Q, x, C.scal + 3, C.lo, prec, n);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  };
  D2_TRY(start_from_x());
  int j = 0, total = 0;
  double theta = 0.0, resid = INFINITY;
  int status = DMRG2D_ENOCONV;
  if (check_every < 1) check_every = 1;
  while (true) {
    float* qj = Q + (int64_t)j * n;
    D2_TRY(C.hv_lo(prec));  // w = H~ q_j (its H~-format copy is in C.lo)
    k_dot_partial32<<<g, VT, 0, C.s>>>(qj, w, n, C.part);
    k_reduce<<<1, VT, 0, C.s>>>(C.part, g, alpha + j, 0);
    k_lz_axpy2_nrm32<<<g, VT, 0, C.s>>>(w, qj, j > 0 ? qj - n : nullptr, alpha + j,
                                        j > 0 ? beta + j - 1 : nullptr, n, C.part);
    k_reduce<<<1, VT, 0, C.s>>>(C.part, g, beta + j, 1);
    for (int pass = 0; pass < gs_passes; ++pass) {  // CGS against q_0..q_j
      dim3 grid(g, (j + 1 + MD_CHUNK - 1) / MD_CHUNK);
      k_multidot_partial32<<<grid, VT, 0, C.s>>>(Q, n, j + 1, w, n, C.part);
      k_reduce<<<j + 1, VT, 0, C.s>>>(C.part, g, h, 0);
      k_combo32<float><<<g, VT, (j + 1) * sizeof(float), C.s>>>(w, Q, n, j + 1, h, n, -1);
      if (pass + 1 == gs_passes) {
        k_dot_partial32<<<g, VT, 0, C.s>>>(w, w, n, C.part);
        k_reduce<<<1, VT, 0, C.s>>>(C.part, g, beta + j, 1);
      }
    }
    D2_CUDA(cudaGetLastError());
    ++j;
    ++total;
    const bool last = total >= max_iter;
    const bool full = j >= kdim;
    if (last || full || total % check_every == 0) {
      k_tridiag_ground<<<1, TD_THREADS, 0, C.s>>>(alpha, beta, j, sv, out3, scr);
      D2_CUDA(cudaGetLastError());
      D2_TRY(C.fetch(out3, 3));
      theta = C.hscal[0];
      resid = C.hscal[1];
      if (C.hscal[2] != 0.0 || !std::isfinite(theta)) {
        status = set_error(DMRG2D_ENAN, "NaN/Inf in the low-precision Lanczos recurrence");
        break;
      }
      const bool conv = resid <= tol * fabs(theta);
      if (conv || last || full) {
        k_combo32<double><<<g, VT, j * sizeof(float), C.s>>>(x, Q, n, j, sv, n, 0);  // Ritz
        D2_CUDA(cudaGetLastError());
        if (conv || last) {
          status = conv ? DMRG2D_OK : DMRG2D_ENOCONV;
          break;
        }
        D2_TRY(start_from_x());  // explicit restart from the Ritz vector
        j = 0;
        continue;
      }
    }
    k_scale_to32<float><<<g, VT, 0, C.s>>>(Q + (int64_t)j * n, w, beta + j - 1, C.lo, prec, n);
    D2_CUDA(cudaGetLastError());
  }
  D2_TRY(C.nrm(x, C.scal + 3));
  D2_TRY(C.scale_inv(x, x, C.scal + 3));
  *theta_out = theta;
  *resid_out = resid;
  *iters_out = total;
  return status;
}

}  // namespace

int convert_f64_to(const double* x, void* out, int precision, int64_t n, cudaStream_t s) {
  if (precision == DMRG2D_BF16X3)
    k_f64_to_bf16x3<<<vgrid(n), VT, 0, s>>>(x, (__nv_bfloat16*)out, n);
  else if (precision == DMRG2D_BF16)
    k_f64_to_bf16<<<vgrid(n), VT, 0, s>>>(x, (__nv_bfloat16*)out, n);
  else if (precision == DMRG2D_TF32)
    k_f64_to_tf32<<<vgrid(n), VT, 0, s>>>(x, (float*)out, n);
  else
    k_f64_to_f32<<<vgrid(n), VT, 0, s>>>(x, (float*)out, n);
  D2_CUDA(cudaGetLastError());
  return DMRG2D_OK;
}

// A fixed sequence of launches (one inner CG step) captured into a CUDA graph on a
// private stream and replayed on the solver's stream: one graph launch per step instead of
// seven kernel launches and a copy.  The captured work reads its scalars (theta, a, beta)
// from device memory, so the same graph serves every outer iteration.
constexpr int HS_THETA = 60;  // pinned-mirror slot holding theta for its upload

struct StepGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;

  template <typename F>
  int capture(Ctx& C, F&& body) {
    if (!cs) D2_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const cudaStream_t saved = C.s;  // captured work is recorded, not run: no ordering needed
    C.s = cs;
    D2_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int st = body();
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    C.s = saved;
    if (st != DMRG2D_OK) return st;
    if (e != cudaSuccess) return set_error(DMRG2D_ECUDA, "CG step capture: %s", cudaGetErrorString(e));
    D2_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    return DMRG2D_OK;
  }
  ~StepGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
  }
};

// Mixed precision: low-precision Lanczos start, FP64 outer Rayleigh-Ritz + CG corrections.
static int mixed_outer(Ctx& C, const dmrg2d_solver_opts* o, double* x, double* energy);

static int mixed_solve(Ctx& C, const dmrg2d_solver_opts* o, double* x, double* energy) {
  // 1. low-precision Lanczos for the start vector
  double th0 = 0, r0 = 0;
  int it0 = 0;
  // basis capped at krylov_dim vectors (explicit restarts), so memory does not grow with
  // inner_iter
  const int kdim1 = std::max(2, std::min(o->inner_iter, o->krylov_dim) + 1);
  const int passes = std::min(2, std::max(0, o->start_reorth));
  int st = lanczos_lo(C, o->precision, x, o->inner_iter, kdim1, 1e-6, 5, &th0, &r0, &it0, passes);
  if (st != DMRG2D_OK && st != DMRG2D_ENOCONV) return st;
  C.st->iters += it0;
  // 2. FP64 outer loop
  return mixed_outer(C, o, x, energy);
}

// FP64 outer loop on a small subspace, starting from x.
static int mixed_outer(Ctx& C, const dmrg2d_solver_opts* o, double* x, double* energy) {
  const int64_t n = C.n;
  const int prec = o->precision;
  const int smax = 6;
  DevBuf Ub, Wb, hxb, rb, tb, r32b, x32b, t32b, p32b, Gb, cb, scb;
  D2_TRY(dmalloc(Ub, sizeof(double) * (size_t)smax * n));
  D2_TRY(dmalloc(Wb, sizeof(double) * (size_t)smax * n));
  D2_TRY(dmalloc(hxb, sizeof(double) * n));
  D2_TRY(dmalloc(rb, sizeof(double) * n));
  D2_TRY(dmalloc(tb, sizeof(double) * n));
  D2_TRY(dmalloc(r32b, sizeof(float) * n));  // the CG's vectors, FP32
  D2_TRY(dmalloc(x32b, sizeof(float) * n));
  D2_TRY(dmalloc(t32b, sizeof(float) * n));
  D2_TRY(dmalloc(p32b, sizeof(float) * n));
  D2_TRY(dmalloc(Gb, sizeof(double) * smax * smax));
  D2_TRY(dmalloc(cb, sizeof(double) * smax));
  D2_TRY(dmalloc(scb, sizeof(double) * 2 * smax * smax));
  double *U = (double*)Ub.p, *W = (double*)Wb.p, *hx = (double*)hxb.p, *r = (double*)rb.p;
  double *t = (double*)tb.p, *G = (double*)Gb.p;
  float *r32 = (float*)r32b.p, *x32 = (float*)x32b.p, *t32 = (float*)t32b.p, *p32 = (float*)p32b.p;
  double *cc = (double*)cb.p, *scr = (double*)scb.p;
  double* sc = C.scal;  // scalars: [4] tmp dot, [5..] host-fetched, [CG_XQ..] CG state
  const int g = vgrid(n);
  StepGraph step;  // the inner CG step, captured once and replayed
  D2_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * smax * smax, C.s));

  D2_TRY(C.nrm(x, sc + 3));
  D2_TRY(C.scale_inv(U, x, sc + 3));
  const int rprec = o->refine_precision == DMRG2D_FP64X ? DMRG2D_FP64X : DMRG2D_FP64;
  D2_TRY(C.hv(rprec, U, W));
  int s = 1;
  std::vector<double> Gh(smax * smax, 0.0);
  auto update_G_col = [&](int jcol) -> int {
    // G[i][jcol] = U_i . W_jcol for i <= jcol; mirror
    D2_TRY(C.multidot(U, n, jcol + 1, W + (int64_t)jcol * n, sc + 8));
    D2_TRY(C.fetch(sc + 8, jcol + 1));
    for (int i = 0; i <= jcol; ++i) Gh[i * smax + jcol] = Gh[jcol * smax + i] = C.hscal[i];
    return DMRG2D_OK;
  };
  D2_TRY(update_G_col(0));
  double theta = 0.0, rn = INFINITY;
  int status = DMRG2D_ENOCONV;
  for (int outer = 0; outer <= o->outer_max; ++outer) {
    D2_CUDA(cudaMemcpyAsync(G, Gh.data(), sizeof(double) * smax * smax, cudaMemcpyHostToDevice, C.s));
    k_small_eigh<<<1, SE_THREADS, 0, C.s>>>(G, s, smax, sc + 5, cc, scr);
    D2_CUDA(cudaGetLastError());
    D2_TRY(C.combo(x, U, n, s, cc, 0));
    D2_TRY(C.combo(hx, W, n, s, cc, 0));
    D2_TRY(C.fetch(sc + 5, 1));
    theta = C.hscal[0];
    D2_CUDA(cudaMemcpyAsync(r, hx, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.s));
    D2_TRY(C.axpby(r, x, -theta, 1.0));  // r = hx - theta x
    D2_TRY(C.nrm(r, sc + 6));
    D2_TRY(C.fetch(sc + 6, 1));
    rn = C.hscal[0];
    C.st->outer = outer;
    if (!std::isfinite(theta) || !std::isfinite(rn)) {
      status = set_error(DMRG2D_ENAN, "NaN/Inf in the FP64 outer loop");
      break;
    }
    if (rn <= o->tol * fabs(theta)) {
      status = DMRG2D_OK;
      break;
    }
    if (outer == o->outer_max) {
      set_error(DMRG2D_ENOCONV, "mixed: %d outer steps, residual %.3e", outer, rn);
      break;
    }
    // ---- inner CG on (I - xx^T)(H~ - theta)(I - xx^T) t = -r, t0 = 0, FP32 vectors ----
    // res (stored in r) = -r projected; r32 = res, x32 = x, t32 = 0, p32 = res
    D2_TRY(C.axpby(r, r, 0.0, -1.0));
    D2_TRY(C.dot(x, r, sc + 4));
    D2_TRY(C.fetch(sc + 4, 1));
    D2_TRY(C.axpby(r, x, -C.hscal[0], 1.0));
    C.hscal[HS_THETA] = theta;
    D2_CUDA(cudaMemcpyAsync(sc + CG_THETA, C.hscal + HS_THETA, sizeof(double),
                            cudaMemcpyHostToDevice, C.s));
    k_cg_start32<<<g, VT, 0, C.s>>>(r, x, r32, x32, t32, p32, C.lo, prec, n, C.part);
    k_reduce<<<1, VT, 0, C.s>>>(C.part, g, sc + CG_RR, 0);
    D2_CUDA(cudaGetLastError());
    D2_TRY(C.fetch(sc + CG_RR, 1));
    const double rr0 = C.hscal[0];
    if (!step.exec) D2_TRY(step.capture(C, [&]() -> int {
      // one CG step: y32 = H~ p, the fused vector passes, scalars to the pinned mirror
      D2_TRY(C.hv_lo(prec, nullptr, nullptr, false));  // counted per replay
      k_cg_dots<<<g, VT, 0, C.s>>>(C.y32, p32, x32, sc, n, C.part);
      k_cg_alpha<<<1, VT, 0, C.s>>>(C.part, g, sc);
      k_cg_update<<<g, VT, 0, C.s>>>(C.y32, p32, x32, t32, r32, sc, n, C.part);
      k_cg_beta<<<1, VT, 0, C.s>>>(C.part, g, sc);
      k_cg_direction<<<g, VT, 0, C.s>>>(p32, r32, sc, C.lo, prec, n);
      D2_CUDA(cudaGetLastError());
      D2_CUDA(cudaMemcpyAsync(C.hscal, sc + CG_PQ, sizeof(double) * (CG_RR1 - CG_PQ + 1),
                              cudaMemcpyDeviceToHost, C.s));
      return DMRG2D_OK;
    }));
    for (int it = 0; it < o->inner_iter; ++it) {
      D2_CUDA(cudaGraphLaunch(step.exec, C.s));
      D2_CUDA(cudaStreamSynchronize(C.s));  // one wait per step
      const double pq = C.hscal[0], rr1 = C.hscal[CG_RR1 - CG_PQ];
      C.st->n_hv_low++;
      C.st->iters++;
      if (!(pq > 0.0)) break;  // (no update was made)
      if (rr1 <= 1e-8 * rr0) break;
    }
    k_f32_to_f64<<<g, VT, 0, C.s>>>(t32, t, n);
    D2_CUDA(cudaGetLastError());
    // ---- orthonormalise t against U and extend the subspace ----
    if (s == smax) {  // restart with the current Ritz pair
      D2_CUDA(cudaMemcpyAsync(U, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.s));
      D2_CUDA(cudaMemcpyAsync(W, hx, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.s));
      s = 1;
      std::fill(Gh.begin(), Gh.end(), 0.0);
      Gh[0] = theta;
    }
    for (int pass = 0; pass < 2; ++pass) {
      D2_TRY(C.multidot(U, n, s, t, sc + 8));
      D2_TRY(C.combo(t, U, n, s, sc + 8, -1));
    }
    D2_TRY(C.nrm(t, sc + 4));
    D2_TRY(C.fetch(sc + 4, 1));
    if (!(C.hscal[0] > 0.0)) {
      set_error(DMRG2D_ENOCONV, "mixed: correction vanished, residual %.3e", rn);
      break;
    }
    D2_TRY(C.scale_inv(U + (int64_t)s * n, t, sc + 4));
    D2_TRY(C.hv(rprec, U + (int64_t)s * n, W + (int64_t)s * n));
    D2_TRY(update_G_col(s));
    ++s;
  }
  C.st->resid = rn;
  *energy = theta;
  return status;
}

}  // namespace dmrg2d

using namespace dmrg2d;

extern "C" int dmrg2d_lanczos_ground(const dmrg2d_ops* ops, const dmrg2d_solver_opts* opts,
                                     double* x_inout, double* energy_out,
                                     dmrg2d_solver_stats* stats, void* stream) {
  if (!ops || !x_inout || !energy_out) return set_error(DMRG2D_EINVAL, "NULL argument");
  clear_error();
  dmrg2d_solver_opts o;
  if (opts) o = *opts; else dmrg2d_default_solver_opts(&o);
  if (o.max_iter < 1) return set_error(DMRG2D_EINVAL, "max_iter < 1");
  if (o.krylov_dim > 512 || o.inner_iter > 511)
    return set_error(DMRG2D_EINVAL, "krylov_dim > 512 or inner_iter > 511");
  if (o.thick_keep < 0 || o.thick_keep > 32)
    return set_error(DMRG2D_EINVAL, "thick_keep must be in [0, 32]");
  if (o.precision != DMRG2D_FP64 && o.precision != DMRG2D_FP32 && o.precision != DMRG2D_TF32 &&
      o.precision != DMRG2D_BF16 && o.precision != DMRG2D_BF16X3)
    return set_error(DMRG2D_EINVAL, "unknown precision %d", o.precision);
  if ((o.precision == DMRG2D_TF32 || o.precision == DMRG2D_BF16 ||
       o.precision == DMRG2D_BF16X3) && !ops->tc_ok)
    return set_error(DMRG2D_EUNSUPPORTED, "tensor-core path unsupported for these shapes");
  if (o.refine_precision != DMRG2D_FP64 && o.refine_precision != DMRG2D_FP64X)
    return set_error(DMRG2D_EINVAL, "refine_precision must be FP64 or FP64X");
  const auto t0 = std::chrono::steady_clock::now();
  dmrg2d_solver_stats local{};
  Ctx C;
  C.ops = ops;
  C.s = (cudaStream_t)stream;
  C.n = ops->n_vec;
  C.st = &local;
  DevBuf part, scal, lo, y32;
  D2_TRY(dmalloc(part, sizeof(double) * (size_t)RED_BLOCKS * 520));
  D2_TRY(dmalloc(scal, sizeof(double) * 64));
  C.part = (double*)part.p;
  C.scal = (double*)scal.p;
  D2_CUDA(cudaMallocHost(&C.hscal, sizeof(double) * 64));
  struct PinnedFree {
    double* p;
    ~PinnedFree() { cudaFreeHost(p); }
  } pf{C.hscal};
  if (o.precision != DMRG2D_FP64) {
    D2_TRY(dmalloc(lo, (o.precision == DMRG2D_BF16 ? 2 : 4) * (size_t)C.n));
    D2_TRY(dmalloc(y32, sizeof(float) * (size_t)C.n));
    C.lo = lo.p;
    C.y32 = (float*)y32.p;
  }
  int st;
  double energy = 0.0;
  D2_TRY(sec_zero_padding(ops, x_inout, C.s));  // restricted layouts: padding rows stay zero
  if (o.refine && o.precision != DMRG2D_FP64) {
    st = mixed_solve(C, &o, x_inout, &energy);
  } else {
    double resid = 0.0;
    int iters = 0;
    st = lanczos(C, o.precision, x_inout, o.max_iter, o.krylov_dim, o.tol, o.fixed_steps,
                 o.check_every, &energy, &resid, &iters, 2, o.thick_keep);
    local.iters = iters;
    local.resid = resid;
  }
  cudaError_t e = cudaStreamSynchronize(C.s);
  if (e != cudaSuccess && st == DMRG2D_OK)
    st = set_error(DMRG2D_ECUDA, "solver: %s", cudaGetErrorString(e));
  int derr = 0;
  if (tc_read_error(ops, &derr) == DMRG2D_OK && derr && st == DMRG2D_OK)
    st = set_error(DMRG2D_ETIMEOUT, "tensor-core kernel gave up waiting (site %d)", derr);
  local.hv_ms = C.hv_ms();
  local.elapsed_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *energy_out = energy;
  if (stats) *stats = local;
  return st;
}

extern "C" int dmrg2d_convert_input(const double* x, void* out, int precision, int64_t n,
                                    void* stream) {
  if (!x || !out) return set_error(DMRG2D_EINVAL, "NULL argument");
  if (n < 0) return set_error(DMRG2D_EINVAL, "n < 0");
  const cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) return DMRG2D_OK;
  switch (precision) {
    case DMRG2D_FP64:
    case DMRG2D_FP64X:
      D2_CUDA(cudaMemcpyAsync(out, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      return DMRG2D_OK;
    case DMRG2D_FP32:
    case DMRG2D_TF32:
    case DMRG2D_BF16:
    case DMRG2D_BF16X3:
      return convert_f64_to(x, out, precision, n, st);
    default:
      return set_error(DMRG2D_EINVAL, "unknown precision %d", precision);
  }
}

extern "C" int dmrg2d_tridiag_lowest(const double* alpha, const double* beta, int k, double* s,
                                     double* out, void* stream) {
  if (!alpha || !beta || !s || !out) return set_error(DMRG2D_EINVAL, "NULL argument");
  if (k < 1 || k > TD_MAX) return set_error(DMRG2D_ESHAPE, "k = %d outside [1, %d]", k, TD_MAX);
  clear_error();
  const cudaStream_t st = (cudaStream_t)stream;
  // the fallback's scratch lives past the 3 outputs: out[3 .. 3 + 5k)
  k_tridiag_ground<<<1, TD_THREADS, 0, st>>>(alpha, beta, k, s, out, out + 3);
  D2_CUDA(cudaGetLastError());
  return DMRG2D_OK;
}

// ---- allocation-free Lanczos for small superblocks ----------------------------------------
// All scratch of this entry point (Krylov basis, work vector, reduction partials, the
// tridiagonal coefficients and eigensolver workspace, device scalars) lives in one
// file-scope device array.  Host code never dereferences the array's name: it asks the
// runtime for the array's device address once per device and hands that to the kernels.
static __device__ __align__(256) double g_noalloc_scratch[DMRG2D_NOALLOC_SCRATCH_DOUBLES];

#include <mutex>

namespace dmrg2d {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up on first use).
int noalloc_scratch(double** out) {
  int dev = 0;
  D2_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(DMRG2D_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(DMRG2D_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s",
                       cudaGetErrorString(e));
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return DMRG2D_OK;
}

// Same recurrence as lanczos() above, with every buffer carved out of `ws`.
int lanczos_in_place(Ctx& C, double* ws, double* x, int max_iter, int kdim, double tol, int fixed,
                     int check_every, double* theta_out, double* resid_out, int* iters_out) {
  const int64_t n = C.n;
  double* Q = ws;
  double* w = Q + (int64_t)(kdim + 1) * n;
  double* alpha = w + n;
  double* beta = alpha + (kdim + 1);
  double* h = beta + (kdim + 1);
  double* sv = h + (kdim + 1);
  double* scr = sv + (kdim + 1);
  double* out3 = C.scal;
  D2_TRY(C.nrm(x, C.scal + 3));
  D2_TRY(C.scale_inv(Q, x, C.scal + 3));
  int j = 0, total = 0;
  double theta = 0.0, resid = INFINITY;
  int status = DMRG2D_ENOCONV;
  if (check_every < 1) check_every = 1;
  while (true) {
    double* qj = Q + (int64_t)j * n;
    D2_TRY(C.hv(DMRG2D_FP64, qj, w));
    D2_TRY(C.dot(qj, w, alpha + j));
    k_lz_axpy2<<<vgrid(n), VT, 0, C.s>>>(w, qj, j > 0 ? qj - n : nullptr, alpha + j,
                                        j > 0 ? beta + j - 1 : nullptr, n);
    D2_CUDA(cudaGetLastError());
    for (int pass = 0; pass < 2; ++pass) {
      D2_TRY(C.multidot(Q, n, j + 1, w, h));
      D2_TRY(C.combo(w, Q, n, j + 1, h, -1));
    }
    D2_TRY(C.nrm(w, beta + j));
    ++j;
    ++total;
    const bool last = total >= max_iter;
    const bool full = j >= kdim;
    if (last || full || (!fixed && total % check_every == 0)) {
      k_tridiag_ground<<<1, TD_THREADS, 0, C.s>>>(alpha, beta, j, sv, out3, scr);
      D2_CUDA(cudaGetLastError());
      D2_TRY(C.fetch(out3, 3));
      theta = C.hscal[0];
      resid = C.hscal[1];
      if (C.hscal[2] != 0.0 || !std::isfinite(theta)) {
        status = set_error(DMRG2D_ENAN, "NaN/Inf in the Lanczos recurrence");
        break;
      }
      const bool conv = !fixed && resid <= tol * fabs(theta);
      if (conv || last || full) {
        D2_TRY(C.combo(x, Q, n, j, sv, 0));
        if (conv) {
          status = DMRG2D_OK;
          break;
        }
        if (last) {
          status = fixed ? DMRG2D_OK : DMRG2D_ENOCONV;
          if (!fixed) set_error(DMRG2D_ENOCONV, "Lanczos: %d steps, residual %.3e", total, resid);
          break;
        }
        D2_TRY(C.nrm(x, C.scal + 3));
        D2_TRY(C.scale_inv(Q, x, C.scal + 3));
        j = 0;
        continue;
      }
    }
    D2_TRY(C.scale_inv(Q + (int64_t)j * n, w, beta + j - 1));
  }
  D2_TRY(C.nrm(x, C.scal + 3));
  D2_TRY(C.scale_inv(x, x, C.scal + 3));
  *theta_out = theta;
  *resid_out = resid;
  *iters_out = total;
  return status;
}

}  // namespace
}  // namespace dmrg2d

extern "C" int dmrg2d_lanczos_ground_noalloc(const dmrg2d_ops* ops, const dmrg2d_solver_opts* opts,
                                             double* x_inout, double* energy_out,
                                             dmrg2d_solver_stats* stats, void* stream) {
  using namespace dmrg2d;
  if (!ops || !x_inout || !energy_out) return set_error(DMRG2D_EINVAL, "NULL argument");
  clear_error();
  dmrg2d_solver_opts o;
  if (opts) o = *opts; else dmrg2d_default_solver_opts(&o);
  if (o.precision != DMRG2D_FP64 || o.refine)
    return set_error(DMRG2D_EUNSUPPORTED, "the allocation-free solver runs plain FP64 Lanczos only");
  if (o.thick_keep != 0)
    return set_error(DMRG2D_EUNSUPPORTED,
                     "the allocation-free solver restarts explicitly (thick_keep must be 0)");
  if (o.max_iter < 1) return set_error(DMRG2D_EINVAL, "max_iter < 1");
  int kdim = o.krylov_dim < 2 ? 2 : o.krylov_dim;
  if (kdim > o.max_iter + 1) kdim = o.max_iter + 1;
  if (kdim > 512)  // the reduction partials and the tridiagonal workspace are sized for 512
    return set_error(DMRG2D_ESHAPE,
                     "allocation-free Lanczos: krylov_dim %d (after clamping to max_iter + 1) "
                     "exceeds 512", kdim);
  const int64_t n = ops->n_vec;
  const int64_t need = (int64_t)(kdim + 2) * n + 10 * (int64_t)(kdim + 1) +
                       (int64_t)RED_BLOCKS * (kdim + 1) + 64;
  if (need > (int64_t)DMRG2D_NOALLOC_SCRATCH_DOUBLES)
    return set_error(DMRG2D_ESHAPE,
                     "allocation-free Lanczos needs %lld scratch doubles for n_vec=%lld, "
                     "krylov_dim=%d; the static scratch holds %lld (reduce krylov_dim or use "
                     "dmrg2d_lanczos_ground)",
                     (long long)need, (long long)n, kdim,
                     (long long)DMRG2D_NOALLOC_SCRATCH_DOUBLES);
  int cur = -1;
  D2_CUDA(cudaGetDevice(&cur));
  if (cur != ops->device)
    return set_error(DMRG2D_EINVAL,
                     "allocation-free Lanczos: device %d is current but the ops were built on "
                     "device %d (the static scratch is per device)", cur, ops->device);
  double* ws = nullptr;
  D2_TRY(noalloc_scratch(&ws));
  const auto t0 = std::chrono::steady_clock::now();
  dmrg2d_solver_stats local{};
  double hscal[64];
  Ctx C;
  C.ops = ops;
  C.s = (cudaStream_t)stream;
  C.n = n;
  C.st = &local;
  C.timing = false;  // no event creation on this path
  C.hscal = hscal;   // pageable host mirror: fetch() copies and synchronises
  // scratch layout: [basis + work + small arrays | reduction partials | device scalars]
  const int64_t vec_part = (int64_t)(kdim + 2) * n + 10 * (int64_t)(kdim + 1);
  C.part = ws + vec_part;
  C.scal = C.part + (int64_t)RED_BLOCKS * (kdim + 1);
  D2_CUDA(cudaMemsetAsync(C.scal, 0, 64 * sizeof(double), C.s));
  D2_TRY(sec_zero_padding(ops, x_inout, C.s));  // restricted layouts: padding rows stay zero
  double energy = 0.0, resid = 0.0;
  int iters = 0;
  int st = lanczos_in_place(C, ws, x_inout, o.max_iter, kdim, o.tol, o.fixed_steps, o.check_every,
                            &energy, &resid, &iters);
  cudaError_t e = cudaStreamSynchronize(C.s);
  if (e != cudaSuccess && st == DMRG2D_OK)
    st = set_error(DMRG2D_ECUDA, "solver: %s", cudaGetErrorString(e));
  local.iters = iters;
  local.resid = resid;
  local.elapsed_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *energy_out = energy;
  if (stats) *stats = local;
  return st;
}

// ---- Davidson with a diagonal (Jacobi) or learned preconditioner ---------------------------
// The paper's exact diagonalisation names no algorithm; Davidson is the standard
// alternative to Lanczos for the lowest eigenpair.  Each step expands an orthonormal
// basis V by the preconditioned residual t = M(theta) r, keeps H V (FP64, or the
// low-precision H~ V followed by the FP64 outer loop when refine is set) and takes the
// Rayleigh-Ritz pair of V^T H V.  Jacobi: t_i = r_i / (theta - D_i).
namespace dmrg2d {
namespace {

__global__ void k_jacobi(double* __restrict__ t, const double* __restrict__ r,
                         const double* __restrict__ D, double theta, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * VT + threadIdx.x; e < n; e += (int64_t)gridDim.x * VT) {
    double den = theta - D[e];
    if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
    t[e] = r[e] / den;
  }
}

}  // namespace

int davidson_solve(Ctx& C, const dmrg2d_davidson_opts* o, double* x, double* energy, double* resid,
                   int* iters) {
  const int64_t n = C.n;
  const int prec = o->precision;
  int smax = o->max_subspace < 4 ? 4 : (o->max_subspace > 48 ? 48 : o->max_subspace);
  DevBuf Vb, Wb, xb, hxb, rb, tb, Db, Gb, cb, scb;
  D2_TRY(dmalloc(Vb, sizeof(double) * (size_t)smax * n));
  D2_TRY(dmalloc(Wb, sizeof(double) * (size_t)smax * n));
  D2_TRY(dmalloc(hxb, sizeof(double) * n));
  D2_TRY(dmalloc(rb, sizeof(double) * n));
  D2_TRY(dmalloc(tb, sizeof(double) * n));
  D2_TRY(dmalloc(Db, sizeof(double) * n));
  D2_TRY(dmalloc(Gb, sizeof(double) * smax * smax));
  D2_TRY(dmalloc(cb, sizeof(double) * smax));
  D2_TRY(dmalloc(scb, sizeof(double) * 2 * smax * smax));
  double *V = (double*)Vb.p, *W = (double*)Wb.p, *hx = (double*)hxb.p, *r = (double*)rb.p;
  double *t = (double*)tb.p, *D = (double*)Db.p, *G = (double*)Gb.p, *cc = (double*)cb.p;
  double* scr = (double*)scb.p;
  double* sc = C.scal;
  D2_TRY(diag_apply(C.ops, D, C.s));
  MlpPrecond mp;
  if (o->precond == DMRG2D_PRECOND_MLP) {
    if (!o->mlp) return set_error(DMRG2D_EINVAL, "MLP preconditioner requested without a network");
    D2_TRY(mlp_precond_setup(o->mlp, C.ops, D, &mp, C.s));
  }
  D2_TRY(C.nrm(x, sc + 3));
  D2_TRY(C.scale_inv(V, x, sc + 3));
  D2_TRY(C.hv(prec, V, W));
  std::vector<double> Gh((size_t)smax * smax, 0.0);
  auto update_G_col = [&](int jcol) -> int {
    D2_TRY(C.multidot(V, n, jcol + 1, W + (int64_t)jcol * n, sc + 8));
    D2_TRY(C.fetch(sc + 8, jcol + 1));
    for (int i = 0; i <= jcol; ++i) Gh[i * smax + jcol] = Gh[jcol * smax + i] = C.hscal[i];
    return DMRG2D_OK;
  };
  D2_TRY(update_G_col(0));
  int s = 1, it = 0, status = DMRG2D_ENOCONV;
  double theta = 0.0, rn = INFINITY;
  for (it = 1; it <= o->max_iter; ++it) {
    D2_CUDA(cudaMemcpyAsync(G, Gh.data(), sizeof(double) * smax * smax, cudaMemcpyHostToDevice, C.s));
    k_small_eigh<<<1, SE_THREADS, 0, C.s>>>(G, s, smax, sc + 5, cc, scr);
    D2_CUDA(cudaGetLastError());
    D2_TRY(C.combo(x, V, n, s, cc, 0));
    D2_TRY(C.combo(hx, W, n, s, cc, 0));
    D2_TRY(C.fetch(sc + 5, 1));
    theta = C.hscal[0];
    D2_CUDA(cudaMemcpyAsync(r, hx, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.s));
    D2_TRY(C.axpby(r, x, -theta, 1.0));
    D2_TRY(C.nrm(r, sc + 6));
    D2_TRY(C.fetch(sc + 6, 1));
    rn = C.hscal[0];
    if (o->log_cap > 0 && it - 1 < o->log_cap) {  // training data for the learned preconditioner
      if (o->log_r)
        D2_CUDA(cudaMemcpyAsync(o->log_r + (int64_t)(it - 1) * n, r, sizeof(double) * n,
                                cudaMemcpyDeviceToDevice, C.s));
      if (o->log_x)
        D2_CUDA(cudaMemcpyAsync(o->log_x + (int64_t)(it - 1) * n, x, sizeof(double) * n,
                                cudaMemcpyDeviceToDevice, C.s));
      if (o->log_theta) o->log_theta[it - 1] = theta;
    }
    if (!std::isfinite(theta) || !std::isfinite(rn)) {
      status = set_error(DMRG2D_ENAN, "NaN/Inf in Davidson");
      break;
    }
    if (rn <= o->tol * fabs(theta)) {
      status = DMRG2D_OK;
      break;
    }
    if (o->precond == DMRG2D_PRECOND_JACOBI) {
      k_jacobi<<<vgrid(n), VT, 0, C.s>>>(t, r, D, theta, n);
      D2_CUDA(cudaGetLastError());
    } else if (o->precond == DMRG2D_PRECOND_MLP) {
      D2_TRY(mlp_precond_apply(o->mlp, &mp, r, D, theta, t, n, C.s));
    } else {
      D2_CUDA(cudaMemcpyAsync(t, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.s));
    }
    if (s == smax) {  // restart from the Ritz pair
      D2_CUDA(cudaMemcpyAsync(V, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.s));
      D2_CUDA(cudaMemcpyAsync(W, hx, sizeof(double) * n, cudaMemcpyDeviceToDevice, C.s));
      s = 1;
      std::fill(Gh.begin(), Gh.end(), 0.0);
      Gh[0] = theta;
    }
    for (int pass = 0; pass < 2; ++pass) {
      D2_TRY(C.multidot(V, n, s, t, sc + 8));
      D2_TRY(C.combo(t, V, n, s, sc + 8, -1));
    }
    D2_TRY(C.nrm(t, sc + 4));
    D2_TRY(C.fetch(sc + 4, 1));
    if (!(C.hscal[0] > 1e-300)) {
      set_error(DMRG2D_ENOCONV, "Davidson: correction vanished, residual %.3e", rn);
      break;
    }
    D2_TRY(C.scale_inv(V + (int64_t)s * n, t, sc + 4));
    D2_TRY(C.hv(prec, V + (int64_t)s * n, W + (int64_t)s * n));
    D2_TRY(update_G_col(s));
    ++s;
  }
  if (it > o->max_iter) {
    it = o->max_iter;
    set_error(DMRG2D_ENOCONV, "Davidson: %d steps, residual %.3e", it, rn);
  }
  mlp_precond_release(&mp);
  *energy = theta;
  *resid = rn;
  *iters = it;
  return status;
}

}  // namespace dmrg2d

extern "C" void dmrg2d_default_davidson_opts(dmrg2d_davidson_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->max_iter = 500;
  o->max_subspace = 24;
  o->tol = 1e-10;
  o->precision = DMRG2D_FP64;
  o->refine = 0;
  o->precond = DMRG2D_PRECOND_JACOBI;
  o->inner_iter = 40;
  o->outer_max = 20;
  o->refine_tol = 1e-10;
}

extern "C" int dmrg2d_davidson_ground(const dmrg2d_ops* ops, const dmrg2d_davidson_opts* opts,
                                      double* x_inout, double* energy_out,
                                      dmrg2d_solver_stats* stats, void* stream) {
  using namespace dmrg2d;
  if (!ops || !x_inout || !energy_out || !opts) return set_error(DMRG2D_EINVAL, "NULL argument");
  clear_error();
  const dmrg2d_davidson_opts& o = *opts;
  if (o.max_iter < 1) return set_error(DMRG2D_EINVAL, "max_iter < 1");
  if (o.precond < DMRG2D_PRECOND_NONE || o.precond > DMRG2D_PRECOND_MLP)
    return set_error(DMRG2D_EINVAL, "unknown preconditioner %d", o.precond);
  if (o.precision != DMRG2D_FP64 && o.precision != DMRG2D_FP32 && o.precision != DMRG2D_TF32 &&
      o.precision != DMRG2D_BF16 && o.precision != DMRG2D_BF16X3)
    return set_error(DMRG2D_EINVAL, "unknown precision %d", o.precision);
  if ((o.precision == DMRG2D_TF32 || o.precision == DMRG2D_BF16 ||
       o.precision == DMRG2D_BF16X3) && !ops->tc_ok)
    return set_error(DMRG2D_EUNSUPPORTED, "tensor-core path unsupported for these shapes");
  const auto t0 = std::chrono::steady_clock::now();
  dmrg2d_solver_stats local{};
  Ctx C;
  C.ops = ops;
  C.s = (cudaStream_t)stream;
  C.n = ops->n_vec;
  C.st = &local;
  DevBuf part, scal, lo, y32;
  D2_TRY(dmalloc(part, sizeof(double) * (size_t)RED_BLOCKS * 520));
  D2_TRY(dmalloc(scal, sizeof(double) * 64));
  C.part = (double*)part.p;
  C.scal = (double*)scal.p;
  D2_CUDA(cudaMallocHost(&C.hscal, sizeof(double) * 64));
  struct PinnedFree {
    double* p;
    ~PinnedFree() { cudaFreeHost(p); }
  } pf{C.hscal};
  if (o.precision != DMRG2D_FP64) {
    D2_TRY(dmalloc(lo, (o.precision == DMRG2D_BF16 ? 2 : 4) * (size_t)C.n));
    D2_TRY(dmalloc(y32, sizeof(float) * (size_t)C.n));
    C.lo = lo.p;
    C.y32 = (float*)y32.p;
  }
  D2_TRY(sec_zero_padding(ops, x_inout, C.s));
  double energy = 0.0, resid = 0.0;
  int iters = 0;
  int st = davidson_solve(C, &o, x_inout, &energy, &resid, &iters);
  local.iters = iters;
  local.resid = resid;
  if ((st == DMRG2D_OK || st == DMRG2D_ENOCONV) && o.refine && o.precision != DMRG2D_FP64) {
    // FP64 outer loop from the Davidson vector (same loop as the mixed Lanczos solver)
    dmrg2d_solver_opts so;
    dmrg2d_default_solver_opts(&so);
    so.precision = o.precision;
    so.refine = 1;
    so.tol = o.refine_tol;
    so.inner_iter = o.inner_iter;
    so.outer_max = o.outer_max;
    st = mixed_outer(C, &so, x_inout, &energy);
    local.resid = C.st->resid;
  }
  cudaError_t e = cudaStreamSynchronize(C.s);
  if (e != cudaSuccess && st == DMRG2D_OK)
    st = set_error(DMRG2D_ECUDA, "solver: %s", cudaGetErrorString(e));
  int derr = 0;
  if (tc_read_error(ops, &derr) == DMRG2D_OK && derr && st == DMRG2D_OK)
    st = set_error(DMRG2D_ETIMEOUT, "tensor-core kernel gave up waiting (site %d)", derr);
  local.hv_ms = C.hv_ms();
  local.elapsed_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *energy_out = energy;
  if (stats) *stats = local;
  return st;
}
