// Learned preconditioner for the Davidson correction: a small MLP, trained and evaluated by
// the kernels in this file (FP32 on CUDA cores).
//
// The network g maps four features of one vector component to a factor that replaces
// the Jacobi factor 1/(theta - D_i):   t_i = (r_i / s_D) * g(x_i).
//   d_i  = (D_i - theta) / s_D,  s_D = RMS over the vector of (D - theta)
//   x0 = clamp(d_i, -8, 8)
//   x1 = clamp(1/d_i, -16, 16) / 16
//   x2 = clamp((mean of D over the component's sector - theta) / s_D, -8, 8)
//   x3 = log(number of components in the sector) / 16
// (Jacobi itself is g = -1/d.)  Architecture: 4 -> H (tanh) -> H (tanh) -> 1.
// Inference: g depends on i only through d_i and its sector, so each Davidson step
// evaluates the network exactly on a grid of G values of d per sector and interpolates
// linearly per component.  Training: weighted least squares on logged Davidson steps,
//   L = 1/(2B) sum_b (w_b g(x_b) - T_b)^2,  w_b = r_i/(s_D s_t),  T_b = alpha delta_i / s_t,
// delta = x_final - (x_k . x_final) x_k, alpha = (delta . t_J)/(delta . delta) (t_J the Jacobi
// correction), s_t = RMS(t_J): the network learns the direction of the ideal correction.
#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "common.h"

struct dmrg2d_mlp {
  int H = 0;
  int np = 0;
  float* p = nullptr;   // parameters: W1[H][4], b1[H], W2[H][H], b2[H], w3[H], b3
  float* g = nullptr;   // gradient
  float* m1 = nullptr;  // Adam moments
  float* m2 = nullptr;
  int step = 0;
  int bcap = 0;         // batch scratch capacity
  float *z1 = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr;
  float *dz2 = nullptr, *dz1 = nullptr;
  float* one = nullptr;  // a single 1.0f (stride-0 operand for column sums)
  double* part = nullptr;
};

namespace dmrg2d {

namespace {

constexpr int MF = 4;       // inputs
constexpr int GRID = 1024;  // table points per sector

inline int off_b1(int H) { return H * MF; }
inline int off_W2(int H) { return H * MF + H; }
inline int off_b2(int H) { return H * MF + H + H * H; }
inline int off_w3(int H) { return H * MF + H + H * H + H; }
inline int off_b3(int H) { return H * MF + H + H * H + 2 * H; }

// C[M x N] (row-major, ldc) = act(sum_k A(i,k) B(k,j) + bias[j]) (+ C if accumulate)
// A(i,k) = A[i*sa0 + k*sa1], B(k,j) = B[k*sb0 + j*sb1]; act: 0 none, 1 tanh
__global__ void __launch_bounds__(256)
k_gemm(const float* __restrict__ A, long long sa0, long long sa1, const float* __restrict__ B,
       long long sb0, long long sb1, float* __restrict__ C, int ldc, int M, int N, int K,
       const float* __restrict__ bias, int act, float* __restrict__ zout) {
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int q = threadIdx.x; q < 16 * 64; q += 256) {
      const int kk = q / 64, ii = q % 64;
      const int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < M && gk < K) ? A[(long long)gi * sa0 + (long long)gk * sa1] : 0.f;
      const int gj = j0 + ii;
      Bs[kk][ii] = (gj < N && gk < K) ? B[(long long)gk * sb0 + (long long)gj * sb1] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = Bs[kk][tx + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      if (i < M && j < N) {
        float z = acc[u][v] + (bias ? bias[j] : 0.f);
        if (zout) zout[(long long)i * ldc + j] = z;
        C[(long long)i * ldc + j] = act ? tanhf(z) : z;
      }
    }
}

int gemm(const float* A, long long sa0, long long sa1, const float* B, long long sb0, long long sb1,
         float* C, int ldc, int M, int N, int K, const float* bias, int act, float* zout,
         cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_gemm<<<grid, 256, 0, s>>>(A, sa0, sa1, B, sb0, sb1, C, ldc, M, N, K, bias, act, zout);
  D2_CUDA(cudaGetLastError());
  return DMRG2D_OK;
}

// dy = (w y - T) w / B ; per-block partial sums of (w y - T)^2
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ w,
                       const float* __restrict__ T, float* __restrict__ dy, int B,
                       double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int b = blockIdx.x * 256 + threadIdx.x; b < B; b += gridDim.x * 256) {
    const float e = w[b] * y[b] - T[b];
    dy[b] = e * w[b] / (float)B;
    s += (double)e * e;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// dz = (g * w3[col]?) (1 - h^2): mode 0: dz[b][o] = dy[b] w3[o] (1 - h2^2)
//                                mode 1: dz[b][i] = dh[b][i] (1 - h1^2)   (in place)
__global__ void k_tanh_back(float* __restrict__ dz, const float* __restrict__ dy,
                            const float* __restrict__ w3, const float* __restrict__ h, int B, int H,
                            int mode) {
  const long long n = (long long)B * H;
  for (long long q = (long long)blockIdx.x * 256 + threadIdx.x; q < n;
       q += (long long)gridDim.x * 256) {
    const int b = (int)(q / H), o = (int)(q % H);
    const float hv = h[q];
    const float up = mode == 0 ? dy[b] * w3[o] : dz[q];
    dz[q] = up * (1.f - hv * hv);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float c1, float c2) {
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
    const float gi = g[i];
    m1[i] = 0.9f * m1[i] + 0.1f * gi;
    m2[i] = 0.999f * m2[i] + 0.001f * gi * gi;
    p[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + 1e-8f);
  }
}

__device__ __forceinline__ void features(double Di, double theta, double sD, float x2, float x3,
                                         float* x) {
  const double d = (Di - theta) / sD;
  x[0] = (float)fmin(fmax(d, -8.0), 8.0);
  double inv = d != 0.0 ? 1.0 / d : 16.0;
  inv = fmin(fmax(inv, -16.0), 16.0);
  x[1] = (float)(inv / 16.0);
  x[2] = x2;
  x[3] = x3;
}

// grid inputs: for sector q, point k: d = dlo_q + k (dhi_q - dlo_q)/(G-1)
__global__ void k_grid_inputs(float* __restrict__ X, const double* __restrict__ qp, int nq,
                              double theta, double sD) {
  const int q = blockIdx.x;
  const double dlo = qp[4 * q], dhi = qp[4 * q + 1];
  const float x2 = (float)qp[4 * q + 2], x3 = (float)qp[4 * q + 3];
  for (int k = threadIdx.x; k < GRID; k += blockDim.x) {
    const double d = dlo + (dhi - dlo) * k / (GRID - 1);
    features(theta + d * sD, theta, sD, x2, x3, X + ((size_t)q * GRID + k) * MF);
  }
}

__device__ __forceinline__ int sector_of(const long long* __restrict__ qstart, int nq, long long i) {
  int lo = 0, hi = nq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (qstart[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The Jacobi factor in units of s_D: t_i = r_i / (theta - D_i) = (r_i / s_D) j(d_i),
// j(d) = -1/d, clamped like the network's input |1/d| <= 16.
__device__ __forceinline__ double jacobi_factor(double d) {
  const double inv = d != 0.0 ? 1.0 / d : 16.0;
  return -fmin(fmax(inv, -16.0), 16.0);
}

// t_i = (r_i / s_D) j(d_i) (1 + y(d_i)), y interpolated from the sector's table
__global__ void k_apply_table(double* __restrict__ t, const double* __restrict__ r,
                              const double* __restrict__ D, const float* __restrict__ table,
                              const double* __restrict__ qp, const long long* __restrict__ qstart,
                              int nq, double theta, double sD, long long n) {
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n;
       i += (long long)gridDim.x * 256) {
    const int q = sector_of(qstart, nq, i);
    const double dlo = qp[4 * q], dhi = qp[4 * q + 1];
    const double d = (D[i] - theta) / sD;
    double u = dhi > dlo ? (d - dlo) / (dhi - dlo) * (GRID - 1) : 0.0;
    u = fmin(fmax(u, 0.0), (double)(GRID - 1));
    const int k = min((int)u, GRID - 2);
    const double f = u - k;
    const float* tq = table + (size_t)q * GRID;
    const double y = (1.0 - f) * tq[k] + f * tq[k + 1];
    t[i] = r[i] / sD * jacobi_factor(d) * (1.0 + y);
  }
}

// training samples: X (features), w = r/(s_D s_t), T = alpha delta / s_t at positions idx
__global__ void k_make_batch(const double* __restrict__ xk, const double* __restrict__ rk,
                             const double* __restrict__ xf, const double* __restrict__ D,
                             const long long* __restrict__ idx, int B, double theta, double sD,
                             double proj, double alpha, double st, const double* __restrict__ qp,
                             const long long* __restrict__ qstart, int nq, float* __restrict__ X,
                             float* __restrict__ w, float* __restrict__ T) {
  for (int b = blockIdx.x * 256 + threadIdx.x; b < B; b += gridDim.x * 256) {
    const long long i = idx[b];
    const int q = sector_of(qstart, nq, i);
    features(D[i], theta, sD, (float)qp[4 * q + 2], (float)qp[4 * q + 3], X + (size_t)b * MF);
    // the preconditioner is (r/s_D) j (1 + y): w y - T with w = (r/s_D) j / s_t and
    // T = (target - (r/s_D) j) / s_t fits the correction y to plain Jacobi
    const double wj = rk[i] / sD * jacobi_factor((D[i] - theta) / sD) / st;
    w[b] = (float)wj;
    T[b] = (float)(alpha * (xf[i] - proj * xk[i]) / st - wj);
  }
}

// per-range partial statistics of D: sum, sum of squares, min, max
__global__ void k_dstats(const double* __restrict__ D, long long n, double* __restrict__ out) {
  __shared__ double s1[256], s2[256], mn[256], mx[256];
  double a = 0, b = 0, lo = 1e300, hi = -1e300;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n;
       i += (long long)gridDim.x * 256) {
    const double v = D[i];
    a += v;
    b += v * v;
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  mn[threadIdx.x] = lo;
  mx[threadIdx.x] = hi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
      mn[threadIdx.x] = fmin(mn[threadIdx.x], mn[threadIdx.x + o]);
      mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[4 * blockIdx.x] = s1[0];
    out[4 * blockIdx.x + 1] = s2[0];
    out[4 * blockIdx.x + 2] = mn[0];
    out[4 * blockIdx.x + 3] = mx[0];
  }
}

// out = [x_k . x_f, delta . t_J, delta . delta, t_J . t_J], delta = x_f - (x_k . x_f) x_k,
// t_J = r / (theta - D): two passes with per-block partials summed on the host
__global__ void k_dot2(const double* __restrict__ a, const double* __restrict__ b, long long n,
                       double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
    s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_delta3(const double* __restrict__ xk, const double* __restrict__ rk,
                         const double* __restrict__ xf, const double* __restrict__ D, double theta,
                         double proj, long long n, double* __restrict__ part) {
  __shared__ double r1[256], r2[256], r3[256];
  double a = 0, b = 0, c = 0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    double den = theta - D[i];
    if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
    const double tj = rk[i] / den;
    const double dl = xf[i] - proj * xk[i];
    a += dl * tj;
    b += dl * dl;
    c += tj * tj;
  }
  r1[threadIdx.x] = a;
  r2[threadIdx.x] = b;
  r3[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
      r3[threadIdx.x] += r3[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = r1[0];
    part[3 * blockIdx.x + 1] = r2[0];
    part[3 * blockIdx.x + 2] = r3[0];
  }
}

int vec_delta_stats(const double* xk, const double* rk, const double* xf, const double* D,
                    double theta, int64_t n, double* out, cudaStream_t s) {
  double* part = nullptr;
  if (cudaMalloc((void**)&part, 3 * 256 * 8) != cudaSuccess)
    return set_error(DMRG2D_ENOMEM, "delta stats");
  std::vector<double> hp(3 * 256, 0.0);
  k_dot2<<<256, 256, 0, s>>>(xk, xf, n, part);
  cudaMemcpyAsync(hp.data(), part, 256 * 8, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  double proj = 0.0;
  for (int i = 0; i < 256; ++i) proj += hp[i];
  k_delta3<<<256, 256, 0, s>>>(xk, rk, xf, D, theta, proj, n, part);
  cudaMemcpyAsync(hp.data(), part, 3 * 256 * 8, cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) return set_error(DMRG2D_ECUDA, "delta stats: %s", cudaGetErrorString(e));
  out[0] = proj;
  out[1] = out[2] = out[3] = 0.0;
  for (int i = 0; i < 256; ++i) {
    out[1] += hp[3 * i];
    out[2] += hp[3 * i + 1];
    out[3] += hp[3 * i + 2];
  }
  return DMRG2D_OK;
}

int grow(dmrg2d_mlp* M, int B) {
  if (B <= M->bcap) return DMRG2D_OK;
  float** bufs[] = {&M->z1, &M->h1, &M->h2, &M->dz2, &M->dz1};
  for (float** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  if (M->y) cudaFree(M->y);
  if (M->dy) cudaFree(M->dy);
  M->y = M->dy = nullptr;
  const size_t big = (size_t)B * M->H * sizeof(float);
  for (float** b : bufs)
    if (cudaMalloc((void**)b, big) != cudaSuccess) return set_error(DMRG2D_ENOMEM, "MLP scratch");
  if (cudaMalloc((void**)&M->y, (size_t)B * 4) != cudaSuccess ||
      cudaMalloc((void**)&M->dy, (size_t)B * 4) != cudaSuccess)
    return set_error(DMRG2D_ENOMEM, "MLP scratch");
  M->bcap = B;
  return DMRG2D_OK;
}

int forward(dmrg2d_mlp* M, const float* X, int B, cudaStream_t s) {
  const int H = M->H;
  const float* p = M->p;
  D2_TRY(gemm(X, MF, 1, p, 1, MF, M->h1, H, B, H, MF, p + off_b1(H), 1, M->z1, s));
  D2_TRY(gemm(M->h1, H, 1, p + off_W2(H), 1, H, M->h2, H, B, H, H, p + off_b2(H), 1, nullptr, s));
  D2_TRY(gemm(M->h2, H, 1, p + off_w3(H), 1, 0, M->y, 1, B, 1, H, p + off_b3(H), 0, nullptr, s));
  return DMRG2D_OK;
}

// gradient of L into M->g; loss (host) optional
int backward(dmrg2d_mlp* M, const float* X, const float* w, const float* T, int B, float* loss,
             cudaStream_t s) {
  const int H = M->H;
  const float* p = M->p;
  float* g = M->g;
  const int nb = 64;
  k_loss<<<nb, 256, 0, s>>>(M->y, w, T, M->dy, B, M->part);
  D2_CUDA(cudaGetLastError());
  // output layer
  D2_TRY(gemm(M->dy, 0, 1, M->h2, H, 1, g + off_w3(H), H, 1, H, B, nullptr, 0, nullptr, s));
  D2_TRY(gemm(M->one, 0, 0, M->dy, 1, 0, g + off_b3(H), 1, 1, 1, B, nullptr, 0, nullptr, s));
  // second hidden layer
  const int eg = (int)std::min<long long>(((long long)B * H + 255) / 256, 4096);
  k_tanh_back<<<eg, 256, 0, s>>>(M->dz2, M->dy, p + off_w3(H), M->h2, B, H, 0);
  D2_TRY(gemm(M->dz2, 1, H, M->h1, H, 1, g + off_W2(H), H, H, H, B, nullptr, 0, nullptr, s));
  D2_TRY(gemm(M->one, 0, 0, M->dz2, H, 1, g + off_b2(H), H, 1, H, B, nullptr, 0, nullptr, s));
  // first hidden layer: dh1 = dz2 W2, then dz1 = dh1 (1 - h1^2)
  D2_TRY(gemm(M->dz2, H, 1, p + off_W2(H), H, 1, M->dz1, H, B, H, H, nullptr, 0, nullptr, s));
  k_tanh_back<<<eg, 256, 0, s>>>(M->dz1, nullptr, nullptr, M->h1, B, H, 1);
  D2_TRY(gemm(M->dz1, 1, H, X, MF, 1, g, MF, H, MF, B, nullptr, 0, nullptr, s));
  D2_TRY(gemm(M->one, 0, 0, M->dz1, H, 1, g + off_b1(H), H, 1, H, B, nullptr, 0, nullptr, s));
  D2_CUDA(cudaGetLastError());
  if (loss) {
    double hp[64];
    D2_CUDA(cudaMemcpyAsync(hp, M->part, sizeof(hp), cudaMemcpyDeviceToHost, s));
    D2_CUDA(cudaStreamSynchronize(s));
    double tot = 0;
    for (int i = 0; i < nb; ++i) tot += hp[i];
    *loss = (float)(tot / (2.0 * B));
  }
  return DMRG2D_OK;
}

// contiguous vector ranges of the sectors (dense: one range)
void ranges(const dmrg2d_ops* ops, std::vector<long long>& start, std::vector<long long>& len) {
  if (ops->sec) {
    std::vector<long long> qb;
    std::vector<int> qld, qc;
    std::vector<double> rd, cd;
    std::vector<int> ri, ci;
    sec_diag_tables(ops, qb, qld, qc, rd, ri, cd, ci);
    for (size_t q = 0; q < qb.size(); ++q) {
      start.push_back(qb[q]);
      len.push_back((long long)qld[q] * qc[q]);
    }
  } else {
    start.push_back(0);
    len.push_back(ops->n_vec);
  }
}

}  // namespace

int mlp_precond_setup(const dmrg2d_mlp* M, const dmrg2d_ops* ops, const double* D, MlpPrecond* P,
                      cudaStream_t s) {
  (void)M;
  std::vector<long long> start, len;
  ranges(ops, start, len);
  P->nq = (int)start.size();
  P->mean.assign(P->nq, 0.0);
  P->dmin.assign(P->nq, 0.0);
  P->dmax.assign(P->nq, 0.0);
  P->count.assign(P->nq, 0.0);
  double* part = nullptr;
  if (cudaMalloc((void**)&part, 4 * 128 * sizeof(double)) != cudaSuccess)
    return set_error(DMRG2D_ENOMEM, "MLP setup");
  double s1 = 0, s2 = 0, n = 0;
  std::vector<double> hp(4 * 128);
  for (int q = 0; q < P->nq; ++q) {
    k_dstats<<<128, 256, 0, s>>>(D + start[q], len[q], part);
    cudaMemcpyAsync(hp.data(), part, hp.size() * 8, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    double a = 0, b = 0, lo = 1e300, hi = -1e300;
    for (int k = 0; k < 128; ++k) {
      a += hp[4 * k];
      b += hp[4 * k + 1];
      lo = std::min(lo, hp[4 * k + 2]);
      hi = std::max(hi, hp[4 * k + 3]);
    }
    P->mean[q] = a / std::max<long long>(len[q], 1);
    P->dmin[q] = lo;
    P->dmax[q] = hi;
    P->count[q] = (double)len[q];
    s1 += a;
    s2 += b;
    n += (double)len[q];
  }
  cudaFree(part);
  P->meanD = s1 / n;
  P->meanD2 = s2 / n;
  std::vector<long long> qs(start);
  qs.push_back(ops->n_vec);
  auto al = [&](void** p, size_t b) -> int {
    if (cudaMalloc(p, b) != cudaSuccess) return set_error(DMRG2D_ENOMEM, "MLP setup");
    return DMRG2D_OK;
  };
  D2_TRY(al((void**)&P->qstart, qs.size() * 8));
  D2_CUDA(cudaMemcpyAsync(P->qstart, qs.data(), qs.size() * 8, cudaMemcpyHostToDevice, s));
  D2_TRY(al((void**)&P->qp, (size_t)P->nq * 4 * 8));
  D2_TRY(al((void**)&P->Xg, (size_t)P->nq * GRID * MF * 4));
  D2_TRY(al((void**)&P->table, (size_t)P->nq * GRID * 4));
  P->hqp.resize((size_t)P->nq * 4);
  D2_CUDA(cudaStreamSynchronize(s));
  return DMRG2D_OK;
}

static int precond_params(MlpPrecond* P, double theta, double* sD, cudaStream_t s) {
  const double var = P->meanD2 - 2.0 * theta * P->meanD + theta * theta;
  *sD = std::sqrt(std::max(var, 1e-300));
  for (int q = 0; q < P->nq; ++q) {
    P->hqp[4 * q] = (P->dmin[q] - theta) / *sD;
    P->hqp[4 * q + 1] = (P->dmax[q] - theta) / *sD;
    P->hqp[4 * q + 2] = std::min(std::max((P->mean[q] - theta) / *sD, -8.0), 8.0);
    P->hqp[4 * q + 3] = std::log(std::max(P->count[q], 1.0)) / 16.0;
  }
  D2_CUDA(cudaMemcpyAsync(P->qp, P->hqp.data(), P->hqp.size() * 8, cudaMemcpyHostToDevice, s));
  return DMRG2D_OK;
}

int mlp_precond_apply(const dmrg2d_mlp* Mc, MlpPrecond* P, const double* r, const double* D,
                      double theta, double* t, int64_t n, cudaStream_t s) {
  dmrg2d_mlp* M = const_cast<dmrg2d_mlp*>(Mc);
  double sD = 1.0;
  D2_TRY(precond_params(P, theta, &sD, s));
  k_grid_inputs<<<P->nq, 256, 0, s>>>(P->Xg, P->qp, P->nq, theta, sD);
  D2_CUDA(cudaGetLastError());
  D2_TRY(grow(M, P->nq * GRID));
  D2_TRY(forward(M, P->Xg, P->nq * GRID, s));
  D2_CUDA(cudaMemcpyAsync(P->table, M->y, (size_t)P->nq * GRID * 4, cudaMemcpyDeviceToDevice, s));
  const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
  k_apply_table<<<grid, 256, 0, s>>>(t, r, D, P->table, P->qp, P->qstart, P->nq, theta, sD, n);
  D2_CUDA(cudaGetLastError());
  return DMRG2D_OK;
}

void mlp_precond_release(MlpPrecond* P) {
  for (void* p : {(void*)P->qstart, (void*)P->qp, (void*)P->Xg, (void*)P->table})
    if (p) cudaFree(p);
  P->qstart = nullptr;
  P->qp = nullptr;
  P->Xg = nullptr;
  P->table = nullptr;
}

}  // namespace dmrg2d

using namespace dmrg2d;

extern "C" int dmrg2d_mlp_create(int hidden, uint64_t seed, dmrg2d_mlp** out) {
  if (!out || hidden < 1 || hidden > 4096) return set_error(DMRG2D_EINVAL, "mlp_create: bad argument");
  *out = nullptr;
  dmrg2d_mlp* M = new dmrg2d_mlp();
  M->H = hidden;
  M->np = off_b3(hidden) + 1;
  std::vector<float> h(M->np, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  const int H = hidden;
  for (int i = 0; i < H * MF; ++i) h[i] = nd(rng) / std::sqrt((float)MF);
  for (int i = 0; i < H * H; ++i) h[off_W2(H) + i] = nd(rng) / std::sqrt((float)H);
  // output layer starts at zero: y = 0 is plain Jacobi (the factor is j(d) (1 + y))
  for (int i = 0; i < H; ++i) h[off_w3(H) + i] = 0.f;
  int st = DMRG2D_OK;
  for (float** b : {&M->p, &M->g, &M->m1, &M->m2})
    if (st == DMRG2D_OK && cudaMalloc((void**)b, (size_t)M->np * 4) != cudaSuccess)
      st = set_error(DMRG2D_ENOMEM, "mlp_create");
  if (st == DMRG2D_OK && (cudaMalloc((void**)&M->one, 4) != cudaSuccess ||
                          cudaMalloc((void**)&M->part, 64 * 8) != cudaSuccess))
    st = set_error(DMRG2D_ENOMEM, "mlp_create");
  if (st == DMRG2D_OK) {
    const float one = 1.f;
    cudaMemcpy(M->p, h.data(), (size_t)M->np * 4, cudaMemcpyHostToDevice);
    cudaMemset(M->m1, 0, (size_t)M->np * 4);
    cudaMemset(M->m2, 0, (size_t)M->np * 4);
    cudaMemcpy(M->one, &one, 4, cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess) st = set_error(DMRG2D_ECUDA, "mlp_create");
  }
  if (st != DMRG2D_OK) {
    dmrg2d_mlp_free(M);
    return st;
  }
  *out = M;
  return DMRG2D_OK;
}

extern "C" void dmrg2d_mlp_free(dmrg2d_mlp* M) {
  if (!M) return;
  for (void* p : {(void*)M->p, (void*)M->g, (void*)M->m1, (void*)M->m2, (void*)M->z1, (void*)M->h1,
                  (void*)M->h2, (void*)M->y, (void*)M->dy, (void*)M->dz2, (void*)M->dz1,
                  (void*)M->one, (void*)M->part})
    if (p) cudaFree(p);
  delete M;
}

extern "C" int dmrg2d_mlp_num_params(const dmrg2d_mlp* M) { return M ? M->np : 0; }

extern "C" int dmrg2d_mlp_get_params(const dmrg2d_mlp* M, float* host) {
  if (!M || !host) return set_error(DMRG2D_EINVAL, "NULL argument");
  D2_CUDA(cudaMemcpy(host, M->p, (size_t)M->np * 4, cudaMemcpyDeviceToHost));
  return DMRG2D_OK;
}

extern "C" int dmrg2d_mlp_set_params(dmrg2d_mlp* M, const float* host) {
  if (!M || !host) return set_error(DMRG2D_EINVAL, "NULL argument");
  D2_CUDA(cudaMemcpy(M->p, host, (size_t)M->np * 4, cudaMemcpyHostToDevice));
  M->step = 0;
  D2_CUDA(cudaMemset(M->m1, 0, (size_t)M->np * 4));
  D2_CUDA(cudaMemset(M->m2, 0, (size_t)M->np * 4));
  return DMRG2D_OK;
}

extern "C" int dmrg2d_mlp_forward(dmrg2d_mlp* M, const float* X, float* Y, int B, void* stream) {
  if (!M || !X || !Y || B < 1) return set_error(DMRG2D_EINVAL, "mlp_forward: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  D2_TRY(grow(M, B));
  D2_TRY(forward(M, X, B, s));
  D2_CUDA(cudaMemcpyAsync(Y, M->y, (size_t)B * 4, cudaMemcpyDeviceToDevice, s));
  return DMRG2D_OK;
}

extern "C" int dmrg2d_mlp_loss_grad(dmrg2d_mlp* M, const float* X, const float* w, const float* T,
                                    int B, float* grad, float* loss, void* stream) {
  if (!M || !X || !w || !T || B < 1) return set_error(DMRG2D_EINVAL, "mlp_loss_grad: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  D2_TRY(grow(M, B));
  D2_TRY(forward(M, X, B, s));
  D2_TRY(backward(M, X, w, T, B, loss, s));
  if (grad) D2_CUDA(cudaMemcpyAsync(grad, M->g, (size_t)M->np * 4, cudaMemcpyDeviceToDevice, s));
  return DMRG2D_OK;
}

extern "C" int dmrg2d_mlp_train_step(dmrg2d_mlp* M, const float* X, const float* w, const float* T,
                                     int B, float lr, float* loss, void* stream) {
  if (!M || !X || !w || !T || B < 1) return set_error(DMRG2D_EINVAL, "mlp_train_step: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  D2_TRY(grow(M, B));
  D2_TRY(forward(M, X, B, s));
  D2_TRY(backward(M, X, w, T, B, loss, s));
  ++M->step;
  const float c1 = 1.f - std::pow(0.9f, (float)M->step), c2 = 1.f - std::pow(0.999f, (float)M->step);
  k_adam<<<(M->np + 255) / 256, 256, 0, s>>>(M->p, M->g, M->m1, M->m2, M->np, lr, c1, c2);
  D2_CUDA(cudaGetLastError());
  return DMRG2D_OK;
}

extern "C" int dmrg2d_mlp_make_batch(const dmrg2d_ops* ops, const double* x_k, const double* r_k,
                                     double theta, const double* x_final, const double* D,
                                     const int64_t* idx, int B, float* X, float* w, float* T,
                                     void* stream) {
  if (!ops || !x_k || !r_k || !x_final || !D || !idx || !X || !w || !T || B < 1)
    return set_error(DMRG2D_EINVAL, "mlp_make_batch: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  MlpPrecond P;
  D2_TRY(mlp_precond_setup(nullptr, ops, D, &P, s));
  double sD = 1.0;
  int st = precond_params(&P, theta, &sD, s);
  // global scalars: proj = x_k . x_f ; delta = x_f - proj x_k ; t_J = r/(theta - D)
  double sc[4] = {0, 0, 0, 0};
  if (st == DMRG2D_OK) st = vec_delta_stats(x_k, r_k, x_final, D, theta, ops->n_vec, sc, s);
  const double proj = sc[0];
  const double alpha = sc[2] > 0 ? sc[1] / sc[2] : 0.0;          // (delta.tJ)/(delta.delta)
  const double stj = std::sqrt(std::max(sc[3] / (double)ops->n_vec, 1e-300));  // RMS(t_J)
  if (st == DMRG2D_OK) {
    k_make_batch<<<(B + 255) / 256, 256, 0, s>>>(x_k, r_k, x_final, D, (const long long*)idx, B,
                                                 theta, sD, proj, alpha, stj, P.qp, P.qstart, P.nq,
                                                 X, w, T);
    if (cudaGetLastError() != cudaSuccess) st = set_error(DMRG2D_ECUDA, "make_batch launch");
  }
  if (st == DMRG2D_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = set_error(DMRG2D_ECUDA, "make_batch");
  mlp_precond_release(&P);
  return st;
}
