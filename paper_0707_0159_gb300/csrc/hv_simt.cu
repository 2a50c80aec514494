// Superblock H·v on CUDA cores (FP64 DFMA or FP32 FMA), and the apply_H entry point.
//
// One CTA computes a BM x BN piece of one output tile (i2, i3) of
//     Y = H_l V + V H_r^T + sum_k A_k V B_k^T        (paper, text after Eq. (dec))
// in three phases that share one register accumulator:
//   1. H_l V:    for every block (i2, i2') of H_l:  acc += HL[i2,i2'] * V_tile(i2', i3)
//   2. V H_r^T:  for every block (i3, i3') of H_r:  acc += V_tile(i2, i3') * HR[i3,i3']^T
//   3. scalar moves (H_c and off-diagonal column terms): acc += c * V_tile(i2', i3')
// and writes Y once.  V is column-major with leading dimension m1*d.
#include "common.h"
#include "ff.cuh"

namespace dmrg2d {

namespace {

struct SimtParams {
  int m1, m4, d;
  int64_t ld;
  const int* Lptr;
  const int* Lcol;
  const int* Rptr;
  const int* Rcol;
  const int* Cptr;
  const int* Csrc;
};

constexpr int BM = 64, BN = 64, BK = 16, TX = 16, TY = 16;  // 256 threads, 4x4 outputs each

// BMt x BNt piece per CTA (64 x 64: 4 x 4 outputs per thread; smaller pieces for small
// superblocks, whose 64 x 64 grid would leave most SMs idle at GB300's FP64 rate)
template <typename T, int BMt, int BNt>
__global__ void __launch_bounds__(TX * TY)
hv_simt_kernel(const T* __restrict__ v, T* __restrict__ y, const T* __restrict__ HL,
               const T* __restrict__ HR, const T* __restrict__ Cval, SimtParams p) {
  constexpr int RA = BMt / TX, RB = BNt / TY;  // outputs per thread along rows / columns
  constexpr int NT = TX * TY;
  __shared__ T As[BK][BMt];
  __shared__ T Bs[BK][BNt];
  const int nbm = (p.m1 + BMt - 1) / BMt;
  const int nbn = (p.m4 + BNt - 1) / BNt;
  const int bm = blockIdx.x % nbm, i2 = blockIdx.x / nbm;
  const int bn = blockIdx.y % nbn, i3 = blockIdx.y / nbn;
  const int i0 = bm * BMt, j0 = bn * BNt;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m1 = p.m1, m4 = p.m4;
  const int64_t ld = p.ld;

  T acc[RA][RB];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[a][b] = T(0);

  auto mma_tile = [&]() {
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T av[RA], bv[RB];
#pragma unroll
      for (int a = 0; a < RA; ++a) av[a] = As[k][tx + TX * a];
#pragma unroll
      for (int b = 0; b < RB; ++b) bv[b] = Bs[k][ty + TY * b];
#pragma unroll
      for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[a][b] += av[a] * bv[b];
    }
  };

  // ---- phase 1: H_l V ----
  for (int e = p.Lptr[i2]; e < p.Lptr[i2 + 1]; ++e) {
    const T* A = HL + (size_t)e * m1 * m1;                    // A[i][k] = A[i*m1 + k]
    const T* B = v + (int64_t)p.Lcol[e] * m1 + ld * ((int64_t)i3 * m4);  // B[k][j] = B[k + ld*j]
    for (int k0 = 0; k0 < m1; k0 += BK) {
      if constexpr (BMt == 64 && BNt == 64) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int k = tid % BK, i = tid / BK + 16 * r;
          const int gi = i0 + i, gk = k0 + k;
          As[k][i] = (gi < m1 && gk < m1) ? A[(size_t)gi * m1 + gk] : T(0);
          const int gj = j0 + i;  // the same (k, row) mapping for B's 64 columns
          Bs[k][i] = (gk < m1 && gj < m4) ? B[gk + ld * gj] : T(0);
        }
      } else {
        for (int idx = tid; idx < BK * BMt; idx += NT) {
          const int k = idx % BK, i = idx / BK;
          const int gi = i0 + i, gk = k0 + k;
          As[k][i] = (gi < m1 && gk < m1) ? A[(size_t)gi * m1 + gk] : T(0);
        }
        for (int idx = tid; idx < BK * BNt; idx += NT) {
          const int k = idx % BK, j = idx / BK;
          const int gj = j0 + j, gk = k0 + k;
          Bs[k][j] = (gk < m1 && gj < m4) ? B[gk + ld * gj] : T(0);
        }
      }
      __syncthreads();
      mma_tile();
      __syncthreads();
    }
  }
  // ---- phase 2: V H_r^T ----
  for (int e = p.Rptr[i3]; e < p.Rptr[i3 + 1]; ++e) {
    const T* A = v + (int64_t)i2 * m1 + ld * ((int64_t)p.Rcol[e] * m4);  // A[i][k] = A[i + ld*k]
    const T* B = HR + (size_t)e * m4 * m4;                    // B[k][j] = B[j*m4 + k]
    for (int k0 = 0; k0 < m4; k0 += BK) {
      if constexpr (BMt == 64 && BNt == 64) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = tid % BM, k = tid / BM + 4 * r;
          const int gi = i0 + i, gk = k0 + k;
          As[k][i] = (gi < m1 && gk < m4) ? A[gi + ld * gk] : T(0);
          const int kb = tid % BK, j = tid / BK + 16 * r;
          const int gj = j0 + j, gkb = k0 + kb;
          Bs[kb][j] = (gj < m4 && gkb < m4) ? B[(size_t)gj * m4 + gkb] : T(0);
        }
      } else {
        for (int idx = tid; idx < BK * BMt; idx += NT) {
          const int i = idx % BMt, k = idx / BMt;
          const int gi = i0 + i, gk = k0 + k;
          As[k][i] = (gi < m1 && gk < m4) ? A[gi + ld * gk] : T(0);
        }
        for (int idx = tid; idx < BK * BNt; idx += NT) {
          const int kb = idx % BK, j = idx / BK;
          const int gj = j0 + j, gkb = k0 + kb;
          Bs[kb][j] = (gj < m4 && gkb < m4) ? B[(size_t)gj * m4 + gkb] : T(0);
        }
      }
      __syncthreads();
      mma_tile();
      __syncthreads();
    }
  }
  // ---- phase 3: scalar tile moves, then the single store of Y ----
  const int t = i2 + p.d * i3;
  for (int e = p.Cptr[t]; e < p.Cptr[t + 1]; ++e) {
    const int src = p.Csrc[e];
    const int s2 = src % p.d, s3 = src / p.d;
    const T c = Cval[e];
    const T* S = v + (int64_t)s2 * m1 + ld * ((int64_t)s3 * m4);
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const int gi = i0 + tx + TX * a, gj = j0 + ty + TY * b;
        if (gi < m1 && gj < m4) acc[a][b] += c * S[gi + ld * gj];
      }
  }
  T* Yt = y + (int64_t)i2 * m1 + ld * ((int64_t)i3 * m4);
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const int gi = i0 + tx + TX * a, gj = j0 + ty + TY * b;
      if (gi < m1 && gj < m4) Yt[gi + ld * gj] = acc[a][b];
    }
}

// ---- FP64 emulated with float pairs (FP64X, ff.cuh) ------------------------------------
// Same tiling as hv_simt_kernel; float-pair arithmetic runs on the FP32 pipes (64x the
// FP64 rate on this part).
__global__ void __launch_bounds__(TX * TY)
hv_simt_ff_kernel(const double* __restrict__ v, double* __restrict__ y,
                  const double* __restrict__ HL, const double* __restrict__ HR,
                  const double* __restrict__ Cval, SimtParams p) {
  __shared__ ff As[BK][BM];
  __shared__ ff Bs[BK][BN];
  const int nbm = (p.m1 + BM - 1) / BM;
  const int nbn = (p.m4 + BN - 1) / BN;
  const int bm = blockIdx.x % nbm, i2 = blockIdx.x / nbm;
  const int bn = blockIdx.y % nbn, i3 = blockIdx.y / nbn;
  const int i0 = bm * BM, j0 = bn * BN;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m1 = p.m1, m4 = p.m4;
  const int64_t ld = p.ld;
  const ff zero = {0.f, 0.f};

  ff acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = zero;

  auto mma_tile = [&]() {
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      ff av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][tx + TX * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][ty + TY * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ff_fma(acc[a][b], av[a], bv[b]);
    }
  };

  // ---- phase 1: H_l V ----
  for (int e = p.Lptr[i2]; e < p.Lptr[i2 + 1]; ++e) {
    const double* A = HL + (size_t)e * m1 * m1;
    const double* B = v + (int64_t)p.Lcol[e] * m1 + ld * ((int64_t)i3 * m4);
    for (int k0 = 0; k0 < m1; k0 += BK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k = tid % BK, i = tid / BK + 16 * r;
        const int gi = i0 + i, gk = k0 + k;
        As[k][i] = (gi < m1 && gk < m1) ? ff_of(A[(size_t)gi * m1 + gk]) : zero;
        const int gj = j0 + i;
        Bs[k][i] = (gk < m1 && gj < m4) ? ff_of(B[gk + ld * gj]) : zero;
      }
      __syncthreads();
      mma_tile();
      __syncthreads();
    }
  }
  // ---- phase 2: V H_r^T ----
  for (int e = p.Rptr[i3]; e < p.Rptr[i3 + 1]; ++e) {
    const double* A = v + (int64_t)i2 * m1 + ld * ((int64_t)p.Rcol[e] * m4);
    const double* B = HR + (size_t)e * m4 * m4;
    for (int k0 = 0; k0 < m4; k0 += BK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = tid % BM, k = tid / BM + 4 * r;
        const int gi = i0 + i, gk = k0 + k;
        As[k][i] = (gi < m1 && gk < m4) ? ff_of(A[gi + ld * gk]) : zero;
        const int kb = tid % BK, j = tid / BK + 16 * r;
        const int gj = j0 + j, gkb = k0 + kb;
        Bs[kb][j] = (gj < m4 && gkb < m4) ? ff_of(B[(size_t)gj * m4 + gkb]) : zero;
      }
      __syncthreads();
      mma_tile();
      __syncthreads();
    }
  }
  // ---- phase 3: scalar tile moves, then the single store of Y ----
  const int t = i2 + p.d * i3;
  for (int e = p.Cptr[t]; e < p.Cptr[t + 1]; ++e) {
    const int src = p.Csrc[e];
    const int s2 = src % p.d, s3 = src / p.d;
    const ff c = ff_of(Cval[e]);
    const double* S = v + (int64_t)s2 * m1 + ld * ((int64_t)s3 * m4);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int gi = i0 + tx + TX * a, gj = j0 + ty + TY * b;
        if (gi < m1 && gj < m4) ff_fma(acc[a][b], c, ff_of(S[gi + ld * gj]));
      }
  }
  double* Yt = y + (int64_t)i2 * m1 + ld * ((int64_t)i3 * m4);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gi = i0 + tx + TX * a, gj = j0 + ty + TY * b;
      if (gi < m1 && gj < m4) Yt[gi + ld * gj] = ff_to_double(acc[a][b]);
    }
}

SimtParams simt_params(const dmrg2d_ops* ops) {
  SimtParams p;
  p.m1 = ops->m1;
  p.m4 = ops->m4;
  p.d = ops->d;
  p.ld = ops->ld;
  p.Lptr = ops->dev.Lptr;
  p.Lcol = ops->dev.Lcol;
  p.Rptr = ops->dev.Rptr;
  p.Rcol = ops->dev.Rcol;
  p.Cptr = ops->dev.Cptr;
  p.Csrc = ops->dev.Csrc;
  return p;
}

template <typename T>
int launch(const dmrg2d_ops* ops, const T* v, T* y, const T* HL, const T* HR, const T* C,
           cudaStream_t s) {
  SimtParams p;
  p.m1 = ops->m1;
  p.m4 = ops->m4;
  p.d = ops->d;
  p.ld = ops->ld;
  p.Lptr = ops->dev.Lptr;
  p.Lcol = ops->dev.Lcol;
  p.Rptr = ops->dev.Rptr;
  p.Rcol = ops->dev.Rcol;
  p.Cptr = ops->dev.Cptr;
  p.Csrc = ops->dev.Csrc;
  // the largest piece (64, 32 or 16 square) whose grid still gives every SM a CTA
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
  }
  auto ctas = [&](int b) {
    return ((int64_t)(ops->m1 + b - 1) / b) * ops->d * ((int64_t)(ops->m4 + b - 1) / b) * ops->d;
  };
  const int tb = ctas(64) >= sms ? 64 : (ctas(32) >= sms ? 32 : 16);
  const int64_t gx = (int64_t)((ops->m1 + tb - 1) / tb) * ops->d;
  const int64_t gy = (int64_t)((ops->m4 + tb - 1) / tb) * ops->d;
  if (gx > 0x7fffffff || gy > 65535)
    return set_error(DMRG2D_EUNSUPPORTED, "SIMT grid %lld x %lld too large", (long long)gx,
                     (long long)gy);
  dim3 grid((unsigned)gx, (unsigned)gy);
  auto ev = prof_slot(ops);
  if (ev.first) D2_CUDA(cudaEventRecord(ev.first, s));
  if (tb == 64)
    hv_simt_kernel<T, 64, 64><<<grid, TX * TY, 0, s>>>(v, y, HL, HR, C, p);
  else if (tb == 32)
    hv_simt_kernel<T, 32, 32><<<grid, TX * TY, 0, s>>>(v, y, HL, HR, C, p);
  else
    hv_simt_kernel<T, 16, 16><<<grid, TX * TY, 0, s>>>(v, y, HL, HR, C, p);
  D2_CUDA(cudaGetLastError());
  if (ev.second) D2_CUDA(cudaEventRecord(ev.second, s));
  return DMRG2D_OK;
}

int launch_ff(const dmrg2d_ops* ops, const double* v, double* y, cudaStream_t s) {
  const SimtParams p = simt_params(ops);
  const int64_t gx = (int64_t)((ops->m1 + BM - 1) / BM) * ops->d;
  const int64_t gy = (int64_t)((ops->m4 + BN - 1) / BN) * ops->d;
  if (gx > 0x7fffffff || gy > 65535)
    return set_error(DMRG2D_EUNSUPPORTED, "SIMT grid %lld x %lld too large", (long long)gx,
                     (long long)gy);
  auto ev = prof_slot(ops);
  if (ev.first) D2_CUDA(cudaEventRecord(ev.first, s));
  hv_simt_ff_kernel<<<dim3((unsigned)gx, (unsigned)gy), TX * TY, 0, s>>>(
      v, y, ops->dev.HL64, ops->dev.HR64, ops->dev.Cval64, p);
  D2_CUDA(cudaGetLastError());
  if (ev.second) D2_CUDA(cudaEventRecord(ev.second, s));
  return DMRG2D_OK;
}

}  // namespace

int launch_hv_simt_ff64(const dmrg2d_ops* ops, const double* v, double* y, cudaStream_t s) {
  if (ops->sec) return sec_apply(ops, v, y, DMRG2D_FP64X, s);
  return launch_ff(ops, v, y, s);
}

int launch_hv_simt_f64(const dmrg2d_ops* ops, const double* v, double* y, cudaStream_t s) {
  if (ops->sec) return sec_apply(ops, v, y, DMRG2D_FP64, s);
  return launch<double>(ops, v, y, ops->dev.HL64, ops->dev.HR64, ops->dev.Cval64, s);
}

int launch_hv_simt_f32(const dmrg2d_ops* ops, const float* v, float* y, cudaStream_t s) {
  if (ops->sec) return sec_apply(ops, v, y, DMRG2D_FP32, s);
  return launch<float>(ops, v, y, ops->dev.HL32, ops->dev.HR32, ops->dev.Cval32, s);
}

}  // namespace dmrg2d

using namespace dmrg2d;

extern "C" int dmrg2d_apply_H(const dmrg2d_ops* ops, const void* v, void* y, int precision,
                              void* stream) {
  if (!ops || !v || !y) return set_error(DMRG2D_EINVAL, "NULL argument to apply_H");
  cudaStream_t s = (cudaStream_t)stream;
  switch (precision) {
    case DMRG2D_FP64:
      return launch_hv_simt_f64(ops, (const double*)v, (double*)y, s);
    case DMRG2D_FP32:
      return launch_hv_simt_f32(ops, (const float*)v, (float*)y, s);
    case DMRG2D_FP64X:
      return launch_hv_simt_ff64(ops, (const double*)v, (double*)y, s);
    case DMRG2D_TF32:
    case DMRG2D_BF16:
    case DMRG2D_BF16X3:
      if (!ops->tc_ok)
        return set_error(DMRG2D_EUNSUPPORTED, "tensor-core path does not support m1=%d m4=%d",
                         ops->m1, ops->m4);
      return launch_hv_tc(ops, v, (float*)y, precision, s);
    default:
      return set_error(DMRG2D_EINVAL, "unknown precision %d", precision);
  }
}
