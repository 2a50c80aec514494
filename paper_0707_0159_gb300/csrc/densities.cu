// Site densities of the two central columns from a superblock vector: the observables
// of the paper's Hubbard study (hole density h(x,y) = 1 - <n_up + n_dn>, its Eq. (hole);
// staggered spin density s(x,y) = <n_up - n_dn>, zero on every site of the finite
// ladder's ground state by the Lieb-Mattis theorem; S(x) = max_y |s(x,y)|).
//
// The occupation numbers are diagonal in the column basis, so one pass over the vector
// bins |x|^2 by the column-2 state i2 of its row and the column-3 state i3 of its column
// (w2, w3: the diagonals of the two columns' reduced density matrices, unnormalised),
// and a small kernel contracts the weights with the occupation numbers.
#include "common.h"

namespace dmrg2d {

namespace {

constexpr int DT = 256;           // threads per block of the binning pass
constexpr int DW = DT / 32;       // warps per block: one (block q, column) per warp
constexpr int DGRID = 8 * 152;    // persistent grid (8 blocks per SM)

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// The vector as sector blocks q (one block for a dense superblock): element (r, c) of
// block q at base[q] + r + ld[q] c.  Packed column g is column colc[g] of block colq[g],
// with column-3 state colI3[g]; row r of block q has column-2 state rowI2[roff[q] + r]
// (-1: a padding row, zero in every vector).  Rows of one i2 are contiguous, so the 32
// rows a warp reads mostly share i2 and are added to its bin once.
__global__ void __launch_bounds__(DT)
k_column_weights(const double* __restrict__ x, const long long* __restrict__ base,
                 const int* __restrict__ ld, const int* __restrict__ colq,
                 const int* __restrict__ colc, const int* __restrict__ colI3, int ncols,
                 const int* __restrict__ roff, const int* __restrict__ rowI2, int d,
                 double* __restrict__ w2, double* __restrict__ w3) {
  extern __shared__ double bins[];  // d column-2 bins of this block
  for (int i = threadIdx.x; i < d; i += DT) bins[i] = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g = blockIdx.x * DW + warp; g < ncols; g += gridDim.x * DW) {
    const int q = colq[g];
    const int nr = ld[q];
    const double* col = x + base[q] + (long long)ld[q] * colc[g];
    const int* ri2 = rowI2 + roff[q];
    double colsum = 0.0;
    for (int r0 = 0; r0 < nr; r0 += 32) {
      const int r = r0 + lane;
      const double v = r < nr ? col[r] : 0.0;
      const int i2 = r < nr ? ri2[r] : -1;
      const double sq = i2 >= 0 ? v * v : 0.0;
      colsum += sq;
      const int i2_0 = __shfl_sync(0xffffffffu, i2, 0);
      if (__all_sync(0xffffffffu, i2 == i2_0)) {
        const double s = warp_sum_d(sq);
        if (lane == 0 && i2_0 >= 0) atomicAdd(&bins[i2_0], s);
      } else if (i2 >= 0) {
        atomicAdd(&bins[i2], sq);
      }
    }
    colsum = warp_sum_d(colsum);
    if (lane == 0) atomicAdd(&w3[colI3[g]], colsum);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += DT)
    if (bins[i] != 0.0) atomicAdd(&w2[i], bins[i]);
}

// out[(c n_legs + y) 4 + k], c = 0 (column 2) / 1 (column 3), k = n_up, n_dn, h, s;
// out[8 n_legs + c] = S(c).  Occupations of column state i: Hubbard mode 2y + s is bit
// 2y + s of i; a spin column's leg y is up when bit y of i is set (n_up + n_dn = 1).
__global__ void k_site_densities(const double* __restrict__ w2, const double* __restrict__ w3,
                                 int d, int n_legs, int hubbard, double* __restrict__ out) {
  __shared__ double red[DT];
  double t = 0.0;
  for (int i = threadIdx.x; i < d; i += DT) t += w2[i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int s = DT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double tot = red[0];
  const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
  for (int k = threadIdx.x; k < 2 * n_legs; k += DT) {
    const int c = k / n_legs, y = k % n_legs;
    const double* w = c == 0 ? w2 : w3;
    double nu = 0.0, nd = 0.0;
    for (int i = 0; i < d; ++i) {
      if (hubbard) {
        nu += ((i >> (2 * y)) & 1) ? w[i] : 0.0;
        nd += ((i >> (2 * y + 1)) & 1) ? w[i] : 0.0;
      } else {
        if ((i >> y) & 1) nu += w[i];
        else nd += w[i];
      }
    }
    nu *= inv;
    nd *= inv;
    double* o = out + 4 * (c * n_legs + y);
    o[0] = nu;
    o[1] = nd;
    o[2] = 1.0 - nu - nd;
    o[3] = nu - nd;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int c = threadIdx.x;
    double m = 0.0;
    for (int y = 0; y < n_legs; ++y) m = fmax(m, fabs(out[4 * (c * n_legs + y) + 3]));
    out[8 * n_legs + c] = m;
  }
}

struct DevArr {
  void* p = nullptr;
  ~DevArr() {
    if (p) cudaFree(p);
  }
  template <typename T>
  int upload(const std::vector<T>& h, cudaStream_t s) {
    if (cudaMalloc(&p, sizeof(T) * std::max<size_t>(h.size(), 1)) != cudaSuccess) {
      p = nullptr;
      return set_error(DMRG2D_ENOMEM, "site_densities: cudaMalloc failed");
    }
    if (!h.empty() &&
        cudaMemcpyAsync(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return set_error(DMRG2D_ECUDA, "site_densities: upload failed");
    return DMRG2D_OK;
  }
};

}  // namespace

}  // namespace dmrg2d

using namespace dmrg2d;

extern "C" int dmrg2d_site_densities(const dmrg2d_ops* ops, const double* x, double* out,
                                     void* stream) {
  if (!ops || !x || !out) return set_error(DMRG2D_EINVAL, "NULL argument");
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  const int d = ops->d, m1 = ops->m1, m4 = ops->m4;
  // layout tables: sector blocks of a restricted superblock, else one dense block
  std::vector<long long> qbase;
  std::vector<int> qld, qcols, rowI2, colI3;
  if (ops->sec) {
    std::vector<double> rowD, colD;
    D2_TRY(sec_diag_tables(ops, qbase, qld, qcols, rowD, rowI2, colD, colI3));
  } else {
    qbase = {0};
    qld = {(int)ops->ld};
    qcols = {d * m4};
    rowI2.resize((size_t)ops->ld);
    for (int64_t r = 0; r < ops->ld; ++r) rowI2[(size_t)r] = (int)(r / m1);
    colI3.resize((size_t)d * m4);
    for (int c = 0; c < d * m4; ++c) colI3[(size_t)c] = c / m4;
  }
  const int nq = (int)qbase.size();
  std::vector<int> roff(nq, 0), colq, colc;
  for (int q = 0; q < nq; ++q) {
    if (q + 1 < nq) roff[q + 1] = roff[q] + qld[q];
    for (int c = 0; c < qcols[q]; ++c) {
      colq.push_back(q);
      colc.push_back(c);
    }
  }
  const int ncols = (int)colq.size();
  if ((size_t)ncols != colI3.size())
    return set_error(DMRG2D_EINVAL, "site_densities: inconsistent sector layout");
  DevArr dbase, dld, dcolq, dcolc, dcolI3, droff, drowI2, dw;
  D2_TRY(dbase.upload(qbase, s));
  D2_TRY(dld.upload(qld, s));
  D2_TRY(dcolq.upload(colq, s));
  D2_TRY(dcolc.upload(colc, s));
  D2_TRY(dcolI3.upload(colI3, s));
  D2_TRY(droff.upload(roff, s));
  D2_TRY(drowI2.upload(rowI2, s));
  D2_TRY(dw.upload(std::vector<double>((size_t)2 * d, 0.0), s));
  double* w2 = (double*)dw.p;
  double* w3 = w2 + d;
  const int grid = std::max(1, std::min(DGRID, (ncols + DW - 1) / DW));
  k_column_weights<<<grid, DT, sizeof(double) * d, s>>>(
      x, (const long long*)dbase.p, (const int*)dld.p, (const int*)dcolq.p,
      (const int*)dcolc.p, (const int*)dcolI3.p, ncols, (const int*)droff.p,
      (const int*)drowI2.p, d, w2, w3);
  D2_CUDA(cudaGetLastError());
  k_site_densities<<<1, DT, 0, s>>>(w2, w3, d, ops->n_legs, ops->kind == DMRG2D_HUBBARD ? 1 : 0,
                                    out);
  D2_CUDA(cudaGetLastError());
  // the scratch above is freed on return: wait for the kernels that read it
  D2_CUDA(cudaStreamSynchronize(s));
  return DMRG2D_OK;
}
