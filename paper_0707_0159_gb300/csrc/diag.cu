// Diagonal of the superblock Hamiltonian in the vector layout (dense or sector-packed).
//
// From Eq. (dec): H(i1 i2 i3 i4; i1 i2 i3 i4) = H_l(i1 i2; i1 i2) + H_r(i3 i4; i3 i4)
// + H_c(i2 i3; i2 i3).  The first two are the diagonals of the diagonal blocks of H_l
// and H_r; the third is the sum of the scalar tile moves whose source tile is their
// destination.  For every matrix V_q the kernel adds a row term, a column term and
// the (i2, i3) term; padding rows of a packed layout get 0.
#include <algorithm>

#include "common.h"

namespace dmrg2d {

namespace {

__global__ void k_diag(double* __restrict__ out, const double* __restrict__ rowD,
                       const int* __restrict__ rowI2, const double* __restrict__ colD,
                       const int* __restrict__ colI3, const double* __restrict__ dC, int d,
                       long long ld, long long ncols) {
  const long long n = ld * ncols;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const long long r = p % ld, c = p / ld;
    const int i2 = rowI2[r];
    out[p] = i2 < 0 ? 0.0 : rowD[r] + colD[c] + dC[i2 + d * colI3[c]];
  }
}

}  // namespace

// Record the diagonal pieces on the host (called by build_ops with the dense blocks).
void diag_pieces(dmrg2d_ops* ops, const std::vector<double>& HL, const std::vector<double>& HR) {
  const int d = ops->d, m1 = ops->m1, m4 = ops->m4;
  ops->hdL.assign((size_t)m1 * d, 0.0);
  ops->hdR.assign((size_t)m4 * d, 0.0);
  ops->hdC.assign((size_t)d * d, 0.0);
  for (int i2 = 0; i2 < d; ++i2)
    for (int e = ops->hLptr[i2]; e < ops->hLptr[i2 + 1]; ++e)
      if (ops->hLcol[e] == i2)
        for (int i = 0; i < m1; ++i)
          ops->hdL[(size_t)i + (size_t)m1 * i2] = HL[(size_t)e * m1 * m1 + (size_t)i * m1 + i];
  for (int i3 = 0; i3 < d; ++i3)
    for (int e = ops->hRptr[i3]; e < ops->hRptr[i3 + 1]; ++e)
      if (ops->hRcol[e] == i3)
        for (int i = 0; i < m4; ++i)
          ops->hdR[(size_t)i + (size_t)m4 * i3] = HR[(size_t)e * m4 * m4 + (size_t)i * m4 + i];
  for (int t = 0; t < d * d; ++t)
    for (int e = ops->hCptr[t]; e < ops->hCptr[t + 1]; ++e)
      if (ops->hCsrc[e] == t) ops->hdC[t] += ops->hCval[e];
}

// Per-matrix row/column tables: dense superblocks are one matrix with row r = i1 + m1 i2
// and column c = i4 + m4 i3.  Sector layouts fill the tables through sec_diag_tables.
int diag_apply(const dmrg2d_ops* ops, double* out, cudaStream_t s) {
  std::vector<long long> qbase;
  std::vector<int> qld, qcols;
  std::vector<double> rowD, colD;
  std::vector<int> rowI2, colI3;
  if (ops->sec) {
    D2_TRY(sec_diag_tables(ops, qbase, qld, qcols, rowD, rowI2, colD, colI3));
  } else {
    const int d = ops->d, m1 = ops->m1, m4 = ops->m4;
    qbase = {0};
    qld = {(int)ops->ld};
    qcols = {d * m4};
    rowD = ops->hdL;
    colD = ops->hdR;
    rowI2.resize((size_t)m1 * d);
    colI3.resize((size_t)m4 * d);
    for (int r = 0; r < m1 * d; ++r) rowI2[r] = r / m1;
    for (int c = 0; c < m4 * d; ++c) colI3[c] = c / m4;
  }
  double *dRow = nullptr, *dCol = nullptr, *dC = nullptr;
  int *dRi = nullptr, *dCi = nullptr;
  auto up = [&](const void* h, size_t bytes, void** dptr) -> int {
    if (cudaMalloc(dptr, bytes) != cudaSuccess)
      return set_error(DMRG2D_ENOMEM, "diagonal: cudaMalloc(%zu)", bytes);
    D2_CUDA(cudaMemcpyAsync(*dptr, h, bytes, cudaMemcpyHostToDevice, s));
    return DMRG2D_OK;
  };
  int st = up(rowD.data(), rowD.size() * 8, (void**)&dRow);
  if (st == DMRG2D_OK) st = up(rowI2.data(), rowI2.size() * 4, (void**)&dRi);
  if (st == DMRG2D_OK) st = up(colD.data(), colD.size() * 8, (void**)&dCol);
  if (st == DMRG2D_OK) st = up(colI3.data(), colI3.size() * 4, (void**)&dCi);
  if (st == DMRG2D_OK) st = up(ops->hdC.data(), ops->hdC.size() * 8, (void**)&dC);
  long long roff = 0, coff = 0;
  for (size_t q = 0; q < qbase.size() && st == DMRG2D_OK; ++q) {
    const long long n = (long long)qld[q] * qcols[q];
    const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
    if (n > 0)
      k_diag<<<grid, 256, 0, s>>>(out + qbase[q], dRow + roff, dRi + roff, dCol + coff,
                                  dCi + coff, dC, ops->d, qld[q], qcols[q]);
    roff += qld[q];
    coff += qcols[q];
  }
  if (st == DMRG2D_OK) {
    cudaError_t e = cudaStreamSynchronize(s);  // the tables are freed below
    if (e != cudaSuccess) st = set_error(DMRG2D_ECUDA, "diagonal: %s", cudaGetErrorString(e));
  }
  for (void* p : {(void*)dRow, (void*)dRi, (void*)dCol, (void*)dCi, (void*)dC})
    if (p) cudaFree(p);
  return st;
}

}  // namespace dmrg2d

using namespace dmrg2d;

extern "C" int dmrg2d_diagonal(const dmrg2d_ops* ops, double* out, void* stream) {
  if (!ops || !out) return set_error(DMRG2D_EINVAL, "NULL argument");
  return diag_apply(ops, out, (cudaStream_t)stream);
}
