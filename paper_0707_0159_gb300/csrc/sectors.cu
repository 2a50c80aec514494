// Sector-restricted superblock H·v: quantum-number blocks of uneven size as one grouped
// launch (the paper's blocks carry conserved quantum numbers, but it does not describe
// their use in H·v).
//
// Packed vector layout (also in include/dmrg2d.h): for every combined left label qL
// (block-1 label + column-2 label), in increasing lexicographic order, one column-major
// matrix V_qL:
//   rows    = for i2 = 0..d-1, the block-1 sector a with label qL - q(i2) (if present),
//             its states i1 in increasing order, each segment padded to a multiple of 8
//             rows (padding is zero on input and written as zero on output);
//   columns = for i3 = 0..d-1, the block-4 sector b with label Q - qL - q(i3) (if present),
//             its states i4 in increasing order;
//   ld      = padded row count; matrices are stored one after another.
// Within each V_qL the order is the paper's (i2 slow, i1 fast) x (i3 slow, i4 fast).
//
// H_l restricted to qL couples row segment (i2, a) to (i2', a') with a' fixed by charge
// conservation; the operator sub-block is the (a, a') part of the dense block
// HL[i2, i2'].  Same for H_r on column segments.  Scalar tile moves keep a and b and may
// change qL (H_c moves charge between the columns).
#include <algorithm>
#include <array>
#include <cmath>
#include <map>

#include "common.h"
#include "ff.cuh"
#include "grouped.h"

namespace dmrg2d {

namespace {

using Lab = std::array<int, 2>;
Lab add(Lab a, Lab b) { return {a[0] + b[0], a[1] + b[1]}; }
Lab sub(Lab a, Lab b) { return {a[0] - b[0], a[1] - b[1]}; }

constexpr int SBM = 64, SBN = 64, SBK = 16;  // CUDA-core tile

struct RowSegD {  // device row segment
  int q, off, dim, dim_pad, k1b, k1e;
};
struct ColSegD {
  int q, off, dim, k2b, k2e;
};
struct K1D {  // phase 1: A = L sub-block, B = rows of V_q
  long long a_off;  // compact FP64/FP32 offset of the sub-block (row-major dim(a) x kdim)
  int a_pool;       // first row of the sub-block in the tensor-core pool
  int b_row;        // first row of segment (i2', a') in V_q
  int kdim;
};
struct K2D {  // phase 2: A = columns of V_q, B = R sub-block
  long long b_off;  // compact offset (row-major dim(b) x kdim)
  int b_pool;
  int a_col;        // first column of segment (i3', b') in V_q
  int kdim;
};
struct TileD {
  int rs, cs;       // row / column segment
  int r_in, c_in;   // first row / column inside the segments
};
struct MoveDst {
  int rs, cs, mb, me;
};
struct MoveSrc {
  int rs, cs;
  double c64;
  float c32;
};
struct MoveItem {
  int dst, c_in;    // destination sub-block, first column of an 8-column chunk
};

struct SecParams {
  const long long* qbase;
  const int* qld;
  const RowSegD* rseg;
  const ColSegD* cseg;
  const K1D* k1;
  const K2D* k2;
  const TileD* tiles;
  const MoveDst* mdst;
  const MoveSrc* msrc;
  const MoveItem* mitems;
};

struct SecState {
  int nQ = 0;
  std::vector<long long> qbase;
  std::vector<int> qld, qcols;
  std::vector<RowSegD> rseg;
  std::vector<ColSegD> cseg;
  std::vector<K1D> k1;
  std::vector<K2D> k2;
  std::vector<TileD> tiles;
  std::vector<MoveDst> mdst;
  std::vector<MoveSrc> msrc;
  std::vector<MoveItem> mitems;
  std::vector<int> rs_i2, rs_a, cs_i3, cs_b;  // host: segment identities
  std::vector<int> a_first, b_first;          // first state of each block sector
  // device copies
  long long* d_qbase = nullptr;
  int* d_qld = nullptr;
  RowSegD* d_rseg = nullptr;
  ColSegD* d_cseg = nullptr;
  K1D* d_k1 = nullptr;
  K2D* d_k2 = nullptr;
  TileD* d_tiles = nullptr;
  MoveDst* d_mdst = nullptr;
  MoveSrc* d_msrc = nullptr;
  MoveItem* d_mitems = nullptr;
  double* d_L64 = nullptr;
  float* d_L32 = nullptr;
  double* d_R64 = nullptr;
  float* d_R32 = nullptr;
  // padding rows (zeroed in solver start vectors): (offset, count) pairs
  std::vector<long long> pad_off;
  std::vector<int> pad_cnt;
  long long* d_pad_off = nullptr;
  int* d_pad_cnt = nullptr;
  std::vector<void*> allocs;
  GroupPlan plan;  // tensor-core form of the same work (pools deduplicated up to sign)
  bool gp_ok = false;

  SecParams params() const {
    return {d_qbase, d_qld, d_rseg, d_cseg, d_k1, d_k2, d_tiles, d_mdst, d_msrc, d_mitems};
  }
};

// ---- kernels ------------------------------------------------------------------------------
// T: storage type of v, y and the operators; Tc: compute type (T, or float pairs ff for
// FP64X with double storage)
template <typename T, typename Tc>
__global__ void __launch_bounds__(256)
hv_simt_sec_kernel(const T* __restrict__ v, T* __restrict__ y, const T* __restrict__ Lsub,
                   const T* __restrict__ Rsub, SecParams p) {
  __shared__ Tc As[SBK][SBM];
  __shared__ Tc Bs[SBK][SBN];
  const TileD t = p.tiles[blockIdx.x];
  const RowSegD rs = p.rseg[t.rs];
  const ColSegD cs = p.cseg[t.cs];
  const long long base = p.qbase[rs.q];
  const long long ld = p.qld[rs.q];
  const int rows = min(SBM, rs.dim - t.r_in), cols = min(SBN, cs.dim - t.c_in);
  const int r0 = rs.off + t.r_in, c0 = cs.off + t.c_in;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const Tc zero = c_zero<Tc>();
  Tc acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = zero;
  auto mma = [&]() {
#pragma unroll
    for (int k = 0; k < SBK; ++k) {
      Tc av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) c_mac(acc[a][b], av[a], bv[b]);
    }
  };
  // phase 1: H_l restricted
  for (int e = rs.k1b; e < rs.k1e; ++e) {
    const K1D k = p.k1[e];
    const T* A = Lsub + k.a_off + (long long)t.r_in * k.kdim;  // A[i][kk] = A[i*kdim + kk]
    const T* B = v + base + k.b_row + ld * c0;                  // B[kk][j] = B[kk + ld*j]
    for (int k0 = 0; k0 < k.kdim; k0 += SBK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int kk = tid % SBK, i = tid / SBK + 16 * r;
        const int gk = k0 + kk;
        As[kk][i] = (i < rows && gk < k.kdim) ? c_in<Tc>(A[(long long)i * k.kdim + gk]) : zero;
        Bs[kk][i] = (i < cols && gk < k.kdim) ? c_in<Tc>(B[gk + ld * i]) : zero;
      }
      __syncthreads();
      mma();
      __syncthreads();
    }
  }
  // phase 2: H_r restricted
  for (int e = cs.k2b; e < cs.k2e; ++e) {
    const K2D k = p.k2[e];
    const T* A = v + base + r0 + ld * k.a_col;                  // A[i][kk] = A[i + ld*kk]
    const T* B = Rsub + k.b_off + (long long)t.c_in * k.kdim;   // B[kk][j] = B[j*kdim + kk]
    for (int k0 = 0; k0 < k.kdim; k0 += SBK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = tid % SBM, kk = tid / SBM + 4 * r;
        const int gk = k0 + kk;
        As[kk][i] = (i < rows && gk < k.kdim) ? c_in<Tc>(A[i + ld * gk]) : zero;
        const int kb = tid % SBK, j = tid / SBK + 16 * r;
        const int gkb = k0 + kb;
        Bs[kb][j] = (j < cols && gkb < k.kdim) ? c_in<Tc>(B[(long long)j * k.kdim + gkb]) : zero;
      }
      __syncthreads();
      mma();
      __syncthreads();
    }
  }
  T* Y = y + base + r0 + ld * c0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = tx + 16 * a, j = ty + 16 * b;
      if (i < rows && j < cols) Y[i + ld * j] = c_out(acc[a][b]);
    }
  // zero padding rows of the segment (last row tile of the segment only)
  if (t.r_in + SBM >= rs.dim) {
    const int npad = rs.dim_pad - rs.dim;
    for (int q = tid; q < npad * SBN; q += 256) {
      const int i = q % npad, j = q / npad;
      if (j < cols) y[base + rs.off + rs.dim + i + ld * (c0 + j)] = T(0);
    }
  }
}

// Y(sub-block) += sum_moves c * V(source sub-block); one block per (sub-block, 8 columns)
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256)
k_sec_moves(const Tin* __restrict__ v, Tout* __restrict__ y, SecParams p, int use64) {
  const MoveItem it = p.mitems[blockIdx.x];
  const MoveDst dst = p.mdst[it.dst];
  const RowSegD rs = p.rseg[dst.rs];
  const ColSegD cs = p.cseg[dst.cs];
  const long long dbase = p.qbase[rs.q] + rs.off;
  const long long dld = p.qld[rs.q];
  const int ncol = min(8, cs.dim - it.c_in);
  for (int i = threadIdx.x; i < rs.dim; i += 256) {
    Tout acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = Tout(0);
    for (int e = dst.mb; e < dst.me; ++e) {
      const MoveSrc ms = p.msrc[e];
      const RowSegD sr = p.rseg[ms.rs];
      const ColSegD sc = p.cseg[ms.cs];
      const long long sld = p.qld[sr.q];
      const Tin* S = v + p.qbase[sr.q] + sr.off + i + sld * (sc.off + it.c_in);
      const Tout c = use64 ? (Tout)ms.c64 : (Tout)ms.c32;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j < ncol) acc[j] += c * (Tout)S[sld * j];
    }
    Tout* Y = y + dbase + i + dld * (cs.off + it.c_in);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j < ncol) Y[dld * j] += acc[j];
  }
}

__global__ void k_zero_pad(double* __restrict__ x, const long long* __restrict__ off,
                           const int* __restrict__ cnt, int n) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  for (int i = 0; i < cnt[w]; ++i) x[off[w] + i] = 0.0;
}

template <typename T>
int up(SecState* S, const std::vector<T>& h, T** d, int64_t* bytes, cudaStream_t s) {
  *d = nullptr;
  if (h.empty()) return DMRG2D_OK;
  const size_t nb = h.size() * sizeof(T);
  if (cudaMalloc((void**)d, nb) != cudaSuccess) {
    *d = nullptr;
    return set_error(DMRG2D_ENOMEM, "cudaMalloc(%zu) failed (sectors)", nb);
  }
  S->allocs.push_back(*d);
  *bytes += (int64_t)nb;
  D2_CUDA(cudaMemcpyAsync(*d, h.data(), nb, cudaMemcpyHostToDevice, s));
  return DMRG2D_OK;
}

}  // namespace

int sec_build(dmrg2d_ops* ops, const dmrg2d_block* L, const dmrg2d_block* R, const int32_t* target,
              const std::vector<double>& HL, const std::vector<double>& HR, cudaStream_t s) {
  const int d = ops->d, m1 = ops->m1, m4 = ops->m4;
  const int nq = ops->kind == DMRG2D_HEISENBERG ? 1 : 2;
  if (!L->qn || !R->qn)
    return set_error(DMRG2D_EINVAL, "sector-restricted build needs qn on both blocks");
  auto lab_of = [&](const int32_t* qn, int i) -> Lab {
    return {qn[i * nq], nq == 2 ? qn[i * nq + 1] : 0};
  };
  const Lab Q = {target[0], nq == 2 ? target[1] : 0};
  // ---- block sectors: maximal runs of equal labels ----
  auto runs = [&](const dmrg2d_block* B, std::vector<Lab>& lab, std::vector<int>& off,
                  std::vector<int>& dim, std::map<Lab, int>& idx, const char* name) -> int {
    for (int i = 0; i < B->m;) {
      const Lab l = lab_of(B->qn, i);
      int j = i + 1;
      while (j < B->m && lab_of(B->qn, j) == l) ++j;
      if (idx.count(l))
        return set_error(DMRG2D_EINVAL, "%s block: states with label (%d,%d) are not contiguous",
                         name, l[0], l[1]);
      idx[l] = (int)lab.size();
      lab.push_back(l);
      off.push_back(i);
      dim.push_back(j - i);
      i = j;
    }
    return DMRG2D_OK;
  };
  std::vector<Lab> lab1, lab4;
  std::vector<int> off1, dim1, off4, dim4;
  std::map<Lab, int> idx1, idx4;
  D2_TRY(runs(L, lab1, off1, dim1, idx1, "left"));
  D2_TRY(runs(R, lab4, off4, dim4, idx4, "right"));
  std::vector<Lab> qc(d);
  for (int i = 0; i < d; ++i) qc[i] = {ops->hqc[2 * i], nq == 2 ? ops->hqc[2 * i + 1] : 0};
  auto find = [](const std::map<Lab, int>& m, Lab l) {
    auto it = m.find(l);
    return it == m.end() ? -1 : it->second;
  };
  // ---- combined left labels with a non-empty right partner ----
  std::map<Lab, int> qset;
  for (int i2 = 0; i2 < d; ++i2)
    for (size_t a = 0; a < lab1.size(); ++a) {
      const Lab qL = add(lab1[a], qc[i2]);
      bool ok = false;
      for (int i3 = 0; i3 < d && !ok; ++i3) ok = find(idx4, sub(sub(Q, qL), qc[i3])) >= 0;
      if (ok) qset[qL] = 0;
    }
  if (qset.empty()) return set_error(DMRG2D_ESHAPE, "target sector is empty");
  SecState* S = new SecState();
  ops->sec = S;
  S->a_first = off1;
  S->b_first = off4;
  std::map<std::pair<int, int>, int> rs_of, cs_of;  // (i2,a) -> row seg, (i3,b) -> col seg
  long long base = 0;
  int qi = 0;
  for (auto& kv : qset) {
    kv.second = qi;
    const Lab qL = kv.first;
    int off = 0;
    for (int i2 = 0; i2 < d; ++i2) {
      const int a = find(idx1, sub(qL, qc[i2]));
      if (a < 0) continue;
      const int pad = (dim1[a] + 7) / 8 * 8;
      rs_of[{i2, a}] = (int)S->rseg.size();
      S->rseg.push_back({qi, off, dim1[a], pad, 0, 0});
      S->rs_i2.push_back(i2);
      S->rs_a.push_back(a);
      off += pad;
    }
    const int ld = off;
    int coff = 0;
    for (int i3 = 0; i3 < d; ++i3) {
      const int b = find(idx4, sub(sub(Q, qL), qc[i3]));
      if (b < 0) continue;
      cs_of[{i3, b}] = (int)S->cseg.size();
      S->cseg.push_back({qi, coff, dim4[b], 0, 0});
      S->cs_i3.push_back(i3);
      S->cs_b.push_back(b);
      coff += dim4[b];
    }
    S->qbase.push_back(base);
    S->qld.push_back(ld);
    S->qcols.push_back(coff);
    base += (long long)ld * coff;
    ++qi;
  }
  S->nQ = qi;
  ops->n_vec = base;
  // padding positions: every column of every padded row segment
  for (size_t r = 0; r < S->rseg.size(); ++r) {
    const RowSegD& rs = S->rseg[r];
    if (rs.dim_pad == rs.dim) continue;
    for (int c = 0; c < S->qcols[rs.q]; ++c) {
      S->pad_off.push_back(S->qbase[rs.q] + rs.off + rs.dim + (long long)S->qld[rs.q] * c);
      S->pad_cnt.push_back(rs.dim_pad - rs.dim);
    }
  }
  // ---- operator sub-blocks and K lists ----
  std::vector<double> Lc, Rc;  // compact row-major sub-blocks
  double flops = 0.0;
  int poolL = 0, poolR = 0;
  std::vector<int> qvalid_rows(S->nQ, 0);
  for (const RowSegD& rs : S->rseg) qvalid_rows[rs.q] += rs.dim;
  for (size_t r = 0; r < S->rseg.size(); ++r) {
    RowSegD& rs = S->rseg[r];
    const int i2 = S->rs_i2[r], a = S->rs_a[r];
    rs.k1b = (int)S->k1.size();
    for (int e = ops->hLptr[i2]; e < ops->hLptr[i2 + 1]; ++e) {
      const int i2p = ops->hLcol[e];
      const int ap = find(idx1, sub(add(lab1[a], qc[i2]), qc[i2p]));
      if (ap < 0) continue;
      auto it = rs_of.find({i2p, ap});
      if (it == rs_of.end()) continue;
      const double* blk = HL.data() + (size_t)e * m1 * m1;
      double mx = 0.0;
      for (int i = 0; i < dim1[a]; ++i)
        for (int k = 0; k < dim1[ap]; ++k)
          mx = std::max(mx, std::fabs(blk[(size_t)(off1[a] + i) * m1 + off1[ap] + k]));
      if (mx == 0.0) continue;  // structurally zero sub-block: no work
      {
        const auto pe = S->plan.poolL.add(blk + (size_t)off1[a] * m1 + off1[ap], dim1[a],
                                          dim1[ap], m1);
        S->plan.k1.push_back({pe.first, S->rseg[it->second].off, dim1[ap], pe.second});
      }
      K1D k;
      k.a_off = (long long)Lc.size();
      k.a_pool = poolL;
      k.b_row = S->rseg[it->second].off;
      k.kdim = dim1[ap];
      for (int i = 0; i < dim1[a]; ++i)
        for (int kk = 0; kk < dim1[ap]; ++kk)
          Lc.push_back(blk[(size_t)(off1[a] + i) * m1 + off1[ap] + kk]);
      poolL += dim1[a];
      S->k1.push_back(k);
      flops += 2.0 * dim1[a] * dim1[ap] * S->qcols[rs.q];
    }
    rs.k1e = (int)S->k1.size();
  }
  for (size_t c = 0; c < S->cseg.size(); ++c) {
    ColSegD& cs = S->cseg[c];
    const int i3 = S->cs_i3[c], b = S->cs_b[c];
    cs.k2b = (int)S->k2.size();
    for (int e = ops->hRptr[i3]; e < ops->hRptr[i3 + 1]; ++e) {
      const int i3p = ops->hRcol[e];
      const int bp = find(idx4, sub(add(lab4[b], qc[i3]), qc[i3p]));
      if (bp < 0) continue;
      auto it = cs_of.find({i3p, bp});
      if (it == cs_of.end()) continue;
      const double* blk = HR.data() + (size_t)e * m4 * m4;
      double mx = 0.0;
      for (int i = 0; i < dim4[b]; ++i)
        for (int k = 0; k < dim4[bp]; ++k)
          mx = std::max(mx, std::fabs(blk[(size_t)(off4[b] + i) * m4 + off4[bp] + k]));
      if (mx == 0.0) continue;
      {
        const auto pe = S->plan.poolR.add(blk + (size_t)off4[b] * m4 + off4[bp], dim4[b],
                                          dim4[bp], m4);
        S->plan.k2.push_back({S->cseg[it->second].off, pe.first, dim4[bp], pe.second});
      }
      K2D k;
      k.b_off = (long long)Rc.size();
      k.b_pool = poolR;
      k.a_col = S->cseg[it->second].off;
      k.kdim = dim4[bp];
      for (int i = 0; i < dim4[b]; ++i)
        for (int kk = 0; kk < dim4[bp]; ++kk)
          Rc.push_back(blk[(size_t)(off4[b] + i) * m4 + off4[bp] + kk]);
      poolR += dim4[b];
      S->k2.push_back(k);
      flops += 2.0 * dim4[b] * dim4[bp] * qvalid_rows[cs.q];
    }
    cs.k2e = (int)S->k2.size();
  }
  // ---- CUDA-core tiles ----
  for (int q = 0; q < S->nQ; ++q)
    for (size_t r = 0; r < S->rseg.size(); ++r) {
      if (S->rseg[r].q != q) continue;
      for (int ri = 0; ri < S->rseg[r].dim; ri += SBM)
        for (size_t c = 0; c < S->cseg.size(); ++c) {
          if (S->cseg[c].q != q) continue;
          for (int ci = 0; ci < S->cseg[c].dim; ci += SBN)
            S->tiles.push_back({(int)r, (int)c, ri, ci});
        }
    }
  // ---- scalar moves per destination sub-block ----
  for (size_t r = 0; r < S->rseg.size(); ++r)
    for (size_t c = 0; c < S->cseg.size(); ++c) {
      if (S->rseg[r].q != S->cseg[c].q) continue;
      const int i2 = S->rs_i2[r], a = S->rs_a[r], i3 = S->cs_i3[c], b = S->cs_b[c];
      const int t = i2 + d * i3;
      MoveDst md{(int)r, (int)c, (int)S->msrc.size(), 0};
      for (int e = ops->hCptr[t]; e < ops->hCptr[t + 1]; ++e) {
        const int src = ops->hCsrc[e];
        const int s2 = src % d, s3 = src / d;
        auto ir = rs_of.find({s2, a});
        auto ic = cs_of.find({s3, b});
        if (ir == rs_of.end() || ic == cs_of.end()) continue;
        if (S->rseg[ir->second].q != S->cseg[ic->second].q) continue;
        S->msrc.push_back({ir->second, ic->second, ops->hCval[e], (float)ops->hCval[e]});
        flops += 2.0 * dim1[a] * dim4[b];
      }
      md.me = (int)S->msrc.size();
      if (md.me == md.mb) continue;
      const int di = (int)S->mdst.size();
      S->mdst.push_back(md);
      for (int ci = 0; ci < S->cseg[c].dim; ci += 8) S->mitems.push_back({di, ci});
    }
  ops->flops = flops;
  // ---- upload ----
  std::vector<float> Lc32(Lc.begin(), Lc.end()), Rc32(Rc.begin(), Rc.end());
  int64_t* nb = &ops->device_bytes;
  int st = DMRG2D_OK;
#define SUP(h, dp) \
  if (st == DMRG2D_OK) st = up(S, h, &dp, nb, s)
  SUP(S->qbase, S->d_qbase);
  SUP(S->qld, S->d_qld);
  SUP(S->rseg, S->d_rseg);
  SUP(S->cseg, S->d_cseg);
  SUP(S->k1, S->d_k1);
  SUP(S->k2, S->d_k2);
  SUP(S->tiles, S->d_tiles);
  SUP(S->mdst, S->d_mdst);
  SUP(S->msrc, S->d_msrc);
  SUP(S->mitems, S->d_mitems);
  SUP(Lc, S->d_L64);
  SUP(Lc32, S->d_L32);
  SUP(Rc, S->d_R64);
  SUP(Rc32, S->d_R32);
  SUP(S->pad_off, S->d_pad_off);
  SUP(S->pad_cnt, S->d_pad_cnt);
#undef SUP
  if (st == DMRG2D_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = set_error(DMRG2D_ECUDA, "sector upload: %s", cudaGetErrorString(e));
  }
  // ---- grouped tensor-core plan over the same segments ----
  if (st == DMRG2D_OK) {
    GroupPlan& g = S->plan;
    g.nQ = S->nQ;
    g.qbase = S->qbase;
    g.qld = S->qld;
    g.qcols = S->qcols;
    for (const RowSegD& r : S->rseg) g.rows.push_back({r.q, r.off, r.dim, r.dim_pad, r.k1b, r.k1e});
    for (const ColSegD& c : S->cseg) g.cols.push_back({c.q, c.off, c.dim, c.k2b, c.k2e});
    for (const MoveDst& md : S->mdst) {  // the scalar moves run in the grouped epilogue
      g.mdst.push_back({md.rs, md.cs, (int)g.moves.size(), 0});
      for (int e = md.mb; e < md.me; ++e)
        g.moves.push_back({S->msrc[e].rs, S->msrc[e].cs, S->msrc[e].c32});
      g.mdst.back().me = (int)g.moves.size();
    }
    const int gs = gp_finalise(ops, &g, s);
    if (gs == DMRG2D_OK) {
      S->gp_ok = true;
      ops->tc_ok = 1;
      for (int p = 0; p < 4; ++p) ops->tc_cfg[p] = 5;  // 128 x 256 longest-first
    } else if (gs == DMRG2D_EUNSUPPORTED) {
      clear_error();  // CUDA-core path only for this sector structure
    } else {
      st = gs;
    }
  }
  return st;
}

void sec_release(dmrg2d_ops* ops) {
  SecState* S = (SecState*)ops->sec;
  if (!S) return;
  gp_release(&S->plan);
  for (void* p : S->allocs) cudaFree(p);
  delete S;
  ops->sec = nullptr;
}

int sec_apply(const dmrg2d_ops* ops, const void* v, void* y, int precision, cudaStream_t s) {
  const SecState* S = (const SecState*)ops->sec;
  if (!S) return set_error(DMRG2D_EINVAL, "not a sector-restricted ops object");
  const SecParams p = S->params();
  const int nt = (int)S->tiles.size(), nm = (int)S->mitems.size();
  // timed kernel: the CUDA-core kernel here; the grouped tensor-core launch times itself
  const bool simt =
      precision == DMRG2D_FP64 || precision == DMRG2D_FP32 || precision == DMRG2D_FP64X;
  auto ev = simt ? prof_slot(ops) : std::pair<cudaEvent_t, cudaEvent_t>(nullptr, nullptr);
  if (ev.first) D2_CUDA(cudaEventRecord(ev.first, s));
  if (precision == DMRG2D_FP64 || precision == DMRG2D_FP64X) {
    // FP64X: the sub-block products in float pairs, the scalar moves in FP64
    if (nt && precision == DMRG2D_FP64)
      hv_simt_sec_kernel<double, double><<<nt, 256, 0, s>>>((const double*)v, (double*)y,
                                                            S->d_L64, S->d_R64, p);
    else if (nt)
      hv_simt_sec_kernel<double, ff><<<nt, 256, 0, s>>>((const double*)v, (double*)y, S->d_L64,
                                                        S->d_R64, p);
    if (ev.second) D2_CUDA(cudaEventRecord(ev.second, s));
    if (nm) k_sec_moves<double, double><<<nm, 256, 0, s>>>((const double*)v, (double*)y, p, 1);
  } else if (precision == DMRG2D_FP32) {
    if (nt) hv_simt_sec_kernel<float, float><<<nt, 256, 0, s>>>((const float*)v, (float*)y,
                                                              S->d_L32, S->d_R32, p);
    if (ev.second) D2_CUDA(cudaEventRecord(ev.second, s));
    if (nm) k_sec_moves<float, float><<<nm, 256, 0, s>>>((const float*)v, (float*)y, p, 0);
  } else if (precision == DMRG2D_BF16X3 && S->gp_ok && ops->tc_cfg[DMRG2D_BF16] == 2 * gp_num_configs()) {
    // segment kernels: three products, then the moves on v_hi and v_lo
    const __nv_bfloat16* vhi = (const __nv_bfloat16*)v;
    const __nv_bfloat16* vlo = vhi + ops->n_vec;
    D2_TRY(gp_launch_seg(ops, &S->plan, vhi, (float*)y, DMRG2D_BF16, s, false, false));
    D2_TRY(gp_launch_seg(ops, &S->plan, vlo, (float*)y, DMRG2D_BF16, s, false, true));
    D2_TRY(gp_launch_seg(ops, &S->plan, vhi, (float*)y, DMRG2D_BF16, s, true, true));
    if (nm) {
      k_sec_moves<__nv_bfloat16, float><<<nm, 256, 0, s>>>(vhi, (float*)y, p, 0);
      k_sec_moves<__nv_bfloat16, float><<<nm, 256, 0, s>>>(vlo, (float*)y, p, 0);
    }
  } else if ((precision == DMRG2D_TF32 || precision == DMRG2D_BF16) && S->gp_ok &&
             ops->tc_cfg[precision] == 2 * gp_num_configs()) {
    // segment kernels (M along the long dimension of each V_q), then the scalar moves
    D2_TRY(gp_launch_seg(ops, &S->plan, v, (float*)y, precision, s));
    if (nm) {
      if (precision == DMRG2D_BF16)
        k_sec_moves<__nv_bfloat16, float><<<nm, 256, 0, s>>>((const __nv_bfloat16*)v, (float*)y,
                                                            p, 0);
      else
        k_sec_moves<float, float><<<nm, 256, 0, s>>>((const float*)v, (float*)y, p, 0);
    }
  } else if (precision == DMRG2D_BF16X3 && S->gp_ok) {
    // v = [v_hi | v_lo]: H_hi v_hi + H_hi v_lo + H_lo v_hi with the layout chosen for BF16,
    // the scalar moves applied to v_hi and v_lo (in the epilogues, or their own kernel)
    const int G = gp_num_configs(), cfg = ops->tc_cfg[DMRG2D_BF16];
    const bool fused = cfg < G;
    const __nv_bfloat16* vhi = (const __nv_bfloat16*)v;
    const __nv_bfloat16* vlo = vhi + ops->n_vec;
    D2_TRY(gp_launch(ops, &S->plan, vhi, (float*)y, DMRG2D_BF16, cfg % G, s, fused, false, false));
    D2_TRY(gp_launch(ops, &S->plan, vlo, (float*)y, DMRG2D_BF16, cfg % G, s, fused, false, true));
    D2_TRY(gp_launch(ops, &S->plan, vhi, (float*)y, DMRG2D_BF16, cfg % G, s, false, true, true));
    if (!fused && nm) {
      k_sec_moves<__nv_bfloat16, float><<<nm, 256, 0, s>>>(vhi, (float*)y, p, 0);
      k_sec_moves<__nv_bfloat16, float><<<nm, 256, 0, s>>>(vlo, (float*)y, p, 0);
    }
  } else if ((precision == DMRG2D_TF32 || precision == DMRG2D_BF16) && S->gp_ok) {
    // tc_cfg < G: one launch, the grouped kernel's epilogue adds the scalar moves;
    // G <= tc_cfg < 2G: the moves run in their own kernel after it (G tile layouts)
    const int G = gp_num_configs(), cfg = ops->tc_cfg[precision];
    const bool fused = cfg < G;
    D2_TRY(gp_launch(ops, &S->plan, v, (float*)y, precision, cfg % G, s, fused));
    if (!fused && nm) {
      if (precision == DMRG2D_BF16)
        k_sec_moves<__nv_bfloat16, float><<<nm, 256, 0, s>>>((const __nv_bfloat16*)v, (float*)y,
                                                            p, 0);
      else
        k_sec_moves<float, float><<<nm, 256, 0, s>>>((const float*)v, (float*)y, p, 0);
    }
  } else {
    return set_error(DMRG2D_EUNSUPPORTED,
                     "sector-restricted H·v: precision %d not available here", precision);
  }
  D2_CUDA(cudaGetLastError());
  return DMRG2D_OK;
}

int sec_dense_index(const dmrg2d_ops* ops, int64_t* out) {
  const SecState* S = (const SecState*)ops->sec;
  if (!S) return set_error(DMRG2D_EINVAL, "not a sector-restricted ops object");
  const int64_t m1 = ops->m1, d = ops->d, m4 = ops->m4;
  for (int64_t p = 0; p < ops->n_vec; ++p) out[p] = -1;
  for (size_t r = 0; r < S->rseg.size(); ++r)
    for (size_t c = 0; c < S->cseg.size(); ++c) {
      const RowSegD& rs = S->rseg[r];
      const ColSegD& cs = S->cseg[c];
      if (rs.q != cs.q) continue;
      const int64_t i2 = S->rs_i2[r], i3 = S->cs_i3[c];
      const int64_t a0 = S->a_first[S->rs_a[r]], b0 = S->b_first[S->cs_b[c]];
      for (int j = 0; j < cs.dim; ++j)
        for (int i = 0; i < rs.dim; ++i) {
          const int64_t pos = S->qbase[rs.q] + rs.off + i + (int64_t)S->qld[rs.q] * (cs.off + j);
          const int64_t i1 = a0 + i, i4 = b0 + j;
          out[pos] = i1 + m1 * i2 + m1 * d * i4 + m1 * d * m4 * i3;
        }
    }
  return DMRG2D_OK;
}

int sec_diag_tables(const dmrg2d_ops* ops, std::vector<long long>& qbase, std::vector<int>& qld,
                    std::vector<int>& qcols, std::vector<double>& rowD, std::vector<int>& rowI2,
                    std::vector<double>& colD, std::vector<int>& colI3) {
  const SecState* S = (const SecState*)ops->sec;
  if (!S) return set_error(DMRG2D_EINVAL, "not a sector-restricted ops object");
  const int m1 = ops->m1, m4 = ops->m4;
  qbase = S->qbase;
  qld = S->qld;
  qcols = S->qcols;
  for (int q = 0; q < S->nQ; ++q) {
    const size_t r0 = rowD.size();
    rowD.resize(r0 + S->qld[q], 0.0);
    rowI2.resize(r0 + S->qld[q], -1);  // padding rows stay -1
    for (size_t r = 0; r < S->rseg.size(); ++r) {
      const RowSegD& rs = S->rseg[r];
      if (rs.q != q) continue;
      const int i2 = S->rs_i2[r], a0 = S->a_first[S->rs_a[r]];
      for (int i = 0; i < rs.dim; ++i) {
        rowD[r0 + rs.off + i] = ops->hdL[(size_t)(a0 + i) + (size_t)m1 * i2];
        rowI2[r0 + rs.off + i] = i2;
      }
    }
    const size_t c0 = colD.size();
    colD.resize(c0 + S->qcols[q], 0.0);
    colI3.resize(c0 + S->qcols[q], 0);
    for (size_t c = 0; c < S->cseg.size(); ++c) {
      const ColSegD& cs = S->cseg[c];
      if (cs.q != q) continue;
      const int i3 = S->cs_i3[c], b0 = S->b_first[S->cs_b[c]];
      for (int j = 0; j < cs.dim; ++j) {
        colD[c0 + cs.off + j] = ops->hdR[(size_t)(b0 + j) + (size_t)m4 * i3];
        colI3[c0 + cs.off + j] = i3;
      }
    }
  }
  return DMRG2D_OK;
}

int sec_layout(const dmrg2d_ops* ops, std::vector<long long>& qbase, std::vector<int>& qld,
               std::vector<int>& qcols, std::vector<int64_t>& row_left,
               std::vector<int64_t>& col_right) {
  const SecState* S = (const SecState*)ops->sec;
  if (!S) return set_error(DMRG2D_EINVAL, "not a sector-restricted ops object");
  const int64_t m1 = ops->m1, m4 = ops->m4;
  qbase = S->qbase;
  qld = S->qld;
  qcols = S->qcols;
  row_left.clear();
  col_right.clear();
  for (int q = 0; q < S->nQ; ++q) {
    const size_t r0 = row_left.size(), c0 = col_right.size();
    row_left.resize(r0 + S->qld[q], -1);  // padding rows stay -1
    col_right.resize(c0 + S->qcols[q], -1);
    for (size_t r = 0; r < S->rseg.size(); ++r) {
      const RowSegD& rs = S->rseg[r];
      if (rs.q != q) continue;
      const int64_t a0 = S->a_first[S->rs_a[r]], i2 = S->rs_i2[r];
      for (int i = 0; i < rs.dim; ++i) row_left[r0 + rs.off + i] = a0 + i + m1 * i2;
    }
    for (size_t c = 0; c < S->cseg.size(); ++c) {
      const ColSegD& cs = S->cseg[c];
      if (cs.q != q) continue;
      const int64_t b0 = S->b_first[S->cs_b[c]], i3 = S->cs_i3[c];
      for (int j = 0; j < cs.dim; ++j) col_right[c0 + cs.off + j] = b0 + j + m4 * i3;
    }
  }
  return DMRG2D_OK;
}

int sec_read_error(const dmrg2d_ops* ops, int* code) {
  *code = 0;
  const SecState* S = (const SecState*)ops->sec;
  if (!S || !S->gp_ok) return DMRG2D_OK;
  return gp_read_error(&S->plan, code);
}

int sec_count(const dmrg2d_ops* ops) {
  const SecState* S = (const SecState*)ops->sec;
  return S ? S->nQ : 0;
}

int sec_zero_padding(const dmrg2d_ops* ops, double* x, cudaStream_t s) {
  const SecState* S = (const SecState*)ops->sec;
  if (!S || S->pad_off.empty()) return DMRG2D_OK;
  const int n = (int)S->pad_off.size();
  k_zero_pad<<<(n + 255) / 256, 256, 0, s>>>(x, S->d_pad_off, S->d_pad_cnt, n);
  D2_CUDA(cudaGetLastError());
  return DMRG2D_OK;
}

}  // namespace dmrg2d
