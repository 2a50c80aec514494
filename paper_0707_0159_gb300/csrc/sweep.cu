// Finite-system direct 2-D DMRG around the superblock H·v (paper: the algorithm around
// Fig. 2) for Heisenberg ladders without quantum-number sectors.
//
// One step: the superblock block 1 + column 2 + column 3 + block 4 is built from the
// stored blocks (dmrg2d_build_ops), its ground state found on the GPU
// (dmrg2d_lanczos_ground: plain FP64 or the mixed-precision solver), the reduced
// density matrix of the growing half formed from V (rho_L = V V^T over rows i1 + m1 i2,
// or rho_R = V^T V over columns i4 + m4 i3; cuBLAS DSYRK, FP64) and diagonalised
// (cuSOLVER dsyevd, FP64).  Its m leading eigenvectors U (n x k, n = m d) define the new
// block: H' = U^T H_enl U and, per leg, the boundary operators U^T (X (x) 1) U of the
// added column.  H_enl is never formed: with U viewed as k matrices W_j (m x d, block
// index fast), (X (x) 1) U is W_j X^T for every j (one strided-batched DGEMM) and
// (1 (x) Y) U is Y [W_0 ... W_k-1] (one DGEMM).  New blocks are copied back to the host
// (k x k), where the next dmrg2d_build_ops reads them.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <vector>

#include "common.h"

namespace dmrg2d {

namespace {

using Mat = std::vector<double>;  // row-major

#define D2_BLAS(call)                                                                 \
  do {                                                                                \
    cublasStatus_t s_ = (call);                                                       \
    if (s_ != CUBLAS_STATUS_SUCCESS)                                                  \
      return set_error(DMRG2D_ECUDA, "%s failed (cuBLAS %d)", #call, (int)s_);        \
  } while (0)
#define D2_SOLV(call)                                                                 \
  do {                                                                                \
    cusolverStatus_t s_ = (call);                                                     \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                \
      return set_error(DMRG2D_ECUDA, "%s failed (cuSOLVER %d)", #call, (int)s_);      \
  } while (0)

struct DBuf;

// a renormalised block on the host: H and the boundary column's S^z_y, S^+_y (m x m);
// U (device, column-major (m_prev d) x m) is the truncation that made it from the block
// of one column less plus a column (block index fast), null for a one-column block
struct Block {
  int m = 0;
  Mat H;
  std::vector<Mat> edge;
  int m_prev = 0;
  std::shared_ptr<DBuf> U;
};

struct DBuf {
  double* p = nullptr;
  size_t n = 0;  // doubles
  ~DBuf() {
    if (p) cudaFree(p);
  }
  int alloc(size_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    if (cudaMalloc((void**)&p, count * sizeof(double)) != cudaSuccess) {
      p = nullptr;
      return set_error(DMRG2D_ENOMEM, "sweep: cudaMalloc(%zu doubles) failed", count);
    }
    n = count;
    return DMRG2D_OK;
  }
  int upload(const Mat& h, cudaStream_t s) {
    D2_TRY(alloc(h.size()));
    D2_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    return DMRG2D_OK;
  }
};

struct Libs {
  cublasHandle_t bl = nullptr;
  cusolverDnHandle_t sv = nullptr;
  ~Libs() {
    if (bl) cublasDestroy(bl);
    if (sv) cusolverDnDestroy(sv);
  }
};

// U[:, j] = Q[:, k-1-j]: Q holds k eigenvectors for ascending eigenvalues (the k largest
// of the spectrum); U lists them largest first
__global__ void k_take_leading(const double* __restrict__ Q, int64_t n, int k,
                               double* __restrict__ U) {
  const int64_t total = n * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = i / n, r = i - j * n;
    U[i] = Q[r + (k - 1 - j) * n];
  }
}

// xorshift64* stream for the start vectors (values in (-1, 1))
struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull) {}
  double next() {
    s ^= s >> 12;
    s ^= s << 25;
    s ^= s >> 27;
    const uint64_t r = s * 0x2545F4914F6CDD1Dull;
    return ((double)(r >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
  }
};

class Sweeper {
 public:
  Sweeper(const dmrg2d_model* M, const dmrg2d_sweep_opts* o, dmrg2d_sweep_report* rep,
          cudaStream_t s)
      : M_(*M), o_(*o), rep_(rep), strm_(s), rng_(o->seed) {}

  int run() {
    spin_column_ops(M_.n_legs, M_.J_rung, M_.rung_pbc != 0, &col_);
    D2_BLAS(cublasCreate(&libs_.bl));
    D2_BLAS(cublasSetStream(libs_.bl, strm_));
    D2_SOLV(cusolverDnCreate(&libs_.sv));
    D2_SOLV(cusolverDnSetStream(libs_.sv, strm_));
    // column operators on the device (row-major buffers)
    D2_TRY(dH_col_.upload(col_.H, strm_));
    dsz_.resize(col_.sz.size());
    dsp_.resize(col_.sp.size());
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      D2_TRY(dsz_[y].upload(col_.sz[y], strm_));
      D2_TRY(dsp_[y].upload(col_.sp[y], strm_));
    }
    const int L = o_.n_columns, half = (L - 2) / 2;
    std::map<int, Block> left, right;
    left[1] = column_block();
    right[1] = column_block();
    for (int l = 1; l < half; ++l) {  // warm-up: block 1 and its mirror image grow together
      Block nb;
      D2_TRY(step(left[l], right[l], true, o_.m_warmup, l, -1, &nb, nullptr));
      left[l + 1] = nb;
      right[l + 1] = nb;
    }
    std::shared_ptr<DBuf> guess;  // start vector of the next step (null: seeded random)
    if (half == 1) {
      D2_TRY(step(left[1], right[1], true, o_.m_warmup, 1, -1, nullptr, nullptr));
      guess = last_x_;  // the sweep's steps use the same superblock
    }
    for (int sw = 0; sw < o_.n_sweeps; ++sw) {
      const int m = o_.m_sweep[sw];
      for (int l = half; l < L - 3; ++l) {  // to the right end
        D2_TRY(step(left[l], right[L - 2 - l], true, m, l, sw, &left[l + 1], guess.get()));
        guess.reset();
        D2_TRY(move_right(left[l + 1], right[L - 2 - l], &guess));
      }
      for (int r = 1; r < L - 3; ++r) {  // to the left end
        const int l = L - 2 - r;
        D2_TRY(step(left[l], right[r], false, m, l, sw, &right[r + 1], guess.get()));
        guess.reset();
        D2_TRY(move_left(right[r + 1], left[l], &guess));
      }
      for (int l = 1; l < half; ++l) {  // back to the middle
        D2_TRY(step(left[l], right[L - 2 - l], true, m, l, sw, &left[l + 1], guess.get()));
        guess.reset();
        D2_TRY(move_right(left[l + 1], right[L - 2 - l], &guess));
      }
      D2_TRY(step(left[half], right[half], true, m, half, sw, nullptr, guess.get()));
      guess = last_x_;  // the next sweep starts on this superblock
    }
    return DMRG2D_OK;
  }

  double solve_seconds = 0.0, build_seconds = 0.0, dm_seconds = 0.0, renorm_seconds = 0.0;

 private:
  static double since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  Block column_block() const {
    Block b;
    b.m = col_.d;
    b.H = col_.H;
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      b.edge.push_back(col_.sz[y]);
      b.edge.push_back(col_.sp[y]);
    }
    return b;
  }

  // out = alpha (X (x) 1_m) W + beta out, W = [W_0 .. W_k-1] (m x d each, column-major);
  // X: row-major d x d on the device, transposed when tX
  int kron_col(const double* X, bool tX, const double* W, double* out, int m, int k,
               double alpha, double beta) {
    const int d = col_.d;
    D2_BLAS(cublasDgemmStridedBatched(libs_.bl, CUBLAS_OP_N, tX ? CUBLAS_OP_T : CUBLAS_OP_N, m, d,
                                      d, &alpha, W, m, (long long)m * d, X, d, 0, &beta, out, m,
                                      (long long)m * d, k));
    return DMRG2D_OK;
  }
  // out = (1_d (x) Y) W: Y row-major m x m on the device, transposed when tY
  int kron_blk(const double* Y, bool tY, const double* W, double* out, int m, int k) {
    const double one = 1.0, zero = 0.0;
    D2_BLAS(cublasDgemm(libs_.bl, tY ? CUBLAS_OP_N : CUBLAS_OP_T, CUBLAS_OP_N, m,
                        col_.d * k, m, &one, Y, m, W, m, &zero, out, m));
    return DMRG2D_OK;
  }

  // One DMRG step on block 1 = L, block 4 = R; grows L (grow_left) or R into *out.
  int step(const Block& Lb, const Block& Rb, bool grow_left, int m_keep, int l, int sweep,
           Block* out, const DBuf* guess) {
    // ---- HMED: superblock ground state -------------------------------------------------
    std::vector<const double*> le, re;
    for (auto& e : Lb.edge) le.push_back(e.data());
    for (auto& e : Rb.edge) re.push_back(e.data());
    dmrg2d_block bl{Lb.m, Lb.H.data(), (int)le.size(), le.data(), nullptr, nullptr};
    dmrg2d_block br{Rb.m, Rb.H.data(), (int)re.size(), re.data(), nullptr, nullptr};
    dmrg2d_ops* ops = nullptr;
    auto tb = std::chrono::steady_clock::now();
    D2_TRY(dmrg2d_build_ops(&M_, &bl, &br, nullptr, &ops, strm_));
    build_seconds += since(tb);
    struct FreeOps {
      dmrg2d_ops* p;
      ~FreeOps() { dmrg2d_free_ops(p); }
    } fo{ops};
    dmrg2d_ops_info info;
    D2_TRY(dmrg2d_ops_get_info(ops, &info));
    const int64_t nv = info.n_vec;
    auto xp = std::make_shared<DBuf>();
    DBuf& x = *xp;
    if (guess && guess->n == (size_t)nv) {  // the previous ground state, in this basis
      D2_TRY(x.alloc((size_t)nv));
      D2_CUDA(cudaMemcpyAsync(x.p, guess->p, nv * sizeof(double), cudaMemcpyDeviceToDevice,
                              strm_));
    } else {
      Mat x0((size_t)nv);
      for (auto& v : x0) v = rng_.next();
      D2_TRY(x.upload(x0, strm_));
    }
    last_x_ = xp;
    last_nv_ = nv;
    dmrg2d_solver_opts so;
    dmrg2d_default_solver_opts(&so);
    so.tol = o_.tol;
    so.krylov_dim = o_.krylov_dim;
    const bool mixed = o_.precision != DMRG2D_FP64 && info.tc_ok;
    if (mixed) {
      so.precision = o_.precision;
      so.refine = 1;
      so.inner_iter = std::min(o_.max_iter, 300);
      so.outer_max = 40;
    } else {
      so.precision = DMRG2D_FP64;
      so.max_iter = o_.max_iter;
    }
    double energy = 0.0;
    dmrg2d_solver_stats stats{};
    const auto t0 = std::chrono::steady_clock::now();
    const int st = dmrg2d_lanczos_ground(ops, &so, x.p, &energy, &stats, strm_);
    solve_seconds += since(t0);
    if (st != DMRG2D_OK && st != DMRG2D_ENOCONV) return st;
    const auto td = std::chrono::steady_clock::now();
    // ---- DMF: reduced density matrix of the growing half --------------------------------
    const int mb = grow_left ? Lb.m : Rb.m;  // block that grows
    const int d = col_.d;
    const int64_t n = (int64_t)mb * d;
    const int64_t other = nv / n;
    DBuf rho;
    D2_TRY(rho.alloc((size_t)(n * n)));
    const double one = 1.0, zero = 0.0;
    // V: (m1 d) x (d m4) column-major view of x; rho_L = V V^T, rho_R = V^T V (lower)
    D2_BLAS(cublasDsyrk(libs_.bl, CUBLAS_FILL_MODE_LOWER, grow_left ? CUBLAS_OP_N : CUBLAS_OP_T,
                        (int)n, (int)other, &one, x.p, grow_left ? (int)n : (int)other, &zero,
                        rho.p, (int)n));
    // ---- DMD: the k leading eigenpairs (selected by index, ascending order) ---------------
    const int k = (int)std::min<int64_t>(m_keep, n);
    double norm2 = 0.0;  // trace of rho = |x|^2
    D2_BLAS(cublasDdot(libs_.bl, (int)nv, x.p, 1, x.p, 1, &norm2));
    DBuf w, work;
    D2_TRY(w.alloc((size_t)n));
    int lwork = 0, meig = 0;
    const int il = (int)n - k + 1, iu = (int)n;  // 1-based eigenvalue indices
    D2_SOLV(cusolverDnDsyevdx_bufferSize(libs_.sv, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                         CUBLAS_FILL_MODE_LOWER, (int)n, rho.p, (int)n, 0.0, 0.0,
                                         il, iu, &meig, w.p, &lwork));
    D2_TRY(work.alloc((size_t)std::max(lwork, 1)));
    int* dinfo = nullptr;
    D2_CUDA(cudaMalloc((void**)&dinfo, sizeof(int)));
    struct FreeInt {
      int* p;
      ~FreeInt() { cudaFree(p); }
    } fi{dinfo};
    D2_SOLV(cusolverDnDsyevdx(libs_.sv, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                              CUBLAS_FILL_MODE_LOWER, (int)n, rho.p, (int)n, 0.0, 0.0, il, iu,
                              &meig, w.p, work.p, lwork, dinfo));
    int hinfo = 0;
    Mat hw((size_t)k);
    D2_CUDA(cudaMemcpyAsync(&hinfo, dinfo, sizeof(int), cudaMemcpyDeviceToHost, strm_));
    D2_CUDA(cudaMemcpyAsync(hw.data(), w.p, k * sizeof(double), cudaMemcpyDeviceToHost, strm_));
    D2_CUDA(cudaStreamSynchronize(strm_));
    dm_seconds += since(td);
    if (hinfo != 0 || meig != k)
      return set_error(DMRG2D_ECUDA, "sweep: dsyevdx info %d, %d of %d eigenpairs", hinfo, meig, k);
    double kept = 0.0;
    for (int j = 0; j < k; ++j) kept += hw[(size_t)j];
    kept /= norm2;
    record(energy, 1.0 - kept, l, sweep, stats.iters);
    if (!out) return DMRG2D_OK;
    // ---- renormalisation: U^T O U for H_enl and the new boundary operators ----------------
    const auto tr = std::chrono::steady_clock::now();
    auto Up = std::make_shared<DBuf>();
    DBuf &U = *Up, HU, T;
    D2_TRY(U.alloc((size_t)(n * k)));
    D2_TRY(HU.alloc((size_t)(n * k)));
    D2_TRY(T.alloc((size_t)(n * k)));
    k_take_leading<<<1024, 256, 0, strm_>>>(rho.p, n, k, U.p);
    D2_CUDA(cudaGetLastError());
    const Block& B = grow_left ? Lb : Rb;
    DBuf dHB;
    D2_TRY(dHB.upload(B.H, strm_));
    // H_enl U = (1 (x) H_B) U + (H_col (x) 1) U
    //         + J sum_y [ (Sz_y (x) SzB_y) + 1/2 (S-_y (x) S+B_y) + 1/2 (S+_y (x) S-B_y) ] U
    D2_TRY(kron_blk(dHB.p, false, U.p, HU.p, mb, k));
    D2_TRY(kron_col(dH_col_.p, false, U.p, HU.p, mb, k, 1.0, 1.0));
    const double J = M_.J_leg;
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      DBuf dz, dp;
      D2_TRY(dz.upload(B.edge[2 * y], strm_));
      D2_TRY(dp.upload(B.edge[2 * y + 1], strm_));
      D2_TRY(kron_blk(dz.p, false, U.p, T.p, mb, k));
      D2_TRY(kron_col(dsz_[y].p, false, T.p, HU.p, mb, k, J, 1.0));
      D2_TRY(kron_blk(dp.p, false, U.p, T.p, mb, k));  // S+ of the block
      D2_TRY(kron_col(dsp_[y].p, true, T.p, HU.p, mb, k, 0.5 * J, 1.0));  // with S- = (S+)^T
      D2_TRY(kron_blk(dp.p, true, U.p, T.p, mb, k));  // S- of the block
      D2_TRY(kron_col(dsp_[y].p, false, T.p, HU.p, mb, k, 0.5 * J, 1.0));
    }
    DBuf small;
    D2_TRY(small.alloc((size_t)k * k));
    Mat hs((size_t)k * k);
    auto project = [&](const double* XU, Mat* dst, bool symmetrise) -> int {
      // dst (row-major) = U^T XU; the column-major product is transposed on the way out
      D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_T, CUBLAS_OP_N, k, k, (int)n, &one, U.p, (int)n, XU,
                          (int)n, &zero, small.p, k));
      D2_CUDA(cudaMemcpyAsync(hs.data(), small.p, (size_t)k * k * sizeof(double),
                              cudaMemcpyDeviceToHost, strm_));
      D2_CUDA(cudaStreamSynchronize(strm_));
      dst->assign((size_t)k * k, 0.0);
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
          const double a = hs[(size_t)i + (size_t)j * k];  // (i, j) of the product
          (*dst)[(size_t)i * k + j] =
              symmetrise ? 0.5 * (a + hs[(size_t)j + (size_t)i * k]) : a;
        }
      return DMRG2D_OK;
    };
    out->m = k;
    out->m_prev = mb;
    out->U = Up;
    D2_TRY(project(HU.p, &out->H, true));
    out->edge.assign(2 * col_.sz.size(), Mat());
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      D2_TRY(kron_col(dsz_[y].p, false, U.p, T.p, mb, k, 1.0, 0.0));
      D2_TRY(project(T.p, &out->edge[2 * y], false));
      D2_TRY(kron_col(dsp_[y].p, false, U.p, T.p, mb, k, 1.0, 0.0));
      D2_TRY(project(T.p, &out->edge[2 * y + 1], false));
    }
    renorm_seconds += since(tr);
    return DMRG2D_OK;
  }

  void record(double e, double trunc, int l, int sweep, int iters) {
    const int i = rep_->n_steps++;
    if (i < rep_->cap) {
      if (rep_->iters) rep_->iters[i] = iters;
      if (rep_->energy) rep_->energy[i] = e;
      if (rep_->trunc) rep_->trunc[i] = trunc;
      if (rep_->l) rep_->l[i] = l;
      if (rep_->sweep) rep_->sweep[i] = sweep;
    }
  }

  std::shared_ptr<DBuf> last_x_;  // ground state of the last step's superblock
  int64_t last_nv_ = 0;

  // Guess for the superblock after moving right: block 1 grew into nl (its U: (m_l d) x k),
  // block 4 = Rs of m_r states (made from a block of m' states plus a column, Rs.U:
  // (m' d) x m_r) splits into that column and that block.  Old V: (m_l d) x (d m_r).
  //   W = U^T V (k x d m_r);  V'[(a + k s3), (b' + m' t)] = sum_b W[a, b + m_r s3] Rs.U[b' + m' t, b]
  int move_right(const Block& nl, const Block& Rs, std::shared_ptr<DBuf>* out) {
    const int d = col_.d, k = nl.m, ml = nl.m_prev, mr = Rs.m, mp = Rs.m_prev;
    const int64_t nL = (int64_t)ml * d, nR = (int64_t)d * mr;
    if (!nl.U || !Rs.U || last_nv_ != nL * nR) return DMRG2D_OK;  // no guess
    DBuf W;
    D2_TRY(W.alloc((size_t)k * nR));
    auto v = std::make_shared<DBuf>();
    D2_TRY(v->alloc((size_t)k * d * d * mp));
    const double one = 1.0, zero = 0.0;
    D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_T, CUBLAS_OP_N, k, (int)nR, (int)nL, &one, nl.U->p,
                        (int)nL, last_x_->p, (int)nL, &zero, W.p, k));
    D2_BLAS(cublasDgemmStridedBatched(libs_.bl, CUBLAS_OP_N, CUBLAS_OP_T, k, mp * d, mr, &one, W.p, k,
                                      (long long)k * mr, Rs.U->p, mp * d, 0, &zero, v->p, k * d,
                                      (long long)k, d));
    *out = v;
    return DMRG2D_OK;
  }
  // Guess after moving left: block 4 grew into nr (its U: (m_r d) x k), block 1 = Ls of
  // m_l states (from m' states plus a column, Ls.U: (m' d) x m_l) splits.  Old V as above.
  //   W = V U (m_l d x k);  V'[(a' + m' t), (b + k s2)] = sum_a Ls.U[a' + m' t, a] W[a + m_l s2, b]
  int move_left(const Block& nr, const Block& Ls, std::shared_ptr<DBuf>* out) {
    const int d = col_.d, k = nr.m, mr = nr.m_prev, ml = Ls.m, mp = Ls.m_prev;
    const int64_t nL = (int64_t)ml * d, nR = (int64_t)d * mr;
    if (!nr.U || !Ls.U || last_nv_ != nL * nR) return DMRG2D_OK;
    DBuf W;
    D2_TRY(W.alloc((size_t)nL * k));
    auto v = std::make_shared<DBuf>();
    D2_TRY(v->alloc((size_t)mp * d * d * k));
    const double one = 1.0, zero = 0.0;
    D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_N, CUBLAS_OP_N, (int)nL, k, (int)nR, &one,
                        last_x_->p, (int)nL, nr.U->p, (int)nR, &zero, W.p, (int)nL));
    D2_BLAS(cublasDgemmStridedBatched(libs_.bl, CUBLAS_OP_N, CUBLAS_OP_N, mp * d, k, ml, &one,
                                      Ls.U->p, mp * d, 0, W.p, (int)nL, (long long)ml, &zero, v->p,
                                      mp * d, (long long)mp * d * k, d));
    *out = v;
    return DMRG2D_OK;
  }

  dmrg2d_model M_;
  dmrg2d_sweep_opts o_;
  dmrg2d_sweep_report* rep_;
  cudaStream_t strm_;
  Rng rng_;
  SpinColumnOps col_;
  Libs libs_;
  DBuf dH_col_;
  std::vector<DBuf> dsz_, dsp_;
};

}  // namespace

}  // namespace dmrg2d

using namespace dmrg2d;

extern "C" int dmrg2d_sweep(const dmrg2d_model* model, const dmrg2d_sweep_opts* opts,
                            dmrg2d_sweep_report* report, void* stream) {
  if (!model || !opts || !report) return set_error(DMRG2D_EINVAL, "sweep: NULL argument");
  clear_error();
  if (model->kind != DMRG2D_HEISENBERG)
    return set_error(DMRG2D_EUNSUPPORTED, "sweep: Heisenberg ladders only");
  if (model->n_legs < 1 || model->n_legs > 8)
    return set_error(DMRG2D_EINVAL, "sweep: n_legs must be in [1, 8]");
  if (opts->n_columns < 4 || opts->n_columns % 2)
    return set_error(DMRG2D_EINVAL, "sweep: n_columns must be even and >= 4");
  if (opts->m_warmup < 1 || opts->n_sweeps < 0 || (opts->n_sweeps > 0 && !opts->m_sweep))
    return set_error(DMRG2D_EINVAL, "sweep: bad m_warmup / n_sweeps / m_sweep");
  for (int i = 0; i < opts->n_sweeps; ++i)
    if (opts->m_sweep[i] < 1) return set_error(DMRG2D_EINVAL, "sweep: m_sweep[%d] < 1", i);
  if (opts->max_iter < 1 || opts->krylov_dim < 2 || !(opts->tol > 0.0))
    return set_error(DMRG2D_EINVAL, "sweep: bad solver options");
  if (report->cap < 0) return set_error(DMRG2D_EINVAL, "sweep: report cap < 0");
  report->n_steps = 0;
  report->seconds = report->solve_seconds = report->build_seconds = 0.0;
  report->dm_seconds = report->renorm_seconds = 0.0;
  const auto t0 = std::chrono::steady_clock::now();
  Sweeper sw(model, opts, report, (cudaStream_t)stream);
  const int st = sw.run();
  report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  report->solve_seconds = sw.solve_seconds;
  report->build_seconds = sw.build_seconds;
  report->dm_seconds = sw.dm_seconds;
  report->renorm_seconds = sw.renorm_seconds;
  return st;
}
