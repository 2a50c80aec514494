// Finite-system direct 2-D DMRG around the superblock H·v (paper: the algorithm around
// Fig. 2) for Heisenberg ladders (dense, or in the S^z_tot = 0 sector) and Hubbard
// ladders (in a target (N_up, N_dn) sector).
//
// One step: the superblock block 1 + column 2 + column 3 + block 4 is built from the
// stored blocks (dmrg2d_build_ops), its ground state found on the GPU
// (dmrg2d_lanczos_ground: plain FP64 or the mixed-precision solver), the reduced
// density matrix of the growing half formed from V (rho_L = V V^T over rows i1 + m1 i2,
// or rho_R = V^T V over columns i4 + m4 i3; cuBLAS DSYRK, FP64) and diagonalised
// (cuSOLVER dsyevd, FP64).  Its m leading eigenvectors U (n x k, n = m d) define the new
// block: H' = U^T H_enl U and, per leg, the boundary operators U^T (X (x) 1) U of the
// added column (Hubbard: its creation operators, carrying the parity of the modes before
// them in the block's mode order).  H_enl is never formed: with U viewed as k matrices
// W_j (m x d, block
// index fast), (X (x) 1) U is W_j X^T for every j (one strided-batched DGEMM) and
// (1 (x) Y) U is Y [W_0 ... W_k-1] (one DGEMM).  New blocks are copied back to the host
// (k x k), where the next dmrg2d_build_ops reads them.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <tuple>
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
  int cols = 1;                 // lattice columns in the block
  std::vector<int32_t> qn;      // sectors: N_up (Hubbard: N_up, N_dn) of each state,
                                // equal labels contiguous
  Mat Sz_tot, Sp_tot;           // the block's total S^z and S^+ (for <S_tot^2>)
  Mat parity;                   // Hubbard: (-1)^N of each state
};

struct IBuf {  // device int64 / int32 arrays for the sector maps
  void* p = nullptr;
  ~IBuf() {
    if (p) cudaFree(p);
  }
  template <typename T>
  int upload(const std::vector<T>& h, cudaStream_t s) {
    if (p) cudaFree(p);
    p = nullptr;
    if (h.empty()) return DMRG2D_OK;
    if (cudaMalloc(&p, h.size() * sizeof(T)) != cudaSuccess) {
      p = nullptr;
      return set_error(DMRG2D_ENOMEM, "sweep: cudaMalloc failed (maps)");
    }
    D2_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return DMRG2D_OK;
  }
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

// library handles on the sweep's stream, and kSide side streams with their own handles
// (the density matrices of different sectors are formed and diagonalised concurrently)
constexpr int kSide = 4;
struct Libs {
  cublasHandle_t bl = nullptr;
  cusolverDnHandle_t sv = nullptr;
  cudaStream_t side[kSide] = {};
  cublasHandle_t sbl[kSide] = {};
  cusolverDnHandle_t ssv[kSide] = {};
  cudaEvent_t ev_main = nullptr, ev_side[kSide] = {};
  ~Libs() {
    if (bl) cublasDestroy(bl);
    if (sv) cusolverDnDestroy(sv);
    for (int k = 0; k < kSide; ++k) {
      if (sbl[k]) cublasDestroy(sbl[k]);
      if (ssv[k]) cusolverDnDestroy(ssv[k]);
      if (ev_side[k]) cudaEventDestroy(ev_side[k]);
      if (side[k]) cudaStreamDestroy(side[k]);
    }
    if (ev_main) cudaEventDestroy(ev_main);
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

// One matrix V_q of a sector-restricted vector against the dense V (ldd rows):
// to_packed: xq[r + qld c] = Vd[rowL[r] + ldd colR[c]] (0 on padding rows); else the reverse.
__global__ void k_pack(double* __restrict__ Vd, int64_t ldd, double* __restrict__ xq, int qld,
                       int qcols, const int64_t* __restrict__ rowL,
                       const int64_t* __restrict__ colR, int to_packed) {
  const int64_t total = (int64_t)qld * qcols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % qld), c = (int)(i / qld);
    const int64_t row = rowL[r];
    if (to_packed)
      xq[i] = row >= 0 ? Vd[row + ldd * colR[c]] : 0.0;
    else if (row >= 0)
      Vd[row + ldd * colR[c]] = xq[i];
  }
}

// G (nr x cols) = the rows rows[0..nr) of X (ldx rows)
__global__ void k_gather_rows(const double* __restrict__ X, int ldx, int cols,
                              const int* __restrict__ rows, int nr, double* __restrict__ G) {
  const int64_t total = (int64_t)nr * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % nr), c = (int)(i / nr);
    G[i] = X[rows[r] + (int64_t)ldx * c];
  }
}

// U[idx[i], col] = Q[i + ldq * qcol] for i < len
__global__ void k_scatter_col(const double* __restrict__ Q, int ldq, int qcol, int len,
                              const int64_t* __restrict__ idx, double* __restrict__ U, int64_t ldu,
                              int col) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x)
    U[idx[i] + ldu * col] = Q[i + (int64_t)ldq * qcol];
}

// U[pos[i]] = 1 (the unit-vector columns of zero-weight kept states)
__global__ void k_set_ones(double* __restrict__ U, const int64_t* __restrict__ pos, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    U[pos[i]] = 1.0;
}

// G[r + nr c] = X[idx[r] + ldx c] (0 where idx[r] < 0): rows of X picked by an index list
__global__ void k_gather_idx(const double* __restrict__ X, int64_t ldx,
                             const int64_t* __restrict__ idx, int nr, int nc,
                             double* __restrict__ G) {
  const int64_t total = (int64_t)nr * nc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % nr), c = (int)(i / nr);
    const int64_t row = idx[r];
    G[i] = row >= 0 ? X[row + ldx * c] : 0.0;
  }
}

// by_rows: Y[idx[r] + ldy c] = G[r + nr c]; else Y[r + ldy idx[c]] = G[r + nr c]
// (entries whose index is negative are skipped)
__global__ void k_scatter_idx(const double* __restrict__ G, int nr, int nc,
                              const int64_t* __restrict__ idx, int by_rows,
                              double* __restrict__ Y, int64_t ldy) {
  const int64_t total = (int64_t)nr * nc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % nr), c = (int)(i / nr);
    if (by_rows) {
      if (idx[r] >= 0) Y[idx[r] + ldy * c] = G[i];
    } else if (idx[c] >= 0) {
      Y[r + ldy * idx[c]] = G[i];
    }
  }
}

// One term of an expectation value on a packed vector: coef * <sub-block 1, sub-block 2>,
// both rows x cols column-major (leading dimensions ld1, ld2) at offsets off1, off2
struct DotItem {
  long long off1, off2;
  int ld1, ld2, rows, cols;
  double coef;
};
// out[i] = value of item i (one CTA per item at a time, block reduction)
__global__ void __launch_bounds__(256) k_item_dots(const double* __restrict__ x,
                                                   const DotItem* __restrict__ items, int n,
                                                   double* __restrict__ out) {
  __shared__ double red[8];
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const DotItem t = items[it];
    const long long total = (long long)t.rows * t.cols;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < total; i += 256) {
      const long long r = i % t.rows, c = i / t.rows;
      acc += x[t.off1 + r + t.ld1 * c] * x[t.off2 + r + t.ld2 * c];
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < 8 ? red[threadIdx.x] : 0.0;
      for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (threadIdx.x == 0) out[it] = t.coef * v;
    }
    __syncthreads();
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
  uint64_t next_u64() {
    s ^= s >> 12;
    s ^= s << 25;
    s ^= s >> 27;
    return s * 0x2545F4914F6CDD1Dull;
  }
};

// the learned preconditioner's training inside a sweep: recorded Davidson steps per
// solve, samples per Adam step, learning rate
constexpr int kTrainLog = 16;
constexpr int kTrainBatch = 8192;
constexpr float kTrainLr = 3e-4f;

class Sweeper {
 public:
  Sweeper(const dmrg2d_model* M, const dmrg2d_sweep_opts* o, dmrg2d_sweep_report* rep,
          cudaStream_t s)
      : M_(*M), o_(*o), rep_(rep), strm_(s), rng_(o->seed), train_rng_(o->seed ^ 0x7A11ull) {}

  // Column operators, their device copies and the library handles (once per run).
  int init() {
    hub_ = M_.kind == DMRG2D_HUBBARD;
    if (hub_) {  // the spin operators stay empty: every per-leg spin loop below is skipped
      hubbard_column_ops(M_.n_legs, M_.t, M_.U, M_.rung_pbc != 0, &hc_);
      col_.d = hc_.d;
      col_.H = hc_.H;
      col_.sz.clear();
      col_.sp.clear();
    } else {
      spin_column_ops(M_.n_legs, M_.J_rung, M_.rung_pbc != 0, &col_);
    }
    D2_BLAS(cublasCreate(&libs_.bl));
    D2_BLAS(cublasSetStream(libs_.bl, strm_));
    D2_SOLV(cusolverDnCreate(&libs_.sv));
    D2_SOLV(cusolverDnSetStream(libs_.sv, strm_));
    D2_CUDA(cudaEventCreateWithFlags(&libs_.ev_main, cudaEventDisableTiming));
    for (int k = 0; k < kSide; ++k) {
      D2_CUDA(cudaStreamCreateWithFlags(&libs_.side[k], cudaStreamNonBlocking));
      D2_CUDA(cudaEventCreateWithFlags(&libs_.ev_side[k], cudaEventDisableTiming));
      D2_BLAS(cublasCreate(&libs_.sbl[k]));
      D2_BLAS(cublasSetStream(libs_.sbl[k], libs_.side[k]));
      D2_SOLV(cusolverDnCreate(&libs_.ssv[k]));
      D2_SOLV(cusolverDnSetStream(libs_.ssv[k], libs_.side[k]));
    }
    // column operators on the device (row-major buffers)
    D2_TRY(dH_col_.upload(col_.H, strm_));
    const int dd = col_.d, nl = (int)col_.sz.size();
    col_Sz_tot_.assign((size_t)dd * dd, 0.0);
    col_Sp_tot_.assign((size_t)dd * dd, 0.0);
    for (int y = 0; y < nl; ++y)
      for (size_t e = 0; e < col_Sz_tot_.size(); ++e) {
        col_Sz_tot_[e] += col_.sz[y][e];
        col_Sp_tot_[e] += col_.sp[y][e];
      }
    D2_TRY(dSz_tot_.upload(col_Sz_tot_, strm_));
    D2_TRY(dSp_tot_.upload(col_Sp_tot_, strm_));
    // rung bond S_y . S_{y+1} of one column (row-major d x d)
    auto mm = [dd](const Mat& a, const Mat& b) {
      Mat c((size_t)dd * dd, 0.0);
      for (int i = 0; i < dd; ++i)
        for (int k = 0; k < dd; ++k) {
          const double x = a[(size_t)i * dd + k];
          if (x != 0.0)
            for (int j = 0; j < dd; ++j) c[(size_t)i * dd + j] += x * b[(size_t)k * dd + j];
        }
      return c;
    };
    auto tr = [dd](const Mat& a) {
      Mat t((size_t)dd * dd);
      for (int i = 0; i < dd; ++i)
        for (int j = 0; j < dd; ++j) t[(size_t)j * dd + i] = a[(size_t)i * dd + j];
      return t;
    };
    drung_.resize(std::max(nl - 1, 0));
    rung_h_.clear();
    for (int y = 0; y + 1 < nl; ++y) {
      Mat b = mm(col_.sz[y], col_.sz[y + 1]);
      const Mat pm = mm(col_.sp[y], tr(col_.sp[y + 1])), mp = mm(tr(col_.sp[y]), col_.sp[y + 1]);
      for (size_t e = 0; e < b.size(); ++e) b[e] += 0.5 * (pm[e] + mp[e]);
      D2_TRY(drung_[y].upload(b, strm_));
      rung_h_.push_back(b);
    }
    dsz_.resize(col_.sz.size());
    dsp_.resize(col_.sp.size());
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      D2_TRY(dsz_[y].upload(col_.sz[y], strm_));
      D2_TRY(dsp_[y].upload(col_.sp[y], strm_));
    }
    if (hub_) {  // c^dag_j and c^dag_j P of the column, row-major
      dcd_.resize(hc_.cd.size());
      dcdP_.resize(hc_.cd.size());
      for (size_t j = 0; j < hc_.cd.size(); ++j) {
        Mat cp = hc_.cd[j];
        for (int r = 0; r < dd; ++r)
          for (int c = 0; c < dd; ++c) cp[(size_t)r * dd + c] *= hc_.parity[(size_t)c];
        D2_TRY(dcd_[j].upload(hc_.cd[j], strm_));
        D2_TRY(dcdP_[j].upload(cp, strm_));
      }
    }
    return DMRG2D_OK;
  }

  // Infinite-system warm-up: block 1 and block 4 grow together until the superblock spans
  // the lattice.
  int warmup() {
    const int L = o_.n_columns, half = (L - 2) / 2;
    left_[1] = column_block();
    right_[1] = column_block();
    for (int l = 1; l < half; ++l) {  // warm-up: block 1 and its mirror image grow together
      if (hub_) {  // electrons: block 4 grows from its own density matrix (a mirrored
                   // block would have the reversed mode order); one ground state serves both
        Block nl, nr;
        D2_TRY(step(left_[l], right_[l], true, o_.m_warmup, l, -1, &nl, nullptr, &nr));
        left_[l + 1] = nl;
        right_[l + 1] = nr;
        continue;
      }
      Block nb;
      D2_TRY(step(left_[l], right_[l], true, o_.m_warmup, l, -1, &nb, nullptr));
      left_[l + 1] = nb;
      right_[l + 1] = nb;
    }
    guess_.reset();  // start vector of the next step (null: seeded random)
    if (half == 1) {
      D2_TRY(step(left_[1], right_[1], true, o_.m_warmup, 1, -1, nullptr, nullptr));
      guess_ = last_x_;  // the sweep's steps use the same superblock
    }
    warm_done_ = true;
    return DMRG2D_OK;
  }

  // n finite sweeps (to the right end, to the left end, back to the middle), sweep s
  // keeping m_sweep[s] states; sweep indices continue those of earlier calls.
  int sweeps(int n, const int* m_sweep) {
    const int L = o_.n_columns, half = (L - 2) / 2;
    for (int s = 0; s < n; ++s) {
      const int m = m_sweep[s], sw = sweeps_done_;
      std::shared_ptr<DBuf>& guess = guess_;
      for (int l = half; l < L - 3; ++l) {  // to the right end
        D2_TRY(step(left_[l], right_[L - 2 - l], true, m, l, sw, &left_[l + 1], guess.get()));
        guess.reset();
        D2_TRY(timed_move(true, left_[l + 1], right_[L - 2 - l], &guess));
      }
      for (int r = 1; r < L - 3; ++r) {  // to the left end
        const int l = L - 2 - r;
        D2_TRY(step(left_[l], right_[r], false, m, l, sw, &right_[r + 1], guess.get()));
        guess.reset();
        D2_TRY(timed_move(false, right_[r + 1], left_[l], &guess));
      }
      for (int l = 1; l < half; ++l) {  // back to the middle
        D2_TRY(step(left_[l], right_[L - 2 - l], true, m, l, sw, &left_[l + 1], guess.get()));
        guess.reset();
        D2_TRY(timed_move(true, left_[l + 1], right_[L - 2 - l], &guess));
      }
      D2_TRY(step(left_[half], right_[half], true, m, half, sw, nullptr, guess.get()));
      guess = last_x_;  // the next sweep starts on this superblock
      ++sweeps_done_;
    }
    return DMRG2D_OK;
  }

  // One call of dmrg2d_sweep on this run: its solver options, report and stream.
  int begin_call(const dmrg2d_sweep_opts* o, dmrg2d_sweep_report* rep, cudaStream_t s) {
    o_.precision = o->precision;
    o_.tol = o->tol;
    o_.max_iter = o->max_iter;
    o_.krylov_dim = o->krylov_dim;
    o_.solver = o->solver;
    o_.precond = o->precond;
    o_.mlp = o->mlp;
    o_.mlp_train_sweeps = o->mlp_train_sweeps;
    o_.mlp_epochs = o->mlp_epochs;
    rep_ = rep;
    strm_ = s;
    solve_seconds = build_seconds = dm_seconds = renorm_seconds = obs_seconds = 0.0;
    train_seconds = transform_seconds = 0.0;
    if (libs_.bl) D2_BLAS(cublasSetStream(libs_.bl, strm_));
    if (libs_.sv) D2_SOLV(cusolverDnSetStream(libs_.sv, strm_));
    return DMRG2D_OK;
  }

  bool warm_done() const { return warm_done_; }
  int sweeps_done() const { return sweeps_done_; }
  double last_energy() const { return last_energy_; }
  const dmrg2d_model& model() const { return M_; }
  const dmrg2d_sweep_opts& opts() const { return o_; }
  int block_states(bool left, int cols) const {
    const auto& mp = left ? left_ : right_;
    auto it = mp.find(cols);
    return it == mp.end() ? 0 : it->second.m;
  }

  double solve_seconds = 0.0, build_seconds = 0.0, dm_seconds = 0.0, renorm_seconds = 0.0,
         obs_seconds = 0.0, train_seconds = 0.0, transform_seconds = 0.0;

 private:
  static double since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  // The wavefunction transformation after a step (the next step's start vector), timed.
  int timed_move(bool right, const Block& grown, const Block& other, std::shared_ptr<DBuf>* g) {
    const auto t0 = std::chrono::steady_clock::now();
    const int st = right ? move_right(grown, other, g) : move_left(grown, other, g);
    if (st == DMRG2D_OK && cudaStreamSynchronize(strm_) != cudaSuccess)
      return set_error(DMRG2D_ECUDA, "sweep: wavefunction transformation");
    transform_seconds += since(t0);
    return st;
  }

  // HMED: the superblock ground state from the start vector x (overwritten).  Lanczos:
  // plain FP64 with thick restart, or the mixed solver (low-precision H·v, FP64 outer
  // loop); Davidson: the same precisions with the chosen preconditioner.  A Davidson solve
  // that trains the learned preconditioner (warm-up and the first mlp_train_sweeps sweeps)
  // runs with Jacobi, records its first steps and then trains the network on them.
  int solve(const dmrg2d_ops* ops, const dmrg2d_ops_info& info, DBuf& x, int sweep,
            double* energy, dmrg2d_solver_stats* stats) {
    const bool mixed = o_.precision != DMRG2D_FP64 && info.tc_ok;
    const auto t0 = std::chrono::steady_clock::now();
    if (o_.solver == DMRG2D_SWEEP_LANCZOS) {
      dmrg2d_solver_opts so;
      dmrg2d_default_solver_opts(&so);
      so.tol = o_.tol;
      so.krylov_dim = o_.krylov_dim;
      if (mixed) {
        so.precision = o_.precision;
        so.refine = 1;
        so.refine_precision = DMRG2D_FP64X;  // outer-loop residuals in float pairs
        so.inner_iter = std::min(o_.max_iter, 300);
        so.outer_max = 40;
      } else {
        so.precision = DMRG2D_FP64;
        so.max_iter = o_.max_iter;
        so.thick_keep = std::min(16, o_.krylov_dim / 4);
      }
      const int st = dmrg2d_lanczos_ground(ops, &so, x.p, energy, stats, strm_);
      solve_seconds += since(t0);
      return st;
    }
    dmrg2d_davidson_opts dv;
    dmrg2d_default_davidson_opts(&dv);
    dv.max_iter = o_.max_iter;
    dv.max_subspace = std::min(48, std::max(4, o_.krylov_dim));
    const bool train =
        o_.precond == DMRG2D_PRECOND_MLP && o_.mlp_epochs > 0 && sweep < o_.mlp_train_sweeps;
    dv.precond = train ? DMRG2D_PRECOND_JACOBI : o_.precond;
    dv.mlp = o_.mlp;
    if (mixed) {
      dv.precision = o_.precision;
      dv.refine = 1;
      dv.tol = std::max(o_.tol, o_.precision == DMRG2D_BF16 ? 1e-2 : 1e-3);
      dv.refine_tol = o_.tol;
      dv.inner_iter = 40;
      dv.outer_max = 40;
    } else {
      dv.precision = DMRG2D_FP64;
      dv.tol = o_.tol;
    }
    const int64_t n = info.n_vec;
    DBuf xl, rl;
    std::vector<double> theta(kTrainLog, std::nan(""));  // NaN: step not recorded
    if (train) {
      D2_TRY(xl.alloc((size_t)kTrainLog * n));
      D2_TRY(rl.alloc((size_t)kTrainLog * n));
      dv.log_cap = kTrainLog;
      dv.log_x = xl.p;
      dv.log_r = rl.p;
      dv.log_theta = theta.data();
    }
    const int st = dmrg2d_davidson_ground(ops, &dv, x.p, energy, stats, strm_);
    solve_seconds += since(t0);
    if (!train || (st != DMRG2D_OK && st != DMRG2D_ENOCONV)) return st;
    // the recorded steps (the Davidson steps, not the outer loop's), less the last one,
    // which is the converged vector itself
    int logged = 0;
    while (logged < kTrainLog && std::isfinite(theta[logged])) ++logged;
    const auto tt = std::chrono::steady_clock::now();
    D2_TRY(train_mlp(ops, n, xl, rl, theta, logged - 1, x.p));
    train_seconds += since(tt);
    return st;
  }

  // mlp_epochs passes over the recorded steps k < steps: per step one batch of samples at
  // seeded random positions (padding positions of a sector layout carry zero weight and
  // target) and one Adam step.
  int train_mlp(const dmrg2d_ops* ops, int64_t n, const DBuf& xl, const DBuf& rl,
                const std::vector<double>& theta, int steps, const double* xf) {
    if (steps < 1) return DMRG2D_OK;
    DBuf D, f;
    D2_TRY(D.alloc((size_t)n));
    D2_TRY(dmrg2d_diagonal(ops, D.p, strm_));
    D2_TRY(f.alloc((size_t)kTrainBatch * 3));  // X (B x 4), w (B), T (B) as floats
    float* X = (float*)f.p;
    float* w = X + 4 * (size_t)kTrainBatch;
    float* T = w + kTrainBatch;
    std::vector<int64_t> idx(kTrainBatch);
    IBuf d_idx;
    for (int e = 0; e < o_.mlp_epochs; ++e)
      for (int k = 0; k < steps; ++k) {
        for (auto& i : idx) i = (int64_t)(train_rng_.next_u64() % (uint64_t)n);
        D2_TRY(d_idx.upload(idx, strm_));
        D2_TRY(dmrg2d_mlp_make_batch(ops, xl.p + (size_t)k * n, rl.p + (size_t)k * n, theta[k],
                                     xf, D.p, (const int64_t*)d_idx.p, kTrainBatch, X, w, T,
                                     strm_));
        D2_TRY(dmrg2d_mlp_train_step(o_.mlp, X, w, T, kTrainBatch, kTrainLr, nullptr, strm_));
      }
    D2_CUDA(cudaStreamSynchronize(strm_));
    return DMRG2D_OK;
  }
  Block column_block() const {
    Block b;
    const int d = col_.d;
    b.m = d;
    if (hub_) {  // states grouped by (N_up, N_dn) (stable), as sector-restricted blocks need
      std::vector<int> perm(d);
      for (int i = 0; i < d; ++i) perm[i] = i;
      std::stable_sort(perm.begin(), perm.end(), [&](int a, int c) {
        return hc_.nup[a] != hc_.nup[c] ? hc_.nup[a] < hc_.nup[c] : hc_.ndn[a] < hc_.ndn[c];
      });
      auto permuted = [&](const Mat& A) {
        Mat P((size_t)d * d);
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j) P[(size_t)i * d + j] = A[(size_t)perm[i] * d + perm[j]];
        return P;
      };
      b.H = permuted(hc_.H);
      for (const Mat& c : hc_.cd) b.edge.push_back(permuted(c));
      for (int i = 0; i < d; ++i) {
        b.parity.push_back(hc_.parity[(size_t)perm[i]]);
        b.qn.push_back(hc_.nup[(size_t)perm[i]]);
        b.qn.push_back(hc_.ndn[(size_t)perm[i]]);
      }
      return b;
    }
    // with sectors the block's states must be grouped by label: order by N_up (stable)
    std::vector<int> perm(d);
    for (int i = 0; i < d; ++i) perm[i] = i;
    if (o_.use_sectors)
      std::stable_sort(perm.begin(), perm.end(), [](int a, int c) {
        return __builtin_popcount((unsigned)a) < __builtin_popcount((unsigned)c);
      });
    auto permuted = [&](const Mat& A) {
      Mat P((size_t)d * d);
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) P[(size_t)i * d + j] = A[(size_t)perm[i] * d + perm[j]];
      return P;
    };
    b.H = permuted(col_.H);
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      b.edge.push_back(permuted(col_.sz[y]));
      b.edge.push_back(permuted(col_.sp[y]));
    }
    if (o_.use_sectors)
      for (int i = 0; i < d; ++i) b.qn.push_back(__builtin_popcount((unsigned)perm[i]));
    b.Sz_tot = permuted(col_Sz_tot_);
    b.Sp_tot = permuted(col_Sp_tot_);
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

  // Dense superblock: rho = V V^T (grow_left) or V^T V of the dense V = x ((n x other) or
  // (other x n)), its k leading eigenvectors (dsyevdx, selected by index) into U, largest
  // first; *kept = their eigenvalue sum.
  int dmd_dense(const double* x, bool grow_left, int64_t n, int64_t other, int k, DBuf& U,
                double* kept) {
    DBuf rho;
    D2_TRY(rho.alloc((size_t)(n * n)));
    const double one = 1.0, zero = 0.0;
    D2_BLAS(cublasDsyrk(libs_.bl, CUBLAS_FILL_MODE_LOWER, grow_left ? CUBLAS_OP_N : CUBLAS_OP_T,
                        (int)n, (int)other, &one, x, grow_left ? (int)n : (int)other, &zero,
                        rho.p, (int)n));
    DBuf w, work;
    D2_TRY(w.alloc((size_t)n));
    int lwork = 0, meig = 0;
    const int il = (int)n - k + 1, iu = (int)n;  // 1-based eigenvalue indices
    D2_SOLV(cusolverDnDsyevdx_bufferSize(libs_.sv, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                         CUBLAS_FILL_MODE_LOWER, (int)n, rho.p, (int)n, 0.0, 0.0,
                                         il, iu, &meig, w.p, &lwork));
    D2_TRY(work.alloc((size_t)std::max(lwork, 1)));
    IBuf info;
    D2_TRY(info.upload(std::vector<int>{0}, strm_));
    D2_SOLV(cusolverDnDsyevdx(libs_.sv, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                              CUBLAS_FILL_MODE_LOWER, (int)n, rho.p, (int)n, 0.0, 0.0, il, iu,
                              &meig, w.p, work.p, lwork, (int*)info.p));
    int hinfo = 0;
    Mat hw((size_t)k);
    D2_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, strm_));
    D2_CUDA(cudaMemcpyAsync(hw.data(), w.p, k * sizeof(double), cudaMemcpyDeviceToHost, strm_));
    D2_CUDA(cudaStreamSynchronize(strm_));
    if (hinfo != 0 || meig != k)
      return set_error(DMRG2D_ECUDA, "sweep: dsyevdx info %d, %d of %d eigenpairs", hinfo, meig, k);
    *kept = 0.0;
    for (int j = 0; j < k; ++j) *kept += hw[(size_t)j];
    k_take_leading<<<1024, 256, 0, strm_>>>(rho.p, n, k, U.p);
    D2_CUDA(cudaGetLastError());
    return DMRG2D_OK;
  }

  // Labels as one integer ordered like the label, N_up (spins) or N_up * 4096 + N_dn
  // (electrons): of block state i, of column state c, of a target
  int blk_label(const std::vector<int32_t>& qn, int i) const {
    return hub_ ? qn[2 * (size_t)i] * 4096 + qn[2 * (size_t)i + 1] : qn[(size_t)i];
  }
  int col_label(int c) const {
    return hub_ ? hc_.nup[(size_t)c] * 4096 + hc_.ndn[(size_t)c] : __builtin_popcount((unsigned)c);
  }
  // [start, end) of every label among n states labelled qn (equal labels contiguous)
  using Ranges = std::map<int, std::pair<int, int>>;
  int label_ranges(const std::vector<int32_t>& qn, int n, Ranges* out) const {
    out->clear();
    for (int i = 0; i < n;) {
      const int lab = blk_label(qn, i);
      int j = i + 1;
      while (j < n && blk_label(qn, j) == lab) ++j;
      if (out->count(lab)) return set_error(DMRG2D_EINVAL, "sweep: block labels not grouped");
      (*out)[lab] = {i, j};
      i = j;
    }
    return DMRG2D_OK;
  }

  // Label of state e = i_blk + m i_col of a block enlarged by a column, as one integer
  // ordered like the label: N_up (spins), N_up * 4096 + N_dn (electrons)
  int enlarged_label(const Block& B, int64_t e) const {
    const int a = (int)(e % B.m), c = (int)(e / B.m);
    if (!hub_) return B.qn[(size_t)a] + __builtin_popcount((unsigned)c);
    return (B.qn[2 * (size_t)a] + hc_.nup[(size_t)c]) * 4096 + B.qn[2 * (size_t)a + 1] +
           hc_.ndn[(size_t)c];
  }

  // Sector-restricted superblock: the density matrix is block diagonal in the growing
  // half's label.  Left: for each V_q, rho_q = G G^T with G its rows without padding;
  // right: rho_q = V_q^T V_q.  All eigenpairs of every rho_q, the k largest eigenvalues
  // over all sectors are kept; the new block's states are grouped by label (ascending)
  // and, within a label, by decreasing weight.  U (n x k, zero outside each state's
  // sector) gets the eigenvectors at their dense indices i1 + m1 i2 (or i4 + m4 i3).
  int dmd_sectors(const double* xpk, bool grow_left, const Block& Lb, const Block& Rb,
                  const std::vector<long long>& qbase, const std::vector<int>& qld,
                  const std::vector<int>& qcols, const std::vector<int64_t>& rowL,
                  const std::vector<int64_t>& colR, int* kio, DBuf& U, double* kept,
                  std::vector<int32_t>* labels) {
    const int nQ = (int)qld.size();
    const double one = 1.0, zero = 0.0;
    std::vector<std::shared_ptr<DBuf>> vecs(nQ);
    std::vector<std::shared_ptr<IBuf>> idx(nQ);
    std::vector<int> dim(nQ), lab(nQ);
    struct Cand {
      double w;
      int q, j;
    };
    std::vector<Cand> cand;
    // host side first (index lists, uploads on the sweep's stream, every buffer), so that
    // no allocation or free falls between the launches of the side streams
    std::vector<std::shared_ptr<IBuf>> d_rows(nQ);
    std::vector<std::shared_ptr<DBuf>> G(nQ), work(nQ);
    std::vector<int> top(nQ), lwork(nQ), meig(nQ), all(nQ);
    std::vector<int64_t> woff(nQ + 1, 0);
    int64_t r0 = 0, c0 = 0;
    for (int q = 0; q < nQ; ++q) {
      std::vector<int64_t> dense;
      vecs[q] = std::make_shared<DBuf>();
      if (grow_left) {
        std::vector<int> rows;
        for (int r = 0; r < qld[q]; ++r)
          if (rowL[r0 + r] >= 0) {
            rows.push_back(r);
            dense.push_back(rowL[r0 + r]);
          }
        dim[q] = (int)rows.size();
        d_rows[q] = std::make_shared<IBuf>();
        D2_TRY(d_rows[q]->upload(rows, strm_));
        G[q] = std::make_shared<DBuf>();
        D2_TRY(G[q]->alloc((size_t)dim[q] * qcols[q]));
        lab[q] = enlarged_label(Lb, dense[0]);  // of the enlarged-left state i1 + m1 i2
      } else {
        for (int c = 0; c < qcols[q]; ++c) dense.push_back(colR[c0 + c]);
        dim[q] = qcols[q];
        lab[q] = enlarged_label(Rb, dense[0]);  // of the enlarged-right state i4 + m4 i3
      }
      D2_TRY(vecs[q]->alloc((size_t)dim[q] * dim[q]));
      idx[q] = std::make_shared<IBuf>();
      D2_TRY(idx[q]->upload(dense, strm_));
      // at most *kio states are kept from any one sector: its *kio largest eigenpairs
      // (dsyevd for the whole spectrum, dsyevdx selected by index otherwise)
      const int n = dim[q], k = q % kSide;
      top[q] = std::min(n, *kio);
      all[q] = top[q] >= n;
      meig[q] = top[q];
      if (all[q])
        D2_SOLV(cusolverDnDsyevd_bufferSize(libs_.ssv[k], CUSOLVER_EIG_MODE_VECTOR,
                                            CUBLAS_FILL_MODE_LOWER, n, vecs[q]->p, n,
                                            vecs[q]->p, &lwork[q]));
      else
        D2_SOLV(cusolverDnDsyevdx_bufferSize(
            libs_.ssv[k], CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, n,
            vecs[q]->p, n, 0.0, 0.0, n - top[q] + 1, n, &meig[q], vecs[q]->p, &lwork[q]));
      work[q] = std::make_shared<DBuf>();
      D2_TRY(work[q]->alloc((size_t)std::max(lwork[q], 1)));
      woff[q + 1] = woff[q] + n;
      r0 += qld[q];
      c0 += qcols[q];
    }
    DBuf w_all;
    IBuf info_all;
    D2_TRY(w_all.alloc((size_t)std::max<int64_t>(woff[nQ], 1)));
    D2_TRY(info_all.upload(std::vector<int>((size_t)nQ, 0), strm_));
    // the sectors' density matrices and eigenpairs on the side streams, after the sweep's
    // stream has produced the ground state and the uploads above
    D2_CUDA(cudaEventRecord(libs_.ev_main, strm_));
    for (int k = 0; k < kSide; ++k) D2_CUDA(cudaStreamWaitEvent(libs_.side[k], libs_.ev_main, 0));
    r0 = 0;
    for (int q = 0; q < nQ; ++q) {
      const int k = q % kSide, n = dim[q];
      const double* xq = xpk + qbase[q];
      if (grow_left) {
        k_gather_rows<<<512, 256, 0, libs_.side[k]>>>(xq, qld[q], qcols[q],
                                                      (const int*)d_rows[q]->p, n, G[q]->p);
        D2_CUDA(cudaGetLastError());
        D2_BLAS(cublasDsyrk(libs_.sbl[k], CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, n, qcols[q], &one,
                            G[q]->p, n, &zero, vecs[q]->p, n));
      } else {
        D2_BLAS(cublasDsyrk(libs_.sbl[k], CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, n, qld[q], &one,
                            xq, qld[q], &zero, vecs[q]->p, n));
      }
      int* info = (int*)info_all.p + q;
      if (all[q])
        D2_SOLV(cusolverDnDsyevd(libs_.ssv[k], CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                 vecs[q]->p, n, w_all.p + woff[q], work[q]->p, lwork[q], info));
      else
        D2_SOLV(cusolverDnDsyevdx(libs_.ssv[k], CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                  CUBLAS_FILL_MODE_LOWER, n, vecs[q]->p, n, 0.0, 0.0,
                                  n - top[q] + 1, n, &meig[q], w_all.p + woff[q], work[q]->p,
                                  lwork[q], info));
    }
    for (int k = 0; k < kSide; ++k) {
      D2_CUDA(cudaEventRecord(libs_.ev_side[k], libs_.side[k]));
      D2_CUDA(cudaStreamWaitEvent(strm_, libs_.ev_side[k], 0));
    }
    Mat w_host((size_t)std::max<int64_t>(woff[nQ], 1));
    std::vector<int> info_host((size_t)nQ, 0);
    D2_CUDA(cudaStreamSynchronize(strm_));
    D2_CUDA(cudaMemcpy(w_host.data(), w_all.p, sizeof(double) * woff[nQ], cudaMemcpyDeviceToHost));
    D2_CUDA(cudaMemcpy(info_host.data(), info_all.p, sizeof(int) * nQ, cudaMemcpyDeviceToHost));
    for (int q = 0; q < nQ; ++q) {
      if (info_host[(size_t)q] != 0 || (!all[q] && meig[q] != top[q]))
        return set_error(DMRG2D_ECUDA, "sweep: dsyevd(x) info %d, %d of %d eigenpairs",
                         info_host[(size_t)q], meig[q], top[q]);
      const int got = all[q] ? dim[q] : top[q];
      for (int j = 0; j < got; ++j) cand.push_back({w_host[(size_t)(woff[q] + j)], q, j});
    }
    // Labels of the enlarged block that no V_q holds (the superblock's target leaves them
    // empty, as the smaller superblocks of the warm-up do for labels only the full filling
    // reaches): the density matrix is zero there, and their states are candidates of
    // weight 0 (unit vectors), kept while m allows, so that later superblocks find them.
    const Block& B = grow_left ? Lb : Rb;
    const int64_t n = (int64_t)B.m * col_.d;
    std::map<int, int> lab_q;  // label -> q
    for (int q = 0; q < nQ; ++q) lab_q[lab[q]] = q;
    std::map<int, std::vector<int64_t>> unreached;  // label -> its states (dense index)
    for (int64_t e = 0; e < n; ++e) {
      const int le = enlarged_label(B, e);
      if (!lab_q.count(le)) unreached[le].push_back(e);
    }
    std::vector<int64_t> unit_idx;  // Cand with q < 0: unit vector at unit_idx[-q-1]
    std::vector<int> unit_lab;
    {  // candidates in label order (ties in weight keep the lower label, then the order)
      std::vector<int> all_labels;
      for (auto& kv : lab_q) all_labels.push_back(kv.first);
      for (auto& kv : unreached) all_labels.push_back(kv.first);
      std::sort(all_labels.begin(), all_labels.end());
      std::vector<Cand> ordered;
      for (int le : all_labels) {
        auto it = lab_q.find(le);
        if (it != lab_q.end()) {
          for (const Cand& c : cand)
            if (c.q == it->second) ordered.push_back(c);
        } else {
          for (int64_t e : unreached[le]) {
            unit_idx.push_back(e);
            unit_lab.push_back(le);
            ordered.push_back({0.0, -(int)unit_idx.size(), 0});
          }
        }
      }
      cand.swap(ordered);
    }
    auto cand_label = [&](const Cand& c) { return c.q >= 0 ? lab[c.q] : unit_lab[-c.q - 1]; };
    std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.w > b.w; });
    const int k = std::min(*kio, (int)cand.size());
    *kio = k;
    std::vector<Cand> keep(cand.begin(), cand.begin() + k);
    std::stable_sort(keep.begin(), keep.end(), [&](const Cand& a, const Cand& b) {
      return cand_label(a) < cand_label(b);  // group by label; stable keeps decreasing weight
    });
    D2_TRY(U.alloc((size_t)(n * k)));
    D2_CUDA(cudaMemsetAsync(U.p, 0, (size_t)n * k * sizeof(double), strm_));
    *kept = 0.0;
    labels->clear();
    std::vector<int64_t> ones;  // flat positions (row + n col) of the unit vectors' 1s
    for (int c = 0; c < k; ++c) {
      const Cand& cd = keep[(size_t)c];
      if (cd.q >= 0) {
        k_scatter_col<<<64, 256, 0, strm_>>>(vecs[cd.q]->p, dim[cd.q], cd.j, dim[cd.q],
                                             (const int64_t*)idx[cd.q]->p, U.p, n, c);
        *kept += cd.w;
      } else {
        ones.push_back(unit_idx[(size_t)(-cd.q - 1)] + n * c);
      }
      labels->push_back(cand_label(cd));
    }
    D2_CUDA(cudaGetLastError());
    if (!ones.empty()) {
      IBuf d_ones;
      D2_TRY(d_ones.upload(ones, strm_));
      k_set_ones<<<64, 256, 0, strm_>>>(U.p, (const int64_t*)d_ones.p, (int)ones.size());
      D2_CUDA(cudaGetLastError());
      D2_CUDA(cudaStreamSynchronize(strm_));  // d_ones is freed on return
    }
    return DMRG2D_OK;
  }

  // ---- observables of the dense V (nL = m1 d rows i1 + m1 i2, nR = d m4 columns
  // i4 + m4 i3) -------------------------------------------------------------------------
  // out = alpha V (op(X) (x) 1_m4)^T + beta out: X acts on i3 (column 3); op(X) = X^T if tX
  int col3(const double* X, bool tX, const double* V, double* out, int64_t nL, int m4,
           double alpha, double beta) {
    const int d = col_.d;
    D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_N, tX ? CUBLAS_OP_T : CUBLAS_OP_N, (int)(nL * m4), d, d,
                        &alpha, V, (int)(nL * m4), X, d, &beta, out, (int)(nL * m4)));
    return DMRG2D_OK;
  }
  // out = alpha V (1_d (x) Y)^T + beta out: Y (row-major m4 x m4) acts on i4 (block 4)
  int blk4(const double* Y, const double* V, double* out, int64_t nL, int m4, double alpha,
           double beta) {
    D2_BLAS(cublasDgemmStridedBatched(libs_.bl, CUBLAS_OP_N, CUBLAS_OP_N, (int)nL, m4, m4, &alpha,
                                      V, (int)nL, (long long)nL * m4, Y, m4, 0, &beta, out, (int)nL,
                                      (long long)nL * m4, col_.d));
    return DMRG2D_OK;
  }
  int dotv(const double* a, const double* b, int64_t n, double* r) {
    D2_BLAS(cublasDdot(libs_.bl, (int)n, a, 1, b, 1, r));
    return DMRG2D_OK;
  }
  // <S_(2,y) . S_(3,y)> (leg bonds between the central columns), <S_(2,y) . S_(2,y+1)>
  // (rung bonds of column 2) and, when with_s2, <S_tot^2> = |S+ x|^2 + |Sz x|^2 + <Sz>.
  int observables(const double* V, const Block& Lb, const Block& Rb, bool with_s2,
                  std::vector<double>* leg, std::vector<double>* rung, double* s2,
                  bool bonds = true) {
    const int m1 = Lb.m, m4 = Rb.m, d = col_.d, nl = (int)col_.sz.size();
    const int64_t nL = (int64_t)m1 * d, nR = (int64_t)d * m4, nd = nL * nR;
    // two work vectors of the dense V's size, kept across steps (the largest so far)
    if (obs_T_.n < (size_t)nd) D2_TRY(obs_T_.alloc((size_t)nd));
    if (obs_T2_.n < (size_t)nd) D2_TRY(obs_T2_.alloc((size_t)nd));
    DBuf &T = obs_T_, &T2 = obs_T2_;
    if (bonds) {
      leg->assign(nl, 0.0);
      rung->assign(std::max(nl - 1, 0), 0.0);
    }
    for (int y = 0; bonds && y < nl; ++y) {
      // (A (x) 1) V (B (x) 1)^T for (A, B) = (Sz, Sz), (S+, S-), (S-, S+) with weights 1, 1/2, 1/2
      const double* sz = dsz_[y].p;
      const double* sp = dsp_[y].p;
      struct P { const double* a; bool ta; const double* b; bool tb; double c; };
      const P terms[3] = {{sz, false, sz, false, 1.0}, {sp, false, sp, true, 0.5},
                          {sp, true, sp, false, 0.5}};
      for (const P& t : terms) {
        D2_TRY(kron_col(t.a, t.ta, V, T.p, m1, (int)nR, 1.0, 0.0));
        D2_TRY(col3(t.b, t.tb, T.p, T2.p, nL, m4, 1.0, 0.0));
        double r = 0.0;
        D2_TRY(dotv(V, T2.p, nd, &r));
        (*leg)[y] += t.c * r;
      }
    }
    for (int y = 0; bonds && y + 1 < nl; ++y) {
      D2_TRY(kron_col(drung_[y].p, false, V, T.p, m1, (int)nR, 1.0, 0.0));
      D2_TRY(dotv(V, T.p, nd, &(*rung)[y]));
    }
    *s2 = std::nan("");
    if (with_s2) {
      DBuf b1z, b1p, b4z, b4p;
      D2_TRY(b1z.upload(Lb.Sz_tot, strm_));
      D2_TRY(b1p.upload(Lb.Sp_tot, strm_));
      D2_TRY(b4z.upload(Rb.Sz_tot, strm_));
      D2_TRY(b4p.upload(Rb.Sp_tot, strm_));
      double a = 0.0, b = 0.0, c = 0.0;
      for (int pass = 0; pass < 2; ++pass) {  // 0: S^+_tot x, 1: S^z_tot x
        const double* cb = pass ? dSz_tot_.p : dSp_tot_.p;
        D2_TRY(kron_blk(pass ? b1z.p : b1p.p, false, V, T.p, m1, (int)nR));
        D2_TRY(kron_col(cb, false, V, T.p, m1, (int)nR, 1.0, 1.0));
        D2_TRY(col3(cb, false, V, T.p, nL, m4, 1.0, 1.0));
        D2_TRY(blk4(pass ? b4z.p : b4p.p, V, T.p, nL, m4, 1.0, 1.0));  // V (1 (x) Y4)^T
        double r = 0.0;
        D2_TRY(dotv(T.p, T.p, nd, &r));
        if (pass == 0) {
          a = r;
        } else {
          b = r;
          D2_TRY(dotv(V, T.p, nd, &c));
        }
      }
      *s2 = a + b + c;
    }
    return DMRG2D_OK;
  }

  // The bond energies of observables() on the packed ground state of the last step.  A
  // column operator A on i2 (and B on i3) moves the row segment (i2, block-1 sector a) of
  // V_qL to (i2', a) of V_qL' and the column segment (i3, block-4 sector b) to (i3', b):
  // <x|(A (x) B)|x> is a sum of coef * <sub-block, sub-block> over those segment pairs,
  // coef = A[i2'][i2] B[i3'][i3] (B = 1 for the rung bonds of column 2).
  int bonds_sectors(int m1, int m4, std::vector<double>* leg, std::vector<double>* rung) {
    const LastSectors& ls = last_sec_;
    const int d = col_.d, nl = (int)col_.sz.size(), nQ = (int)ls.qld.size();
    struct Seg {
      int q, off, len;
    };
    std::map<std::pair<int, int>, Seg> rseg;                 // (i2, first i1) -> row segment
    std::map<std::tuple<int, int, int>, std::pair<int, int>> cseg;  // (q, i3, first i4)
    std::vector<std::vector<std::array<int, 4>>> qcols(nQ);  // per q: (i3, i4, off, len)
    std::vector<std::vector<std::array<int, 4>>> qrows(nQ);  // per q: (i2, i1, off, len)
    int64_t r0 = 0, c0 = 0;
    for (int q = 0; q < nQ; ++q) {
      for (int r = 0; r < ls.qld[q];) {
        const int64_t e = ls.rowL[r0 + r];
        if (e < 0) {
          ++r;
          continue;
        }
        const int i2 = (int)(e / m1), i1 = (int)(e % m1);
        int len = 1;
        while (r + len < ls.qld[q] && ls.rowL[r0 + r + len] == e + len &&
               (e + len) / m1 == i2)
          ++len;
        rseg[{i2, i1}] = {q, r, len};
        qrows[q].push_back({i2, i1, r, len});
        r += len;
      }
      for (int c = 0; c < ls.qcols[q];) {
        const int64_t e = ls.colR[c0 + c];
        const int i3 = (int)(e / m4), i4 = (int)(e % m4);
        int len = 1;
        while (c + len < ls.qcols[q] && ls.colR[c0 + c + len] == e + len &&
               (e + len) / m4 == i3)
          ++len;
        cseg[std::make_tuple(q, i3, i4)] = {c, len};
        qcols[q].push_back({i3, i4, c, len});
        c += len;
      }
      r0 += ls.qld[q];
      c0 += ls.qcols[q];
    }
    std::vector<DotItem> items;
    std::vector<size_t> first;  // item range of each output: legs, then rungs
    // A[i2'][i2] of a row-major d x d operator, transposed when t
    auto el = [d](const Mat& X, bool t, int r, int c) {
      return t ? X[(size_t)c * d + r] : X[(size_t)r * d + c];
    };
    auto add = [&](const Mat& A, bool ta, const Mat* B, bool tb, double coef) {
      for (int q = 0; q < nQ; ++q)
        for (const auto& rs : qrows[q])
          for (int i2p = 0; i2p < d; ++i2p) {
            const double a = el(A, ta, i2p, rs[0]);
            if (a == 0.0) continue;
            auto pr = rseg.find({i2p, rs[1]});
            if (pr == rseg.end() || pr->second.len != rs[3]) continue;
            const int qp = pr->second.q;
            for (const auto& cs : qcols[q])
              for (int i3p = 0; i3p < d; ++i3p) {
                const double b = B ? el(*B, tb, i3p, cs[0]) : (i3p == cs[0] ? 1.0 : 0.0);
                if (b == 0.0) continue;
                auto pc = cseg.find(std::make_tuple(qp, i3p, cs[1]));
                if (pc == cseg.end() || pc->second.second != cs[3]) continue;
                DotItem t;
                t.off1 = ls.qbase[qp] + pr->second.off + (long long)ls.qld[qp] * pc->second.first;
                t.ld1 = ls.qld[qp];
                t.off2 = ls.qbase[q] + rs[2] + (long long)ls.qld[q] * cs[2];
                t.ld2 = ls.qld[q];
                t.rows = rs[3];
                t.cols = cs[3];
                t.coef = coef * a * b;
                items.push_back(t);
              }
          }
    };
    for (int y = 0; y < nl; ++y) {
      first.push_back(items.size());
      add(col_.sz[y], false, &col_.sz[y], false, 1.0);
      add(col_.sp[y], false, &col_.sp[y], true, 0.5);
      add(col_.sp[y], true, &col_.sp[y], false, 0.5);
    }
    for (int y = 0; y + 1 < nl; ++y) {
      first.push_back(items.size());
      add(rung_h_[(size_t)y], false, nullptr, false, 1.0);
    }
    first.push_back(items.size());
    leg->assign(nl, 0.0);
    rung->assign(std::max(nl - 1, 0), 0.0);
    if (items.empty()) return DMRG2D_OK;
    IBuf d_items;
    DBuf d_out;
    {
      std::vector<int64_t> raw(items.size() * sizeof(DotItem) / sizeof(int64_t));
      std::memcpy(raw.data(), items.data(), items.size() * sizeof(DotItem));
      D2_TRY(d_items.upload(raw, strm_));
    }
    D2_TRY(d_out.alloc(items.size()));
    const int grid = (int)std::min<size_t>(items.size(), 152 * 8);
    k_item_dots<<<grid, 256, 0, strm_>>>(ls.x->p, (const DotItem*)d_items.p, (int)items.size(),
                                         d_out.p);
    D2_CUDA(cudaGetLastError());
    Mat vals(items.size());
    D2_CUDA(cudaMemcpyAsync(vals.data(), d_out.p, items.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, strm_));
    D2_CUDA(cudaStreamSynchronize(strm_));
    for (size_t o = 0; o + 1 < first.size(); ++o) {
      double v = 0.0;
      for (size_t i = first[o]; i < first[o + 1]; ++i) v += vals[i];
      if ((int)o < nl)
        (*leg)[o] = v;
      else
        (*rung)[o - nl] = v;
    }
    return DMRG2D_OK;
  }

  // One DMRG step on block 1 = L, block 4 = R; grows L (grow_left) or R into *out.
  int step(const Block& Lb, const Block& Rb, bool grow_left, int m_keep, int l, int sweep,
           Block* out, const DBuf* guess, Block* out_other = nullptr) {
    // ---- HMED: superblock ground state -------------------------------------------------
    std::vector<const double*> le, re;
    for (auto& e : Lb.edge) le.push_back(e.data());
    for (auto& e : Rb.edge) re.push_back(e.data());
    const bool sec = o_.use_sectors != 0;
    dmrg2d_block bl{Lb.m, Lb.H.data(), (int)le.size(), le.data(),
                    hub_ ? Lb.parity.data() : nullptr, sec ? Lb.qn.data() : nullptr};
    dmrg2d_block br{Rb.m, Rb.H.data(), (int)re.size(), re.data(),
                    hub_ ? Rb.parity.data() : nullptr, sec ? Rb.qn.data() : nullptr};
    // spins: S^z_tot = 0 (half the superblock's sites up); electrons: the ladder's filling
    // (N_up, N_dn), on a superblock of fewer columns (warm-up) the same filling rounded
    // half up: floor(N cols / L + 1/2)
    const int cols = Lb.cols + Rb.cols + 2;
    int32_t target[2] = {M_.n_legs * cols / 2, 0};
    if (hub_) {
      target[0] = (int32_t)std::floor((double)o_.n_up * cols / o_.n_columns + 0.5);
      target[1] = (int32_t)std::floor((double)o_.n_dn * cols / o_.n_columns + 0.5);
    }
    dmrg2d_ops* ops = nullptr;
    auto tb = std::chrono::steady_clock::now();
    D2_TRY(dmrg2d_build_ops(&M_, &bl, &br, sec ? target : nullptr, &ops, strm_));
    build_seconds += since(tb);
    struct FreeOps {
      dmrg2d_ops* p;
      ~FreeOps() { dmrg2d_free_ops(p); }
    } fo{ops};
    dmrg2d_ops_info info;
    D2_TRY(dmrg2d_ops_get_info(ops, &info));
    const int64_t nv = info.n_vec;
    const int d = col_.d;
    const int64_t nL = (int64_t)Lb.m * d, nR = (int64_t)d * Rb.m, nd = nL * nR;  // dense V
    // sector layout of the packed vector (rows/columns of each V_q in the dense V)
    std::vector<long long> qbase;
    std::vector<int> qld, qcols;
    std::vector<int64_t> rowL, colR;
    auto d_rowL = std::make_shared<IBuf>(), d_colR = std::make_shared<IBuf>();
    if (sec) {
      D2_TRY(sec_layout(ops, qbase, qld, qcols, rowL, colR));
      D2_TRY(d_rowL->upload(rowL, strm_));
      D2_TRY(d_colR->upload(colR, strm_));
    }
    auto pack = [&](double* Vd, double* xpk, int to_packed) -> int {
      int64_t r0 = 0, c0 = 0;
      for (size_t q = 0; q < qld.size(); ++q) {
        k_pack<<<512, 256, 0, strm_>>>(Vd, nL, xpk + qbase[q], qld[q], qcols[q],
                                       (const int64_t*)d_rowL->p + r0,
                                       (const int64_t*)d_colR->p + c0, to_packed);
        r0 += qld[q];
        c0 += qcols[q];
      }
      D2_CUDA(cudaGetLastError());
      return DMRG2D_OK;
    };
    auto xs = std::make_shared<DBuf>();
    DBuf& x = *xs;
    if (guess && guess->n == (size_t)nd) {  // the previous ground state, in this basis
      D2_TRY(x.alloc((size_t)nv));
      if (sec)
        D2_TRY(pack(guess->p, x.p, 1));
      else
        D2_CUDA(cudaMemcpyAsync(x.p, guess->p, nv * sizeof(double), cudaMemcpyDeviceToDevice,
                                strm_));
    } else {
      Mat x0((size_t)nv);
      for (auto& v : x0) v = rng_.next();
      if (sec) {  // zero on the padding rows
        int64_t r0 = 0;
        for (size_t q = 0; q < qld.size(); ++q) {
          for (int c = 0; c < qcols[q]; ++c)
            for (int r = 0; r < qld[q]; ++r)
              if (rowL[r0 + r] < 0) x0[(size_t)(qbase[q] + r + (int64_t)qld[q] * c)] = 0.0;
          r0 += qld[q];
        }
      }
      D2_TRY(x.upload(x0, strm_));
    }
    double energy = 0.0;
    dmrg2d_solver_stats stats{};
    const int st = solve(ops, info, x, sweep, &energy, &stats);
    if (st != DMRG2D_OK && st != DMRG2D_ENOCONV) return st;
    const auto td = std::chrono::steady_clock::now();
    // the ground state as the dense V ((m1 d) x (d m4)) for the next step's start vector
    auto xd = std::make_shared<DBuf>();
    D2_TRY(xd->alloc((size_t)nd));
    if (sec) {
      D2_CUDA(cudaMemsetAsync(xd->p, 0, nd * sizeof(double), strm_));
      D2_TRY(pack(xd->p, x.p, 0));
    } else {
      D2_CUDA(cudaMemcpyAsync(xd->p, x.p, nd * sizeof(double), cudaMemcpyDeviceToDevice, strm_));
    }
    last_x_ = xd;
    last_nv_ = nd;
    last_sec_.valid = sec;
    if (sec) {
      last_sec_.m1 = Lb.m;
      last_sec_.m4 = Rb.m;
      last_sec_.target = hub_ ? target[0] * 4096 + target[1] : target[0];
      last_sec_.x = xs;
      last_sec_.qbase = qbase;
      last_sec_.qld = qld;
      last_sec_.qcols = qcols;
      last_sec_.qlab.assign(qld.size(), 0);
      int64_t r0 = 0;
      for (size_t q = 0; q < qld.size(); ++q) {
        int r = 0;
        while (r < qld[q] && rowL[r0 + r] < 0) ++r;
        if (r == qld[q]) return set_error(DMRG2D_EINVAL, "sweep: empty sector matrix");
        last_sec_.qlab[q] = enlarged_label(Lb, rowL[r0 + r]);
        r0 += qld[q];
      }
      last_sec_.d_rowL = d_rowL;
      last_sec_.d_colR = d_colR;
      last_sec_.rowL = rowL;
      last_sec_.colR = colR;
    }
    double norm2 = 0.0;  // trace of rho = |x|^2
    D2_BLAS(cublasDdot(libs_.bl, (int)nv, x.p, 1, x.p, 1, &norm2));
    // ---- DMF + DMD: k leading eigenvectors of the growing half's density matrix ----------
    const SecLayout lay{sec, nd, &qbase, &qld, &qcols, &rowL, &colR};
    Grown g;
    D2_TRY(dmd(grow_left, Lb, Rb, m_keep, x.p, norm2, lay, &g));
    dm_seconds += since(td);
    // observables of this step's ground state (<S_tot^2> only where no block is grown:
    // the last step of each sweep)
    const auto to = std::chrono::steady_clock::now();
    std::vector<double> leg, rung, dens;
    double s2 = std::nan("");
    if (hub_) {  // site densities of the central columns (normalised by the call)
      DBuf dd;
      D2_TRY(dd.alloc((size_t)(8 * M_.n_legs + 2)));
      D2_TRY(dmrg2d_site_densities(ops, x.p, dd.p, strm_));
      dens.resize(dd.n);
      D2_CUDA(cudaMemcpyAsync(dens.data(), dd.p, dd.n * sizeof(double), cudaMemcpyDeviceToHost,
                              strm_));
      D2_CUDA(cudaStreamSynchronize(strm_));
    } else {
      if (sec) {  // bond energies on the packed state; <S_tot^2> on the dense V
        D2_TRY(bonds_sectors(Lb.m, Rb.m, &leg, &rung));
        if (out == nullptr) D2_TRY(observables(xd->p, Lb, Rb, true, &leg, &rung, &s2, false));
      } else {
        D2_TRY(observables(xd->p, Lb, Rb, out == nullptr, &leg, &rung, &s2));
      }
      for (double& v : leg) v /= norm2;
      for (double& v : rung) v /= norm2;
      s2 /= norm2;
    }
    obs_seconds += since(to);
    record(energy, 1.0 - g.kept, l, sweep, stats.iters, leg, rung, s2, dens);
    if (!out) return DMRG2D_OK;
    D2_TRY(renorm(grow_left, Lb, Rb, g, out));
    if (out_other) {  // the other half from the same ground state (Hubbard warm-up)
      const auto t2 = std::chrono::steady_clock::now();
      Grown g2;
      D2_TRY(dmd(!grow_left, Lb, Rb, m_keep, x.p, norm2, lay, &g2));
      dm_seconds += since(t2);
      D2_TRY(renorm(!grow_left, Lb, Rb, g2, out_other));
    }
    return DMRG2D_OK;
  }

  // The sector layout of a superblock vector (empty for a dense superblock), as dmd needs it.
  struct SecLayout {
    bool sec;
    int64_t nd;  // elements of the dense V
    const std::vector<long long>* qbase;
    const std::vector<int>* qld;
    const std::vector<int>* qcols;
    const std::vector<int64_t>* rowL;
    const std::vector<int64_t>* colR;
  };
  // What DMD hands to the renormalisation: U (n x k, n = mb d), the kept states' labels
  // (sectors) and the kept weight (divided by |x|^2).
  struct Grown {
    std::shared_ptr<DBuf> U;
    std::vector<int32_t> labels;
    int k = 0, mb = 0;
    int64_t n = 0;
    double kept = 0.0;
  };

  // DMF + DMD of the half that grows (grow_left: block 1 + column 2), from the ground state
  // x of the superblock of Lb and Rb (packed if lay.sec).
  int dmd(bool grow_left, const Block& Lb, const Block& Rb, int m_keep, const double* x,
          double norm2, const SecLayout& lay, Grown* g) {
    const int d = col_.d;
    g->mb = grow_left ? Lb.m : Rb.m;  // block that grows
    g->n = (int64_t)g->mb * d;
    int k = (int)std::min<int64_t>(m_keep, g->n);
    g->U = std::make_shared<DBuf>();
    double kept = 0.0;
    if (lay.sec) {
      D2_TRY(dmd_sectors(x, grow_left, Lb, Rb, *lay.qbase, *lay.qld, *lay.qcols, *lay.rowL,
                         *lay.colR, &k, *g->U, &kept, &g->labels));
    } else {
      D2_TRY(g->U->alloc((size_t)(g->n * k)));
      D2_TRY(dmd_dense(x, grow_left, g->n, lay.nd / g->n, k, *g->U, &kept));
    }
    g->k = k;
    g->kept = kept / norm2;
    return DMRG2D_OK;
  }

  // Renormalisation: the new block U^T O U from the block B that grew (Lb if grow_left).
  int renorm(bool grow_left, const Block& Lb, const Block& Rb, Grown& g, Block* out) {
    auto Up = g.U;
    DBuf& U = *Up;
    const int mb = g.mb, k = g.k;
    const int64_t n = g.n;
    const std::vector<int32_t>& labels = g.labels;
    const auto tr = std::chrono::steady_clock::now();
    const Block& B = grow_left ? Lb : Rb;
    DBuf dHB;
    D2_TRY(dHB.upload(B.H, strm_));
    if (hub_) {
      D2_TRY(renormalize_hubbard(B, grow_left, U, dHB, mb, n, k, labels, out));
      out->U = Up;
      renorm_seconds += since(tr);
      return DMRG2D_OK;
    }
    if (o_.use_sectors) {
      D2_TRY(renorm_sectors(grow_left ? Lb : Rb, U, dHB, g, out));
      out->m_prev = mb;
      out->U = Up;
      out->cols = (grow_left ? Lb.cols : Rb.cols) + 1;
      renorm_seconds += since(tr);
      return DMRG2D_OK;
    }
    const double one = 1.0, zero = 0.0;
    DBuf HU, T;
    D2_TRY(HU.alloc((size_t)(n * k)));
    D2_TRY(T.alloc((size_t)(n * k)));
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
    out->cols = (grow_left ? Lb.cols : Rb.cols) + 1;
    out->qn = labels;
    D2_TRY(project(HU.p, &out->H, true));
    out->edge.assign(2 * col_.sz.size(), Mat());
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      D2_TRY(kron_col(dsz_[y].p, false, U.p, T.p, mb, k, 1.0, 0.0));
      D2_TRY(project(T.p, &out->edge[2 * y], false));
      D2_TRY(kron_col(dsp_[y].p, false, U.p, T.p, mb, k, 1.0, 0.0));
      D2_TRY(project(T.p, &out->edge[2 * y + 1], false));
    }
    // total S^z, S^+ of the new block: U^T (1 (x) S_B + S_col (x) 1) U
    for (int pass = 0; pass < 2; ++pass) {
      DBuf dB;
      D2_TRY(dB.upload(pass ? B.Sp_tot : B.Sz_tot, strm_));
      D2_TRY(kron_blk(dB.p, false, U.p, T.p, mb, k));
      D2_TRY(kron_col(pass ? dSp_tot_.p : dSz_tot_.p, false, U.p, T.p, mb, k, 1.0, 1.0));
      D2_TRY(project(T.p, pass ? &out->Sp_tot : &out->Sz_tot, pass == 0));
    }
    renorm_seconds += since(tr);
    return DMRG2D_OK;
  }

  // Renormalisation of a spin block in sectors.  U (n x k) is zero outside each kept
  // state's sector: column j (label q) lives on the rows i + m c with label(i) = q - q(c),
  // a contiguous range of the block's states for every column state c.  A block operator
  // that shifts block labels by dY then maps those rows onto the range of q - q(c) + dY:
  // (1 (x) Y) U is one GEMM per column state and kept label (out zero elsewhere).  A
  // projection U^T (X U) with X shifting labels by dX has only the blocks (q + dX, q),
  // one GEMM each over the n rows.  Same operators and order as the dense renormalisation.
  int kron_blk_sec(const double* Y, bool tY, int dY, const double* W, double* out, int m, int k,
                   const Ranges& rb, const Ranges& rk) {
    const int d = col_.d;
    const int64_t n = (int64_t)m * d;
    const double one = 1.0, zero = 0.0;
    D2_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * n * k, strm_));
    for (int c = 0; c < d; ++c)
      for (const auto& kq : rk) {
        const int a = kq.first - col_label(c);
        auto ia = rb.find(a), ib = rb.find(a + dY);
        if (ia == rb.end() || ib == rb.end()) continue;
        const int s0 = ia->second.first, ms = ia->second.second - s0;
        const int r0 = ib->second.first, mr = ib->second.second - r0;
        const int j0 = kq.second.first, nk = kq.second.second - j0;
        // Y row-major: Y[r][s] is the column-major (s, r) entry
        const double* A = tY ? Y + r0 + (int64_t)m * s0 : Y + s0 + (int64_t)m * r0;
        D2_BLAS(cublasDgemm(libs_.bl, tY ? CUBLAS_OP_N : CUBLAS_OP_T, CUBLAS_OP_N, mr, nk, ms,
                            &one, A, m, W + s0 + (int64_t)m * c + n * j0, (int)n, &zero,
                            out + r0 + (int64_t)m * c + n * j0, (int)n));
      }
    return DMRG2D_OK;
  }
  int project_sec(const double* U, const double* XU, int dX, int64_t n, int k, const Ranges& rk,
                  Mat* dst, bool symmetrise) {
    const double one = 1.0, zero = 0.0;
    DBuf small;
    D2_TRY(small.alloc((size_t)k * k));
    D2_CUDA(cudaMemsetAsync(small.p, 0, sizeof(double) * k * k, strm_));
    for (const auto& kq : rk) {
      auto it = rk.find(kq.first + dX);
      if (it == rk.end()) continue;
      const int j0 = kq.second.first, nj = kq.second.second - j0;
      const int i0 = it->second.first, ni = it->second.second - i0;
      D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_T, CUBLAS_OP_N, ni, nj, (int)n, &one, U + n * i0,
                          (int)n, XU + n * j0, (int)n, &zero, small.p + i0 + (int64_t)k * j0, k));
    }
    Mat hs((size_t)k * k);
    D2_CUDA(cudaMemcpyAsync(hs.data(), small.p, (size_t)k * k * sizeof(double),
                            cudaMemcpyDeviceToHost, strm_));
    D2_CUDA(cudaStreamSynchronize(strm_));
    dst->assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        const double a = hs[(size_t)i + (size_t)j * k];
        (*dst)[(size_t)i * k + j] = symmetrise ? 0.5 * (a + hs[(size_t)j + (size_t)i * k]) : a;
      }
    return DMRG2D_OK;
  }
  int renorm_sectors(const Block& B, DBuf& U, DBuf& dHB, const Grown& g, Block* out) {
    const int mb = g.mb, k = g.k;
    const int64_t n = g.n;
    Ranges rb, rk;
    D2_TRY(label_ranges(B.qn, mb, &rb));
    D2_TRY(label_ranges(g.labels, k, &rk));
    DBuf HU, T;
    D2_TRY(HU.alloc((size_t)(n * k)));
    D2_TRY(T.alloc((size_t)(n * k)));
    // H_enl U as in the dense renormalisation: S+ raises N_up by one, S- lowers it
    D2_TRY(kron_blk_sec(dHB.p, false, 0, U.p, HU.p, mb, k, rb, rk));
    D2_TRY(kron_col(dH_col_.p, false, U.p, HU.p, mb, k, 1.0, 1.0));
    const double J = M_.J_leg;
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      DBuf dz, dp;
      D2_TRY(dz.upload(B.edge[2 * y], strm_));
      D2_TRY(dp.upload(B.edge[2 * y + 1], strm_));
      D2_TRY(kron_blk_sec(dz.p, false, 0, U.p, T.p, mb, k, rb, rk));
      D2_TRY(kron_col(dsz_[y].p, false, T.p, HU.p, mb, k, J, 1.0));
      D2_TRY(kron_blk_sec(dp.p, false, 1, U.p, T.p, mb, k, rb, rk));
      D2_TRY(kron_col(dsp_[y].p, true, T.p, HU.p, mb, k, 0.5 * J, 1.0));
      D2_TRY(kron_blk_sec(dp.p, true, -1, U.p, T.p, mb, k, rb, rk));
      D2_TRY(kron_col(dsp_[y].p, false, T.p, HU.p, mb, k, 0.5 * J, 1.0));
    }
    out->m = k;
    out->qn = g.labels;
    D2_TRY(project_sec(U.p, HU.p, 0, n, k, rk, &out->H, true));
    out->edge.assign(2 * col_.sz.size(), Mat());
    for (size_t y = 0; y < col_.sz.size(); ++y) {
      D2_TRY(kron_col(dsz_[y].p, false, U.p, T.p, mb, k, 1.0, 0.0));
      D2_TRY(project_sec(U.p, T.p, 0, n, k, rk, &out->edge[2 * y], false));
      D2_TRY(kron_col(dsp_[y].p, false, U.p, T.p, mb, k, 1.0, 0.0));
      D2_TRY(project_sec(U.p, T.p, 1, n, k, rk, &out->edge[2 * y + 1], false));
    }
    for (int pass = 0; pass < 2; ++pass) {
      DBuf dB;
      D2_TRY(dB.upload(pass ? B.Sp_tot : B.Sz_tot, strm_));
      D2_TRY(kron_blk_sec(dB.p, false, pass, U.p, T.p, mb, k, rb, rk));
      D2_TRY(kron_col(pass ? dSp_tot_.p : dSz_tot_.p, false, U.p, T.p, mb, k, 1.0, 1.0));
      D2_TRY(project_sec(U.p, T.p, pass, n, k, rk, pass ? &out->Sp_tot : &out->Sz_tot, pass == 0));
    }
    return DMRG2D_OK;
  }

  // dst (row-major k x k) = U^T XU, symmetrised when asked; U, XU: n x k column-major
  int project(const DBuf& U, const double* XU, int64_t n, int k, Mat* dst, bool symmetrise) {
    const double one = 1.0, zero = 0.0;
    DBuf small;
    D2_TRY(small.alloc((size_t)k * k));
    Mat hs((size_t)k * k);
    D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_T, CUBLAS_OP_N, k, k, (int)n, &one, U.p, (int)n, XU,
                        (int)n, &zero, small.p, k));
    D2_CUDA(cudaMemcpyAsync(hs.data(), small.p, (size_t)k * k * sizeof(double),
                            cudaMemcpyDeviceToHost, strm_));
    D2_CUDA(cudaStreamSynchronize(strm_));
    dst->assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        const double a = hs[(size_t)i + (size_t)j * k];
        (*dst)[(size_t)i * k + j] = symmetrise ? 0.5 * (a + hs[(size_t)j + (size_t)i * k]) : a;
      }
    return DMRG2D_OK;
  }

  // Electrons: the new block from the growing block B (mb states) and a column, U (n x k,
  // n = mb d, block index fast).  H_enl = 1 (x) H_B + H_col (x) 1 - t sum_j h_j with the
  // hopping between B's boundary mode j and the column's mode j:
  //   block 1 grows: h_j = c_j (x) E_j + c^dag_j (x) E_j^T, E_j = c^dag_{B,j} P_B, and the
  //                  new boundary operators are c^dag_j (x) P_B (the column's modes come
  //                  after block 1's: their string runs over the whole block);
  //   block 4 grows: h_j = (c^dag_j P) (x) c_{B,j} + (P c_j) (x) c^dag_{B,j}, and the new
  //                  boundary operators are c^dag_j (x) 1 (the column comes first).
  // Labels (N_up * 4096 + N_dn, from the density matrix's sectors) give the new block's
  // (N_up, N_dn) and parity.
  int renormalize_hubbard(const Block& B, bool grow_left, const DBuf& U, const DBuf& dHB, int mb,
                          int64_t n, int k, const std::vector<int32_t>& labels, Block* out) {
    DBuf HU, T, T2;
    D2_TRY(HU.alloc((size_t)(n * k)));
    D2_TRY(T.alloc((size_t)(n * k)));
    D2_TRY(kron_blk(dHB.p, false, U.p, HU.p, mb, k));
    D2_TRY(kron_col(dH_col_.p, false, U.p, HU.p, mb, k, 1.0, 1.0));
    const double t = M_.t;
    const int nm = (int)hc_.cd.size();
    DBuf dPb;
    if (grow_left) {
      Mat Pb((size_t)mb * mb, 0.0);
      for (int i = 0; i < mb; ++i) Pb[(size_t)i * mb + i] = B.parity[(size_t)i];
      D2_TRY(dPb.upload(Pb, strm_));
      D2_TRY(T2.alloc((size_t)(n * k)));
    }
    for (int j = 0; j < nm; ++j) {
      DBuf dE;
      if (grow_left) {
        Mat E = B.edge[(size_t)j];  // c^dag_{B,j} P_B: column c of the matrix times P_B[c]
        for (int r = 0; r < mb; ++r)
          for (int c = 0; c < mb; ++c) E[(size_t)r * mb + c] *= B.parity[(size_t)c];
        D2_TRY(dE.upload(E, strm_));
        D2_TRY(kron_blk(dE.p, false, U.p, T.p, mb, k));                  // (1 (x) E_j) U
        D2_TRY(kron_col(dcd_[j].p, true, T.p, HU.p, mb, k, -t, 1.0));    // c_j (x) E_j
        D2_TRY(kron_blk(dE.p, true, U.p, T.p, mb, k));                   // (1 (x) E_j^T) U
        D2_TRY(kron_col(dcd_[j].p, false, T.p, HU.p, mb, k, -t, 1.0));   // c^dag_j (x) E_j^T
      } else {
        D2_TRY(dE.upload(B.edge[(size_t)j], strm_));                     // c^dag_{B,j}
        D2_TRY(kron_blk(dE.p, true, U.p, T.p, mb, k));                   // (1 (x) c_{B,j}) U
        D2_TRY(kron_col(dcdP_[j].p, false, T.p, HU.p, mb, k, -t, 1.0));  // c^dag_j P
        D2_TRY(kron_blk(dE.p, false, U.p, T.p, mb, k));                  // (1 (x) c^dag_{B,j}) U
        D2_TRY(kron_col(dcdP_[j].p, true, T.p, HU.p, mb, k, -t, 1.0));   // P c_j
      }
    }
    out->m = k;
    out->m_prev = mb;
    out->cols = B.cols + 1;
    D2_TRY(project(U, HU.p, n, k, &out->H, true));
    out->edge.assign((size_t)nm, Mat());
    for (int j = 0; j < nm; ++j) {
      if (grow_left) {
        D2_TRY(kron_blk(dPb.p, false, U.p, T2.p, mb, k));                // (1 (x) P_B) U
        D2_TRY(kron_col(dcd_[j].p, false, T2.p, T.p, mb, k, 1.0, 0.0));  // c^dag_j (x) P_B
      } else {
        D2_TRY(kron_col(dcd_[j].p, false, U.p, T.p, mb, k, 1.0, 0.0));   // c^dag_j (x) 1
      }
      D2_TRY(project(U, T.p, n, k, &out->edge[(size_t)j], false));
    }
    out->qn.clear();
    out->parity.clear();
    for (int32_t lab : labels) {
      const int nu = lab / 4096, nd = lab % 4096;
      out->qn.push_back(nu);
      out->qn.push_back(nd);
      out->parity.push_back((nu + nd) % 2 ? -1.0 : 1.0);
    }
    return DMRG2D_OK;
  }

  void record(double e, double trunc, int l, int sweep, int iters, const std::vector<double>& leg,
              const std::vector<double>& rung, double s2, const std::vector<double>& dens) {
    last_energy_ = e;
    const int i = rep_->n_steps++;
    if (i < rep_->cap) {
      if (rep_->densities && !dens.empty())
        for (size_t j = 0; j < dens.size(); ++j) rep_->densities[(size_t)i * dens.size() + j] = dens[j];
      const int nl = (int)col_.sz.size(), nr = std::max(nl - 1, 1);
      if (rep_->leg_bond)
        for (int y = 0; y < nl; ++y) rep_->leg_bond[(size_t)i * nl + y] = leg[(size_t)y];
      if (rep_->rung_bond)
        for (int y = 0; y < nr; ++y)
          rep_->rung_bond[(size_t)i * nr + y] = y < (int)rung.size() ? rung[(size_t)y] : 0.0;
      if (rep_->s2) rep_->s2[i] = s2;
      if (rep_->iters) rep_->iters[i] = iters;
      if (rep_->energy) rep_->energy[i] = e;
      if (rep_->trunc) rep_->trunc[i] = trunc;
      if (rep_->l) rep_->l[i] = l;
      if (rep_->sweep) rep_->sweep[i] = sweep;
    }
  }

  Mat col_Sz_tot_, col_Sp_tot_;
  DBuf dSz_tot_, dSp_tot_;
  std::vector<DBuf> drung_;
  std::vector<Mat> rung_h_;  // the same rung-bond operators on the host (row-major)
  std::shared_ptr<DBuf> last_x_;  // ground state of the last step's superblock
  int64_t last_nv_ = 0;
  // the last step's sector-restricted ground state: packed vector, its layout (the rows
  // and columns of each V_q in the dense V), the enlarged-left label of each V_q, the
  // target label and the block sizes
  struct LastSectors {
    bool valid = false;
    int m1 = 0, m4 = 0, target = 0;
    std::shared_ptr<DBuf> x;
    std::vector<long long> qbase;
    std::vector<int> qld, qcols, qlab;
    std::vector<int64_t> rowL, colR;
    std::shared_ptr<IBuf> d_rowL, d_colR;
  } last_sec_;

  // Guess for the superblock after moving right: block 1 grew into nl (its U: (m_l d) x k),
  // block 4 = Rs of m_r states (made from a block of m' states plus a column, Rs.U:
  // (m' d) x m_r) splits into that column and that block.  Old V: (m_l d) x (d m_r).
  //   W = U^T V (k x d m_r);  V'[(a + k s3), (b' + m' t)] = sum_b W[a, b + m_r s3] Rs.U[b' + m' t, b]
  int move_right(const Block& nl, const Block& Rs, std::shared_ptr<DBuf>* out) {
    const int d = col_.d, k = nl.m, ml = nl.m_prev, mr = Rs.m, mp = Rs.m_prev;
    const int64_t nL = (int64_t)ml * d, nR = (int64_t)d * mr;
    if (!nl.U || !Rs.U || last_nv_ != nL * nR) return DMRG2D_OK;  // no guess
    if (last_sec_.valid && last_sec_.m1 == ml && last_sec_.m4 == mr)
      return move_right_sectors(nl, Rs, out);
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
    if (last_sec_.valid && last_sec_.m1 == ml && last_sec_.m4 == mr)
      return move_left_sectors(nr, Ls, out);
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

  // The same two transformations on a sector-restricted ground state, label by label.
  // W = U^T V from the packed matrices V_q: the kept states of label qL (a contiguous range
  // of U's columns) see only V_q of that enlarged-left label, W_q = U_q^T V_q with U_q the
  // rows of U at V_q's rows (0 on padding).  Then, per split-off column i3 and label p of
  // block 4 (a contiguous range of its states), the kept states of label
  // target - q(i3) - p take the product with the range's columns of Rs.U.  Everything
  // else of W and of the new V is zero.
  int move_right_sectors(const Block& nl, const Block& Rs, std::shared_ptr<DBuf>* out) {
    const int d = col_.d, k = nl.m, ml = nl.m_prev, mr = Rs.m, mp = Rs.m_prev;
    const int64_t nL = (int64_t)ml * d, nR = (int64_t)d * mr;
    const LastSectors& ls = last_sec_;
    Ranges rk, r4;
    D2_TRY(label_ranges(nl.qn, k, &rk));
    D2_TRY(label_ranges(Rs.qn, mr, &r4));
    const double one = 1.0, zero = 0.0;
    DBuf W, G, Wq;
    D2_TRY(W.alloc((size_t)k * nR));
    D2_CUDA(cudaMemsetAsync(W.p, 0, sizeof(double) * k * nR, strm_));
    size_t gmax = 0, wmax = 0;
    for (size_t q = 0; q < ls.qld.size(); ++q) {
      auto it = rk.find(ls.qlab[q]);
      if (it == rk.end()) continue;
      const size_t kq = it->second.second - it->second.first;
      gmax = std::max(gmax, (size_t)ls.qld[q] * kq);
      wmax = std::max(wmax, kq * ls.qcols[q]);
    }
    D2_TRY(G.alloc(std::max<size_t>(gmax, 1)));
    D2_TRY(Wq.alloc(std::max<size_t>(wmax, 1)));
    int64_t r0 = 0, c0 = 0;
    for (size_t q = 0; q < ls.qld.size(); ++q) {
      const int ld = ls.qld[q], nc = ls.qcols[q];
      auto it = rk.find(ls.qlab[q]);
      if (it != rk.end()) {
        const int j0 = it->second.first, kq = it->second.second - j0;
        k_gather_idx<<<512, 256, 0, strm_>>>(nl.U->p + nL * j0, nL,
                                             (const int64_t*)ls.d_rowL->p + r0, ld, kq, G.p);
        D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_T, CUBLAS_OP_N, kq, nc, ld, &one, G.p, ld,
                            ls.x->p + ls.qbase[q], ld, &zero, Wq.p, kq));
        k_scatter_idx<<<512, 256, 0, strm_>>>(Wq.p, kq, nc, (const int64_t*)ls.d_colR->p + c0, 0,
                                              W.p + j0, k);
        D2_CUDA(cudaGetLastError());
      }
      r0 += ld;
      c0 += nc;
    }
    auto v = std::make_shared<DBuf>();
    const int64_t nv = (int64_t)k * d * d * mp;
    D2_TRY(v->alloc((size_t)nv));
    D2_CUDA(cudaMemsetAsync(v->p, 0, sizeof(double) * nv, strm_));
    for (int i3 = 0; i3 < d; ++i3)
      for (const auto& pr : r4) {
        auto it = rk.find(ls.target - col_label(i3) - pr.first);
        if (it == rk.end()) continue;
        const int b0 = it->second.first, kq = it->second.second - b0;
        const int a0 = pr.second.first, np = pr.second.second - a0;
        D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_N, CUBLAS_OP_T, kq, mp * d, np, &one,
                            W.p + b0 + (int64_t)k * (a0 + (int64_t)mr * i3), k,
                            Rs.U->p + (int64_t)mp * d * a0, mp * d, &zero,
                            v->p + b0 + (int64_t)k * i3, k * d));
      }
    *out = v;
    return DMRG2D_OK;
  }
  // W = V U from the packed matrices: the kept states of label target - qL see only V_q,
  // W_q = V_q U_q with U_q the rows of U at V_q's columns; per split-off column s2 and
  // label p of block 1, the kept states of label target - p - q(s2) take Ls.U's range.
  int move_left_sectors(const Block& nr, const Block& Ls, std::shared_ptr<DBuf>* out) {
    const int d = col_.d, k = nr.m, mr = nr.m_prev, ml = Ls.m, mp = Ls.m_prev;
    const int64_t nL = (int64_t)ml * d, nR = (int64_t)d * mr;
    const LastSectors& ls = last_sec_;
    Ranges rk, r1;
    D2_TRY(label_ranges(nr.qn, k, &rk));
    D2_TRY(label_ranges(Ls.qn, ml, &r1));
    const double one = 1.0, zero = 0.0;
    DBuf W, G, Wq;
    D2_TRY(W.alloc((size_t)nL * k));
    D2_CUDA(cudaMemsetAsync(W.p, 0, sizeof(double) * nL * k, strm_));
    size_t gmax = 0, wmax = 0;
    for (size_t q = 0; q < ls.qld.size(); ++q) {
      auto it = rk.find(ls.target - ls.qlab[q]);
      if (it == rk.end()) continue;
      const size_t kq = it->second.second - it->second.first;
      gmax = std::max(gmax, (size_t)ls.qcols[q] * kq);
      wmax = std::max(wmax, (size_t)ls.qld[q] * kq);
    }
    D2_TRY(G.alloc(std::max<size_t>(gmax, 1)));
    D2_TRY(Wq.alloc(std::max<size_t>(wmax, 1)));
    int64_t r0 = 0, c0 = 0;
    for (size_t q = 0; q < ls.qld.size(); ++q) {
      const int ld = ls.qld[q], nc = ls.qcols[q];
      auto it = rk.find(ls.target - ls.qlab[q]);
      if (it != rk.end()) {
        const int j0 = it->second.first, kq = it->second.second - j0;
        k_gather_idx<<<512, 256, 0, strm_>>>(nr.U->p + nR * j0, nR,
                                             (const int64_t*)ls.d_colR->p + c0, nc, kq, G.p);
        D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_N, CUBLAS_OP_N, ld, kq, nc, &one,
                            ls.x->p + ls.qbase[q], ld, G.p, nc, &zero, Wq.p, ld));
        k_scatter_idx<<<512, 256, 0, strm_>>>(Wq.p, ld, kq, (const int64_t*)ls.d_rowL->p + r0, 1,
                                              W.p + nL * j0, nL);
        D2_CUDA(cudaGetLastError());
      }
      r0 += ld;
      c0 += nc;
    }
    auto v = std::make_shared<DBuf>();
    const int64_t nv = (int64_t)mp * d * d * k;
    D2_TRY(v->alloc((size_t)nv));
    D2_CUDA(cudaMemsetAsync(v->p, 0, sizeof(double) * nv, strm_));
    for (int s2 = 0; s2 < d; ++s2)
      for (const auto& pr : r1) {
        auto it = rk.find(ls.target - pr.first - col_label(s2));
        if (it == rk.end()) continue;
        const int b0 = it->second.first, kq = it->second.second - b0;
        const int a0 = pr.second.first, np = pr.second.second - a0;
        D2_BLAS(cublasDgemm(libs_.bl, CUBLAS_OP_N, CUBLAS_OP_N, mp * d, kq, np, &one,
                            Ls.U->p + (int64_t)mp * d * a0, mp * d,
                            W.p + a0 + (int64_t)ml * s2 + nL * b0, (int)nL, &zero,
                            v->p + (int64_t)mp * d * (b0 + (int64_t)k * s2), mp * d));
      }
    *out = v;
    return DMRG2D_OK;
  }

  dmrg2d_model M_;
  dmrg2d_sweep_opts o_;
  dmrg2d_sweep_report* rep_;
  std::map<int, Block> left_, right_;  // blocks by lattice columns (block 1 / block 4)
  std::shared_ptr<DBuf> guess_;        // start vector of the next step (null: seeded random)
  bool warm_done_ = false;
  int sweeps_done_ = 0;
  double last_energy_ = 0.0;
  cudaStream_t strm_;
  Rng rng_;
  Rng train_rng_;  // sample positions of the learned preconditioner's training batches
  DBuf obs_T_, obs_T2_;  // work vectors of the observables
  SpinColumnOps col_;
  Libs libs_;
  DBuf dH_col_;
  std::vector<DBuf> dsz_, dsp_;
  bool hub_ = false;              // Hubbard ladder (electrons) instead of spins
  HubbardColumnOps hc_;
  std::vector<DBuf> dcd_, dcdP_;  // per mode j: c^dag_j and c^dag_j P of the column
};

}  // namespace

}  // namespace dmrg2d

using namespace dmrg2d;

struct dmrg2d_state {
  dmrg2d::Sweeper* sw = nullptr;
  bool ready = false;   // column operators and handles set up (first sweep call)
  bool failed = false;  // an earlier call failed part-way: the blocks may be inconsistent
};

namespace {

// The lattice, model and filling fields (fixed for a state).
int check_lattice(const dmrg2d_model* model, const dmrg2d_sweep_opts* opts) {
  if (model->kind != DMRG2D_HEISENBERG && model->kind != DMRG2D_HUBBARD)
    return set_error(DMRG2D_EUNSUPPORTED, "sweep: Heisenberg or Hubbard ladders only");
  if (model->kind == DMRG2D_HUBBARD) {
    if (!opts->use_sectors)
      return set_error(DMRG2D_EUNSUPPORTED,
                       "sweep: Hubbard ladders run in a target (N_up, N_dn) sector (use_sectors)");
    const int sites = model->n_legs * opts->n_columns;
    if (opts->n_up < 0 || opts->n_dn < 0 || opts->n_up > sites || opts->n_dn > sites)
      return set_error(DMRG2D_EINVAL, "sweep: n_up, n_dn must be in [0, %d]", sites);
  }
  if (model->n_legs < 1 || model->n_legs > (model->kind == DMRG2D_HUBBARD ? 4 : 8))
    return set_error(DMRG2D_EINVAL, "sweep: n_legs must be in [1, %d]",
                     model->kind == DMRG2D_HUBBARD ? 4 : 8);
  if (opts->n_columns < 4 || opts->n_columns % 2)
    return set_error(DMRG2D_EINVAL, "sweep: n_columns must be even and >= 4");
  if (opts->m_warmup < 1) return set_error(DMRG2D_EINVAL, "sweep: m_warmup < 1");
  return DMRG2D_OK;
}

// The per-call fields: sweeps and solver options.
int check_call(const dmrg2d_sweep_opts* opts) {
  if (opts->n_sweeps < 0 || (opts->n_sweeps > 0 && !opts->m_sweep))
    return set_error(DMRG2D_EINVAL, "sweep: bad n_sweeps / m_sweep");
  for (int i = 0; i < opts->n_sweeps; ++i)
    if (opts->m_sweep[i] < 1) return set_error(DMRG2D_EINVAL, "sweep: m_sweep[%d] < 1", i);
  if (opts->max_iter < 1 || opts->krylov_dim < 2 || !(opts->tol > 0.0))
    return set_error(DMRG2D_EINVAL, "sweep: bad solver options");
  if (opts->solver != DMRG2D_SWEEP_LANCZOS && opts->solver != DMRG2D_SWEEP_DAVIDSON)
    return set_error(DMRG2D_EINVAL, "sweep: unknown solver %d", opts->solver);
  if (opts->solver == DMRG2D_SWEEP_DAVIDSON) {
    if (opts->precond < DMRG2D_PRECOND_NONE || opts->precond > DMRG2D_PRECOND_MLP)
      return set_error(DMRG2D_EINVAL, "sweep: unknown preconditioner %d", opts->precond);
    if (opts->precond == DMRG2D_PRECOND_MLP && !opts->mlp)
      return set_error(DMRG2D_EINVAL, "sweep: the MLP preconditioner needs a network");
    if (opts->mlp_epochs < 0) return set_error(DMRG2D_EINVAL, "sweep: mlp_epochs < 0");
  }
  return DMRG2D_OK;
}

}  // namespace

extern "C" int dmrg2d_state_create(const dmrg2d_model* model, const dmrg2d_sweep_opts* opts,
                                   dmrg2d_state** out) {
  if (!model || !opts || !out) return set_error(DMRG2D_EINVAL, "state_create: NULL argument");
  *out = nullptr;
  clear_error();
  D2_TRY(check_lattice(model, opts));
  dmrg2d_sweep_opts o = *opts;
  o.n_sweeps = 0;  // sweeps come with each dmrg2d_sweep call
  o.m_sweep = nullptr;
  dmrg2d_state* st = new (std::nothrow) dmrg2d_state();
  if (!st) return set_error(DMRG2D_ENOMEM, "state_create: out of host memory");
  st->sw = new (std::nothrow) Sweeper(model, &o, nullptr, nullptr);
  if (!st->sw) {
    delete st;
    return set_error(DMRG2D_ENOMEM, "state_create: out of host memory");
  }
  *out = st;
  return DMRG2D_OK;
}

extern "C" void dmrg2d_state_free(dmrg2d_state* st) {
  if (!st) return;
  delete st->sw;
  delete st;
}

extern "C" int dmrg2d_state_get_info(const dmrg2d_state* st, dmrg2d_state_info* info) {
  if (!st || !info) return set_error(DMRG2D_EINVAL, "state_get_info: NULL argument");
  const Sweeper& sw = *st->sw;
  const int L = sw.opts().n_columns, half = (L - 2) / 2;
  info->n_columns = L;
  info->warmed_up = sw.warm_done() ? 1 : 0;
  info->sweeps_done = sw.sweeps_done();
  info->last_energy = sw.last_energy();
  info->m_left = sw.block_states(true, half);
  info->m_right = sw.block_states(false, half);
  info->failed = st->failed ? 1 : 0;
  return DMRG2D_OK;
}

extern "C" int dmrg2d_sweep(dmrg2d_state* state, const dmrg2d_sweep_opts* opts,
                            dmrg2d_sweep_report* report, void* stream) {
  if (!state || !opts || !report) return set_error(DMRG2D_EINVAL, "sweep: NULL argument");
  clear_error();
  Sweeper& sw = *state->sw;
  const dmrg2d_sweep_opts& so = sw.opts();
  if (state->failed)
    return set_error(DMRG2D_EINVAL, "sweep: an earlier call on this state failed; free it");
  if (opts->n_columns != so.n_columns || opts->use_sectors != so.use_sectors ||
      opts->n_up != so.n_up || opts->n_dn != so.n_dn)
    return set_error(DMRG2D_EINVAL,
                     "sweep: n_columns, use_sectors, n_up, n_dn differ from the state's");
  D2_TRY(check_call(opts));
  if (report->cap < 0) return set_error(DMRG2D_EINVAL, "sweep: report cap < 0");
  report->n_steps = 0;
  report->seconds = report->solve_seconds = report->build_seconds = 0.0;
  report->dm_seconds = report->renorm_seconds = report->obs_seconds = 0.0;
  report->train_seconds = report->transform_seconds = 0.0;
  const auto t0 = std::chrono::steady_clock::now();
  int st = sw.begin_call(opts, report, (cudaStream_t)stream);
  if (st == DMRG2D_OK && !state->ready) {
    st = sw.init();
    state->ready = st == DMRG2D_OK;
  }
  if (st == DMRG2D_OK && !sw.warm_done()) st = sw.warmup();
  if (st == DMRG2D_OK) st = sw.sweeps(opts->n_sweeps, opts->m_sweep);
  if (st != DMRG2D_OK) state->failed = true;
  report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  report->solve_seconds = sw.solve_seconds;
  report->build_seconds = sw.build_seconds;
  report->dm_seconds = sw.dm_seconds;
  report->renorm_seconds = sw.renorm_seconds;
  report->obs_seconds = sw.obs_seconds;
  report->train_seconds = sw.train_seconds;
  report->transform_seconds = sw.transform_seconds;
  return st;
}
