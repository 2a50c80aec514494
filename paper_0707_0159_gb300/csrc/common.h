// Internal declarations shared by the translation units of libdmrg2d.
// Not part of the public ABI (see include/dmrg2d.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/dmrg2d.h"

namespace dmrg2d {

// ---- exact spin-column operators (row-major d x d), shared with the DMRG sweep --------
struct SpinColumnOps {
  int d = 0;
  std::vector<double> H;                     // rung bonds of one column
  std::vector<std::vector<double>> sz, sp;   // per leg: S^z_y, S^+_y
};
void spin_column_ops(int n, double J_rung, bool pbc, SpinColumnOps* out);
// exact Hubbard column: rung hopping + on-site U; c^dag of mode j = 2y + s (with the
// in-column string), the parity (-1)^N and the (N_up, N_dn) of every state (bit j of a
// state index is the occupation of mode j)
struct HubbardColumnOps {
  int d = 0;
  std::vector<double> H;
  std::vector<std::vector<double>> cd;
  std::vector<double> parity;
  std::vector<int> nup, ndn;
};
void hubbard_column_ops(int n, double t, double U, bool pbc, HubbardColumnOps* out);

// ---- error reporting (thread-local message, negative status codes) --------------------
int set_error(int code, const char* fmt, ...);
void clear_error();

#define D2_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ::dmrg2d::set_error(DMRG2D_ECUDA, "%s failed: %s (%s:%d)", #call,          \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);           \
  } while (0)

#define D2_TRY(expr)                                                                    \
  do {                                                                                  \
    int s_ = (expr);                                                                    \
    if (s_ != DMRG2D_OK) return s_;                                                     \
  } while (0)

// ---- packed operators -------------------------------------------------------------------
// Output tile (i2, i3) of V is the m1 x m4 sub-matrix with rows i1 + m1*i2 and
// columns i4 + m4*i3; its flat tile id is i2 + d*i3.
struct DeviceOps {
  // H_l: CSR over block rows i2; block e couples (i2, Lcol[e]); m1 x m1 row-major
  int nL = 0;
  int* Lptr = nullptr;
  int* Lcol = nullptr;
  double* HL64 = nullptr;
  float* HL32 = nullptr;
  __nv_bfloat16* HL16 = nullptr;
  // H_r: CSR over block columns i3; block e couples (i3, Rcol[e]); m4 x m4 row-major
  // stored as [i4][i4'] so that Y(:, i4) += sum_i4' V(:, i4') * HR[i4][i4']
  int nR = 0;
  int* Rptr = nullptr;
  int* Rcol = nullptr;
  double* HR64 = nullptr;
  float* HR32 = nullptr;
  __nv_bfloat16* HR16 = nullptr;
  // scalar tile moves: CSR over destination tiles t = i2 + d*i3
  int nC = 0;
  int* Cptr = nullptr;
  int* Csrc = nullptr;
  double* Cval64 = nullptr;
  float* Cval32 = nullptr;
};

}  // namespace dmrg2d

struct dmrg2d_ops {
  int kind = 0, n_legs = 0, d = 0, m1 = 0, m4 = 0;
  int64_t n_vec = 0;
  int64_t ld = 0;  // rows of V = m1*d (leading dimension of the column-major V)
  double flops = 0.0;
  int64_t device_bytes = 0;
  int tc_ok = 0;
  int device = 0;
  dmrg2d::DeviceOps dev;
  // host copies of the CSR structure (tile schedulers, tests)
  std::vector<int> hLptr, hLcol, hRptr, hRcol, hCptr, hCsrc;
  std::vector<double> hCval;
  std::vector<int> hqc;  // column quantum numbers, (N_up, N_dn) per column state
  // diagonal of H: H_l diagonal per (i1 + m1 i2), H_r per (i4 + m4 i3), H_c per (i2 + d i3)
  std::vector<double> hdL, hdR, hdC;
  // sector-restricted operation (NULL for the dense superblock), opaque here
  void* sec = nullptr;
  // tensor-core path state (tensor maps of the operator blocks), opaque here
  void* tc = nullptr;
  // tensor-core kernel choice per precision: -1 the dense kernel, >= 0 a grouped-kernel
  // tile configuration (set by dmrg2d_autotune; defaults chosen at build time)
  int tc_cfg[4] = {-1, -1, -1, -1};
  // kernel timing (dmrg2d_profile_start/stop); apply_H only records into it
  mutable std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  mutable size_t prof_used = 0;
  mutable bool prof_on = false;
};

namespace dmrg2d {

// event pair around the dominant kernel of one apply_H call (null when not profiling)
inline std::pair<cudaEvent_t, cudaEvent_t> prof_slot(const dmrg2d_ops* ops) {
  if (!ops->prof_on || ops->prof_used >= ops->prof_ev.size()) return {nullptr, nullptr};
  return ops->prof_ev[ops->prof_used++];
}

// hv_simt.cu
int launch_hv_simt_f64(const dmrg2d_ops* ops, const double* v, double* y, cudaStream_t s);
int launch_hv_simt_ff64(const dmrg2d_ops* ops, const double* v, double* y, cudaStream_t s);
int launch_hv_simt_f32(const dmrg2d_ops* ops, const float* v, float* y, cudaStream_t s);

// hv_tc.cu
int tc_prepare(dmrg2d_ops* ops, cudaStream_t s, const std::vector<double>& HL,
               const std::vector<double>& HR);
int tc_gemm(const dmrg2d_ops* ops, const void* v, float* y, int precision, int cfg,
            cudaStream_t s);
int sec_read_error(const dmrg2d_ops* ops, int* code);
void tc_release(dmrg2d_ops* ops);
int launch_hv_tc(const dmrg2d_ops* ops, const void* v, float* y, int precision, cudaStream_t s);
int tc_read_error(const dmrg2d_ops* ops, int* code);

// sectors.cu
int sec_build(dmrg2d_ops* ops, const dmrg2d_block* L, const dmrg2d_block* R, const int32_t* target,
              const std::vector<double>& HL, const std::vector<double>& HR, cudaStream_t s);
void sec_release(dmrg2d_ops* ops);
int sec_apply(const dmrg2d_ops* ops, const void* v, void* y, int precision, cudaStream_t s);
int sec_zero_padding(const dmrg2d_ops* ops, double* x, cudaStream_t s);
int sec_dense_index(const dmrg2d_ops* ops, int64_t* out);
int sec_count(const dmrg2d_ops* ops);
// per matrix V_q of a sector-restricted vector: row r -> enlarged-left index i1 + m1 i2
// (-1 for padding rows), column c -> enlarged-right index i4 + m4 i3 (concatenated over q)
int sec_layout(const dmrg2d_ops* ops, std::vector<long long>& qbase, std::vector<int>& qld,
               std::vector<int>& qcols, std::vector<int64_t>& row_left,
               std::vector<int64_t>& col_right);
int sec_diag_tables(const dmrg2d_ops* ops, std::vector<long long>& qbase, std::vector<int>& qld,
                    std::vector<int>& qcols, std::vector<double>& rowD, std::vector<int>& rowI2,
                    std::vector<double>& colD, std::vector<int>& colI3);

// diag.cu
void diag_pieces(dmrg2d_ops* ops, const std::vector<double>& HL, const std::vector<double>& HR);
int diag_apply(const dmrg2d_ops* ops, double* out, cudaStream_t s);

// mlp.cu: learned Davidson preconditioner state
struct MlpPrecond {
  int nq = 0;
  std::vector<double> mean, dmin, dmax, count, hqp;
  double meanD = 0.0, meanD2 = 0.0;
  long long* qstart = nullptr;
  double* qp = nullptr;
  float* Xg = nullptr;
  float* table = nullptr;
};
int mlp_precond_setup(const dmrg2d_mlp* M, const dmrg2d_ops* ops, const double* D, MlpPrecond* P,
                      cudaStream_t s);
int mlp_precond_apply(const dmrg2d_mlp* M, MlpPrecond* P, const double* r, const double* D,
                      double theta, double* t, int64_t n, cudaStream_t s);
void mlp_precond_release(MlpPrecond* P);

// vector kernels used by the solvers (solver.cu)
int convert_f64_to(const double* x, void* out, int precision, int64_t n, cudaStream_t s);

}  // namespace dmrg2d
