// Operator assembly for the superblock H·v (paper Eq. (dec)) and the small ABI entries.
//
// build_ops turns the model and the two renormalised blocks into
//   * dense m1 x m1 blocks of H_l, one per nonzero block position (i2, i2'),
//   * dense m4 x m4 blocks of H_r, one per nonzero block position (i3, i3'),
//   * scalar tile moves  Y_tile(i2, i3) += c * V_tile(i2', i3')  for every term
//     that is a multiple of the identity on both blocks (H_c, off-diagonal column
//     terms),
// and uploads them.  Column operators are built here from bit arithmetic on
// the column basis (layout in include/dmrg2d.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <new>
#include <thread>

#include "common.h"

namespace dmrg2d {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

namespace {

using Mat = std::vector<double>;  // row-major square matrix

Mat zeros(int n) { return Mat((size_t)n * n, 0.0); }

Mat matmul(const Mat& a, const Mat& b, int n) {
  Mat c = zeros(n);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      double x = a[(size_t)i * n + k];
      if (x == 0.0) continue;
      for (int j = 0; j < n; ++j) c[(size_t)i * n + j] += x * b[(size_t)k * n + j];
    }
  return c;
}

Mat transpose(const Mat& a, int n) {
  Mat t = zeros(n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) t[(size_t)j * n + i] = a[(size_t)i * n + j];
  return t;
}

int popcount_below(unsigned s, int j) { return __builtin_popcount(s & ((1u << j) - 1u)); }

// ---- exact column operators --------------------------------------------------------------
struct Column {
  int d = 0;
  Mat H;                        // column Hamiltonian (rung bonds, on-site U)
  std::vector<Mat> sz, sp, sm;  // spins: per leg
  std::vector<Mat> c, cd;       // electrons: per mode j = 2y + s
  std::vector<double> parity;   // electrons: (-1)^N
  std::vector<int> nup, ndn;
};

std::vector<std::pair<int, int>> rung_bonds(int n, bool pbc) {
  std::vector<std::pair<int, int>> b;
  for (int y = 0; y + 1 < n; ++y) b.push_back({y, y + 1});
  if (pbc && n > 2) b.push_back({n - 1, 0});
  return b;
}

Column spin_column(int n, double J_rung, bool pbc) {
  Column col;
  const int d = 1 << n;
  col.d = d;
  for (int y = 0; y < n; ++y) {
    Mat z = zeros(d), p = zeros(d);
    for (int s = 0; s < d; ++s) {
      z[(size_t)s * d + s] = ((s >> y) & 1) ? 0.5 : -0.5;
      if (!((s >> y) & 1)) p[(size_t)(s | (1 << y)) * d + s] = 1.0;  // S^+ |down> = |up>
    }
    col.sz.push_back(z);
    col.sp.push_back(p);
    col.sm.push_back(transpose(p, d));
  }
  col.H = zeros(d);
  for (auto [a, b] : rung_bonds(n, pbc))
    for (int s = 0; s < d; ++s) {
      int ba = (s >> a) & 1, bb = (s >> b) & 1;
      col.H[(size_t)s * d + s] += J_rung * (ba == bb ? 0.25 : -0.25);
      if (ba != bb) col.H[(size_t)(s ^ ((1 << a) | (1 << b))) * d + s] += 0.5 * J_rung;
    }
  for (int s = 0; s < d; ++s) {
    col.nup.push_back(__builtin_popcount((unsigned)s));
    col.ndn.push_back(0);
  }
  return col;
}

Column hubbard_column(int n, double t, double U, bool pbc) {
  Column col;
  const int nm = 2 * n;
  const int d = 1 << nm;
  col.d = d;
  for (int j = 0; j < nm; ++j) {
    Mat a = zeros(d);
    for (int s = 0; s < d; ++s)
      if ((s >> j) & 1) a[(size_t)(s ^ (1 << j)) * d + s] = (popcount_below(s, j) & 1) ? -1.0 : 1.0;
    col.c.push_back(a);
    col.cd.push_back(transpose(a, d));
  }
  col.H = zeros(d);
  for (auto [a, b] : rung_bonds(n, pbc))
    for (int sg = 0; sg < 2; ++sg) {
      Mat hop = matmul(col.cd[2 * a + sg], col.c[2 * b + sg], d);
      for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) {
          double h = hop[(size_t)i * d + k];
          if (h != 0.0) {
            col.H[(size_t)i * d + k] += -t * h;
            col.H[(size_t)k * d + i] += -t * h;
          }
        }
    }
  for (int s = 0; s < d; ++s) {
    int nu = 0, nd = 0;
    for (int y = 0; y < n; ++y) {
      int u = (s >> (2 * y)) & 1, dn = (s >> (2 * y + 1)) & 1;
      nu += u;
      nd += dn;
      if (u && dn) col.H[(size_t)s * d + s] += U;
    }
    col.nup.push_back(nu);
    col.ndn.push_back(nd);
    col.parity.push_back(((nu + nd) & 1) ? -1.0 : 1.0);
  }
  return col;
}

// X_col (d x d) (x) Y_block (m x m) with a coefficient
struct Term {
  double coef;
  Mat X;
  Mat Y;
};

Mat block_mat(const double* p, int m) { return Mat(p, p + (size_t)m * m); }

Mat col_times_parity(const Mat& a, const std::vector<double>& P, int d, bool right) {
  // right: a * P ; else P * a
  Mat r = a;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) r[(size_t)i * d + j] *= right ? P[j] : P[i];
  return r;
}

template <typename T>
int upload(const std::vector<T>& h, T** d, int64_t* bytes, cudaStream_t s) {
  if (h.empty()) {
    *d = nullptr;
    return DMRG2D_OK;
  }
  size_t nb = h.size() * sizeof(T);
  cudaError_t e = cudaMalloc((void**)d, nb);
  if (e != cudaSuccess) {
    *d = nullptr;
    return set_error(DMRG2D_ENOMEM, "cudaMalloc(%zu) failed: %s", nb, cudaGetErrorString(e));
  }
  *bytes += (int64_t)nb;
  D2_CUDA(cudaMemcpyAsync(*d, h.data(), nb, cudaMemcpyHostToDevice, s));
  return DMRG2D_OK;
}

int check_block(const dmrg2d_block* b, int n_legs, int kind, const char* name) {
  if (!b) return set_error(DMRG2D_EINVAL, "%s block is NULL", name);
  if (b->m < 1) return set_error(DMRG2D_EINVAL, "%s block: m = %d < 1", name, b->m);
  if (!b->H) return set_error(DMRG2D_EINVAL, "%s block: H is NULL", name);
  if (b->n_edge != 0 && b->n_edge != 2 * n_legs)
    return set_error(DMRG2D_ESHAPE, "%s block: n_edge = %d, expected 0 or %d", name, b->n_edge,
                     2 * n_legs);
  if (b->n_edge && !b->edge) return set_error(DMRG2D_EINVAL, "%s block: edge is NULL", name);
  for (int k = 0; k < b->n_edge; ++k)
    if (!b->edge[k]) return set_error(DMRG2D_EINVAL, "%s block: edge[%d] is NULL", name, k);
  (void)kind;
  return DMRG2D_OK;
}

}  // namespace

void spin_column_ops(int n, double J_rung, bool pbc, SpinColumnOps* out) {
  const Column c = spin_column(n, J_rung, pbc);
  out->d = c.d;
  out->H = c.H;
  out->sz = c.sz;
  out->sp = c.sp;
}

void hubbard_column_ops(int n, double t, double U, bool pbc, HubbardColumnOps* out) {
  const Column c = hubbard_column(n, t, U, pbc);
  out->d = c.d;
  out->H = c.H;
  out->cd = c.cd;
  out->parity = c.parity;
  out->nup = c.nup;
  out->ndn = c.ndn;
}

// Assemble the packed operators on the host.
// f(0 .. n-1) on the host's cores (the operator blocks of a superblock are independent)
template <typename F>
static void parallel_for(int n, F f) {
  const int nt = (int)std::min<unsigned>((unsigned)std::max(n, 1),
                                         std::max(1u, std::thread::hardware_concurrency()));
  if (nt <= 1 || n < 2) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int> next{0};
  auto worker = [&] {
    for (int i = next++; i < n; i = next++) f(i);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) {
    try {
      pool.emplace_back(worker);
    } catch (...) {  // no more threads: the ones started and this one finish the work
      break;
    }
  }
  worker();
  for (auto& th : pool) th.join();
}

static int assemble(const dmrg2d_model* M, const dmrg2d_block* L, const dmrg2d_block* R,
                    dmrg2d_ops* ops, std::vector<double>& HL, std::vector<double>& HR) {
  const bool heis = M->kind == DMRG2D_HEISENBERG;
  Column col = heis ? spin_column(M->n_legs, M->J_rung, M->rung_pbc != 0)
                    : hubbard_column(M->n_legs, M->t, M->U, M->rung_pbc != 0);
  const int d = col.d, m1 = L->m, m4 = R->m;
  ops->hqc.assign((size_t)d * 2, 0);
  for (int i = 0; i < d; ++i) {
    ops->hqc[2 * i] = col.nup[i];
    ops->hqc[2 * i + 1] = col.ndn[i];
  }
  ops->d = d;
  ops->m1 = m1;
  ops->m4 = m4;
  ops->ld = (int64_t)m1 * d;
  ops->n_vec = (int64_t)m1 * d * d * m4;

  // ---- Kronecker terms of H_l (X on i2, Y on i1) and H_r (X on i3, Y on i4) ----
  std::vector<Term> tl, tr;
  std::vector<std::pair<double, std::pair<Mat, Mat>>> tc;  // (coef, (a on i2, b on i3))
  if (heis) {
    const double J = M->J_leg;
    for (int y = 0; y < M->n_legs; ++y) {
      if (L->n_edge) {
        Mat sz1 = block_mat(L->edge[2 * y], m1), sp1 = block_mat(L->edge[2 * y + 1], m1);
        tl.push_back({J, col.sz[y], sz1});
        tl.push_back({0.5 * J, col.sm[y], sp1});
        tl.push_back({0.5 * J, col.sp[y], transpose(sp1, m1)});
      }
      if (R->n_edge) {
        Mat sz4 = block_mat(R->edge[2 * y], m4), sp4 = block_mat(R->edge[2 * y + 1], m4);
        tr.push_back({J, col.sz[y], sz4});
        tr.push_back({0.5 * J, col.sp[y], transpose(sp4, m4)});
        tr.push_back({0.5 * J, col.sm[y], sp4});
      }
      tc.push_back({J, {col.sz[y], col.sz[y]}});
      tc.push_back({0.5 * J, {col.sp[y], col.sm[y]}});
      tc.push_back({0.5 * J, {col.sm[y], col.sp[y]}});
    }
  } else {
    const double t = M->t;
    std::vector<double> P1(m1, 1.0);
    if (L->parity)
      for (int i = 0; i < m1; ++i) P1[i] = L->parity[i];
    for (int y = 0; y < M->n_legs; ++y)
      for (int s = 0; s < 2; ++s) {
        const int j = 2 * y + s;
        if (L->n_edge) {
          // c^dag_{1,e} c_{2,j} = (c^dag_e P_1) (x) c_j ; written column-op first: c_j (x) E
          Mat E = block_mat(L->edge[j], m1);
          for (int a = 0; a < m1; ++a)
            for (int b = 0; b < m1; ++b) E[(size_t)a * m1 + b] *= P1[b];
          tl.push_back({-t, col.c[j], E});
          tl.push_back({-t, col.cd[j], transpose(E, m1)});
        }
        if (R->n_edge) {
          // c^dag_{3,j} c_{4,e} = (c^dag_j P_3) (x) c_e
          Mat c4d = block_mat(R->edge[j], m4);
          tr.push_back({-t, col_times_parity(col.cd[j], col.parity, d, true), transpose(c4d, m4)});
          tr.push_back({-t, col_times_parity(col.c[j], col.parity, d, false), c4d});
        }
        // c^dag_{2,j} c_{3,j} = (c^dag_j P_2) (x) c_j
        tc.push_back({-t, {col_times_parity(col.cd[j], col.parity, d, true), col.c[j]}});
        tc.push_back({-t, {col_times_parity(col.c[j], col.parity, d, false), col.cd[j]}});
      }
  }

  // ---- dense blocks of H_l / H_r at every touched block position ----
  auto build_side = [&](const std::vector<Term>& terms, const double* HB, int m,
                        std::vector<int>& ptr, std::vector<int>& cidx, std::vector<double>& blocks,
                        std::vector<std::vector<char>>& is_pos) {
    is_pos.assign(d, std::vector<char>(d, 0));
    for (int i = 0; i < d; ++i) is_pos[i][i] = 1;
    for (const Term& tm : terms)
      for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k)
          if (tm.X[(size_t)i * d + k] != 0.0) is_pos[i][k] = 1;
    ptr.assign(d + 1, 0);
    cidx.clear();
    for (int i = 0; i < d; ++i) {
      for (int k = 0; k < d; ++k)
        if (is_pos[i][k]) cidx.push_back(k);
      ptr[i + 1] = (int)cidx.size();
    }
    const size_t mm = (size_t)m * m;
    std::vector<int> row_of(cidx.size());
    for (int i = 0; i < d; ++i)
      for (int e = ptr[i]; e < ptr[i + 1]; ++e) row_of[(size_t)e] = i;
    blocks.resize(cidx.size() * mm);
    parallel_for((int)cidx.size(), [&](int e) {  // one block position per task
      const int i = row_of[(size_t)e], k = cidx[(size_t)e];
      double* B = blocks.data() + (size_t)e * mm;
      if (i == k)
        std::copy(HB, HB + mm, B);
      else
        std::fill(B, B + mm, 0.0);
      const double hc = col.H[(size_t)i * d + k];
      if (hc != 0.0)
        for (int q = 0; q < m; ++q) B[(size_t)q * m + q] += hc;
      for (const Term& tm : terms) {
        const double x = tm.coef * tm.X[(size_t)i * d + k];
        if (x == 0.0) continue;
        for (size_t q = 0; q < mm; ++q) B[q] += x * tm.Y[q];
      }
    });
  };
  std::vector<std::vector<char>> posL, posR;
  build_side(tl, L->H, m1, ops->hLptr, ops->hLcol, HL, posL);
  build_side(tr, R->H, m4, ops->hRptr, ops->hRcol, HR, posR);

  // ---- scalar tile moves: Y(i2,i3) += c V(i2',i3') ----
  std::vector<std::map<int, double>> mv((size_t)d * d);
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k) {
      const double hc = col.H[(size_t)i * d + k];
      if (i == k || hc == 0.0) continue;
      if (!posL[i][k])
        for (int i3 = 0; i3 < d; ++i3) mv[(size_t)i + (size_t)d * i3][k + d * i3] += hc;
      if (!posR[i][k])
        for (int i2 = 0; i2 < d; ++i2) mv[(size_t)i2 + (size_t)d * i][i2 + d * k] += hc;
    }
  for (const auto& ct : tc) {
    const double c = ct.first;
    const Mat& a = ct.second.first;
    const Mat& b = ct.second.second;
    for (int i2 = 0; i2 < d; ++i2)
      for (int j2 = 0; j2 < d; ++j2) {
        const double av = a[(size_t)i2 * d + j2];
        if (av == 0.0) continue;
        for (int i3 = 0; i3 < d; ++i3)
          for (int j3 = 0; j3 < d; ++j3) {
            const double bv = b[(size_t)i3 * d + j3];
            if (bv == 0.0) continue;
            mv[(size_t)i2 + (size_t)d * i3][j2 + d * j3] += c * av * bv;
          }
      }
  }
  ops->hCptr.assign((size_t)d * d + 1, 0);
  ops->hCsrc.clear();
  ops->hCval.clear();
  for (size_t tid = 0; tid < (size_t)d * d; ++tid) {
    for (const auto& kv : mv[tid])
      if (kv.second != 0.0) {
        ops->hCsrc.push_back(kv.first);
        ops->hCval.push_back(kv.second);
      }
    ops->hCptr[tid + 1] = (int)ops->hCsrc.size();
  }
  ops->dev.nL = (int)ops->hLcol.size();
  ops->dev.nR = (int)ops->hRcol.size();
  ops->dev.nC = (int)ops->hCsrc.size();
  ops->flops = 2.0 * ops->dev.nL * (double)m1 * m1 * ((double)d * m4) +
               2.0 * ops->dev.nR * (double)m4 * m4 * ((double)m1 * d) +
               2.0 * ops->dev.nC * (double)m1 * m4;
  return DMRG2D_OK;
}

static void release_device(dmrg2d_ops* ops) {
  DeviceOps& D = ops->dev;
  void* ptrs[] = {D.Lptr, D.Lcol, D.HL64, D.HL32, D.HL16, D.Rptr, D.Rcol,  D.HR64,
                  D.HR32, D.HR16, D.Cptr, D.Csrc, D.Cval64, D.Cval32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  D = DeviceOps();
}

}  // namespace dmrg2d

using namespace dmrg2d;

extern "C" int dmrg2d_build_ops(const dmrg2d_model* model, const dmrg2d_block* left,
                                const dmrg2d_block* right, const int32_t* target,
                                dmrg2d_ops** out, void* stream) {
  clear_error();
  if (!out) return set_error(DMRG2D_EINVAL, "out is NULL");
  *out = nullptr;
  if (!model) return set_error(DMRG2D_EINVAL, "model is NULL");
  if (model->kind != DMRG2D_HEISENBERG && model->kind != DMRG2D_HUBBARD)
    return set_error(DMRG2D_EINVAL, "unknown model kind %d", model->kind);
  const int max_legs = model->kind == DMRG2D_HEISENBERG ? 10 : 5;
  if (model->n_legs < 1 || model->n_legs > max_legs)
    return set_error(DMRG2D_EINVAL, "n_legs = %d outside [1, %d]", model->n_legs, max_legs);
  D2_TRY(check_block(left, model->n_legs, model->kind, "left"));
  D2_TRY(check_block(right, model->n_legs, model->kind, "right"));
  cudaStream_t s = (cudaStream_t)stream;

  dmrg2d_ops* ops = new dmrg2d_ops();
  ops->kind = model->kind;
  ops->n_legs = model->n_legs;
  cudaGetDevice(&ops->device);
  std::vector<double> HL, HR;
  int st;
  try {
    st = assemble(model, left, right, ops, HL, HR);
  } catch (const std::bad_alloc&) {
    st = set_error(DMRG2D_ENOMEM, "build_ops: out of host memory for the operator blocks");
  }
  if (st != DMRG2D_OK) {
    delete ops;
    return st;
  }
  diag_pieces(ops, HL, HR);
  if (target) {  // sector-restricted: pack the sub-blocks, skip the dense uploads
    st = sec_build(ops, left, right, target, HL, HR, s);
    if (st != DMRG2D_OK) {
      sec_release(ops);
      delete ops;
      return st;
    }
    *out = ops;
    return DMRG2D_OK;
  }
  std::vector<float> HL32(HL.begin(), HL.end()), HR32(HR.begin(), HR.end());
  std::vector<__nv_bfloat16> HL16(HL.size()), HR16(HR.size());
  for (size_t i = 0; i < HL.size(); ++i) HL16[i] = __float2bfloat16_rn((float)HL[i]);
  for (size_t i = 0; i < HR.size(); ++i) HR16[i] = __float2bfloat16_rn((float)HR[i]);
  std::vector<float> C32(ops->hCval.begin(), ops->hCval.end());
  DeviceOps& D = ops->dev;
  int64_t* nb = &ops->device_bytes;
  st = DMRG2D_OK;
#define UP(h, dptr) \
  if (st == DMRG2D_OK) st = upload(h, &dptr, nb, s)
  UP(ops->hLptr, D.Lptr);
  UP(ops->hLcol, D.Lcol);
  UP(HL, D.HL64);
  UP(HL32, D.HL32);
  UP(HL16, D.HL16);
  UP(ops->hRptr, D.Rptr);
  UP(ops->hRcol, D.Rcol);
  UP(HR, D.HR64);
  UP(HR32, D.HR32);
  UP(HR16, D.HR16);
  UP(ops->hCptr, D.Cptr);
  UP(ops->hCsrc, D.Csrc);
  UP(ops->hCval, D.Cval64);
  UP(C32, D.Cval32);
#undef UP
  if (st == DMRG2D_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = set_error(DMRG2D_ECUDA, "upload: %s", cudaGetErrorString(e));
  }
  if (st == DMRG2D_OK) st = tc_prepare(ops, s, HL, HR);
  if (st != DMRG2D_OK) {
    tc_release(ops);
    release_device(ops);
    delete ops;
    return st;
  }
  *out = ops;
  return DMRG2D_OK;
}

extern "C" int dmrg2d_ops_get_info(const dmrg2d_ops* ops, dmrg2d_ops_info* info) {
  if (!ops || !info) return set_error(DMRG2D_EINVAL, "NULL argument");
  info->n_vec = ops->n_vec;
  info->m1 = ops->m1;
  info->m4 = ops->m4;
  info->d = ops->d;
  info->n_legs = ops->n_legs;
  info->n_blk_left = ops->dev.nL;
  info->n_blk_right = ops->dev.nR;
  info->n_scalar = ops->dev.nC;
  info->flops_per_apply = ops->flops;
  info->tc_ok = ops->tc_ok;
  info->device_bytes = ops->device_bytes;
  info->n_sectors = sec_count(ops);
  return DMRG2D_OK;
}

extern "C" int dmrg2d_sector_dense_index(const dmrg2d_ops* ops, int64_t* out) {
  if (!ops || !out) return set_error(DMRG2D_EINVAL, "NULL argument");
  return sec_dense_index(ops, out);
}

static void prof_clear(dmrg2d_ops* ops) {
  for (auto& e : ops->prof_ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  ops->prof_ev.clear();
  ops->prof_used = 0;
  ops->prof_on = false;
}

extern "C" int dmrg2d_profile_start(dmrg2d_ops* ops, int max_launches) {
  if (!ops || max_launches < 1) return set_error(DMRG2D_EINVAL, "profile_start: bad argument");
  prof_clear(ops);
  for (int i = 0; i < max_launches; ++i) {
    cudaEvent_t a, b;
    D2_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return set_error(DMRG2D_ECUDA, "cudaEventCreate failed");
    }
    ops->prof_ev.push_back({a, b});
  }
  ops->prof_on = true;
  return DMRG2D_OK;
}

extern "C" int dmrg2d_profile_stop(dmrg2d_ops* ops, double* total_ms, int* launches) {
  if (!ops || !total_ms || !launches) return set_error(DMRG2D_EINVAL, "profile_stop: NULL");
  double tot = 0.0;
  for (size_t i = 0; i < ops->prof_used; ++i) {
    D2_CUDA(cudaEventSynchronize(ops->prof_ev[i].second));
    float ms = 0.f;
    D2_CUDA(cudaEventElapsedTime(&ms, ops->prof_ev[i].first, ops->prof_ev[i].second));
    tot += ms;
  }
  *total_ms = tot;
  *launches = (int)ops->prof_used;
  prof_clear(ops);
  return DMRG2D_OK;
}

extern "C" void dmrg2d_free_ops(dmrg2d_ops* ops) {
  if (!ops) return;
  prof_clear(ops);
  sec_release(ops);
  tc_release(ops);
  release_device(ops);
  delete ops;
}

extern "C" int dmrg2d_check_device(const dmrg2d_ops* ops) {
  if (!ops) return set_error(DMRG2D_EINVAL, "NULL ops");
  D2_CUDA(cudaDeviceSynchronize());
  int code = 0;
  D2_TRY(tc_read_error(ops, &code));
  if (code) return set_error(DMRG2D_ETIMEOUT, "tensor-core kernel gave up waiting (site %d)", code);
  return DMRG2D_OK;
}

extern "C" const char* dmrg2d_last_error(void) { return g_err.c_str(); }

extern "C" const char* dmrg2d_version(void) { return "dmrg2d-gb300 0.1 (sm_103a)"; }

extern "C" size_t dmrg2d_struct_size(int which) {
  switch (which) {
    case DMRG2D_STRUCT_MODEL: return sizeof(dmrg2d_model);
    case DMRG2D_STRUCT_BLOCK: return sizeof(dmrg2d_block);
    case DMRG2D_STRUCT_OPS_INFO: return sizeof(dmrg2d_ops_info);
    case DMRG2D_STRUCT_SOLVER_OPTS: return sizeof(dmrg2d_solver_opts);
    case DMRG2D_STRUCT_SOLVER_STATS: return sizeof(dmrg2d_solver_stats);
    case DMRG2D_STRUCT_DAVIDSON_OPTS: return sizeof(dmrg2d_davidson_opts);
    case DMRG2D_STRUCT_SWEEP_OPTS: return sizeof(dmrg2d_sweep_opts);
    case DMRG2D_STRUCT_SWEEP_REPORT: return sizeof(dmrg2d_sweep_report);
    case DMRG2D_STRUCT_STATE_INFO: return sizeof(dmrg2d_state_info);
    default: return 0;
  }
}

extern "C" void dmrg2d_default_solver_opts(dmrg2d_solver_opts* o) {
  if (!o) return;
  o->max_iter = 300;
  o->krylov_dim = 64;
  o->tol = 1e-10;
  o->fixed_steps = 0;
  o->precision = DMRG2D_FP64;
  o->refine = 0;
  o->inner_iter = 30;
  o->outer_max = 20;
  o->check_every = 5;
  o->start_reorth = 0;
  o->refine_precision = DMRG2D_FP64;
  o->thick_keep = 0;
}
