// Grouped tcgen05 H·v over a work list of (row segment x column segment) pieces.
//
// Same pipeline as hv_tc_kernel (TMA ring, one MMA-issuing thread, two TMEM
// accumulators, four epilogue warps, bounded waits), but every piece reads its
// operator blocks and its V_q slices from per-segment lists, so one persistent launch
// covers uneven quantum-number sectors (or the dense superblock as a single sector).
// Rows of a piece beyond its segment and K beyond a block's width meet zero-padded
// pool columns or are masked in the epilogue; the epilogue also writes the zero
// padding rows of the segment.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include <cudaTypedefs.h>

#include "grouped.h"
#include "tc_ptx.cuh"

namespace dmrg2d {

namespace {

using namespace tc;

constexpr int GQ_MAX = 64;  // sectors per launch (V tensor maps travel as kernel parameters)
constexpr int G_THREADS = 320;  // producer, MMA issuer, 8 epilogue warps
constexpr int G_EPI_WARPS = 8;
constexpr int G_STAGES = 4;
constexpr int G_BM = 128;
constexpr uint32_t G_STAGE_A = 16384, G_STAGE_B = 32768, G_STAGE = G_STAGE_A + G_STAGE_B;
constexpr uint32_t G_TMEM_COLS = 512, G_ACC_COLS = 256;
constexpr size_t G_SMEM = G_STAGES * G_STAGE + 1024 + 256;
constexpr int N_ORDERS = 3;  // column-slab raster, row-slab raster, longest piece first

// a scalar move as the epilogue reads it: element offset of the source segment's first
// row and column in the packed vector, the source matrix's leading dimension, coefficient
struct GMoveD {
  long long src;
  int ld;
  float c;
};

struct GMaps {
  CUtensorMap L, R;
  CUtensorMap vk[GQ_MAX];
  CUtensorMap vm[GQ_MAX];
};

struct GParams {
  int ntiles, bn, BK;
  const GTile* tiles;
  const GRow* rows;
  const GCol* cols;
  const GK1* k1;
  const GK2* k2;
  const long long* qbase;
  const int* qld;
  float* y;
  int* err;
  const GMoveD* moves;  // scalar moves, read by the epilogue
  const void* v;       // the input vector (TF32 as float, or BF16)
  uint32_t idesc1[2], idesc2[2];
  uint32_t a2_lbo, a2_sbo, a2_kstep, a2_layout;
  int a2_boxes, a2_box_rows;
  uint32_t tx_bytes;
  int bf16;
  int accum_y;  // add the Y already stored (BF16X3's second and third products)
};

struct SItem;

struct GDev {
  GTile* tiles[2][N_ORDERS] = {};
  int ntiles[2][N_ORDERS] = {};
  GRow* rows = nullptr;
  GCol* cols = nullptr;
  GK1* k1 = nullptr;
  GK2* k2 = nullptr;
  GMoveD* moves = nullptr;
  long long* qbase = nullptr;
  int* qld = nullptr;
  float* pL32 = nullptr;
  float* pR32 = nullptr;
  __nv_bfloat16* pL16 = nullptr;
  __nv_bfloat16* pR16 = nullptr;
  __nv_bfloat16* pL16lo = nullptr;  // BF16X3: x - bf16(x) rounded to BF16
  __nv_bfloat16* pR16lo = nullptr;
  CUtensorMap mLlo, mRlo[2];
  CUtensorMap mL32[2], mR32[2], mL32lo, mR32lo;  // the pools in 32-row boxes (segment kernels)
  int KPL = 0, KPR = 0, prL = 0, prR = 0, copies = 1;
  CUtensorMap mL[2], mR[2][2];  // [precision][piece width 128/256]
  int* err = nullptr;
  int sms = 0;
  std::vector<void*> allocs;
  int* d_qcols = nullptr;
  SItem* sitems[2] = {nullptr, nullptr};  // segment kernels: pass 1 and pass 2 pieces
  int nsitems[2] = {0, 0};
};

template <int BF16>
__global__ void __launch_bounds__(G_THREADS, 1)
hv_tc_grouped_kernel(const __grid_constant__ GMaps maps, const GParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + G_STAGES * G_STAGE);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * G_STAGES + 4);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + G_STAGES + s); };
  auto tfull = [&](int b) { return smem_u32(bars + 2 * G_STAGES + b); };
  auto tempty = [&](int b) { return smem_u32(bars + 2 * G_STAGES + 2 + b); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), G_EPI_WARPS);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(G_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int BK = p.BK;

  if (warp == 0 && lane == 0) {
    // ------------------------------- TMA producer -------------------------------
    int stage = 0;
    uint32_t phase = 0;
    for (int ti = blockIdx.x; ti < p.ntiles && !*abort; ti += gridDim.x) {
      const GTile t = p.tiles[ti];
      const GRow rs = p.rows[t.rs];
      const GCol cs = p.cols[t.cs];
      const int r0 = rs.off + t.r_in, c0 = cs.off + t.c_in;
      const CUtensorMap* vk = &maps.vk[rs.q];
      const CUtensorMap* vm = &maps.vm[rs.q];
      for (int ph = 0; ph < 2; ++ph) {
        const int e0 = ph == 0 ? rs.k1b : cs.k2b, e1 = ph == 0 ? rs.k1e : cs.k2e;
        for (int e = e0; e < e1; ++e) {
          int kdim, a_pool = 0, b_row = 0, a_col = 0, b_pool = 0;
          if (ph == 0) {
            const GK1 k = p.k1[e];
            kdim = k.kdim;
            a_pool = k.a_pool;
            b_row = k.b_row;
          } else {
            const GK2 k = p.k2[e];
            kdim = k.kdim;
            a_col = k.a_col;
            b_pool = k.b_pool;
          }
          const int nk = (kdim + BK - 1) / BK;
          for (int kc = 0; kc < nk; ++kc) {
            if (!mbar_wait(empty(stage), phase ^ 1u, abort)) {
              raise_abort(abort, p.err, 11);
              goto producer_done;
            }
            const uint32_t a_s = smem_u32(smem + stage * G_STAGE);
            const uint32_t b_s = a_s + G_STAGE_A;
            mbar_expect_tx(full(stage), p.tx_bytes);
            if (ph == 0) {
              tma_load_2d(a_s, &maps.L, full(stage), kc * BK, a_pool + t.r_in);
              tma_load_2d(b_s, vk, full(stage), b_row + kc * BK, c0);
            } else {
              for (int b = 0; b < p.a2_boxes; ++b)
                tma_load_2d(a_s + b * p.a2_lbo, vm, full(stage), r0 + b * p.a2_box_rows,
                            a_col + kc * BK);
              tma_load_2d(b_s, &maps.R, full(stage), kc * BK, b_pool + t.c_in);
            }
            if (++stage == G_STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
    }
  producer_done:;
  } else if (warp == 1 && lane == 0) {
    // ------------------------------- MMA issuer ---------------------------------
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t aphase = 0;
    for (int ti = blockIdx.x; ti < p.ntiles && !*abort; ti += gridDim.x) {
      const GTile t = p.tiles[ti];
      const GRow rs = p.rows[t.rs];
      const GCol cs = p.cols[t.cs];
      if (!mbar_wait(tempty(acc), aphase ^ 1u, abort)) {
        raise_abort(abort, p.err, 12);
        break;
      }
      tc_fence_after();
      const uint32_t dt = tmem_base + acc * G_ACC_COLS;
      uint32_t accum = 0;
      bool ok = true;
      for (int ph = 0; ph < 2 && ok; ++ph) {
        const int e0 = ph == 0 ? rs.k1b : cs.k2b, e1 = ph == 0 ? rs.k1e : cs.k2e;
        // descriptor fields fixed for the phase (no branch between two MMAs: the tensor
        // pipe's instruction queue is shallow)
        const uint64_t a_hi = ph == 0 ? sdesc(0, 16, 1024)
                                      : sdesc(0, p.a2_lbo, p.a2_sbo, p.a2_layout);
        const uint32_t a_step = ph == 0 ? 32u : p.a2_kstep;
        const uint64_t b_hi = sdesc(0, 16, 1024);
        for (int e = e0; e < e1 && ok; ++e) {
          const int kdim = ph == 0 ? p.k1[e].kdim : p.k2[e].kdim;
          const int neg = ph == 0 ? p.k1[e].neg : p.k2[e].neg;
          const uint32_t id = ph == 0 ? (neg ? p.idesc1[1] : p.idesc1[0])
                                      : (neg ? p.idesc2[1] : p.idesc2[0]);
          const int nk = (kdim + BK - 1) / BK;
          for (int kc = 0; kc < nk; ++kc) {
            // the mbarrier's completion orders the TMA writes before these MMAs
            if (!mbar_wait(full(stage), phase, abort)) {
              raise_abort(abort, p.err, 13);
              ok = false;
              break;
            }
            const uint32_t a_s = smem_u32(smem + stage * G_STAGE);
            const uint32_t b_s = a_s + G_STAGE_A;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              umma_t<BF16>(dt, a_hi | sdesc_addr(a_s + k * a_step),
                           b_hi | sdesc_addr(b_s + k * 32), id, accum);
              accum = 1;
            }
            umma_commit(empty(stage));
            stage = stage + 1 == G_STAGES ? 0 : stage + 1;
            phase ^= stage == 0 ? 1u : 0u;
          }
        }
      }
      if (!ok) break;
      umma_commit(tfull(acc));
      if (++acc == 2) {
        acc = 0;
        aphase ^= 1u;
      }
    }
  } else if (warp >= 2) {
    // ------------------------------- epilogue -----------------------------------
    // two warps per TMEM lane quadrant, alternating 32-column chunks; the scalar moves of
    // the tile's (row segment, column segment) are added from V before the store
    const int q4 = warp & 3;
    const int half = (warp - 2) >> 2;
    int acc = 0;
    uint32_t aphase = 0;
    for (int ti = blockIdx.x; ti < p.ntiles; ti += gridDim.x) {
      const GTile t = p.tiles[ti];
      const GRow rs = p.rows[t.rs];
      const GCol cs = p.cols[t.cs];
      if (!mbar_wait(tfull(acc), aphase, abort)) {
        raise_abort(abort, p.err, 14);
        break;
      }
      tc_fence_after();
      const bool has_k = rs.k1e > rs.k1b || cs.k2e > cs.k2b;
      const int rows_valid = min(G_BM, rs.dim - t.r_in);
      const int rows_out = min(G_BM, rs.dim_pad - t.r_in);  // valid rows + zero padding rows
      const int cols_valid = min(p.bn, cs.dim - t.c_in);
      const int row = 32 * q4 + lane;
      const long long ld = p.qld[rs.q];
      float* yq = p.y + p.qbase[rs.q] + rs.off + t.r_in + row + ld * (cs.off + t.c_in);
      for (int ch = half; ch < p.bn / 32 && ch * 32 < cols_valid; ch += 2) {
        uint32_t v[32];
        if (has_k) {
          tmem_ld32(tmem_base + ((uint32_t)(32 * q4) << 16) + acc * G_ACC_COLS + ch * 32, v);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0u;
        }
        float o[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) o[j] = __uint_as_float(v[j]);
        const bool real = row < rows_valid;
        if (real && p.moves) {
          // two moves per iteration: 64 loads in flight per thread
          const long long rc = t.r_in + row;
          const long long cc = t.c_in + ch * 32;
          for (int e = t.mb; e < t.me; e += 2) {
            const bool two = e + 1 < t.me;
            const GMoveD ma = p.moves[e];
            const GMoveD mb = two ? p.moves[e + 1] : ma;
            const float cb = two ? mb.c : 0.f;
            const long long oa = ma.src + rc + (long long)ma.ld * cc;
            const long long ob = mb.src + rc + (long long)mb.ld * cc;
            float va[32], vb[32];
            if (p.bf16) {
              const __nv_bfloat16* A = (const __nv_bfloat16*)p.v + oa;
              const __nv_bfloat16* B = (const __nv_bfloat16*)p.v + ob;
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const bool in = ch * 32 + j < cols_valid;
                va[j] = in ? __bfloat162float(A[(long long)ma.ld * j]) : 0.f;
                vb[j] = in ? __bfloat162float(B[(long long)mb.ld * j]) : 0.f;
              }
            } else {
              const float* A = (const float*)p.v + oa;
              const float* B = (const float*)p.v + ob;
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const bool in = ch * 32 + j < cols_valid;
                va[j] = in ? __ldg(A + (long long)ma.ld * j) : 0.f;
                vb[j] = in ? __ldg(B + (long long)mb.ld * j) : 0.f;
              }
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) o[j] += ma.c * va[j] + cb * vb[j];
          }
        }
        if (row < rows_out) {
          if (p.accum_y && real) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (ch * 32 + j < cols_valid) o[j] += yq[ld * (ch * 32 + j)];
          }
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (ch * 32 + j < cols_valid) yq[ld * (ch * 32 + j)] = real ? o[j] : 0.f;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(acc));
      if (++acc == 2) {
        acc = 0;
        aphase ^= 1u;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(G_TMEM_COLS)
                 : "memory");
  }
}

// ---- sectors of tens of states: M = 128 along the long dimension of V_q ---------------------
// A piece of the grouped kernel is 128 rows of one row segment: with quantum-number sectors of
// tens of states most of its rows, columns and K are padding.  These two passes keep the
// MMA's M = 128 on the long dimension of V_q instead, and its N on one segment (rounded up to
// the instruction's 16):
//   pass 1 (H_l V): for a row segment r and 128 columns of V_q,
//       Y_q(rows of r, cols)^T = sum_e V_q(rows of r_e, cols)^T H_l[r, r_e]^T,
//     the grouped kernel's phase-1 operands with their roles swapped (A = the V tile, M =
//     its 128 columns; B = the operator block, N = the rows of r);
//   pass 2 (V H_r^T): for a column segment c and 128 rows of V_q (across row segments),
//       Y_q(rows, cols of c) += sum_e V_q(rows, cols of c_e) H_r[c, c_e]^T  (N = c's columns).
// The K loop skips the instruction steps past an operator block's K.  The scalar moves run in
// their own kernel after pass 2.
struct SItem {
  int q, seg, n0, m0;  // matrix; segment (row segment in pass 1, column segment in pass 2);
                       // offset of the N range in the segment; first of the 128 M indices
};

struct SParams {
  int nitems;
  const SItem* items;
  const GRow* rows;
  const GCol* cols;
  const GK1* k1;
  const GK2* k2;
  const long long* qbase;
  const int* qld;
  const int* qcols;
  float* y;
  int* err;
  uint32_t idesc[16][2];  // N = 16 (i + 1); [negate the operator block]
  uint32_t a2_lbo, a2_sbo, a2_kstep, a2_layout;  // pass 2: MN-major A (as the grouped kernel)
  int a2_boxes, a2_box_rows;
  uint32_t a_bytes, b_box_bytes;  // per stage: the A tile; one 32-row box of B
  int BK, KSTEP;  // K per stage; K per instruction
  int accum_y;    // pass 1: add the Y already stored (BF16X3)
};

template <int BF16, int PASS>
__global__ void __launch_bounds__(G_THREADS, 1)
hv_tc_seg_kernel(const __grid_constant__ GMaps maps, const SParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + G_STAGES * G_STAGE);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * G_STAGES + 4);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + G_STAGES + s); };
  auto tfull = [&](int b) { return smem_u32(bars + 2 * G_STAGES + b); };
  auto tempty = [&](int b) { return smem_u32(bars + 2 * G_STAGES + 2 + b); };
  constexpr int NMAX = PASS == 0 ? 128 : 256;  // N per piece (pool boxes of 128 / 256 rows)

  if (threadIdx.x == 0) {
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), G_EPI_WARPS);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(G_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int BK = p.BK;

  if (warp == 0 && lane == 0) {
    // ------------------------------- TMA producer -------------------------------
    int stage = 0;
    uint32_t phase = 0;
    for (int ti = blockIdx.x; ti < p.nitems && !*abort; ti += gridDim.x) {
      const SItem it = p.items[ti];
      const int e0 = PASS == 0 ? p.rows[it.seg].k1b : p.cols[it.seg].k2b;
      const int e1 = PASS == 0 ? p.rows[it.seg].k1e : p.cols[it.seg].k2e;
      // the operator rows this piece needs, in 32-row boxes (N rounded up to 16 <= 32 nb)
      const int sdim = PASS == 0 ? p.rows[it.seg].dim : p.cols[it.seg].dim;
      const int nb = (min(NMAX, sdim - it.n0) + 31) / 32;
      const uint32_t tx = p.a_bytes + (uint32_t)nb * p.b_box_bytes;
      for (int e = e0; e < e1; ++e) {
        int kdim, pool, voff;
        if (PASS == 0) {
          const GK1 k = p.k1[e];
          kdim = k.kdim;
          pool = k.a_pool;
          voff = k.b_row;
        } else {
          const GK2 k = p.k2[e];
          kdim = k.kdim;
          pool = k.b_pool;
          voff = k.a_col;
        }
        const int nk = (kdim + BK - 1) / BK;
        for (int kc = 0; kc < nk; ++kc) {
          if (!mbar_wait(empty(stage), phase ^ 1u, abort)) {
            raise_abort(abort, p.err, 21);
            goto producer_done;
          }
          const uint32_t a_s = smem_u32(smem + stage * G_STAGE);
          const uint32_t b_s = a_s + G_STAGE_A;
          mbar_expect_tx(full(stage), tx);
          if (PASS == 0) {
            // A: V_q rows voff + kc BK .. (K), columns m0 .. m0 + 127 (M)
            tma_load_2d(a_s, &maps.vk[it.q], full(stage), voff + kc * BK, it.m0);
          } else {
            // A: V_q rows m0 .. m0 + 127 (M, MN-major), columns voff + kc BK .. (K)
            for (int b = 0; b < p.a2_boxes; ++b)
              tma_load_2d(a_s + b * p.a2_lbo, &maps.vm[it.q], full(stage),
                          it.m0 + b * p.a2_box_rows, voff + kc * BK);
          }
          // B: operator rows pool + n0 .., 32 at a time (the 128B swizzle is a function of
          // the shared-memory address, so the boxes line up as one tile)
          for (int b = 0; b < nb; ++b)
            tma_load_2d(b_s + b * 32 * 128, PASS == 0 ? &maps.L : &maps.R, full(stage), kc * BK,
                        pool + it.n0 + 32 * b);
          if (++stage == G_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  producer_done:;
  } else if (warp == 1 && lane == 0) {
    // ------------------------------- MMA issuer ---------------------------------
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t aphase = 0;
    const uint64_t a_hi = PASS == 0 ? sdesc(0, 16, 1024) : sdesc(0, p.a2_lbo, p.a2_sbo, p.a2_layout);
    const uint32_t a_step = PASS == 0 ? 32u : p.a2_kstep;
    const uint64_t b_hi = sdesc(0, 16, 1024);
    const int ksteps = BK / p.KSTEP;  // 4
    for (int ti = blockIdx.x; ti < p.nitems && !*abort; ti += gridDim.x) {
      const SItem it = p.items[ti];
      const int sdim = PASS == 0 ? p.rows[it.seg].dim : p.cols[it.seg].dim;
      const int nvalid = min(NMAX, sdim - it.n0);
      const int nidx = (nvalid + 15) / 16 - 1;
      const int e0 = PASS == 0 ? p.rows[it.seg].k1b : p.cols[it.seg].k2b;
      const int e1 = PASS == 0 ? p.rows[it.seg].k1e : p.cols[it.seg].k2e;
      if (!mbar_wait(tempty(acc), aphase ^ 1u, abort)) {
        raise_abort(abort, p.err, 22);
        break;
      }
      tc_fence_after();
      const uint32_t dt = tmem_base + acc * G_ACC_COLS;
      uint32_t accum = 0;
      bool ok = true;
      for (int e = e0; e < e1 && ok; ++e) {
        const int kdim = PASS == 0 ? p.k1[e].kdim : p.k2[e].kdim;
        const int neg = PASS == 0 ? p.k1[e].neg : p.k2[e].neg;
        const uint32_t id = p.idesc[nidx][neg];
        const int nk = (kdim + BK - 1) / BK;
        const int last = (kdim - (nk - 1) * BK + p.KSTEP - 1) / p.KSTEP;  // steps in the last stage
        for (int kc = 0; kc < nk; ++kc) {
          if (!mbar_wait(full(stage), phase, abort)) {
            raise_abort(abort, p.err, 23);
            ok = false;
            break;
          }
          const uint32_t a_s = smem_u32(smem + stage * G_STAGE);
          const uint32_t b_s = a_s + G_STAGE_A;
          const int nks = kc + 1 == nk ? last : ksteps;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            umma_if_t<BF16>(dt, a_hi | sdesc_addr(a_s + k * a_step), b_hi | sdesc_addr(b_s + k * 32),
                            id, accum, (uint32_t)(k < nks));
            accum = 1;  // step 0 is always issued
          }
          umma_commit(empty(stage));
          stage = stage + 1 == G_STAGES ? 0 : stage + 1;
          phase ^= stage == 0 ? 1u : 0u;
        }
      }
      if (!ok) break;
      umma_commit(tfull(acc));
      if (++acc == 2) {
        acc = 0;
        aphase ^= 1u;
      }
    }
  } else if (warp >= 2) {
    // ------------------------------- epilogue -----------------------------------
    // TMEM lane = M index (a column of V_q in pass 1, a row in pass 2), TMEM column = N
    // index; two warps per lane quadrant take alternate 32-column chunks
    const int q4 = warp & 3;
    const int half = (warp - 2) >> 2;
    int acc = 0;
    uint32_t aphase = 0;
    for (int ti = blockIdx.x; ti < p.nitems; ti += gridDim.x) {
      const SItem it = p.items[ti];
      if (!mbar_wait(tfull(acc), aphase, abort)) {
        raise_abort(abort, p.err, 24);
        break;
      }
      tc_fence_after();
      const long long ld = p.qld[it.q];
      float* yq = p.y + p.qbase[it.q];
      const int mi = it.m0 + 32 * q4 + lane;  // this thread's M index
      if (PASS == 0) {
        const GRow rs = p.rows[it.seg];
        const bool has_k = rs.k1e > rs.k1b;
        // rows n0 .. of the segment: valid up to dim, zero padding up to dim_pad
        const int nout = min(NMAX, rs.dim_pad - it.n0);
        const int nval = min(NMAX, rs.dim - it.n0);
        const int nch = (nout + 31) / 32;
        const bool col_ok = mi < p.qcols[it.q];
        float* ycol = yq + rs.off + it.n0 + ld * mi;
        for (int ch = half; ch < nch; ch += 2) {
          uint32_t v[32];
          if (has_k) {
            tmem_ld32(tmem_base + acc * G_ACC_COLS + ((uint32_t)(32 * q4) << 16) + ch * 32, v);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0u;
          }
          if (col_ok) {
            // 16-byte stores: the segment offset, n0 and ld are multiples of 8 and nout of 8
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4) {
              const int n = ch * 32 + 4 * j4;
              if (n < nout) {
                float4 o;
                o.x = n + 0 < nval ? __uint_as_float(v[4 * j4 + 0]) : 0.f;
                o.y = n + 1 < nval ? __uint_as_float(v[4 * j4 + 1]) : 0.f;
                o.z = n + 2 < nval ? __uint_as_float(v[4 * j4 + 2]) : 0.f;
                o.w = n + 3 < nval ? __uint_as_float(v[4 * j4 + 3]) : 0.f;
                float4* dst = reinterpret_cast<float4*>(ycol + n);
                if (p.accum_y) {
                  const float4 old = *dst;  // padding entries hold 0: adding keeps them 0
                  o.x += old.x;
                  o.y += old.y;
                  o.z += old.z;
                  o.w += old.w;
                }
                *dst = o;
              }
            }
          }
        }
      } else {
        const GCol cs = p.cols[it.seg];
        const bool has_k = cs.k2e > cs.k2b;
        const int nval = min(NMAX, cs.dim - it.n0);
        const int nch = (nval + 31) / 32;
        const bool row_ok = mi < ld;
        float* yrow = yq + mi + ld * (cs.off + it.n0);
        for (int ch = half; ch < nch && has_k; ch += 2) {
          uint32_t v[32];
          tmem_ld32(tmem_base + acc * G_ACC_COLS + ((uint32_t)(32 * q4) << 16) + ch * 32, v);
          if (row_ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int n = ch * 32 + j;
              if (n < nval) yrow[ld * n] += __uint_as_float(v[j]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(acc));
      if (++acc == 2) {
        acc = 0;
        aphase ^= 1u;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(G_TMEM_COLS)
                 : "memory");
  }
}

// the pool in TF32 (rounded to nearest), BF16, and the BF16 rounding of x - bf16(x)
__global__ void k_pool_convert(const double* __restrict__ x, float* __restrict__ o32,
                               __nv_bfloat16* __restrict__ o16, __nv_bfloat16* __restrict__ o16lo,
                               int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float f = (float)x[i];
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(f));
    o32[i] = __uint_as_float(u);
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    o16[i] = h;
    o16lo[i] = __float2bfloat16_rn((float)(x[i] - (double)__bfloat162float(h)));
  }
}

uint64_t hash_vals(const double* a, int rows, int cols, int64_t ld, double sign) {
  uint64_t h = 1469598103934665603ull ^ ((uint64_t)rows << 32 | (uint32_t)cols);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) {
      double x = sign * a[(int64_t)i * ld + j];
      if (x == 0.0) x = 0.0;  // +0 and -0 hash alike
      uint64_t u;
      memcpy(&u, &x, 8);
      h = (h ^ u) * 1099511628211ull;
    }
  return h;
}

PFN_cuTensorMapEncodeTiled_v12000 encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault,
                                         &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)q;
  }
  return fn;
}

int map2d(CUtensorMap* m, const void* base, bool bf16, uint64_t inner, uint64_t outer,
          uint32_t bi, uint32_t bo, CUtensorMapSwizzle swz) {
  auto fn = encode();
  if (!fn) return set_error(DMRG2D_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const uint32_t elt = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * elt};
  cuuint32_t box[2] = {bi, bo};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return set_error(DMRG2D_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DMRG2D_OK;
}

template <typename T>
int gup(GDev* D, const std::vector<T>& h, T** d, int64_t* bytes, cudaStream_t s) {
  *d = nullptr;
  if (h.empty()) return DMRG2D_OK;
  const size_t nb = h.size() * sizeof(T);
  if (cudaMalloc((void**)d, nb) != cudaSuccess) {
    *d = nullptr;
    return set_error(DMRG2D_ENOMEM, "cudaMalloc(%zu) failed (grouped plan)", nb);
  }
  D->allocs.push_back(*d);
  *bytes += (int64_t)nb;
  D2_CUDA(cudaMemcpyAsync(*d, h.data(), nb, cudaMemcpyHostToDevice, s));
  return DMRG2D_OK;
}

const char* kNames[2 * N_ORDERS] = {"128x128 column-slab", "128x128 row-slab", "128x128 longest-first",
                                    "128x256 column-slab", "128x256 row-slab", "128x256 longest-first"};

}  // namespace

std::pair<int, int> BlockPool::add(const double* src, int rows, int cols, int64_t ld) {
  const uint64_t hp = hash_vals(src, rows, cols, ld, 1.0);
  const uint64_t hn = hash_vals(src, rows, cols, ld, -1.0);
  for (size_t i = 0; i < ent.size(); ++i) {
    const Entry& e = ent[i];
    if (e.rows != rows || e.cols != cols || (e.h != hp && e.h != hn)) continue;
    for (int sg = 0; sg < 2; ++sg) {
      const double sign = sg ? -1.0 : 1.0;
      if (e.h != (sg ? hn : hp)) continue;
      bool same = true;
      for (int r = 0; r < rows && same; ++r)
        for (int c = 0; c < cols; ++c)
          if (e.a[(size_t)r * cols + c] != sign * src[(int64_t)r * ld + c]) {
            same = false;
            break;
          }
      if (same) return {(int)i, sg};
    }
  }
  Entry e;
  e.rows = rows;
  e.cols = cols;
  e.h = hp;
  e.a.resize((size_t)rows * cols);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) e.a[(size_t)r * cols + c] = src[(int64_t)r * ld + c];
  ent.push_back(std::move(e));
  return {(int)ent.size() - 1, 0};
}

int gp_num_configs() { return 2 * N_ORDERS; }
const char* gp_config_name(int cfg) {
  return cfg >= 0 && cfg < 2 * N_ORDERS ? kNames[cfg] : "?";
}

int gp_finalise(dmrg2d_ops* ops, GroupPlan* g, cudaStream_t s) {
  if (g->nQ > GQ_MAX)
    return set_error(DMRG2D_EUNSUPPORTED, "%d sectors exceed the grouped kernel's %d", g->nQ,
                     GQ_MAX);
  for (int q = 0; q < g->nQ; ++q)
    if (g->qld[q] % 8 != 0 || g->qbase[q] % 8 != 0)
      return set_error(DMRG2D_EUNSUPPORTED, "V_q not 8-element aligned");
  GDev* D = new GDev();
  g->dev = D;
  // ---- pools: entries laid out row after row, K padded with zeros to a multiple of 64 ----
  auto layout = [&](BlockPool& P, int& KP, int& prow, std::vector<int>& first) {
    KP = 64;
    for (auto& e : P.ent) KP = std::max(KP, (e.cols + 63) / 64 * 64);
    prow = 0;
    first.resize(P.ent.size());
    for (size_t i = 0; i < P.ent.size(); ++i) {
      first[i] = prow;
      prow += P.ent[i].rows;
    }
    prow = std::max(prow, 256);  // never smaller than one TMA box of rows
  };
  std::vector<int> fL, fR;
  layout(g->poolL, D->KPL, D->prL, fL);
  layout(g->poolR, D->KPR, D->prR, fR);
  for (auto& k : g->k1) k.a_pool = fL[k.a_pool];
  for (auto& k : g->k2) k.b_pool = fR[k.b_pool];
  const int copies = std::max(1, g->copies);
  auto fill = [copies](const BlockPool& P, int KP, int prow, const std::vector<int>& first) {
    std::vector<double> h((size_t)copies * std::max(prow, 1) * KP, 0.0);
    for (int cp = 0; cp < copies; ++cp)
      for (size_t i = 0; i < P.ent.size(); ++i)
        for (int r = 0; r < P.ent[i].rows; ++r)
          for (int c = 0; c < P.ent[i].cols; ++c)
            h[((size_t)cp * prow + first[i] + r) * KP + c] =
                P.ent[i].a[(size_t)r * P.ent[i].cols + c];
    return h;
  };
  std::vector<double> hL = fill(g->poolL, D->KPL, D->prL, fL);
  std::vector<double> hR = fill(g->poolR, D->KPR, D->prR, fR);
  // ---- tile lists: two piece widths x three orders ----
  auto cost = [&](const GTile& t) {
    const GRow& r = g->rows[t.rs];
    const GCol& c = g->cols[t.cs];
    long long w = 0;
    for (int e = r.k1b; e < r.k1e; ++e) w += (g->k1[e].kdim + 63) / 64;
    for (int e = c.k2b; e < c.k2e; ++e) w += (g->k2[e].kdim + 63) / 64;
    return w;
  };
  // move range of each destination (row segment, column segment)
  std::unordered_map<long long, std::pair<int, int>> mv_of;
  for (const GMoveDst& md : g->mdst)
    mv_of[(long long)md.rs * (long long)g->cols.size() + md.cs] = {md.mb, md.me};
  auto tile = [&](int r, int c, int ri, int ci) {
    auto it = mv_of.find((long long)r * (long long)g->cols.size() + c);
    const int mb = it == mv_of.end() ? 0 : it->second.first;
    const int me = it == mv_of.end() ? 0 : it->second.second;
    return GTile{r, c, ri, ci, mb, me};
  };
  std::vector<GTile> lists[2][N_ORDERS];
  for (int b = 0; b < 2; ++b) {
    const int bn = b ? 256 : 128;
    std::vector<GTile> colmaj, rowmaj;
    for (int q = 0; q < g->nQ; ++q) {
      for (size_t c = 0; c < g->cols.size(); ++c) {
        if (g->cols[c].q != q) continue;
        for (int ci = 0; ci < g->cols[c].dim; ci += bn)
          for (size_t r = 0; r < g->rows.size(); ++r) {
            if (g->rows[r].q != q) continue;
            for (int ri = 0; ri < g->rows[r].dim; ri += G_BM)
              colmaj.push_back(tile((int)r, (int)c, ri, ci));
          }
      }
      for (size_t r = 0; r < g->rows.size(); ++r) {
        if (g->rows[r].q != q) continue;
        for (int ri = 0; ri < g->rows[r].dim; ri += G_BM)
          for (size_t c = 0; c < g->cols.size(); ++c) {
            if (g->cols[c].q != q) continue;
            for (int ci = 0; ci < g->cols[c].dim; ci += bn)
              rowmaj.push_back(tile((int)r, (int)c, ri, ci));
          }
      }
    }
    std::vector<GTile> lpt = colmaj;
    std::stable_sort(lpt.begin(), lpt.end(),
                     [&](const GTile& x, const GTile& y) { return cost(x) > cost(y); });
    lists[b][0] = colmaj;
    lists[b][1] = rowmaj;
    lists[b][2] = lpt;
  }
  // ---- upload ----
  int64_t* nb = &ops->device_bytes;
  int st = DMRG2D_OK;
  for (int b = 0; b < 2 && st == DMRG2D_OK; ++b)
    for (int o = 0; o < N_ORDERS && st == DMRG2D_OK; ++o) {
      st = gup(D, lists[b][o], &D->tiles[b][o], nb, s);
      D->ntiles[b][o] = (int)lists[b][o].size();
    }
  {  // segment-kernel pieces: pass 1 walks 128-column tiles of each V_q and, within one,
     // its row segments (consecutive pieces read the same V tiles); pass 2 walks 128-row
     // tiles and, within one, the column segments
    std::vector<SItem> s1, s2;
    for (int q = 0; q < g->nQ; ++q) {
      for (int m0 = 0; m0 < g->qcols[q]; m0 += 128)
        for (size_t r = 0; r < g->rows.size(); ++r) {
          if (g->rows[r].q != q) continue;
          for (int n0 = 0; n0 < g->rows[r].dim; n0 += 128) s1.push_back({q, (int)r, n0, m0});
        }
      for (int m0 = 0; m0 < g->qld[q]; m0 += 128)
        for (size_t c = 0; c < g->cols.size(); ++c) {
          if (g->cols[c].q != q) continue;
          for (int n0 = 0; n0 < g->cols[c].dim; n0 += 256) s2.push_back({q, (int)c, n0, m0});
        }
    }
    st = gup(D, s1, &D->sitems[0], nb, s);
    D->nsitems[0] = (int)s1.size();
    if (st == DMRG2D_OK) st = gup(D, s2, &D->sitems[1], nb, s);
    D->nsitems[1] = (int)s2.size();
    if (st == DMRG2D_OK) st = gup(D, g->qcols, &D->d_qcols, nb, s);
  }
  if (st == DMRG2D_OK) st = gup(D, g->rows, &D->rows, nb, s);
  if (st == DMRG2D_OK) st = gup(D, g->cols, &D->cols, nb, s);
  if (st == DMRG2D_OK) st = gup(D, g->k1, &D->k1, nb, s);
  if (st == DMRG2D_OK) st = gup(D, g->k2, &D->k2, nb, s);
  std::vector<GMoveD> mvd;
  mvd.reserve(g->moves.size());
  for (const GMove& m : g->moves) {
    const GRow& r = g->rows[m.rs];
    const GCol& c = g->cols[m.cs];
    if (r.q != c.q) return set_error(DMRG2D_EINVAL, "grouped plan: move across matrices");
    const long long ldq = g->qld[r.q];
    mvd.push_back({g->qbase[r.q] + r.off + ldq * c.off, (int)ldq, m.c});
  }
  if (st == DMRG2D_OK) st = gup(D, mvd, &D->moves, nb, s);
  if (st == DMRG2D_OK) st = gup(D, g->qbase, &D->qbase, nb, s);
  if (st == DMRG2D_OK) st = gup(D, g->qld, &D->qld, nb, s);
  double *dL = nullptr, *dR = nullptr;
  if (st == DMRG2D_OK) st = gup(D, hL, &dL, nb, s);
  if (st == DMRG2D_OK) st = gup(D, hR, &dR, nb, s);
  auto alloc = [&](void** p, size_t bytes) {
    if (st != DMRG2D_OK) return;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      *p = nullptr;
      st = set_error(DMRG2D_ENOMEM, "cudaMalloc(%zu) failed (pools)", bytes);
      return;
    }
    D->allocs.push_back(*p);
    *nb += (int64_t)bytes;
  };
  alloc((void**)&D->pL32, hL.size() * 4);
  alloc((void**)&D->pL16, hL.size() * 2);
  alloc((void**)&D->pL16lo, hL.size() * 2);
  alloc((void**)&D->pR16lo, hR.size() * 2);
  alloc((void**)&D->pR32, hR.size() * 4);
  alloc((void**)&D->pR16, hR.size() * 2);
  alloc((void**)&D->err, sizeof(int));
  if (st == DMRG2D_OK) {
    k_pool_convert<<<1024, 256, 0, s>>>(dL, D->pL32, D->pL16, D->pL16lo, (int64_t)hL.size());
    k_pool_convert<<<1024, 256, 0, s>>>(dR, D->pR32, D->pR16, D->pR16lo, (int64_t)hR.size());
    if (cudaMemsetAsync(D->err, 0, sizeof(int), s) != cudaSuccess)
      st = set_error(DMRG2D_ECUDA, "memset failed");
  }
  if (st == DMRG2D_OK) {
    const int rowsL = std::max(D->prL, 1) * copies, rowsR = std::max(D->prR, 1) * copies;
    D->copies = copies;
    st = map2d(&D->mL[0], D->pL32, false, D->KPL, rowsL, 32, G_BM, CU_TENSOR_MAP_SWIZZLE_128B);
    if (st == DMRG2D_OK)
      st = map2d(&D->mL[1], D->pL16, true, D->KPL, rowsL, 64, G_BM, CU_TENSOR_MAP_SWIZZLE_128B);
    if (st == DMRG2D_OK)
      st = map2d(&D->mLlo, D->pL16lo, true, D->KPL, rowsL, 64, G_BM, CU_TENSOR_MAP_SWIZZLE_128B);
    for (int b = 0; b < 2 && st == DMRG2D_OK; ++b) {
      const bool bf = b == 1;
      st = map2d(&D->mL32[b], bf ? (const void*)D->pL16 : (const void*)D->pL32, bf, D->KPL,
                 rowsL, bf ? 64 : 32, 32, CU_TENSOR_MAP_SWIZZLE_128B);
      if (st == DMRG2D_OK)
        st = map2d(&D->mR32[b], bf ? (const void*)D->pR16 : (const void*)D->pR32, bf, D->KPR,
                   rowsR, bf ? 64 : 32, 32, CU_TENSOR_MAP_SWIZZLE_128B);
    }
    if (st == DMRG2D_OK)
      st = map2d(&D->mL32lo, D->pL16lo, true, D->KPL, rowsL, 64, 32, CU_TENSOR_MAP_SWIZZLE_128B);
    if (st == DMRG2D_OK)
      st = map2d(&D->mR32lo, D->pR16lo, true, D->KPR, rowsR, 64, 32, CU_TENSOR_MAP_SWIZZLE_128B);
    for (int b = 0; b < 2 && st == DMRG2D_OK; ++b) {
      const uint32_t rows_box = b ? 256 : 128;
      st = map2d(&D->mR[0][b], D->pR32, false, D->KPR, rowsR, 32, rows_box,
                 CU_TENSOR_MAP_SWIZZLE_128B);
      if (st == DMRG2D_OK)
        st = map2d(&D->mR[1][b], D->pR16, true, D->KPR, rowsR, 64, rows_box,
                   CU_TENSOR_MAP_SWIZZLE_128B);
      if (st == DMRG2D_OK)
        st = map2d(&D->mRlo[b], D->pR16lo, true, D->KPR, rowsR, 64, rows_box,
                   CU_TENSOR_MAP_SWIZZLE_128B);
    }
  }
  if (st == DMRG2D_OK) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&D->sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(hv_tc_grouped_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(hv_tc_grouped_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(hv_tc_seg_kernel<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(hv_tc_seg_kernel<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(hv_tc_seg_kernel<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(hv_tc_seg_kernel<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)G_SMEM) != cudaSuccess)
      st = set_error(DMRG2D_ECUDA, "cannot set %zu bytes of shared memory", G_SMEM);
  }
  if (st == DMRG2D_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = set_error(DMRG2D_ECUDA, "grouped plan: %s", cudaGetErrorString(e));
  }
  return st;
}

void gp_release(GroupPlan* g) {
  GDev* D = (GDev*)g->dev;
  if (!D) return;
  for (void* p : D->allocs) cudaFree(p);
  delete D;
  g->dev = nullptr;
}

int gp_launch(const dmrg2d_ops* ops, const GroupPlan* g, const void* v, float* y, int precision,
              int cfg, cudaStream_t s, bool fuse_moves, bool lo_ops, bool accum) {
  const GDev* D = (const GDev*)g->dev;
  if (!D) return set_error(DMRG2D_EUNSUPPORTED, "grouped plan not prepared");
  if (cfg < 0 || cfg >= 2 * N_ORDERS) return set_error(DMRG2D_EINVAL, "bad tile config %d", cfg);
  const bool bf = precision == DMRG2D_BF16;
  const int b = cfg / N_ORDERS, o = cfg % N_ORDERS;
  const int bn = b ? 256 : 128;
  const uint32_t BK = bf ? 64 : 32;
  GMaps maps;  // 16 KB: filled per call, copied into the launch parameters
  if (lo_ops && !bf) return set_error(DMRG2D_EINVAL, "low operator parts are BF16 only");
  maps.L = lo_ops ? D->mLlo : D->mL[bf ? 1 : 0];
  maps.R = lo_ops ? D->mRlo[b] : D->mR[bf ? 1 : 0][b];
  const int elt = bf ? 2 : 4;
  const int box_rows = bf ? 64 : 32;
  for (int q = 0; q < g->nQ; ++q) {
    const char* base = (const char*)v + (size_t)g->qbase[q] * elt;
    D2_TRY(map2d(&maps.vk[q], base, bf, (uint64_t)g->qld[q], (uint64_t)g->qcols[q], BK, bn,
                 CU_TENSOR_MAP_SWIZZLE_128B));
    D2_TRY(map2d(&maps.vm[q], base, bf, (uint64_t)g->qld[q], (uint64_t)g->qcols[q],
                 (uint32_t)box_rows, BK,
                 bf ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B));
  }
  GParams p;
  p.ntiles = D->ntiles[b][o];
  p.bn = bn;
  p.BK = (int)BK;
  p.tiles = D->tiles[b][o];
  p.rows = D->rows;
  p.cols = D->cols;
  p.k1 = D->k1;
  p.k2 = D->k2;
  p.qbase = D->qbase;
  p.qld = D->qld;
  p.y = y;
  p.err = D->err;
  p.moves = fuse_moves ? D->moves : nullptr;
  p.v = v;
  const int fmt = bf ? 1 : 2;
  for (int n = 0; n < 2; ++n) {
    p.idesc1[n] = make_idesc(fmt, 0, G_BM, bn, n, 0);
    p.idesc2[n] = make_idesc(fmt, 1, G_BM, bn, 0, n);
  }
  p.a2_box_rows = box_rows;
  p.a2_boxes = G_BM / box_rows;
  p.a2_lbo = (uint32_t)box_rows * BK * elt;
  p.a2_kstep = bf ? 2048 : 1024;
  p.a2_layout = bf ? 2u : 1u;
  p.a2_sbo = bf ? 1024u : 512u;
  p.tx_bytes = G_STAGE_A + (uint32_t)bn * 128;
  p.bf16 = bf ? 1 : 0;
  p.accum_y = accum ? 1 : 0;
  if (p.ntiles == 0) return DMRG2D_OK;
  const int grid = std::min(p.ntiles, D->sms);
  auto ev = prof_slot(ops);
  if (ev.first) D2_CUDA(cudaEventRecord(ev.first, s));
  if (bf)
    hv_tc_grouped_kernel<1><<<grid, G_THREADS, G_SMEM, s>>>(maps, p);
  else
    hv_tc_grouped_kernel<0><<<grid, G_THREADS, G_SMEM, s>>>(maps, p);
  D2_CUDA(cudaGetLastError());
  if (ev.second) D2_CUDA(cudaEventRecord(ev.second, s));
  return DMRG2D_OK;
}

int gp_launch_seg(const dmrg2d_ops* ops, const GroupPlan* g, const void* v, float* y,
                  int precision, cudaStream_t s, bool lo_ops, bool accum) {
  const GDev* D = (const GDev*)g->dev;
  if (!D) return set_error(DMRG2D_EUNSUPPORTED, "grouped plan not prepared");
  if (((uintptr_t)y & 15) != 0)
    return set_error(DMRG2D_EINVAL, "segment kernels: y must be 16-byte aligned");
  const bool bf = precision == DMRG2D_BF16;
  if (lo_ops && !bf) return set_error(DMRG2D_EINVAL, "low operator parts are BF16 only");
  const uint32_t BK = bf ? 64 : 32;
  const int elt = bf ? 2 : 4;
  const int box_rows = bf ? 64 : 32;
  GMaps maps;
  maps.L = lo_ops ? D->mL32lo : D->mL32[bf ? 1 : 0];  // 32-row boxes of the pools
  maps.R = lo_ops ? D->mR32lo : D->mR32[bf ? 1 : 0];
  for (int q = 0; q < g->nQ; ++q) {
    const char* base = (const char*)v + (size_t)g->qbase[q] * elt;
    D2_TRY(map2d(&maps.vk[q], base, bf, (uint64_t)g->qld[q], (uint64_t)g->qcols[q], BK, 128,
                 CU_TENSOR_MAP_SWIZZLE_128B));
    D2_TRY(map2d(&maps.vm[q], base, bf, (uint64_t)g->qld[q], (uint64_t)g->qcols[q],
                 (uint32_t)box_rows, BK,
                 bf ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B));
  }
  SParams p;
  p.rows = D->rows;
  p.cols = D->cols;
  p.k1 = D->k1;
  p.k2 = D->k2;
  p.qbase = D->qbase;
  p.qld = D->qld;
  p.qcols = D->d_qcols;
  p.y = y;
  p.err = D->err;
  p.a2_box_rows = box_rows;
  p.a2_boxes = G_BM / box_rows;
  p.a2_lbo = (uint32_t)box_rows * BK * elt;
  p.a2_kstep = bf ? 2048 : 1024;
  p.a2_layout = bf ? 2u : 1u;
  p.a2_sbo = bf ? 1024u : 512u;
  p.BK = (int)BK;
  p.KSTEP = bf ? 16 : 8;
  const int fmt = bf ? 1 : 2;
  auto ev = prof_slot(ops);
  if (ev.first) D2_CUDA(cudaEventRecord(ev.first, s));
  for (int pass = 0; pass < 2; ++pass) {
    p.nitems = D->nsitems[pass];
    p.items = D->sitems[pass];
    p.accum_y = accum ? 1 : 0;
    for (int i = 0; i < 16; ++i)
      for (int n = 0; n < 2; ++n) p.idesc[i][n] = make_idesc(fmt, pass, G_BM, 16 * (i + 1), 0, n);
    // A = the V tile (16 KB); B = 32-row boxes of operator rows (4 KB each)
    p.a_bytes = G_STAGE_A;
    p.b_box_bytes = 32 * 128;
    if (p.nitems == 0) continue;
    const int grid = std::min(p.nitems, D->sms);
    if (bf) {
      if (pass) hv_tc_seg_kernel<1, 1><<<grid, G_THREADS, G_SMEM, s>>>(maps, p);
      else hv_tc_seg_kernel<1, 0><<<grid, G_THREADS, G_SMEM, s>>>(maps, p);
    } else {
      if (pass) hv_tc_seg_kernel<0, 1><<<grid, G_THREADS, G_SMEM, s>>>(maps, p);
      else hv_tc_seg_kernel<0, 0><<<grid, G_THREADS, G_SMEM, s>>>(maps, p);
    }
    D2_CUDA(cudaGetLastError());
  }
  if (ev.second) D2_CUDA(cudaEventRecord(ev.second, s));
  return DMRG2D_OK;
}

int gp_pool_views(const GroupPlan* g, int precision, int bn, const CUtensorMap** mL,
                  const CUtensorMap** mR, const GK1** k1, const GK2** k2, int* rowsL, int* rowsR,
                  int* copies) {
  const GDev* D = g ? (const GDev*)g->dev : nullptr;
  if (!D) return set_error(DMRG2D_EUNSUPPORTED, "grouped plan not prepared");
  const int pi = precision == DMRG2D_BF16 ? 1 : 0;
  *mL = &D->mL[pi];
  *mR = &D->mR[pi][bn == 256 ? 1 : 0];
  *k1 = D->k1;
  *k2 = D->k2;
  *rowsL = std::max(D->prL, 1);  // replica r of a pool starts at row r * rows
  *rowsR = std::max(D->prR, 1);
  *copies = D->copies;
  return DMRG2D_OK;
}

int gp_read_error(const GroupPlan* g, int* code) {
  *code = 0;
  const GDev* D = g ? (const GDev*)g->dev : nullptr;
  if (!D || !D->err) return DMRG2D_OK;
  D2_CUDA(cudaMemcpy(code, D->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (*code) D2_CUDA(cudaMemset(D->err, 0, sizeof(int)));
  return DMRG2D_OK;
}

}  // namespace dmrg2d
