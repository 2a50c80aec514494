// Superblock H·v on the 5th-generation tensor cores (tcgen05, sm_103a), TF32 or BF16
// operands with FP32 accumulation in tensor memory.
//
// Output tile (i2, i3) of Y = H_l V + V H_r^T + H_c V_c (paper, text after Eq. (dec)) is
// split into 128 x BN pieces (rows i1 of block row i2, columns i4 of block column i3).
// For one piece the K loop runs over
//   phase 1 (H_l V):   A = HL[i2,i2'] rows, K-major       B = V(i2' rows, i3 cols), K-major
//   phase 2 (V H_r^T): A = V(i2 rows, i3' cols), MN-major  B = HR[i3,i3'] rows, K-major
// into ONE accumulator, so Y is written once.  The epilogue adds the scalar tile moves
// (H_c, off-diagonal column terms), Y(i2,i3) += c V(i2',i3'), reading the source rows
// from L2 while the MMAs of the next piece run in the other accumulator.
//
// Kernel organisation (one persistent CTA per SM, 320 threads):
//   warp 0   TMA producer: 4-stage ring of 48 KB (A 16 KB + B up to 32 KB), 128B swizzle
//   warp 1   TMEM owner (512 columns = two 128 x 256 FP32 accumulators) and MMA issuer
//   warps 2-9 epilogue: tcgen05.ld of the finished accumulator, scalar moves, FP32 stores
// Every mbarrier wait is bounded (globaltimer); on timeout the CTA raises an error flag,
// stops issuing work, releases its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.h"
#include "grouped.h"
#include "tc_ptx.cuh"

namespace dmrg2d {

namespace {

using namespace tc;

constexpr int TC_THREADS = 320;  // producer, MMA issuer, 8 epilogue warps
constexpr int EPI_WARPS = 8;
constexpr int STAGES = 4;
constexpr int BM = 128;
constexpr uint32_t STAGE_A = 16384;
constexpr uint32_t STAGE_B = 32768;
constexpr uint32_t STAGE_BYTES = STAGE_A + STAGE_B;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COLS = 256;
constexpr size_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;

struct TcParams {
  int m1, m4, d, BN;
  int n_mt, n_nt;
  int tiles;
  const int* order;  // piece order (column-slab numbering), nullptr: column-slab order
  int kblk1, kblk2;
  int BK;
  int64_t ld;
  const int* Lptr;
  const int* Lcol;
  const int* Rptr;
  const int* Rcol;
  float* y;
  int* err;
  uint32_t idesc1[2], idesc2[2];  // [negate the operator block]
  uint32_t a2_lbo, a2_sbo, a2_kstep, a2_layout;
  int a2_boxes, a2_box_rows;
  uint32_t tx_bytes;
  int bf16;
  // operator blocks from the deduplicated pool: entry e of H_l / H_r reads pool rows
  // k1[e].a_pool / k2[e].b_pool, negated when .neg is set (pooled = 0: block e itself)
  int pooled;
  const GK1* k1;
  const GK2* k2;
  int poolL_rows, poolR_rows, copies;  // rows of one pool replica; replicas
  // phases run by this launch: [ph0, ph1) of {0: H_l V, 1: V H_r^T}; accum_y: the
  // epilogue adds the Y already stored (second pass of the two-pass form)
  int ph0, ph1, accum_y;
  // the phase-2 V operand in one 3-D box (its a2_boxes row blocks) instead of a2_boxes 2-D
  // boxes; the shared-memory image is the same
  int a2_3d;
  // scalar tile moves fused into the epilogue (H_c and off-diagonal column terms)
  int fuse;
  const void* v;
  const int* Cptr;
  const int* Csrc;
  const float* Cval;
};

struct TileCoord {
  int i2, mt, i3, nt;
};
__device__ __forceinline__ TileCoord decode(const TcParams& p, int t) {
  if (p.order) t = __ldg(p.order + t);
  const int nm = p.d * p.n_mt;
  const int mg = t % nm, ng = t / nm;  // consecutive tiles walk down one column slab of V
  return {mg / p.n_mt, mg % p.n_mt, ng / p.n_nt, ng % p.n_nt};
}

// Epilogue of one piece (rows mt*128.. of block row i2, columns of block column i3 / nt):
// accumulator columns from tensor memory at tacc, plus the scalar tile moves, stored to Y.
// Warp (q, half) handles TMEM lane quadrant q and half of the 32-column chunks.
__device__ __forceinline__ void epilogue_piece(const TcParams& p, const TileCoord& c, int mt,
                                               uint32_t tacc, int q, int half, int lane) {
  const int row = 32 * q + lane;
  const int64_t r = (int64_t)c.i2 * p.m1 + mt * BM + row;
  const int64_t col0 = (int64_t)c.i3 * p.m4 + (int64_t)c.nt * p.BN;
  const int tt = c.i2 + p.d * c.i3;
  const int e0 = p.fuse ? p.Cptr[tt] : 0, e1 = p.fuse ? p.Cptr[tt + 1] : 0;
  const int nch = p.BN / 32;
  for (int ch = half * (nch / 2); ch < (half + 1) * (nch / 2); ++ch) {
    uint32_t v[32];
    tmem_ld32(tacc + ((uint32_t)(32 * q) << 16) + ch * 32, v);
    float o[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) o[j] = __uint_as_float(v[j]);
    // scalar tile moves of this piece: Y(i2,i3) += c V(i2',i3') on the same rows and
    // columns of the source tile; a warp reads 32 consecutive rows per column, MV moves
    // at a time (MV x 32 loads in flight per thread: the moves are bound by the loads in
    // flight; four spill registers)
    constexpr int MV = 3;
    for (int e = e0; e < e1; e += MV) {
      float cm[MV];
      int64_t off[MV];
#pragma unroll
      for (int m = 0; m < MV; ++m) {
        const bool have = e + m < e1;
        const int sm = p.Csrc[have ? e + m : e];
        cm[m] = have ? p.Cval[e + m] : 0.f;
        const int64_t rm = (int64_t)(sm % p.d) * p.m1 + mt * BM + row;
        const int64_t km = (int64_t)(sm / p.d) * p.m4 + (int64_t)c.nt * p.BN + ch * 32;
        off[m] = rm + p.ld * km;
      }
      float vm[MV][32];
      if (p.bf16) {
#pragma unroll
        for (int m = 0; m < MV; ++m) {
          const __nv_bfloat16* A = (const __nv_bfloat16*)p.v + off[m];
#pragma unroll
          for (int j = 0; j < 32; ++j) vm[m][j] = __bfloat162float(A[p.ld * j]);
        }
      } else {
#pragma unroll
        for (int m = 0; m < MV; ++m) {
          const float* A = (const float*)p.v + off[m];
#pragma unroll
          for (int j = 0; j < 32; ++j) vm[m][j] = __ldg(A + p.ld * j);
        }
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        float s = o[j];
#pragma unroll
        for (int m = 0; m < MV; ++m) s = fmaf(cm[m], vm[m][j], s);
        o[j] = s;
      }
    }
    float* yp = p.y + r + p.ld * (col0 + ch * 32);
    if (p.accum_y) {
#pragma unroll
      for (int j = 0; j < 32; ++j) o[j] += yp[p.ld * j];
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) yp[p.ld * j] = o[j];
  }
}

template <int BF16>
__global__ void __launch_bounds__(TC_THREADS, 1)
hv_tc_kernel(const __grid_constant__ CUtensorMap mHL, const __grid_constant__ CUtensorMap mHR,
             const __grid_constant__ CUtensorMap mVk, const __grid_constant__ CUtensorMap mVm,
             const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 4);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + STAGES + s); };
  auto tfull = [&](int b) { return smem_u32(bars + 2 * STAGES + b); };
  auto tempty = [&](int b) { return smem_u32(bars + 2 * STAGES + 2 + b); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), EPI_WARPS);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------- TMA producer -------------------------------
    int stage = 0;
    uint32_t phase = 0;
    for (int t = blockIdx.x; t < p.tiles && !*abort; t += gridDim.x) {
      const TileCoord c = decode(p, t);
      const int r0 = c.i2 * p.m1 + c.mt * BM;
      const int c0 = c.i3 * p.m4 + c.nt * p.BN;
      for (int ph = p.ph0; ph < p.ph1; ++ph) {
        const int e0 = ph == 0 ? p.Lptr[c.i2] : p.Rptr[c.i3];
        const int e1 = ph == 0 ? p.Lptr[c.i2 + 1] : p.Rptr[c.i3 + 1];
        const int kb = ph == 0 ? p.kblk1 : p.kblk2;
        for (int e = e0; e < e1; ++e) {
          const int nb = ph == 0 ? p.Lcol[e] : p.Rcol[e];
          for (int kc = 0; kc < kb; ++kc) {
            if (!mbar_wait(empty(stage), phase ^ 1u, abort)) {
              raise_abort(abort, p.err, 1);
              goto producer_done;
            }
            const uint32_t a_s = smem_u32(smem + stage * STAGE_BYTES);
            const uint32_t b_s = a_s + STAGE_A;
            mbar_expect_tx(full(stage), p.tx_bytes);
            if (ph == 0) {
              tma_load_2d(a_s, &mHL, full(stage), kc * p.BK,
                          (p.pooled ? p.k1[e].a_pool + (int)(blockIdx.x % p.copies) * p.poolL_rows
                                    : e * p.m1) +
                              c.mt * BM);
              tma_load_2d(b_s, &mVk, full(stage), nb * p.m1 + kc * p.BK, c0);
            } else {
              if (p.a2_3d)
                tma_load_3d(a_s, &mVm, full(stage), 0, nb * p.m4 + kc * p.BK, r0 / p.a2_box_rows);
              else
                for (int b = 0; b < p.a2_boxes; ++b)
                  tma_load_2d(a_s + b * p.a2_lbo, &mVm, full(stage), r0 + b * p.a2_box_rows,
                              nb * p.m4 + kc * p.BK);
              tma_load_2d(b_s, &mHR, full(stage), kc * p.BK,
                          (p.pooled ? p.k2[e].b_pool + (int)(blockIdx.x % p.copies) * p.poolR_rows
                                    : e * p.m4) +
                              c.nt * p.BN);
            }
            if (++stage == STAGES) {
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
    for (int t = blockIdx.x; t < p.tiles && !*abort; t += gridDim.x) {
      const TileCoord c = decode(p, t);
      if (!mbar_wait(tempty(acc), aphase ^ 1u, abort)) {
        raise_abort(abort, p.err, 2);
        break;
      }
      tc_fence_after();
      const uint32_t dt = tmem_base + acc * ACC_COLS;
      uint32_t accum = 0;
      bool ok = true;
      for (int ph = p.ph0; ph < p.ph1 && ok; ++ph) {
        const int e0 = ph == 0 ? p.Lptr[c.i2] : p.Rptr[c.i3];
        const int e1 = ph == 0 ? p.Lptr[c.i2 + 1] : p.Rptr[c.i3 + 1];
        const int kb = ph == 0 ? p.kblk1 : p.kblk2;
        // descriptor fields fixed for the phase (the A operand of phase 2 is V, MN-major)
        const uint64_t a_hi = ph == 0 ? sdesc(0, 16, 1024)
                                      : sdesc(0, p.a2_lbo, p.a2_sbo, p.a2_layout);
        const uint32_t a_step = ph == 0 ? 32u : p.a2_kstep;
        const uint64_t b_hi = sdesc(0, 16, 1024);
        for (int e = e0; e < e1 && ok; ++e) {
          // instruction descriptor of this operator block, chosen once per block
          const int neg = p.pooled ? (ph == 0 ? p.k1[e].neg : p.k2[e].neg) : 0;
          const uint32_t idb = ph == 0 ? (neg ? p.idesc1[1] : p.idesc1[0])
                                       : (neg ? p.idesc2[1] : p.idesc2[0]);
          for (int kc = 0; kc < kb; ++kc) {
            // the mbarrier's completion orders the TMA writes before these MMAs; no
            // tcgen05 fence is needed per stage
            if (!mbar_wait(full(stage), phase, abort)) {
              raise_abort(abort, p.err, 3);
              ok = false;
              break;
            }
            const uint32_t a_s = smem_u32(smem + stage * STAGE_BYTES);
            const uint32_t b_s = a_s + STAGE_A;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              umma_t<BF16>(dt, a_hi | sdesc_addr(a_s + k * a_step),
                           b_hi | sdesc_addr(b_s + k * 32), idb, accum);
              accum = 1;
            }
            umma_commit(empty(stage));
            stage = stage + 1 == STAGES ? 0 : stage + 1;
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
    const int q = warp & 3;             // TMEM lane quadrant this warp may access
    const int half = (warp - 2) >> 2;   // two warps per quadrant split the column chunks
    int acc = 0;
    uint32_t aphase = 0;
    for (int t = blockIdx.x; t < p.tiles; t += gridDim.x) {
      const TileCoord c = decode(p, t);
      if (!mbar_wait(tfull(acc), aphase, abort)) {
        raise_abort(abort, p.err, 4);
        break;
      }
      tc_fence_after();
      epilogue_piece(p, c, c.mt, tmem_base + acc * ACC_COLS, q, half, lane);
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
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---- CTA-pair variant (cluster of 2, tcgen05 cta_group::2) -------------------------------
// The two CTAs of a cluster compute one 256 x BN tile (both 128-row pieces of a 256-row
// block row) with M = 256 MMAs issued by the even CTA: each CTA stages its own 128 rows
// of A and HALF of the B columns, so a stage is 32 KB instead of 48 KB per SM, six stages
// fit, and the B bytes each SM pulls from L2 halve.  The accumulator rows of CTA r live
// in its own tensor memory; its epilogue warps handle piece mt = 2 * pair + r as in the
// single-CTA kernel.
//   full[s]   (even CTA) : its producer's expect_tx for both CTAs' bytes; both CTAs'
//                          TMA loads complete on it
//   empty[s]  (both)     : multicast commit after the MMAs that read stage s
//   tfull[b]  (both)     : multicast commit after the last MMA of a tile
//   tempty[b] (even CTA) : one arrival per epilogue warp of both CTAs
// Both CTAs meet at cluster barriers after set-up and before releasing tensor memory, so
// neither exits while the other may still touch its shared or tensor memory.
constexpr int P_STAGES = 6;
constexpr uint32_t P_STAGE_A = 16384;
constexpr uint32_t P_STAGE = 32768;  // A 128 rows + B 128 columns, BK of K
constexpr size_t P_SMEM = P_STAGES * P_STAGE + 1024 + 256;
constexpr int P_HALF = 128;          // B columns per CTA

template <int BF16>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
hv_tc_pair_kernel(const __grid_constant__ CUtensorMap mHL, const __grid_constant__ CUtensorMap mHR,
                  const __grid_constant__ CUtensorMap mVk, const __grid_constant__ CUtensorMap mVm,
                  const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + P_STAGES * P_STAGE);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * P_STAGES + 4);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const bool even = rank == 0;
  auto full = [&](int s) { return smem_u32(bars + s); };
  auto empty = [&](int s) { return smem_u32(bars + P_STAGES + s); };
  auto tfull = [&](int b) { return smem_u32(bars + 2 * P_STAGES + b); };
  auto tempty = [&](int b) { return smem_u32(bars + 2 * P_STAGES + 2 + b); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), 2 * EPI_WARPS);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {  // one warp of each CTA allocates the pair's tensor memory together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int cid = (int)cluster_id_x(), ncl = (int)ncluster_x();

  if (warp == 0 && lane == 0) {
    // ------------------------- TMA producer (both CTAs) -------------------------
    int stage = 0;
    uint32_t phase = 0;
    for (int t = cid; t < p.tiles && !*abort; t += ncl) {
      const TileCoord c = decode(p, t);  // c.mt: pair of 128-row pieces
      const int mt = 2 * c.mt + (int)rank;
      const int r0 = c.i2 * p.m1 + mt * BM;
      const int cb = c.nt * p.BN + (int)rank * P_HALF;  // this CTA's B columns
      for (int ph = p.ph0; ph < p.ph1; ++ph) {
        const int e0 = ph == 0 ? p.Lptr[c.i2] : p.Rptr[c.i3];
        const int e1 = ph == 0 ? p.Lptr[c.i2 + 1] : p.Rptr[c.i3 + 1];
        const int kb = ph == 0 ? p.kblk1 : p.kblk2;
        for (int e = e0; e < e1; ++e) {
          const int nb = ph == 0 ? p.Lcol[e] : p.Rcol[e];
          for (int kc = 0; kc < kb; ++kc) {
            if (!mbar_wait(empty(stage), phase ^ 1u, abort)) {
              raise_abort(abort, p.err, 11);
              goto producer_done;
            }
            const uint32_t a_s = smem_u32(smem + stage * P_STAGE);
            const uint32_t b_s = a_s + P_STAGE_A;
            if (even) mbar_expect_tx(full(stage), 2 * p.tx_bytes);
            const uint32_t fb = mapa(full(stage), 0);
            if (ph == 0) {
              const int arow = p.pooled ? p.k1[e].a_pool + (int)(cid % p.copies) * p.poolL_rows
                                        : e * p.m1;
              tma_load_2d_pair(a_s, &mHL, fb, kc * p.BK, arow + mt * BM);
              tma_load_2d_pair(b_s, &mVk, fb, nb * p.m1 + kc * p.BK, c.i3 * p.m4 + cb);
            } else {
              if (p.a2_3d)
                tma_load_3d_pair(a_s, &mVm, fb, 0, nb * p.m4 + kc * p.BK, r0 / p.a2_box_rows);
              else
                for (int b = 0; b < p.a2_boxes; ++b)
                  tma_load_2d_pair(a_s + b * p.a2_lbo, &mVm, fb, r0 + b * p.a2_box_rows,
                                   nb * p.m4 + kc * p.BK);
              const int brow = p.pooled ? p.k2[e].b_pool + (int)(cid % p.copies) * p.poolR_rows
                                        : e * p.m4;
              tma_load_2d_pair(b_s, &mHR, fb, kc * p.BK, brow + cb);
            }
            if (++stage == P_STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
    }
  producer_done:;
  } else if (warp == 1 && lane == 0 && even) {
    // ------------------------- MMA issuer (even CTA) ----------------------------
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t aphase = 0;
    for (int t = cid; t < p.tiles && !*abort; t += ncl) {
      const TileCoord c = decode(p, t);
      if (!mbar_wait(tempty(acc), aphase ^ 1u, abort)) {
        raise_abort(abort, p.err, 12);
        break;
      }
      tc_fence_after();
      const uint32_t dt = tmem_base + acc * ACC_COLS;
      uint32_t accum = 0;
      bool ok = true;
      for (int ph = p.ph0; ph < p.ph1 && ok; ++ph) {
        const int e0 = ph == 0 ? p.Lptr[c.i2] : p.Rptr[c.i3];
        const int e1 = ph == 0 ? p.Lptr[c.i2 + 1] : p.Rptr[c.i3 + 1];
        const int kb = ph == 0 ? p.kblk1 : p.kblk2;
        // descriptor fields fixed for the phase (the A operand of phase 2 is V, MN-major)
        const uint64_t a_hi = ph == 0 ? sdesc(0, 16, 1024)
                                      : sdesc(0, p.a2_lbo, p.a2_sbo, p.a2_layout);
        const uint32_t a_step = ph == 0 ? 32u : p.a2_kstep;
        const uint64_t b_hi = sdesc(0, 16, 1024);
        for (int e = e0; e < e1 && ok; ++e) {
          // instruction descriptor of this operator block, chosen once per block
          const int neg = p.pooled ? (ph == 0 ? p.k1[e].neg : p.k2[e].neg) : 0;
          const uint32_t idb = ph == 0 ? (neg ? p.idesc1[1] : p.idesc1[0])
                                       : (neg ? p.idesc2[1] : p.idesc2[0]);
          for (int kc = 0; kc < kb; ++kc) {
            // the mbarrier's completion orders the TMA writes before these MMAs; no
            // tcgen05 fence is needed per stage
            if (!mbar_wait(full(stage), phase, abort)) {
              raise_abort(abort, p.err, 13);
              ok = false;
              break;
            }
            const uint32_t a_s = smem_u32(smem + stage * P_STAGE);
            const uint32_t b_s = a_s + P_STAGE_A;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              umma_pair_t<BF16>(dt, a_hi | sdesc_addr(a_s + k * a_step),
                                b_hi | sdesc_addr(b_s + k * 32), idb, accum);
              accum = 1;
            }
            umma_commit_pair(empty(stage));
            stage = stage + 1 == P_STAGES ? 0 : stage + 1;
            phase ^= stage == 0 ? 1u : 0u;
          }
        }
      }
      if (!ok) break;
      umma_commit_pair(tfull(acc));
      if (++acc == 2) {
        acc = 0;
        aphase ^= 1u;
      }
    }
  } else if (warp >= 2) {
    // ------------------------- epilogue (both CTAs) -----------------------------
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint32_t te0 = mapa(tempty(0), 0), te1 = mapa(tempty(1), 0);
    int acc = 0;
    uint32_t aphase = 0;
    for (int t = cid; t < p.tiles; t += ncl) {
      const TileCoord c = decode(p, t);
      if (!mbar_wait(tfull(acc), aphase, abort)) {
        raise_abort(abort, p.err, 14);
        break;
      }
      tc_fence_after();
      epilogue_piece(p, c, 2 * c.mt + (int)rank, tmem_base + acc * ACC_COLS, q, half, lane);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(acc ? te1 : te0);
      if (++acc == 2) {
        acc = 0;
        aphase ^= 1u;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Self-test of the bounded waits: one thread waits on an mbarrier that nothing arrives on,
// with the same routine the tensor-core kernels use, gives up after limit_ns, and records
// the give-up in *err as the kernels do (site 99).
__global__ void k_wait_selftest(int* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  mbar_init(smem_u32(&bar), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(smem_u32(&bar), 0, (volatile int*)&abort_flag, limit_ns))
    raise_abort((volatile int*)&abort_flag, err, 99);
}

// ---- host side ----------------------------------------------------------------------------
struct TcState {
  bool dense_ok = false;
  GroupPlan* plan = nullptr;  // grouped form of the same superblock (m1 % 8 == 0)
  float* HLt = nullptr;  // TF32-rounded copies of the operator blocks
  float* HRt = nullptr;
  int* err = nullptr;
  int* order = nullptr;   // blocked piece order of the dense kernel
  int* order2 = nullptr;  // the same for the CTA-pair kernel (256-row pieces)
  int* order2p[2] = {nullptr, nullptr};  // the CTA-pair kernel in 4 x 4 / 16 x 16 patches
  // two-pass form: pass A (H_l V, column-slab order) and pass B (V H_r^T, row-slab
  // order), for 128-row pieces [0] and CTA-pair pieces [1]; the scalar moves split so
  // that each pass reads the sources its order keeps in L2
  int* orderA[2] = {nullptr, nullptr};
  int* orderB[2] = {nullptr, nullptr};
  int *CptrA = nullptr, *CsrcA = nullptr, *CptrB = nullptr, *CsrcB = nullptr;
  float *CvalA = nullptr, *CvalB = nullptr;
  bool pair_ok = false;   // CTA-pair kernel applies (m1 % 256 == 0, 256-wide pieces)
  int pairs = 0;          // CTA pairs resident at once (persistent grid of the pair kernel)
  CUtensorMap mHR2[2];    // H_r blocks in 128-row boxes (half a piece's columns)
  CUtensorMap mHL[2], mHR[2];  // [0] TF32, [1] BF16
  // BF16X3: the low BF16 parts of the operator blocks, x - bf16(x) rounded to BF16
  __nv_bfloat16* HLlo = nullptr;
  __nv_bfloat16* HRlo = nullptr;
  CUtensorMap mHLlo, mHRlo, mHR2lo;
  int sms = 0;
  int BN = 0;
};

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

int make_map(CUtensorMap* m, const void* base, bool bf16, uint64_t inner, uint64_t outer,
             uint32_t box_inner, uint32_t box_outer,
             CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  auto fn = encode_fn();
  if (!fn) return set_error(DMRG2D_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const uint32_t elt = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * elt};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(DMRG2D_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DMRG2D_OK;
}

// lo = the BF16 rounding of x - bf16(x): with hi = bf16(x), hi + lo carries ~16 bits of x
__global__ void k_bf16_lo(const double* __restrict__ x, __nv_bfloat16* __restrict__ o, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double hi = (double)__bfloat162float(__float2bfloat16_rn((float)x[i]));
    o[i] = __float2bfloat16_rn((float)(x[i] - hi));
  }
}

// A 3-D view of a column-major matrix with leading dimension ld: dim 0 = a row within a
// block of d0 rows, dim 1 = the column (stride ld), dim 2 = the row block (stride d0); one
// box {d0, b1, b2} lands in shared memory as b2 consecutive {d0, b1} tiles.
int make_map3(CUtensorMap* m, const void* base, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2,
              uint64_t ld, uint32_t b0, uint32_t b1, uint32_t b2, CUtensorMapSwizzle swz) {
  auto fn = encode_fn();
  if (!fn) return set_error(DMRG2D_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const uint64_t elt = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {ld * elt, d0 * elt};
  cuuint32_t box[3] = {b0, b1, b2};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                  const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return set_error(DMRG2D_EUNSUPPORTED, "3-D tensor map rejected (%d)", (int)r);
  return DMRG2D_OK;
}

__global__ void k_round_tf32(const double* __restrict__ x, float* __restrict__ o, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float f = (float)x[i];
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(f));
    o[i] = __uint_as_float(u);
  }
}


// Blocked piece order of the dense kernel.  A piece (i2, mt, i3, nt) reads the column
// operators' neighbours of i2 (phase 1, column slab i3), of i3 (phase 2, row slab i2)
// and the scalar-move sources; the column-slab order streams all of H_l through L2 once
// per wave.  Here consecutive pieces cover a B x B patch of output tiles (i2, i3), with
// both halves mt (and all nt) of a tile next to each other, so one wave touches B rows
// of H_l, B rows of H_r and the V tiles around the patch.  Patches follow a Gray code of
// their linear index when both patch counts are powers of two (one patch coordinate
// bit changes per step: for column bases whose operators flip bits of the state label,
// successive patches share neighbours), else a serpentine walk.  Returns column-slab
// numbers (t = i2 n_mt + mt + d n_mt (i3 n_nt + nt)).
// tc_cfg value of the CTA-pair kernel in blocked order (dense-kernel variant 6)
constexpr int kPairBlockedCfg = -1 - 6;

std::vector<int> blocked_order(int d, int n_mt, int n_nt, int B) {
  const int nb = (d + B - 1) / B;
  const bool pow2 = (nb & (nb - 1)) == 0;
  std::vector<int> out;
  out.reserve((size_t)d * n_mt * d * n_nt);
  for (int h = 0; h < nb * nb; ++h) {
    int h2, h3;
    if (pow2) {
      const int g = h ^ (h >> 1);
      h2 = g % nb;
      h3 = g / nb;
    } else {
      h3 = h / nb;
      h2 = (h3 & 1) ? nb - 1 - h % nb : h % nb;
    }
    for (int i3 = h3 * B; i3 < std::min(d, (h3 + 1) * B); ++i3)
      for (int i2 = h2 * B; i2 < std::min(d, (h2 + 1) * B); ++i2)
        for (int nt = 0; nt < n_nt; ++nt)
          for (int mt = 0; mt < n_mt; ++mt)
            out.push_back(i2 * n_mt + mt + d * n_mt * (i3 * n_nt + nt));
  }
  return out;
}

// Orders of the two-pass form (column-slab numbers, as blocked_order).  Pass A walks one
// block column i3 at a time (all pieces of the column, so H_l V reads each V tile of the
// column from L2 once it is there); pass B walks one block row i2 at a time.  Columns
// (rows) follow a Gray code when d is a power of two, so consecutive slabs differ in one
// bit of the state label and share the sources of the moves between slabs.
std::vector<int> slab_order(int d, int n_mt, int n_nt, bool columns) {
  const bool pow2 = (d & (d - 1)) == 0;
  std::vector<int> out;
  out.reserve((size_t)d * n_mt * d * n_nt);
  for (int a = 0; a < d; ++a) {
    const int s = pow2 ? (a ^ (a >> 1)) : a;
    for (int b = 0; b < d; ++b) {
      const int i2 = columns ? b : s, i3 = columns ? s : b;
      for (int nt = 0; nt < n_nt; ++nt)
        for (int mt = 0; mt < n_mt; ++mt)
          out.push_back(i2 * n_mt + mt + d * n_mt * (i3 * n_nt + nt));
    }
  }
  return out;
}

}  // namespace

int tc_prepare(dmrg2d_ops* ops, cudaStream_t s, const std::vector<double>& HL,
               const std::vector<double>& HR) {
  ops->tc_ok = 0;
  if (ops->sec) return DMRG2D_OK;  // sector-restricted superblocks build their own plan
  const int m1 = ops->m1, m4 = ops->m4, d = ops->d;
  if (!encode_fn()) return DMRG2D_OK;
  const bool dense_ok = m1 % BM == 0 && (m4 == 128 || m4 % 256 == 0);
  const bool grouped_ok = m1 % 8 == 0;
  if (!dense_ok && !grouped_ok) return DMRG2D_OK;  // CUDA-core path only
  TcState* T = new TcState();
  ops->tc = T;
  T->dense_ok = dense_ok;
  T->BN = m4 == 128 ? 128 : 256;
  const int64_t nL = ops->dev.nL, nR = ops->dev.nR;
  int st = DMRG2D_OK;
  auto alloc = [&](void** p, size_t b) {
    if (st != DMRG2D_OK) return;
    if (cudaMalloc(p, b) != cudaSuccess) {
      *p = nullptr;
      st = set_error(DMRG2D_ENOMEM, "cudaMalloc(%zu) failed", b);
    } else {
      ops->device_bytes += (int64_t)b;
    }
  };
  alloc((void**)&T->err, sizeof(int));
  if (st == DMRG2D_OK && cudaMemsetAsync(T->err, 0, sizeof(int), s) != cudaSuccess)
    st = set_error(DMRG2D_ECUDA, "memset failed");
  if (dense_ok) {
    alloc((void**)&T->HLt, sizeof(float) * nL * m1 * m1);
    alloc((void**)&T->HRt, sizeof(float) * nR * m4 * m4);
    alloc((void**)&T->HLlo, sizeof(__nv_bfloat16) * nL * m1 * m1);
    alloc((void**)&T->HRlo, sizeof(__nv_bfloat16) * nR * m4 * m4);
    if (st == DMRG2D_OK) {
      k_round_tf32<<<1024, 256, 0, s>>>(ops->dev.HL64, T->HLt, nL * m1 * m1);
      k_round_tf32<<<1024, 256, 0, s>>>(ops->dev.HR64, T->HRt, nR * m4 * m4);
      k_bf16_lo<<<1024, 256, 0, s>>>(ops->dev.HL64, T->HLlo, nL * m1 * m1);
      k_bf16_lo<<<1024, 256, 0, s>>>(ops->dev.HR64, T->HRlo, nR * m4 * m4);
    }
    if (st == DMRG2D_OK) st = make_map(&T->mHLlo, T->HLlo, true, m1, nL * m1, 64, BM);
    if (st == DMRG2D_OK) st = make_map(&T->mHRlo, T->HRlo, true, m4, nR * m4, 64, T->BN);
    for (int b = 0; b < 2 && st == DMRG2D_OK; ++b) {
      const bool bf = b == 1;
      const uint32_t BK = bf ? 64 : 32;
      const void* hl = bf ? (const void*)ops->dev.HL16 : (const void*)T->HLt;
      const void* hr = bf ? (const void*)ops->dev.HR16 : (const void*)T->HRt;
      st = make_map(&T->mHL[b], hl, bf, m1, nL * m1, BK, BM);
      if (st == DMRG2D_OK) st = make_map(&T->mHR[b], hr, bf, m4, nR * m4, BK, T->BN);
    }
    T->pair_ok = m1 % 256 == 0 && T->BN == 256;
    for (int b = 0; b < 2 && st == DMRG2D_OK && T->pair_ok; ++b) {
      const bool bf = b == 1;
      st = make_map(&T->mHR2[b], bf ? (const void*)ops->dev.HR16 : (const void*)T->HRt, bf, m4,
                    nR * m4, bf ? 64 : 32, P_HALF);
    }
    if (st == DMRG2D_OK && T->pair_ok)
      st = make_map(&T->mHR2lo, T->HRlo, true, m4, nR * m4, 64, P_HALF);
    auto upload_order = [&](int** dst, int pieces_mt, int patch = 8) {
      const std::vector<int> ord = blocked_order(d, pieces_mt, m4 / T->BN, patch);
      alloc((void**)dst, sizeof(int) * ord.size());
      if (st == DMRG2D_OK &&
          cudaMemcpy(*dst, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice) !=
              cudaSuccess)
        st = set_error(DMRG2D_ECUDA, "order upload failed");
    };
    upload_order(&T->order, m1 / BM);
    if (T->pair_ok) {
      upload_order(&T->order2, m1 / 256);
      upload_order(&T->order2p[0], m1 / 256, 4);
      upload_order(&T->order2p[1], m1 / 256, 16);
    }
    // two-pass form: slab orders and the moves split by pass (same column: pass A,
    // same row: pass B, the rest (H_c between the two columns): pass A)
    auto upload_ints = [&](int** dst, const std::vector<int>& h) {
      alloc((void**)dst, sizeof(int) * std::max<size_t>(h.size(), 1));
      if (st == DMRG2D_OK && !h.empty() &&
          cudaMemcpy(*dst, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice) !=
              cudaSuccess)
        st = set_error(DMRG2D_ECUDA, "upload failed");
    };
    for (int k = 0; k < 2; ++k) {
      if (k == 1 && !T->pair_ok) break;
      const int pieces = k ? m1 / 256 : m1 / BM;
      upload_ints(&T->orderA[k], slab_order(d, pieces, m4 / T->BN, true));
      upload_ints(&T->orderB[k], slab_order(d, pieces, m4 / T->BN, false));
    }
    {
      std::vector<int> pa(1, 0), pb(1, 0), sa, sb;
      std::vector<float> va, vb;
      for (int tt = 0; tt < d * d; ++tt) {
        const int i2 = tt % d;
        for (int e = ops->hCptr[tt]; e < ops->hCptr[tt + 1]; ++e) {
          const int src = ops->hCsrc[e];
          const bool row = src % d == i2 && src / d != tt / d;  // same block row: pass B
          (row ? sb : sa).push_back(src);
          (row ? vb : va).push_back((float)ops->hCval[e]);
        }
        pa.push_back((int)sa.size());
        pb.push_back((int)sb.size());
      }
      upload_ints(&T->CptrA, pa);
      upload_ints(&T->CptrB, pb);
      upload_ints(&T->CsrcA, sa);
      upload_ints(&T->CsrcB, sb);
      alloc((void**)&T->CvalA, sizeof(float) * std::max<size_t>(va.size(), 1));
      alloc((void**)&T->CvalB, sizeof(float) * std::max<size_t>(vb.size(), 1));
      if (st == DMRG2D_OK &&
          ((!va.empty() && cudaMemcpy(T->CvalA, va.data(), sizeof(float) * va.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess) ||
           (!vb.empty() && cudaMemcpy(T->CvalB, vb.data(), sizeof(float) * vb.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess)))
        st = set_error(DMRG2D_ECUDA, "upload failed");
    }
    if (st == DMRG2D_OK) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&T->sms, cudaDevAttrMultiProcessorCount, dev);
      if (cudaFuncSetAttribute(hv_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_BYTES) != cudaSuccess ||
          cudaFuncSetAttribute(hv_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_BYTES) != cudaSuccess ||
          (T->pair_ok &&
           (cudaFuncSetAttribute(hv_tc_pair_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)P_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(hv_tc_pair_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)P_SMEM) != cudaSuccess)))
        st = set_error(DMRG2D_ECUDA, "cannot set %zu bytes of shared memory", SMEM_BYTES);
      if (st == DMRG2D_OK && T->pair_ok) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(T->sms);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = P_SMEM;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, hv_tc_pair_kernel<0>, &cfg) != cudaSuccess) {
          cudaGetLastError();
          ncl = 0;
        }
        T->pairs = std::min(ncl, T->sms / 2);
        T->pair_ok = T->pairs > 0;
      }
    }
  }
  if (grouped_ok && st == DMRG2D_OK) {
    // the dense superblock as one sector: row segment per i2, column segment per i3,
    // operator blocks stored once up to sign
    GroupPlan* g = new GroupPlan();
    T->plan = g;
    g->copies = 8;
    g->nQ = 1;
    g->qbase = {0};
    g->qld = {(int)ops->ld};
    g->qcols = {d * m4};
    for (int i2 = 0; i2 < d; ++i2) {
      GRow r{0, m1 * i2, m1, m1, (int)g->k1.size(), 0};
      for (int e = ops->hLptr[i2]; e < ops->hLptr[i2 + 1]; ++e) {
        auto pe = g->poolL.add(HL.data() + (size_t)e * m1 * m1, m1, m1, m1);
        g->k1.push_back({pe.first, m1 * ops->hLcol[e], m1, pe.second});
      }
      r.k1e = (int)g->k1.size();
      g->rows.push_back(r);
    }
    for (int i3 = 0; i3 < d; ++i3) {
      GCol c{0, m4 * i3, m4, (int)g->k2.size(), 0};
      for (int e = ops->hRptr[i3]; e < ops->hRptr[i3 + 1]; ++e) {
        auto pe = g->poolR.add(HR.data() + (size_t)e * m4 * m4, m4, m4, m4);
        g->k2.push_back({m4 * ops->hRcol[e], pe.first, m4, pe.second});
      }
      c.k2e = (int)g->k2.size();
      g->cols.push_back(c);
    }
    // scalar moves: destination tile (i2, i3) = (row segment i2, column segment i3)
    for (int i3 = 0; i3 < d; ++i3)
      for (int i2 = 0; i2 < d; ++i2) {
        const int tt = i2 + d * i3;
        if (ops->hCptr[tt] == ops->hCptr[tt + 1]) continue;
        GMoveDst md{i2, i3, (int)g->moves.size(), 0};
        for (int e = ops->hCptr[tt]; e < ops->hCptr[tt + 1]; ++e)
          g->moves.push_back({ops->hCsrc[e] % d, ops->hCsrc[e] / d, (float)ops->hCval[e]});
        md.me = (int)g->moves.size();
        g->mdst.push_back(md);
      }
    st = gp_finalise(ops, g, s);
  }
  if (st == DMRG2D_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = set_error(DMRG2D_ECUDA, "tc_prepare: %s", cudaGetErrorString(e));
  }
  if (st != DMRG2D_OK) return st;
  ops->tc_ok = 1;
  // default before any autotuning: the CTA-pair kernel in blocked order where it applies
  // (fastest on the shapes measured), else the single-CTA dense kernel, else grouped
  const int dflt = dense_ok ? (T->pair_ok ? kPairBlockedCfg : -1) : 5;
  for (int p = 0; p < 4; ++p) ops->tc_cfg[p] = dflt;
  return DMRG2D_OK;
}

void tc_release(dmrg2d_ops* ops) {
  TcState* T = (TcState*)ops->tc;
  if (!T) return;
  if (T->HLt) cudaFree(T->HLt);
  if (T->HRt) cudaFree(T->HRt);
  if (T->HLlo) cudaFree(T->HLlo);
  if (T->HRlo) cudaFree(T->HRlo);
  if (T->err) cudaFree(T->err);
  if (T->order) cudaFree(T->order);
  if (T->order2) cudaFree(T->order2);
  for (int k = 0; k < 2; ++k)
    if (T->order2p[k]) cudaFree(T->order2p[k]);
  for (int k = 0; k < 2; ++k) {
    if (T->orderA[k]) cudaFree(T->orderA[k]);
    if (T->orderB[k]) cudaFree(T->orderB[k]);
  }
  for (void* q : {(void*)T->CptrA, (void*)T->CsrcA, (void*)T->CvalA, (void*)T->CptrB,
                  (void*)T->CsrcB, (void*)T->CvalB})
    if (q) cudaFree(q);
  if (T->plan) {
    gp_release(T->plan);
    delete T->plan;
  }
  delete T;
  ops->tc = nullptr;
}

// dense-kernel variants: tc_cfg = -1 - variant, variant bit 0 = operator pool, bit 1 =
// blocked piece order, bit 2 = CTA-pair kernel, bit 3 = two passes (H_l V with the moves
// of the same column and H_c in column-slab order, then V H_r^T with the moves of the
// same row in row-slab order, adding to the stored Y); autotuner index 0 / 7 / 8 / 9 /
// 10 / 11 / 12 / 13 / 20 / 21 = variant 0 / 1 / 2 / 3 / 4 / 6 / 5 / 7 / 8 / 12
// lo_ops: the operator blocks' low BF16 parts (BF16X3); accum: add to the stored Y
static int launch_dense_kernel(const dmrg2d_ops* ops, const TcState* T, const void* v, float* y,
                               bool bf, bool fuse_moves, int variant, cudaStream_t s,
                               bool lo_ops = false, bool accum = false) {
  const bool pair = (variant & 4) != 0;
  const bool use_pool = (variant & 1) != 0;
  const bool two = (variant & 8) != 0;
  const bool a3 = (variant & 16) != 0;
  const int b = bf ? 1 : 0;
  const int m1 = ops->m1, m4 = ops->m4, d = ops->d;
  const uint32_t BK = bf ? 64 : 32;
  TcParams p;
  p.m1 = m1;
  p.m4 = m4;
  p.d = d;
  p.BN = T->BN;
  p.n_mt = pair ? m1 / 256 : m1 / BM;  // pieces (pairs of pieces) per block row
  p.n_nt = m4 / T->BN;
  p.tiles = d * p.n_mt * d * p.n_nt;
  // blocked order: 8 x 8 tile patches, or (CTA pairs, bits 5 / 6) 4 x 4 / 16 x 16
  const int* pair_order = (variant & 32) ? T->order2p[0] : (variant & 64) ? T->order2p[1]
                                                                          : T->order2;
  p.order = (variant & 2) ? (pair ? pair_order : T->order) : nullptr;
  p.ph0 = 0;
  p.ph1 = 2;
  p.accum_y = accum ? 1 : 0;
  p.a2_3d = a3 ? 1 : 0;
  p.BK = (int)BK;
  p.kblk1 = m1 / (int)BK;
  p.kblk2 = m4 / (int)BK;
  p.ld = ops->ld;
  p.Lptr = ops->dev.Lptr;
  p.Lcol = ops->dev.Lcol;
  p.Rptr = ops->dev.Rptr;
  p.Rcol = ops->dev.Rcol;
  p.y = y;
  p.err = T->err;
  const int fmt = bf ? 1 : 2;
  const int M = pair ? 2 * BM : BM;
  for (int n = 0; n < 2; ++n) {
    p.idesc1[n] = make_idesc(fmt, 0, M, T->BN, n, 0);
    p.idesc2[n] = make_idesc(fmt, 1, M, T->BN, 0, n);
  }
  const CUtensorMap* mA = lo_ops ? &T->mHLlo : &T->mHL[b];
  const CUtensorMap* mB =
      lo_ops ? (pair ? &T->mHR2lo : &T->mHRlo) : (pair ? &T->mHR2[b] : &T->mHR[b]);
  p.pooled = 0;
  p.k1 = nullptr;
  p.k2 = nullptr;
  p.poolL_rows = p.poolR_rows = 0;
  p.copies = 1;
  // (the pair kernel reads H_r rows in 128-row boxes: the pool's 128-wide view)
  if (use_pool && T->plan &&
      gp_pool_views(T->plan, bf ? DMRG2D_BF16 : DMRG2D_TF32, pair ? P_HALF : T->BN, &mA, &mB,
                    &p.k1, &p.k2, &p.poolL_rows, &p.poolR_rows, &p.copies) == DMRG2D_OK)
    p.pooled = 1;
  p.a2_box_rows = bf ? 64 : 32;
  p.a2_boxes = BM / p.a2_box_rows;
  p.a2_lbo = (uint32_t)p.a2_box_rows * BK * (bf ? 2 : 4);  // bytes of one {rows, BK} box
  p.a2_kstep = bf ? 2048 : 1024;                           // 16 (bf16) / 8 (tf32) k-rows
  p.a2_layout = bf ? 2u : 1u;
  // k-row groups: 8 rows (1024 B) for the 16-byte-atom swizzle, 4 rows (512 B) for the
  // 32-byte-atom swizzle whose pattern repeats every four 128-byte rows
  p.a2_sbo = bf ? 1024u : 512u;
  p.tx_bytes = STAGE_A + (uint32_t)(pair ? P_HALF : T->BN) * 128;  // per CTA and stage
  p.bf16 = bf ? 1 : 0;
  p.fuse = fuse_moves ? 1 : 0;
  p.v = v;
  p.Cptr = ops->dev.Cptr;
  p.Csrc = ops->dev.Csrc;
  p.Cval = ops->dev.Cval32;
  CUtensorMap mVk, mVm;
  const uint64_t rows = (uint64_t)ops->ld, cols = (uint64_t)d * m4;
  D2_TRY(make_map(&mVk, v, bf, rows, cols, BK, pair ? P_HALF : T->BN));
  if (a3) {  // dims {row in block, column, row block}: the four boxes in one copy
    D2_TRY(make_map3(&mVm, v, bf, (uint64_t)p.a2_box_rows, cols, rows / (uint64_t)p.a2_box_rows,
                     (uint64_t)ops->ld, (uint32_t)p.a2_box_rows, BK, (uint32_t)p.a2_boxes,
                     bf ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B));
  } else {
    D2_TRY(make_map(&mVm, v, bf, rows, cols, (uint32_t)p.a2_box_rows, BK,
                    bf ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B));
  }
  auto ev = prof_slot(ops);
  if (ev.first) D2_CUDA(cudaEventRecord(ev.first, s));
  auto launch = [&](const TcParams& q) {
    if (pair) {
      const int pairs = std::min(q.tiles, T->pairs);
      if (bf)
        hv_tc_pair_kernel<1><<<2 * pairs, TC_THREADS, P_SMEM, s>>>(*mA, *mB, mVk, mVm, q);
      else
        hv_tc_pair_kernel<0><<<2 * pairs, TC_THREADS, P_SMEM, s>>>(*mA, *mB, mVk, mVm, q);
    } else {
      const int grid = std::min(q.tiles, T->sms);
      if (bf)
        hv_tc_kernel<1><<<grid, TC_THREADS, SMEM_BYTES, s>>>(*mA, *mB, mVk, mVm, q);
      else
        hv_tc_kernel<0><<<grid, TC_THREADS, SMEM_BYTES, s>>>(*mA, *mB, mVk, mVm, q);
    }
  };
  if (two) {
    TcParams a = p, b2 = p;
    a.order = T->orderA[pair ? 1 : 0];
    a.ph1 = 1;
    a.Cptr = T->CptrA;
    a.Csrc = T->CsrcA;
    a.Cval = T->CvalA;
    b2.order = T->orderB[pair ? 1 : 0];
    b2.ph0 = 1;
    b2.accum_y = 1;
    b2.Cptr = T->CptrB;
    b2.Csrc = T->CsrcB;
    b2.Cval = T->CvalB;
    launch(a);
    launch(b2);
  } else {
    launch(p);
  }
  D2_CUDA(cudaGetLastError());
  if (ev.second) D2_CUDA(cudaEventRecord(ev.second, s));
  return DMRG2D_OK;
}

// H·v with an explicit kernel choice (dense kernel: moves only when fuse_moves)
int tc_gemm(const dmrg2d_ops* ops, const void* v, float* y, int precision, int cfg,
            cudaStream_t s) {
  const TcState* T = (const TcState*)ops->tc;
  if (!T) return set_error(DMRG2D_EUNSUPPORTED, "tensor-core path not prepared");
  if (cfg < 0) {
    if (!T->dense_ok) return set_error(DMRG2D_EUNSUPPORTED, "dense kernel unsupported here");
    return launch_dense_kernel(ops, T, v, y, precision == DMRG2D_BF16, false, -1 - cfg, s);
  }
  if (!T->plan) return set_error(DMRG2D_EUNSUPPORTED, "grouped kernel unsupported here");
  return gp_launch(ops, T->plan, v, y, precision, cfg, s);
}

int launch_hv_tc(const dmrg2d_ops* ops, const void* v, float* y, int precision, cudaStream_t s) {
  if (ops->sec) return sec_apply(ops, v, y, precision, s);
  if (!ops->tc || !ops->tc_ok)
    return set_error(DMRG2D_EUNSUPPORTED, "tensor-core path not prepared");
  if (precision == DMRG2D_BF16X3) {
    // v = [v_hi | v_lo] (BF16); Y = H_hi v_hi + H_hi v_lo + H_lo v_hi in three BF16
    // launches of the kernel chosen for BF16 (per-position operator blocks, one pass),
    // the scalar moves (exact coefficients) applied to v_hi and v_lo
    const TcState* T = (const TcState*)ops->tc;
    const void* vlo = (const __nv_bfloat16*)v + ops->n_vec;
    const int cfg = ops->tc_cfg[DMRG2D_BF16];
    if (cfg < 0) {
      const int var = (-1 - cfg) & ~9;  // no operator pool, no two-pass form
      D2_TRY(launch_dense_kernel(ops, T, v, y, true, true, var, s, false, false));
      D2_TRY(launch_dense_kernel(ops, T, vlo, y, true, true, var, s, false, true));
      return launch_dense_kernel(ops, T, v, y, true, false, var, s, true, true);
    }
    if (!T->plan) return set_error(DMRG2D_EUNSUPPORTED, "grouped kernel unsupported here");
    D2_TRY(gp_launch(ops, T->plan, v, y, DMRG2D_BF16, cfg, s, true, false, false));
    D2_TRY(gp_launch(ops, T->plan, vlo, y, DMRG2D_BF16, cfg, s, true, false, true));
    return gp_launch(ops, T->plan, v, y, DMRG2D_BF16, cfg, s, false, true, true);
  }
  const bool bf = precision == DMRG2D_BF16;
  if (ops->tc_cfg[precision] < 0) {  // dense kernel: the moves run in its epilogue
    return launch_dense_kernel(ops, (const TcState*)ops->tc, v, y, bf, true,
                               -1 - ops->tc_cfg[precision], s);
  }
  // grouped kernel: its epilogue adds the scalar moves of the plan
  return tc_gemm(ops, v, y, precision, ops->tc_cfg[precision], s);
}

int tc_read_error(const dmrg2d_ops* ops, int* code) {
  *code = 0;
  const TcState* T = (const TcState*)ops->tc;
  if (T && T->err) {
    D2_CUDA(cudaMemcpy(code, T->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (*code) D2_CUDA(cudaMemset(T->err, 0, sizeof(int)));
  }
  int c2 = 0;
  if (T && T->plan) D2_TRY(gp_read_error(T->plan, &c2));
  if (!*code) *code = c2;
  int c3 = 0;
  D2_TRY(sec_read_error(ops, &c3));
  if (!*code) *code = c3;
  return DMRG2D_OK;
}

}  // namespace dmrg2d

// ---- tile-configuration autotuner ---------------------------------------------------------
namespace dmrg2d {

// candidate index: 0 = dense kernel, 1 + c = grouped kernel configuration c, 7 = dense
// kernel reading the deduplicated (replicated) operator pool, 8 / 9 = dense kernel in the
// blocked piece order (per-position blocks / pool)
// 14 + c = grouped configuration c with the scalar moves in a separate kernel (sectors)
// 20 / 21 = two-pass dense kernel (128-row pieces / CTA pairs)
// 22 = segment kernels (sectors: M along the long dimension of each V_q, moves separate)
// 23 / 24 = CTA-pair kernel / dense kernel in blocked order, the phase-2 V operand in one
// 3-D copy per stage
// 25 / 26 = candidate 23 with the output tiles in 4 x 4 / 16 x 16 patches
constexpr int N_CANDIDATES = 27;
static int idx_to_cfg(int idx) {
  static const int dense_variant[14] = {0, -1, -1, -1, -1, -1, -1, 1, 2, 3, 4, 6, 5, 7};
  if (idx >= 1 && idx <= 6) return idx - 1;
  if (idx == 20) return -1 - 8;
  if (idx == 21) return -1 - 12;
  if (idx == 22) return 2 * gp_num_configs();
  if (idx == 23) return -1 - (6 | 16);
  if (idx == 24) return -1 - (2 | 16);
  if (idx == 25) return -1 - (6 | 16 | 32);
  if (idx == 26) return -1 - (6 | 16 | 64);
  if (idx >= 14) return gp_num_configs() + idx - 14;
  return -1 - dense_variant[idx];
}

static bool tc_candidate_ok(const dmrg2d_ops* ops, int idx) {
  if (idx < 0 || idx >= N_CANDIDATES) return false;
  if (idx >= 14 && idx < 20) return ops->sec && ops->tc_ok;  // grouped, separate moves
  if (idx == 22) return ops->sec && ops->tc_ok;               // segment kernels
  if (idx >= 23) {                                             // dense kernels, 3-D V copies
    const TcState* T = (const TcState*)ops->tc;
    return !ops->sec && T && T->dense_ok && (idx == 24 || T->pair_ok);
  }
  if (idx == 0 || idx >= 7) {                                // dense-kernel variants
    const TcState* T = (const TcState*)ops->tc;
    if (ops->sec || !T || !T->dense_ok) return false;
    const int variant = -1 - idx_to_cfg(idx);
    if ((variant & 4) && !T->pair_ok) return false;
    return (variant & 1) == 0 || T->plan != nullptr;  // the pool lives in the grouped plan
  }
  if (idx > gp_num_configs()) return false;
  if (ops->sec) return ops->tc_ok != 0;
  const TcState* T = (const TcState*)ops->tc;
  return T && T->plan;
}

// one full H·v (operator blocks and scalar moves) with candidate idx
static int tc_run_candidate(dmrg2d_ops* ops, const void* v, float* y, int prec, int idx,
                            cudaStream_t s) {
  const int saved = ops->tc_cfg[prec];
  ops->tc_cfg[prec] = idx_to_cfg(idx);
  const int st = launch_hv_tc(ops, v, y, prec, s);
  ops->tc_cfg[prec] = saved;
  return st;
}

}  // namespace dmrg2d

using namespace dmrg2d;

extern "C" const char* dmrg2d_tile_config_name(int index) {
  if (index == 0) return "dense kernel 128x256 (column-slab raster)";
  if (index == 7) return "dense kernel 128x256, deduplicated operator pool";
  if (index == 8) return "dense kernel 128x256 (8x8-tile blocked raster)";
  if (index == 9) return "dense kernel 128x256 (8x8-tile blocked raster), operator pool";
  if (index == 10) return "CTA-pair kernel 256x256 (column-slab raster)";
  if (index == 11) return "CTA-pair kernel 256x256 (8x8-tile blocked raster)";
  if (index == 12) return "CTA-pair kernel 256x256 (column-slab raster), operator pool";
  if (index == 13) return "CTA-pair kernel 256x256 (8x8-tile blocked raster), operator pool";
  if (index == 20) return "dense kernel 128x256, two passes (H_l V by column slabs, V H_r^T by row slabs)";
  if (index == 21) return "CTA-pair kernel 256x256, two passes (H_l V by column slabs, V H_r^T by row slabs)";
  if (index == 22) return "segment kernels (M = 128 along V's long dimension, N = one sector), separate moves";
  if (index == 23) return "CTA-pair kernel 256x256 (8x8-tile blocked raster), phase-2 V in one 3-D copy";
  if (index == 24) return "dense kernel 128x256 (8x8-tile blocked raster), phase-2 V in one 3-D copy";
  if (index == 25) return "CTA-pair kernel 256x256 (4x4-tile blocked raster), phase-2 V in one 3-D copy";
  if (index == 26) return "CTA-pair kernel 256x256 (16x16-tile blocked raster), phase-2 V in one 3-D copy";
  static const char* sep[6] = {
      "grouped 128x128 column-slab, separate moves kernel",
      "grouped 128x128 row-slab, separate moves kernel",
      "grouped 128x128 longest-first, separate moves kernel",
      "grouped 128x256 column-slab, separate moves kernel",
      "grouped 128x256 row-slab, separate moves kernel",
      "grouped 128x256 longest-first, separate moves kernel"};
  if (index >= 14 && index < 20) return sep[index - 14];
  return gp_config_name(index - 1);
}

extern "C" int dmrg2d_set_tile_config(dmrg2d_ops* ops, int precision, int index) {
  if (!ops || (precision != DMRG2D_TF32 && precision != DMRG2D_BF16))
    return set_error(DMRG2D_EINVAL, "set_tile_config: bad argument");
  if (!tc_candidate_ok(ops, index))
    return set_error(DMRG2D_EUNSUPPORTED, "tile configuration %d not available here", index);
  ops->tc_cfg[precision] = idx_to_cfg(index);
  return DMRG2D_OK;
}

extern "C" int dmrg2d_autotune(dmrg2d_ops* ops, int precision, int* best, double* ms, int n_ms,
                               void* stream) {
  if (!ops || (precision != DMRG2D_TF32 && precision != DMRG2D_BF16))
    return set_error(DMRG2D_EINVAL, "autotune: bad argument");
  if (!ops->tc_ok) return set_error(DMRG2D_EUNSUPPORTED, "no tensor-core path for these shapes");
  cudaStream_t s = (cudaStream_t)stream;
  const bool bf = precision == DMRG2D_BF16;
  const size_t n = (size_t)ops->n_vec;
  void* v = nullptr;
  float* y = nullptr;
  if (cudaMalloc(&v, n * (bf ? 2 : 4)) != cudaSuccess)
    return set_error(DMRG2D_ENOMEM, "autotune: cudaMalloc failed");
  if (cudaMalloc((void**)&y, n * 4) != cudaSuccess) {
    cudaFree(v);
    return set_error(DMRG2D_ENOMEM, "autotune: cudaMalloc failed");
  }
  struct Free {
    void* a;
    void* b;
    ~Free() {
      cudaFree(a);
      cudaFree(b);
    }
  } fr{v, y};
  D2_CUDA(cudaMemsetAsync(v, 0x3C, n * (bf ? 2 : 4), s));  // small positive values
  cudaEvent_t e0, e1;
  D2_CUDA(cudaEventCreate(&e0));
  D2_CUDA(cudaEventCreate(&e1));
  int chosen = -1;
  double tbest = 1e300;
  const int ncand = N_CANDIDATES;
  int st = DMRG2D_OK;
  for (int c = 0; c < ncand && st == DMRG2D_OK; ++c) {
    double t = -1.0;
    if (tc_candidate_ok(ops, c)) {
      st = tc_run_candidate(ops, v, y, precision, c, s);  // warm-up
      if (st == DMRG2D_EUNSUPPORTED) {  // a candidate whose tensor maps cannot be encoded
        st = DMRG2D_OK;
        clear_error();
        if (ms && c < n_ms) ms[c] = -1.0;
        continue;
      }
      float tmin = 1e30f;
      for (int r = 0; r < 3 && st == DMRG2D_OK; ++r) {
        cudaEventRecord(e0, s);
        st = tc_run_candidate(ops, v, y, precision, c, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          st = set_error(DMRG2D_ECUDA, "autotune: launch failed");
          break;
        }
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        tmin = x < tmin ? x : tmin;
      }
      t = tmin;
      if (st == DMRG2D_OK && t < tbest) {
        tbest = t;
        chosen = c;
      }
    }
    if (ms && c < n_ms) ms[c] = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DMRG2D_OK) return st;
  int derr = 0;
  D2_TRY(tc_read_error(ops, &derr));
  if (derr) return set_error(DMRG2D_ETIMEOUT, "tensor-core kernel gave up waiting (site %d)", derr);
  if (chosen < 0) return set_error(DMRG2D_EUNSUPPORTED, "no tile configuration applies");
  ops->tc_cfg[precision] = idx_to_cfg(chosen);
  if (best) *best = chosen;
  return DMRG2D_OK;
}

extern "C" int dmrg2d_wait_selftest(double seconds, void* stream) {
  if (!(seconds > 0.0) || seconds > 2.0)
    return set_error(DMRG2D_EINVAL, "wait_selftest: seconds must be in (0, 2]");
  cudaStream_t s = (cudaStream_t)stream;
  int* err = nullptr;
  D2_CUDA(cudaMalloc((void**)&err, sizeof(int)));
  struct Free {
    int* p;
    ~Free() { cudaFree(p); }
  } fr{err};
  D2_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_wait_selftest<<<1, 32, 0, s>>>(err, (uint64_t)(seconds * 1e9));
  D2_CUDA(cudaGetLastError());
  int code = 0;
  D2_CUDA(cudaMemcpyAsync(&code, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  D2_CUDA(cudaStreamSynchronize(s));
  if (code == 99)
    return set_error(DMRG2D_ETIMEOUT, "wait_selftest: the bounded wait gave up as designed");
  return set_error(DMRG2D_ECUDA, "wait_selftest: the wait did not report its timeout (%d)", code);
}
