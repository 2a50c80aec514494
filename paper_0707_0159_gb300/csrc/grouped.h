// Work list of the grouped tensor-core H·v, shared by dense and sector-restricted
// superblocks.  Internal header.
//
// The vector is a list of column-major matrices V_q (one for a dense superblock).  Rows
// of V_q are grouped in row segments (one per block row i2, or per (i2, block sector)),
// columns in column segments.  Output pieces ("tiles") are 128 rows of one row segment
// by BN columns of one column segment.  A row segment's phase-1 list holds one entry per
// H_l block that feeds it (A = operator block from the pool, B = rows of V_q); a column
// segment's phase-2 list one entry per H_r block (A = columns of V_q, B = pool block).
// The pool stores every distinct operator block once; an entry may use it negated.
#pragma once
#include <cuda.h>
#include <cstdint>
#include <vector>

#include "common.h"

namespace dmrg2d {

struct GRow {
  int q, off, dim, dim_pad, k1b, k1e;
};
struct GCol {
  int q, off, dim, k2b, k2e;
};
struct GK1 {
  int a_pool, b_row, kdim, neg;
};
struct GK2 {
  int a_col, b_pool, kdim, neg;
};
struct GTile {
  int rs, cs, r_in, c_in;
  int mb, me;  // scalar moves into this tile's (row segment, column segment): moves[mb..me)
};
// scalar tile move Y(dst rs, dst cs) += c V(rs, cs): same rows within the row segments,
// same columns within the column segments (H_c and off-diagonal column terms)
struct GMove {
  int rs, cs;
  float c;
};
struct GMoveDst {
  int rs, cs, mb, me;  // destination segments, range in GroupPlan::moves
};

// Distinct operator blocks, deduplicated up to sign.
struct BlockPool {
  struct Entry {
    int rows, cols;
    std::vector<double> a;
    uint64_t h;
  };
  std::vector<Entry> ent;
  // returns (entry index, negated?) for the rows x cols block src[i*ld + j]
  std::pair<int, int> add(const double* src, int rows, int cols, int64_t ld);
};

struct GroupPlan {
  int nQ = 0;
  std::vector<long long> qbase;
  std::vector<int> qld, qcols;
  std::vector<GRow> rows;
  std::vector<GCol> cols;
  std::vector<GK1> k1;  // a_pool holds the pool ENTRY index until finalise()
  std::vector<GK2> k2;
  std::vector<GMoveDst> mdst;  // scalar moves, grouped by destination (optional)
  std::vector<GMove> moves;
  BlockPool poolL, poolR;
  int copies = 1;       // pool replicas (CTAs read replica blockIdx % copies: no L2 hot spot)
  void* dev = nullptr;  // device state (grouped.cu)
};

// Lays out the pools, builds the tile lists, uploads everything.  `ops` receives the
// device bytes.  Fails with EUNSUPPORTED when the plan does not fit the kernel.
int gp_finalise(dmrg2d_ops* ops, GroupPlan* g, cudaStream_t s);
void gp_release(GroupPlan* g);
// Y(all V_q) = grouped H_l V + V H_r^T, plus the plan's scalar moves when fuse_moves;
// cfg = tile layout 0 .. gp_num_configs() - 1
// lo_ops: the pools' low BF16 parts (BF16X3, precision BF16); accum: add to the stored Y
int gp_launch(const dmrg2d_ops* ops, const GroupPlan* g, const void* v, float* y, int precision,
              int cfg, cudaStream_t s, bool fuse_moves = true, bool lo_ops = false,
              bool accum = false);
// Segment kernels (sectors of tens of states): pass 1 = H_l V with M along the columns of
// V_q, written to Y (added when accum); pass 2 = V H_r^T with M along the rows, added to Y.
// No scalar moves.  y must be 16-byte aligned.
int gp_launch_seg(const dmrg2d_ops* ops, const GroupPlan* g, const void* v, float* y,
                  int precision, cudaStream_t s, bool lo_ops = false, bool accum = false);
int gp_read_error(const GroupPlan* g, int* code);
// pool tensor maps and per-block entries (CSR order of the build) for another kernel
int gp_pool_views(const GroupPlan* g, int precision, int bn, const CUtensorMap** mL,
                  const CUtensorMap** mR, const GK1** k1, const GK2** k2, int* rowsL, int* rowsR,
                  int* copies);
int gp_num_configs();
const char* gp_config_name(int cfg);

}  // namespace dmrg2d
