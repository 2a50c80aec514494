/*
 * dmrg2d.h — C ABI of the GB300 superblock H·v library for the direct n-leg DMRG
 * of Yamada, Okumura and Machida (arXiv 0707.0159).
 *
 * The superblock is block 1 (m1 states, index i1) · block 2 = one lattice
 * column of n sites (d states, i2) · block 3 = one column (d states, i3) ·
 * block 4 (m4 states, i4) — paper Fig. 2.  Its Hamiltonian is split as in
 * Eq. (dec):  H = H_l (x) 1_{34} + H_r (x) 1_{12} + H_c (x) 1_{14},
 * and with the superblock vector v viewed as the (m1 d) x (d m4) matrix V,
 *     H v  ->  Y = H_l V + V H_r^T + H_c V_c
 * (paper, text after Eq. (dec)).  This library evaluates the last term as
 * sum_k A_k V B_k^T with A_k = a_k (x) 1_{m1}, B_k = b_k (x) 1_{m4}, the same
 * product written on V instead of the permuted V_c.
 *
 * Layouts (all fixed by the paper's index map):
 *   - vector v, dense (no sectors): element of state |i1 i2 i3 i4> at
 *       i1 + m1*i2 + m1*d*i4 + m1*d*m4*i3          (0-based)
 *     i.e. V = column-major (m1 d) x (d m4) matrix, leading dimension m1*d.
 *   - column basis: spin column i = sum_y b_y 2^y (b_y = 1: spin up on leg y);
 *     Hubbard column i = sum_y (n_{y,up} + 2 n_{y,dn}) 4^y, fermion modes
 *     ordered by that bit position (leg 0 up, leg 0 down, leg 1 up, ...).
 *   - fermion signs: global mode order block 1, column 2, column 3, block 4;
 *     each subsystem's operators carry the parities of the subsystems before it.
 *   - block operators (inputs): host arrays, row-major m x m, <i|op|j> at i*m+j.
 *   - sector-restricted vectors (target != NULL): see dmrg2d_build_ops.
 *
 * Ownership: every function copies what it needs from its inputs; the caller
 * keeps ownership of all pointers passed in.  dmrg2d_ops owns the device memory
 * it allocates until dmrg2d_free_ops.  Device vectors passed to apply/solve are
 * caller-owned.  No function throws; errors are returned as negative codes and
 * dmrg2d_last_error() gives a thread-local message.
 */
#ifndef DMRG2D_H
#define DMRG2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------- */
enum {
  DMRG2D_OK = 0,
  DMRG2D_EINVAL = -1,       /* bad argument (NULL, out-of-range value)               */
  DMRG2D_ESHAPE = -2,       /* inconsistent sizes                                    */
  DMRG2D_ENOMEM = -3,       /* device or host allocation failed                      */
  DMRG2D_ECUDA = -4,        /* a CUDA runtime call failed                            */
  DMRG2D_ENOCONV = -5,      /* solver hit its iteration budget (best estimate kept)  */
  DMRG2D_ETIMEOUT = -6,     /* a device-side bounded wait gave up                    */
  DMRG2D_ENAN = -7,         /* NaN/Inf met in a reduction                            */
  DMRG2D_EUNSUPPORTED = -8  /* precision/shape combination not built                 */
};

/* ---- models (paper: Heisenberg J_z = J_xy, Hubbard U/t; open boundaries) ------------ */
enum { DMRG2D_HEISENBERG = 0, DMRG2D_HUBBARD = 1 };

/* arithmetic of the H·v products */
enum {
  DMRG2D_FP64 = 0,   /* v, y double; DFMA                                            */
  DMRG2D_TF32 = 1,   /* v float, y float; tcgen05 kind::tf32, FP32 accumulate in TMEM */
  DMRG2D_BF16 = 2,   /* v bf16 (uint16 bits), y float; tcgen05 kind::f16, FP32 acc  */
  DMRG2D_FP32 = 3,   /* v float, y float; FP32 FMA on CUDA cores                      */
  DMRG2D_FP64X = 4,  /* v, y double; float-pair arithmetic (~48-bit significands) on
                        the FP32 CUDA cores: FP64 emulated for the mixed solver's
                        residuals (sector layouts: the scalar moves in FP64)         */
  DMRG2D_BF16X3 = 5  /* split BF16: v = [v_hi | v_lo], 2 n_vec bf16 values with
                        v_hi = bf16(x), v_lo = bf16(x - v_hi) (dmrg2d_convert_input);
                        y float; three BF16 tensor-core products into FP32,
                        H_hi v_hi + H_hi v_lo + H_lo v_hi (the operators split the same
                        way): relative error ~1e-5 instead of BF16's ~2e-3              */
};

typedef struct dmrg2d_model {
  int kind;          /* DMRG2D_HEISENBERG or DMRG2D_HUBBARD                            */
  int n_legs;        /* sites per column n >= 1; d = 2^n (spins) or 4^n (electrons)  */
  double J_leg;      /* Heisenberg coupling along the legs (between columns)          */
  double J_rung;     /* Heisenberg coupling along a column                            */
  double t;          /* Hubbard hopping (same along legs and rungs)                  */
  double U;          /* Hubbard on-site repulsion                                    */
  int rung_pbc;      /* 1: close each column into a ring (n > 2 only)                */
} dmrg2d_model;

/* One renormalised block (block 1 or block 4), host memory, row-major m x m.
 * edge[] holds the operators of the block's sites that touch the neighbouring
 * column, one entry per leg y:
 *   Heisenberg: edge[2y] = S^z_y, edge[2y+1] = S^+_y   (S^- = (S^+)^T)
 *   Hubbard:    edge[2y] = c^dag_{y,up}, edge[2y+1] = c^dag_{y,dn} (c = (c^dag)^T),
 *               each carrying the block's own Jordan-Wigner string;
 *               parity[i] = +1/-1 is the block's fermion parity (diagonal).
 * n_edge = 0 describes a lattice end (the block is not coupled to the column).
 * qn (optional): per-state quantum numbers, row-major m x nq with nq = 1
 * (N_up) for spins and nq = 2 (N_up, N_dn) for electrons; needed only for
 * sector-restricted operation. */
typedef struct dmrg2d_block {
  int m;
  const double* H;
  int n_edge;
  const double* const* edge;
  const double* parity;
  const int32_t* qn;
} dmrg2d_block;

typedef struct dmrg2d_ops dmrg2d_ops;

typedef struct dmrg2d_ops_info {
  int64_t n_vec;           /* length of v                                          */
  int m1, m4, d, n_legs;
  int n_blk_left;          /* dense m1 x m1 blocks of H_l (nonzero block positions) */
  int n_blk_right;         /* dense m4 x m4 blocks of H_r                           */
  int n_scalar;            /* scalar tile moves (H_c terms + off-diagonal column    */
                           /* terms of H_l/H_r, both of the form c * I_m1 (x) I_m4) */
  double flops_per_apply;  /* algorithmic flops of one H·v (see dmrg2d_apply_H)     */
  int tc_ok;               /* 1 if the tcgen05 path supports these shapes          */
  int64_t device_bytes;    /* device memory owned by the ops object                */
  int n_sectors;           /* combined left labels (0 for a dense superblock)       */
} dmrg2d_ops_info;

/* Build the packed operators of H_l, H_r and H_c (paper Eq. (dec)).
 *   H_l = 1_d (x) H_B1 + H_col (x) 1_m1 + sum_k X_k (x) E_k   (row index i1 + m1*i2)
 *   H_r = 1_d (x) H_B4 + H_col (x) 1_m4 + sum_k X'_k (x) E'_k (row index i4 + m4*i3)
 *   H_c = sum_k a_k (on i2) b_k (on i3), the n leg bonds between the columns.
 * Column operators are built here from the model.  Every block position
 * (i2, i2') of H_l touched by a block operator becomes one dense m1 x m1 block;
 * terms that are multiples of the identity in block space (off-diagonal
 * column terms, all of H_c) become scalar tile moves.
 * target: NULL for the dense superblock.  Otherwise the superblock is restricted
 * to the states whose quantum numbers add up to target[0..nq) (nq = 1: N_up for
 * spins, nq = 2: (N_up, N_dn) for electrons); both blocks need qn, and states with
 * equal labels must be contiguous.  Packed vector layout of a restricted superblock:
 * for every combined left label qL = q(i1) + q(i2), in increasing lexicographic
 * order, one column-major matrix V_qL whose rows are, for i2 = 0..d-1, the block-1
 * sector with label qL - q(i2) (its states in order), each such segment padded with
 * zero rows to a multiple of 8, and whose columns are, for i3 = 0..d-1, the block-4
 * sector with label target - qL - q(i3); leading dimension = padded row count; the
 * matrices follow one another.  Padding entries must be zero on input and are written
 * as zero on output.  dmrg2d_sector_dense_index returns the map.
 * stream: cudaStream_t (may be NULL) used for the uploads.
 * Errors: EINVAL for NULL/invalid fields, ESHAPE if n_edge != 0 and != 2*n_legs,
 * ENOMEM/ECUDA on device failures (nothing leaks; *out is left NULL). */
int dmrg2d_build_ops(const dmrg2d_model* model, const dmrg2d_block* left,
                     const dmrg2d_block* right, const int32_t* target,
                     dmrg2d_ops** out, void* stream);

int dmrg2d_ops_get_info(const dmrg2d_ops* ops, dmrg2d_ops_info* info);

/* Sector-restricted ops only: out[p] (host array of info.n_vec entries) receives the
 * dense superblock index i1 + m1*i2 + m1*d*i4 + m1*d*m4*i3 of packed position p, or
 * -1 for a padding row.  EINVAL for a dense ops object. */
int dmrg2d_sector_dense_index(const dmrg2d_ops* ops, int64_t* out);

/* y = H v (paper: H_l V + V H_r^T + H_c V_c).  v and y are caller-owned device
 * buffers of info.n_vec elements in the layout above; they must not overlap.
 * Element types by precision: FP64 double/double; FP32 and TF32 float/float;
 * BF16 bf16/float; BF16X3 2 n_vec bf16 (hi part, then lo part)/float.  TF32, BF16 and
 * BF16X3 need info.tc_ok (else EUNSUPPORTED); BF16X3 uses the tile configuration
 * chosen for BF16 without the operator pool or the two-pass form (three launches).
 * Algorithmic flops: 2*n_blk_left*m1^2*(d*m4) + 2*n_blk_right*m4^2*(m1*d)
 * + 2*n_scalar*m1*m4.  Asynchronous on `stream`; allocates nothing; no host
 * synchronisation, so the call can be captured in a CUDA graph. */
int dmrg2d_apply_H(const dmrg2d_ops* ops, const void* v, void* y, int precision, void* stream);

/* The input format of apply_H at `precision` from an FP64 vector x (device, n doubles):
 * FP32 rounds to float; TF32 rounds to the nearest TF32 value (stored as float); BF16
 * rounds to bf16; BF16X3 writes 2n bf16, hi = bf16(x) then lo = bf16(x - hi); FP64 and
 * FP64X copy.  out: device buffer of that format.  Asynchronous; allocates nothing.
 * EINVAL for an unknown precision or a NULL pointer. */
int dmrg2d_convert_input(const double* x, void* out, int precision, int64_t n, void* stream);

/* Ground state of H by Lanczos (implied by the paper's "exact diagonalization"
 * of the superblock; the algorithm is not named there). */
typedef struct dmrg2d_solver_opts {
  int max_iter;        /* Lanczos steps (plain) or total inner steps budget (mixed) */
  int krylov_dim;      /* basis vectors kept before an explicit restart (>= 2)      */
  double tol;          /* stop when ||H x - theta x|| <= tol * |theta|              */
  int fixed_steps;     /* 1: run exactly max_iter steps with no convergence test    */
  int precision;       /* precision of the inner H·v (FP64 for the plain method)    */
  int refine;          /* 1: FP64 outer residual correction (mixed precision)       */
  int inner_iter;      /* mixed: low-precision steps per correction solve          */
  int outer_max;       /* mixed: maximum FP64 outer iterations                      */
  int check_every;     /* plain: convergence test every this many steps             */
  int start_reorth;    /* mixed: Gram-Schmidt passes per step of the low-precision
                          start (2 = full reorthogonalisation as in the plain solve,
                          1 = one pass, 0 = the three-term recurrence only)          */
  int refine_precision;/* mixed: H·v of the outer loop's residuals, DMRG2D_FP64 or
                          DMRG2D_FP64X (float pairs)                                 */
  int thick_keep;      /* plain Lanczos, at a full basis: 0 = explicit restart from the
                          lowest Ritz vector; p in 1..32 = thick restart (Wu and Simon)
                          keeping the p lowest Ritz vectors and the next Lanczos vector,
                          the kept space re-tridiagonalised so the recurrence goes on  */
} dmrg2d_solver_opts;

typedef struct dmrg2d_solver_stats {
  int iters;           /* Lanczos / inner steps taken                               */
  int outer;           /* FP64 outer iterations (mixed)                             */
  int n_hv_fp64;       /* FP64 H·v calls                                            */
  int n_hv_low;        /* low-precision H·v calls                                   */
  double resid;        /* final ||H x - theta x|| (FP64)                            */
  double hv_ms;        /* device time spent in H·v launches (CUDA events)           */
  double elapsed_ms;   /* wall time of the call                                     */
} dmrg2d_solver_stats;

/* x_inout: device double[n_vec]; on entry the start vector (any norm, nonzero),
 * on exit the normalised ground-state estimate.  energy_out: host double.
 * Allocates its Krylov basis on the device for the duration of the call.
 * Returns OK, ENOCONV (estimate kept), ENAN, or an allocation/CUDA error. */
int dmrg2d_lanczos_ground(const dmrg2d_ops* ops, const dmrg2d_solver_opts* opts,
                          double* x_inout, double* energy_out,
                          dmrg2d_solver_stats* stats, void* stream);

/* Lowest eigenpair of the symmetric tridiagonal matrix T (diagonal alpha[0..k),
 * off-diagonal beta[0..k-1)) — the small eigenproblem inside every Lanczos solve of the
 * superblock (the paper's exact diagonalisation names no eigensolver).  One block: the
 * eigenvalue by multisection on Sturm counts (257 points per round), the eigenvector by
 * the twisted factorisation of T - theta (inverse iteration as the fallback).
 *   alpha, beta: device, k doubles each (beta[k-1] is the coupling of the Krylov space to
 *   the next Lanczos vector: it enters only the residual estimate out[1]).
 *   s: device, k doubles, receives the unit eigenvector (first nonzero entry positive).
 *   out: device, 3 + 5k doubles: out[0] = eigenvalue, out[1] = |beta[k-1] s[k-1]|,
 *   out[2] = 0 (ok) or 1 (a non-finite entry); the rest is workspace.
 * 1 <= k <= 512 (else ESHAPE).  Asynchronous on `stream`; allocates nothing. */
int dmrg2d_tridiag_lowest(const double* alpha, const double* beta, int k, double* s,
                          double* out, void* stream);

/* Allocation-free variant of dmrg2d_lanczos_ground for small superblocks.  The
 * paper has no counterpart; it exists for callers that cannot call cudaMalloc:
 * applications whose device memory is owned by another allocator (for example a
 * framework's caching allocator that has reserved most of the device up front, so a
 * second allocation fails or fragments its pool), and latency-critical loops that
 * cannot afford cudaMalloc's implicit synchronisation.  This call allocates nothing
 * (no cudaMalloc, cudaFree, pinned host buffer or CUDA event).  Its scratch — the
 * Krylov basis (krylov_dim + 1 vectors), one work vector, reduction partials and
 * small arrays — lives in one static device array of DMRG2D_NOALLOC_SCRATCH_DOUBLES
 * doubles (16 MiB) that every GPU which loads the library holds until the process
 * exits.
 *   Limits: plain FP64 Lanczos only (precision = DMRG2D_FP64, refine = 0, else
 *   EUNSUPPORTED); krylov_dim, after clamping to max_iter + 1, at most 512 (else
 *   ESHAPE); (krylov_dim + 2) * n_vec + 1226 * (krylov_dim + 1) + 64 doubles must fit
 *   in the array, else ESHAPE with the sizes in dmrg2d_last_error().
 *   Device: the ops object's device must be current (else EINVAL), since the array is
 *   one per device.
 *   Sector-restricted ops: the padding rows of x_inout are set to zero first, as in
 *   dmrg2d_lanczos_ground.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before
 *   any stream capture.
 *   Sharing: all calls on a device use the same array and it keeps the last call's
 *   contents; every value the solver reads from it is written earlier in the same
 *   call.  Calls that overlap on the GPU (other streams or host threads) race and
 *   corrupt each other's results: serialise them.
 * Arguments, results and status codes are those of dmrg2d_lanczos_ground; stats
 * hv_ms is not measured (0). */
#define DMRG2D_NOALLOC_SCRATCH_DOUBLES (2u << 20)
int dmrg2d_lanczos_ground_noalloc(const dmrg2d_ops* ops, const dmrg2d_solver_opts* opts,
                                  double* x_inout, double* energy_out,
                                  dmrg2d_solver_stats* stats, void* stream);

/* Tensor-core tile configurations of the H_l V + V H_r^T kernel.  Index 0 is the
 * dense kernel (dense superblocks with m1 % 128 == 0 and m4 = 128 or m4 % 256 == 0);
 * index 1 + c is the grouped kernel (any sector structure; dense superblocks with
 * m1 % 8 == 0) with pieces of 128 x 128 (c = 0..2) or 128 x 256 (c = 3..5) in
 * column-slab, row-slab or longest-first order; index 7 is the dense kernel reading
 * each distinct operator block once (up to sign) from a small replicated pool; indices
 * 8 and 9 are the dense kernel (per-position blocks / pool) visiting the output tiles
 * (i2, i3) in 8 x 8 patches instead of column slabs, so that the operator rows and V
 * tiles one wave of pieces reads stay in L2; indices 10 and 11 are the CTA-pair kernel
 * (m1 % 256 == 0, m4 % 256 == 0: two SMs share one 256 x 256 tile through M = 256
 * tensor-core instructions) in column-slab / blocked order, and 12 and 13 the same
 * reading the deduplicated operator pool; 14 + c (c = 0..5, sector-restricted
 * superblocks) is grouped configuration c with the scalar moves in a separate kernel
 * instead of the grouped kernel's epilogue; 20 and 21 are the dense kernel / CTA-pair
 * kernel in two passes over the output: H_l V with the moves inside a block column and
 * H_c in column-slab order, then V H_r^T with the moves inside a block row in row-slab
 * order, added to the stored Y (each pass finds the V tiles it reads in L2); 22
 * (sector-restricted superblocks) is the pair of segment kernels for sectors of tens of
 * states: H_l V with the MMA's M = 128 along the columns of each V_q and N = one row
 * segment (the grouped kernel's operands with their roles swapped), then V H_r^T with M
 * along the rows and N = one column segment, N rounded up to 16, K steps past a block's K
 * skipped, the scalar moves in their own kernel (y must be 16-byte aligned); 23 and 24
 * are configurations 11 (CTA pair, blocked order) and 8 (dense kernel, blocked order)
 * with the MN-major V operand of V H_r^T fetched per pipeline stage by one 3-D tensor
 * copy (a row within a block of rows, the column, the row block) instead of one 2-D box
 * per block of rows (same shared-memory image, same results); 25 and 26 are configuration
 * 23 with the output tiles visited in 4 x 4 / 16 x 16 patches instead of 8 x 8.
 * dmrg2d_autotune times a complete H·v (scalar moves included) with every
 * configuration that applies (one warm-up and three timed launches each, on scratch
 * buffers it allocates and frees), keeps the fastest for later apply_H and solver
 * calls at `precision` (TF32 or BF16), and returns its index in *best; ms[i]
 * (optional, n_ms entries) receives candidate i's time, -1 when it does not apply.
 * The call synchronises the stream.  dmrg2d_set_tile_config makes an explicit choice
 * (EUNSUPPORTED if the index does not apply). */
int dmrg2d_autotune(dmrg2d_ops* ops, int precision, int* best, double* ms, int n_ms,
                    void* stream);
int dmrg2d_set_tile_config(dmrg2d_ops* ops, int precision, int index);
const char* dmrg2d_tile_config_name(int index);

void dmrg2d_default_solver_opts(dmrg2d_solver_opts* opts);

/* Failure-detection self-test (library infrastructure; the paper has no counterpart).
 * Every mbarrier wait in the tensor-core kernels is bounded: when it runs out, the
 * kernel records the site in a device flag, stops issuing work, releases its tensor
 * memory and returns, so the context stays usable and dmrg2d_check_device (or the
 * solver) reports ETIMEOUT.  This call runs one kernel whose wait, through the same
 * routine, is on an mbarrier that nothing arrives on, with a limit of `seconds`
 * (0 < seconds <= 2).  Returns ETIMEOUT when the wait gave up and reported it (the
 * expected outcome), ECUDA otherwise, EINVAL for a bad limit.  Synchronises `stream`. */
int dmrg2d_wait_selftest(double seconds, void* stream);

/* Kernel timing for benchmarks.  After dmrg2d_profile_start, every apply_H call
 * records a CUDA event pair around its dominant kernel (the fused H_l V + V H_r^T
 * contraction) on the call's stream, for at most max_launches calls; the event
 * pairs are created here, so apply_H still allocates nothing.
 * dmrg2d_profile_stop waits for the recorded events, returns the summed kernel
 * time in milliseconds and the number of timed launches, and turns timing off. */
int dmrg2d_profile_start(dmrg2d_ops* ops, int max_launches);
int dmrg2d_profile_stop(dmrg2d_ops* ops, double* total_ms, int* launches);

/* Waits for the device, then reports whether a tensor-core kernel launched with
 * these ops gave up a bounded wait since the last check (every wait on the
 * device ends after at most 2 s and sets a flag instead of hanging).
 * Returns OK, ETIMEOUT (flag found and cleared) or ECUDA. */
int dmrg2d_check_device(const dmrg2d_ops* ops);

/* Diagonal of H in the vector layout of `ops` (dense or packed; 0 on padding rows):
 * H(i1 i2 i3 i4; same) = H_l diagonal + H_r diagonal + H_c diagonal (Eq. (dec)).
 * out: caller-owned device double[info.n_vec].  Synchronises the stream. */
int dmrg2d_diagonal(const dmrg2d_ops* ops, double* out, void* stream);

/* ---- Davidson with a diagonal or learned preconditioner ----------------------------
 * Lowest eigenpair by Davidson: expand an orthonormal basis V by the preconditioned
 * residual t = M(theta) r, Rayleigh-Ritz on V^T H V, restart from the Ritz vector when
 * V holds max_subspace vectors.  Preconditioners: NONE (t = r), JACOBI
 * (t_i = r_i / (theta - D_i), D = diag H), MLP (t_i = (r_i / s_D) j(d_i) (1 + y(x_i)):
 * the Jacobi factor j(d) = -clamp(1/d, +-16) in units of s_D, corrected by the output y
 * of a trained dmrg2d_mlp, see below; y = 0 is plain Jacobi).  With precision TF32/BF16 the basis images H V use the
 * low-precision H~·v; refine = 1 then finishes with the FP64 outer loop of
 * dmrg2d_lanczos_ground (tolerance refine_tol, inner_iter CG steps, outer_max steps).
 * Stops when ||H x - theta x|| <= tol * |theta|.  log_cap > 0 records the first
 * log_cap Ritz vectors (log_x) and residuals (log_r) — caller-owned device arrays of
 * log_cap * n_vec doubles, either may be NULL — and theta values (log_theta, host). */
enum { DMRG2D_PRECOND_NONE = 0, DMRG2D_PRECOND_JACOBI = 1, DMRG2D_PRECOND_MLP = 2 };
typedef struct dmrg2d_mlp dmrg2d_mlp;
typedef struct dmrg2d_davidson_opts {
  int max_iter;
  int max_subspace;     /* 4..48                                                     */
  double tol;
  int precision;
  int refine;
  int precond;
  const dmrg2d_mlp* mlp;
  int inner_iter, outer_max;
  double refine_tol;
  int log_cap;
  double* log_x;
  double* log_r;
  double* log_theta;
} dmrg2d_davidson_opts;
void dmrg2d_default_davidson_opts(dmrg2d_davidson_opts* opts);
int dmrg2d_davidson_ground(const dmrg2d_ops* ops, const dmrg2d_davidson_opts* opts,
                           double* x_inout, double* energy_out, dmrg2d_solver_stats* stats,
                           void* stream);

/* ---- the learned preconditioner's network -------------------------------------------
 * A pointwise MLP, 4 inputs -> hidden (tanh) -> hidden (tanh) -> 1, FP32 parameters in
 * one device array: W1[hidden][4], b1[hidden], W2[hidden][hidden], b2[hidden],
 * w3[hidden], b3.  Inputs of component i (d_i = (D_i - theta)/s_D, s_D the RMS of
 * D - theta): clamp(d_i, +-8), clamp(1/d_i, +-16)/16, clamp of the sector's mean
 * (D - theta)/s_D, log(sector size)/16.  Output layer initialised to zero (y = 0:
 * Jacobi).  Trained on weighted least squares
 *   L = 1/(2B) sum_b (w_b y(X_b) - T_b)^2
 * with batches built by dmrg2d_mlp_make_batch from a logged Davidson step (x_k, r_k,
 * theta_k) and the converged vector x_f: w = (r_i/s_D) j(d_i)/s_t,
 * T = alpha delta_i / s_t - w, delta = x_f - (x_k . x_f) x_k,
 * alpha = (delta . t_J)/(delta . delta), t_J the Jacobi correction and s_t its RMS (so
 * w y - T = ((r/s_D) j (1 + y) - alpha delta)/s_t).  All arrays are device arrays unless
 * noted; X is B x 4.  The Davidson solver evaluates y exactly on 1024 values of d per
 * sector each step and interpolates linearly in between. */
int dmrg2d_mlp_create(int hidden, uint64_t seed, dmrg2d_mlp** out);
void dmrg2d_mlp_free(dmrg2d_mlp* mlp);
int dmrg2d_mlp_num_params(const dmrg2d_mlp* mlp);
int dmrg2d_mlp_get_params(const dmrg2d_mlp* mlp, float* host_params);
int dmrg2d_mlp_set_params(dmrg2d_mlp* mlp, const float* host_params);  /* resets Adam */
int dmrg2d_mlp_forward(dmrg2d_mlp* mlp, const float* X, float* Y, int B, void* stream);
int dmrg2d_mlp_loss_grad(dmrg2d_mlp* mlp, const float* X, const float* w, const float* T, int B,
                         float* grad, float* loss_host, void* stream);
int dmrg2d_mlp_train_step(dmrg2d_mlp* mlp, const float* X, const float* w, const float* T, int B,
                          float lr, float* loss_host, void* stream);  /* one Adam step */
int dmrg2d_mlp_make_batch(const dmrg2d_ops* ops, const double* x_k, const double* r_k,
                          double theta, const double* x_final, const double* D,
                          const int64_t* idx, int B, float* X, float* w, float* T,
                          void* stream);

void dmrg2d_free_ops(dmrg2d_ops* ops);

/* ---- finite-system direct 2-D DMRG around the superblock H·v ----------------------------
 * The paper's algorithm (its description around Fig. 2): a DMRG step takes the
 * superblock block 1 + column 2 + column 3 + block 4, finds its ground state (HMED:
 * dmrg2d_lanczos_ground on dmrg2d_build_ops), forms the reduced density matrix of the
 * half that grows (DMF: rho_L = V V^T over (i1, i2), or rho_R = V^T V over (i3, i4)),
 * diagonalises it (DMD) and keeps its m leading eigenvectors U as the basis of the new
 * block, into which the block Hamiltonian and the boundary-column operators are
 * transformed (U^T O U).  Blocks grow by one whole column.  The infinite-system warm-up
 * grows block 1 and its mirror image block 4 together until the superblock spans the
 * lattice; each finite sweep then moves to the right end, to the left end and back to
 * the middle.
 * Supported: Heisenberg ladders (model->kind == DMRG2D_HEISENBERG, n_legs <= 8), open
 * along the legs, n_columns even and >= 4; dense superblocks, or (use_sectors) the
 * S^z_tot = 0 sector: blocks carry their states' N_up (grouped by label), the superblock
 * H·v runs on the sector-restricted layout, and the density matrix, block diagonal in
 * the growing half's label, is diagonalised sector by sector (dsyevd; dsyevdx for the m
 * largest eigenpairs of a sector with more than m states; sectors on concurrent streams),
 * keeping the m largest eigenvalues over all sectors; the renormalisation of spin blocks
 * and the wavefunction transformation run label by label on the sector structure.  Hubbard ladders (DMRG2D_HUBBARD, n_legs <= 4,
 * use_sectors = 1, else EUNSUPPORTED): the target sector is (n_up, n_dn) electrons on
 * the whole ladder (on the warm-up's smaller superblocks the same filling per column,
 * rounded half up); blocks carry the creation operators of their boundary column, their
 * parity and (N_up, N_dn) labels; block 4 grows from its own density matrix during the
 * warm-up (a mirrored fermion block would have the reversed mode order), both blocks from
 * one ground state; every step records the site densities of its central columns
 * (report->densities).  Labels of a growing block that the superblock's target leaves
 * empty (its density matrix is zero there, as on the warm-up's smaller superblocks) keep
 * their states with weight 0 while m allows, so that larger superblocks find them.
 * Density matrices and their eigenvectors are FP64 on the GPU (cuBLAS DSYRK, cuSOLVER
 * dsyevd / dsyevdx); ties in the density-matrix spectrum keep the eigenvectors the solver
 * returns last.
 * Ground states: `precision` FP64 runs the plain Lanczos (thick restart keeping
 * krylov_dim / 4 Ritz vectors, at most 16); TF32/BF16/BF16X3 the mixed solver with FP64
 * refinement (its outer-loop H·v in float pairs, DMRG2D_FP64X) where the tensor-core path
 * supports the superblock's shapes (plain FP64 otherwise).  solver =
 * DMRG2D_SWEEP_DAVIDSON takes dmrg2d_davidson_ground instead (basis of krylov_dim
 * vectors, clamped to 4..48; max_iter Davidson steps; with TF32/BF16/BF16X3
 * the low-precision stage stops at a residual of 1e-3 |E| (1e-2 for BF16) and the FP64
 * outer loop finishes at tol), preconditioned by `precond` (DMRG2D_PRECOND_NONE / JACOBI
 * / MLP).  With DMRG2D_PRECOND_MLP, `mlp` (caller-owned, not NULL) is the learned
 * preconditioner, trained inside the sweep when mlp_epochs > 0: every solve of the
 * warm-up and of the sweeps with index < mlp_train_sweeps runs plain Jacobi Davidson,
 * records its first 16 steps (Ritz vector, residual, Ritz value) and then takes
 * mlp_epochs passes over them, one Adam step (learning rate 3e-4) of 8192 samples drawn
 * by a seeded generator per recorded step, on the pairs dmrg2d_mlp_make_batch forms with
 * the converged vector; the later solves precondition with the network.  mlp_epochs = 0
 * uses the network as given.  Training time is reported apart (train_seconds).
 * Warm-up steps start from a seeded random vector; every
 * finite-sweep step starts from the previous ground state carried into its basis (the
 * wavefunction transformation: the new block's U and the stored U of the block that
 * splits into a smaller block and a column).
 * report: caller-owned arrays of `cap` entries receive, per step in order, the
 * superblock ground energy, the truncation error 1 - (kept weight), the number of
 * columns in block 1, the sweep index (-1 for the warm-up) and the solver's steps
 * (Lanczos steps, low-precision inner steps of the mixed solver, or Davidson steps plus,
 * in mixed precision, the outer loop's inner steps); n_steps counts all
 * steps (entries beyond cap are not stored).  Synchronises `stream`.
 * Errors: EINVAL (bad options), EUNSUPPORTED (model), solver and CUDA errors. */
typedef struct dmrg2d_sweep_opts {
  int n_columns;       /* L: columns of the ladder (even, >= 4)                       */
  int m_warmup;        /* states kept during the warm-up                              */
  int n_sweeps;        /* finite sweeps                                               */
  const int* m_sweep;  /* states kept in sweep s (n_sweeps entries)                  */
  int precision;       /* H·v precision of the ground-state solves                    */
  double tol;          /* ground-state residual tolerance (relative to |E|)           */
  int max_iter;        /* Lanczos steps per solve (plain) / inner steps (mixed)       */
  int krylov_dim;      /* Lanczos basis before restart                                */
  uint64_t seed;       /* start vectors                                               */
  int use_sectors;     /* 1: S^z_tot = 0 sector-restricted superblocks (blocks carry  */
                       /*    N_up labels, density matrices per sector)               */
  int n_up, n_dn;      /* Hubbard ladders: electrons of each spin on the whole ladder */
  int solver;          /* DMRG2D_SWEEP_LANCZOS (0) or DMRG2D_SWEEP_DAVIDSON (1)         */
  int precond;         /* Davidson preconditioner (DMRG2D_PRECOND_*)                    */
  dmrg2d_mlp* mlp;     /* DMRG2D_PRECOND_MLP: the network (trained in place, see above) */
  int mlp_train_sweeps;/* the warm-up and sweeps below this index train the network     */
  int mlp_epochs;      /* passes over each training solve's recorded steps (0: none)    */
} dmrg2d_sweep_opts;
enum { DMRG2D_SWEEP_LANCZOS = 0, DMRG2D_SWEEP_DAVIDSON = 1 };

typedef struct dmrg2d_sweep_report {
  int cap;             /* entries the arrays below hold                               */
  int n_steps;         /* steps done                                                  */
  double* energy;
  double* trunc;
  int* l;
  int* sweep;
  int* iters;          /* ground-state solver steps (Lanczos or inner low-precision)  */
  /* observables of each step's superblock ground state (the paper's bond energies):
   * leg_bond[step * n_legs + y] = <S_(2,y) . S_(3,y)> between the two central columns,
   * rung_bond[step * max(n_legs - 1, 1) + y] = <S_(2,y) . S_(2,y+1)> in column 2,
   * s2[step] = <S_tot^2> at the last step of each sweep (back in the middle; also the
   * single warm-up step of a 4-column lattice) — the Lieb-Mattis check: 0 for the
   * ladder's ground state — NaN elsewhere.  Column 2 is
   * lattice column l (0-based).  Any of the three may be NULL. */
  double* leg_bond;
  double* rung_bond;
  double* s2;
  /* Hubbard ladders: the site densities of the two central columns of each step's
   * ground state, densities[step * (8 n_legs + 2) + ...] in the layout of
   * dmrg2d_site_densities (n_up, n_dn, hole density, staggered spin density per site;
   * then S(x) of both columns).  May be NULL. */
  double* densities;
  double seconds;      /* wall time of the call, of which:                            */
  double solve_seconds;/*   ground-state solves (dmrg2d_lanczos_ground)              */
  double build_seconds;/*   superblock operator assembly (dmrg2d_build_ops)          */
  double dm_seconds;   /*   density matrix and its eigenvectors                      */
  double renorm_seconds;/*  new block operators U^T O U and their copy to the host   */
  double obs_seconds;  /*   observables                                              */
  double train_seconds;/* training of the learned preconditioner (not in solve_seconds)  */
  double transform_seconds; /* wavefunction transformations (the next step's start)   */
} dmrg2d_sweep_report;

/* A DMRG run in progress: the model, the lattice and its filling, every block built so far
 * (block 1 and block 4 of each length: host operators, device truncation matrices), the
 * ground state carried to the next step and the sweep count.  dmrg2d_state_create takes
 * the model and, from opts, the fields that fix the run: n_columns, m_warmup, seed,
 * use_sectors, n_up, n_dn (validated as for dmrg2d_sweep; EINVAL / EUNSUPPORTED); it does
 * no device work.  dmrg2d_sweep then runs the warm-up on the first call and, on every
 * call, opts->n_sweeps more finite sweeps (sweep indices in the report continue from the
 * earlier calls; each sweep's first step starts from the ground state the previous call
 * left), with that call's solver options (precision, tol, max_iter, krylov_dim, solver,
 * precond, mlp, mlp_train_sweeps, mlp_epochs); its
 * lattice fields must equal the state's (else EINVAL).  Two calls of one sweep each do
 * exactly what one call of two sweeps does.  After a failed call the state is unusable
 * (later calls return EINVAL): free it.  A state is used by one host thread at a time. */
typedef struct dmrg2d_state dmrg2d_state;
typedef struct dmrg2d_state_info {
  int n_columns;       /* L                                                              */
  int warmed_up;       /* 1 once the warm-up has run                                     */
  int sweeps_done;     /* finite sweeps completed over all calls                         */
  double last_energy;  /* superblock ground energy of the last step                      */
  int m_left, m_right; /* states of block 1 and block 4 at the middle (L/2 - 1 columns)   */
  int failed;          /* 1 after a failed call                                          */
} dmrg2d_state_info;
int dmrg2d_state_create(const dmrg2d_model* model, const dmrg2d_sweep_opts* opts,
                        dmrg2d_state** out);
void dmrg2d_state_free(dmrg2d_state* state);
int dmrg2d_state_get_info(const dmrg2d_state* state, dmrg2d_state_info* info);
int dmrg2d_sweep(dmrg2d_state* state, const dmrg2d_sweep_opts* opts,
                 dmrg2d_sweep_report* report, void* stream);

/* Site densities of the two central columns of a superblock state: the observables of
 * the paper's Hubbard study, hole density h(x,y) = 1 - <n_{x,y,up} + n_{x,y,dn}> (its
 * Eq. (hole)) and staggered spin density s(x,y) = <n_{x,y,up} - n_{x,y,dn}> (which the
 * Lieb-Mattis theorem makes vanish on every site of the finite ladder's ground state),
 * with S(x) = max_y |s(x,y)|.  A DMRG step measures the sites of columns 2 and 3, which
 * one superblock holds exactly.
 *   x:   device, FP64, n_vec elements in the layout of ops (dense, or the packed sector
 *        layout of a sector-restricted ops; padding rows are ignored); not modified and
 *        need not be normalised (the densities are divided by <x|x>).
 *   out: device, 8 n_legs + 2 doubles, written: out[4 (c n_legs + y) + k] for column
 *        c = 0 (block 2) / 1 (block 3), leg y, k = 0 n_up, 1 n_dn, 2 h, 3 s; then
 *        out[8 n_legs + c] = S(c).  For a spin model n_up / n_dn are the probabilities
 *        of up / down on the site (h = 0, s = 2 <S^z>).
 * One pass over x bins |x|^2 by each element's column states (i2, i3); the occupation
 * numbers are diagonal in the column basis.  The call allocates small scratch
 * (layout tables and 2 d bins) and synchronises the stream.  Errors: EINVAL on a NULL
 * argument; ENOMEM / ECUDA from the allocation or launches. */
int dmrg2d_site_densities(const dmrg2d_ops* ops, const double* x, double* out, void* stream);

/* Thread-local text of the last error of this thread ("" if none). */
const char* dmrg2d_last_error(void);

/* Library version string. */
const char* dmrg2d_version(void);

/* sizeof of a public struct as this library was compiled, for bindings that mirror the
 * structs (an ABI check; no device work): which = DMRG2D_STRUCT_*; 0 for an unknown
 * value. */
enum {
  DMRG2D_STRUCT_MODEL = 0, DMRG2D_STRUCT_BLOCK = 1, DMRG2D_STRUCT_OPS_INFO = 2,
  DMRG2D_STRUCT_SOLVER_OPTS = 3, DMRG2D_STRUCT_SOLVER_STATS = 4,
  DMRG2D_STRUCT_DAVIDSON_OPTS = 5, DMRG2D_STRUCT_SWEEP_OPTS = 6,
  DMRG2D_STRUCT_SWEEP_REPORT = 7, DMRG2D_STRUCT_STATE_INFO = 8
};
size_t dmrg2d_struct_size(int which);

#ifdef __cplusplus
}
#endif
#endif /* DMRG2D_H */
