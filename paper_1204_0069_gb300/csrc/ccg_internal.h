// ccg_internal.h -- state and launch parameters shared by the C-ABI layer and
// the persistent FP64 solver kernel.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace ccg {

constexpr int kMaxP = 32;          // agents per solve (warp width)
constexpr int kThreads = 256;      // threads per CTA of the persistent kernel
constexpr int kWarps = kThreads / 32;
// SM sub-partitions, one FP64 pipe each (warp w issues on sub-partition
// w mod 4); FP64-bound work that needs few warps uses one per sub-partition
constexpr int kSubParts = 4;
constexpr int kSq = kMaxP * kMaxP;
// Per-CTA partial-sum slot: two p x p Grams, one p-vector, one scalar, each
// entry as an unevaluated sum hi + lo (compensated accumulation): hi at
// [slot], lo at [kPartHalf + slot].
constexpr int kSlotGram0 = 0;
constexpr int kSlotGram1 = kSq;
constexpr int kSlotVec = 2 * kSq;
constexpr int kSlotScalar = 2 * kSq + kMaxP;
constexpr int kPartHalf = 2 * kSq + 2 * kMaxP;
constexpr int kPartStride = 2 * kPartHalf;

// Control word written by the CTA that runs a serial step; every CTA follows
// it after the grid barrier, so control flow is uniform across the grid.
enum Ctrl : int {
  CTRL_LOOP = 0,     // run one cCG iteration
  CTRL_CHECK = 1,    // true residual of the best agent
  CTRL_REPLACE = 2,  // residual replacement R = A X - b 1^T, D = R
  CTRL_FINISH = 3    // write x_out / X_out and leave
};

enum Mode : int {
  MODE_SOLVE = 0,
  MODE_BLOCK_PRODUCT = 1,
  MODE_BARRIER_SELFTEST = 2,
  MODE_REFINE = 3,     // x += c delta; r = b - A x (FP64); scaled residual
  MODE_CHEB = 4        // Z = q(A_lp) R: Chebyshev polynomial preconditioner
};

// Preconditioned FP64 solve (outer loop of the mixed-precision path): the
// step the next launch resumes with once the preconditioner launch has
// written Z = q(A_lp) R.
enum PcStage : int {
  PC_NONE = 0,
  PC_SET_D = 1,   // D_k = Z (after the initial block or a residual replacement)
  PC_BETA = 2     // H = Z'W, beta_k, D_{k+1} = Z + D_k beta_k^T
};

// A-pass policy of the persistent kernel: FP64 A on the FP64 pipe, a
// quantised A on the tensor cores (inner solves of the mixed-precision path),
// or an FP32 copy of A on the FP32 pipe (inner solves of the batched
// mixed-precision path).
enum Policy : int {
  POL_FP64 = 0, POL_BF16 = 1, POL_FP8 = 2, POL_TF32X3 = 3, POL_F32 = 4,
  POL_SLICED = 5  // FP64 cCG with the block product formed exactly from FP8 slices
};

// Status values mirror ccg_status in include/ccg.h.
enum Status : int {
  ST_OK = 0,
  ST_NOT_CONVERGED = 1,
  ST_ERR_INVALID = -1,
  ST_ERR_NOT_SPD = -2,
  ST_ERR_NUMERICAL = -3,
  ST_ERR_OOM = -4,
  ST_ERR_TIMEOUT = -5,
  ST_ERR_CUDA = -6
};

// Device-resident solver state (one per launch, in the handle workspace).
struct DevState {
  unsigned int bar_count;   // grid barrier arrivals
  unsigned int bar_gen;     // grid barrier generation
  int error;                // first error (negative status), 0 if none
  int result;               // ST_OK / ST_NOT_CONVERGED once finished
  int ctrl;                 // Ctrl for the next phase
  int k;                    // iterations so far
  int pk;                   // active agents
  int prev_pk;              // active agents before the last rank test
  int changed;              // 1 if the last rank test removed agents
  int jbest;                // column of the agent returned
  int replacements;
  int drops;
  int k_replaced;           // iteration count at the last replacement
  int zero_rhs;             // b == 0
  int err_where;            // diagnostic: phase that set `error`
  int pc_stage;             // PcStage: preconditioned solve waits for Z
  int cur;                  // preconditioned solve: current direction buffer (0: D0)
  int pad1;
  int keep[kMaxP];          // kept columns (pre-compaction indices)
  int agent[kMaxP];         // original agent id of each active column
  int old_agent[kMaxP];     // agent ids before the last compaction
  double bnorm;
  double relres_true;
  double relres_recur;
  double s[kMaxP];          // ||R e_j||
  double sc[kMaxP];         // diag(M)^{-1/2} of the kept columns
  double L[kSq];            // Cholesky factor of S M S (stride kMaxP)
  double alphaT[kSq];       // (alpha_k^T)[b][a], stride kMaxP
  double betaT[kSq];        // (beta_k^T)[b][a], stride kMaxP
  double gram_out[2 * kSq]; // block-product mode: M, G (stride kMaxP)
  float sigma[kMaxP];       // FP8 operand column scales
  double rnorm;             // refinement mode: ||b - A x||
  double red[kPartHalf];    // cross-CTA sums of the partial slots (same offsets)
};

// Serving kernel: one request of the ring (written by the host).
struct ServeDesc {
  int64_t n, lda;
  const double* A;
  const double* b;
  double* x;
  double tol;
  int maxit;
  int p;
  int64_t seq;             // ring position + 1 once written (guards against stale reads)
};
// Claim and result of one ring entry (written by the kernel, read by the host).
struct ServeOut {
  int64_t claimed;         // seq once a slot took the request
  int64_t done;            // seq once the result below is final
  int status;
  int iterations;
  double relres_true;
  int slot;
  int pad;
  long long t_start_ns;    // device clock (%globaltimer) at claim and at the end
  long long t_end_ns;
};
// Per slot: arrival counter and generation of the slot barrier, the ticket
// (ring position of the slot's next request, or -1: leave).
struct SlotSync {
  unsigned count;
  unsigned gen;
  int ticket;
  int pad;
};
struct ServeCtl {
  unsigned head;           // requests claimed
  int busy;                // slots working on a request
  int closing;             // 1: every slot leaves once idle
  int error;               // a slot barrier gave up (CCG_ERR_TIMEOUT)
};

struct Params {
  int64_t n;
  int64_t lda;
  const double* A;
  const double* b;
  const double* x0;        // ccg_solve: single initial guess (nullable)
  const double* X0;        // ccg_solve_block: explicit initial block
  double spread;
  unsigned long long seed;
  double* X;
  double* R;
  double* D0;
  double* D1;
  double* W;
  double* part;            // gridDim.x * kPartStride partial sums
  DevState* st;
  double* x_out;
  double* X_out;           // nullable, n x p
  int p;                   // agents requested (leading dimension of blocks)
  int maxit;
  double tol;
  double rank_tol;
  int replacement;
  int explicit_residual;   // R_{k+1} = A X_{k+1} - b 1^T instead of the recurrence
  int apass_variant;       // FP64 A-pass shape (0 tiled; 1, 2 narrow with 8 / 2 loads)
  int mode;
  long long timeout_ns;
  unsigned int expected_ctas;  // barrier arrival count
  // block-product mode
  const double* V;
  const double* U;
  double* Wout;
  int q;
  // inner solves (mixed precision): stop on the recurrence residual alone
  int skip_true_check;
  // CTAs that solve one system together (0 = the whole grid) and this CTA's
  // rank in its group; the batched solver runs groups of one CTA
  int group_ctas;
  int group_rank;
  // batched solve: systems taken from a queue, one per CTA at a time
  int64_t batch_count;
  const int64_t* batch_desc;   // per queued system: n, A offset, vector offset, index
  int64_t batch_slot_stride;   // doubles of X, R, D0, D1, W workspace per CTA
  unsigned int* batch_next;    // queue head
  int* batch_status;
  int* batch_iters;
  double* batch_relres;
  // batched FP32 refinement: per CTA slot, r, b_in, delta, x_best (n each)
  // and the FP32 copy of A with the FP32 operand rows
  double* batch_vec;
  int64_t batch_vec_stride;    // doubles per slot
  float* batch_f32;
  int64_t batch_f32_stride;    // floats per slot
  double batch_inner_tol;
  int batch_max_outer;
  int* batch_outer;            // refinement steps per system
  int batch_variant[8];        // A-pass variant per size bucket [2^(b+5), 2^(b+6))
  // FP32 A-pass (POL_F32): A32 row-major with leading dimension a32_ld (a
  // multiple of 4), operand columns as FP32 rows vt32 (stride a32_ld)
  const float* a32;
  int64_t a32_ld;
  float* vt32;
  // tensor-core A-pass (policy != POL_FP64)
  int lp_kc;               // k-chunks per 128-row tile
  int lp_kelems;           // K elements per chunk
  int64_t lp_units;        // row tiles x k-chunks (x slices for POL_SLICED)
  int64_t lp_tiles;        // row tiles of one slice (POL_SLICED)
  const float* lp_row_scale;
  void* lp_dq;             // quantised operand rows (NB x lp_ldk)
  int64_t lp_ldk;
  float* lp_part;          // partial tiles, (grid + tiles) x 128 x NP floats
  // refinement mode
  double* ref_x;
  const double* ref_delta;
  double ref_coef;
  double* ref_r;           // A x - b
  double* ref_bin;         // -(A x - b) * sqrt(n) / ||b - A x||
  // preconditioned FP64 solve: D_{k+1} = Z_{k+1} + D_k beta_k^T with
  // Z = q(A_lp) R written by a MODE_CHEB launch between two launches of the
  // solve (resume = 1 continues from the state in st)
  int precond;
  int resume;
  double* Z;               // n x p, leading dimension p
  // MODE_CHEB: scratch blocks (n x p each) and the polynomial
  double* cheb_d;
  double* cheb_s;
  double* cheb_w;
  int cheb_steps;          // products with A_lp per application
  double cheb_lo;          // interval [cheb_lo, cheb_hi] of the Chebyshev polynomial
  double cheb_hi;
  // serving kernel (continuous batching): slots of serve_group CTAs, each
  // taking requests from a queue the host appends to while the kernel runs
  int serve_group;               // CTAs per slot
  int serve_capacity;            // request ring entries
  const ServeDesc* serve_desc;   // request ring (host memory mapped into the device)
  const int* serve_tail;         // requests posted (host writes, mapped)
  const int* serve_stop;         // 1: leave once idle (host writes, mapped)
  ServeOut* serve_out;           // per ring entry: claim and result (mapped)
  SlotSync* serve_sync;          // per slot: barrier words and ticket (device)
  ServeCtl* serve_ctl;           // claim counter, busy slots, closing flag (device)
  int64_t serve_ws_stride;       // doubles of X, R, D0, D1, W per slot
  long long serve_idle_ns;       // leave after this long with nothing to do
  CUtensorMap lp_tmA;  // A_lp tiles (the type carries its alignment)
  CUtensorMap lp_tmB;  // operand tiles
};

// Launch helpers implemented in ccg_fp64.cu.
// Bucket (1, 2, 4, 8, 16, 32) >= p used for the register tiles.
int p_bucket(int p);
// Dynamic shared memory the kernel needs for bucket P and policy pol.
size_t fp64_smem_bytes(int P, int pol = POL_FP64);
// Max co-resident CTAs per SM of the persistent kernel (0 on error).
int fp64_ctas_per_sm(int P, bool vec, int pol = POL_FP64);
cudaError_t launch_fp64(const Params& prm, int P, bool vec, int ctas,
                        cudaStream_t stream, int pol = POL_FP64);
// Batched solver (groups of one CTA): occupancy and launch.
// ir: the FP32-refinement variant (batch_ir_kernel).
int batch_ctas_per_sm(int P, bool ir = false);
cudaError_t launch_batch(const Params& prm, int P, int ctas, cudaStream_t stream, bool ir = false);
// Serving kernel (slots of CTAs over a request ring): occupancy and launch.
int serve_ctas_per_sm(int P);
cudaError_t launch_serve(const Params& prm, int P, int ctas, cudaStream_t stream);

}  // namespace ccg
