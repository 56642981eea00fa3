// Internal declarations shared by the translation units of libmc.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mc.h"

#define MCL MC_MAX_CONTINUA
// partial-sum quantities reserved per reduction slot (all persistent kernels)
#define MC_KMAX_ALLOC (8 * MCL)
// Threads per CTA of the FP64 step kernels (the stencil tile code is built for
// this count; launches must use it).
#define MC_STEP_THREADS 256

// Everything the persistent time-stepping kernel needs, passed by value.
// Field pointers address ny rows of `pitch` doubles, cell (i, j) at
// j*pitch + i; the pitch is nx rounded up to 16 and the padding stays zero.
struct StepParams {
  int nx, ny, L, pitch;
  long long N;         // nx * ny
  long long Np;        // ny * pitch
  int scheme;          // MC_SCHEME_*
  int nsteps;
  int max_iter;
  int tiles_x, tiles_y;  // stencil tiles per continuum
  double rtol;
  double tau;
  double mtau[MCL];                // c_a h^2 / tau
  double mass[MCL];                // c_a h^2
  double qconst[MCL][MCL];         // sigma_ab h^2 where no per-cell array
  const double* qcell[MCL][MCL];   // per-cell sigma_ab h^2 or nullptr
  double diagc_const[MCL];         // c_a h^2/tau + sum_b q_ab (constant case)
  const double* diagc[MCL];        // same per cell, or nullptr
  const double* TE[MCL];
  const double* TN[MCL];
  const double* invd[MCL];
  const double* F[MCL];
  const double* W[MCL];            // well index q_w |cell| per cell, or nullptr
  const double* FW[MCL];           // W p_w per cell, or nullptr
  double* p[MCL];
  double* pprev[MCL];
  double* r[MCL];
  double* z[MCL];                  // M r, written by the pointwise phase
  double* P[2][MCL];
  double* q[MCL];
  double* partials;                // [2 slots][4 quantities][MCL][nblocks]
  unsigned* bar_count;
  unsigned* bar_gen;
  int* status;                     // mc_status of the run (0 = OK)
  int* steps_done;
  long long* iters;                // [MCL]
  int* max_iters;                  // [MCL]
  double* relres;                  // [MCL]
  double* mass_defect;             // [1]
  long long spin_limit;
  // Jacobi PCG in scaled variables (decoupled FP64 path): sqrt of the
  // diagonal and the scaled face values T / sqrt(d_i d_j); nullptr: the
  // unscaled flux-form iteration
  const double* sqd[MCL];
  const double* tE[MCL];
  const double* tN[MCL];
  const double* qs[MCL][MCL];      // coupled: q_ab / sqrt(d_a d_b) per cell
  // single-pass form of the scaled iteration: w = A~ r (double-buffered) and
  // the search direction p; single_pass selects it
  double* w[2][MCL];
  double* pd[MCL];
  int single_pass;
  // two-level preconditioner (FP64 path; two_level = 0: Jacobi)
  int two_level;
  int nc;                          // coarse unknowns per continuum (stencil tiles)
  int tl_full;                     // coupled: one (L nc)^2 coarse operator in Ainv[0]
  const double* Ainv[MCL];         // nc x nc inverse of the coarse operator
  double* gsum[MCL];               // P^T r (tile sums)
  double* ccor[MCL];               // coarse correction A_c^-1 P^T r
};

// TMA descriptors of the arrays the stencil phase reads through tiles.
// The precision form's single-reduction inner solve also reads a second
// residual buffer (q) and the double-buffered w = A M r through tiles.
struct TmaMaps {
  CUtensorMap r[MCL];
  CUtensorMap P[2][MCL];
  CUtensorMap invd[MCL];
  CUtensorMap q[MCL];
  CUtensorMap w[2][MCL];
  CUtensorMap z[MCL];            // FP64 step kernel: z = M r
};

// Extra state of the precision form (FP32 inner PCG in FP64 refinement).
struct IrParams {
  StepParams sp;                 // FP64 state, coefficients, outer residual in sp.r
  float* r32[MCL];
  float* P32[2][MCL];
  float* q32[MCL];
  float* d32[MCL];
  float* w32[2][MCL];            // single-reduction form: w = A M r (double-buffered)
  float* p32[MCL];               // single-reduction form: search direction
  const float* invd32[MCL];
  const void* TElo[MCL];         // float or bf16 transmissibilities
  const void* TNlo[MCL];
  const float* dc32[MCL];        // FP32 copy of the per-cell diag(A0 - D), or nullptr
  float dcf[MCL];                // its constant value otherwise
  double inner_rtol;
  int ir_max;
  int inner_form;                // MC_INNER_*
  int* ir_sweeps;
  unsigned* abort_word;          // raised by a timed-out barrier; every barrier polls it
};

// Per-instance record of the batched precision form (device memory).
struct BatchInst {
  int status;                    // mc_status of the instance (0 = OK)
  int steps_done;                // steps completed since the last reset
  int ir_sweeps;
  int busy;                      // 1 while a team holds the instance mid-step
  long long iters[MCL];
  int max_iters[MCL];
  double relres[MCL];            // ||r|| / ||b|| at the end of the last solve
};

// Everything the batched persistent kernel needs, passed by value. The grid
// is split into `teams` teams of `team` CTAs; each team takes instances from
// a shared counter in the order `order` (largest first) and runs the
// precision-form step of that instance with team-scoped barriers.
struct BatchParams {
  const IrParams* inst;          // [n] (device), per-instance pointers and constants
  const TmaMaps* maps;           // [n] (device)
  const int* order;              // [n] instance indices, largest first
  BatchInst* st;                 // [n]
  int n;
  int team, teams;
  int scheme;
  double rtol;
  double inner_rtol;
  int max_iter, ir_max;
  int inner_form;                // MC_INNER_*
  long long spin_limit;
  unsigned* ctrl;                // [0] queue; team t: u64 barrier count at 32(t+1),
                                 // ticket at 32(t+1)+4 (zeroed before each launch)
  unsigned* abort_word;          // zeroed before each batched call
  double* partials;              // team t: [2 slots][MC_KMAX_ALLOC][team] from t*2*KM*team
};

struct mc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, L = 0, pitch = 0;
  long long N = 0, Np = 0;
  TmaMaps maps;
  double h = 0, tau = 0;
  double c[MCL] = {};
  double sigma[MCL][MCL] = {};
  mc_opts opts{};
  int num_sms = 0;
  // device buffers
  double* k[MCL] = {};      // permeability (pitched), kept for the NLMC build
  double* TE[MCL] = {};
  double* TN[MCL] = {};
  double* invd[MCL] = {};
  double* sqd[MCL] = {};           // sqrt(diag) and scaled faces (FP64 scaled PCG)
  double* tE[MCL] = {};
  double* tN[MCL] = {};
  double* qs[MCL][MCL] = {};       // scaled exchange of each pair (qs[a][b] == qs[b][a])
  double* w64[2][MCL] = {};        // single-pass FP64 iteration: w buffers, search direction
  double* pd[MCL] = {};
  double* diagc[MCL] = {};
  double* qcell[MCL][MCL] = {};
  double* F[MCL] = {};
  double* W[MCL] = {};             // wells in effect (mc_set_well), nullptr when none
  double* FW[MCL] = {};
  double* W_buf[MCL] = {};         // the well buffers, kept across removal / re-adding
  double* FW_buf[MCL] = {};
  double* p[MCL] = {};
  double* pprev[MCL] = {};
  double* r[MCL] = {};
  double* z[MCL] = {};
  double* P[2][MCL] = {};
  double* q[MCL] = {};
  double* partials = nullptr;
  size_t partials_len = 0;
  // two-level preconditioner (allocated and factorised on first use)
  double* tl_Ainv[MCL] = {};
  double* tl_g[MCL] = {};
  double* tl_c[MCL] = {};
  double* tl_work = nullptr;
  unsigned* tl_bar = nullptr;
  int tl_nc = 0;
  int tl_ready = 0;
  double* tl_Afull = nullptr;      // coupled: (L nc)^2 inverse of the Galerkin coarse operator
  double* tl_work_full = nullptr;
  int tl_full_ready = 0;
  int maxb = 0;                    // CTAs the partials buffer is sized for
  // precision form (allocated on first use)
  float* r32[MCL] = {};
  float* P32[2][MCL] = {};
  float* q32[MCL] = {};
  float* d32[MCL] = {};
  float* w32[2][MCL] = {};
  float* p32[MCL] = {};
  float* invd32[MCL] = {};
  float* TElo32[MCL] = {};         // FP32 copies, or BF16 in their first half
  float* TNlo32[MCL] = {};
  float* dc32[MCL] = {};           // FP32 per-cell diag(A0 - D) when exchange varies per cell
  int lo_kind = 0;                 // 0 none, 1 FP32, 2 BF16
  TmaMaps maps32;
  int* dsweeps = nullptr;
  unsigned* bar = nullptr;         // [0] count, [32] generation (own sector)
  int* dstatus = nullptr;
  int* dsteps = nullptr;
  long long* diters = nullptr;
  int* dmaxit = nullptr;
  double* drelres = nullptr;
  double* dmass = nullptr;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  std::string err;
};

// Allocation helper: zero-filled device buffer tracked by the context.
cudaError_t mc_alloc(mc_ctx* ctx, void** ptr, size_t bytes);

// Fill StepParams from a context (device pointers, constants).
void mc_fill_params(const mc_ctx* ctx, StepParams* sp, int scheme, int nsteps);

// Launch the persistent time-stepping kernel (mc_step.cu).
cudaError_t mc_launch_steps(mc_ctx* ctx, const StepParams& sp, int blocks,
                            int threads);
cudaError_t mc_launch_steps_raw(const StepParams& sp, const TmaMaps& maps, int blocks,
                                int threads, cudaStream_t stream);

// In-place Gauss-Jordan inverse of an n x n SPD matrix on the device (one
// cooperative launch; work holds 2n doubles, bar 96 zeroed words of its own).
cudaError_t mc_gj_invert(double* M, int n, double* work, unsigned* bar, int* status,
                         long long spin_limit, int num_sms, cudaStream_t stream);

// Two-level preconditioner (mc_step.cu): coarse operator A_c = P^T (M/tau + A0) P
// of continuum a on the 64 x 16 stencil tiles (P = tile indicators), dense
// nc x nc, assembled into Ac (overwritten).
cudaError_t mc_launch_coarse_assemble(const mc_ctx* ctx, int a, double* Ac);
// The coupled scheme's Galerkin coarse operator P^T A P with P = blockdiag(P_a):
// (L nc)^2, the per-continuum blocks above plus the exchange blocks.
cudaError_t mc_launch_coarse_assemble_coupled(const mc_ctx* ctx, double* Ac);
int mc_step_tiles(int nx, int ny);

// Maximum co-resident CTAs for the step kernel of this L (cooperative grid).
int mc_step_max_blocks(int L, int threads, int num_sms);
int mc_step_max_blocks_any(int L, int threads, int num_sms);
int mc_step_blocks_for(const StepParams& sp, int threads, int num_sms);
int mc_step_box_x();
int mc_step_box_y();

// Precision form (mc_ir.cu).
int mc_ir_max_blocks(int L, bool bf16, int num_sms);
cudaError_t mc_ir_prepare(mc_ctx* ctx, int bf16);
cudaError_t mc_launch_ir(mc_ctx* ctx, const StepParams& sp, int bf16, int blocks);
// IrParams of a prepared context (mc_ir_prepare done) around StepParams sp.
void mc_ir_fill(const mc_ctx* ctx, const StepParams& sp, IrParams* ip);
// Batched form: co-resident CTAs of the batched kernel, and one launch (one
// time step of every instance) queued on `stream` (cooperative attribute set,
// so it may be captured into a CUDA graph).
int mc_ir_batch_max_blocks(bool bf16, int num_sms);
cudaError_t mc_launch_ir_batch(const BatchParams& bp, int bf16, int blocks, cudaStream_t stream);

// Encode a 2-D tiled tensor map (x innermost) over a pitched array.
cudaError_t mc_encode_map(CUtensorMap* map, CUtensorMapDataType dtype, int esize, void* base,
                          int nx, int ny, int pitch_elems, int box_x, int box_y);

// Row pitch (elements) used for every device field of an nx-wide grid.
inline int mc_pitch_for(int nx) { return (nx + 15) / 16 * 16; }

// Setup kernels (mc_setup_kernels.cu).
cudaError_t mc_launch_setup(mc_ctx* ctx, int a, const double* k_dev);
// Context-free set-up of one continuum without exchange: TE, TN from k and
// invd = 1 / (c h^2 / tau + sum of face T), all pitched.
cudaError_t mc_launch_single_setup(int nx, int ny, int pitch, double h, double c, double tau,
                                   const double* k, double* TE, double* TN, double* invd,
                                   cudaStream_t stream);
cudaError_t mc_launch_diag(mc_ctx* ctx, int a);
// Scaled exchange q_ab / sqrt(d_a d_b) of every pair (after mc_launch_diag of
// every continuum).
cudaError_t mc_launch_pairs(mc_ctx* ctx);
// The same two set-ups into caller-owned arrays, with the diagonal term W
// (per cell, or nullptr) in place of the context's wells.
cudaError_t mc_launch_diag_into(const mc_ctx* ctx, int a, const double* W, double* diagc, double* invd,
                                double* sqd, double* tE, double* tN);
cudaError_t mc_launch_pairs_into(const mc_ctx* ctx, double* const* sqd, double* const (*qs)[MCL]);
// Persistent FP64 step kernel with caller-filled StepParams on the context's
// stream and TMA maps (cooperative launch, default grid).
cudaError_t mc_launch_steps_default(mc_ctx* ctx, const StepParams& sp);
// FW = W * pw in place (FW holds pw on entry), pitched arrays.
cudaError_t mc_launch_well(mc_ctx* ctx, int a);
cudaError_t mc_launch_apply(mc_ctx* ctx, int scheme, double* const* x,
                            double* const* y);
cudaError_t mc_launch_rhs(mc_ctx* ctx, double* const* b);
