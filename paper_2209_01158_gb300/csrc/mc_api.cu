// C ABI of libmc.so: context life cycle, host <-> device copies, and the
// step entry points that launch the persistent time-stepping kernel.

#include <math.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <new>
#include <string>

#include "mc_internal.h"

namespace {

// Host <-> device copies between dense nx*ny host arrays and pitched fields.
cudaError_t h2d(const mc_ctx* ctx, double* dst, const double* src) {
  return cudaMemcpy2DAsync(dst, ctx->pitch * sizeof(double), src, ctx->nx * sizeof(double),
                           ctx->nx * sizeof(double), ctx->ny, cudaMemcpyHostToDevice, ctx->stream);
}

cudaError_t d2h(const mc_ctx* ctx, double* dst, const double* src) {
  return cudaMemcpy2DAsync(dst, ctx->nx * sizeof(double), src, ctx->pitch * sizeof(double),
                           ctx->nx * sizeof(double), ctx->ny, cudaMemcpyDeviceToHost, ctx->stream);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

thread_local std::string g_setup_err;

mc_status set_err(mc_ctx* ctx, mc_status s, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_setup_err = msg;
  return s;
}

mc_status cuda_err(mc_ctx* ctx, const char* what, cudaError_t e) {
  return set_err(ctx, MC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return cuda_err(ctx, #call, e_);             \
  } while (0)

bool finite_nonneg(const double* x, long long n) {
  for (long long i = 0; i < n; ++i)
    if (!(x[i] >= 0.0) || !isfinite(x[i])) return false;
  return true;
}

void free_all(mc_ctx* ctx) {
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
}

int launch_threads(const mc_ctx* ctx) { return ctx->opts.threads > 0 ? ctx->opts.threads : MC_STEP_THREADS; }

// CTAs of a step launch: the kernel's co-resident count (at most the count the
// partial-sum buffer was sized for), or fewer when mc_opts.blocks asks.
int launch_blocks(const mc_ctx* ctx, const StepParams& sp) {
  int maxb = mc_step_blocks_for(sp, launch_threads(ctx), ctx->num_sms);
  if (maxb > ctx->maxb) maxb = ctx->maxb;
  int b = ctx->opts.blocks > 0 ? ctx->opts.blocks : maxb;
  if (b > maxb) b = maxb;
  return b;
}

mc_status check_opts(const mc_opts* o, std::string* why) {
  if (o->precision < MC_PREC_FP64 || o->precision > MC_PREC_BF16T_IR) { *why = "precision"; return MC_E_ARG; }
  if (o->precond != MC_PRECOND_JACOBI && o->precond != MC_PRECOND_TWO_LEVEL) {
    *why = "precond";
    return MC_E_ARG;
  }
  if (o->max_iter < 1) { *why = "max_iter < 1"; return MC_E_ARG; }
  if (!(o->rtol > 0.0) || !(o->rtol < 1.0)) { *why = "rtol must be in (0, 1)"; return MC_E_ARG; }
  if (o->spin_limit < 1) { *why = "spin_limit < 1"; return MC_E_ARG; }
  if (o->threads != 0 && o->threads != MC_STEP_THREADS) {
    *why = "threads must be 0 or " + std::to_string(MC_STEP_THREADS);
    return MC_E_ARG;
  }
  if (o->blocks < 0) { *why = "blocks < 0"; return MC_E_ARG; }
  if (o->inner_form != MC_INNER_SINGLE_REDUCTION && o->inner_form != MC_INNER_TWO_REDUCTIONS) {
    *why = "inner_form";
    return MC_E_ARG;
  }
  if (o->fp64_form != MC_FP64_TWO_PASS && o->fp64_form != MC_FP64_SINGLE_PASS) {
    *why = "fp64_form";
    return MC_E_ARG;
  }
  return MC_OK;
}

}  // namespace

cudaError_t mc_encode_map(CUtensorMap* map, CUtensorMapDataType dtype, int esize, void* base, int nx,
                          int ny, int pitch_elems, int box_x, int box_y) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
  cuuint64_t strides[1] = {(cuuint64_t)pitch_elems * (cuuint64_t)esize};
  cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dtype, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t mc_alloc(mc_ctx* ctx, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) return e;
  ctx->allocs.push_back(*ptr);
  ctx->bytes += (int64_t)bytes;
  return cudaMemset(*ptr, 0, bytes);
}

void mc_fill_params(const mc_ctx* ctx, StepParams* sp, int scheme, int nsteps) {
  memset(sp, 0, sizeof(*sp));
  sp->nx = ctx->nx;
  sp->ny = ctx->ny;
  sp->L = ctx->L;
  sp->pitch = ctx->pitch;
  sp->N = ctx->N;
  sp->Np = ctx->Np;
  sp->scheme = scheme;
  sp->nsteps = nsteps;
  sp->max_iter = ctx->opts.max_iter;
  sp->rtol = ctx->opts.rtol;
  sp->tau = ctx->tau;
  const double area = ctx->h * ctx->h;
  for (int a = 0; a < ctx->L; ++a) {
    sp->mass[a] = ctx->c[a] * area;
    sp->mtau[a] = ctx->c[a] * area / ctx->tau;
    double dc = sp->mtau[a];
    for (int b = 0; b < ctx->L; ++b) {
      sp->qconst[a][b] = ctx->sigma[a][b] * area;
      sp->qcell[a][b] = ctx->qcell[a][b];
      if (b != a) dc += sp->qconst[a][b];
    }
    sp->diagc_const[a] = dc;
    sp->diagc[a] = ctx->diagc[a];
    sp->TE[a] = ctx->TE[a];
    sp->TN[a] = ctx->TN[a];
    sp->invd[a] = ctx->invd[a];
    sp->sqd[a] = ctx->sqd[a];
    sp->tE[a] = ctx->tE[a];
    sp->tN[a] = ctx->tN[a];
    for (int b = 0; b < ctx->L; ++b) sp->qs[a][b] = ctx->qs[a][b];
    sp->w[0][a] = ctx->w64[0][a];
    sp->w[1][a] = ctx->w64[1][a];
    sp->pd[a] = ctx->pd[a];
    sp->F[a] = ctx->F[a];
    sp->W[a] = ctx->W[a];
    sp->FW[a] = ctx->FW[a];
    sp->p[a] = ctx->p[a];
    sp->pprev[a] = ctx->pprev[a];
    sp->r[a] = ctx->r[a];
    sp->z[a] = ctx->z[a];
    sp->P[0][a] = ctx->P[0][a];
    sp->P[1][a] = ctx->P[1][a];
    sp->q[a] = ctx->q[a];
  }
  sp->partials = ctx->partials;
  sp->bar_count = ctx->bar;
  sp->bar_gen = ctx->bar + 32;
  sp->status = ctx->dstatus;
  sp->steps_done = ctx->dsteps;
  sp->iters = ctx->diters;
  sp->max_iters = ctx->dmaxit;
  sp->relres = ctx->drelres;
  sp->mass_defect = ctx->dmass;
  sp->spin_limit = ctx->opts.spin_limit;
  sp->single_pass = ctx->opts.fp64_form == MC_FP64_SINGLE_PASS ? 1 : 0;
}

cudaError_t mc_launch_steps_default(mc_ctx* ctx, const StepParams& sp) {
  return mc_launch_steps(ctx, sp, launch_blocks(ctx, sp), launch_threads(ctx));
}

extern "C" {

mc_status mc_default_opts(mc_opts* o) {
  if (!o) return MC_E_ARG;
  memset(o, 0, sizeof(*o));
  o->precision = MC_PREC_FP64;
  o->precond = MC_PRECOND_JACOBI;
  o->max_iter = 100000;
  o->ir_max = 50;
  o->rtol = 1e-12;
  o->inner_rtol = 1e-3;
  o->spin_limit = 2000000;
  o->blocks = 0;
  o->threads = 0;
  o->inner_form = MC_INNER_SINGLE_REDUCTION;
  return MC_OK;
}

const char* mc_status_string(mc_status s) {
  switch (s) {
    case MC_OK: return "ok";
    case MC_E_ARG: return "invalid argument";
    case MC_E_ALLOC: return "allocation failed";
    case MC_E_CUDA: return "CUDA error";
    case MC_E_NOCONV: return "no convergence within max_iter";
    case MC_E_TIMEOUT: return "device barrier timeout";
    case MC_E_STATE: return "invalid state";
    case MC_E_BREAKDOWN: return "PCG breakdown";
  }
  return "unknown status";
}

const char* mc_last_error(const mc_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_setup_err.c_str();
}

mc_status mc_setup(const mc_grid* g, int32_t L, const double* const* k, const double* c,
                   const double* sigma, const double* const* sigma_cell, double tau,
                   const mc_opts* opts, void* stream, mc_ctx** out) {
  mc_ctx* ctx = nullptr;
  if (!out) return set_err(nullptr, MC_E_ARG, "out is NULL");
  *out = nullptr;
  if (!g || g->nx < 1 || g->ny < 1) return set_err(nullptr, MC_E_ARG, "grid must have nx, ny >= 1");
  if ((long long)g->nx * g->ny > (1LL << 31)) return set_err(nullptr, MC_E_ARG, "grid larger than 2^31 cells");
  if (L < 1 || L > MC_MAX_CONTINUA) return set_err(nullptr, MC_E_ARG, "L must be in 1..MC_MAX_CONTINUA");
  if (!k || !c) return set_err(nullptr, MC_E_ARG, "k and c are required");
  if (!(tau > 0.0) || !isfinite(tau)) return set_err(nullptr, MC_E_ARG, "tau must be > 0 and finite");
  const long long N = (long long)g->nx * g->ny;
  for (int a = 0; a < L; ++a) {
    if (!(c[a] > 0.0) || !isfinite(c[a])) return set_err(nullptr, MC_E_ARG, "c must be > 0 and finite");
    if (!k[a]) return set_err(nullptr, MC_E_ARG, "k[a] is NULL");
    if (!finite_nonneg(k[a], N)) return set_err(nullptr, MC_E_ARG, "k must be finite and >= 0");
  }
  if (sigma) {
    for (int a = 0; a < L; ++a)
      for (int b = 0; b < L; ++b) {
        if (a == b) continue;
        const double s = sigma[a * L + b];
        if (!(s >= 0.0) || !isfinite(s)) return set_err(nullptr, MC_E_ARG, "sigma must be finite and >= 0");
        if (s != sigma[b * L + a]) return set_err(nullptr, MC_E_ARG, "sigma must be symmetric");
      }
  }
  if (sigma_cell) {
    int pi = 0;
    for (int a = 0; a < L; ++a)
      for (int b = a + 1; b < L; ++b, ++pi)
        if (sigma_cell[pi] && !finite_nonneg(sigma_cell[pi], N))
          return set_err(nullptr, MC_E_ARG, "sigma_cell must be finite and >= 0");
  }
  mc_opts o;
  mc_default_opts(&o);
  if (opts) o = *opts;
  std::string why;
  if (check_opts(&o, &why) != MC_OK) return set_err(nullptr, MC_E_ARG, "opts: " + why);

  ctx = new (std::nothrow) mc_ctx();
  if (!ctx) return set_err(nullptr, MC_E_ALLOC, "host allocation failed");
  ctx->nx = g->nx;
  ctx->ny = g->ny;
  ctx->L = L;
  ctx->N = N;
  ctx->pitch = mc_pitch_for(g->nx);
  ctx->Np = (long long)g->ny * ctx->pitch;
  ctx->h = 1.0 / g->nx;
  ctx->tau = tau;
  ctx->opts = o;
  ctx->stream = (cudaStream_t)stream;
  for (int a = 0; a < L; ++a) {
    ctx->c[a] = c[a];
    for (int b = 0; b < L; ++b) ctx->sigma[a][b] = (sigma && a != b) ? sigma[a * L + b] : 0.0;
  }
  auto bail = [&](mc_status s) {
    g_setup_err = ctx->err;
    free_all(ctx);
    delete ctx;
    return s;
  };
  cudaError_t e;
#define CKS(call)                                                   \
  do {                                                              \
    e = (call);                                                     \
    if (e != cudaSuccess) {                                         \
      cuda_err(ctx, #call, e);                                      \
      return bail(e == cudaErrorMemoryAllocation ? MC_E_ALLOC : MC_E_CUDA); \
    }                                                               \
  } while (0)
  CKS(cudaGetDevice(&ctx->device));
  CKS(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const size_t fb = (size_t)ctx->Np * sizeof(double);
  // Per-cell exchange arrays (sigma first, scaled to q = sigma h^2 on device).
  if (sigma_cell) {
    int pi = 0;
    for (int a = 0; a < L; ++a)
      for (int b = a + 1; b < L; ++b, ++pi) {
        if (!sigma_cell[pi]) continue;
        CKS(mc_alloc(ctx, (void**)&ctx->qcell[a][b], fb));
        ctx->qcell[b][a] = ctx->qcell[a][b];
        CKS(h2d(ctx, ctx->qcell[a][b], sigma_cell[pi]));
      }
  }
  for (int a = 0; a < L; ++a) {
    bool percell = false;
    for (int b = 0; b < L; ++b) percell |= (ctx->qcell[a][b] != nullptr);
    CKS(mc_alloc(ctx, (void**)&ctx->k[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->TE[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->TN[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->invd[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->sqd[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->tE[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->tN[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->w64[0][a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->w64[1][a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->pd[a], fb));
    if (percell) CKS(mc_alloc(ctx, (void**)&ctx->diagc[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->F[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->p[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->pprev[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->r[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->z[a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->P[0][a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->P[1][a], fb));
    CKS(mc_alloc(ctx, (void**)&ctx->q[a], fb));
  }
  for (int a = 0; a < L; ++a)
    for (int b = a + 1; b < L; ++b) {
      CKS(mc_alloc(ctx, (void**)&ctx->qs[a][b], fb));
      ctx->qs[b][a] = ctx->qs[a][b];
    }
  const int maxb = mc_step_max_blocks_any(L, MC_STEP_THREADS, ctx->num_sms);
  if (maxb < 1) {
    cuda_err(ctx, "occupancy query", cudaGetLastError());
    return bail(MC_E_CUDA);
  }
  ctx->maxb = maxb;
  ctx->partials_len = (size_t)2 * MC_KMAX_ALLOC * maxb;
  CKS(mc_alloc(ctx, (void**)&ctx->partials, ctx->partials_len * sizeof(double)));
  CKS(mc_alloc(ctx, (void**)&ctx->bar, 96 * sizeof(unsigned)));
  CKS(mc_alloc(ctx, (void**)&ctx->dstatus, sizeof(int)));
  CKS(mc_alloc(ctx, (void**)&ctx->dsteps, sizeof(int)));
  CKS(mc_alloc(ctx, (void**)&ctx->diters, MCL * sizeof(long long)));
  CKS(mc_alloc(ctx, (void**)&ctx->dmaxit, MCL * sizeof(int)));
  CKS(mc_alloc(ctx, (void**)&ctx->drelres, MCL * sizeof(double)));
  CKS(mc_alloc(ctx, (void**)&ctx->dmass, sizeof(double)));
  CKS(mc_alloc(ctx, (void**)&ctx->dsweeps, sizeof(int)));
  // Coefficients: k (kept on the device for the NLMC build) into TE / TN.
  for (int a = 0; a < L; ++a) {
    CKS(h2d(ctx, ctx->k[a], k[a]));
    CKS(mc_launch_setup(ctx, a, ctx->k[a]));
  }
  for (int a = 0; a < L; ++a) CKS(mc_launch_diag(ctx, a));
  CKS(mc_launch_pairs(ctx));
  // TMA descriptors of the tiles the stencil phase stages in shared memory.
  for (int a = 0; a < L; ++a) {
    const int bx = mc_step_box_x(), by = mc_step_box_y();
    CKS(mc_encode_map(&ctx->maps.z[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, ctx->z[a], ctx->nx, ctx->ny,
                      ctx->pitch, bx, by));
    CKS(mc_encode_map(&ctx->maps.r[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, ctx->r[a], ctx->nx, ctx->ny,
                      ctx->pitch, bx, by));
    CKS(mc_encode_map(&ctx->maps.P[0][a], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, ctx->P[0][a], ctx->nx,
                      ctx->ny, ctx->pitch, bx, by));
    CKS(mc_encode_map(&ctx->maps.P[1][a], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, ctx->P[1][a], ctx->nx,
                      ctx->ny, ctx->pitch, bx, by));
    CKS(mc_encode_map(&ctx->maps.invd[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, ctx->invd[a], ctx->nx,
                      ctx->ny, ctx->pitch, bx, by));
    CKS(mc_encode_map(&ctx->maps.q[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, ctx->q[a], ctx->nx, ctx->ny,
                      ctx->pitch, bx, by));
    for (int k = 0; k < 2; ++k)
      CKS(mc_encode_map(&ctx->maps.w[k][a], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, ctx->w64[k][a], ctx->nx,
                        ctx->ny, ctx->pitch, bx, by));
  }
  CKS(cudaStreamSynchronize(ctx->stream));
#undef CKS
  *out = ctx;
  return MC_OK;
}

void mc_destroy(mc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
}

mc_status mc_set_opts(mc_ctx* ctx, const mc_opts* opts) {
  if (!ctx || !opts) return MC_E_ARG;
  std::string why;
  if (check_opts(opts, &why) != MC_OK) return set_err(ctx, MC_E_ARG, "opts: " + why);
  ctx->opts = *opts;
  return MC_OK;
}

mc_status mc_set_source(mc_ctx* ctx, int32_t alpha, const double* F) {
  if (!ctx) return MC_E_ARG;
  if (alpha < 0 || alpha >= ctx->L || !F) return set_err(ctx, MC_E_ARG, "bad alpha or F");
  for (long long i = 0; i < ctx->N; ++i)
    if (!isfinite(F[i])) return set_err(ctx, MC_E_ARG, "F must be finite");
  CK(cudaSetDevice(ctx->device));
  CK(h2d(ctx, ctx->F[alpha], F));
  CK(cudaStreamSynchronize(ctx->stream));
  return MC_OK;
}

mc_status mc_set_well(mc_ctx* ctx, int32_t alpha, const double* W, const double* pw) {
  if (!ctx) return MC_E_ARG;
  if (alpha < 0 || alpha >= ctx->L) return set_err(ctx, MC_E_ARG, "bad alpha");
  if (W) {
    if (!pw) return set_err(ctx, MC_E_ARG, "pw is NULL");
    for (long long i = 0; i < ctx->N; ++i) {
      if (!isfinite(W[i]) || W[i] < 0.0) return set_err(ctx, MC_E_ARG, "W must be finite and >= 0");
      if (!isfinite(pw[i])) return set_err(ctx, MC_E_ARG, "pw must be finite");
    }
  }
  CK(cudaSetDevice(ctx->device));
  const size_t fb = (size_t)ctx->Np * sizeof(double);
  if (W) {
    if (!ctx->W_buf[alpha]) {
      CK(mc_alloc(ctx, (void**)&ctx->W_buf[alpha], fb));
      CK(mc_alloc(ctx, (void**)&ctx->FW_buf[alpha], fb));
    }
    // the well makes diag(A0 - D) vary per cell
    if (!ctx->diagc[alpha]) CK(mc_alloc(ctx, (void**)&ctx->diagc[alpha], fb));
    ctx->W[alpha] = ctx->W_buf[alpha];
    ctx->FW[alpha] = ctx->FW_buf[alpha];
    CK(h2d(ctx, ctx->W[alpha], W));
    CK(h2d(ctx, ctx->FW[alpha], pw));
    CK(mc_launch_well(ctx, alpha));
  } else {
    // out of effect; the buffers are kept for a later mc_set_well
    ctx->W[alpha] = nullptr;
    ctx->FW[alpha] = nullptr;
  }
  CK(mc_launch_diag(ctx, alpha));
  CK(mc_launch_pairs(ctx));
  ctx->lo_kind = 0;  // FP32 / BF16 copies of diag and invd are stale
  ctx->tl_ready = 0;  // so is the two-level coarse operator
  ctx->tl_full_ready = 0;
  CK(cudaStreamSynchronize(ctx->stream));
  return MC_OK;
}

mc_status mc_set_state(mc_ctx* ctx, const double* const* p) {
  if (!ctx) return MC_E_ARG;
  if (!p) return set_err(ctx, MC_E_ARG, "p is NULL");
  for (int a = 0; a < ctx->L; ++a)
    if (!p[a]) return set_err(ctx, MC_E_ARG, "p[a] is NULL");
  CK(cudaSetDevice(ctx->device));
  for (int a = 0; a < ctx->L; ++a) CK(h2d(ctx, ctx->p[a], p[a]));
  CK(cudaStreamSynchronize(ctx->stream));
  return MC_OK;
}

mc_status mc_get_state(mc_ctx* ctx, double* const* p) {
  if (!ctx) return MC_E_ARG;
  if (!p) return set_err(ctx, MC_E_ARG, "p is NULL");
  for (int a = 0; a < ctx->L; ++a)
    if (!p[a]) return set_err(ctx, MC_E_ARG, "p[a] is NULL");
  CK(cudaSetDevice(ctx->device));
  for (int a = 0; a < ctx->L; ++a) CK(d2h(ctx, p[a], ctx->p[a]));
  CK(cudaStreamSynchronize(ctx->stream));
  return MC_OK;
}

mc_status mc_state_device(mc_ctx* ctx, int32_t alpha, double** dev) {
  if (!ctx || !dev || alpha < 0 || alpha >= ctx->L) return MC_E_ARG;
  *dev = ctx->p[alpha];
  return MC_OK;
}

// Two-level preconditioner set-up: the coarse operator of every continuum on
// the stencil tiles and its dense inverse (Gauss-Jordan on the device), once
// per context and again after the diagonal changes (mc_set_well); for the
// coupled scheme the Galerkin operator over all continua instead.
static mc_status tl_prepare_coupled(mc_ctx* ctx);

static mc_status tl_prepare(mc_ctx* ctx, bool coupled) {
  const int nc = mc_step_tiles(ctx->nx, ctx->ny);
  if (nc > MC_TWO_LEVEL_MAX_TILES)
    return set_err(ctx, MC_E_ARG, "two-level preconditioner: more than MC_TWO_LEVEL_MAX_TILES tiles");
  if (coupled && (long long)ctx->L * nc > MC_TWO_LEVEL_MAX_COUPLED)
    return set_err(ctx, MC_E_ARG, "two-level preconditioner: L x tiles above MC_TWO_LEVEL_MAX_COUPLED");
  if (ctx->tl_ready) return coupled ? tl_prepare_coupled(ctx) : MC_OK;
  if (!ctx->tl_work) {
    CK(mc_alloc(ctx, (void**)&ctx->tl_work, 2 * (size_t)nc * sizeof(double)));
    CK(mc_alloc(ctx, (void**)&ctx->tl_bar, 96 * sizeof(unsigned)));
    for (int a = 0; a < ctx->L; ++a) {
      CK(mc_alloc(ctx, (void**)&ctx->tl_Ainv[a], (size_t)nc * nc * sizeof(double)));
      CK(mc_alloc(ctx, (void**)&ctx->tl_g[a], (size_t)nc * sizeof(double)));
      CK(mc_alloc(ctx, (void**)&ctx->tl_c[a], (size_t)nc * sizeof(double)));
    }
    ctx->tl_nc = nc;
  }
  CK(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), ctx->stream));
  for (int a = 0; a < ctx->L; ++a) {
    CK(mc_launch_coarse_assemble(ctx, a, ctx->tl_Ainv[a]));
    CK(mc_gj_invert(ctx->tl_Ainv[a], nc, ctx->tl_work, ctx->tl_bar, ctx->dstatus, ctx->opts.spin_limit,
                    ctx->num_sms, ctx->stream));
  }
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st != MC_OK) return set_err(ctx, (mc_status)st, "two-level preconditioner set-up");
  ctx->tl_ready = 1;
  return coupled ? tl_prepare_coupled(ctx) : MC_OK;
}

static mc_status tl_prepare_coupled(mc_ctx* ctx) {
  if (ctx->tl_full_ready) return MC_OK;
  const long long n = (long long)ctx->L * ctx->tl_nc;
  if (!ctx->tl_Afull) {
    CK(mc_alloc(ctx, (void**)&ctx->tl_Afull, (size_t)(n * n) * sizeof(double)));
    CK(mc_alloc(ctx, (void**)&ctx->tl_work_full, 2 * (size_t)n * sizeof(double)));
  }
  CK(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), ctx->stream));
  CK(mc_launch_coarse_assemble_coupled(ctx, ctx->tl_Afull));
  CK(mc_gj_invert(ctx->tl_Afull, (int)n, ctx->tl_work_full, ctx->tl_bar, ctx->dstatus, ctx->opts.spin_limit,
                  ctx->num_sms, ctx->stream));
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st != MC_OK) return set_err(ctx, (mc_status)st, "two-level preconditioner set-up (coupled)");
  ctx->tl_full_ready = 1;
  return MC_OK;
}

static mc_status run_steps(mc_ctx* ctx, int scheme, int nsteps, mc_stats* stats) {
  if (stats) memset(stats, 0, sizeof(*stats));
  if (nsteps < 0) return set_err(ctx, MC_E_ARG, "nsteps < 0");
  const bool ir = ctx->opts.precision != MC_PREC_FP64;
  if (ir && scheme == MC_SCHEME_COUPLED)
    return set_err(ctx, MC_E_ARG, "the precision form applies to the decoupled schemes");
  const bool tl = ctx->opts.precond == MC_PRECOND_TWO_LEVEL;
  if (tl && ir)
    return set_err(ctx, MC_E_ARG, "the two-level preconditioner applies to the FP64 schemes");
  if (nsteps == 0) return MC_OK;
  CK(cudaSetDevice(ctx->device));
  if (tl) {
    const mc_status ps = tl_prepare(ctx, scheme == MC_SCHEME_COUPLED);
    if (ps != MC_OK) return ps;
  }
  StepParams sp;
  mc_fill_params(ctx, &sp, scheme, nsteps);
  if (tl) {
    sp.two_level = 1;
    sp.nc = ctx->tl_nc;
    for (int a = 0; a < ctx->L; ++a) {
      sp.Ainv[a] = ctx->tl_Ainv[a];
      sp.gsum[a] = ctx->tl_g[a];
      sp.ccor[a] = ctx->tl_c[a];
    }
    if (scheme == MC_SCHEME_COUPLED) {
      sp.tl_full = 1;
      sp.Ainv[0] = ctx->tl_Afull;
    }
  }
  CK(cudaMemsetAsync(ctx->bar, 0, 96 * sizeof(unsigned), ctx->stream));
  CK(cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->dsteps, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->diters, 0, MCL * sizeof(long long), ctx->stream));
  CK(cudaMemsetAsync(ctx->dmaxit, 0, MCL * sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(ctx->drelres, 0, MCL * sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->dmass, 0, sizeof(double), ctx->stream));
  CK(cudaMemsetAsync(ctx->dsweeps, 0, sizeof(int), ctx->stream));
  if (ir) {
    const int bf16 = ctx->opts.precision == MC_PREC_BF16T_IR ? 1 : 0;
    CK(mc_ir_prepare(ctx, bf16));
    int blocks = mc_ir_max_blocks(ctx->L, bf16 != 0, ctx->num_sms);
    if (blocks > ctx->maxb) blocks = ctx->maxb;
    if (ctx->opts.blocks > 0 && ctx->opts.blocks < blocks) blocks = ctx->opts.blocks;
    if (blocks < 1) return set_err(ctx, MC_E_CUDA, "no co-resident CTAs for the precision form");
    CK(mc_launch_ir(ctx, sp, bf16, blocks));
  } else {
    const int blocks = launch_blocks(ctx, sp);
    CK(mc_launch_steps(ctx, sp, blocks, launch_threads(ctx)));
  }
  int st = 0, done = 0;
  mc_stats s;
  memset(&s, 0, sizeof(s));
  CK(cudaMemcpyAsync(&st, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&done, ctx->dsteps, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(s.iters, ctx->diters, MCL * sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(s.max_iters, ctx->dmaxit, MCL * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(s.rel_residual, ctx->drelres, MCL * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&s.mass_defect, ctx->dmass, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&s.ir_sweeps, ctx->dsweeps, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  s.steps_done = done;
  s.status = st;
  if (st != MC_OK) {
    // Roll the state back to the start of the failed step.
    for (int a = 0; a < ctx->L; ++a)
      CK(cudaMemcpyAsync(ctx->p[a], ctx->pprev[a], ctx->Np * sizeof(double), cudaMemcpyDeviceToDevice,
                         ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (stats) *stats = s;
  if (st != MC_OK)
    return set_err(ctx, (mc_status)st, std::string("step ") + std::to_string(done + 1) + ": " +
                                           mc_status_string((mc_status)st));
  return MC_OK;
}

mc_status mc_step_decoupled(mc_ctx* ctx, int32_t scheme, int32_t nsteps, mc_stats* stats) {
  if (!ctx) return MC_E_ARG;
  if (scheme != MC_SCHEME_D && scheme != MC_SCHEME_L && scheme != MC_SCHEME_U)
    return set_err(ctx, MC_E_ARG, "scheme must be MC_SCHEME_D, _L or _U");
  return run_steps(ctx, scheme, nsteps, stats);
}

mc_status mc_step_coupled(mc_ctx* ctx, int32_t nsteps, mc_stats* stats) {
  if (!ctx) return MC_E_ARG;
  return run_steps(ctx, MC_SCHEME_COUPLED, nsteps, stats);
}

mc_status mc_get_coefficients(mc_ctx* ctx, int32_t alpha, double* TE, double* TN, double* diag) {
  if (!ctx || alpha < 0 || alpha >= ctx->L) return MC_E_ARG;
  CK(cudaSetDevice(ctx->device));
  if (TE) CK(d2h(ctx, TE, ctx->TE[alpha]));
  if (TN) CK(d2h(ctx, TN, ctx->TN[alpha]));
  if (diag) CK(d2h(ctx, diag, ctx->invd[alpha]));
  CK(cudaStreamSynchronize(ctx->stream));
  if (diag)
    for (long long i = 0; i < ctx->N; ++i) diag[i] = 1.0 / diag[i];
  return MC_OK;
}

mc_status mc_apply(mc_ctx* ctx, int32_t scheme, const double* const* x, double* const* y) {
  if (!ctx || !x || !y) return MC_E_ARG;
  if (scheme != MC_SCHEME_COUPLED && (scheme < MC_SCHEME_D || scheme > MC_SCHEME_U))
    return set_err(ctx, MC_E_ARG, "bad scheme");
  CK(cudaSetDevice(ctx->device));
  // r and q are step work space: free between steps.
  for (int a = 0; a < ctx->L; ++a) {
    if (!x[a] || !y[a]) return set_err(ctx, MC_E_ARG, "x[a] / y[a] NULL");
    CK(h2d(ctx, ctx->r[a], x[a]));
  }
  CK(mc_launch_apply(ctx, scheme, ctx->r, ctx->q));
  for (int a = 0; a < ctx->L; ++a) CK(d2h(ctx, y[a], ctx->q[a]));
  CK(cudaStreamSynchronize(ctx->stream));
  return MC_OK;
}

mc_status mc_rhs_decoupled(mc_ctx* ctx, double* const* b) {
  if (!ctx || !b) return MC_E_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(mc_launch_rhs(ctx, ctx->q));
  for (int a = 0; a < ctx->L; ++a) {
    if (!b[a]) return set_err(ctx, MC_E_ARG, "b[a] NULL");
    CK(d2h(ctx, b[a], ctx->q[a]));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return MC_OK;
}

mc_status mc_device_bytes(const mc_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return MC_E_ARG;
  *bytes = ctx->bytes;
  return MC_OK;
}

}  // extern "C"
