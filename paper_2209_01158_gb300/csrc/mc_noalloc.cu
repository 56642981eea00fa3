// mc_step_single_noalloc: a variant of the persistent time-stepping kernel's
// entry point for callers that must not allocate device memory.
//
// Every buffer the solver needs beyond the caller's inputs and outputs -- the
// pitched copies of k, F and p, the transmissibilities, the Jacobi inverse,
// the PCG vectors, the per-CTA partial sums, the grid-barrier words and the
// run statistics -- lives in ONE file-scope device array of fixed size. The
// array belongs to the loaded module, so every GPU that loads this library
// holds it (about 6 MB) until the process exits.
//
// In host code the array's name is only a host-side stand-in for the device
// symbol. Its device address is looked up once per device with
// cudaGetSymbolAddress (that device current) and that address is what the
// kernels receive.

#include <math.h>
#include <string.h>

#include <mutex>

#include "mc_internal.h"

namespace {

constexpr long long kMaxCells = 65536;   // ny * pitch, pitch = nx rounded up to 16
constexpr int kFields = 11;              // k/r, TE, TN, invd, F, p, pprev, P0, P1, q, z
constexpr int kMaxBlocks = 1024;
constexpr long long kPartials = 2LL * 4 * MCL * kMaxBlocks;
constexpr long long kCtrl = 256;         // barrier words, status, statistics
constexpr long long kDoubles = kFields * kMaxCells + kPartials + kCtrl;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kDoubles];

std::mutex g_lock;
double* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" mc_status mc_step_single_noalloc(int32_t nx, int32_t ny, const double* k, double c,
                                            double tau, const double* F, double* p,
                                            int32_t nsteps, double rtol, int32_t max_iter,
                                            void* stream, mc_stats* stats) {
  if (stats) memset(stats, 0, sizeof(*stats));
  if (nx < 1 || ny < 1) return MC_E_ARG;
  const int pitch = mc_pitch_for(nx);
  const long long Np = (long long)ny * pitch;
  if (Np > kMaxCells) return MC_E_ARG;  // beyond the fixed scratch array
  if (!k || !F || !p) return MC_E_ARG;
  if (!(c > 0.0) || !isfinite(c) || !(tau > 0.0) || !isfinite(tau)) return MC_E_ARG;
  if (!(rtol > 0.0) || !(rtol < 1.0) || max_iter < 1 || nsteps < 0) return MC_E_ARG;
  if (nsteps == 0) return MC_OK;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, num_sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MC_E_CUDA;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MC_E_CUDA;
  double* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return MC_E_CUDA;

  // Carve the array: kFields pitched fields, then partials, then control.
  double* fld[kFields];
  for (int f = 0; f < kFields; ++f) fld[f] = base + f * kMaxCells;
  double* kk = fld[0];  // holds k during set-up, then serves as r
  double *TE = fld[1], *TN = fld[2], *invd = fld[3], *Fp = fld[4], *pp = fld[5], *pprev = fld[6];
  double *P0 = fld[7], *P1 = fld[8], *q = fld[9], *zb = fld[10];
  double* partials = base + kFields * kMaxCells;
  double* ctrl = partials + kPartials;
  unsigned* bar = reinterpret_cast<unsigned*>(ctrl);               // 96 words
  int* dstatus = reinterpret_cast<int*>(ctrl + 48);
  int* dsteps = reinterpret_cast<int*>(ctrl + 49);
  long long* diters = reinterpret_cast<long long*>(ctrl + 50);     // [4]
  int* dmaxit = reinterpret_cast<int*>(ctrl + 54);                 // [4]
  double* drelres = ctrl + 56;                                     // [4]
  double* dmass = ctrl + 60;

  const size_t row = (size_t)nx * sizeof(double), prow = (size_t)pitch * sizeof(double);
#define NA_CK(x)                                  \
  do {                                            \
    if ((x) != cudaSuccess) return MC_E_CUDA;     \
  } while (0)
  // The array keeps the previous call's contents: zero everything this call
  // reads before writing (padding columns, barrier words, statistics).
  NA_CK(cudaMemsetAsync(base, 0, (size_t)kDoubles * sizeof(double), st));
  NA_CK(cudaMemcpy2DAsync(kk, prow, k, row, row, ny, cudaMemcpyDeviceToDevice, st));
  NA_CK(cudaMemcpy2DAsync(Fp, prow, F, row, row, ny, cudaMemcpyDeviceToDevice, st));
  NA_CK(cudaMemcpy2DAsync(pp, prow, p, row, row, ny, cudaMemcpyDeviceToDevice, st));
  const double h = 1.0 / nx;
  NA_CK(mc_launch_single_setup(nx, ny, pitch, h, c, tau, kk, TE, TN, invd, st));

  TmaMaps maps;
  memset(&maps, 0, sizeof(maps));
  const int bx = mc_step_box_x(), by = mc_step_box_y();
  NA_CK(mc_encode_map(&maps.z[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, zb, nx, ny, pitch, bx, by));
  NA_CK(mc_encode_map(&maps.P[0][0], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, P0, nx, ny, pitch, bx, by));
  NA_CK(mc_encode_map(&maps.P[1][0], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, P1, nx, ny, pitch, bx, by));
  NA_CK(mc_encode_map(&maps.invd[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, invd, nx, ny, pitch, bx, by));

  StepParams sp;
  memset(&sp, 0, sizeof(sp));
  sp.nx = nx;
  sp.ny = ny;
  sp.L = 1;
  sp.pitch = pitch;
  sp.N = (long long)nx * ny;
  sp.Np = Np;
  sp.scheme = MC_SCHEME_D;
  sp.nsteps = nsteps;
  sp.max_iter = max_iter;
  sp.rtol = rtol;
  sp.tau = tau;
  sp.mass[0] = c * h * h;
  sp.mtau[0] = c * h * h / tau;
  sp.diagc_const[0] = sp.mtau[0];
  sp.TE[0] = TE;
  sp.TN[0] = TN;
  sp.invd[0] = invd;
  sp.F[0] = Fp;
  sp.p[0] = pp;
  sp.pprev[0] = pprev;
  sp.r[0] = kk;
  sp.z[0] = zb;
  sp.P[0][0] = P0;
  sp.P[1][0] = P1;
  sp.q[0] = q;
  sp.partials = partials;
  sp.bar_count = bar;
  sp.bar_gen = bar + 32;
  sp.status = dstatus;
  sp.steps_done = dsteps;
  sp.iters = diters;
  sp.max_iters = dmaxit;
  sp.relres = drelres;
  sp.mass_defect = dmass;
  sp.spin_limit = 2000000;
  int blocks = mc_step_max_blocks(1, MC_STEP_THREADS, num_sms);
  if (blocks < 1) return MC_E_CUDA;
  if (blocks > kMaxBlocks) blocks = kMaxBlocks;
  NA_CK(mc_launch_steps_raw(sp, maps, blocks, MC_STEP_THREADS, st));

  double ctl[16];
  NA_CK(cudaMemcpyAsync(ctl, ctrl + 48, sizeof(ctl), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  int status = 0, done = 0;
  memcpy(&status, &ctl[0], sizeof(int));
  memcpy(&done, &ctl[1], sizeof(int));
  // On failure the caller's p receives the state at the start of the failed step.
  const double* src = status == MC_OK ? pp : pprev;
  NA_CK(cudaMemcpy2DAsync(p, row, src, prow, row, ny, cudaMemcpyDeviceToDevice, st));
  NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
  if (stats) {
    stats->steps_done = done;
    stats->status = status;
    memcpy(&stats->iters[0], &ctl[2], sizeof(long long));
    memcpy(&stats->max_iters[0], &ctl[6], sizeof(int));
    stats->rel_residual[0] = ctl[8];
    stats->mass_defect = ctl[12];
  }
  return static_cast<mc_status>(status);
}
