// Coefficient set-up (once per context) and the standalone operator /
// right-hand-side kernels used to inspect a context. Fields are pitched:
// cell (i, j) at j*pitch + i, padding columns zero and never written.
//
// Section 3.1, Eq. app-md: T_ij = k_face |E_ij| / d_ij. Cells are squares, so
// |E| = d = h and T = k_face; the face value is the harmonic mean of the two
// cell permeabilities (0 when both vanish). Boundary faces carry no
// transmissibility (zero-flux condition, Eq. mm-bc). Exchange between
// co-located continua: q_ab,i = sigma_ab,i |cell| = sigma_ab,i h^2.
// Diagonal of M_a/tau + D_a + sum_b Q_ab (Section 3.3, D-scheme A0 block):
//   d_i = c_a h^2 / tau + sum_b q_ab,i + sum over the four faces of T,
// its inverse (Jacobi), its square root and the scaled face values
// T_ij / sqrt(d_i d_j) of the unit-diagonal operator the FP64 PCG iterates on.

#include "mc_internal.h"

namespace {

__global__ void faces_kernel(int nx, int ny, int pitch, const double* __restrict__ k,
                             double* __restrict__ TE, double* __restrict__ TN) {
  const long long Np = (long long)ny * pitch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Np;
       i += (long long)gridDim.x * blockDim.x) {
    const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
    if (gx >= nx) continue;
    const double kc = k[i];
    double te = 0.0, tn = 0.0;
    if (gx + 1 < nx) {
      const double kn = k[i + 1];
      const double s = kc + kn;
      te = s > 0.0 ? 2.0 * kc * kn / s : 0.0;
    }
    if (gy + 1 < ny) {
      const double kn = k[i + pitch];
      const double s = kc + kn;
      tn = s > 0.0 ? 2.0 * kc * kn / s : 0.0;
    }
    TE[i] = te;
    TN[i] = tn;
  }
}

__global__ void scale_kernel(long long N, double* __restrict__ x, double s) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    x[i] *= s;
}

struct DiagArgs {
  int nx, ny, pitch, L, a;
  double mtau;
  double qconst[MCL];
  const double* qcell[MCL];
  const double* TE;
  const double* TN;
  const double* W;  // well index per cell, or nullptr
  double* diagc;  // may be nullptr (constant case)
  double* invd;
  double* sqd;    // sqrt of the diagonal, or nullptr
};

__global__ void diag_kernel(DiagArgs g) {
  const long long Np = (long long)g.ny * g.pitch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Np;
       i += (long long)gridDim.x * blockDim.x) {
    const int gy = (int)(i / g.pitch), gx = (int)(i - (long long)gy * g.pitch);
    if (gx >= g.nx) continue;
    double dc = g.mtau;
    for (int b = 0; b < g.L; ++b) {
      if (b == g.a) continue;
      dc += g.qcell[b] ? g.qcell[b][i] : g.qconst[b];
    }
    if (g.W) dc += g.W[i];
    double t = g.TE[i] + g.TN[i];
    if (gx > 0) t += g.TE[i - 1];
    if (gy > 0) t += g.TN[i - g.pitch];
    if (g.diagc) g.diagc[i] = dc;
    g.invd[i] = 1.0 / (dc + t);
    if (g.sqd) g.sqd[i] = sqrt(dc + t);
  }
}

// Symmetrically scaled face transmissibilities of the Jacobi-scaled operator
// D^-1/2 A D^-1/2 (unit diagonal): t_ij = T_ij / (sqrt(d_i) sqrt(d_j)).
__global__ void scaled_faces_kernel(int nx, int ny, int pitch, const double* __restrict__ TE,
                                    const double* __restrict__ TN, const double* __restrict__ sqd,
                                    double* __restrict__ tE, double* __restrict__ tN) {
  const long long Np = (long long)ny * pitch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Np;
       i += (long long)gridDim.x * blockDim.x) {
    const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
    if (gx >= nx) continue;
    const double sc = sqd[i];
    tE[i] = gx + 1 < nx ? TE[i] / (sc * sqd[i + 1]) : 0.0;
    tN[i] = gy + 1 < ny ? TN[i] / (sc * sqd[i + pitch]) : 0.0;
  }
}

// Scaled exchange of a pair of co-located continua: q_ab,i / sqrt(d_a,i d_b,i).
__global__ void pair_scale_kernel(int nx, int ny, int pitch, const double* __restrict__ qcell,
                                  double qconst, const double* __restrict__ sa,
                                  const double* __restrict__ sb, double* __restrict__ qs) {
  const long long Np = (long long)ny * pitch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Np;
       i += (long long)gridDim.x * blockDim.x) {
    const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
    if (gx >= nx) continue;
    const double q = qcell ? qcell[i] : qconst;
    qs[i] = q / (sa[i] * sb[i]);
  }
}

struct ApplyArgs {
  int nx, ny, pitch, L;
  bool coupled;
  double mtau[MCL];
  double qconst[MCL][MCL];
  const double* qcell[MCL][MCL];
  const double* TE[MCL];
  const double* TN[MCL];
  const double* x[MCL];
  double* y[MCL];
  const double* F[MCL];
  const double* W[MCL];   // wells, or nullptr
  const double* FW[MCL];
  bool rhs;  // y_a = mtau x_a + F_a (+ W_a pw_a) + sum_b q_ab x_b instead of the operator
};

__device__ __forceinline__ double q_of(const ApplyArgs& g, int a, int b, long long i) {
  return g.qcell[a][b] ? g.qcell[a][b][i] : g.qconst[a][b];
}

__global__ void apply_kernel(ApplyArgs g) {
  const long long Np = (long long)g.ny * g.pitch;
  const int nx = g.nx, pitch = g.pitch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Np;
       i += (long long)gridDim.x * blockDim.x) {
    const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
    if (gx >= nx) continue;
    for (int a = 0; a < g.L; ++a) {
      const double xc = g.x[a][i];
      double v;
      if (g.rhs) {
        v = g.mtau[a] * xc + g.F[a][i];
        if (g.FW[a]) v += g.FW[a][i];
        for (int b = 0; b < g.L; ++b)
          if (b != a) v += q_of(g, a, b, i) * g.x[b][i];
      } else {
        v = g.mtau[a] * xc;
        if (g.W[a]) v += g.W[a][i] * xc;
        if (gx + 1 < nx) v += g.TE[a][i] * (xc - g.x[a][i + 1]);
        if (gx > 0) v += g.TE[a][i - 1] * (xc - g.x[a][i - 1]);
        if (gy + 1 < g.ny) v += g.TN[a][i] * (xc - g.x[a][i + pitch]);
        if (gy > 0) v += g.TN[a][i - pitch] * (xc - g.x[a][i - pitch]);
        for (int b = 0; b < g.L; ++b) {
          if (b == a) continue;
          const double qv = q_of(g, a, b, i);
          v += qv * xc;
          if (g.coupled) v -= qv * g.x[b][i];
        }
      }
      g.y[a][i] = v;
    }
  }
}

int grid_for(long long N) {
  long long b = (N + 255) / 256;
  if (b > 4096) b = 4096;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t mc_launch_setup(mc_ctx* ctx, int a, const double* k_dev) {
  const long long N = ctx->Np;
  const int blocks = grid_for(N);
  faces_kernel<<<blocks, 256, 0, ctx->stream>>>(ctx->nx, ctx->ny, ctx->pitch, k_dev, ctx->TE[a],
                                                ctx->TN[a]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // Per-cell exchange arrays hold sigma on upload; scale them to q = sigma h^2
  // once, when the lower-indexed continuum of the pair is set up.
  for (int b = a + 1; b < ctx->L; ++b) {
    if (ctx->qcell[a][b]) {
      scale_kernel<<<blocks, 256, 0, ctx->stream>>>(N, ctx->qcell[a][b], ctx->h * ctx->h);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t mc_launch_diag(mc_ctx* ctx, int a) {
  return mc_launch_diag_into(ctx, a, ctx->W[a], ctx->diagc[a], ctx->invd[a], ctx->sqd[a], ctx->tE[a],
                             ctx->tN[a]);
}

cudaError_t mc_launch_diag_into(const mc_ctx* ctx, int a, const double* W, double* diagc, double* invd,
                                double* sqd, double* tE, double* tN) {
  DiagArgs g{};
  g.nx = ctx->nx;
  g.ny = ctx->ny;
  g.pitch = ctx->pitch;
  g.L = ctx->L;
  g.a = a;
  g.mtau = ctx->c[a] * ctx->h * ctx->h / ctx->tau;
  for (int b = 0; b < ctx->L; ++b) {
    g.qconst[b] = ctx->sigma[a][b] * ctx->h * ctx->h;
    g.qcell[b] = ctx->qcell[a][b];
  }
  g.TE = ctx->TE[a];
  g.TN = ctx->TN[a];
  g.W = W;
  g.diagc = diagc;
  g.invd = invd;
  g.sqd = sqd;
  diag_kernel<<<grid_for(ctx->Np), 256, 0, ctx->stream>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !sqd) return e;
  scaled_faces_kernel<<<grid_for(ctx->Np), 256, 0, ctx->stream>>>(
      ctx->nx, ctx->ny, ctx->pitch, ctx->TE[a], ctx->TN[a], sqd, tE, tN);
  return cudaGetLastError();
}

cudaError_t mc_launch_pairs(mc_ctx* ctx) { return mc_launch_pairs_into(ctx, ctx->sqd, ctx->qs); }

cudaError_t mc_launch_pairs_into(const mc_ctx* ctx, double* const* sqd, double* const (*qs)[MCL]) {
  for (int a = 0; a < ctx->L; ++a)
    for (int b = a + 1; b < ctx->L; ++b) {
      if (!qs[a][b] || !sqd[a] || !sqd[b]) continue;
      pair_scale_kernel<<<grid_for(ctx->Np), 256, 0, ctx->stream>>>(
          ctx->nx, ctx->ny, ctx->pitch, ctx->qcell[a][b], ctx->sigma[a][b] * ctx->h * ctx->h,
          sqd[a], sqd[b], qs[a][b]);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

namespace {

__global__ void well_kernel(long long Np, const double* __restrict__ W, double* __restrict__ FW) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Np;
       i += (long long)gridDim.x * blockDim.x)
    FW[i] = W[i] * FW[i];
}

}  // namespace

cudaError_t mc_launch_well(mc_ctx* ctx, int a) {
  well_kernel<<<grid_for(ctx->Np), 256, 0, ctx->stream>>>(ctx->Np, ctx->W[a], ctx->FW[a]);
  return cudaGetLastError();
}

static void fill_apply(const mc_ctx* ctx, ApplyArgs* g) {
  g->nx = ctx->nx;
  g->ny = ctx->ny;
  g->pitch = ctx->pitch;
  g->L = ctx->L;
  for (int a = 0; a < ctx->L; ++a) {
    g->mtau[a] = ctx->c[a] * ctx->h * ctx->h / ctx->tau;
    g->TE[a] = ctx->TE[a];
    g->TN[a] = ctx->TN[a];
    g->F[a] = ctx->F[a];
    g->W[a] = ctx->W[a];
    g->FW[a] = ctx->FW[a];
    for (int b = 0; b < ctx->L; ++b) {
      g->qconst[a][b] = ctx->sigma[a][b] * ctx->h * ctx->h;
      g->qcell[a][b] = ctx->qcell[a][b];
    }
  }
}

cudaError_t mc_launch_apply(mc_ctx* ctx, int scheme, double* const* x, double* const* y) {
  ApplyArgs g{};
  fill_apply(ctx, &g);
  g.coupled = scheme == MC_SCHEME_COUPLED;
  g.rhs = false;
  for (int a = 0; a < ctx->L; ++a) {
    g.x[a] = x[a];
    g.y[a] = y[a];
  }
  apply_kernel<<<grid_for(ctx->Np), 256, 0, ctx->stream>>>(g);
  return cudaGetLastError();
}

cudaError_t mc_launch_rhs(mc_ctx* ctx, double* const* b) {
  ApplyArgs g{};
  fill_apply(ctx, &g);
  g.rhs = true;
  for (int a = 0; a < ctx->L; ++a) {
    g.x[a] = ctx->p[a];
    g.y[a] = b[a];
  }
  apply_kernel<<<grid_for(ctx->Np), 256, 0, ctx->stream>>>(g);
  return cudaGetLastError();
}

cudaError_t mc_launch_single_setup(int nx, int ny, int pitch, double h, double c, double tau,
                                   const double* k, double* TE, double* TN, double* invd,
                                   cudaStream_t stream) {
  const long long Np = (long long)ny * pitch;
  faces_kernel<<<grid_for(Np), 256, 0, stream>>>(nx, ny, pitch, k, TE, TN);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  DiagArgs g{};
  g.nx = nx;
  g.ny = ny;
  g.pitch = pitch;
  g.L = 1;
  g.a = 0;
  g.mtau = c * h * h / tau;
  g.TE = TE;
  g.TN = TN;
  g.diagc = nullptr;
  g.invd = invd;
  diag_kernel<<<grid_for(Np), 256, 0, stream>>>(g);
  return cudaGetLastError();
}
