// Nonlocal multicontinuum (NLMC) coarse model on the GPU (Section 4).
//
// Build (Section 4.1):
//   * For every coarse block K_i (bx x by fine cells) and continuum beta, the
//     basis function psi^{i,beta} on the oversampled region K_i^+ (K_i grown
//     by `layers` coarse layers, clipped to the domain) minimises the energy
//     of the coupled fine operator D + Q restricted to K_i^+ (zero Dirichlet
//     data on the part of the region boundary inside the domain, through a
//     ghost value at h/2: T = 2 k) subject to Eq. eq:basis's constraints
//     mean_{K_j^alpha}(psi_alpha) = delta_ij delta_alpha,beta for every coarse
//     block K_j of the region and every alpha, K_j^alpha = Omega_alpha ∩ K_j:
//     a continuum given a support mask (an embedded fracture continuum: its
//     fracture cells) is averaged over its own cells only, and a block
//     without such cells has no coarse unknown of that continuum (no basis
//     function, zero rows and columns of A_bar, state 0).
//     Solver: projected preconditioned CG in the null space of the
//     constraints. psi = psi0 + w with psi0 the indicator of K_i in continuum
//     beta; the Jacobi-preconditioned residual is projected by subtracting,
//     on every coarse block and continuum, its invd-weighted mean (which is
//     exactly the M^{-1}-orthogonal projection for block-mean constraints),
//     and the residual itself is re-projected every iteration so that it
//     cannot drift out of the constraint-compatible space. One CTA per
//     (block, beta), all reductions inside the CTA.
//   * V = A psi for the global steady operator A = D + Q (zero flux on the
//     domain boundary), on the region plus a one-cell ring.
//   * A_bar = R A R^T: A_bar[(i,alpha),(j,beta)] = sum psi^{i,alpha} . V^{j,beta}
//     over the overlap, one CTA per pair of blocks that can interact.
//   * Optional conservative form: every diagonal entry of A_bar is set to
//     minus the sum of the other entries of its row, so that A_bar 1 = 0 as
//     for the exact (globally oversampled) basis; the truncated local basis
//     breaks this, and with very permeable fractures the defect outweighs
//     the coarse mass term.
//   * M_bar = diag(c_alpha |K_i^alpha|), F_bar = block sums of the fine
//     sources, wells W_bar = sums of W over K_i^alpha with right-hand side the
//     sums of W p_w (the coarse finite-volume forms the paper gives for
//     piecewise-constant data).
// Coarse stepping (Sections 4.2-4.3): coupled (Eq. is-nlmc) or the D-, L-,
// U-schemes with A0_bar from the diagonal / lower / upper blocks of A_bar.
// The coarse systems are small and dense: their inverses are formed once by
// Gauss-Jordan elimination (SPD, no pivoting) and every solve is a GEMV plus
// one residual-correction sweep.

#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "mc_internal.h"
#include "mc_sync.cuh"

struct mc_nlmc {
  mc_ctx* ctx = nullptr;
  int ncx = 0, ncy = 0, layers = 0, bx = 0, by = 0, Nc = 0, L = 0;
  int RX = 0, RY = 0;        // largest region extent (fine cells)
  long long rsz = 0;         // L * RX * RY
  long long vsz = 0;         // L * (RX + 2) * (RY + 2)
  int nbr = 0;               // block-distance range of interacting pairs
  double tau = 0.0;
  double basis_rtol = 1e-12;
  int basis_max_iter = 50000;
  double* psi = nullptr;     // [Nc][L beta][L gamma][RY][RX]
  double* V = nullptr;       // [Nc][L beta][L gamma][RY+2][RX+2]
  double* work = nullptr;    // per CTA slot: r, p, q, invd ([4][rsz])
  int nslots = 0;
  double* Abar = nullptr;    // (L Nc)^2, row-major
  double* mbar = nullptr;    // L Nc
  double* fbar = nullptr;    // L Nc
  double* wbar = nullptr;    // L Nc: coarse well index (sum of W over K_i^alpha)
  double* wpbar = nullptr;   // L Nc: sum of W p_w over K_i^alpha
  int* nsup = nullptr;       // L Nc: cells of K_i^alpha (0: no coarse unknown)
  unsigned char* sup = nullptr;  // L pitched masks of Omega_alpha (continua given one)
  int flags = 0;
  double* Gd = nullptr;      // L blocks of Nc^2: inverses of M_bar_a/tau + A_bar_aa
  double* Gc = nullptr;      // (L Nc)^2: inverse of M_bar/tau + A_bar
  double* gjrow = nullptr;   // Gauss-Jordan pivot row / column buffers (2 * L Nc)
  double* pbar = nullptr;    // L Nc
  double* pprev = nullptr;
  double* rhs = nullptr;
  double* xt = nullptr;
  double* res = nullptr;
  unsigned* bar = nullptr;   // [0..1] counter, [64] abort
  int* dstatus = nullptr;
  int* dsteps = nullptr;
  long long* dits = nullptr; // [0] total basis iterations, [1] max, [2] non-converged count
  std::vector<void*> allocs;
  int64_t bytes = 0;
  std::string err;
};

namespace {

constexpr int BT = 1024;  // basis-solve threads (32 warps)

struct Region {
  int x0, y0, lnx, lny, nbx, nby, centre;
};

__host__ __device__ inline Region region_of(int I, int J, int ncx, int ncy, int layers, int bx,
                                            int by) {
  const int I0 = I - layers < 0 ? 0 : I - layers;
  const int I1 = I + layers + 1 > ncx ? ncx : I + layers + 1;
  const int J0 = J - layers < 0 ? 0 : J - layers;
  const int J1 = J + layers + 1 > ncy ? ncy : J + layers + 1;
  Region r;
  r.x0 = I0 * bx;
  r.y0 = J0 * by;
  r.lnx = (I1 - I0) * bx;
  r.lny = (J1 - J0) * by;
  r.nbx = I1 - I0;
  r.nby = J1 - J0;
  r.centre = (J - J0) * r.nbx + (I - I0);
  return r;
}

struct FineRef {
  int nx, ny, pitch, L;
  const double* TE[MCL];
  const double* TN[MCL];
  const double* k[MCL];
  double qconst[MCL][MCL];
  const double* qcell[MCL][MCL];
  const unsigned char* sup[MCL];   // pitched mask of Omega_a, or nullptr (every cell)
};

// Cell gi (pitched index) of continuum a belongs to Omega_a.
__device__ __forceinline__ bool in_sup(const FineRef& f, int a, long long gi) {
  return f.sup[a] == nullptr || f.sup[a][gi] != 0;
}

__device__ __forceinline__ double fq(const FineRef& f, int a, int b, long long gi) {
  return f.qcell[a][b] ? __ldg(f.qcell[a][b] + gi) : f.qconst[a][b];
}

struct BasisArgs {
  FineRef f;
  int ncx, ncy, layers, bx, by, RX, RY;
  long long rsz;
  double* psi;
  double* work;
  double rtol;
  int max_iter;
  long long* dits;
  const int* nsup;   // [L][Nc] cells of K_j^alpha
};

// A_loc x at local cell (g, ly, lx) of region R (Dirichlet ghosts inside the
// domain, zero flux on the domain boundary, exchange between continua).
__device__ __forceinline__ double apply_loc(const BasisArgs& A, const Region& R, const double* x,
                                            int g, int ly, int lx) {
  const FineRef& f = A.f;
  const int gx = R.x0 + lx, gy = R.y0 + ly;
  const long long gi = (long long)gy * f.pitch + gx;
  const long long li = (long long)g * A.RX * A.RY + (long long)ly * A.RX + lx;
  const double xc = x[li];
  double v = 0.0;
  if (lx + 1 < R.lnx) v += __ldg(f.TE[g] + gi) * (xc - x[li + 1]);
  else if (gx + 1 < f.nx) v += 2.0 * __ldg(f.k[g] + gi) * xc;
  if (lx > 0) v += __ldg(f.TE[g] + gi - 1) * (xc - x[li - 1]);
  else if (gx > 0) v += 2.0 * __ldg(f.k[g] + gi) * xc;
  if (ly + 1 < R.lny) v += __ldg(f.TN[g] + gi) * (xc - x[li + A.RX]);
  else if (gy + 1 < f.ny) v += 2.0 * __ldg(f.k[g] + gi) * xc;
  if (ly > 0) v += __ldg(f.TN[g] + gi - f.pitch) * (xc - x[li - A.RX]);
  else if (gy > 0) v += 2.0 * __ldg(f.k[g] + gi) * xc;
  for (int d = 0; d < f.L; ++d) {
    if (d == g) continue;
    v += fq(f, g, d, gi) * (xc - x[li + (long long)(d - g) * A.RX * A.RY]);
  }
  return v;
}

// Diagonal of A_loc at the local cell.
__device__ __forceinline__ double diag_loc(const BasisArgs& A, const Region& R, int g, int ly, int lx) {
  const FineRef& f = A.f;
  const int gx = R.x0 + lx, gy = R.y0 + ly;
  const long long gi = (long long)gy * f.pitch + gx;
  const double kc = __ldg(f.k[g] + gi);
  double v = 0.0;
  if (lx + 1 < R.lnx) v += __ldg(f.TE[g] + gi); else if (gx + 1 < f.nx) v += 2.0 * kc;
  if (lx > 0) v += __ldg(f.TE[g] + gi - 1); else if (gx > 0) v += 2.0 * kc;
  if (ly + 1 < R.lny) v += __ldg(f.TN[g] + gi); else if (gy + 1 < f.ny) v += 2.0 * kc;
  if (ly > 0) v += __ldg(f.TN[g] + gi - f.pitch); else if (gy > 0) v += 2.0 * kc;
  for (int d = 0; d < f.L; ++d)
    if (d != g) v += fq(f, g, d, gi);
  return v;
}

// Cells of the region are visited by "segments" (one row of one coarse block
// of one continuum); warp w takes segments w, w+32, ..., lanes stride the
// segment. Per-block sums therefore land in per-warp slots and are added in a
// fixed order: deterministic.
template <typename Fn>
__device__ __forceinline__ void for_cells(const BasisArgs& A, const Region& R, Fn fn) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int L = A.f.L;
  const int nseg = L * R.lny * R.nbx;
  for (int s = warp; s < nseg; s += BT / 32) {
    const int cb = s % R.nbx;
    const int rowg = s / R.nbx;
    const int ly = rowg % R.lny;
    const int g = rowg / R.lny;
    const int blk = g * (R.nbx * R.nby) + (ly / A.by) * R.nbx + cb;
    for (int c0 = 0; c0 < A.bx; c0 += 32) {  // same trip count on every lane
      const int c = c0 + lane;
      fn(g, ly, cb * A.bx + (c < A.bx ? c : 0), blk, c < A.bx);
    }
  }
}

// part[warp][block] -> totals[block] (fixed order); nblk <= 2 * MCL * 25.
constexpr int MAXBLK = MCL * 25;

__device__ __forceinline__ void block_totals(double* part, double* tot, int nblk) {
  __syncthreads();
  for (int b = threadIdx.x; b < nblk; b += BT) {
    double s = 0.0;
    for (int w = 0; w < BT / 32; ++w) s += part[w * MAXBLK + b];
    tot[b] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(BT, 1) nlmc_basis_kernel(const BasisArgs A) {
  __shared__ double part[(BT / 32) * MAXBLK];
  __shared__ double sinv[MAXBLK];
  __shared__ double mean[MAXBLK];
  __shared__ double s_red[(BT / 32) * 2];
  __shared__ double s_res[2];
  const int L = A.f.L;
  const int Nc = A.ncx * A.ncy;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* r = A.work + (size_t)blockIdx.x * 4 * A.rsz;
  double* p = r + A.rsz;
  double* q = p + A.rsz;
  double* iv = q + A.rsz;
  const long long plane = (long long)A.RX * A.RY;
  auto idx = [&](int g, int ly, int lx) -> long long {
    return (long long)g * plane + (long long)ly * A.RX + lx;
  };
  auto clear_part = [&]() {
    for (int b = threadIdx.x; b < (BT / 32) * MAXBLK; b += BT) part[b] = 0.0;
    __syncthreads();
  };
  long long it_total = 0, it_max = 0, nonconv = 0;
  for (int task = blockIdx.x; task < Nc * L; task += gridDim.x) {
    const int i = task / L, beta = task - i * L;
    const int I = i % A.ncx, J = i / A.ncx;
    const Region R = region_of(I, J, A.ncx, A.ncy, A.layers, A.bx, A.by);
    if (A.nsup[beta * Nc + i] == 0) continue;  // K_i^beta empty: no coarse unknown (uniform)
    const int nb = R.nbx * R.nby;
    const int nblk = L * nb;
    const int cblk = beta * nb + R.centre;
    double* w = A.psi + ((size_t)i * L + beta) * A.rsz;
    auto sup_of = [&](int g, int ly, int lx) -> bool {
      return in_sup(A.f, g, (long long)(R.y0 + ly) * A.f.pitch + R.x0 + lx);
    };
    // w = p = psi0 (indicator of K_i^beta in continuum beta); invd and its
    // sums over every K_j^alpha (constrained cells only)
    clear_part();
    for_cells(A, R, [&](int g, int ly, int lx, int blk, bool ok) {
      double d = 0.0;
      if (ok) {
        const long long li = idx(g, ly, lx);
        const bool s_in = sup_of(g, ly, lx);
        const double v = (blk == cblk && s_in) ? 1.0 : 0.0;
        w[li] = v;
        p[li] = v;
        const double dv = 1.0 / diag_loc(A, R, g, ly, lx);
        iv[li] = dv;
        d = s_in ? dv : 0.0;
      }
      const double s = warp_sum_d(d);
      if (lane == 0) part[warp * MAXBLK + blk] += s;
    });
    block_totals(part, sinv, nblk);
    // r = -A psi0, then its invd-weighted block means
    clear_part();
    for_cells(A, R, [&](int g, int ly, int lx, int blk, bool ok) {
      double t = 0.0;
      if (ok) {
        const long long li = idx(g, ly, lx);
        const double rv = -apply_loc(A, R, p, g, ly, lx);
        r[li] = rv;
        t = sup_of(g, ly, lx) ? iv[li] * rv : 0.0;
      }
      const double s = warp_sum_d(t);
      if (lane == 0) part[warp * MAXBLK + blk] += s;
    });
    block_totals(part, mean, nblk);
    for (int b = threadIdx.x; b < nblk; b += BT) mean[b] = sinv[b] > 0.0 ? mean[b] / sinv[b] : 0.0;
    __syncthreads();
    double acc[1] = {0.0};
    for_cells(A, R, [&](int g, int ly, int lx, int blk, bool ok) {
      if (!ok) return;
      const long long li = idx(g, ly, lx);
      const double rv = r[li] - (sup_of(g, ly, lx) ? mean[blk] : 0.0);
      r[li] = rv;
      const double z = iv[li] * rv;
      p[li] = z;
      acc[0] += rv * z;
    });
    cta_sum<1>(acc, s_red, s_res);
    double rz = acc[0];
    const double rz0 = rz;
    const double tol2 = A.rtol * A.rtol;
    int it = 0;
    bool conv = !(rz > tol2 * rz0) || rz0 == 0.0;
    while (!conv && it < A.max_iter) {
      double pq[1] = {0.0};
      for_cells(A, R, [&](int g, int ly, int lx, int blk, bool ok) {
        if (!ok) return;
        const long long li = idx(g, ly, lx);
        const double qv = apply_loc(A, R, p, g, ly, lx);
        q[li] = qv;
        pq[0] += p[li] * qv;
      });
      cta_sum<1>(pq, s_red, s_res);
      if (!(pq[0] > 0.0)) break;
      const double al = rz / pq[0];
      clear_part();
      for_cells(A, R, [&](int g, int ly, int lx, int blk, bool ok) {
        double t = 0.0;
        if (ok) {
          const long long li = idx(g, ly, lx);
          w[li] += al * p[li];
          const double rv = r[li] - al * q[li];
          r[li] = rv;
          t = sup_of(g, ly, lx) ? iv[li] * rv : 0.0;
        }
        const double s = warp_sum_d(t);
        if (lane == 0) part[warp * MAXBLK + blk] += s;
      });
      block_totals(part, mean, nblk);
      for (int b = threadIdx.x; b < nblk; b += BT) mean[b] = sinv[b] > 0.0 ? mean[b] / sinv[b] : 0.0;
      __syncthreads();
      double rzn[1] = {0.0};
      for_cells(A, R, [&](int g, int ly, int lx, int blk, bool ok) {
        if (!ok) return;
        const long long li = idx(g, ly, lx);
        const double rv = r[li] - (sup_of(g, ly, lx) ? mean[blk] : 0.0);
        r[li] = rv;
        rzn[0] += rv * (iv[li] * rv);
      });
      cta_sum<1>(rzn, s_red, s_res);
      ++it;
      if (!(rzn[0] > tol2 * rz0)) { conv = true; break; }
      const double bt = rzn[0] / rz;
      rz = rzn[0];
      for_cells(A, R, [&](int g, int ly, int lx, int blk, bool ok) {
        if (!ok) return;
        const long long li = idx(g, ly, lx);
        p[li] = iv[li] * r[li] + bt * p[li];
      });
      __syncthreads();
    }
    it_total += it;
    if (it > it_max) it_max = it;
    if (!conv) ++nonconv;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(A.dits), (unsigned long long)it_total);
    atomicMax(reinterpret_cast<unsigned long long*>(A.dits + 1), (unsigned long long)it_max);
    atomicAdd(reinterpret_cast<unsigned long long*>(A.dits + 2), (unsigned long long)nonconv);
  }
}

// V^{i,beta} = A psi^{i,beta} on the region plus a one-cell ring.
__global__ void nlmc_apply_kernel(const BasisArgs A, double* V, long long vsz) {
  const int L = A.f.L;
  const int Nc = A.ncx * A.ncy;
  const FineRef& f = A.f;
  const int VX = A.RX + 2, VY = A.RY + 2;
  for (long long task = blockIdx.x; task < (long long)Nc * L; task += gridDim.x) {
    const int i = (int)(task / L), beta = (int)(task - (long long)i * L);
    const Region R = region_of(i % A.ncx, i / A.ncx, A.ncx, A.ncy, A.layers, A.bx, A.by);
    const double* ps = A.psi + ((size_t)i * L + beta) * A.rsz;
    double* v = V + ((size_t)i * L + beta) * vsz;
    const int ex = R.lnx + 2, ey = R.lny + 2;
    for (long long e = threadIdx.x; e < (long long)L * ex * ey; e += blockDim.x) {
      const int g = (int)(e / (ex * ey));
      const int rem = (int)(e - (long long)g * ex * ey);
      const int ly = rem / ex - 1, lx = rem % ex - 1;
      const int gx = R.x0 + lx, gy = R.y0 + ly;
      double out = 0.0;
      if (gx >= 0 && gx < f.nx && gy >= 0 && gy < f.ny) {
        auto val = [&](int gg, int yy, int xx) -> double {
          if (xx < 0 || xx >= R.lnx || yy < 0 || yy >= R.lny) return 0.0;
          return ps[(long long)gg * A.RX * A.RY + (long long)yy * A.RX + xx];
        };
        const long long gi = (long long)gy * f.pitch + gx;
        const double xc = val(g, ly, lx);
        if (gx + 1 < f.nx) out += __ldg(f.TE[g] + gi) * (xc - val(g, ly, lx + 1));
        if (gx > 0) out += __ldg(f.TE[g] + gi - 1) * (xc - val(g, ly, lx - 1));
        if (gy + 1 < f.ny) out += __ldg(f.TN[g] + gi) * (xc - val(g, ly + 1, lx));
        if (gy > 0) out += __ldg(f.TN[g] + gi - f.pitch) * (xc - val(g, ly - 1, lx));
        for (int d = 0; d < L; ++d)
          if (d != g) out += fq(f, g, d, gi) * (xc - val(d, ly, lx));
      }
      v[(long long)g * VX * VY + (long long)(ly + 1) * VX + (lx + 1)] = out;
    }
  }
}

// A_bar entries of one (i, j) block pair: sum over the overlap of
// psi^{i,alpha}_gamma * V^{j,beta}_gamma for all alpha, beta.
__global__ void nlmc_galerkin_kernel(const BasisArgs A, const double* V, long long vsz, int nbr,
                                     double* Abar) {
  __shared__ double s_red[(256 / 32) * MCL * MCL];
  __shared__ double s_res[MCL * MCL];
  const int L = A.f.L;
  const int Nc = A.ncx * A.ncy;
  const int span = 2 * nbr + 1;
  const long long npair = (long long)Nc * span * span;
  const int VX = A.RX + 2, VY = A.RY + 2;
  for (long long task = blockIdx.x; task < npair; task += gridDim.x) {
    const int i = (int)(task / (span * span));
    const int off = (int)(task - (long long)i * span * span);
    const int Ii = i % A.ncx, Ji = i / A.ncx;
    const int Ij = Ii + off % span - nbr, Jj = Ji + off / span - nbr;
    if (Ij < 0 || Ij >= A.ncx || Jj < 0 || Jj >= A.ncy) continue;  // uniform per CTA
    const int j = Jj * A.ncx + Ij;
    const Region Ri = region_of(Ii, Ji, A.ncx, A.ncy, A.layers, A.bx, A.by);
    const Region Rj = region_of(Ij, Jj, A.ncx, A.ncy, A.layers, A.bx, A.by);
    const int xs = max(Ri.x0, Rj.x0 - 1), xe = min(Ri.x0 + Ri.lnx, Rj.x0 + Rj.lnx + 1);
    const int ys = max(Ri.y0, Rj.y0 - 1), ye = min(Ri.y0 + Ri.lny, Rj.y0 + Rj.lny + 1);
    double acc[MCL * MCL];
#pragma unroll
    for (int k = 0; k < MCL * MCL; ++k) acc[k] = 0.0;
    if (xs < xe && ys < ye) {
      const int wx = xe - xs;
      const long long ncell = (long long)wx * (ye - ys);
      for (long long e = threadIdx.x; e < ncell; e += blockDim.x) {
        const int gy = ys + (int)(e / wx), gx = xs + (int)(e % wx);
        const int lxi = gx - Ri.x0, lyi = gy - Ri.y0;
        const int lxj = gx - Rj.x0 + 1, lyj = gy - Rj.y0 + 1;
        for (int g = 0; g < L; ++g) {
          double pv[MCL], vv[MCL];
          for (int a = 0; a < L; ++a)
            pv[a] = A.psi[((size_t)i * L + a) * A.rsz + (long long)g * A.RX * A.RY +
                          (long long)lyi * A.RX + lxi];
          for (int b = 0; b < L; ++b)
            vv[b] = V[((size_t)j * L + b) * vsz + (long long)g * VX * VY + (long long)lyj * VX + lxj];
          for (int a = 0; a < L; ++a)
            for (int b = 0; b < L; ++b) acc[a * MCL + b] += pv[a] * vv[b];
        }
      }
    }
    cta_sum<MCL * MCL>(acc, s_red, s_res);
    if (threadIdx.x == 0) {
      const long long n = (long long)L * Nc;
      for (int a = 0; a < L; ++a)
        for (int b = 0; b < L; ++b) Abar[((long long)a * Nc + i) * n + (long long)b * Nc + j] = acc[a * MCL + b];
    }
  }
}

// Cells of K_i^alpha for every block and continuum (one warp each).
__global__ void nlmc_support_count(FineRef f, int ncx, int ncy, int bx, int by, int* nsup) {
  const int Nc = ncx * ncy;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < f.L * Nc; t += nwarps) {
    const int a = t / Nc, i = t - a * Nc;
    const int I = i % ncx, J = i / ncx;
    int cnt = 0;
    for (int e = lane; e < bx * by; e += 32) {
      const long long gi = (long long)(J * by + e / bx) * f.pitch + I * bx + e % bx;
      cnt += in_sup(f, a, gi) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) nsup[t] = cnt;
  }
}

// Coarse mass c |K_i^alpha|, block sums of F, means of p over K_i^alpha, and
// the coarse well terms (sums of W and W p_w over K_i^alpha); 0 for the
// unknowns that do not exist.
__global__ void nlmc_coarse_vectors(FineRef f, const double* const* F, const double* const* p,
                                    const double* const* W, const double* const* FW, int ncx, int ncy,
                                    int bx, int by, double area, const double* c, const int* nsup,
                                    double* mbar, double* fbar, double* pbar, double* wbar,
                                    double* wpbar) {
  const int Nc = ncx * ncy;
  const int L = f.L;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < L * Nc; t += nwarps) {
    const int a = t / Nc, i = t - a * Nc;
    const int I = i % ncx, J = i / ncx;
    const int ns = nsup[t];
    double sf = 0.0, sp = 0.0, sw = 0.0, swp = 0.0;
    for (int e = lane; e < bx * by; e += 32) {
      const long long gi = (long long)(J * by + e / bx) * f.pitch + I * bx + e % bx;
      if (F) sf += F[a][gi];
      if (!in_sup(f, a, gi)) continue;
      if (p) sp += p[a][gi];
      if (W[a]) {
        sw += W[a][gi];
        swp += FW[a][gi];
      }
    }
    sf = warp_sum_d(sf);
    sp = warp_sum_d(sp);
    sw = warp_sum_d(sw);
    swp = warp_sum_d(swp);
    if (lane == 0) {
      if (mbar) mbar[t] = ns > 0 ? c[a] * ns * area : 0.0;
      if (fbar) fbar[t] = ns > 0 ? sf : 0.0;
      if (pbar) pbar[t] = ns > 0 ? sp / ns : 0.0;
      if (wbar) wbar[t] = ns > 0 ? sw : 0.0;
      if (wpbar) wpbar[t] = ns > 0 ? swp : 0.0;
    }
  }
}

// Conservative form: A_bar[r][r] -= sum of row r (one warp per row; a warp
// reads only its own row and writes only its diagonal).
__global__ void nlmc_conserve_kernel(double* Abar, long long n) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < n; r += nw) {
    double s = 0.0;
    for (long long c = lane; c < n; c += 32) s += Abar[r * n + c];
    s = warp_sum_d(s);
    if (lane == 0) Abar[r * n + r] -= s;
  }
}

struct GJArgs {
  GridBar bar;
  double* M;       // n x n, inverted in place
  double* row;     // n
  double* col;     // n
  int n;
};

// In-place Gauss-Jordan inversion of an SPD matrix (no pivoting needed).
__global__ void gj_invert_kernel(const GJArgs g) {
  const long long n = g.n;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  for (long long k = 0; k < n; ++k) {
    const double piv = __ldcg(g.M + k * n + k);
    for (long long j = gt; j < n; j += gs) {
      g.row[j] = __ldcg(g.M + k * n + j) / piv;
      g.col[j] = __ldcg(g.M + j * n + k);
    }
    if (!grid_barrier(g.bar)) return;
    for (long long e = gt; e < n * n; e += gs) {
      const long long i = e / n, j = e - i * n;
      double v;
      if (i == k && j == k) v = 1.0 / piv;
      else if (i == k) v = __ldcg(g.row + j);
      else if (j == k) v = -__ldcg(g.col + i) / piv;
      else v = __ldcg(g.M + e) - __ldcg(g.col + i) * __ldcg(g.row + j);
      g.M[e] = v;
    }
    if (!grid_barrier(g.bar)) return;
  }
}

struct CoarseArgs {
  GridBar bar;
  int L, Nc, scheme, nsteps;
  double tau;
  const double* Abar;
  const double* mbar;
  const double* fbar;
  const double* wbar;    // coarse well index (diagonal)
  const double* wpbar;   // coarse well right-hand side
  const double* Gd;
  const double* Gc;
  double* pbar;
  double* pprev;
  double* rhs;
  double* xt;
  double* res;
  int* steps_done;
};

// y[r] = sum_c M[r * ld + c] x[c] for rows r in [r0, r1), one warp per row.
__device__ __forceinline__ void gemv_rows(const double* M, long long ld, const double* x, int ncol,
                                          double* y, int r0, int r1, double scale, bool accumulate) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = r0 + warp; r < r1; r += nw) {
    double s = 0.0;
    for (int c = lane; c < ncol; c += 32) s += __ldcg(M + r * ld + c) * __ldcg(x + c);
    s = warp_sum_d(s);
    if (lane == 0) y[r] = accumulate ? y[r] + scale * s : scale * s;
  }
}

__global__ void nlmc_step_kernel(const CoarseArgs A) {
  const int L = A.L, Nc = A.Nc;
  const long long n = (long long)L * Nc;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  int done = 0;
  for (int step = 0; step < A.nsteps; ++step) {
    for (long long e = gt; e < n; e += gs) A.pprev[e] = __ldcg(A.pbar + e);
    if (!grid_barrier(A.bar)) return;
    if (A.scheme == MC_SCHEME_COUPLED) {
      for (long long e = gt; e < n; e += gs)
        A.rhs[e] = A.mbar[e] / A.tau * __ldcg(A.pprev + e) + A.fbar[e] + A.wpbar[e];
      if (!grid_barrier(A.bar)) return;
      gemv_rows(A.Gc, n, A.rhs, (int)n, A.xt, 0, (int)n, 1.0, false);
      if (!grid_barrier(A.bar)) return;
      // res = rhs - (M_bar/tau + A_bar) xt
      gemv_rows(A.Abar, n, A.xt, (int)n, A.res, 0, (int)n, 1.0, false);
      if (!grid_barrier(A.bar)) return;
      for (long long e = gt; e < n; e += gs)
        A.res[e] = __ldcg(A.rhs + e) - (A.mbar[e] / A.tau + A.wbar[e]) * __ldcg(A.xt + e) -
                   __ldcg(A.res + e);
      if (!grid_barrier(A.bar)) return;
      gemv_rows(A.Gc, n, A.res, (int)n, A.xt, 0, (int)n, 1.0, true);
      if (!grid_barrier(A.bar)) return;
      for (long long e = gt; e < n; e += gs) A.pbar[e] = __ldcg(A.xt + e);
      if (!grid_barrier(A.bar)) return;
    } else {
      const int groups = A.scheme == MC_SCHEME_D ? 1 : L;
      for (int gi = 0; gi < groups; ++gi) {
        const int a0 = A.scheme == MC_SCHEME_D ? 0 : (A.scheme == MC_SCHEME_L ? gi : L - 1 - gi);
        const int a1 = A.scheme == MC_SCHEME_D ? L : a0 + 1;
        const double* src = A.scheme == MC_SCHEME_D ? A.pprev : A.pbar;
        // rhs_a = M_a/tau p_a^{n-1} + F_a - sum_{b != a} A_ab src_b
        for (int a = a0; a < a1; ++a) {
          for (long long e = gt; e < Nc; e += gs) A.rhs[a * Nc + e] = 0.0;
        }
        if (!grid_barrier(A.bar)) return;
        for (int a = a0; a < a1; ++a)
          for (int b = 0; b < L; ++b) {
            if (b == a) continue;
            gemv_rows(A.Abar + (long long)b * Nc, n, src + (long long)b * Nc, Nc, A.rhs,
                      a * Nc, (a + 1) * Nc, -1.0, true);
            if (!grid_barrier(A.bar)) return;
          }
        for (int a = a0; a < a1; ++a)
          for (long long e = gt; e < Nc; e += gs) {
            const long long r = a * Nc + e;
            A.rhs[r] = __ldcg(A.rhs + r) + A.mbar[r] / A.tau * __ldcg(A.pprev + r) + A.fbar[r] +
                       A.wpbar[r];
          }
        if (!grid_barrier(A.bar)) return;
        for (int a = a0; a < a1; ++a) {
          const double* G = A.Gd + (long long)a * Nc * Nc;
          // xt_a = G_a rhs_a, one warp per row
          const int lane = threadIdx.x & 31;
          const long long warp = (gt) >> 5;
          const long long nw = gs >> 5;
          for (long long r = warp; r < Nc; r += nw) {
            double s = 0.0;
            for (int c = lane; c < Nc; c += 32) s += __ldcg(G + r * Nc + c) * __ldcg(A.rhs + a * Nc + c);
            s = warp_sum_d(s);
            if (lane == 0) A.xt[a * Nc + r] = s;
          }
        }
        if (!grid_barrier(A.bar)) return;
        // res_a = rhs_a - (M_a/tau + A_aa) xt_a, then xt_a += G_a res_a
        for (int a = a0; a < a1; ++a) {
          const int lane = threadIdx.x & 31;
          const long long warp = gt >> 5;
          const long long nw = gs >> 5;
          for (long long r = warp; r < Nc; r += nw) {
            const long long row = a * Nc + r;
            double s = 0.0;
            for (int c = lane; c < Nc; c += 32)
              s += __ldcg(A.Abar + row * n + a * Nc + c) * __ldcg(A.xt + a * Nc + c);
            s = warp_sum_d(s);
            if (lane == 0)
              A.res[row] = __ldcg(A.rhs + row) - (A.mbar[row] / A.tau + A.wbar[row]) * __ldcg(A.xt + row) - s;
          }
        }
        if (!grid_barrier(A.bar)) return;
        for (int a = a0; a < a1; ++a) {
          const double* G = A.Gd + (long long)a * Nc * Nc;
          const int lane = threadIdx.x & 31;
          const long long warp = gt >> 5;
          const long long nw = gs >> 5;
          for (long long r = warp; r < Nc; r += nw) {
            double s = 0.0;
            for (int c = lane; c < Nc; c += 32) s += __ldcg(G + r * Nc + c) * __ldcg(A.res + a * Nc + c);
            s = warp_sum_d(s);
            if (lane == 0) A.pbar[a * Nc + r] = __ldcg(A.xt + a * Nc + r) + s;
          }
        }
        if (!grid_barrier(A.bar)) return;
      }
    }
    ++done;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.steps_done = done;
}

mc_status nerr(mc_nlmc* m, mc_status s, const std::string& msg) {
  if (m) m->err = msg;
  if (m && m->ctx) m->ctx->err = msg;
  return s;
}

cudaError_t nalloc(mc_nlmc* m, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return e;
  m->allocs.push_back(*p);
  m->bytes += (int64_t)bytes;
  return cudaMemsetAsync(*p, 0, bytes, m->ctx->stream);
}

void nfree(mc_nlmc* m) {
  for (void* p : m->allocs) cudaFree(p);
  m->allocs.clear();
}

FineRef fine_ref(const mc_ctx* ctx, double* const* k) {
  FineRef f{};
  f.nx = ctx->nx;
  f.ny = ctx->ny;
  f.pitch = ctx->pitch;
  f.L = ctx->L;
  for (int a = 0; a < ctx->L; ++a) {
    f.TE[a] = ctx->TE[a];
    f.TN[a] = ctx->TN[a];
    f.k[a] = k[a];
    for (int b = 0; b < ctx->L; ++b) {
      f.qconst[a][b] = ctx->sigma[a][b] * ctx->h * ctx->h;
      f.qcell[a][b] = ctx->qcell[a][b];
    }
  }
  return f;
}

int coop_blocks(void* fn, int threads, int num_sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0) != cudaSuccess) return 0;
  return per * num_sms;
}

cudaError_t gj_invert(mc_nlmc* m, double* M, int n) {
  GJArgs g{};
  g.bar.count = reinterpret_cast<unsigned long long*>(m->bar);
  g.bar.abort_word = m->bar + 64;
  g.bar.status = m->dstatus;
  g.bar.spin_limit = m->ctx->opts.spin_limit;
  g.M = M;
  g.row = m->gjrow;
  g.col = m->gjrow + (long long)m->L * m->Nc;
  g.n = n;
  cudaError_t e = cudaMemsetAsync(m->bar, 0, 96 * sizeof(unsigned), m->ctx->stream);
  if (e != cudaSuccess) return e;
  const int blocks = coop_blocks((void*)gj_invert_kernel, 512, m->ctx->num_sms);
  if (blocks < 1) return cudaErrorInvalidConfiguration;
  void* args[] = {&g};
  return cudaLaunchCooperativeKernel((void*)gj_invert_kernel, dim3(blocks), dim3(512), args, 0,
                                     m->ctx->stream);
}

// M_bar/tau + W_bar + A_bar restricted to continuum a; a coarse unknown that
// does not exist (zero mass, zero row and column of A_bar) gets a unit
// diagonal, so that the inverse exists and maps its zero right-hand side to 0.
__global__ void copy_block_kernel(const double* Abar, long long n, int a, int Nc, const double* mbar,
                                  const double* wbar, double tau, double* G) {
  const long long tot = (long long)Nc * Nc;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / Nc, c = e - r * Nc;
    const long long ra = (long long)a * Nc + r;
    double v = Abar[ra * n + (long long)a * Nc + c];
    if (r == c) v += mbar[ra] > 0.0 ? mbar[ra] / tau + wbar[ra] : 1.0;
    G[e] = v;
  }
}

__global__ void copy_full_kernel(const double* Abar, long long n, const double* mbar,
                                 const double* wbar, double tau, double* G) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, c = e - r * n;
    G[e] = Abar[e] + (r == c ? (mbar[r] > 0.0 ? mbar[r] / tau + wbar[r] : 1.0) : 0.0);
  }
}

}  // namespace

cudaError_t mc_gj_invert(double* M, int n, double* work, unsigned* bar, int* status,
                         long long spin_limit, int num_sms, cudaStream_t stream) {
  GJArgs g{};
  g.bar.count = reinterpret_cast<unsigned long long*>(bar);
  g.bar.abort_word = bar + 64;
  g.bar.status = status;
  g.bar.spin_limit = spin_limit;
  g.M = M;
  g.row = work;
  g.col = work + n;
  g.n = n;
  cudaError_t e = cudaMemsetAsync(bar, 0, 96 * sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  const int blocks = coop_blocks((void*)gj_invert_kernel, 512, num_sms);
  if (blocks < 1) return cudaErrorInvalidConfiguration;
  void* args[] = {&g};
  return cudaLaunchCooperativeKernel((void*)gj_invert_kernel, dim3(blocks), dim3(512), args, 0, stream);
}

extern "C" {

mc_status mc_nlmc_build(mc_ctx* ctx, int32_t ncx, int32_t ncy, int32_t layers,
                        double basis_rtol, int32_t basis_max_iter, mc_nlmc** out) {
  return mc_nlmc_build_ex(ctx, ncx, ncy, layers, basis_rtol, basis_max_iter, nullptr, 0, out);
}

mc_status mc_nlmc_build_ex(mc_ctx* ctx, int32_t ncx, int32_t ncy, int32_t layers,
                           double basis_rtol, int32_t basis_max_iter,
                           const uint8_t* const* support, int32_t flags, mc_nlmc** out) {
  if (!ctx || !out) return MC_E_ARG;
  *out = nullptr;
  if (ncx < 1 || ncy < 1 || layers < 0) return MC_E_ARG;
  if (ctx->nx % ncx || ctx->ny % ncy) {
    ctx->err = "coarse grid must divide the fine grid";
    return MC_E_ARG;
  }
  if (!(basis_rtol > 0.0) || !(basis_rtol < 1.0) || basis_max_iter < 1) return MC_E_ARG;
  if (flags & ~MC_NLMC_CONSERVATIVE) {
    ctx->err = "unknown NLMC flags";
    return MC_E_ARG;
  }
  const int bx = ctx->nx / ncx, by = ctx->ny / ncy;
  const int span = 2 * layers + 1;
  if ((span < ncx ? span : ncx) * (span < ncy ? span : ncy) * ctx->L > MAXBLK) {
    ctx->err = "too many coarse blocks per oversampled region";
    return MC_E_ARG;
  }
  mc_nlmc* m = new (std::nothrow) mc_nlmc();
  if (!m) return MC_E_ALLOC;
  m->ctx = ctx;
  m->ncx = ncx;
  m->ncy = ncy;
  m->layers = layers;
  m->bx = bx;
  m->by = by;
  m->Nc = ncx * ncy;
  m->L = ctx->L;
  m->RX = (span < ncx ? span : ncx) * bx;
  m->RY = (span < ncy ? span : ncy) * by;
  m->rsz = (long long)m->L * m->RX * m->RY;
  m->vsz = (long long)m->L * (m->RX + 2) * (m->RY + 2);
  m->nbr = 2 * layers + 1;
  m->tau = ctx->tau;
  m->basis_rtol = basis_rtol;
  m->basis_max_iter = basis_max_iter;
  m->flags = flags;
  cudaStream_t st = ctx->stream;
  const int L = m->L, Nc = m->Nc;
  const long long n = (long long)L * Nc;
  auto bail = [&](mc_status s, const std::string& msg) {
    nerr(m, s, msg);
    nfree(m);
    delete m;
    return s;
  };
  cudaError_t e;
#define NK(x)                                                                    \
  do {                                                                           \
    e = (x);                                                                     \
    if (e != cudaSuccess)                                                        \
      return bail(e == cudaErrorMemoryAllocation ? MC_E_ALLOC : MC_E_CUDA,       \
                  std::string(#x) + ": " + cudaGetErrorString(e));               \
  } while (0)
  NK(cudaSetDevice(ctx->device));
  // the context's permeability copies serve the Dirichlet ghost terms
  double* kd[MCL] = {};
  for (int a = 0; a < L; ++a) kd[a] = ctx->k[a];
  int bblocks = coop_blocks((void*)nlmc_basis_kernel, BT, ctx->num_sms);
  if (bblocks < 1) bblocks = ctx->num_sms;
  m->nslots = (int)(bblocks < n ? bblocks : n);
  NK(nalloc(m, (void**)&m->psi, (size_t)Nc * L * m->rsz * sizeof(double)));
  NK(nalloc(m, (void**)&m->work, (size_t)m->nslots * 4 * m->rsz * sizeof(double)));
  NK(nalloc(m, (void**)&m->V, (size_t)Nc * L * m->vsz * sizeof(double)));
  NK(nalloc(m, (void**)&m->Abar, (size_t)n * n * sizeof(double)));
  NK(nalloc(m, (void**)&m->Gd, (size_t)L * Nc * Nc * sizeof(double)));
  NK(nalloc(m, (void**)&m->Gc, (size_t)n * n * sizeof(double)));
  NK(nalloc(m, (void**)&m->gjrow, (size_t)2 * n * sizeof(double)));
  NK(nalloc(m, (void**)&m->mbar, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->fbar, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->wbar, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->wpbar, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->nsup, (size_t)n * sizeof(int)));
  NK(nalloc(m, (void**)&m->pbar, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->pprev, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->rhs, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->xt, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->res, (size_t)n * sizeof(double)));
  NK(nalloc(m, (void**)&m->bar, 96 * sizeof(unsigned)));
  NK(nalloc(m, (void**)&m->dstatus, sizeof(int)));
  NK(nalloc(m, (void**)&m->dsteps, sizeof(int)));
  NK(nalloc(m, (void**)&m->dits, 4 * sizeof(long long)));
  double* cdev = nullptr;
  NK(nalloc(m, (void**)&cdev, MCL * sizeof(double)));
  NK(cudaMemcpyAsync(cdev, ctx->c, MCL * sizeof(double), cudaMemcpyHostToDevice, st));
  const double** Fptr = nullptr;
  const double** Pptr = nullptr;
  const double** Wptr = nullptr;
  const double** FWptr = nullptr;
  NK(nalloc(m, (void**)&Fptr, MCL * sizeof(double*)));
  NK(nalloc(m, (void**)&Pptr, MCL * sizeof(double*)));
  NK(nalloc(m, (void**)&Wptr, MCL * sizeof(double*)));
  NK(nalloc(m, (void**)&FWptr, MCL * sizeof(double*)));
  NK(cudaMemcpyAsync(Fptr, ctx->F, MCL * sizeof(double*), cudaMemcpyHostToDevice, st));
  NK(cudaMemcpyAsync(Pptr, ctx->p, MCL * sizeof(double*), cudaMemcpyHostToDevice, st));
  NK(cudaMemcpyAsync(Wptr, ctx->W, MCL * sizeof(double*), cudaMemcpyHostToDevice, st));
  NK(cudaMemcpyAsync(FWptr, ctx->FW, MCL * sizeof(double*), cudaMemcpyHostToDevice, st));
  // Omega_alpha masks, pitched like the fine fields (only continua given one)
  const unsigned char* supd[MCL] = {};
  int nmask = 0;
  for (int a = 0; a < L; ++a) nmask += (support && support[a]) ? 1 : 0;
  if (nmask > 0) {
    NK(nalloc(m, (void**)&m->sup, (size_t)nmask * ctx->Np));
    int slot = 0;
    for (int a = 0; a < L; ++a) {
      if (!support[a]) continue;
      unsigned char* dst = m->sup + (size_t)slot++ * ctx->Np;
      NK(cudaMemcpy2DAsync(dst, ctx->pitch, support[a], ctx->nx, ctx->nx, ctx->ny,
                           cudaMemcpyHostToDevice, st));
      supd[a] = dst;
    }
  }

  BasisArgs A{};
  A.f = fine_ref(ctx, kd);
  for (int a = 0; a < L; ++a) A.f.sup[a] = supd[a];
  A.nsup = m->nsup;
  nlmc_support_count<<<256, 256, 0, st>>>(A.f, ncx, ncy, bx, by, m->nsup);
  NK(cudaGetLastError());
  A.ncx = ncx;
  A.ncy = ncy;
  A.layers = layers;
  A.bx = bx;
  A.by = by;
  A.RX = m->RX;
  A.RY = m->RY;
  A.rsz = m->rsz;
  A.psi = m->psi;
  A.work = m->work;
  A.rtol = basis_rtol;
  A.max_iter = basis_max_iter;
  A.dits = m->dits;
  nlmc_basis_kernel<<<m->nslots, BT, 0, st>>>(A);
  NK(cudaGetLastError());
  const int g2 = (int)(n < 4096 ? n : 4096);
  nlmc_apply_kernel<<<g2, 256, 0, st>>>(A, m->V, m->vsz);
  NK(cudaGetLastError());
  const long long npair = (long long)Nc * (2 * m->nbr + 1) * (2 * m->nbr + 1);
  nlmc_galerkin_kernel<<<(int)(npair < 65536 ? npair : 65536), 256, 0, st>>>(A, m->V, m->vsz, m->nbr,
                                                                               m->Abar);
  NK(cudaGetLastError());
  if (flags & MC_NLMC_CONSERVATIVE) {
    nlmc_conserve_kernel<<<(int)((n + 7) / 8), 256, 0, st>>>(m->Abar, n);
    NK(cudaGetLastError());
  }
  nlmc_coarse_vectors<<<256, 256, 0, st>>>(A.f, Fptr, Pptr, Wptr, FWptr, ncx, ncy, bx, by,
                                           ctx->h * ctx->h, cdev, m->nsup, m->mbar, m->fbar,
                                           m->pbar, m->wbar, m->wpbar);
  NK(cudaGetLastError());
  for (int a = 0; a < L; ++a) {
    copy_block_kernel<<<1024, 256, 0, st>>>(m->Abar, n, a, Nc, m->mbar, m->wbar, m->tau,
                                            m->Gd + (long long)a * Nc * Nc);
    NK(cudaGetLastError());
    NK(gj_invert(m, m->Gd + (long long)a * Nc * Nc, Nc));
  }
  copy_full_kernel<<<1024, 256, 0, st>>>(m->Abar, n, m->mbar, m->wbar, m->tau, m->Gc);
  NK(cudaGetLastError());
  NK(gj_invert(m, m->Gc, (int)n));
  long long its[4] = {0, 0, 0, 0};
  int stt = 0;
  NK(cudaMemcpyAsync(its, m->dits, sizeof(its), cudaMemcpyDeviceToHost, st));
  NK(cudaMemcpyAsync(&stt, m->dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
  NK(cudaStreamSynchronize(st));
#undef NK
  if (stt != 0) return bail((mc_status)stt, "coarse inverse: device barrier timeout");
  if (its[2] != 0) return bail(MC_E_NOCONV, "basis solves did not converge within basis_max_iter");
  *out = m;
  return MC_OK;
}

void mc_nlmc_destroy(mc_nlmc* m) {
  if (!m) return;
  cudaSetDevice(m->ctx->device);
  cudaStreamSynchronize(m->ctx->stream);
  nfree(m);
  delete m;
}

mc_status mc_nlmc_info(const mc_nlmc* m, int64_t* info) {
  if (!m || !info) return MC_E_ARG;
  long long its[4] = {0, 0, 0, 0};
  if (cudaMemcpy(its, m->dits, sizeof(its), cudaMemcpyDeviceToHost) != cudaSuccess) return MC_E_CUDA;
  info[0] = m->Nc;
  info[1] = m->L;
  info[2] = its[0];
  info[3] = its[1];
  info[4] = m->bytes;
  return MC_OK;
}

mc_status mc_nlmc_active(mc_nlmc* m, uint8_t* active) {
  if (!m || !active) return MC_E_ARG;
  const size_t n = (size_t)m->L * m->Nc;
  std::vector<int> ns(n);
  if (cudaMemcpyAsync(ns.data(), m->nsup, n * sizeof(int), cudaMemcpyDeviceToHost, m->ctx->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(m->ctx->stream) != cudaSuccess)
    return MC_E_CUDA;
  for (size_t i = 0; i < n; ++i) active[i] = ns[i] > 0 ? 1 : 0;
  return MC_OK;
}

mc_status mc_nlmc_set_state(mc_nlmc* m, const double* pbar) {
  if (!m || !pbar) return MC_E_ARG;
  if (cudaMemcpyAsync(m->pbar, pbar, (size_t)m->L * m->Nc * sizeof(double), cudaMemcpyHostToDevice,
                      m->ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->ctx->stream) != cudaSuccess)
    return MC_E_CUDA;
  return MC_OK;
}

mc_status mc_nlmc_get_state(mc_nlmc* m, double* pbar) {
  if (!m || !pbar) return MC_E_ARG;
  if (cudaMemcpyAsync(pbar, m->pbar, (size_t)m->L * m->Nc * sizeof(double), cudaMemcpyDeviceToHost,
                      m->ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->ctx->stream) != cudaSuccess)
    return MC_E_CUDA;
  return MC_OK;
}

mc_status mc_nlmc_get_operator(mc_nlmc* m, double* Abar, double* mbar, double* fbar) {
  if (!m) return MC_E_ARG;
  const size_t n = (size_t)m->L * m->Nc;
  cudaStream_t st = m->ctx->stream;
  if (Abar && cudaMemcpyAsync(Abar, m->Abar, n * n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MC_E_CUDA;
  if (mbar && cudaMemcpyAsync(mbar, m->mbar, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MC_E_CUDA;
  if (fbar && cudaMemcpyAsync(fbar, m->fbar, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MC_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MC_E_CUDA;
  return MC_OK;
}

mc_status mc_nlmc_get_basis(mc_nlmc* m, int32_t block, int32_t beta, double* psi) {
  if (!m || !psi || block < 0 || block >= m->Nc || beta < 0 || beta >= m->L) return MC_E_ARG;
  const mc_ctx* ctx = m->ctx;
  const Region R = region_of(block % m->ncx, block / m->ncx, m->ncx, m->ncy, m->layers, m->bx, m->by);
  memset(psi, 0, (size_t)m->L * ctx->nx * ctx->ny * sizeof(double));
  cudaStream_t st = m->ctx->stream;
  for (int g = 0; g < m->L; ++g) {
    const double* src = m->psi + ((size_t)block * m->L + beta) * m->rsz + (size_t)g * m->RX * m->RY;
    double* dst = psi + (size_t)g * ctx->nx * ctx->ny + (size_t)R.y0 * ctx->nx + R.x0;
    if (cudaMemcpy2DAsync(dst, ctx->nx * sizeof(double), src, m->RX * sizeof(double),
                          R.lnx * sizeof(double), R.lny, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return MC_E_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return MC_E_CUDA;
  return MC_OK;
}

mc_status mc_nlmc_step(mc_nlmc* m, int32_t scheme, int32_t nsteps, mc_stats* stats) {
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!m) return MC_E_ARG;
  if (scheme != MC_SCHEME_COUPLED && scheme != MC_SCHEME_D && scheme != MC_SCHEME_L &&
      scheme != MC_SCHEME_U)
    return nerr(m, MC_E_ARG, "bad scheme");
  if (nsteps < 0) return MC_E_ARG;
  if (nsteps == 0) return MC_OK;
  mc_ctx* ctx = m->ctx;
  cudaStream_t st = ctx->stream;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MC_E_CUDA;
  CoarseArgs A{};
  A.bar.count = reinterpret_cast<unsigned long long*>(m->bar);
  A.bar.abort_word = m->bar + 64;
  A.bar.status = m->dstatus;
  A.bar.spin_limit = ctx->opts.spin_limit;
  A.L = m->L;
  A.Nc = m->Nc;
  A.scheme = scheme;
  A.nsteps = nsteps;
  A.tau = m->tau;
  A.Abar = m->Abar;
  A.mbar = m->mbar;
  A.fbar = m->fbar;
  A.wbar = m->wbar;
  A.wpbar = m->wpbar;
  A.Gd = m->Gd;
  A.Gc = m->Gc;
  A.pbar = m->pbar;
  A.pprev = m->pprev;
  A.rhs = m->rhs;
  A.xt = m->xt;
  A.res = m->res;
  A.steps_done = m->dsteps;
  if (cudaMemsetAsync(m->bar, 0, 96 * sizeof(unsigned), st) != cudaSuccess) return MC_E_CUDA;
  if (cudaMemsetAsync(m->dstatus, 0, sizeof(int), st) != cudaSuccess) return MC_E_CUDA;
  const int blocks = coop_blocks((void*)nlmc_step_kernel, 512, ctx->num_sms);
  if (blocks < 1) return MC_E_CUDA;
  void* args[] = {&A};
  if (cudaLaunchCooperativeKernel((void*)nlmc_step_kernel, dim3(blocks), dim3(512), args, 0, st) !=
      cudaSuccess)
    return nerr(m, MC_E_CUDA, "coarse step launch failed");
  int stt = 0, done = 0;
  if (cudaMemcpyAsync(&stt, m->dstatus, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&done, m->dsteps, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MC_E_CUDA;
  if (stats) {
    stats->steps_done = done;
    stats->status = stt;
  }
  if (stt != 0) return nerr(m, (mc_status)stt, "coarse step: device barrier timeout");
  return MC_OK;
}

}  // extern "C"
