// Persistent time-stepping kernel: right-hand side assembly, per-continuum
// (or coupled) Jacobi-preconditioned CG on the 5-point TPFA stencil, and the
// mass-balance check, for nsteps time steps in ONE cooperative launch.
//
// Section 3.2 (Eq. ct-mc, coupled backward Euler) and Section 3.3 (Eq. si-mc,
// D-, L-, U-schemes). Per step and continuum a the decoupled schemes solve
//   (M_a/tau + D_a + sum_b Q_ab) p_a^n = M_a/tau p_a^{n-1} + F_a
//                                        + sum_b Q_ab p_b^{n-1 or n},
// the coupled scheme (M/tau + D + Q) p^n = M/tau p^{n-1} + F.
//
// Layout: every field is ny rows of `pitch` doubles (pitch = nx rounded up to
// 16, padding zero), cell (i, j) at j*pitch + i. TE holds the east-face
// transmissibility (0 on the last column), TN the north face (0 on the last
// row). The PCG warm-starts from p^{n-1} and updates p in place.
//
// PCG iteration = two phases separated by grid barriers:
//   A (stencil): per 64 x 16 tile, TMA brings the halo boxes of z = M r and
//     P_old into shared memory (a ring of up to 8 stages: the next tiles'
//     boxes load while this one computes); P_new = z + beta*P_old on the
//     66 x 18 halo region, then q = A P_new on the tile and <P_new, q>.
//   B (pointwise, vectorised): x += alpha P_new, r -= alpha q, z = invd r
//     (stored for the next phase A), <r, r>, <r, z>.
// Decoupled Jacobi solves run the same two phases in scaled variables
// (pcg_solve_scaled): with S = diag(sqrt(d)), Jacobi PCG on A is plain CG on
// S^-1 A S^-1, whose diagonal is 1 and whose face entries are
// T_ij / sqrt(d_i d_j), so the stencil costs 4 FMA and 1 add per cell and
// z = r needs no multiply, no invd read and no z store.
// Cross-CTA data written inside the launch is read through L2 (ld.cg or TMA,
// after a proxy fence); read-only coefficients use the read-only path.
// Reductions are deterministic: warp butterflies, then fixed-order sums over
// warps and over CTAs.

#include <math.h>

#include "mc_internal.h"
#include "mc_sync.cuh"
#include "mc_tma.h"

namespace {

constexpr int TX = 64;          // stencil tile width (cells along x)
constexpr int TY = 16;          // stencil tile height
constexpr int HOFF = 2;         // box starts 2 doubles (16 B) left of the tile
constexpr int BX = TX + 2 * HOFF;   // 68: box width (doubles), 544 B rows
constexpr int BY = TY + 2;          // 18: box height
constexpr int ABOX = 1232;      // box slot in doubles (9856 B, 128-B multiple)
constexpr uint32_t BOX_BYTES = BX * BY * 8;
constexpr int PX = TX + 2;      // 66: P_new halo region width
constexpr int PN = PX * BY;     // 1188 cells
constexpr int NT = MC_STEP_THREADS;  // threads per CTA
constexpr int RPT = NT / TX;    // 4: tile rows covered by one pass of the CTA
constexpr int CPT = TY / RPT;   // 4: own cells per thread
constexpr int KMAX = 4 * MCL;   // partial-sum quantities per slot

// TMA pipeline depth per CTA. Two 256-thread CTAs share an SM (each with its
// own CTA barriers, so one computes while the other waits), so each CTA keeps
// its ring within half of the SM's shared memory; the two rings together keep
// enough boxes in flight to cover the DRAM latency (Little's law: ~64 KB per
// SM). Measured on the three-continuum D-scheme at 1024^2: 500 ms per step
// against 547 ms with one 512-thread CTA per SM and an 8-deep ring.
__host__ __device__ constexpr int nstage(int L, bool coupled) {
  return !coupled ? 4 : (L <= 1 ? 4 : (L == 2 ? 2 : 1));
}

__device__ __forceinline__ double ldc(const double* p) { return __ldcg(p); }
__device__ __forceinline__ double ldr(const double* p) { return __ldg(p); }

__device__ __forceinline__ double warp_sum(double v) { return warp_sum_d(v); }

__device__ __forceinline__ GridBar bar_of(const StepParams& sp) {
  GridBar g;
  g.count = reinterpret_cast<unsigned long long*>(sp.bar_count);
  g.abort_word = sp.bar_gen + 32;
  g.status = sp.status;
  g.spin_limit = sp.spin_limit;
  return g;
}

__device__ __forceinline__ void raise_abort(const StepParams& sp, int code) {
  grid_raise_abort(bar_of(sp), code);
}

// Grid-wide barrier (mc_sync.cuh); afterwards thread 0, which issues the TMA
// loads, orders the other CTAs' generic stores before its async-proxy reads.
__device__ bool grid_sync(const StepParams& sp) {
  const bool ok = grid_barrier(bar_of(sp));
  if (threadIdx.x == 0) fence_proxy_async();
  return ok;
}

// CTA reduction through the (idle) TMA box area of shared memory.
template <int NQ>
__device__ __forceinline__ void block_store(const double (&v)[NQ], unsigned qmask, double* stage,
                                            double* partials, int slot) {
  cta_reduce_store<NQ, NT, KMAX, double>(v, qmask, stage, partials, slot);
}

// Sum over b = lane, lane + 32, ... < nb of src[b], in that order. The first
// PMAX loads are issued together (one L2 round trip for up to 32 * PMAX CTAs)
// before the adds; the order of the adds, and so the result, is that of the
// plain loop.
constexpr int PMAX = 12;
__device__ __forceinline__ double lane_partial_sum(const double* src, int lane, int nb) {
  double v[PMAX];
#pragma unroll
  for (int j = 0; j < PMAX; ++j) v[j] = lane + 32 * j < nb ? ldc(src + lane + 32 * j) : 0.0;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PMAX; ++j)
    if (lane + 32 * j < nb) s += v[j];
  for (int b = lane + 32 * PMAX; b < nb; b += 32) s += ldc(src + b);
  return s;
}

// Grid totals of NQ quantities into s_res (shared), readable by all threads.
// Quantities whose bit is clear in qmask (stored as 0 by block_store) are not
// summed: their totals are 0.
template <int NQ>
__device__ void grid_totals(const double* partials, int slot, double* s_res, unsigned qmask = ~0u) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int k = warp; k < NQ; k += nw) {
    const double s =
        (qmask >> k) & 1u ? warp_sum(lane_partial_sum(partials + ((size_t)slot * KMAX + k) * nb, lane, nb)) : 0.0;
    if (lane == 0) s_res[k] = s;
  }
  __syncthreads();
}

template <int NQ>
__device__ void grid_sum(const double* partials, int slot, double* s_res, double (&out)[NQ]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int k = warp; k < NQ; k += nw) {
    const double s = warp_sum(lane_partial_sum(partials + ((size_t)slot * KMAX + k) * nb, lane, nb));
    if (lane == 0) s_res[k] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NQ; ++k) out[k] = s_res[k];
  __syncthreads();
}

__device__ __forceinline__ double qab(const StepParams& sp, int a, int b, long long i) {
  const double* c = sp.qcell[a][b];
  return c ? ldr(c + i) : sp.qconst[a][b];
}

__device__ __forceinline__ double diagc(const StepParams& sp, int a, long long i) {
  const double* d = sp.diagc[a];
  return d ? ldr(d + i) : sp.diagc_const[a];
}

// D_a x at cell (gx, gy): sum over faces of T (x_i - x_neighbour).
__device__ __forceinline__ double stencil_flux(const StepParams& sp, int a, const double* x,
                                               int gx, int gy, long long i, double xc) {
  const int pitch = sp.pitch;
  double s = 0.0;
  if (gx + 1 < sp.nx) s += ldr(sp.TE[a] + i) * (xc - ldc(x + i + 1));
  if (gx > 0) s += ldr(sp.TE[a] + i - 1) * (xc - ldc(x + i - 1));
  if (gy + 1 < sp.ny) s += ldr(sp.TN[a] + i) * (xc - ldc(x + i + pitch));
  if (gy > 0) s += ldr(sp.TN[a] + i - pitch) * (xc - ldc(x + i - pitch));
  return s;
}

// Per-continuum PCG scalars in shared memory, updated by thread 0 only: the
// FP64 divisions and convergence tests run once per CTA, not per thread.
struct Scal64 {
  double bb[MCL], rr[MCL], rz[MCL], beta[MCL], alpha[MCL];
  double rzl[MCL];  // two-level: (r, D^-1 r) before the coarse term is added
  int iters[MCL];
  unsigned active;
  int flag;  // 1 breakdown
};

struct Smem {
  Scal64* sc;
  double* box;      // [NST stages][NARR][ABOX]
  double* pn;       // [NL][PN]
  double* red;      // [NT/32][KMAX]
  double* res;      // [KMAX]
  uint64_t* bar;    // [NST]
  double* cn;       // [9] coarse corrections of a tile and its neighbours
};

// ---------------------------------------------------------------------------
// Two-level preconditioner (an option beside Jacobi):
//   M^-1 r = D^-1 r + P A_c^-1 P^T r,  A_c = P^T A P,
// where P holds the indicator vectors of the 64 x 16 stencil tiles and A is
// the continuum's own system matrix M_a/tau + D_a + sum_b Q_ab (+ W_a). A_c is
// the Galerkin coarse operator (5-point on the tile grid); its dense inverse
// is formed once at set-up. Both terms are symmetric positive (semi)definite,
// so M^-1 is SPD and the CG recurrences are unchanged. The coarse space holds
// the constant vector, the near-null mode of the zero-flux systems.

// P^T r: the sum of r over every tile of the continua in `act`, tiles handed
// out to the CTAs as in the stencil phase (deterministic sums).
template <int L>
__device__ void tile_rsums(const StepParams& sp, unsigned act, Smem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int alist[L];
  int nact = 0;
#pragma unroll
  for (int a = 0; a < L; ++a) if (act & (1u << a)) alist[nact++] = a;
  const int tiles = sp.tiles_x * sp.tiles_y;
  const int lx = tid % TX, ly = tid / TX;
  for (int t = blockIdx.x; t < nact * tiles; t += gridDim.x) {
    const int w = t / tiles, tt = t - w * tiles;
    int a0 = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) if (k == w) a0 = alist[k];
    const int gx = (tt % sp.tiles_x) * TX + lx, y0 = (tt / sp.tiles_x) * TY;
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int gy = y0 + ly + RPT * j;
      if (gx < sp.nx && gy < sp.ny) v += ldc(sp.r[a0] + (long long)gy * sp.pitch + gx);
    }
    v = warp_sum(v);
    if (lane == 0) sm.red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double g = 0.0;
      for (int k = 0; k < NT / 32; ++k) g += sm.red[k];
      sp.gsum[a0][tt] = g;
    }
    __syncthreads();
  }
}

// c_a = A_c^-1 (P^T r)_a for the continua in `act`, one warp per row, and
// this CTA's share of (P^T r_a) . c_a in gc (lane 0 of each warp).
template <int L>
__device__ void coarse_correct(const StepParams& sp, unsigned act, Smem& sm, double (&gc)[L]) {
  const int nc = sp.nc;
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * NT + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * NT) >> 5;
  double* sg = sm.box;  // P^T r staged in the idle TMA ring
  if (sp.tl_full) {
    // coupled: one Galerkin system over all continua (exchange blocks included)
#pragma unroll
    for (int a = 0; a < L; ++a) gc[a] = 0.0;
    const int n = L * nc;
    for (int J = threadIdx.x; J < n; J += NT) {
      const int a = J / nc;
      sg[J] = ldc(sp.gsum[a] + (J - a * nc));
    }
    __syncthreads();
    const double* Ai = sp.Ainv[0];
    for (long long R = gw; R < n; R += nw) {
      const double* row = Ai + R * n;
      double v = 0.0;
      for (int J = lane; J < n; J += 32) v = fma(ldr(row + J), sg[J], v);
      v = warp_sum(v);
      if (lane == 0) {
        const int a = (int)(R / nc);
        sp.ccor[a][R - (long long)a * nc] = v;
#pragma unroll
        for (int k = 0; k < L; ++k)
          if (k == a) gc[k] = fma(sg[R], v, gc[k]);
      }
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int a = 0; a < L; ++a) {
    gc[a] = 0.0;
    if (!(act & (1u << a))) continue;
    for (int J = threadIdx.x; J < nc; J += NT) sg[J] = ldc(sp.gsum[a] + J);
    __syncthreads();
    const double* Ai = sp.Ainv[a];
    for (long long I = gw; I < nc; I += nw) {
      const double* row = Ai + I * nc;
      double v = 0.0;
      for (int J = lane; J < nc; J += 32) v = fma(ldr(row + J), sg[J], v);
      v = warp_sum(v);
      if (lane == 0) {
        sp.ccor[a][I] = v;
        gc[a] = fma(sg[I], v, gc[a]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// One linear solve: the continua in `mask` (decoupled, independent systems),
// or all L continua as one coupled system. Warm start from p, result in p.
// Returns false when the run must stop (timeout, breakdown, no convergence).
template <int L, bool COUPLED, bool TLV>
__device__ bool pcg_solve(const StepParams& sp, const TmaMaps& maps, unsigned mask, Smem& sm,
                          uint32_t& phb) {
  constexpr int NL = COUPLED ? L : 1;
  constexpr int NARR = 2 * NL;
  constexpr int NST = nstage(L, COUPLED);
  const int nx = sp.nx, ny = sp.ny, pitch = sp.pitch;
  const long long Np = sp.Np;
  const int tid = threadIdx.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
  const long long gstride = (long long)gridDim.x * blockDim.x;

  // ---- fused right-hand side + initial residual (slot 0: bb, rr, rz) -----
  double acc[3 * L];
#pragma unroll
  for (int k = 0; k < 3 * L; ++k) acc[k] = 0.0;
#pragma unroll
  for (int a = 0; a < L; ++a) {
    if (!(mask & (1u << a))) continue;
    const double* pa = sp.p[a];
    for (long long i = gtid; i < Np; i += gstride) {
      const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
      if (gx >= nx) continue;
      const double xc = ldc(pa + i);
      double f = ldr(sp.F[a] + i);
      double wx = 0.0;  // implicit well term: b += W p_w, A x += W x
      if (sp.W[a]) {
        f += ldr(sp.FW[a] + i);
        wx = ldr(sp.W[a] + i) * xc;
      }
      double ex = 0.0, exb = 0.0;
#pragma unroll
      for (int b = 0; b < L; ++b) {
        if (b == a) continue;
        const double qv = qab(sp, a, b, i);
        const double pb = ldc(sp.p[b] + i);
        ex += qv * (pb - xc);
        exb += qv * pb;
      }
      const double rv = (f - wx) + ex - stencil_flux(sp, a, pa, gx, gy, i, xc);
      const double bv = COUPLED ? sp.mtau[a] * xc + f : sp.mtau[a] * xc + f + exb;
      const double z = ldr(sp.invd[a] + i) * rv;
      sp.r[a][i] = rv;
      sp.z[a][i] = z;
      sp.P[0][a][i] = z;  // P_old of the first iteration (beta = 0): any finite value
      acc[0 * L + a] += bv * bv;
      acc[1 * L + a] += rv * rv;
      acc[2 * L + a] += rv * z;
    }
  }
  block_store<3 * L>(acc, qbits(mask, L, 3), sm.box, sp.partials, 0);
  if (!grid_sync(sp)) return false;
  grid_totals<3 * L>(sp.partials, 0, sm.res, qbits(mask, L, 3));
  const double rtol2 = sp.rtol * sp.rtol;
  Scal64& S = *sm.sc;
  if (tid == 0) {
    double sb = 0, sr = 0, sz = 0;
    for (int a = 0; a < L; ++a) {
      S.bb[a] = sm.res[a];
      S.rr[a] = sm.res[L + a];
      S.rz[a] = sm.res[2 * L + a];
      S.beta[a] = 0.0;
      S.alpha[a] = 0.0;
      S.iters[a] = 0;
      if (mask & (1u << a)) { sb += S.bb[a]; sr += S.rr[a]; sz += S.rz[a]; }
    }
    if (COUPLED)
      for (int a = 0; a < L; ++a) { S.bb[a] = sb; S.rr[a] = sr; S.rz[a] = sz; }
    unsigned act = 0;
    for (int a = 0; a < L; ++a)
      if ((mask & (1u << a)) && S.rr[a] > rtol2 * S.bb[a]) act |= 1u << a;
    S.active = act;
    S.flag = 0;
  }
  __syncthreads();
  unsigned active = S.active;
  int it = 0;
  int cur = 0;
  int slot = 1;
  bool ok = true;
  // Two-level: the coarse correction of every continuum. The coupled scheme
  // takes the coarse space blockdiag(P_a) with the Galerkin operator P^T A P
  // of the coupled matrix (exchange blocks included, sp.tl_full), its (r, z)
  // the sum over the continua.
  constexpr bool TL = TLV;
  if (TL && active) {
    // z_0 = D^-1 r_0 + P c_0: the coarse term, and its share of (r_0, z_0)
    tile_rsums<L>(sp, active, sm);
    if (!grid_sync(sp)) return false;
    double gc[L];
    coarse_correct<L>(sp, active, sm, gc);
    block_store<L>(gc, active, sm.box, sp.partials, slot);
    if (!grid_sync(sp)) return false;
    grid_totals<L>(sp.partials, slot, sm.res, active);
    slot ^= 1;
    if (tid == 0) {
      double gsum = 0.0;
      for (int a = 0; a < L; ++a) gsum += sm.res[a];
      for (int a = 0; a < L; ++a)
        if (active & (1u << a)) S.rz[a] += COUPLED ? gsum : sm.res[a];
    }
    __syncthreads();
  }

  const int tiles = sp.tiles_x * sp.tiles_y;
  const int lx = tid % TX, ly = tid / TX;  // own cells (lx, ly + RPT * j), j < CPT
  while (active) {
    if (it >= sp.max_iter) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(sp.status, 0, (int)MC_E_NOCONV);
      ok = false;
      break;
    }
    // ---- phase A: TMA halo tiles, P_new = z + beta P_old, q = A P_new -----
    int act_list[L];
    int nact = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) if (active & (1u << a)) act_list[nact++] = a;
    double pq[L];
#pragma unroll
    for (int a = 0; a < L; ++a) pq[a] = 0.0;
    const int ntask = COUPLED ? tiles : nact * tiles;

    // issue the TMA boxes of task t into stage s (thread 0 only)
    auto issue = [&](int t, int s) {
      int a0 = 0, tt = t;
      if (!COUPLED) {
        const int w = t / tiles;
        tt = t - w * tiles;
#pragma unroll
        for (int k = 0; k < L; ++k) if (k == w) a0 = act_list[k];
      }
      const int bx0 = (tt % sp.tiles_x) * TX - HOFF;
      const int by0 = (tt / sp.tiles_x) * TY - 1;
      uint64_t* bar = sm.bar + s;
      fence_proxy_async();
      mbar_expect_tx(bar, NARR * BOX_BYTES);
      double* base = sm.box + (size_t)s * NARR * ABOX;
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const int a = COUPLED ? l : a0;
        tma_load_2d(base + (2 * l + 0) * ABOX, &maps.z[a], bx0, by0, bar);
        tma_load_2d(base + (2 * l + 1) * ABOX, &maps.P[cur][a], bx0, by0, bar);
      }
    };

    const int G = gridDim.x;
    int t = blockIdx.x;
    int k = 0;
    unsigned pend = 0;  // stages with a TMA load in flight (uniform in the CTA)
    // prologue: the first NST-1 tasks of this CTA in flight
#pragma unroll
    for (int j = 0; j < NST - 1; ++j) {
      const int tj = t + j * G;
      if (tj < ntask) {
        if (tid == 0) issue(tj, j);
        pend |= 1u << j;
      }
    }
    bool tma_ok = true;
    for (; t < ntask; t += G, ++k) {
      const int s = k % NST;
      {
        // refill the stage freed by the previous task with the task NST-1 ahead
        const int tn = t + (NST - 1) * G;
        const int sn = (k + NST - 1) % NST;
        if (tn < ntask) {
          if (tid == 0) issue(tn, sn);
          pend |= 1u << sn;
        }
      }
      int a0 = 0, tt = t;
      if (!COUPLED) {
        const int w = t / tiles;
        tt = t - w * tiles;
#pragma unroll
        for (int kk = 0; kk < L; ++kk) if (kk == w) a0 = act_list[kk];
      }
      const int x0 = (tt % sp.tiles_x) * TX;
      const int y0 = (tt / sp.tiles_x) * TY;
      const int gx = x0 + lx;
      // read-only coefficients of the own cells, fetched while TMA lands
      // (decoupled tiles; the coupled tile loads them in the compute loop)
      double te[CPT], tw[CPT], tn[CPT], ts[CPT], dc[CPT];
      if (!COUPLED) {
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int gy = y0 + ly + RPT * j;
          const long long i = (long long)gy * pitch + gx;
          te[j] = tw[j] = tn[j] = ts[j] = dc[j] = 0.0;
          if (gx < nx && gy < ny) {
            te[j] = ldr(sp.TE[a0] + i);
            tn[j] = ldr(sp.TN[a0] + i);
            if (gx > 0) tw[j] = ldr(sp.TE[a0] + i - 1);
            if (gy > 0) ts[j] = ldr(sp.TN[a0] + i - pitch);
            dc[j] = diagc(sp, a0, i);
          }
        }
      }
      if (!mbar_wait(sm.bar + s, (phb >> s) & 1u, sp.spin_limit)) {
        if (tid == 0) raise_abort(sp, (int)MC_E_TIMEOUT);
        tma_ok = false;
        break;
      }
      phb ^= 1u << s;
      pend &= ~(1u << s);
      if (TL) {
        // c of this tile and of its 8 neighbours (0 outside the tile grid),
        // for every continuum of the tile
        if (tid < 9 * NL) {
          const int l = tid / 9, kk = tid - 9 * l;
          const int a = COUPLED ? l : a0;
          const int cx = tt % sp.tiles_x + kk % 3 - 1, cy = tt / sp.tiles_x + kk / 3 - 1;
          sm.cn[tid] = (cx >= 0 && cx < sp.tiles_x && cy >= 0 && cy < sp.tiles_y)
                           ? ldc(sp.ccor[a] + cy * sp.tiles_x + cx)
                           : 0.0;
        }
        __syncthreads();
      }
      const double* base = sm.box + (size_t)s * NARR * ABOX;
      // P_new on the 66 x 18 halo region (box columns 1..66)
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const int a = COUPLED ? l : a0;
        const double bt = S.beta[a];
        const double* bz = base + (2 * l + 0) * ABOX;
        const double* bp = base + (2 * l + 1) * ABOX;
        double* pn = sm.pn + l * PN;
        for (int e = tid; e < PN; e += NT) {
          const int ry = e / PX, rx = e - ry * PX;
          const int bidx = ry * BX + rx + 1;
          double zc = bz[bidx];
          if (TL)
            zc += sm.cn[9 * l + (ry == 0 ? 0 : (ry == BY - 1 ? 6 : 3)) + (rx == 0 ? 0 : (rx == PX - 1 ? 2 : 1))];
          pn[e] = fma(bt, bp[bidx], zc);
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int lyj = ly + RPT * j;
        const int gy = y0 + lyj;
        if (gx >= nx || gy >= ny) continue;
        const long long i = (long long)gy * pitch + gx;
        const int c = (lyj + 1) * PX + lx + 1;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          const int a = COUPLED ? l : a0;
          double cte, ctw, ctn, cts, cdc;
          if (COUPLED) {
            cte = ldr(sp.TE[a] + i);
            ctn = ldr(sp.TN[a] + i);
            ctw = gx > 0 ? ldr(sp.TE[a] + i - 1) : 0.0;
            cts = gy > 0 ? ldr(sp.TN[a] + i - pitch) : 0.0;
            cdc = diagc(sp, a, i);
          } else {
            cte = te[j]; ctw = tw[j]; ctn = tn[j]; cts = ts[j]; cdc = dc[j];
          }
          const double* pn = sm.pn + l * PN;
          const double pc = pn[c];
          double qv = cdc * pc + cte * (pc - pn[c + 1]) + ctw * (pc - pn[c - 1]) +
                      ctn * (pc - pn[c + PX]) + cts * (pc - pn[c - PX]);
          if (COUPLED) {
#pragma unroll
            for (int b = 0; b < L; ++b) {
              if (b == a) continue;
              qv -= qab(sp, a, b, i) * sm.pn[b * PN + c];
            }
          }
          sp.P[cur ^ 1][a][i] = pc;
          sp.q[a][i] = qv;
#pragma unroll
          for (int kk = 0; kk < L; ++kk) if (kk == a) pq[kk] += pc * qv;
        }
      }
      __syncthreads();
    }
    if (!tma_ok) {
      // Leave no TMA copy landing in this CTA's shared memory after it exits:
      // wait (bounded again) for every load still in flight.
      for (int st = 0; st < NST; ++st)
        if (pend & (1u << st)) mbar_wait(sm.bar + st, (phb >> st) & 1u, 1LL << 24);
      ok = false;
      break;
    }
    block_store<L>(pq, active, sm.box, sp.partials, slot);
    if (!grid_sync(sp)) { ok = false; break; }
    grid_totals<L>(sp.partials, slot, sm.res, active);
    slot ^= 1;
    if (tid == 0) {
      double pqs = 0.0;
      for (int a = 0; a < L; ++a) pqs += sm.res[a];
      int brk = 0;
      for (int a = 0; a < L; ++a) {
        S.alpha[a] = 0.0;
        if (active & (1u << a)) {
          const double pqt = COUPLED ? pqs : sm.res[a];
          if (!(pqt > 0.0) || !isfinite(pqt)) brk = 1;
          else S.alpha[a] = S.rz[a] / pqt;
        }
      }
      S.flag = brk;
    }
    __syncthreads();
    if (S.flag) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(sp.status, 0, (int)MC_E_BREAKDOWN);
      ok = false;
      break;
    }
    // ---- phase B: x += alpha P, r -= alpha q (slot: rr, rz), 2 cells/thread --
    double acc2[2 * L];
#pragma unroll
    for (int kk = 0; kk < 2 * L; ++kk) acc2[kk] = 0.0;
    const long long Np2 = Np >> 1;
    if (TL) {
      // tile by tile (same hand-out as phase A), so that P^T r of every tile
      // is summed inside one CTA
      const int lane = tid & 31, warp = tid >> 5;
      for (int t = blockIdx.x; t < nact * tiles; t += gridDim.x) {
        const int w = t / tiles, tt = t - w * tiles;
        int a0 = 0;
#pragma unroll
        for (int kk = 0; kk < L; ++kk) if (kk == w) a0 = act_list[kk];
        const double al = S.alpha[a0];
        const int gx = (tt % sp.tiles_x) * TX + lx, y0 = (tt / sp.tiles_x) * TY;
        double* x = sp.p[a0];
        double* r = sp.r[a0];
        double* zz = sp.z[a0];
        const double* Pn = sp.P[cur ^ 1][a0];
        double rs = 0.0;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int gy = y0 + ly + RPT * j;
          if (gx >= nx || gy >= ny) continue;
          const long long i = (long long)gy * pitch + gx;
          const double rv = ldc(r + i) - al * ldc(sp.q[a0] + i);
          const double xn = ldc(x + i) + al * ldc(Pn + i);
          const double zv = ldr(sp.invd[a0] + i) * rv;
          x[i] = xn;
          r[i] = rv;
          zz[i] = zv;
#pragma unroll
          for (int kk = 0; kk < L; ++kk)
            if (kk == a0) {
              acc2[kk] += rv * rv;
              acc2[L + kk] += rv * zv;
            }
          rs += rv;
        }
        rs = warp_sum(rs);
        if (lane == 0) sm.red[warp] = rs;
        __syncthreads();
        if (tid == 0) {
          double g = 0.0;
          for (int k2 = 0; k2 < NT / 32; ++k2) g += sm.red[k2];
          sp.gsum[a0][tt] = g;
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (TL || !(active & (1u << a))) continue;
      const double al = S.alpha[a];
      double2* x = reinterpret_cast<double2*>(sp.p[a]);
      double2* r = reinterpret_cast<double2*>(sp.r[a]);
      const double2* Pn = reinterpret_cast<const double2*>(sp.P[cur ^ 1][a]);
      const double2* qq = reinterpret_cast<const double2*>(sp.q[a]);
      const double2* iv = reinterpret_cast<const double2*>(sp.invd[a]);
      double2* zz = reinterpret_cast<double2*>(sp.z[a]);
#pragma unroll 2
      for (long long j = gtid; j < Np2; j += gstride) {
        const double2 rv0 = __ldcg(r + j);
        const double2 qv = __ldcg(qq + j);
        const double2 xv = __ldcg(x + j);
        const double2 pv = __ldcg(Pn + j);
        const double2 dv = __ldg(iv + j);
        double2 rv, xn, zv;
        rv.x = rv0.x - al * qv.x;
        rv.y = rv0.y - al * qv.y;
        xn.x = xv.x + al * pv.x;
        xn.y = xv.y + al * pv.y;
        zv.x = dv.x * rv.x;
        zv.y = dv.y * rv.y;
        x[j] = xn;
        r[j] = rv;
        zz[j] = zv;
        acc2[a] += rv.x * rv.x + rv.y * rv.y;
        acc2[L + a] += rv.x * zv.x + rv.y * zv.y;
      }
    }
    block_store<2 * L>(acc2, qbits(active, L, 2), sm.box, sp.partials, slot);
    if (!grid_sync(sp)) { ok = false; break; }
    grid_totals<2 * L>(sp.partials, slot, sm.res, qbits(active, L, 2));
    slot ^= 1;
    ++it;
    if (tid == 0) {
      double s0 = 0, s1 = 0;
      for (int a = 0; a < L; ++a) { s0 += sm.res[a]; s1 += sm.res[L + a]; }
      unsigned act = active;
      int bad = 0;
      for (int a = 0; a < L; ++a) {
        if (!(active & (1u << a))) continue;
        const double rra = COUPLED ? s0 : sm.res[a];
        const double rzn = COUPLED ? s1 : sm.res[L + a];
        S.rr[a] = rra;
        if (TL) {
          S.rzl[a] = rzn;  // beta after the coarse term
        } else {
          S.beta[a] = rzn / S.rz[a];
          S.rz[a] = rzn;
        }
        S.iters[a] = it;
        if (!(rra > rtol2 * S.bb[a])) act &= ~(1u << a);
        if (!isfinite(rra)) bad = 1;
      }
      S.active = act;
      S.flag = bad;
    }
    __syncthreads();
    active = S.active;
    if (S.flag) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(sp.status, 0, (int)MC_E_BREAKDOWN);
      ok = false;
      break;
    }
    if (TL && active) {
      double gc[L];
      coarse_correct<L>(sp, active, sm, gc);
      block_store<L>(gc, active, sm.box, sp.partials, slot);
      if (!grid_sync(sp)) { ok = false; break; }
      grid_totals<L>(sp.partials, slot, sm.res, active);
      slot ^= 1;
      if (tid == 0) {
        double gsum = 0.0;
        for (int a = 0; a < L; ++a) gsum += sm.res[a];
        for (int a = 0; a < L; ++a)
          if (active & (1u << a)) {
            const double rzn = S.rzl[a] + (COUPLED ? gsum : sm.res[a]);
            S.beta[a] = rzn / S.rz[a];
            S.rz[a] = rzn;
          }
      }
      __syncthreads();
    }
    cur ^= 1;
  }
  // ---- constant-mode correction --------------------------------------------
  // The zero-flux systems have near-null modes that only the mass and
  // exchange diagonal holds: the constant of each solved continuum. Because
  // 1^T D = 0, the exact solution satisfies, for every such constant 1_a,
  //   1_a^T (b - A x) = sum_i (F + m_a/tau (p_a^{n-1} - x_a) + exchange)_i = 0.
  // Rounding in A P leaves a residual in these directions that the small
  // diagonal amplifies; a Galerkin correction x += sum_a c_a 1_a with
  // G c = 1^T (b - A x), G_ab = 1_a^T A 1_b, restores the identities
  // (decoupled: one independent 1 x 1 system per continuum; coupled: L x L).
  // The per-cell terms are differences of nearby values, so the sums are
  // accurate.
  if (ok) {
    constexpr int NPAIR = L * (L - 1) / 2;
    // decoupled: [1^T r, 1^T diag(A0 - D)] per continuum; coupled:
    // [1^T r per continuum, Q sums per pair, well sums per continuum]
    constexpr int NQC = COUPLED ? 2 * L + NPAIR : 2 * L;
    double cs[NQC];
#pragma unroll
    for (int kk = 0; kk < NQC; ++kk) cs[kk] = 0.0;
    const bool lag_prev = sp.scheme == MC_SCHEME_D;
    for (long long i = gtid; i < Np; i += gstride) {
      const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
      if (gx >= nx) continue;
      double xv[L];
#pragma unroll
      for (int a = 0; a < L; ++a) xv[a] = (mask & (1u << a)) ? ldc(sp.p[a] + i) : 0.0;
      int pi = 0;
#pragma unroll
      for (int a = 0; a < L; ++a) {
        if (!(mask & (1u << a))) continue;
        double tv = ldr(sp.F[a] + i) + sp.mtau[a] * (ldc(sp.pprev[a] + i) - xv[a]);
        if (sp.W[a]) {
          const double wv = ldr(sp.W[a] + i);
          tv += ldr(sp.FW[a] + i) - wv * xv[a];
          if (COUPLED) cs[L + NPAIR + a] += wv;
        }
#pragma unroll
        for (int b = 0; b < L; ++b) {
          if (b == a) continue;
          const double pb = COUPLED ? xv[b] : (lag_prev ? ldc(sp.pprev[b] + i) : ldc(sp.p[b] + i));
          tv += qab(sp, a, b, i) * (pb - xv[a]);
        }
        cs[a] += tv;
        if (!COUPLED) cs[L + a] += diagc(sp, a, i);
      }
      if (COUPLED) {
#pragma unroll
        for (int a = 0; a < L; ++a)
#pragma unroll
          for (int b = a + 1; b < L; ++b) cs[L + pi++] += qab(sp, a, b, i);
      }
    }
    block_store<NQC>(cs, (1u << NQC) - 1u, sm.box, sp.partials, slot);
    if (!grid_sync(sp)) {
      ok = false;
    } else {
      double ct[NQC];
      grid_sum<NQC>(sp.partials, slot, sm.res, ct);
      slot ^= 1;
      double shift[L];
      if (COUPLED) {
        // G_aa = N m_a/tau + sum_b Q_ab + W_a, G_ab = -Q_ab (Q, W summed over cells)
        double G[L][L], c[L];
#pragma unroll
        for (int a = 0; a < L; ++a) {
#pragma unroll
          for (int b = 0; b < L; ++b) G[a][b] = 0.0;
          G[a][a] = (double)sp.N * sp.mtau[a] + ct[L + NPAIR + a];
          c[a] = ct[a];
        }
        int pi = 0;
#pragma unroll
        for (int a = 0; a < L; ++a)
#pragma unroll
          for (int b = a + 1; b < L; ++b) {
            const double Q = ct[L + pi++];
            G[a][a] += Q;
            G[b][b] += Q;
            G[a][b] -= Q;
            G[b][a] -= Q;
          }
        // Gaussian elimination (G is SPD: no pivoting needed)
#pragma unroll
        for (int kk = 0; kk < L; ++kk) {
#pragma unroll
          for (int r = kk + 1; r < L; ++r) {
            const double f = G[r][kk] / G[kk][kk];
#pragma unroll
            for (int cc = kk; cc < L; ++cc) G[r][cc] -= f * G[kk][cc];
            c[r] -= f * c[kk];
          }
        }
#pragma unroll
        for (int r = L - 1; r >= 0; --r) {
          double v = c[r];
#pragma unroll
          for (int cc = r + 1; cc < L; ++cc) v -= G[r][cc] * shift[cc];
          shift[r] = v / G[r][r];
        }
      } else {
#pragma unroll
        for (int a = 0; a < L; ++a) shift[a] = ct[L + a] > 0.0 ? ct[a] / ct[L + a] : 0.0;
      }
#pragma unroll
      for (int a = 0; a < L; ++a) {
        if (!(mask & (1u << a))) continue;
        const double sh = shift[a];
        if (!isfinite(sh)) continue;
        for (long long i = gtid; i < Np; i += gstride) {
          const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
          if (gx >= nx) continue;
          sp.p[a][i] = ldc(sp.p[a] + i) + sh;
        }
      }
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(mask & (1u << a))) continue;
      if (COUPLED && a != 0) continue;
      const int ka = COUPLED ? 0 : a;
      sp.iters[ka] += S.iters[a];
      if (S.iters[a] > sp.max_iters[ka]) sp.max_iters[ka] = S.iters[a];
      sp.relres[ka] = S.bb[a] > 0 ? sqrt(S.rr[a] / S.bb[a]) : sqrt(S.rr[a]);
    }
  }
  // The next solve's first pass reads p and rewrites partial slot 0: every
  // CTA must be past this solve's last reads first.
  if (ok && !grid_sync(sp)) ok = false;
  return ok;
}

// ---------------------------------------------------------------------------
// Jacobi PCG in scaled variables. With S = diag(sqrt(d)) (d the diagonal of
// the system matrix A: a continuum's block for the decoupled schemes, the
// whole coupled matrix for the coupled one -- the same d), Jacobi-
// preconditioned CG on A x = b is, iterate for iterate, plain CG on
// (S^-1 A S^-1) y = S^-1 b with y = S x: the scaled residual r~ = S^-1 r
// satisfies r~.r~ = r.(D^-1 r), and the scaled search direction is p~ = S p.
// The scaled operator has a unit diagonal, face entries
// t_ij = T_ij / sqrt(d_i d_j) and (coupled) exchange entries
// q_ab,i / sqrt(d_a,i d_b,i) (set-up kernels), so
//   q~_a = p~_a - sum_faces t p~_a(neighbour) [- sum_b qs_ab p~_b (coupled)].
// The stopping test stays the unscaled one, ||b - A x||_2 = ||S r~||_2 <=
// rtol ||b||_2, evaluated every CHK-th iteration (at most CHK - 1 extra
// iterations). The initial residual (fused with the right-hand side) and the
// constant-mode correction after the solve use the unscaled flux form, as in
// pcg_solve. y lives in the z buffer during the solve; p keeps the unscaled
// x until the end.
// The three stages are separate (not inlined) functions so that the
// iteration loop gets a register allocation of its own.
constexpr int CHK = 4;

template <int L, bool C>
__device__ __noinline__ bool scaled_init(const StepParams& sp, unsigned mask, Smem& sm, bool sp1) {
  const int nx = sp.nx, pitch = sp.pitch;
  const long long Np = sp.Np;
  const int tid = threadIdx.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  // ---- fused right-hand side + initial residual (slot 0: bb, rr, rz) -----
  double acc[3 * L];
#pragma unroll
  for (int k = 0; k < 3 * L; ++k) acc[k] = 0.0;
#pragma unroll
  for (int a = 0; a < L; ++a) {
    if (!(mask & (1u << a))) continue;
    const double* pa = sp.p[a];
    for (long long i = gtid; i < Np; i += gstride) {
      const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
      if (gx >= nx) continue;
      const double xc = ldc(pa + i);
      double f = ldr(sp.F[a] + i);
      double wx = 0.0;
      if (sp.W[a]) {
        f += ldr(sp.FW[a] + i);
        wx = ldr(sp.W[a] + i) * xc;
      }
      double ex = 0.0, exb = 0.0;
#pragma unroll
      for (int b = 0; b < L; ++b) {
        if (b == a) continue;
        const double qv = qab(sp, a, b, i);
        const double pb = ldc(sp.p[b] + i);
        ex += qv * (pb - xc);
        exb += qv * pb;
      }
      const double rv = (f - wx) + ex - stencil_flux(sp, a, pa, gx, gy, i, xc);
      const double bv = C ? sp.mtau[a] * xc + f : sp.mtau[a] * xc + f + exb;
      const double s = ldr(sp.sqd[a] + i);
      const double rt = rv / s;
      sp.r[a][i] = rt;
      sp.z[a][i] = xc * s;
      sp.P[0][a][i] = rt;  // P_old of the first iteration (beta = 0): any finite value
      if (sp1) {           // single-pass form: s = w = p = 0 before pass -1
        sp.P[0][a][i] = 0.0;
        sp.w[0][a][i] = 0.0;
        sp.pd[a][i] = 0.0;
      }
      acc[0 * L + a] += bv * bv;
      acc[1 * L + a] += rv * rv;
      acc[2 * L + a] += rt * rt;
    }
  }
  block_store<3 * L>(acc, qbits(mask, L, 3), sm.box, sp.partials, 0);
  if (!grid_sync(sp)) return false;
  grid_totals<3 * L>(sp.partials, 0, sm.res, qbits(mask, L, 3));
  const double rtol2 = sp.rtol * sp.rtol;
  Scal64& S = *sm.sc;
  if (tid == 0) {
    double sb = 0, sr = 0, sz = 0;
    for (int a = 0; a < L; ++a) {
      S.bb[a] = sm.res[a];
      S.rr[a] = sm.res[L + a];
      S.rz[a] = sm.res[2 * L + a];
      S.beta[a] = 0.0;
      S.alpha[a] = 0.0;
      S.iters[a] = 0;
      if (mask & (1u << a)) { sb += S.bb[a]; sr += S.rr[a]; sz += S.rz[a]; }
    }
    if (C)
      for (int a = 0; a < L; ++a) { S.bb[a] = sb; S.rr[a] = sr; S.rz[a] = sz; }
    unsigned act = 0;
    for (int a = 0; a < L; ++a)
      if ((mask & (1u << a)) && S.rr[a] > rtol2 * S.bb[a]) act |= 1u << a;
    S.active = act;
    S.flag = 0;
  }
  __syncthreads();
  return true;
}

// The iterations of the scaled solve; slot: next partial-sum slot (in/out).
template <int L, bool C>
__device__ __noinline__ bool scaled_loop(const StepParams& sp, const TmaMaps& maps, Smem& sm,
                                         uint32_t& phb, int& slot_io) {
  constexpr int NL = C ? L : 1;
  constexpr int NARR = 2 * NL;
  constexpr int NST = nstage(L, C);
  const int nx = sp.nx, ny = sp.ny, pitch = sp.pitch;
  const long long Np = sp.Np;
  const int tid = threadIdx.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  const double rtol2 = sp.rtol * sp.rtol;
  Scal64& S = *sm.sc;
  unsigned active = S.active;
  int it = 0;
  int cur = 0;
  int slot = slot_io;
  bool ok = true;

  const int tiles = sp.tiles_x * sp.tiles_y;
  const int lx = tid % TX, ly = tid / TX;  // own cells (lx, ly + RPT * j), j < CPT
  while (active) {
    if (it >= sp.max_iter) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(sp.status, 0, (int)MC_E_NOCONV);
      ok = false;
      break;
    }
    // ---- phase A: TMA halo tiles of r~ and P_old, P_new = r~ + beta P_old,
    //      q~ = (S^-1 A S^-1) P_new, <P_new, q~> -------------------------------
    int act_list[L];
    int nact = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) if (active & (1u << a)) act_list[nact++] = a;
    double pq[L];
#pragma unroll
    for (int a = 0; a < L; ++a) pq[a] = 0.0;
    const int ntask = C ? tiles : nact * tiles;

    auto issue = [&](int t, int s) {
      int a0 = 0, tt = t;
      if (!C) {
        const int w = t / tiles;
        tt = t - w * tiles;
#pragma unroll
        for (int k = 0; k < L; ++k) if (k == w) a0 = act_list[k];
      }
      const int bx0 = (tt % sp.tiles_x) * TX - HOFF;
      const int by0 = (tt / sp.tiles_x) * TY - 1;
      uint64_t* bar = sm.bar + s;
      fence_proxy_async();
      mbar_expect_tx(bar, NARR * BOX_BYTES);
      double* base = sm.box + (size_t)s * NARR * ABOX;
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const int a = C ? l : a0;
        tma_load_2d(base + (2 * l + 0) * ABOX, &maps.r[a], bx0, by0, bar);
        tma_load_2d(base + (2 * l + 1) * ABOX, &maps.P[cur][a], bx0, by0, bar);
      }
    };

    const int G = gridDim.x;
    int t = blockIdx.x;
    int k = 0;
    unsigned pend = 0;
#pragma unroll
    for (int j = 0; j < NST - 1; ++j) {
      const int tj = t + j * G;
      if (tj < ntask) {
        if (tid == 0) issue(tj, j);
        pend |= 1u << j;
      }
    }
    bool tma_ok = true;
    for (; t < ntask; t += G, ++k) {
      const int s = k % NST;
      {
        const int tn = t + (NST - 1) * G;
        const int sn = (k + NST - 1) % NST;
        if (tn < ntask) {
          if (tid == 0) issue(tn, sn);
          pend |= 1u << sn;
        }
      }
      int a0 = 0, tt = t;
      if (!C) {
        const int w = t / tiles;
        tt = t - w * tiles;
#pragma unroll
        for (int kk = 0; kk < L; ++kk) if (kk == w) a0 = act_list[kk];
      }
      const int x0 = (tt % sp.tiles_x) * TX;
      const int y0 = (tt / sp.tiles_x) * TY;
      const int gx = x0 + lx;
      // scaled face values of the own cells, fetched while TMA lands
      // (decoupled tiles; the coupled tile loads them in the compute loop)
      double te[CPT], tw[CPT], tn[CPT], ts[CPT];
      if (!C) {
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int gy = y0 + ly + RPT * j;
          const long long i = (long long)gy * pitch + gx;
          te[j] = tw[j] = tn[j] = ts[j] = 0.0;
          if (gx < nx && gy < ny) {
            te[j] = ldr(sp.tE[a0] + i);
            tn[j] = ldr(sp.tN[a0] + i);
            if (gx > 0) tw[j] = ldr(sp.tE[a0] + i - 1);
            if (gy > 0) ts[j] = ldr(sp.tN[a0] + i - pitch);
          }
        }
      }
      if (!mbar_wait(sm.bar + s, (phb >> s) & 1u, sp.spin_limit)) {
        if (tid == 0) raise_abort(sp, (int)MC_E_TIMEOUT);
        tma_ok = false;
        break;
      }
      phb ^= 1u << s;
      pend &= ~(1u << s);
      const double* base = sm.box + (size_t)s * NARR * ABOX;
      // decoupled tiles alternate between two P_new areas, so that no CTA
      // barrier is needed after the stencil (a thread can write area k % 2
      // only after every thread passed this tile's barrier below, i.e.
      // finished reading area k % 2 two tiles back)
      double* pnb = sm.pn + (C ? 0 : (k & 1) * PN);
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const int a = C ? l : a0;
        const double bt = S.beta[a];
        const double* br = base + (2 * l + 0) * ABOX;
        const double* bp = base + (2 * l + 1) * ABOX;
        double* pn = pnb + l * PN;
        for (int e = tid; e < PN; e += NT) {
          const int ry = e / PX, rx = e - ry * PX;
          const int bidx = ry * BX + rx + 1;
          pn[e] = fma(bt, bp[bidx], br[bidx]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int lyj = ly + RPT * j;
        const int gy = y0 + lyj;
        if (gx >= nx || gy >= ny) continue;
        const long long i = (long long)gy * pitch + gx;
        const int c = (lyj + 1) * PX + lx + 1;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          const int a = C ? l : a0;
          double cte, ctw, ctn, cts;
          if (C) {
            cte = ldr(sp.tE[a] + i);
            ctn = ldr(sp.tN[a] + i);
            ctw = gx > 0 ? ldr(sp.tE[a] + i - 1) : 0.0;
            cts = gy > 0 ? ldr(sp.tN[a] + i - pitch) : 0.0;
          } else {
            cte = te[j]; ctw = tw[j]; ctn = tn[j]; cts = ts[j];
          }
          const double* pn = pnb + l * PN;
          const double pc = pn[c];
          double nb = fma(cte, pn[c + 1], fma(ctw, pn[c - 1], fma(ctn, pn[c + PX], cts * pn[c - PX])));
          if (C) {
#pragma unroll
            for (int b = 0; b < L; ++b) {
              if (b == a) continue;
              nb = fma(ldr(sp.qs[a][b] + i), pnb[b * PN + c], nb);
            }
          }
          const double qv = pc - nb;
          sp.P[cur ^ 1][a][i] = pc;
          sp.q[a][i] = qv;
#pragma unroll
          for (int kk = 0; kk < L; ++kk) if (kk == a) pq[kk] = fma(pc, qv, pq[kk]);
        }
      }
      if (C) __syncthreads();
    }
    if (!tma_ok) {
      for (int st = 0; st < NST; ++st)
        if (pend & (1u << st)) mbar_wait(sm.bar + st, (phb >> st) & 1u, 1LL << 24);
      ok = false;
      break;
    }
    block_store<L>(pq, active, sm.box, sp.partials, slot);
    if (!grid_sync(sp)) { ok = false; break; }
    grid_totals<L>(sp.partials, slot, sm.res, active);
    slot ^= 1;
    if (tid == 0) {
      double pqs = 0.0;
      for (int a = 0; a < L; ++a) pqs += sm.res[a];
      int brk = 0;
      for (int a = 0; a < L; ++a) {
        S.alpha[a] = 0.0;
        if (active & (1u << a)) {
          const double pqt = C ? pqs : sm.res[a];
          if (!(pqt > 0.0) || !isfinite(pqt)) brk = 1;
          else S.alpha[a] = S.rz[a] / pqt;
        }
      }
      S.flag = brk;
    }
    __syncthreads();
    if (S.flag) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(sp.status, 0, (int)MC_E_BREAKDOWN);
      ok = false;
      break;
    }
    // ---- phase B: y += alpha P_new, r~ -= alpha q~, (r~, r~); every CHK-th
    //      iteration also ||S r~||^2 for the stopping test ------------------
    const bool chk = ((it + 1) % CHK) == 0;
    double acc2[2 * L];
#pragma unroll
    for (int kk = 0; kk < 2 * L; ++kk) acc2[kk] = 0.0;
    const long long Np2 = Np >> 1;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(active & (1u << a))) continue;
      const double al = S.alpha[a];
      double2* y = reinterpret_cast<double2*>(sp.z[a]);
      double2* r = reinterpret_cast<double2*>(sp.r[a]);
      const double2* Pn = reinterpret_cast<const double2*>(sp.P[cur ^ 1][a]);
      const double2* qq = reinterpret_cast<const double2*>(sp.q[a]);
      const double2* sq = reinterpret_cast<const double2*>(sp.sqd[a]);
      if (chk) {
        for (long long j = gtid; j < Np2; j += gstride) {
          const double2 rv0 = __ldcg(r + j);
          const double2 qv = __ldcg(qq + j);
          const double2 yv = __ldcg(y + j);
          const double2 pv = __ldcg(Pn + j);
          const double2 sv = __ldg(sq + j);
          double2 rv, yn;
          rv.x = fma(-al, qv.x, rv0.x);
          rv.y = fma(-al, qv.y, rv0.y);
          yn.x = fma(al, pv.x, yv.x);
          yn.y = fma(al, pv.y, yv.y);
          y[j] = yn;
          r[j] = rv;
          acc2[L + a] = fma(rv.x, rv.x, fma(rv.y, rv.y, acc2[L + a]));
          const double ux = sv.x * rv.x, uy = sv.y * rv.y;
          acc2[a] = fma(ux, ux, fma(uy, uy, acc2[a]));
        }
      } else {
#pragma unroll 2
        for (long long j = gtid; j < Np2; j += gstride) {
          const double2 rv0 = __ldcg(r + j);
          const double2 qv = __ldcg(qq + j);
          const double2 yv = __ldcg(y + j);
          const double2 pv = __ldcg(Pn + j);
          double2 rv, yn;
          rv.x = fma(-al, qv.x, rv0.x);
          rv.y = fma(-al, qv.y, rv0.y);
          yn.x = fma(al, pv.x, yv.x);
          yn.y = fma(al, pv.y, yv.y);
          y[j] = yn;
          r[j] = rv;
          acc2[L + a] = fma(rv.x, rv.x, fma(rv.y, rv.y, acc2[L + a]));
        }
      }
    }
    const unsigned qm = chk ? qbits(active, L, 2) : (active << L);
    block_store<2 * L>(acc2, qm, sm.box, sp.partials, slot);
    if (!grid_sync(sp)) { ok = false; break; }
    grid_totals<2 * L>(sp.partials, slot, sm.res, qm);
    slot ^= 1;
    ++it;
    if (tid == 0) {
      double s0 = 0, s1 = 0;
      for (int a = 0; a < L; ++a) { s0 += sm.res[a]; s1 += sm.res[L + a]; }
      unsigned act = active;
      int bad = 0;
      for (int a = 0; a < L; ++a) {
        if (!(active & (1u << a))) continue;
        const double rzn = C ? s1 : sm.res[L + a];
        S.beta[a] = rzn / S.rz[a];
        S.rz[a] = rzn;
        S.iters[a] = it;
        if (!isfinite(rzn)) bad = 1;
        if (rzn == 0.0) {  // exact solution (tiny grids): converged
          S.rr[a] = 0.0;
          act &= ~(1u << a);
        } else if (chk) {
          const double rra = C ? s0 : sm.res[a];
          S.rr[a] = rra;
          if (!(rra > rtol2 * S.bb[a])) act &= ~(1u << a);
          if (!isfinite(rra)) bad = 1;
        }
      }
      S.active = act;
      S.flag = bad;
    }
    __syncthreads();
    active = S.active;
    if (S.flag) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(sp.status, 0, (int)MC_E_BREAKDOWN);
      ok = false;
      break;
    }
    cur ^= 1;
  }
  slot_io = slot;
  return ok;
}

// Back to x = y / sqrt(d) with the constant-mode correction of pcg_solve:
// decoupled, per solved continuum c_a = 1^T (b - A x)_a / 1^T diag(A0 - D)_a;
// coupled, one constant per continuum from the L x L Galerkin system; the
// sums use the non-diffusive terms only (1^T D = 0).
template <int L, bool C>
__device__ __noinline__ bool scaled_finish(const StepParams& sp, unsigned mask, Smem& sm, int slot) {
  constexpr int NPAIR = L * (L - 1) / 2;
  constexpr int NQC = C ? 2 * L + NPAIR : 2 * L;
  const int nx = sp.nx, pitch = sp.pitch;
  const long long Np = sp.Np;
  const int tid = threadIdx.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  Scal64& S = *sm.sc;
  bool ok = true;
  double cs[NQC];
#pragma unroll
  for (int kk = 0; kk < NQC; ++kk) cs[kk] = 0.0;
  const bool lag_prev = sp.scheme == MC_SCHEME_D;
  for (long long i = gtid; i < Np; i += gstride) {
    const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
    if (gx >= nx) continue;
    double xv[L];
#pragma unroll
    for (int a = 0; a < L; ++a)
      xv[a] = (mask & (1u << a)) ? ldc(sp.z[a] + i) / ldr(sp.sqd[a] + i) : 0.0;
    int pi = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(mask & (1u << a))) continue;
      double tv = ldr(sp.F[a] + i) + sp.mtau[a] * (ldc(sp.pprev[a] + i) - xv[a]);
      if (sp.W[a]) {
        const double wv = ldr(sp.W[a] + i);
        tv += ldr(sp.FW[a] + i) - wv * xv[a];
        if (C) cs[L + NPAIR + a] += wv;
      }
#pragma unroll
      for (int b = 0; b < L; ++b) {
        if (b == a) continue;
        const double pb = C ? xv[b] : (lag_prev ? ldc(sp.pprev[b] + i) : ldc(sp.p[b] + i));
        tv += qab(sp, a, b, i) * (pb - xv[a]);
      }
      cs[a] += tv;
      if (!C) cs[L + a] += diagc(sp, a, i);
    }
    if (C) {
#pragma unroll
      for (int a = 0; a < L; ++a)
#pragma unroll
        for (int b = a + 1; b < L; ++b) cs[L + pi++] += qab(sp, a, b, i);
    }
  }
  block_store<NQC>(cs, (1u << NQC) - 1u, sm.box, sp.partials, slot);
  if (!grid_sync(sp)) {
    ok = false;
  } else {
    double ct[NQC];
    grid_sum<NQC>(sp.partials, slot, sm.res, ct);
    double shift[L];
    if (C) {
      // G_aa = N m_a/tau + sum_b Q_ab + W_a, G_ab = -Q_ab (Q, W summed over cells)
      double G[L][L], c[L];
#pragma unroll
      for (int a = 0; a < L; ++a) {
#pragma unroll
        for (int b = 0; b < L; ++b) G[a][b] = 0.0;
        G[a][a] = (double)sp.N * sp.mtau[a] + ct[L + NPAIR + a];
        c[a] = ct[a];
      }
      int pi = 0;
#pragma unroll
      for (int a = 0; a < L; ++a)
#pragma unroll
        for (int b = a + 1; b < L; ++b) {
          const double Q = ct[L + pi++];
          G[a][a] += Q;
          G[b][b] += Q;
          G[a][b] -= Q;
          G[b][a] -= Q;
        }
#pragma unroll
      for (int kk = 0; kk < L; ++kk) {
#pragma unroll
        for (int r = kk + 1; r < L; ++r) {
          const double f = G[r][kk] / G[kk][kk];
#pragma unroll
          for (int cc = kk; cc < L; ++cc) G[r][cc] -= f * G[kk][cc];
          c[r] -= f * c[kk];
        }
      }
#pragma unroll
      for (int r = L - 1; r >= 0; --r) {
        double v = c[r];
#pragma unroll
        for (int cc = r + 1; cc < L; ++cc) v -= G[r][cc] * shift[cc];
        shift[r] = v / G[r][r];
      }
    } else {
#pragma unroll
      for (int a = 0; a < L; ++a) shift[a] = ct[L + a] > 0.0 ? ct[a] / ct[L + a] : 0.0;
    }
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(mask & (1u << a))) continue;
      const double sh = isfinite(shift[a]) ? shift[a] : 0.0;
      for (long long i = gtid; i < Np; i += gstride) {
        const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
        if (gx >= nx) continue;
        sp.p[a][i] = ldc(sp.z[a] + i) / ldr(sp.sqd[a] + i) + sh;
      }
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(mask & (1u << a))) continue;
      if (C && a != 0) continue;
      sp.iters[a] += S.iters[a];
      if (S.iters[a] > sp.max_iters[a]) sp.max_iters[a] = S.iters[a];
      sp.relres[a] = S.bb[a] > 0 ? sqrt(S.rr[a] / S.bb[a]) : sqrt(S.rr[a]);
    }
  }
  // The next solve's first pass reads p and rewrites partial slot 0: every
  // CTA must be past this solve's last reads first.
  if (ok && !grid_sync(sp)) ok = false;
  return ok;
}

// ---------------------------------------------------------------------------
// Single-pass form of the scaled iteration: the Chronopoulos-Gear recurrences
// of CG on the unit-diagonal system (u = r there, w = A~ r, s = A~ p carried
// by recurrence), ONE tile pass and ONE grid reduction per iteration. In exact
// arithmetic the iterates are those of scaled_loop (plain CG); the two inner
// products gamma = (r, r) and delta = (w, r) of an iteration are formed after
// the same pass, and alpha = gamma / (delta - beta gamma / alpha_prev).
// Pass i, tile by tile with a one-cell halo:
//   s_i = w_i + beta_i s_{i-1},  r_{i+1} = r_i - alpha_i s_i     (tile + halo)
//   p_i = r_i + beta_i p_{i-1},  y += alpha_i p_i                 (tile)
//   w_{i+1} = A~ r_{i+1},  gamma, delta (and every CHK-th pass ||S r||^2)
// The halo values are recomputed from the previous pass's r, s, w (the same
// fused multiply-adds as their owner tile, so both copies agree bit for bit).
// r, s, w are double-buffered (buffer `cur` read through TMA, `cur ^ 1`
// written): r in (r, q), s in (P[0], P[1]), w in (w[0], w[1]); p and y are
// touched only at their own cells. Pass -1 runs with alpha = beta = 0 on
// s = w = p = 0 and forms w_0 = A~ r_0 and the first inner products.
__host__ __device__ constexpr int nstage1(int L, bool coupled) {
  return !coupled ? 3 : (L <= 1 ? 3 : 1);
}

template <int L, bool C>
__device__ __noinline__ bool sp1_loop(const StepParams& sp, const TmaMaps& maps, Smem& sm, uint32_t& phb,
                                      int& slot_io) {
  constexpr int NL = C ? L : 1;
  constexpr int NARR = 3 * NL;
  constexpr int NST = nstage1(L, C);
  const int nx = sp.nx, ny = sp.ny, pitch = sp.pitch;
  const int tid = threadIdx.x;
  const double rtol2 = sp.rtol * sp.rtol;
  Scal64& S = *sm.sc;
  unsigned active = S.active;
  int it = -1;
  int cur = 0;
  int slot = slot_io;
  bool ok = true;
  if (tid == 0)
    for (int a = 0; a < L; ++a) { S.alpha[a] = 0.0; S.beta[a] = 0.0; }
  __syncthreads();

  const int tiles = sp.tiles_x * sp.tiles_y;
  const int lx = tid % TX, ly = tid / TX;
  while (active) {
    if (it >= sp.max_iter) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(sp.status, 0, (int)MC_E_NOCONV);
      ok = false;
      break;
    }
    const bool chk = it >= 0 && ((it + 1) % CHK) == 0;
    int act_list[L];
    int nact = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) if (active & (1u << a)) act_list[nact++] = a;
    double dots[3 * L];   // gamma, delta, ||S r||^2 per continuum
#pragma unroll
    for (int a = 0; a < 3 * L; ++a) dots[a] = 0.0;
    const int ntask = C ? tiles : nact * tiles;

    auto issue = [&](int t, int s) {
      int a0 = 0, tt = t;
      if (!C) {
        const int w = t / tiles;
        tt = t - w * tiles;
#pragma unroll
        for (int k = 0; k < L; ++k) if (k == w) a0 = act_list[k];
      }
      const int bx0 = (tt % sp.tiles_x) * TX - HOFF;
      const int by0 = (tt / sp.tiles_x) * TY - 1;
      uint64_t* bar = sm.bar + s;
      fence_proxy_async();
      mbar_expect_tx(bar, NARR * BOX_BYTES);
      double* base = sm.box + (size_t)s * NARR * ABOX;
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const int a = C ? l : a0;
        tma_load_2d(base + (3 * l + 0) * ABOX, cur ? &maps.q[a] : &maps.r[a], bx0, by0, bar);
        tma_load_2d(base + (3 * l + 1) * ABOX, &maps.P[cur][a], bx0, by0, bar);
        tma_load_2d(base + (3 * l + 2) * ABOX, &maps.w[cur][a], bx0, by0, bar);
      }
    };

    const int G = gridDim.x;
    int t = blockIdx.x;
    int k = 0;
    unsigned pend = 0;
#pragma unroll
    for (int j = 0; j < NST - 1; ++j) {
      const int tj = t + j * G;
      if (tj < ntask) {
        if (tid == 0) issue(tj, j);
        pend |= 1u << j;
      }
    }
    bool tma_ok = true;
    for (; t < ntask; t += G, ++k) {
      const int s = k % NST;
      {
        const int tn = t + (NST - 1) * G;
        const int sn = (k + NST - 1) % NST;
        if (tn < ntask) {
          if (tid == 0) issue(tn, sn);
          pend |= 1u << sn;
        }
      }
      int a0 = 0, tt = t;
      if (!C) {
        const int w = t / tiles;
        tt = t - w * tiles;
#pragma unroll
        for (int kk = 0; kk < L; ++kk) if (kk == w) a0 = act_list[kk];
      }
      const int x0 = (tt % sp.tiles_x) * TX;
      const int y0 = (tt / sp.tiles_x) * TY;
      const int gx = x0 + lx;
      double te[CPT], tw[CPT], tn[CPT], ts[CPT], pold[CPT], yold[CPT];
      if (!C) {
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int gy = y0 + ly + RPT * j;
          const long long i = (long long)gy * pitch + gx;
          te[j] = tw[j] = tn[j] = ts[j] = pold[j] = yold[j] = 0.0;
          if (gx < nx && gy < ny) {
            te[j] = ldr(sp.tE[a0] + i);
            tn[j] = ldr(sp.tN[a0] + i);
            if (gx > 0) tw[j] = ldr(sp.tE[a0] + i - 1);
            if (gy > 0) ts[j] = ldr(sp.tN[a0] + i - pitch);
            pold[j] = ldc(sp.pd[a0] + i);
            yold[j] = ldc(sp.z[a0] + i);
          }
        }
      }
      if (!mbar_wait(sm.bar + s, (phb >> s) & 1u, sp.spin_limit)) {
        if (tid == 0) raise_abort(sp, (int)MC_E_TIMEOUT);
        tma_ok = false;
        break;
      }
      phb ^= 1u << s;
      pend &= ~(1u << s);
      const double* base = sm.box + (size_t)s * NARR * ABOX;
      // r_{i+1} on the 66 x 18 region of every continuum of the tile
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const int a = C ? l : a0;
        const double al = S.alpha[a], bt = S.beta[a];
        const double* bR = base + (3 * l + 0) * ABOX;
        const double* bS = base + (3 * l + 1) * ABOX;
        const double* bW = base + (3 * l + 2) * ABOX;
        double* pn = sm.pn + l * PN;
        for (int e = tid; e < PN; e += NT) {
          const int ry = e / PX, rx = e - ry * PX;
          const int b = ry * BX + rx + 1;
          const double sn = fma(bt, bS[b], bW[b]);
          pn[e] = fma(-al, sn, bR[b]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int lyj = ly + RPT * j;
        const int gy = y0 + lyj;
        if (gx >= nx || gy >= ny) continue;
        const long long i = (long long)gy * pitch + gx;
        const int c = (lyj + 1) * PX + lx + 1;
        const int b = (lyj + 1) * BX + lx + HOFF;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          const int a = C ? l : a0;
          const double al = S.alpha[a], bt = S.beta[a];
          const double* bR = base + (3 * l + 0) * ABOX;
          const double* bS = base + (3 * l + 1) * ABOX;
          const double* bW = base + (3 * l + 2) * ABOX;
          double cte, ctw, ctn, cts, po, yo;
          if (C) {
            cte = ldr(sp.tE[a] + i);
            ctn = ldr(sp.tN[a] + i);
            ctw = gx > 0 ? ldr(sp.tE[a] + i - 1) : 0.0;
            cts = gy > 0 ? ldr(sp.tN[a] + i - pitch) : 0.0;
            po = ldc(sp.pd[a] + i);
            yo = ldc(sp.z[a] + i);
          } else {
            cte = te[j]; ctw = tw[j]; ctn = tn[j]; cts = ts[j]; po = pold[j]; yo = yold[j];
          }
          const double* pn = sm.pn + l * PN;
          const double sn = fma(bt, bS[b], bW[b]);
          const double rn = pn[c];
          const double pv = fma(bt, po, bR[b]);
          const double yv = fma(al, pv, yo);
          double nb = fma(cte, pn[c + 1], fma(ctw, pn[c - 1], fma(ctn, pn[c + PX], cts * pn[c - PX])));
          if (C) {
#pragma unroll
            for (int bb = 0; bb < L; ++bb) {
              if (bb == a) continue;
              nb = fma(ldr(sp.qs[a][bb] + i), sm.pn[bb * PN + c], nb);
            }
          }
          const double wv = rn - nb;
          (cur ? sp.r[a] : sp.q[a])[i] = rn;
          sp.P[cur ^ 1][a][i] = sn;
          sp.w[cur ^ 1][a][i] = wv;
          sp.pd[a][i] = pv;
          sp.z[a][i] = yv;
#pragma unroll
          for (int kk = 0; kk < L; ++kk)
            if (kk == a) {
              dots[kk] = fma(rn, rn, dots[kk]);
              dots[L + kk] = fma(wv, rn, dots[L + kk]);
              if (chk) {
                const double u = ldr(sp.sqd[a] + i) * rn;
                dots[2 * L + kk] = fma(u, u, dots[2 * L + kk]);
              }
            }
        }
      }
      __syncthreads();
    }
    if (!tma_ok) {
      for (int st = 0; st < NST; ++st)
        if (pend & (1u << st)) mbar_wait(sm.bar + st, (phb >> st) & 1u, 1LL << 24);
      ok = false;
      break;
    }
    const unsigned qm = chk ? qbits(active, L, 3) : qbits(active, L, 2);
    block_store<3 * L>(dots, qm, sm.box, sp.partials, slot);
    if (!grid_sync(sp)) { ok = false; break; }
    grid_totals<3 * L>(sp.partials, slot, sm.res, qm);
    slot ^= 1;
    if (tid == 0) {
      double sg = 0.0, sd = 0.0, sr = 0.0;
      for (int a = 0; a < L; ++a) { sg += sm.res[a]; sd += sm.res[L + a]; sr += sm.res[2 * L + a]; }
      unsigned act = active;
      int bad = 0;
      for (int a = 0; a < L; ++a) {
        const unsigned bit = 1u << a;
        if (!(active & bit)) continue;
        const double gam = C ? sg : sm.res[a];
        const double del = C ? sd : sm.res[L + a];
        if (!isfinite(gam) || !isfinite(del)) { bad = 1; continue; }
        if (it >= 0) S.iters[a] = it + 1;
        if (gam == 0.0) {  // exact solution (tiny grids)
          S.rr[a] = 0.0;
          act &= ~bit;
          continue;
        }
        if (chk) {
          const double rra = C ? sr : sm.res[2 * L + a];
          S.rr[a] = rra;
          if (!(rra > rtol2 * S.bb[a])) { act &= ~bit; continue; }
        }
        if (it < 0) {
          if (!(del > 0.0)) { bad = 1; continue; }
          S.rz[a] = gam;               // gamma of the last pass
          S.rzl[a] = gam / del;        // alpha of the last pass
          S.alpha[a] = S.rzl[a];
          S.beta[a] = 0.0;
          continue;
        }
        const double be = gam / S.rz[a];
        const double den = del - be * gam / S.rzl[a];
        if (!(den > 0.0)) { bad = 1; continue; }
        S.rz[a] = gam;
        S.rzl[a] = gam / den;
        S.alpha[a] = S.rzl[a];
        S.beta[a] = be;
      }
      S.active = act;
      S.flag = bad;
    }
    __syncthreads();
    active = S.active;
    if (S.flag) {
      if (blockIdx.x == 0 && tid == 0) atomicCAS(sp.status, 0, (int)MC_E_BREAKDOWN);
      ok = false;
      break;
    }
    cur ^= 1;
    ++it;
  }
  slot_io = slot;
  return ok;
}

template <int L, bool C, bool SP1>
__device__ bool pcg_solve_scaled(const StepParams& sp, const TmaMaps& maps, unsigned mask, Smem& sm,
                                 uint32_t& phb) {
  if (!scaled_init<L, C>(sp, mask, sm, SP1)) return false;
  int slot = 1;
  bool ok;
  if constexpr (SP1) ok = sp1_loop<L, C>(sp, maps, sm, phb, slot);
  else ok = scaled_loop<L, C>(sp, maps, sm, phb, slot);
  if (ok) return scaled_finish<L, C>(sp, mask, sm, slot);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // keep the iteration counts of the failed solve
    const Scal64& S = *sm.sc;
    for (int a = 0; a < L; ++a) {
      if (!(mask & (1u << a)) || (C && a != 0)) continue;
      sp.iters[a] += S.iters[a];
      if (S.iters[a] > sp.max_iters[a]) sp.max_iters[a] = S.iters[a];
    }
  }
  return false;
}

// MODE 0: Jacobi PCG, flux-form stencil; 1: two-level preconditioner; 2:
// Jacobi PCG in scaled variables, two passes; 3: the same, single pass.
template <int L, bool COUPLED, int MODE>
__global__ void __launch_bounds__(NT, 512 / NT)
    step_kernel(const __grid_constant__ StepParams sp, const __grid_constant__ TmaMaps maps) {
  constexpr int NL = COUPLED ? L : 1;
  constexpr int NARR = (MODE == 3 ? 3 : 2) * NL;
  constexpr int NST = MODE == 3 ? nstage1(L, COUPLED) : nstage(L, COUPLED);
  constexpr int NPN = (MODE == 2 && !COUPLED) ? 2 : 1;  // P_new areas (scaled_loop)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations need 128-B aligned slots: align the dynamic base.
  unsigned char* smem_base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  __shared__ Scal64 s_scal;
  __shared__ double s_cn[9 * MCL];
  Smem sm;
  sm.sc = &s_scal;
  sm.cn = s_cn;
  sm.box = reinterpret_cast<double*>(smem_base);
  sm.pn = sm.box + NST * NARR * ABOX;
  sm.red = sm.pn + NPN * NL * PN;
  sm.res = sm.red + (NT / 32) * KMAX;
  sm.bar = reinterpret_cast<uint64_t*>(sm.res + KMAX);
  if (threadIdx.x == 0) {
    for (int st = 0; st < NST; ++st) mbar_init(sm.bar + st, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phb = 0u;  // parity of the next completion of each stage

  const long long Np = sp.Np;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;

  int done = 0;
  bool ok = true;
  for (int step = 0; step < sp.nsteps && ok; ++step) {
    for (int a = 0; a < L; ++a)
      for (long long i = gtid; i < Np; i += gstride) sp.pprev[a][i] = ldc(sp.p[a] + i);
    if (COUPLED) {
      if (MODE >= 2) ok = pcg_solve_scaled<L, true, MODE == 3>(sp, maps, (1u << L) - 1u, sm, phb);
      else ok = pcg_solve<L, true, MODE == 1>(sp, maps, (1u << L) - 1u, sm, phb);
    } else if (sp.scheme == MC_SCHEME_D) {
      if (MODE >= 2) ok = pcg_solve_scaled<L, false, MODE == 3>(sp, maps, (1u << L) - 1u, sm, phb);
      else ok = pcg_solve<L, false, MODE == 1>(sp, maps, (1u << L) - 1u, sm, phb);
    } else {
      for (int k = 0; k < L && ok; ++k) {
        const int a = sp.scheme == MC_SCHEME_U ? L - 1 - k : k;
        if (MODE >= 2) ok = pcg_solve_scaled<L, false, MODE == 3>(sp, maps, 1u << a, sm, phb);
        else ok = pcg_solve<L, false, MODE == 1>(sp, maps, 1u << a, sm, phb);
      }
    }
    if (ok) ++done;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sp.steps_done = done;
  if (!ok || done == 0) return;

  // ---- mass identity of the last step (Section 3.3, summed equations) ----
  // sum_a m_a dp_a + tau sum_{a<b} q_ab (w_a dp_a + w_b dp_b)
  //   = tau sum (F + W (p_w - p^n)),
  // with (w_a, w_b) = (1,1) D, (0,1) L, (1,0) U, (0,0) coupled; the implicit
  // well term enters every scheme the same way.
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const double wa = (!COUPLED && (sp.scheme == MC_SCHEME_D || sp.scheme == MC_SCHEME_U)) ? 1.0 : 0.0;
  const double wb = (!COUPLED && (sp.scheme == MC_SCHEME_D || sp.scheme == MC_SCHEME_L)) ? 1.0 : 0.0;
  for (long long i = gtid; i < Np; i += gstride) {
    double dp[L];
#pragma unroll
    for (int a = 0; a < L; ++a) {
      dp[a] = ldc(sp.p[a] + i) - ldc(sp.pprev[a] + i);
      const double m = sp.mass[a] * dp[a];
      double f = ldr(sp.F[a] + i);
      if (sp.W[a]) f += ldr(sp.FW[a] + i) - ldr(sp.W[a] + i) * ldc(sp.p[a] + i);
      acc[0] += m;
      acc[1] += f;
      acc[3] += fabs(m) + sp.tau * fabs(f);
    }
#pragma unroll
    for (int a = 0; a < L; ++a)
#pragma unroll
      for (int b = a + 1; b < L; ++b) {
        const double e = qab(sp, a, b, i) * (wa * dp[a] + wb * dp[b]);
        acc[2] += e;
        acc[3] += sp.tau * fabs(e);
      }
  }
  block_store<4>(acc, 0xfu, sm.box, sp.partials, 0);
  if (!grid_sync(sp)) return;
  double t[4];
  grid_sum<4>(sp.partials, 0, sm.res, t);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double num = t[0] + sp.tau * t[2] - sp.tau * t[1];
    *sp.mass_defect = fabs(num) / fmax(t[3], 1e-300);
  }
}

template <int L, bool C, int M>
constexpr size_t smem_bytes() {
  constexpr int NL = C ? L : 1;
  constexpr int NST = M == 3 ? nstage1(L, C) : nstage(L, C);
  constexpr int NB = M == 3 ? 3 : 2;
  constexpr int NPN = (M == 2 && !C) ? 2 : 1;
  return (size_t)(NST * NB * NL * ABOX + NPN * NL * PN + (NT / 32) * KMAX + KMAX) * sizeof(double) +
         NST * sizeof(uint64_t) + 128;
}

struct KInfo {
  void* fn;
  size_t smem;
};

// Each variant (flux-form Jacobi, two-level, scaled Jacobi, coupled) is a
// separate instantiation, so that no kernel carries another's code.
template <int L, bool C, int M>
KInfo info() {
  return KInfo{(void*)step_kernel<L, C, M>, smem_bytes<L, C, M>()};
}

template <int L>
KInfo pick_l(bool coupled, int mode) {
  if (coupled) {
    switch (mode) {
      case 1: return info<L, true, 1>();
      case 2: return info<L, true, 2>();
      case 3: return info<L, true, 3>();
      default: return info<L, true, 0>();
    }
  }
  switch (mode) {
    case 1: return info<L, false, 1>();
    case 2: return info<L, false, 2>();
    case 3: return info<L, false, 3>();
    default: return info<L, false, 0>();
  }
}

// mode: 0 flux-form Jacobi, 1 two-level, 2 scaled Jacobi
// (two phases, two reductions per iteration), 3 scaled Jacobi single-pass
KInfo pick(int L, bool coupled, int mode = 0) {
  switch (L) {
    case 1: return pick_l<1>(coupled, mode);
    case 2: return pick_l<2>(coupled, mode);
    case 3: return pick_l<3>(coupled, mode);
    default: return pick_l<4>(coupled, mode);
  }
}

int max_blocks_for(KInfo k, int threads, int num_sms) {
  if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, threads, k.smem) != cudaSuccess) return 0;
  return per_sm * num_sms;
}

// A_c = P^T (M/tau + A0)_a P on the tile grid: one thread per coarse row I
// sums diag(A0 - D) over the tile and the face transmissibilities across each
// tile side; the off-diagonal entry to a neighbouring tile is minus that side's
// sum (the same faces in the same order from both sides, so A_c is exactly
// symmetric). Ac must be zero on entry.
__global__ void coarse_assemble_kernel(int nx, int ny, int pitch, int tiles_x, int tiles_y,
                                       const double* TE, const double* TN, const double* diagc,
                                       double diagc_const, double* Ac, long long ld) {
  const int nc = tiles_x * tiles_y;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    const int x0 = (I % tiles_x) * TX, y0 = (I / tiles_x) * TY;
    const int x1 = min(x0 + TX, nx), y1 = min(y0 + TY, ny);
    double d = 0.0, te = 0.0, tw = 0.0, tn = 0.0, ts = 0.0;
    for (int y = y0; y < y1; ++y)
      for (int x = x0; x < x1; ++x) d += diagc ? diagc[(long long)y * pitch + x] : diagc_const;
    for (int y = y0; y < y1; ++y) {
      if (x1 < nx) te += TE[(long long)y * pitch + x1 - 1];
      if (x0 > 0) tw += TE[(long long)y * pitch + x0 - 1];
    }
    for (int x = x0; x < x1; ++x) {
      if (y1 < ny) tn += TN[(long long)(y1 - 1) * pitch + x];
      if (y0 > 0) ts += TN[(long long)(y0 - 1) * pitch + x];
    }
    double* row = Ac + (long long)I * ld;
    row[I] = d + te + tw + tn + ts;
    if (x1 < nx) row[I + 1] = -te;
    if (x0 > 0) row[I - 1] = -tw;
    if (y1 < ny) row[I + tiles_x] = -tn;
    if (y0 > 0) row[I - tiles_x] = -ts;
  }
}

// Exchange blocks of the coupled Galerkin coarse operator P^T A P, P =
// blockdiag(P_a): entry ((a, I), (b, I)) = -(sum over the cells of tile I of
// q_ab), the same cells in the same order for (a, b) and (b, a), so the
// operator stays exactly symmetric. The diagonal blocks already carry +sum_b
// q_ab through diagc. Ac holds the (L nc)^2 matrix, row stride ld.
struct ExchArgs {
  const double* qcell[MCL][MCL];
  double qconst[MCL][MCL];
};

__global__ void coarse_exchange_kernel(int nx, int ny, int pitch, int tiles_x, int nc, int L,
                                       const __grid_constant__ ExchArgs q, double* Ac, long long ld) {
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    const int x0 = (I % tiles_x) * TX, y0 = (I / tiles_x) * TY;
    const int x1 = min(x0 + TX, nx), y1 = min(y0 + TY, ny);
    for (int a = 0; a < L; ++a)
      for (int b = a + 1; b < L; ++b) {
        const double* qc = q.qcell[a][b];
        double sq = 0.0;
        for (int y = y0; y < y1; ++y)
          for (int x = x0; x < x1; ++x) sq += qc ? qc[(long long)y * pitch + x] : q.qconst[a][b];
        Ac[((long long)a * nc + I) * ld + (long long)b * nc + I] = -sq;
        Ac[((long long)b * nc + I) * ld + (long long)a * nc + I] = -sq;
      }
  }
}

}  // namespace

int mc_step_tiles(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }

cudaError_t mc_launch_coarse_assemble(const mc_ctx* ctx, int a, double* Ac) {
  const int tx = (ctx->nx + TX - 1) / TX, ty = (ctx->ny + TY - 1) / TY;
  const long long nc = (long long)tx * ty;
  cudaError_t e = cudaMemsetAsync(Ac, 0, (size_t)(nc * nc) * sizeof(double), ctx->stream);
  if (e != cudaSuccess) return e;
  double dconst = ctx->c[a] * ctx->h * ctx->h / ctx->tau;
  for (int b = 0; b < ctx->L; ++b)
    if (b != a) dconst += ctx->sigma[a][b] * ctx->h * ctx->h;
  const int blocks = (int)((nc + 127) / 128);
  coarse_assemble_kernel<<<blocks, 128, 0, ctx->stream>>>(ctx->nx, ctx->ny, ctx->pitch, tx, ty,
                                                          ctx->TE[a], ctx->TN[a], ctx->diagc[a],
                                                          dconst, Ac, nc);
  return cudaGetLastError();
}

cudaError_t mc_launch_coarse_assemble_coupled(const mc_ctx* ctx, double* Ac) {
  const int tx = (ctx->nx + TX - 1) / TX, ty = (ctx->ny + TY - 1) / TY;
  const long long nc = (long long)tx * ty;
  const long long n = (long long)ctx->L * nc;
  cudaError_t e = cudaMemsetAsync(Ac, 0, (size_t)(n * n) * sizeof(double), ctx->stream);
  if (e != cudaSuccess) return e;
  const int blocks = (int)((nc + 127) / 128);
  ExchArgs q{};
  for (int a = 0; a < ctx->L; ++a) {
    double dconst = ctx->c[a] * ctx->h * ctx->h / ctx->tau;
    for (int b = 0; b < ctx->L; ++b) {
      if (b != a) dconst += ctx->sigma[a][b] * ctx->h * ctx->h;
      q.qcell[a][b] = ctx->qcell[a][b];
      q.qconst[a][b] = ctx->sigma[a][b] * ctx->h * ctx->h;
    }
    coarse_assemble_kernel<<<blocks, 128, 0, ctx->stream>>>(ctx->nx, ctx->ny, ctx->pitch, tx, ty,
                                                            ctx->TE[a], ctx->TN[a], ctx->diagc[a], dconst,
                                                            Ac + (a * nc) * n + a * nc, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  coarse_exchange_kernel<<<blocks, 128, 0, ctx->stream>>>(ctx->nx, ctx->ny, ctx->pitch, tx, (int)nc, ctx->L, q,
                                                          Ac, n);
  return cudaGetLastError();
}

int mc_step_max_blocks(int L, int threads, int num_sms) {
  int m = max_blocks_for(pick(L, true), threads, num_sms);
  for (int mode = 1; mode < 4; ++mode) {
    const int c = max_blocks_for(pick(L, true, mode), threads, num_sms);
    if (c < m) m = c;
  }
  for (int mode = 0; mode < 4; ++mode) {
    const int a = max_blocks_for(pick(L, false, mode), threads, num_sms);
    if (a < m) m = a;
  }
  return m;
}

// Co-resident CTAs of the kernel that a launch with these parameters runs.
int mc_step_blocks_for(const StepParams& sp, int threads, int num_sms) {
  const int mode = sp.two_level ? 1 : (sp.sqd[0] == nullptr ? 0 : (sp.single_pass ? 3 : 2));
  return max_blocks_for(pick(sp.L, sp.scheme == MC_SCHEME_COUPLED, mode), threads, num_sms);
}

// The largest co-resident count over every step kernel of L continua.
int mc_step_max_blocks_any(int L, int threads, int num_sms) {
  int m = 0;
  for (int mode = 0; mode < 4; ++mode)
    for (int c = 0; c < 2; ++c) {
      const int v = max_blocks_for(pick(L, c != 0, mode), threads, num_sms);
      if (v > m) m = v;
    }
  return m;
}

int mc_step_box_x() { return BX; }
int mc_step_box_y() { return BY; }

cudaError_t mc_launch_steps_raw(const StepParams& sp_in, const TmaMaps& maps_in, int blocks,
                                int threads, cudaStream_t stream) {
  StepParams sp = sp_in;
  TmaMaps maps = maps_in;
  sp.tiles_x = (sp.nx + TX - 1) / TX;
  sp.tiles_y = (sp.ny + TY - 1) / TY;
  const int mode = sp.two_level ? 1 : (sp.sqd[0] == nullptr ? 0 : (sp.single_pass ? 3 : 2));
  KInfo k = pick(sp.L, sp.scheme == MC_SCHEME_COUPLED, mode);
  cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&sp, &maps};
  return cudaLaunchCooperativeKernel(k.fn, dim3(blocks), dim3(threads), args, k.smem, stream);
}

cudaError_t mc_launch_steps(mc_ctx* ctx, const StepParams& sp, int blocks, int threads) {
  return mc_launch_steps_raw(sp, ctx->maps, blocks, threads, ctx->stream);
}
