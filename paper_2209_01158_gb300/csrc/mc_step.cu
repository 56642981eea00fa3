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
// Layout: every field is nx*ny doubles, cell (i, j) at j*nx + i. TE holds the
// east-face transmissibility (0 on the last column), TN the north face (0 on
// the last row). The PCG warm-starts from p^{n-1} and updates p in place.
//
// Cross-CTA data written inside the launch (r, P, q, p, partial sums) is read
// with ld.global.cg so no SM serves it from a stale L1 line; read-only
// coefficients go through the read-only path. Reductions are deterministic:
// warp butterflies, then a fixed-order sum over warps and over CTAs.

#include <math.h>

#include "mc_internal.h"

namespace {

constexpr int TX = 64;   // stencil tile width (cells along x)
constexpr int TY = 8;    // stencil tile height
constexpr int HX = TX + 2;
constexpr int HY = TY + 2;
constexpr int NT = 512;  // threads per CTA (launch bound)
constexpr int KMAX = 4 * MCL;  // partial-sum quantities per slot

__device__ __forceinline__ double ldc(const double* p) { return __ldcg(p); }
__device__ __forceinline__ double ldr(const double* p) { return __ldg(p); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid-wide barrier for a cooperative launch. Every wait is bounded by
// spin_limit polls; a CTA that gives up raises the abort word and the status
// MC_E_TIMEOUT, and every CTA that sees the abort word leaves the kernel.
__device__ bool grid_sync(const StepParams& sp) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned* count = sp.bar_count;
    unsigned* gen = sp.bar_gen;
    unsigned* abort_word = sp.bar_gen + 32;
    unsigned g = ld_acquire(gen);
    __threadfence();
    unsigned arrived = atomicAdd(count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      long long n = 0;
      while (ld_acquire(gen) == g) {
        if (ld_acquire(abort_word) != 0u) { ok = 0; break; }
        if (++n > sp.spin_limit) {
          atomicExch(abort_word, 1u);
          atomicCAS(sp.status, 0, (int)MC_E_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (ok && ld_acquire(abort_word) != 0u) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block-reduce NQ values and store them as this CTA's partials:
// partials[slot][k][blockIdx.x], KMAX quantities reserved per slot so the
// two alternating slots never overlap whatever NQ each phase uses.
template <int NQ>
__device__ void block_store(double (&v)[NQ], double* s_red, double* partials, int slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) s_red[warp * NQ + k] = s;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += s_red[w * NQ + threadIdx.x];
    partials[((size_t)slot * KMAX + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
  __syncthreads();
}

// Sum the NQ partials over all CTAs in a fixed order; every thread gets them.
template <int NQ>
__device__ void grid_sum(const double* partials, int slot, double* s_res, double (&out)[NQ]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int k = warp; k < NQ; k += nw) {
    const double* src = partials + ((size_t)slot * KMAX + k) * nb;
    double s = 0.0;
#pragma unroll 4
    for (int b = lane; b < nb; b += 32) s += ldc(src + b);
    s = warp_sum(s);
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
  const int nx = sp.nx;
  double s = 0.0;
  const double te = ldr(sp.TE[a] + i);
  const double tn = ldr(sp.TN[a] + i);
  if (gx + 1 < nx) s += te * (xc - ldc(x + i + 1));
  if (gx > 0) s += ldr(sp.TE[a] + i - 1) * (xc - ldc(x + i - 1));
  if (gy + 1 < sp.ny) s += tn * (xc - ldc(x + i + nx));
  if (gy > 0) s += ldr(sp.TN[a] + i - nx) * (xc - ldc(x + i - nx));
  return s;
}

// ---------------------------------------------------------------------------
// One linear solve: the continua in `mask` (decoupled, independent systems),
// or all L continua as one coupled system. Warm start from p, result in p.
// Returns false when the run must stop (timeout, breakdown, no convergence).
template <int L, bool COUPLED>
__device__ bool pcg_solve(const StepParams& sp, unsigned mask, double* s_tile,
                          double* s_red, double* s_res) {
  const long long N = sp.N;
  const int nx = sp.nx;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;

  // ---- fused right-hand side + initial residual (slot 0: bb, rr, rz) -----
  double acc[3 * L];
#pragma unroll
  for (int k = 0; k < 3 * L; ++k) acc[k] = 0.0;
#pragma unroll
  for (int a = 0; a < L; ++a) {
    if (!(mask & (1u << a))) continue;
    const double* pa = sp.p[a];
    for (long long i = gtid; i < N; i += gstride) {
      const int gx = (int)(i % nx), gy = (int)(i / nx);
      const double xc = ldc(pa + i);
      const double f = ldr(sp.F[a] + i);
      double ex = 0.0, exb = 0.0;
#pragma unroll
      for (int b = 0; b < L; ++b) {
        if (b == a) continue;
        const double qv = qab(sp, a, b, i);
        const double pb = ldc(sp.p[b] + i);
        ex += qv * (pb - xc);
        exb += qv * pb;
      }
      const double rv = f + ex - stencil_flux(sp, a, pa, gx, gy, i, xc);
      const double bv = COUPLED ? sp.mtau[a] * xc + f : sp.mtau[a] * xc + f + exb;
      const double z = ldr(sp.invd[a] + i) * rv;
      sp.r[a][i] = rv;
      sp.P[0][a][i] = z;
      acc[0 * L + a] += bv * bv;
      acc[1 * L + a] += rv * rv;
      acc[2 * L + a] += rv * z;
    }
  }
  block_store<3 * L>(acc, s_red, sp.partials, 0);
  if (!grid_sync(sp)) return false;
  double tot[3 * L];
  grid_sum<3 * L>(sp.partials, 0, s_res, tot);

  double bb[L], rr[L], rz[L], beta[L];
#pragma unroll
  for (int a = 0; a < L; ++a) {
    bb[a] = tot[a];
    rr[a] = tot[L + a];
    rz[a] = tot[2 * L + a];
    beta[a] = 0.0;
  }
  if (COUPLED) {
    double sb = 0, sr = 0, sz = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (mask & (1u << a)) { sb += bb[a]; sr += rr[a]; sz += rz[a]; }
    }
#pragma unroll
    for (int a = 0; a < L; ++a) { bb[a] = sb; rr[a] = sr; rz[a] = sz; }
  }
  const double rtol2 = sp.rtol * sp.rtol;
  unsigned active = 0;
#pragma unroll
  for (int a = 0; a < L; ++a) {
    if ((mask & (1u << a)) && rr[a] > rtol2 * bb[a]) active |= 1u << a;
  }
  int it = 0;
  int cur = 0;
  int slot = 1;
  bool ok = true;
  int my_iters[L];
#pragma unroll
  for (int a = 0; a < L; ++a) my_iters[a] = 0;

  const int tiles = sp.tiles_x * sp.tiles_y;
  while (active) {
    if (it >= sp.max_iter) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(sp.status, 0, (int)MC_E_NOCONV);
      ok = false;
      break;
    }
    // ---- phase A: P_new = z + beta P_old on a halo tile, q = A P_new ------
    int act_list[L];
    int nact = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) if (active & (1u << a)) act_list[nact++] = a;
    double pq[L];
#pragma unroll
    for (int a = 0; a < L; ++a) pq[a] = 0.0;
    const int ntask = COUPLED ? tiles : nact * tiles;
    for (int t = blockIdx.x; t < ntask; t += gridDim.x) {
      int a0 = 0, tt = t;
      if (!COUPLED) {
        const int w = t / tiles;
        tt = t - w * tiles;
#pragma unroll
        for (int k = 0; k < L; ++k) if (k == w) a0 = act_list[k];
      }
      const int x0 = (tt % sp.tiles_x) * TX;
      const int y0 = (tt / sp.tiles_x) * TY;
      constexpr int NL = COUPLED ? L : 1;
#pragma unroll
      for (int l = 0; l < NL; ++l) {
        const int a = COUPLED ? l : a0;
        const double* r = sp.r[a];
        const double* Po = sp.P[cur][a];
        const double* iv = sp.invd[a];
        const double bt = beta[a];
        double* st = s_tile + l * HX * HY;
        for (int e = threadIdx.x; e < HX * HY; e += blockDim.x) {
          const int ly = e / HX, lx = e - ly * HX;
          const int gx = x0 + lx - 1, gy = y0 + ly - 1;
          double v = 0.0;
          if (gx >= 0 && gx < nx && gy >= 0 && gy < sp.ny) {
            const long long i = (long long)gy * nx + gx;
            v = ldr(iv + i) * ldc(r + i) + bt * ldc(Po + i);
          }
          st[e] = v;
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < TX * TY; e += blockDim.x) {
        const int ly = e / TX, lx = e - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= sp.ny) continue;
        const long long i = (long long)gy * nx + gx;
        const int c = (ly + 1) * HX + lx + 1;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          const int a = COUPLED ? l : a0;
          const double* st = s_tile + l * HX * HY;
          const double pc = st[c];
          const double te = ldr(sp.TE[a] + i);
          const double tn = ldr(sp.TN[a] + i);
          const double tw = gx > 0 ? ldr(sp.TE[a] + i - 1) : 0.0;
          const double ts = gy > 0 ? ldr(sp.TN[a] + i - nx) : 0.0;
          double qv = diagc(sp, a, i) * pc + te * (pc - st[c + 1]) + tw * (pc - st[c - 1]) +
                      tn * (pc - st[c + HX]) + ts * (pc - st[c - HX]);
          if (COUPLED) {
#pragma unroll
            for (int b = 0; b < L; ++b) {
              if (b == a) continue;
              qv -= qab(sp, a, b, i) * s_tile[b * HX * HY + c];
            }
          }
          sp.P[cur ^ 1][a][i] = pc;
          sp.q[a][i] = qv;
#pragma unroll
          for (int k = 0; k < L; ++k) if (k == a) pq[k] += pc * qv;
        }
      }
      __syncthreads();
    }
    block_store<L>(pq, s_red, sp.partials, slot);
    if (!grid_sync(sp)) { ok = false; break; }
    double pqt[L];
    grid_sum<L>(sp.partials, slot, s_res, pqt);
    slot ^= 1;
    if (COUPLED) {
      double s = 0;
#pragma unroll
      for (int a = 0; a < L; ++a) s += pqt[a];
#pragma unroll
      for (int a = 0; a < L; ++a) pqt[a] = s;
    }
    double alpha[L];
    bool brk = false;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      alpha[a] = 0.0;
      if (active & (1u << a)) {
        if (!(pqt[a] > 0.0) || !isfinite(pqt[a])) brk = true;
        else alpha[a] = rz[a] / pqt[a];
      }
    }
    if (brk) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(sp.status, 0, (int)MC_E_BREAKDOWN);
      ok = false;
      break;
    }
    // ---- phase B: x += alpha P, r -= alpha q, z = invd r (slot: rr, rz) ----
    double acc2[2 * L];
#pragma unroll
    for (int k = 0; k < 2 * L; ++k) acc2[k] = 0.0;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(active & (1u << a))) continue;
      const double al = alpha[a];
      double* x = sp.p[a];
      double* r = sp.r[a];
      const double* Pn = sp.P[cur ^ 1][a];
      const double* qq = sp.q[a];
      const double* iv = sp.invd[a];
      for (long long i = gtid; i < N; i += gstride) {
        const double rv = ldc(r + i) - al * ldc(qq + i);
        x[i] = ldc(x + i) + al * ldc(Pn + i);
        r[i] = rv;
        acc2[a] += rv * rv;
        acc2[L + a] += rv * (ldr(iv + i) * rv);
      }
    }
    block_store<2 * L>(acc2, s_red, sp.partials, slot);
    if (!grid_sync(sp)) { ok = false; break; }
    double t2[2 * L];
    grid_sum<2 * L>(sp.partials, slot, s_res, t2);
    slot ^= 1;
    if (COUPLED) {
      double s0 = 0, s1 = 0;
#pragma unroll
      for (int a = 0; a < L; ++a) { s0 += t2[a]; s1 += t2[L + a]; }
#pragma unroll
      for (int a = 0; a < L; ++a) { t2[a] = s0; t2[L + a] = s1; }
    }
    ++it;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(active & (1u << a))) continue;
      rr[a] = t2[a];
      const double rzn = t2[L + a];
      beta[a] = rzn / rz[a];
      rz[a] = rzn;
      my_iters[a] = it;
      if (!(rr[a] > rtol2 * bb[a])) active &= ~(1u << a);
      if (!isfinite(rr[a])) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(sp.status, 0, (int)MC_E_BREAKDOWN);
        ok = false;
      }
    }
    if (!ok) break;
    cur ^= 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(mask & (1u << a))) continue;
      const int ka = COUPLED ? 0 : a;
      if (COUPLED && a != 0) continue;
      sp.iters[ka] += my_iters[a];
      if (my_iters[a] > sp.max_iters[ka]) sp.max_iters[ka] = my_iters[a];
      sp.relres[ka] = bb[a] > 0 ? sqrt(rr[a] / bb[a]) : sqrt(rr[a]);
    }
  }
  // The next solve reads p of this one's continua: make p visible to all.
  if (ok && !grid_sync(sp)) ok = false;
  return ok;
}

template <int L, bool COUPLED>
__global__ void __launch_bounds__(NT, 1) step_kernel(StepParams sp) {
  constexpr int NL = COUPLED ? L : 1;
  __shared__ double s_tile[NL * HX * HY];
  __shared__ double s_red[(NT / 32) * KMAX];
  __shared__ double s_res[KMAX];
  const long long N = sp.N;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;

  int done = 0;
  bool ok = true;
  for (int step = 0; step < sp.nsteps && ok; ++step) {
    for (int a = 0; a < L; ++a)
      for (long long i = gtid; i < N; i += gstride) sp.pprev[a][i] = ldc(sp.p[a] + i);
    if (COUPLED) {
      ok = pcg_solve<L, true>(sp, (1u << L) - 1u, s_tile, s_red, s_res);
    } else if (sp.scheme == MC_SCHEME_D) {
      ok = pcg_solve<L, false>(sp, (1u << L) - 1u, s_tile, s_red, s_res);
    } else {
      for (int k = 0; k < L && ok; ++k) {
        const int a = sp.scheme == MC_SCHEME_U ? L - 1 - k : k;
        ok = pcg_solve<L, false>(sp, 1u << a, s_tile, s_red, s_res);
      }
    }
    if (ok) ++done;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sp.steps_done = done;
  if (!ok || done == 0) return;

  // ---- mass identity of the last step (Section 3.3, summed equations) ----
  // sum_a m_a dp_a + tau sum_{a<b} q_ab (w_a dp_a + w_b dp_b) = tau sum F,
  // with (w_a, w_b) = (1,1) D, (0,1) L, (1,0) U, (0,0) coupled.
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const double wa = (!COUPLED && (sp.scheme == MC_SCHEME_D || sp.scheme == MC_SCHEME_U)) ? 1.0 : 0.0;
  const double wb = (!COUPLED && (sp.scheme == MC_SCHEME_D || sp.scheme == MC_SCHEME_L)) ? 1.0 : 0.0;
  for (long long i = gtid; i < N; i += gstride) {
    double dp[L];
#pragma unroll
    for (int a = 0; a < L; ++a) {
      dp[a] = ldc(sp.p[a] + i) - ldc(sp.pprev[a] + i);
      const double m = sp.mass[a] * dp[a];
      const double f = ldr(sp.F[a] + i);
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
  block_store<4>(acc, s_red, sp.partials, 0);
  if (!grid_sync(sp)) return;
  double t[4];
  grid_sum<4>(sp.partials, 0, s_res, t);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double num = t[0] + sp.tau * t[2] - sp.tau * t[1];
    *sp.mass_defect = fabs(num) / fmax(t[3], 1e-300);
  }
}

template <int L, bool C>
void* kernel_ptr() { return (void*)step_kernel<L, C>; }

void* pick(int L, bool coupled) {
  switch (L) {
    case 1: return coupled ? kernel_ptr<1, true>() : kernel_ptr<1, false>();
    case 2: return coupled ? kernel_ptr<2, true>() : kernel_ptr<2, false>();
    case 3: return coupled ? kernel_ptr<3, true>() : kernel_ptr<3, false>();
    default: return coupled ? kernel_ptr<4, true>() : kernel_ptr<4, false>();
  }
}

}  // namespace

int mc_step_max_blocks(int L, int threads, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick(L, false), threads, 0) != cudaSuccess)
    return 0;
  int per_sm_c = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_c, pick(L, true), threads, 0) != cudaSuccess)
    return 0;
  return (per_sm < per_sm_c ? per_sm : per_sm_c) * num_sms;
}

cudaError_t mc_launch_steps(mc_ctx* ctx, const StepParams& sp_in, int blocks, int threads) {
  StepParams sp = sp_in;
  sp.tiles_x = (sp.nx + TX - 1) / TX;
  sp.tiles_y = (sp.ny + TY - 1) / TY;
  void* fn = pick(sp.L, sp.scheme == MC_SCHEME_COUPLED);
  void* args[] = {&sp};
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, 0, ctx->stream);
}
