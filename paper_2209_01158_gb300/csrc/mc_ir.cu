// Precision form of the decoupled step: FP32 inner PCG inside FP64 iterative
// refinement, one persistent cooperative launch per call.
//
// Each continuum's system of the D-, L- or U-scheme (Section 3.3)
//   (M_a/tau + D_a + sum_b Q_ab) x = b
// is solved by refinement sweeps:
//   1. FP64 residual, flux form, every term a difference of nearby values:
//        r = F + m/tau (p^{n-1} - x) + sum_b q_ab (p_b - x) - D x
//   2. constant-mode deflation: the exact solution satisfies 1^T r = 0
//      (1^T D = 0), so x += c, r -= c diag(A0 - D) with
//      c = 1^T r / 1^T diag(A0 - D); the FP32 solve cannot resolve this
//      near-null mode, the FP64 shift does;
//   3. stop when ||r|| <= rtol ||b|| (FP64), or when refinement has reached
//      its floor: the last inner solve met its own target but the sweep did
//      not halve ||r|| (the rule LAPACK's refinement uses: stop once the
//      backward error no longer halves), with ||r|| already within
//      1e3 rtol ||b|| or the last correction below 100 rtol ||x||. On
//      fracture continua (k 1e4 on thin networks, 1e-2
//      around them) FP32-corrected refinement levels off near 1e-11 ||b||
//      while the error is ~1e-13: the FP32 corrections carry large
//      near-null components that the operator maps to small residuals;
//   4. FP32 PCG on A d = r (transmissibilities stored FP32 or BF16, FP32
//      vectors, Jacobi), to a relative residual inner_rtol; the dot products
//      are summed per thread in FP32 and then across the grid in FP64;
//   5. x += d in FP64.
// The inner PCG runs in one of two forms (mc_opts.inner_form): the default
// single-reduction recurrences (`inner_single`: one tile pass and one grid
// reduction per iteration, halo values recomputed from double-buffered
// vectors), or the two-reduction textbook recurrences with the structure of
// the FP64 kernel (TMA halo tiles of r, P_old and invd in a shared-memory
// ring, then a pointwise vector phase), with 4-byte data.

#include <cuda_bf16.h>
#include <math.h>

#include "mc_internal.h"
#include "mc_sync.cuh"
#include "mc_tma.h"

namespace {

constexpr int TX = 64, TY = 16;
constexpr int HOFF = 4;                 // 16 B of floats left of the tile
constexpr int BX = TX + 2 * HOFF;       // 72 floats, 288 B rows
constexpr int BY = TY + 2;
constexpr int ABOX = 1312;              // floats per box slot (5248 B, 128-B multiple)
constexpr uint32_t BOX_BYTES = BX * BY * 4;
constexpr int PX = TX + 2, PN = PX * BY;
// Two 256-thread CTAs per SM, each with its own CTA barriers and a 4-stage
// ring, so that one computes while the other waits (the same split as the
// FP64 step kernels). Measured on the two-continuum 4096^2 precision step:
// 5.75 s against 7.27 s with one 512-thread CTA per SM and a 6-stage ring.
constexpr int NT = 256;
constexpr int RPT = NT / TX;            // 4 tile rows per pass of the CTA
constexpr int CPT = TY / RPT;           // 4 own cells per thread
constexpr int NST = 4;
constexpr int NBOX = 4;                 // box slots per ring stage (3 used by the two-reduction form)
constexpr int KM = MC_KMAX_ALLOC;

__device__ __forceinline__ float tload(const float* p, long long i) { return __ldg(p + i); }

// The face transmissibilities of this lane's cell (gx, gy): east te = TE[i],
// west tw = TE[i - 1], north tn = TN[i], south ts = TN[i - pitch] (0 where
// the face does not exist). All 32 lanes of the warp call it, for the 32
// consecutive cells gx = x0w + lane of one row (x0w a multiple of 32); cells
// outside the grid get 0 and load nothing.
__device__ __forceinline__ void tfaces(const float* TE, const float* TN, long long i, int gx, int gy, int nx,
                                       int ny, int pitch, float& te, float& tw, float& tn, float& ts) {
  te = tw = tn = ts = 0.f;
  if (gx < nx && gy < ny) {
    te = tload(TE, i);
    tn = tload(TN, i);
    if (gx > 0) tw = tload(TE, i - 1);
    if (gy > 0) ts = tload(TN, i - pitch);
  }
}

// BF16: the row's values are read as 32-bit words (two BF16 each, rows start
// on 32-byte boundaries since the pitch is a multiple of 16) and handed out by
// warp shuffles. TE: lanes 0..16 read the 17 words covering columns
// x0w - 2 .. x0w + 31, which hold every lane's east and west face. TN: lanes
// 0..15 read the 16 words of row gy, lanes 16..31 those of row gy - 1. Two
// loads per row instead of four; a word that lies outside the grid's rows or
// the array is not read (0). The values are exactly those of the scalar loads.
__device__ __forceinline__ float bf16_half(unsigned w, int hi) {
  return __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
}
__device__ __forceinline__ void tfaces(const __nv_bfloat16* TE, const __nv_bfloat16* TN, long long i, int gx,
                                       int gy, int nx, int ny, int pitch, float& te, float& tw, float& tn,
                                       float& ts) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int x0w = gx - lane;
  const long long row = i - gx;  // gy * pitch
  const unsigned* E = reinterpret_cast<const unsigned*>(TE);
  const unsigned* Nn = reinterpret_cast<const unsigned*>(TN);
  unsigned we = 0u, wn = 0u;
  {
    const int c = x0w - 2 + 2 * lane;  // first column of this lane's TE word
    if (lane <= 16 && gy < ny && c >= 0 && c + 1 < pitch) we = __ldg(E + ((row + c) >> 1));
  }
  {
    const int k = lane & 15;
    const int c = x0w + 2 * k;
    const int r = lane < 16 ? gy : gy - 1;
    if (r >= 0 && r < ny && c + 1 < pitch) wn = __ldg(Nn + (((long long)r * pitch + c) >> 1));
  }
  const unsigned e1 = __shfl_sync(full, we, (lane + 2) >> 1);
  const unsigned e0 = __shfl_sync(full, we, (lane + 1) >> 1);
  const unsigned n1 = __shfl_sync(full, wn, lane >> 1);
  const unsigned n0 = __shfl_sync(full, wn, 16 + (lane >> 1));
  te = tw = tn = ts = 0.f;
  if (gx < nx && gy < ny) {
    te = bf16_half(e1, lane & 1);
    tn = bf16_half(n1, lane & 1);
    if (gx > 0) tw = bf16_half(e0, (lane + 1) & 1);
    if (gy > 0) ts = bf16_half(n0, lane & 1);
  }
}

// The CTAs that cooperate on one solve: the whole grid, or one team of the
// batched kernel. rank/size replace blockIdx.x/gridDim.x everywhere below.
struct Team {
  int rank, size;
};

__device__ __forceinline__ GridBar irbar(const IrParams& ip, const Team& tm) {
  const StepParams& sp = ip.sp;
  GridBar g;
  g.count = reinterpret_cast<unsigned long long*>(sp.bar_count);
  g.abort_word = ip.abort_word;
  g.status = sp.status;
  g.spin_limit = sp.spin_limit;
  g.nparts = (unsigned)tm.size;
  return g;
}

__device__ __forceinline__ bool gsync(const IrParams& ip, const Team& tm) {
  const bool ok = grid_barrier(irbar(ip, tm));
  if (threadIdx.x == 0) fence_proxy_async();
  return ok;
}

// CTA reductions through the (idle) TMA box area of shared memory: FP64 for
// the refinement passes, FP32 within warps (then FP64) for the inner PCG.
template <int NQ>
__device__ __forceinline__ void store_part(const double (&v)[NQ], unsigned qmask, float* box,
                                           double* partials, int slot, const Team& tm) {
  cta_reduce_store<NQ, NT, KM, double>(v, qmask, reinterpret_cast<double*>(box), partials, slot,
                                       tm.size, tm.rank);
}

template <int NQ>
__device__ __forceinline__ void store_part_f(const float (&v)[NQ], unsigned qmask, float* box,
                                             double* partials, int slot, const Team& tm) {
  cta_reduce_store<NQ, NT, KM, float>(v, qmask, box, partials, slot, tm.size, tm.rank);
}

// Grid totals of NQ quantities into s_res (shared); all threads may read
// s_res after the call.
template <int NQ>
__device__ void sum_totals(const double* partials, int slot, double* s_res, const Team& tm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = tm.size;
  for (int k = warp; k < NQ; k += NT / 32) {
    const double* src = partials + ((size_t)slot * KM + k) * nb;
    double s = 0.0;
#pragma unroll 4
    for (int b = lane; b < nb; b += 32) s += __ldcg(src + b);
    s = warp_sum_d(s);
    if (lane == 0) s_res[k] = s;
  }
  __syncthreads();
}

template <int NQ>
__device__ void sum_part(const double* partials, int slot, double* s_res, double (&out)[NQ],
                         const Team& tm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = tm.size;
  for (int k = warp; k < NQ; k += NT / 32) {
    const double* src = partials + ((size_t)slot * KM + k) * nb;
    double s = 0.0;
#pragma unroll 4
    for (int b = lane; b < nb; b += 32) s += __ldcg(src + b);
    s = warp_sum_d(s);
    if (lane == 0) s_res[k] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NQ; ++k) out[k] = s_res[k];
  __syncthreads();
}

__device__ __forceinline__ double qab(const StepParams& sp, int a, int b, long long i) {
  const double* c = sp.qcell[a][b];
  return c ? __ldg(c + i) : sp.qconst[a][b];
}

__device__ __forceinline__ double dcell(const StepParams& sp, int a, long long i) {
  const double* d = sp.diagc[a];
  return d ? __ldg(d + i) : sp.diagc_const[a];
}

// Per-continuum scalars of the inner PCG, kept in shared memory and updated
// by thread 0 only: the FP64 divisions and tests run once per CTA instead of
// once per thread (FP64 issue slots are scarce on this GPU).
struct InnerScal {
  double rr0[MCL], rz[MCL], rr[MCL], rmin[MCL], rck[MCL];
  double gam[MCL], alp[MCL];  // single-reduction form: (r, M r) and alpha of the last pass
  float alpha[MCL], beta[MCL];
  int its[MCL];
  unsigned act;
  unsigned iok;    // continua whose last inner solve met inner_rtol
  int brk;
};

struct Sm {
  Team team;
  InnerScal* sc;
  float* box;      // [NST][NBOX][ABOX]
  float* pn;       // [PN]
  double* red;     // [NT/32][KM]
  double* res;     // [KM]
  uint64_t* bar;   // [NST]
};

// Inner FP32 PCG with ONE grid-wide reduction per iteration: the
// Chronopoulos-Gear recurrences of Jacobi PCG (u = M r, w = A u, s = A p
// carried by recurrence). In exact arithmetic they produce the iterates of
// textbook PCG on A d = r0; the two inner products of an iteration,
// gamma = (r, u) and delta = (w, u), are formed after the same pass, and
// alpha follows from delta - beta gamma / alpha_prev = (p, A p).
//
// One pass per iteration i, tile by tile with a one-cell halo:
//   s_i = w_i + beta_i s_{i-1},  r_{i+1} = r_i - alpha_i s_i   (tile + halo)
//   u_{i+1} = M r_{i+1}                                         (tile + halo)
//   p_i = M r_i + beta_i p_{i-1},  d += alpha_i p_i             (tile)
//   w_{i+1} = A u_{i+1},  (r,r), (r,u), (w,u) of i+1             (tile)
// The halo values are recomputed from the previous pass's vectors (the same
// fused multiply-adds as their owner tile, so both copies agree bit for bit),
// which is what lets the stencil of w_{i+1} follow the update without a
// second grid barrier. r, s and w are double-buffered (buffer `cur` is read
// through TMA, `cur ^ 1` written); p and d are only touched at their own cells
// and stay in place. Pass -1 runs with alpha = beta = 0 on s = w = p = 0 and
// forms w_0 = A M r_0 and the first inner products.
//
// Returns false only when the launch must stop (barrier timeout / abort);
// convergence, the progress window and breakdown end a continuum's solve and
// leave d consistent with the last residual formed.
template <int L, typename TT>
__device__ bool inner_single(const IrParams& ip, const TmaMaps& maps, unsigned active, Sm& sm,
                             uint32_t& phb, int& slot, int inner_cap) {
  const StepParams& sp = ip.sp;
  const int nx = sp.nx, ny = sp.ny, pitch = sp.pitch;
  const int tid = threadIdx.x;
  const Team tm = sm.team;
  const double in2 = ip.inner_rtol * ip.inner_rtol;
  InnerScal& S = *sm.sc;
  if (tid == 0) {
    for (int a = 0; a < L; ++a) {
      S.alpha[a] = 0.f;
      S.beta[a] = 0.f;
    }
    S.act = active;
    S.iok = 0;
    S.brk = 0;
  }
  __syncthreads();
  unsigned act = active;
  int cur = 0;
  int it = -1;
  const int tiles = sp.tiles_x * sp.tiles_y;
  const int lx = tid % TX, ly = tid / TX;
  while (act) {
    if (it >= inner_cap) break;
    int alist[L];
    int nact = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) if (act & (1u << a)) alist[nact++] = a;
    // per continuum: (r, r), (r, u), (w, u) of the new residual
    float dots[3 * L];
#pragma unroll
    for (int k = 0; k < 3 * L; ++k) dots[k] = 0.f;
    const int ntask = nact * tiles;
    auto issue = [&](int task, int s) {
      const int w = task / tiles, tt = task - w * tiles;
      int a0 = 0;
#pragma unroll
      for (int k = 0; k < L; ++k) if (k == w) a0 = alist[k];
      const int bx0 = (tt % sp.tiles_x) * TX - HOFF;
      const int by0 = (tt / sp.tiles_x) * TY - 1;
      uint64_t* bar = sm.bar + s;
      fence_proxy_async();
      mbar_expect_tx(bar, 4 * BOX_BYTES);
      float* base = sm.box + (size_t)s * NBOX * ABOX;
      tma_load_2d(base, cur ? &maps.q[a0] : &maps.r[a0], bx0, by0, bar);
      tma_load_2d(base + ABOX, &maps.P[cur][a0], bx0, by0, bar);
      tma_load_2d(base + 2 * ABOX, &maps.w[cur][a0], bx0, by0, bar);
      tma_load_2d(base + 3 * ABOX, &maps.invd[a0], bx0, by0, bar);
    };
    const int G = tm.size;
    int tk = tm.rank, k = 0;
    unsigned pend = 0;
#pragma unroll
    for (int j = 0; j < NST - 1; ++j) {
      const int tj = tk + j * G;
      if (tj < ntask) {
        if (tid == 0) issue(tj, j);
        pend |= 1u << j;
      }
    }
    bool tma_ok = true;
    for (; tk < ntask; tk += G, ++k) {
      const int s = k % NST;
      {
        const int tn = tk + (NST - 1) * G, sn = (k + NST - 1) % NST;
        if (tn < ntask) {
          if (tid == 0) issue(tn, sn);
          pend |= 1u << sn;
        }
      }
      const int w = tk / tiles, tt = tk - w * tiles;
      int a0 = 0;
#pragma unroll
      for (int kk = 0; kk < L; ++kk) if (kk == w) a0 = alist[kk];
      const int x0 = (tt % sp.tiles_x) * TX, y0 = (tt / sp.tiles_x) * TY;
      const int gx = x0 + lx;
      const TT* TE = static_cast<const TT*>(ip.TElo[a0]);
      const TT* TN = static_cast<const TT*>(ip.TNlo[a0]);
      float te[CPT], tw[CPT], tn[CPT], ts[CPT], dc[CPT], pold[CPT], dold[CPT];
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int gy = y0 + ly + RPT * j;
        const long long i = (long long)gy * pitch + gx;
        tfaces(TE, TN, i, gx, gy, nx, ny, pitch, te[j], tw[j], tn[j], ts[j]);
        dc[j] = pold[j] = dold[j] = 0.f;
        if (gx < nx && gy < ny) {
          dc[j] = ip.dc32[a0] ? __ldg(ip.dc32[a0] + i) : ip.dcf[a0];
          pold[j] = __ldcg(ip.p32[a0] + i);
          dold[j] = __ldcg(ip.d32[a0] + i);
        }
      }
      if (!mbar_wait(sm.bar + s, (phb >> s) & 1u, sp.spin_limit)) {
        if (tid == 0) grid_raise_abort(irbar(ip, tm), (int)MC_E_TIMEOUT);
        tma_ok = false;
        break;
      }
      phb ^= 1u << s;
      pend &= ~(1u << s);
      const float* bR = sm.box + (size_t)s * NBOX * ABOX;
      const float* bS = bR + ABOX;
      const float* bW = bR + 2 * ABOX;
      const float* bD = bR + 3 * ABOX;
      const float al = S.alpha[a0], bt = S.beta[a0];
      // u_{i+1} = M (r_i - alpha (w_i + beta s_{i-1})) on the 66 x 18 region
      for (int e = tid; e < PN; e += NT) {
        const int ry = e / PX, rx = e - ry * PX;
        const int b = ry * BX + rx + (HOFF - 1);
        const float sn = __fmaf_rn(bt, bS[b], bW[b]);
        const float rn = __fmaf_rn(-al, sn, bR[b]);
        sm.pn[e] = __fmul_rn(bD[b], rn);
      }
      __syncthreads();
      float* rN = cur ? ip.r32[a0] : ip.q32[a0];
      float* sN = ip.P32[cur ^ 1][a0];
      float* wN = ip.w32[cur ^ 1][a0];
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int lyj = ly + RPT * j;
        const int gy = y0 + lyj;
        if (gx >= nx || gy >= ny) continue;
        const long long i = (long long)gy * pitch + gx;
        const int c = (lyj + 1) * PX + lx + 1;
        const int b = (lyj + 1) * BX + lx + HOFF;
        const float sn = __fmaf_rn(bt, bS[b], bW[b]);
        const float rn = __fmaf_rn(-al, sn, bR[b]);
        const float uc = sm.pn[c];
        const float pv = __fmaf_rn(bt, pold[j], __fmul_rn(bD[b], bR[b]));
        const float dv = __fmaf_rn(al, pv, dold[j]);
        const float wv = dc[j] * uc + te[j] * (uc - sm.pn[c + 1]) + tw[j] * (uc - sm.pn[c - 1]) +
                         tn[j] * (uc - sm.pn[c + PX]) + ts[j] * (uc - sm.pn[c - PX]);
        rN[i] = rn;
        sN[i] = sn;
        wN[i] = wv;
        ip.p32[a0][i] = pv;
        ip.d32[a0][i] = dv;
#pragma unroll
        for (int kk = 0; kk < L; ++kk)
          if (kk == a0) {
            dots[kk] += rn * rn;
            dots[L + kk] += rn * uc;
            dots[2 * L + kk] += wv * uc;
          }
      }
      __syncthreads();
    }
    if (!tma_ok) {
      for (int st = 0; st < NST; ++st)
        if (pend & (1u << st)) mbar_wait(sm.bar + st, (phb >> st) & 1u, 1LL << 24);
      return false;
    }
    store_part_f<3 * L>(dots, qbits(act, L, 3), sm.box, sp.partials, slot, tm);
    if (!gsync(ip, tm)) return false;
    sum_totals<3 * L>(sp.partials, slot, sm.res, tm);
    slot ^= 1;
    if (tid == 0) {
      unsigned a_act = act;
      for (int a = 0; a < L; ++a) {
        const unsigned bit = 1u << a;
        if (!(act & bit)) continue;
        const double rr = sm.res[a], gam = sm.res[L + a], del = sm.res[2 * L + a];
        if (it < 0) {
          // pass -1: r_0, u_0 = M r_0, w_0 = A u_0; alpha_0 = gamma / delta
          S.rr0[a] = S.rr[a] = S.rmin[a] = S.rck[a] = rr;
          if (!(rr > 0.0) || !(gam > 0.0) || !(del > 0.0) || !isfinite(gam) || !isfinite(del)) {
            a_act &= ~bit;
            continue;
          }
          S.gam[a] = gam;
          S.alp[a] = gam / del;
          S.alpha[a] = (float)S.alp[a];
          S.beta[a] = 0.f;
          continue;
        }
        S.rr[a] = rr;
        S.its[a] += 1;
        if (!(rr > in2 * S.rr0[a])) S.iok |= bit;
        if (!(rr > in2 * S.rr0[a]) || !isfinite(rr)) {
          a_act &= ~bit;
          continue;
        }
        // FP32 progress test, as in the two-reduction form: the smallest
        // residual seen must halve in every window of 2048 iterations
        if (rr < S.rmin[a]) S.rmin[a] = rr;
        if (((it + 1) & 2047) == 0) {
          if (!(S.rmin[a] < 0.25 * S.rck[a])) a_act &= ~bit;
          S.rck[a] = S.rmin[a];
        }
        const double be = gam / S.gam[a];
        const double den = del - be * gam / S.alp[a];
        if (!(gam > 0.0) || !(den > 0.0) || !isfinite(den)) {
          a_act &= ~bit;  // breakdown: keep what the sweep reached
          continue;
        }
        S.gam[a] = gam;
        S.alp[a] = gam / den;
        S.alpha[a] = (float)S.alp[a];
        S.beta[a] = (float)be;
      }
      S.act = a_act;
    }
    __syncthreads();
    act = S.act;
    cur ^= 1;
    ++it;
  }
  return true;
}

// One solve of the continua in `mask` (all at once for D; one for L/U).
template <int L, typename TT>
__device__ bool ir_solve(const IrParams& ip, const TmaMaps& maps, unsigned mask, Sm& sm,
                         uint32_t& phb, int& slot) {
  const StepParams& sp = ip.sp;
  const int nx = sp.nx, ny = sp.ny, pitch = sp.pitch;
  const long long Np = sp.Np;
  const int tid = threadIdx.x;
  const Team tm = sm.team;
  const long long gtid = (long long)tm.rank * NT + tid;
  const long long gs = (long long)tm.size * NT;
  const bool lag_prev = sp.scheme == MC_SCHEME_D;
  const double rtol2 = sp.rtol * sp.rtol;
  const double in2 = ip.inner_rtol * ip.inner_rtol;
  const bool single = ip.inner_form == MC_INNER_SINGLE_REDUCTION;
  double bb[L], rr_prev[L], rr_last[L];
#pragma unroll
  for (int a = 0; a < L; ++a) bb[a] = rr_prev[a] = rr_last[a] = 0.0;
  unsigned active = mask;
  unsigned iok = 0;
  if (tid == 0)
    for (int a = 0; a < MCL; ++a) sm.sc->its[a] = 0;
  __syncthreads();
  int sweeps = 0;
  bool ok = true;
  for (int sweep = 0; ok; ++sweep) {
    // ---- 1. FP64 residual and the sums of the constant-mode correction -----
    // q: [rr, sum r, sum dc, sum r dc, sum dc^2, bb, xx, dd] per continuum
    // (dd: the last inner correction, still in d32)
    double acc[8 * L];
#pragma unroll
    for (int k = 0; k < 8 * L; ++k) acc[k] = 0.0;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(active & (1u << a))) continue;
      const double* x = sp.p[a];
      for (long long i = gtid; i < Np; i += gs) {
        const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
        if (gx >= nx) continue;
        const double xc = __ldcg(x + i);
        const double xp = __ldcg(sp.pprev[a] + i);
        const double f = __ldg(sp.F[a] + i);
        double rv = f + sp.mtau[a] * (xp - xc);
        double bv = sp.mtau[a] * xp + f;
        if (sp.W[a]) {  // implicit well term: b += W p_w, A x += W x
          const double fw = __ldg(sp.FW[a] + i);
          rv += fw - __ldg(sp.W[a] + i) * xc;
          bv += fw;
        }
#pragma unroll
        for (int b = 0; b < L; ++b) {
          if (b == a) continue;
          const double pb = lag_prev ? __ldcg(sp.pprev[b] + i) : __ldcg(sp.p[b] + i);
          const double qv = qab(sp, a, b, i);
          rv += qv * (pb - xc);
          bv += qv * pb;
        }
        if (gx + 1 < nx) rv -= __ldg(sp.TE[a] + i) * (xc - __ldcg(x + i + 1));
        if (gx > 0) rv -= __ldg(sp.TE[a] + i - 1) * (xc - __ldcg(x + i - 1));
        if (gy + 1 < ny) rv -= __ldg(sp.TN[a] + i) * (xc - __ldcg(x + i + pitch));
        if (gy > 0) rv -= __ldg(sp.TN[a] + i - pitch) * (xc - __ldcg(x + i - pitch));
        const double dc = dcell(sp, a, i);
        sp.r[a][i] = rv;
        acc[a] += rv * rv;
        acc[L + a] += rv;
        acc[2 * L + a] += dc;
        acc[3 * L + a] += rv * dc;
        acc[4 * L + a] += dc * dc;
        acc[5 * L + a] += bv * bv;
        acc[6 * L + a] += xc * xc;
        if (sweep > 0) {
          const double dv = (double)__ldcg(ip.d32[a] + i);
          acc[7 * L + a] += dv * dv;
        }
      }
    }
    store_part<8 * L>(acc, qbits(active, L, 8), sm.box, sp.partials, slot, tm);
    if (!gsync(ip, tm)) return false;
    double t[8 * L];
    sum_part<8 * L>(sp.partials, slot, sm.res, t, tm);
    slot ^= 1;
    double shift[L];
    unsigned inner = 0;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      shift[a] = 0.0;
      if (!(active & (1u << a))) continue;
      if (sweep == 0) bb[a] = t[5 * L + a];
      const double c = t[2 * L + a] > 0.0 ? t[L + a] / t[2 * L + a] : 0.0;
      shift[a] = c;
      double rr = t[a] - 2.0 * c * t[3 * L + a] + c * c * t[4 * L + a];
      if (rr < 0.0) rr = 0.0;
      rr_last[a] = rr;
      if (rr > rtol2 * bb[a]) {
        // refinement floor: the inner solve met its target, ||r|| did not
        // halve, and either ||r|| is within 1e3 rtol ||b|| or the last
        // correction moved x by at most 100 rtol ||x||
        const bool flat = sweep > 0 && (iok & (1u << a)) && rr > 0.25 * rr_prev[a];
        const bool near = rr <= 1e6 * rtol2 * bb[a] || t[7 * L + a] <= 1e4 * rtol2 * t[6 * L + a];
        if (!(flat && near)) inner |= 1u << a;
      }
      rr_prev[a] = rr;
    }
    if (inner && sweep >= ip.ir_max) {
      if (tm.rank == 0 && tid == 0) {
        atomicCAS(sp.status, 0, (int)MC_E_NOCONV);
        // what the failed solve reached, for the caller's diagnosis
        for (int a = 0; a < L; ++a) {
          if (!(mask & (1u << a))) continue;
          sp.iters[a] += sm.sc->its[a];
          if (sm.sc->its[a] > sp.max_iters[a]) sp.max_iters[a] = sm.sc->its[a];
          sp.relres[a] = bb[a] > 0.0 ? sqrt(rr_last[a] / bb[a]) : sqrt(rr_last[a]);
        }
        atomicAdd(ip.ir_sweeps, sweeps);
      }
      return false;
    }
    // ---- 2. apply the shift; start the inner solve on the corrected residual
    double acc2[2 * L];
#pragma unroll
    for (int k = 0; k < 2 * L; ++k) acc2[k] = 0.0;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(active & (1u << a))) continue;
      const double c = shift[a];
      const bool go = inner & (1u << a);
      for (long long i = gtid; i < Np; i += gs) {
        const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
        if (gx >= nx) continue;
        sp.p[a][i] = __ldcg(sp.p[a] + i) + c;
        if (go) {
          const double rv = __ldcg(sp.r[a] + i) - c * dcell(sp, a, i);
          const float r32 = (float)rv;
          ip.r32[a][i] = r32;
          ip.d32[a][i] = 0.0f;
          if (single) {
            // s_{-1} = w_{-1} = p_{-1} = 0: the first pass of the
            // single-reduction loop then forms w_0 = A M r_0
            ip.P32[0][a][i] = 0.0f;
            ip.w32[0][a][i] = 0.0f;
            ip.p32[a][i] = 0.0f;
          } else {
            const float z = __ldg(ip.invd32[a] + i) * r32;
            ip.P32[0][a][i] = z;
            acc2[a] += (double)r32 * (double)r32;
            acc2[L + a] += (double)r32 * (double)z;
          }
        }
      }
    }
    active = inner;
    if (!active) break;
    ++sweeps;
    // The inner solve ends at inner_rtol, when FP32 CG stops making progress
    // (the window test), or at a cap of 16 max(nx, ny) iterations within
    // [2048, 16384] (and max_iter). The cap has two sides: on a fracture
    // continuum (k 1e4 in thin connected networks, 1e-2 around them)
    // Jacobi-PCG needs about 10 n iterations for the 1e-3 reduction, and
    // cutting that short multiplies the total work; but a very long FP32 run
    // drifts (its recursive residual keeps falling while the true one does
    // not: 100000-iteration sweeps at 4096^2 and contrast 1e5 gained
    // nothing), so the FP64 sweep restarts it.
    int inner_cap = 16 * (nx > ny ? nx : ny);
    if (inner_cap < 2048) inner_cap = 2048;
    if (inner_cap > 16384) inner_cap = 16384;
    if (inner_cap > sp.max_iter) inner_cap = sp.max_iter;
    if (single) {
      if (!gsync(ip, tm)) return false;
      if (!inner_single<L, TT>(ip, maps, active, sm, phb, slot, inner_cap)) return false;
      iok = sm.sc->iok;
    } else {
    store_part<2 * L>(acc2, qbits(inner, L, 2), sm.box, sp.partials, slot, tm);
    if (!gsync(ip, tm)) return false;
    sum_totals<2 * L>(sp.partials, slot, sm.res, tm);
    slot ^= 1;
    InnerScal& S = *sm.sc;
    if (tid == 0) {
      unsigned a_act = 0;
      for (int a = 0; a < L; ++a) {
        S.rr0[a] = S.rr[a] = S.rmin[a] = S.rck[a] = sm.res[a];
        S.rz[a] = sm.res[L + a];
        S.beta[a] = 0.f;
        S.alpha[a] = 0.f;
        if ((active & (1u << a)) && sm.res[a] > 0.0) a_act |= 1u << a;
      }
      S.act = a_act;
      S.iok = 0;
      S.brk = 0;
    }
    __syncthreads();
    // ---- 3. FP32 inner PCG ----------------------------------------------------
    unsigned act = S.act;
    int cur = 0;
    int it = 0;
    const int tiles = sp.tiles_x * sp.tiles_y;
    const int lx = tid % TX, ly = tid / TX;
    while (act) {
      if (it >= inner_cap) break;  // the outer loop measures what was reached
      int alist[L];
      int nact = 0;
#pragma unroll
      for (int a = 0; a < L; ++a) if (act & (1u << a)) alist[nact++] = a;
      float pq[L];
#pragma unroll
      for (int a = 0; a < L; ++a) pq[a] = 0.f;
      const int ntask = nact * tiles;
      auto issue = [&](int task, int s) {
        const int w = task / tiles, tt = task - w * tiles;
        int a0 = 0;
#pragma unroll
        for (int k = 0; k < L; ++k) if (k == w) a0 = alist[k];
        const int bx0 = (tt % sp.tiles_x) * TX - HOFF;
        const int by0 = (tt / sp.tiles_x) * TY - 1;
        uint64_t* bar = sm.bar + s;
        fence_proxy_async();
        mbar_expect_tx(bar, 3 * BOX_BYTES);
        float* base = sm.box + (size_t)s * NBOX * ABOX;
        tma_load_2d(base, &maps.r[a0], bx0, by0, bar);
        tma_load_2d(base + ABOX, &maps.P[cur][a0], bx0, by0, bar);
        tma_load_2d(base + 2 * ABOX, &maps.invd[a0], bx0, by0, bar);
      };
      const int G = tm.size;
      int tk = tm.rank, k = 0;
      unsigned pend = 0;
#pragma unroll
      for (int j = 0; j < NST - 1; ++j) {
        const int tj = tk + j * G;
        if (tj < ntask) {
          if (tid == 0) issue(tj, j);
          pend |= 1u << j;
        }
      }
      bool tma_ok = true;
      for (; tk < ntask; tk += G, ++k) {
        const int s = k % NST;
        {
          const int tn = tk + (NST - 1) * G, sn = (k + NST - 1) % NST;
          if (tn < ntask) {
            if (tid == 0) issue(tn, sn);
            pend |= 1u << sn;
          }
        }
        const int w = tk / tiles, tt = tk - w * tiles;
        int a0 = 0;
#pragma unroll
        for (int kk = 0; kk < L; ++kk) if (kk == w) a0 = alist[kk];
        const int x0 = (tt % sp.tiles_x) * TX, y0 = (tt / sp.tiles_x) * TY;
        const int gx = x0 + lx;
        const TT* TE = static_cast<const TT*>(ip.TElo[a0]);
        const TT* TN = static_cast<const TT*>(ip.TNlo[a0]);
        float te[CPT], tw[CPT], tn[CPT], ts[CPT], dc[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int gy = y0 + ly + RPT * j;
          const long long i = (long long)gy * pitch + gx;
          tfaces(TE, TN, i, gx, gy, nx, ny, pitch, te[j], tw[j], tn[j], ts[j]);
          dc[j] = 0.f;
          if (gx < nx && gy < ny) {
            dc[j] = ip.dc32[a0] ? __ldg(ip.dc32[a0] + i) : ip.dcf[a0];
          }
        }
        if (!mbar_wait(sm.bar + s, (phb >> s) & 1u, sp.spin_limit)) {
          if (tid == 0) grid_raise_abort(irbar(ip, tm), (int)MC_E_TIMEOUT);
          tma_ok = false;
          break;
        }
        phb ^= 1u << s;
        pend &= ~(1u << s);
        const float* base = sm.box + (size_t)s * NBOX * ABOX;
        const float bt = S.beta[a0];
        for (int e = tid; e < PN; e += NT) {
          const int ry = e / PX, rx = e - ry * PX;
          const int bidx = ry * BX + rx + (HOFF - 1);
          sm.pn[e] = base[2 * ABOX + bidx] * base[bidx] + bt * base[ABOX + bidx];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int lyj = ly + RPT * j;
          const int gy = y0 + lyj;
          if (gx >= nx || gy >= ny) continue;
          const long long i = (long long)gy * pitch + gx;
          const int c = (lyj + 1) * PX + lx + 1;
          const float pc = sm.pn[c];
          const float qv = dc[j] * pc + te[j] * (pc - sm.pn[c + 1]) + tw[j] * (pc - sm.pn[c - 1]) +
                           tn[j] * (pc - sm.pn[c + PX]) + ts[j] * (pc - sm.pn[c - PX]);
          ip.P32[cur ^ 1][a0][i] = pc;
          ip.q32[a0][i] = qv;
#pragma unroll
          for (int kk = 0; kk < L; ++kk) if (kk == a0) pq[kk] += pc * qv;
        }
        __syncthreads();
      }
      if (!tma_ok) {
        for (int st = 0; st < NST; ++st)
          if (pend & (1u << st)) mbar_wait(sm.bar + st, (phb >> st) & 1u, 1LL << 24);
        return false;
      }
      store_part_f<L>(pq, act, sm.box, sp.partials, slot, tm);
      if (!gsync(ip, tm)) return false;
      sum_totals<L>(sp.partials, slot, sm.res, tm);
      slot ^= 1;
      if (tid == 0) {
        int b = 0;
        for (int a = 0; a < L; ++a) {
          S.alpha[a] = 0.f;
          if (act & (1u << a)) {
            const double pqt = sm.res[a];
            if (!(pqt > 0.0) || !isfinite(pqt)) b = 1;
            else S.alpha[a] = (float)(S.rz[a] / pqt);
          }
        }
        S.brk = b;
      }
      __syncthreads();
      if (S.brk) break;  // FP32 breakdown: keep what the sweep reached
      float acc3[2 * L];
#pragma unroll
      for (int kk = 0; kk < 2 * L; ++kk) acc3[kk] = 0.f;
      const long long Np4 = Np >> 2;
#pragma unroll
      for (int a = 0; a < L; ++a) {
        if (!(act & (1u << a))) continue;
        const float al = S.alpha[a];
        float4* d = reinterpret_cast<float4*>(ip.d32[a]);
        float4* r = reinterpret_cast<float4*>(ip.r32[a]);
        const float4* Pn = reinterpret_cast<const float4*>(ip.P32[cur ^ 1][a]);
        const float4* qq = reinterpret_cast<const float4*>(ip.q32[a]);
        const float4* iv = reinterpret_cast<const float4*>(ip.invd32[a]);
        float srr = 0.f, srz = 0.f;
#pragma unroll 2
        for (long long j = gtid; j < Np4; j += gs) {
          const float4 r0 = __ldcg(r + j), qv = __ldcg(qq + j), dv = __ldcg(d + j),
                       pv = __ldcg(Pn + j), iw = __ldg(iv + j);
          float4 rn, dn;
          rn.x = r0.x - al * qv.x; rn.y = r0.y - al * qv.y;
          rn.z = r0.z - al * qv.z; rn.w = r0.w - al * qv.w;
          dn.x = dv.x + al * pv.x; dn.y = dv.y + al * pv.y;
          dn.z = dv.z + al * pv.z; dn.w = dv.w + al * pv.w;
          d[j] = dn;
          r[j] = rn;
          srr += rn.x * rn.x + rn.y * rn.y + rn.z * rn.z + rn.w * rn.w;
          srz += rn.x * (iw.x * rn.x) + rn.y * (iw.y * rn.y) + rn.z * (iw.z * rn.z) +
                 rn.w * (iw.w * rn.w);
        }
        acc3[a] += srr;
        acc3[L + a] += srz;
      }
      store_part_f<2 * L>(acc3, qbits(act, L, 2), sm.box, sp.partials, slot, tm);
      if (!gsync(ip, tm)) return false;
      sum_totals<2 * L>(sp.partials, slot, sm.res, tm);
      slot ^= 1;
      ++it;
      if (tid == 0) {
        unsigned a_act = act;
        for (int a = 0; a < L; ++a) {
          if (!(act & (1u << a))) continue;
          const double rr = sm.res[a];
          const double rzn = sm.res[L + a];
          S.rr[a] = rr;
          S.beta[a] = (float)(rzn / S.rz[a]);
          S.rz[a] = rzn;
          S.its[a] += 1;
          if (!(rr > in2 * S.rr0[a])) S.iok |= 1u << a;
          if (!(rr > in2 * S.rr0[a]) || !isfinite(rr)) a_act &= ~(1u << a);
          // FP32 progress test: the smallest residual seen must halve in
          // every window of 2048 iterations (CG residual norms are not
          // monotone, so the running minimum is compared); a slower FP32 run
          // has hit its rounding limits and the outer FP64 sweep restarts
          // from what was reached
          if (rr < S.rmin[a]) S.rmin[a] = rr;
          if ((it & 2047) == 0) {
            if (!(S.rmin[a] < 0.25 * S.rck[a])) a_act &= ~(1u << a);
            S.rck[a] = S.rmin[a];
          }
        }
        S.act = a_act;
      }
      __syncthreads();
      act = S.act;
      cur ^= 1;
    }
    iok = S.iok;
    }
    // ---- 4. x += d (FP64) -------------------------------------------------------
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(active & (1u << a))) continue;
      for (long long i = gtid; i < Np; i += gs) sp.p[a][i] = __ldcg(sp.p[a] + i) + (double)__ldcg(ip.d32[a] + i);
    }
    if (!gsync(ip, tm)) return false;
  }
  if (tm.rank == 0 && tid == 0) {
#pragma unroll
    for (int a = 0; a < L; ++a) {
      if (!(mask & (1u << a))) continue;
      sp.iters[a] += sm.sc->its[a];
      if (sm.sc->its[a] > sp.max_iters[a]) sp.max_iters[a] = sm.sc->its[a];
      sp.relres[a] = bb[a] > 0.0 ? sqrt(rr_last[a] / bb[a]) : sqrt(rr_last[a]);
    }
    atomicAdd(ip.ir_sweeps, sweeps);
  }
  return gsync(ip, tm);
}

// One time step of one instance: the D-scheme solves every continuum at once,
// the L- and U-schemes one continuum after the other (index / reverse order).
template <int L, typename TT>
__device__ bool ir_instance_step(const IrParams& ip, const TmaMaps& maps, Sm& sm, uint32_t& phb,
                                 int& slot) {
  const int scheme = ip.sp.scheme;
  if (scheme == MC_SCHEME_D) return ir_solve<L, TT>(ip, maps, (1u << L) - 1u, sm, phb, slot);
  for (int k = 0; k < L; ++k) {
    const int a = scheme == MC_SCHEME_U ? L - 1 - k : k;
    if (!ir_solve<L, TT>(ip, maps, 1u << a, sm, phb, slot)) return false;
  }
  return true;
}

// Shared-memory carve-up common to both kernels.
__device__ __forceinline__ void carve(Sm& sm, unsigned char* smem_raw, InnerScal* sc) {
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  sm.sc = sc;
  sm.box = reinterpret_cast<float*>(base);
  sm.pn = sm.box + NST * NBOX * ABOX;
  sm.red = reinterpret_cast<double*>(sm.pn + ((PN + 1) / 2) * 2);
  sm.res = sm.red + (NT / 32) * KM;
  sm.bar = reinterpret_cast<uint64_t*>(sm.res + KM);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(sm.bar + s, 1);
    fence_mbar_init();
  }
  __syncthreads();
}

template <int L, typename TT>
__global__ void __launch_bounds__(NT, 2)
    ir_step_kernel(const __grid_constant__ IrParams ip, const __grid_constant__ TmaMaps maps) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ InnerScal s_scal;
  Sm sm;
  sm.team.rank = blockIdx.x;
  sm.team.size = gridDim.x;
  carve(sm, smem_raw, &s_scal);
  uint32_t phb = 0u;
  int slot = 0;
  const StepParams& sp = ip.sp;
  const long long gtid = (long long)blockIdx.x * NT + threadIdx.x;
  const long long gs = (long long)gridDim.x * NT;
  int done = 0;
  bool ok = true;
  for (int step = 0; step < sp.nsteps && ok; ++step) {
    for (int a = 0; a < L; ++a)
      for (long long i = gtid; i < sp.Np; i += gs) sp.pprev[a][i] = __ldcg(sp.p[a] + i);
    if (!gsync(ip, sm.team)) { ok = false; break; }
    ok = ir_instance_step<L, TT>(ip, maps, sm, phb, slot);
    if (ok) ++done;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sp.steps_done = done;
}

// Batched form: one launch advances every instance of a batch by one step.
// CTA b belongs to team b / team; each team takes the next instance from the
// shared counter (instances are listed largest first, so the long solves
// start early and the short ones fill the tail), copies its parameters to
// shared memory, points the reductions and barriers at the team's own words,
// and runs the step with team-scoped barriers. Continua converge
// independently inside each solve (per-continuum active masks; converged
// continua drop out of the tile list). An instance whose solve fails
// (refinement limit) is put back to the start of the step and skipped until
// the host resets it; a barrier timeout anywhere raises the abort word and
// every team leaves.
template <typename TT>
__global__ void __launch_bounds__(NT, 2) ir_batch_kernel(const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ InnerScal s_scal;
  __shared__ __align__(16) IrParams s_ip;
  __shared__ int s_idx, s_flag;
  static_assert(sizeof(IrParams) % 8 == 0, "IrParams copy in 8-byte words");
  const int t = blockIdx.x / bp.team;
  if (t >= bp.teams) return;
  Sm sm;
  sm.team.rank = blockIdx.x - t * bp.team;
  sm.team.size = bp.team;
  carve(sm, smem_raw, &s_scal);
  const int tid = threadIdx.x;
  const bool lead = sm.team.rank == 0 && tid == 0;
  unsigned* tc = bp.ctrl + 32 * (t + 1);
  GridBar tb;
  tb.count = reinterpret_cast<unsigned long long*>(tc);
  tb.abort_word = bp.abort_word;
  tb.status = reinterpret_cast<int*>(bp.ctrl + 1);
  tb.spin_limit = bp.spin_limit;
  tb.nparts = (unsigned)bp.team;
  if (tid == 0) s_flag = ld_acquire_u32(bp.abort_word) != 0u;
  __syncthreads();
  if (s_flag) return;
  uint32_t phb = 0u;
  int slot = 0;
  const long long gtid = (long long)sm.team.rank * NT + tid;
  const long long gs = (long long)bp.team * NT;
  for (;;) {
    // the team lead draws the next instance; the barrier publishes it
    if (lead) {
      const unsigned v = atomicAdd(bp.ctrl, 1u);
      *reinterpret_cast<volatile unsigned*>(tc + 4) = v;
    }
    if (!grid_barrier(tb)) break;
    if (tid == 0) s_idx = (int)ld_acquire_u32(tc + 4);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= bp.n) break;
    const int inst = __ldg(bp.order + idx);
    {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(bp.inst + inst);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_ip);
      for (int w = tid; w < (int)(sizeof(IrParams) / 8); w += NT) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    BatchInst* rec = bp.st + inst;
    if (tid == 0) {
      StepParams& sp = s_ip.sp;
      sp.scheme = bp.scheme;
      sp.rtol = bp.rtol;
      sp.max_iter = bp.max_iter;
      sp.spin_limit = bp.spin_limit;
      sp.partials = bp.partials + (size_t)t * 2 * KM * bp.team;
      sp.bar_count = tc;
      sp.status = &rec->status;
      sp.iters = rec->iters;
      sp.max_iters = rec->max_iters;
      sp.relres = rec->relres;
      s_ip.inner_rtol = bp.inner_rtol;
      s_ip.ir_max = bp.ir_max;
      s_ip.inner_form = bp.inner_form;
      s_ip.ir_sweeps = &rec->ir_sweeps;
      s_ip.abort_word = bp.abort_word;
      s_flag = __ldcg(&rec->status) != 0;
    }
    __syncthreads();
    if (s_flag) {  // failed earlier in this call: leave it as it is
      if (!grid_barrier(tb)) break;
      continue;
    }
    const StepParams& sp = s_ip.sp;
    const int L = sp.L;
    for (int a = 0; a < L; ++a)
      for (long long i = gtid; i < sp.Np; i += gs) sp.pprev[a][i] = __ldcg(sp.p[a] + i);
    if (!gsync(s_ip, sm.team)) break;
    if (lead) rec->busy = 1;
    const TmaMaps& maps = bp.maps[inst];
    bool ok;
    switch (L) {
      case 1: ok = ir_instance_step<1, TT>(s_ip, maps, sm, phb, slot); break;
      case 2: ok = ir_instance_step<2, TT>(s_ip, maps, sm, phb, slot); break;
      case 3: ok = ir_instance_step<3, TT>(s_ip, maps, sm, phb, slot); break;
      default: ok = ir_instance_step<4, TT>(s_ip, maps, sm, phb, slot); break;
    }
    if (ok) {
      if (lead) {
        rec->steps_done += 1;
        rec->busy = 0;
      }
      continue;
    }
    if (tid == 0) s_flag = ld_acquire_u32(bp.abort_word) != 0u;
    __syncthreads();
    if (s_flag) break;  // timeout: the host restores instances left busy
    for (int a = 0; a < L; ++a)
      for (long long i = gtid; i < sp.Np; i += gs) sp.p[a][i] = __ldcg(sp.pprev[a] + i);
    if (!gsync(s_ip, sm.team)) break;
    if (lead) rec->busy = 0;
  }
}

template <int L, typename TT>
size_t ir_smem() {
  return (size_t)NST * NBOX * ABOX * 4 + (size_t)((PN + 1) / 2) * 2 * 4 +
         (size_t)((NT / 32) * KM + KM) * 8 + NST * 8 + 128;
}

struct IKInfo {
  void* fn;
  size_t smem;
};

template <int L, typename TT>
IKInfo iinfo() {
  return IKInfo{(void*)ir_step_kernel<L, TT>, ir_smem<L, TT>()};
}

IKInfo ipick(int L, bool bf16) {
  if (bf16) {
    switch (L) {
      case 1: return iinfo<1, __nv_bfloat16>();
      case 2: return iinfo<2, __nv_bfloat16>();
      case 3: return iinfo<3, __nv_bfloat16>();
      default: return iinfo<4, __nv_bfloat16>();
    }
  }
  switch (L) {
    case 1: return iinfo<1, float>();
    case 2: return iinfo<2, float>();
    case 3: return iinfo<3, float>();
    default: return iinfo<4, float>();
  }
}

__global__ void lo_copy_kernel(long long Np, const double* TE, const double* TN, const double* invd,
                               const double* dc, void* TElo, void* TNlo, float* invd32,
                               float* dc32, int bf16) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Np;
       i += (long long)gridDim.x * blockDim.x) {
    if (bf16) {
      static_cast<__nv_bfloat16*>(TElo)[i] = __double2bfloat16(TE[i]);
      static_cast<__nv_bfloat16*>(TNlo)[i] = __double2bfloat16(TN[i]);
    } else {
      static_cast<float*>(TElo)[i] = (float)TE[i];
      static_cast<float*>(TNlo)[i] = (float)TN[i];
    }
    invd32[i] = (float)invd[i];
    if (dc32) dc32[i] = (float)dc[i];
  }
}

}  // namespace

int mc_ir_max_blocks(int L, bool bf16, int num_sms) {
  IKInfo k = ipick(L, bf16);
  if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) != cudaSuccess)
    return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k.fn, NT, k.smem) != cudaSuccess) return 0;
  return per * num_sms;
}

int mc_ir_box_x() { return BX; }
int mc_ir_box_y() { return BY; }

cudaError_t mc_ir_prepare(mc_ctx* ctx, int bf16) {
  const size_t fb4 = (size_t)ctx->Np * 4;
  const size_t tb = bf16 ? (size_t)ctx->Np * 2 : fb4;
  cudaError_t e;
  if (ctx->lo_kind != 1 + bf16) {
    for (int a = 0; a < ctx->L; ++a) {
      if (!ctx->r32[a]) {
        if ((e = mc_alloc(ctx, (void**)&ctx->r32[a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->P32[0][a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->P32[1][a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->q32[a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->d32[a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->w32[0][a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->w32[1][a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->p32[a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->invd32[a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->TElo32[a], fb4)) != cudaSuccess) return e;
        if ((e = mc_alloc(ctx, (void**)&ctx->TNlo32[a], fb4)) != cudaSuccess) return e;
      }
      if (ctx->diagc[a] && !ctx->dc32[a] && (e = mc_alloc(ctx, (void**)&ctx->dc32[a], fb4)) != cudaSuccess)
        return e;
      // bf16 copies live in the first half of the FP32 buffers
      lo_copy_kernel<<<1024, 256, 0, ctx->stream>>>(ctx->Np, ctx->TE[a], ctx->TN[a], ctx->invd[a],
                                                    ctx->diagc[a], ctx->TElo32[a], ctx->TNlo32[a],
                                                    ctx->invd32[a], ctx->dc32[a], bf16);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      const int bx = BX, by = BY;
      if ((e = mc_encode_map(&ctx->maps32.r[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->r32[a], ctx->nx,
                             ctx->ny, ctx->pitch, bx, by)) != cudaSuccess) return e;
      if ((e = mc_encode_map(&ctx->maps32.P[0][a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->P32[0][a],
                             ctx->nx, ctx->ny, ctx->pitch, bx, by)) != cudaSuccess) return e;
      if ((e = mc_encode_map(&ctx->maps32.P[1][a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->P32[1][a],
                             ctx->nx, ctx->ny, ctx->pitch, bx, by)) != cudaSuccess) return e;
      if ((e = mc_encode_map(&ctx->maps32.invd[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->invd32[a],
                             ctx->nx, ctx->ny, ctx->pitch, bx, by)) != cudaSuccess) return e;
      if ((e = mc_encode_map(&ctx->maps32.q[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->q32[a],
                             ctx->nx, ctx->ny, ctx->pitch, bx, by)) != cudaSuccess) return e;
      for (int h = 0; h < 2; ++h)
        if ((e = mc_encode_map(&ctx->maps32.w[h][a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ctx->w32[h][a],
                               ctx->nx, ctx->ny, ctx->pitch, bx, by)) != cudaSuccess) return e;
    }
    ctx->lo_kind = 1 + bf16;
  }
  (void)tb;
  return cudaSuccess;
}

void mc_ir_fill(const mc_ctx* ctx, const StepParams& sp_in, IrParams* ip) {
  memset(ip, 0, sizeof(*ip));
  ip->sp = sp_in;
  ip->sp.tiles_x = (sp_in.nx + TX - 1) / TX;
  ip->sp.tiles_y = (sp_in.ny + TY - 1) / TY;
  for (int a = 0; a < ctx->L; ++a) {
    ip->r32[a] = ctx->r32[a];
    ip->P32[0][a] = ctx->P32[0][a];
    ip->P32[1][a] = ctx->P32[1][a];
    ip->q32[a] = ctx->q32[a];
    ip->d32[a] = ctx->d32[a];
    ip->w32[0][a] = ctx->w32[0][a];
    ip->w32[1][a] = ctx->w32[1][a];
    ip->p32[a] = ctx->p32[a];
    ip->invd32[a] = ctx->invd32[a];
    ip->TElo[a] = ctx->TElo32[a];
    ip->TNlo[a] = ctx->TNlo32[a];
    ip->dc32[a] = ctx->dc32[a];
    ip->dcf[a] = (float)sp_in.diagc_const[a];
  }
  ip->inner_rtol = ctx->opts.inner_rtol;
  ip->ir_max = ctx->opts.ir_max;
  ip->inner_form = ctx->opts.inner_form;
  ip->ir_sweeps = ctx->dsweeps;
  ip->abort_word = sp_in.bar_gen + 32;
}

cudaError_t mc_launch_ir(mc_ctx* ctx, const StepParams& sp_in, int bf16, int blocks) {
  IrParams ip;
  mc_ir_fill(ctx, sp_in, &ip);
  IKInfo k = ipick(ctx->L, bf16 != 0);
  cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&ip, &ctx->maps32};
  return cudaLaunchCooperativeKernel(k.fn, dim3(blocks), dim3(NT), args, k.smem, ctx->stream);
}

static void* batch_fn(bool bf16) {
  return bf16 ? (void*)ir_batch_kernel<__nv_bfloat16> : (void*)ir_batch_kernel<float>;
}

int mc_ir_batch_max_blocks(bool bf16, int num_sms) {
  void* fn = batch_fn(bf16);
  const size_t smem = ir_smem<1, float>();
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, NT, smem) != cudaSuccess) return 0;
  return per * num_sms;
}

cudaError_t mc_launch_ir_batch(const BatchParams& bp, int bf16, int blocks, cudaStream_t stream) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = ir_smem<1, float>();
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  BatchParams copy = bp;
  void* args[] = {&copy};
  return cudaLaunchKernelExC(&cfg, batch_fn(bf16 != 0), args);
}
