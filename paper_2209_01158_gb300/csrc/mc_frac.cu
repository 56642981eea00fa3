// Lower-dimensional fracture continuum on its own 1-D mesh, coupled to the
// context's matrix continua (Section 2, Eqs. mm-md and mm-tc; Section 3.1,
// Eqs. app-md and app-tc; schemes of Sections 3.2-3.3).
//
// Mesh (host, once): every segment is clipped to the unit square and split at
// the grid lines it crosses and at its intersections with the other segments;
// each piece iota_l is a fracture cell of length |iota_l| hosted by the matrix
// cell holding its midpoint. A junction is a point where pieces meet (split
// point, crossing, or both); pieces of a junction are coupled pairwise by the
// storage-free flux balance T_ln = t_l t_n / sum_m t_m, t_l = k_f / (|iota_l|/2)
// (two pieces: the two-point value k_f / (d_l + d_n)). The topology and the
// geometry (lengths, midpoints, hosts, junction membership) are built on the
// host; every coefficient is computed by the set-up kernels below.
//
// Coefficients (device): mass c_f |iota_l|, exchange with matrix continuum a
// q_al = sigma_af |iota_l| / (h/4) (interface |iota_l|, distance h/4: the mean
// distance from the points of a cell to a line through its centre), the
// junction sums and T_ln, and the fracture diagonal. On the matrix side the
// exchange is a per-cell diagonal term W = sum over hosted pieces of q_al
// (plus the context's own wells) with right-hand side sum q_al p_f,l: the
// persistent FP64 step kernel takes it like a well, with its own copies of the
// Jacobi diagonal, sqrt(d), scaled faces and scaled exchange.
//
// Time step (D-scheme; continua in ascending permeability, the fracture
// last): snapshot p_f; right-hand side of the matrix from p_f^{n-1}; the step
// kernel solves every matrix continuum (exchange among them lagged); the
// fracture is solved from p_m^{n-1}. L-scheme: the fracture uses p_m^n. U-scheme:
// the fracture first (p_m^{n-1}), then the matrix from p_f^n. The fracture
// solve is one CTA: PCG on the CSR graph with the line preconditioner (block
// Jacobi over the tridiagonal rows of each segment's pieces), flux-form
// operator, and the constant-mode correction of the matrix kernels. The
// coupled scheme runs one cooperative kernel: PCG over all matrix cells and
// pieces, point Jacobi on the matrix rows and the same line blocks on the
// fracture rows.

#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "mc_internal.h"
#include "mc_sync.cuh"

struct mc_frac {
  mc_ctx* ctx = nullptr;
  int L = 0;                 // matrix continua (the context's)
  int P = 0;                 // pieces
  int nnz = 0;               // off-diagonal CSR entries
  int NJ = 0;                // junctions
  int NH = 0;                // matrix cells hosting pieces
  double kf = 0, cf = 0;
  double sigma_f[MCL] = {};
  // host copies of the geometry
  std::vector<double> len, mid;
  std::vector<int> host;     // j * nx + i
  // device: mesh
  double* len_d = nullptr;
  int* rowptr = nullptr;     // P + 1
  int* col = nullptr;        // nnz
  int* ejct = nullptr;       // nnz: junction of each entry
  int* jptr = nullptr;       // NJ + 1
  int* jmem = nullptr;       // junction members
  int* hcell = nullptr;      // NH pitched indices of hosting cells
  int* hptr = nullptr;       // NH + 1
  int* hpiece = nullptr;     // pieces by hosting cell
  int* hostp = nullptr;      // P: pitched host index
  int NS = 0;                // segments (each a run of consecutive pieces)
  int* segptr = nullptr;     // NS + 1
  double* llo = nullptr;     // P: line factors (per-segment tridiagonal block,
  double* lcp = nullptr;     //    Thomas elimination): sub-diagonal, modified
  double* ldinv = nullptr;   //    super-diagonal, inverse pivots
  // device: coefficients
  double* jsum = nullptr;    // NJ
  double* T = nullptr;       // nnz
  double* q[MCL] = {};       // P per matrix continuum
  double* mf = nullptr;      // P: c_f |iota|
  double* dcf = nullptr;     // P: c_f|iota|/tau + sum_a q + W_f (non-diffusive diagonal)
  double* invdf = nullptr;   // P: 1 / (dcf + sum T)
  double* Ff = nullptr, *Wf = nullptr, *FWf = nullptr;
  // device: state and work
  double* pf = nullptr, *pf_prev = nullptr;
  double* r = nullptr, *z = nullptr, *pp = nullptr, *qq = nullptr, *bf = nullptr;
  // matrix side
  double* Wm[MCL] = {};      // user wells + hosted exchange
  double* FWm[MCL] = {};     // user W p_w + exchange right-hand side (per step)
  double* diagc[MCL] = {}, *invd[MCL] = {}, *sqd[MCL] = {}, *tE[MCL] = {}, *tN[MCL] = {};
  double* qs[MCL][MCL] = {};
  // status words of the fracture and coupled kernels
  int* dstat = nullptr;      // [0] status, [1] fracture iterations, [2] coupled iterations
  double* drel = nullptr;    // [0] fracture relres, [1] coupled relres
  double* cpart = nullptr;   // coupled kernel partial sums
  unsigned* cbar = nullptr;  // coupled kernel barrier words
  int* hidx = nullptr;       // per pitched matrix cell: hosting-cell list index or -1
  double* Pf2 = nullptr;     // second search-direction buffer (coupled and grid fracture kernels)
  int cblocks = 0;
  double* gpart = nullptr;   // grid fracture solve: partial sums
  unsigned* gbar = nullptr;  // grid fracture solve: barrier words
  int gblocks = 0;           // grid fracture solve: CTAs of the launch
  int gcap = 0;              // grid fracture solve: co-resident CTAs
  std::vector<void*> allocs;
  int64_t bytes = 0;
};

namespace {

// ------------------------------------------------------------- host mesh ---

bool clip_unit(double x0, double y0, double x1, double y1, double* t0o, double* t1o) {
  const double dx = x1 - x0, dy = y1 - y0;
  double t0 = 0.0, t1 = 1.0;
  const double p[4] = {-dx, dx, -dy, dy};
  const double qv[4] = {x0, 1.0 - x0, y0, 1.0 - y0};
  for (int k = 0; k < 4; ++k) {
    if (p[k] == 0.0) {
      if (qv[k] < 0.0) return false;
      continue;
    }
    const double t = qv[k] / p[k];
    if (p[k] < 0.0) t0 = std::max(t0, t);
    else t1 = std::min(t1, t);
    if (t0 >= t1) return false;
  }
  *t0o = t0;
  *t1o = t1;
  return true;
}

struct Seg {
  double x0, y0, x1, y1;
};

bool cross(const Seg& a, const Seg& b, double* s, double* u) {
  const double ax = a.x1 - a.x0, ay = a.y1 - a.y0, bx = b.x1 - b.x0, by = b.y1 - b.y0;
  const double den = ax * by - ay * bx;
  if (den == 0.0) return false;
  const double cx = b.x0 - a.x0, cy = b.y0 - a.y0;
  const double ss = (cx * by - cy * bx) / den;
  const double uu = (cx * ay - cy * ax) / den;
  if (ss >= 0.0 && ss <= 1.0 && uu >= 0.0 && uu <= 1.0) {
    *s = ss;
    *u = uu;
    return true;
  }
  return false;
}

struct Mesh {
  std::vector<double> len, mid;
  std::vector<int> host;
  std::vector<int> segptr;   // pieces of segment s: segptr[s] .. segptr[s+1]-1
  std::vector<std::vector<int>> junctions;
};

std::pair<int, int> root_of(std::map<std::pair<int, int>, std::pair<int, int>>& parent,
                            std::pair<int, int> x) {
  while (true) {
    auto it = parent.find(x);
    if (it == parent.end()) {
      parent[x] = x;
      return x;
    }
    if (it->second == x) return x;
    auto jt = parent.find(it->second);
    if (jt != parent.end()) it->second = jt->second;
    x = it->second;
  }
}

Mesh build_mesh(const double* segs, int nseg, int nx, int ny) {
  const double tol = 1e-12;
  const double h = 1.0 / nx;
  std::vector<Seg> cl;
  for (int k = 0; k < nseg; ++k) {
    const double x0 = segs[4 * k], y0 = segs[4 * k + 1], x1 = segs[4 * k + 2], y1 = segs[4 * k + 3];
    double t0, t1;
    if (!clip_unit(x0, y0, x1, y1, &t0, &t1)) continue;
    Seg e{x0 + t0 * (x1 - x0), y0 + t0 * (y1 - y0), x0 + t1 * (x1 - x0), y0 + t1 * (y1 - y0)};
    if (std::hypot(e.x1 - e.x0, e.y1 - e.y0) > tol) cl.push_back(e);
  }
  const int S = (int)cl.size();
  std::vector<std::vector<double>> brk(S, std::vector<double>{0.0, 1.0});
  struct Cr { int a; double s; int b; double u; };
  std::vector<Cr> crs;
  for (int k = 0; k < S; ++k) {
    const Seg& g = cl[k];
    const double lo[2] = {g.x0, g.y0}, hi[2] = {g.x1, g.y1};
    for (int d = 0; d < 2; ++d) {
      const double dd = hi[d] - lo[d];
      if (dd == 0.0) continue;
      const double a = std::min(lo[d], hi[d]), b = std::max(lo[d], hi[d]);
      const long long g0 = (long long)std::ceil(a / h), g1 = (long long)std::floor(b / h);
      for (long long gg = g0; gg <= g1; ++gg) {
        const double t = ((double)gg * h - lo[d]) / dd;
        if (t > 0.0 && t < 1.0) brk[k].push_back(t);
      }
    }
  }
  for (int a = 0; a < S; ++a)
    for (int b = a + 1; b < S; ++b) {
      double s, u;
      if (cross(cl[a], cl[b], &s, &u)) {
        brk[a].push_back(s);
        brk[b].push_back(u);
        crs.push_back(Cr{a, s, b, u});
      }
    }
  Mesh m;
  std::vector<std::vector<double>> pts(S);
  std::vector<int> first(S);
  for (int k = 0; k < S; ++k) {
    const Seg& g = cl[k];
    const double Lk = std::hypot(g.x1 - g.x0, g.y1 - g.y0);
    std::vector<double> ts = brk[k];
    std::sort(ts.begin(), ts.end());
    std::vector<double> keep{ts[0]};
    for (size_t i = 1; i < ts.size(); ++i)
      if ((ts[i] - keep.back()) * Lk > tol) keep.push_back(ts[i]);
    keep.back() = 1.0;
    pts[k] = keep;
    first[k] = (int)m.len.size();
    m.segptr.push_back(first[k]);
    for (size_t i = 0; i + 1 < keep.size(); ++i) {
      const double t0 = keep[i], t1 = keep[i + 1];
      const double tm = 0.5 * (t0 + t1);
      const double mx = g.x0 + tm * (g.x1 - g.x0), my = g.y0 + tm * (g.y1 - g.y0);
      int ci = (int)std::floor(mx / h), cj = (int)std::floor(my / h);
      ci = std::min(std::max(ci, 0), nx - 1);
      cj = std::min(std::max(cj, 0), ny - 1);
      m.len.push_back((t1 - t0) * Lk);
      m.mid.push_back(mx);
      m.mid.push_back(my);
      m.host.push_back(cj * nx + ci);
    }
  }
  m.segptr.push_back((int)m.len.size());
  auto nearest = [&](int k, double t) {
    const std::vector<double>& ts = pts[k];
    int best = 0;
    double bd = fabs(ts[0] - t);
    for (size_t i = 1; i < ts.size(); ++i)
      if (fabs(ts[i] - t) < bd) { bd = fabs(ts[i] - t); best = (int)i; }
    return best;
  };
  std::map<std::pair<int, int>, std::pair<int, int>> parent;
  for (const Cr& c : crs) {
    const auto ra = root_of(parent, {c.a, nearest(c.a, c.s)});
    const auto rb = root_of(parent, {c.b, nearest(c.b, c.u)});
    if (ra != rb) parent[ra] = rb;
  }
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (int k = 0; k < S; ++k) {
    const int npc = (int)pts[k].size() - 1;
    for (int qi = 0; qi <= npc; ++qi) {
      std::vector<int>& gvec = groups[root_of(parent, {k, qi})];
      if (qi >= 1) gvec.push_back(first[k] + qi - 1);
      if (qi <= npc - 1) gvec.push_back(first[k] + qi);
    }
  }
  for (auto& kv : groups) {
    std::vector<int> g = kv.second;
    std::sort(g.begin(), g.end());
    g.erase(std::unique(g.begin(), g.end()), g.end());
    if (g.size() >= 2) m.junctions.push_back(g);
  }
  return m;
}

// ------------------------------------------------------- set-up kernels ---

__global__ void frac_jsum_kernel(int NJ, const int* jptr, const int* jmem, const double* len, double kf,
                                 double* jsum) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NJ; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = jptr[j]; e < jptr[j + 1]; ++e) s += kf / (0.5 * len[jmem[e]]);
    jsum[j] = s;
  }
}

struct FracCoef {
  int P, L;
  double kf, cf, tau, h;
  double sigma[MCL];
  const int* rowptr;
  const int* col;
  const int* ejct;
  const double* len;
  const double* jsum;
  const double* Wf;
  double* T;
  double* q[MCL];
  double* mf;
  double* dcf;
  double* invdf;
};

// T of every CSR entry (star-delta), masses, exchange, diagonals.
__global__ void frac_coef_kernel(FracCoef g) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < g.P; l += gridDim.x * blockDim.x) {
    const double tl = g.kf / (0.5 * g.len[l]);
    double sT = 0.0;
    for (int e = g.rowptr[l]; e < g.rowptr[l + 1]; ++e) {
      const double tn = g.kf / (0.5 * g.len[g.col[e]]);
      const double v = tl * tn / g.jsum[g.ejct[e]];
      g.T[e] = v;
      sT += v;
    }
    const double m = g.cf * g.len[l];
    double dc = m / g.tau + g.Wf[l];
    for (int a = 0; a < g.L; ++a) {
      const double qa = g.sigma[a] * g.len[l] / (0.25 * g.h);
      g.q[a][l] = qa;
      dc += qa;
    }
    g.mf[l] = m;
    g.dcf[l] = dc;
    g.invdf[l] = 1.0 / (dc + sT);
  }
}

// Line preconditioner of the fracture: block Jacobi whose blocks are the
// tridiagonal rows of each segment's pieces (diagonal: the full diagonal of
// the fracture rows; off-diagonals: -T between consecutive pieces of the
// segment). Thomas elimination without pivoting (the blocks are strictly
// diagonally dominant: the mass and exchange terms lie on the diagonal), one
// thread per segment.
__device__ __forceinline__ double t_between(const int* rowptr, const int* col, const double* T, int l,
                                            int n) {
  for (int e = rowptr[l]; e < rowptr[l + 1]; ++e)
    if (col[e] == n) return T[e];
  return 0.0;
}

__global__ void frac_line_factor_kernel(int NS, const int* segptr, const int* rowptr, const int* col,
                                        const double* T, const double* invdf, double* lo, double* cp,
                                        double* dinv) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < NS; s += gridDim.x * blockDim.x) {
    const int l0 = segptr[s], l1 = segptr[s + 1];
    double cprev = 0.0;
    for (int l = l0; l < l1; ++l) {
      const double d = 1.0 / invdf[l];
      const double a = l > l0 ? -t_between(rowptr, col, T, l, l - 1) : 0.0;
      const double c = l + 1 < l1 ? -t_between(rowptr, col, T, l, l + 1) : 0.0;
      const double den = d - a * cprev;
      const double di = 1.0 / den;
      lo[l] = a;
      cprev = c * di;
      cp[l] = cprev;
      dinv[l] = di;
    }
  }
}

// z = M^-1 r on the pieces l0..l1-1 of one segment, by one warp (all 32 lanes
// call it). Forward substitution y_l = (r_l - lo_l y_{l-1}) dinv_l and back
// substitution z_l = y_l - cp_l z_{l+1} are affine recurrences x_l = a_l +
// b_l x_prev. Lane k owns the contiguous run [k m, (k+1) m) of the segment,
// m = ceil(n / 32): it composes the maps of its run (compose (a2, b2) after
// (a1, b1): (a2 + b2 a1, b2 b1)), an inclusive warp scan of the 32 run maps
// (5 shuffle steps) gives every run its incoming value, and a second walk over
// the run writes the results. Each lane's walk is one dependent FMA chain over
// independent loads, so a long segment costs about 4 m FMA latencies rather
// than a load round trip per 32 pieces. |b_l| < 1 (diagonal dominance), so
// the products only shrink.
__device__ __forceinline__ void line_apply_warp(int l0, int l1, const double* lo, const double* cp,
                                                const double* dinv, const double* r, double* z) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int n = l1 - l0;
  const int m = (n + 31) >> 5;
  const int s0 = l0 + min(n, lane * m), s1 = l0 + min(n, (lane + 1) * m);
  // forward: y_l = A_l + B_l y_{l-1}, A_l = r_l dinv_l, B_l = -lo_l dinv_l
  double a = 0.0, b = 1.0;
#pragma unroll 4
  for (int l = s0; l < s1; ++l) {
    const double di = __ldg(dinv + l);
    a = fma(-__ldg(lo + l) * di, a, __ldcg(r + l) * di);
    b *= -__ldg(lo + l) * di;
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double ap = __shfl_up_sync(full, a, o), bp = __shfl_up_sync(full, b, o);
    if (lane >= o) {
      a = fma(b, ap, a);
      b *= bp;
    }
  }
  double y = __shfl_up_sync(full, a, 1);  // y before the run (0 before the segment)
  if (lane == 0) y = 0.0;
#pragma unroll 4
  for (int l = s0; l < s1; ++l) {
    const double di = __ldg(dinv + l);
    y = fma(-__ldg(lo + l) * di, y, __ldcg(r + l) * di);
    z[l] = y;
  }
  // backward: z_l = y_l + B'_l z_{l+1}, B'_l = -cp_l, walked from the run's end
  a = 0.0;
  b = 1.0;
#pragma unroll 4
  for (int l = s1 - 1; l >= s0; --l) {
    const double bl = -__ldg(cp + l);
    a = fma(bl, a, z[l]);
    b *= bl;
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double ad = __shfl_down_sync(full, a, o), bd = __shfl_down_sync(full, b, o);
    if (lane + o < 32) {
      a = fma(b, ad, a);
      b *= bd;
    }
  }
  double x = __shfl_down_sync(full, a, 1);  // z after the run (0 after the segment)
  if (lane == 31) x = 0.0;
#pragma unroll 4
  for (int l = s1 - 1; l >= s0; --l) {
    x = fma(-__ldg(cp + l), x, z[l]);
    z[l] = x;
  }
  __syncwarp();
}

struct HostArgs {
  int NH, L;
  const int* hcell;
  const int* hptr;
  const int* hpiece;
  const double* q[MCL];
  const double* base[MCL];   // user wells (W or W p_w), or nullptr
  const double* pf;          // nullptr: sum q (the diagonal); else sum q p_f
  double* out[MCL];
};

// Per hosting cell: out = base + sum over its pieces of q (or q p_f), summed
// in piece order (deterministic).
__global__ void frac_host_kernel(HostArgs g) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.NH; c += gridDim.x * blockDim.x) {
    const int cell = g.hcell[c];
    for (int a = 0; a < g.L; ++a) {
      double s = g.base[a] ? g.base[a][cell] : 0.0;
      for (int e = g.hptr[c]; e < g.hptr[c + 1]; ++e) {
        const int l = g.hpiece[e];
        s += g.pf ? g.q[a][l] * g.pf[l] : g.q[a][l];
      }
      g.out[a][cell] = s;
    }
  }
}

// ------------------------------------------------------- fracture solve ---

constexpr int FT = 1024;  // threads of the one-CTA fracture solve

struct FracSolve {
  int P, L, NS;
  const int* segptr;
  const double* llo;
  const double* lcp;
  const double* ldinv;
  const int* rowptr;
  const int* col;
  const double* T;
  const double* dcf;
  const double* invdf;
  const double* mf;
  const double* Ff;
  const double* FWf;
  const double* q[MCL];
  const int* hostp;
  const double* pm[MCL];     // matrix state the exchange reads (p^{n-1} or p^n)
  double* x;                 // p_f: warm start, result
  const double* xprev;       // p_f^{n-1}
  double* r;
  double* z;
  double* p;
  double* qv;
  double* xb;                // right-hand side kept for the constant-mode correction
  double tau, rtol;
  int max_iter;
  int* stat;                 // [0] status, [1] iterations (accumulated)
  double* relres;
};

__device__ __forceinline__ double frac_flux(const FracSolve& A, const double* x, int l, double xl) {
  double s = A.dcf[l] * xl;
  for (int e = A.rowptr[l]; e < A.rowptr[l + 1]; ++e) s += A.T[e] * (xl - x[A.col[e]]);
  return s;
}

__global__ void __launch_bounds__(FT, 1) frac_solve_kernel(const FracSolve A) {
  __shared__ double s_red[(FT / 32) * 3];
  __shared__ double s_res[3];
  const int P = A.P;
  double acc[3] = {0.0, 0.0, 0.0};
  // b, r = b - A x (flux form); b kept in qv for the constant-mode correction
  for (int l = threadIdx.x; l < P; l += FT) {
    double b = A.mf[l] / A.tau * A.xprev[l] + A.Ff[l] + A.FWf[l];
    for (int a = 0; a < A.L; ++a) b += A.q[a][l] * A.pm[a][A.hostp[l]];
    const double rv = b - frac_flux(A, A.x, l, A.x[l]);
    A.r[l] = rv;
    A.qv[l] = b;
    acc[0] += b * b;
    acc[1] += rv * rv;
  }
  __syncthreads();
  // z = M^-1 r (line blocks), p = z, (r, z)
  for (int s = threadIdx.x >> 5; s < A.NS; s += FT / 32)
    line_apply_warp(A.segptr[s], A.segptr[s + 1], A.llo, A.lcp, A.ldinv, A.r, A.z);
  __syncthreads();
  for (int l = threadIdx.x; l < P; l += FT) {
    A.p[l] = A.z[l];
    acc[2] += A.r[l] * A.z[l];
  }
  cta_sum<3>(acc, s_red, s_res);
  // b of the constant-mode correction moves to xb (qv is the PCG's q)
  for (int l = threadIdx.x; l < P; l += FT) A.xb[l] = A.qv[l];
  __syncthreads();
  const double bb = acc[0];
  double rr = acc[1], rz = acc[2];
  const double tol2 = A.rtol * A.rtol;
  int it = 0;
  int status = 0;
  while (rr > tol2 * bb) {
    if (it >= A.max_iter) { status = MC_E_NOCONV; break; }
    double pq[1] = {0.0};
    for (int l = threadIdx.x; l < P; l += FT) {
      const double v = frac_flux(A, A.p, l, A.p[l]);
      A.qv[l] = v;
      pq[0] += A.p[l] * v;
    }
    cta_sum<1>(pq, s_red, s_res);
    if (!(pq[0] > 0.0) || !isfinite(pq[0])) { status = MC_E_BREAKDOWN; break; }
    const double al = rz / pq[0];
    double d2[2] = {0.0, 0.0};
    for (int l = threadIdx.x; l < P; l += FT) {
      A.x[l] += al * A.p[l];
      const double rv = A.r[l] - al * A.qv[l];
      A.r[l] = rv;
      d2[0] += rv * rv;
    }
    __syncthreads();
    for (int s = threadIdx.x >> 5; s < A.NS; s += FT / 32)
      line_apply_warp(A.segptr[s], A.segptr[s + 1], A.llo, A.lcp, A.ldinv, A.r, A.z);
    __syncthreads();
    for (int l = threadIdx.x; l < P; l += FT) d2[1] += A.r[l] * A.z[l];
    cta_sum<2>(d2, s_red, s_res);
    ++it;
    rr = d2[0];
    if (!isfinite(rr)) { status = MC_E_BREAKDOWN; break; }
    const double bt = d2[1] / rz;
    rz = d2[1];
    for (int l = threadIdx.x; l < P; l += FT) A.p[l] = A.z[l] + bt * A.p[l];
    __syncthreads();
  }
  // constant-mode correction: c = 1^T (b - A x) / 1^T dcf (the T terms cancel)
  if (status == 0) {
    double cs[2] = {0.0, 0.0};
    for (int l = threadIdx.x; l < P; l += FT) {
      cs[0] += A.xb[l] - A.dcf[l] * A.x[l];
      cs[1] += A.dcf[l];
    }
    cta_sum<2>(cs, s_red, s_res);
    const double c = cs[1] > 0.0 ? cs[0] / cs[1] : 0.0;
    if (isfinite(c))
      for (int l = threadIdx.x; l < P; l += FT) A.x[l] += c;
  }
  if (threadIdx.x == 0) {
    if (status) atomicCAS(A.stat, 0, status);
    A.stat[1] += it;
    *A.relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
  }
}

__global__ void frac_wp_kernel(int P, const double* W, double* FW) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < P; l += gridDim.x * blockDim.x)
    FW[l] = W[l] * FW[l];
}

cudaError_t falloc(mc_frac* f, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return e;
  f->allocs.push_back(*p);
  f->bytes += (int64_t)bytes;
  return cudaMemsetAsync(*p, 0, bytes, f->ctx->stream);
}

void ffree(mc_frac* f) {
  for (void* p : f->allocs) cudaFree(p);
  f->allocs.clear();
}

mc_status ferr(mc_frac* f, mc_status s, const std::string& msg) {
  if (f && f->ctx) f->ctx->err = msg;
  return s;
}

int grid256(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 4096) b = 4096;
  return (int)b;
}

cudaError_t launch_host(mc_frac* f, const double* const* base, const double* pf, double* const* out) {
  if (f->NH == 0) return cudaSuccess;
  HostArgs g{};
  g.NH = f->NH;
  g.L = f->L;
  g.hcell = f->hcell;
  g.hptr = f->hptr;
  g.hpiece = f->hpiece;
  for (int a = 0; a < f->L; ++a) {
    g.q[a] = f->q[a];
    g.base[a] = base[a];
    g.out[a] = out[a];
  }
  g.pf = pf;
  frac_host_kernel<<<grid256(f->NH), 256, 0, f->ctx->stream>>>(g);
  return cudaGetLastError();
}

// Matrix step (one time step) with the fracture exchange as a diagonal term.
mc_status matrix_step(mc_frac* f, int scheme, mc_stats* st) {
  mc_ctx* ctx = f->ctx;
  StepParams sp;
  mc_fill_params(ctx, &sp, scheme, 1);
  for (int a = 0; a < f->L; ++a) {
    sp.W[a] = f->Wm[a];
    sp.FW[a] = f->FWm[a];
    sp.diagc[a] = f->diagc[a];
    sp.invd[a] = f->invd[a];
    sp.sqd[a] = f->sqd[a];
    sp.tE[a] = f->tE[a];
    sp.tN[a] = f->tN[a];
    for (int b = 0; b < f->L; ++b) sp.qs[a][b] = f->qs[a][b];
  }
  cudaStream_t s = ctx->stream;
  if (cudaMemsetAsync(ctx->bar, 0, 96 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(ctx->dstatus, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(ctx->dsteps, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(ctx->diters, 0, MCL * sizeof(long long), s) != cudaSuccess ||
      cudaMemsetAsync(ctx->dmaxit, 0, MCL * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(ctx->dmass, 0, sizeof(double), s) != cudaSuccess)
    return ferr(f, MC_E_CUDA, "fracture step: memset");
  if (mc_launch_steps_default(ctx, sp) != cudaSuccess) return ferr(f, MC_E_CUDA, "fracture step: matrix launch");
  int stt = 0;
  long long its[MCL] = {};
  int mx[MCL] = {};
  double rel[MCL] = {};
  if (cudaMemcpyAsync(&stt, ctx->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(its, ctx->diters, sizeof(its), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(mx, ctx->dmaxit, sizeof(mx), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(rel, ctx->drelres, sizeof(rel), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ferr(f, MC_E_CUDA, "fracture step: matrix status");
  for (int a = 0; a < f->L; ++a) {
    st->iters[a] += its[a];
    if (mx[a] > st->max_iters[a]) st->max_iters[a] = mx[a];
    st->rel_residual[a] = rel[a];
  }
  if (stt != 0) return ferr(f, (mc_status)stt, std::string("matrix solve: ") + mc_status_string((mc_status)stt));
  return MC_OK;
}

// Networks of at least this many pieces take the fracture solve over a
// cooperative grid (frac_solve_grid_kernel); smaller ones the one-CTA kernel,
// whose CTA barriers are cheaper than grid barriers.
constexpr int FRAC_GRID_MIN_PIECES = 8192;

mc_status frac_solve_grid(mc_frac* f, const FracSolve& A);

mc_status frac_solve(mc_frac* f, double* const* pm, mc_stats* st) {
  mc_ctx* ctx = f->ctx;
  cudaStream_t s = ctx->stream;
  FracSolve A{};
  A.P = f->P;
  A.L = f->L;
  A.rowptr = f->rowptr;
  A.col = f->col;
  A.T = f->T;
  A.dcf = f->dcf;
  A.invdf = f->invdf;
  A.mf = f->mf;
  A.Ff = f->Ff;
  A.FWf = f->FWf;
  for (int a = 0; a < f->L; ++a) {
    A.q[a] = f->q[a];
    A.pm[a] = pm[a];
  }
  A.hostp = f->hostp;
  A.x = f->pf;
  A.xprev = f->pf_prev;
  A.r = f->r;
  A.z = f->z;
  A.p = f->pp;
  A.qv = f->qq;
  A.xb = f->bf;
  A.NS = f->NS;
  A.segptr = f->segptr;
  A.llo = f->llo;
  A.lcp = f->lcp;
  A.ldinv = f->ldinv;
  A.tau = ctx->tau;
  A.rtol = ctx->opts.rtol;
  A.max_iter = ctx->opts.max_iter;
  A.stat = f->dstat;
  A.relres = f->drel;
  if (cudaMemsetAsync(f->dstat, 0, 2 * sizeof(int), s) != cudaSuccess) return ferr(f, MC_E_CUDA, "memset");
  if (f->P >= FRAC_GRID_MIN_PIECES) {
    const mc_status gs = frac_solve_grid(f, A);
    if (gs != MC_OK) return gs;
  } else {
    frac_solve_kernel<<<1, FT, 0, s>>>(A);
    if (cudaGetLastError() != cudaSuccess) return ferr(f, MC_E_CUDA, "fracture solve launch");
  }
  int ss[2] = {0, 0};
  double rel = 0.0;
  if (cudaMemcpyAsync(ss, f->dstat, sizeof(ss), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&rel, f->drel, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ferr(f, MC_E_CUDA, "fracture solve status");
  const int k = f->L;
  st->iters[k] += ss[1];
  if (ss[1] > st->max_iters[k]) st->max_iters[k] = ss[1];
  st->rel_residual[k] = rel;
  if (ss[0] != 0) return ferr(f, (mc_status)ss[0], std::string("fracture solve: ") + mc_status_string((mc_status)ss[0]));
  return MC_OK;
}

mc_status coupled_step(mc_frac* f, mc_stats* st);

}  // namespace

extern "C" {

mc_status mc_frac_create(mc_ctx* ctx, int32_t nseg, const double* seg, double kf, double cf,
                         const double* sigma_f, mc_frac** out) {
  if (!ctx || !out) return MC_E_ARG;
  *out = nullptr;
  if (nseg < 1 || !seg || !sigma_f) {
    ctx->err = "mc_frac_create: segments and sigma_f are required";
    return MC_E_ARG;
  }
  if (!(kf > 0.0) || !isfinite(kf) || !(cf > 0.0) || !isfinite(cf)) {
    ctx->err = "mc_frac_create: kf and cf must be > 0 and finite";
    return MC_E_ARG;
  }
  if (ctx->L + 1 > MCL) {
    ctx->err = "mc_frac_create: at most MC_MAX_CONTINUA - 1 matrix continua";
    return MC_E_ARG;
  }
  if (ctx->nx != ctx->ny) {
    ctx->err = "mc_frac_create: the unit square needs nx == ny";
    return MC_E_ARG;
  }
  for (int k = 0; k < 4 * nseg; ++k)
    if (!isfinite(seg[k])) {
      ctx->err = "mc_frac_create: segment coordinates must be finite";
      return MC_E_ARG;
    }
  for (int a = 0; a < ctx->L; ++a)
    if (!(sigma_f[a] >= 0.0) || !isfinite(sigma_f[a])) {
      ctx->err = "mc_frac_create: sigma_f must be >= 0 and finite";
      return MC_E_ARG;
    }
  if (ctx->opts.precision != MC_PREC_FP64 || ctx->opts.precond != MC_PRECOND_JACOBI) {
    ctx->err = "mc_frac_create: the context must use FP64 with the Jacobi preconditioner";
    return MC_E_ARG;
  }
  Mesh mesh = build_mesh(seg, nseg, ctx->nx, ctx->ny);
  if (mesh.len.empty()) {
    ctx->err = "mc_frac_create: no segment crosses the domain";
    return MC_E_ARG;
  }
  mc_frac* f = new (std::nothrow) mc_frac();
  if (!f) return MC_E_ALLOC;
  f->ctx = ctx;
  f->L = ctx->L;
  f->P = (int)mesh.len.size();
  f->kf = kf;
  f->cf = cf;
  for (int a = 0; a < ctx->L; ++a) f->sigma_f[a] = sigma_f[a];
  f->len = mesh.len;
  f->mid = mesh.mid;
  f->host = mesh.host;
  const int P = f->P, L = f->L;
  // CSR of the fracture graph (entries: the other members of each junction)
  std::vector<std::vector<std::pair<int, int>>> rows(P);
  std::vector<int> jptr{0}, jmem;
  for (size_t j = 0; j < mesh.junctions.size(); ++j) {
    const std::vector<int>& g = mesh.junctions[j];
    for (int l : g) {
      jmem.push_back(l);
      for (int n : g)
        if (n != l) rows[l].push_back({n, (int)j});
    }
    jptr.push_back((int)jmem.size());
  }
  std::vector<int> rowptr{0}, col, ejct;
  for (int l = 0; l < P; ++l) {
    std::sort(rows[l].begin(), rows[l].end());
    for (auto& e : rows[l]) {
      col.push_back(e.first);
      ejct.push_back(e.second);
    }
    rowptr.push_back((int)col.size());
  }
  f->nnz = (int)col.size();
  f->NJ = (int)mesh.junctions.size();
  // hosting cells (pitched), pieces grouped by cell in piece order
  std::map<int, std::vector<int>> byc;
  std::vector<int> hostp(P);
  for (int l = 0; l < P; ++l) {
    const int c = mesh.host[l];
    const int pc = (c / ctx->nx) * ctx->pitch + c % ctx->nx;
    hostp[l] = pc;
    byc[pc].push_back(l);
  }
  std::vector<int> hcell, hptr{0}, hpiece;
  for (auto& kv : byc) {
    hcell.push_back(kv.first);
    for (int l : kv.second) hpiece.push_back(l);
    hptr.push_back((int)hpiece.size());
  }
  f->NH = (int)hcell.size();
  cudaStream_t st = ctx->stream;
  auto bail = [&](mc_status s, const std::string& msg) {
    ctx->err = msg;
    ffree(f);
    delete f;
    return s;
  };
  cudaError_t e;
#define FK(x)                                                                   \
  do {                                                                          \
    e = (x);                                                                    \
    if (e != cudaSuccess)                                                       \
      return bail(e == cudaErrorMemoryAllocation ? MC_E_ALLOC : MC_E_CUDA,      \
                  std::string(#x) + ": " + cudaGetErrorString(e));              \
  } while (0)
  FK(cudaSetDevice(ctx->device));
  auto up_i = [&](int** d, const std::vector<int>& v) -> cudaError_t {
    cudaError_t ee = falloc(f, (void**)d, v.size() * sizeof(int));
    if (ee != cudaSuccess || v.empty()) return ee;
    return cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  };
  FK(up_i(&f->rowptr, rowptr));
  FK(up_i(&f->col, col));
  FK(up_i(&f->ejct, ejct));
  FK(up_i(&f->jptr, jptr));
  FK(up_i(&f->jmem, jmem));
  FK(up_i(&f->hcell, hcell));
  FK(up_i(&f->hptr, hptr));
  FK(up_i(&f->hpiece, hpiece));
  FK(up_i(&f->hostp, hostp));
  const size_t pb = (size_t)P * sizeof(double);
  FK(falloc(f, (void**)&f->len_d, pb));
  FK(cudaMemcpyAsync(f->len_d, mesh.len.data(), pb, cudaMemcpyHostToDevice, st));
  FK(falloc(f, (void**)&f->jsum, (size_t)(f->NJ > 0 ? f->NJ : 1) * sizeof(double)));
  FK(falloc(f, (void**)&f->T, (size_t)(f->nnz > 0 ? f->nnz : 1) * sizeof(double)));
  for (int a = 0; a < L; ++a) FK(falloc(f, (void**)&f->q[a], pb));
  for (double** p : {&f->mf, &f->dcf, &f->invdf, &f->Ff, &f->Wf, &f->FWf, &f->pf, &f->pf_prev, &f->r,
                     &f->z, &f->pp, &f->qq, &f->bf, &f->llo, &f->lcp, &f->ldinv})
    FK(falloc(f, (void**)p, pb));
  f->NS = (int)mesh.segptr.size() - 1;
  FK(up_i(&f->segptr, mesh.segptr));
  FK(falloc(f, (void**)&f->dstat, 4 * sizeof(int)));
  FK(falloc(f, (void**)&f->drel, 2 * sizeof(double)));
  const size_t fb = (size_t)ctx->Np * sizeof(double);
  for (int a = 0; a < L; ++a) {
    for (double** p : {&f->Wm[a], &f->FWm[a], &f->diagc[a], &f->invd[a], &f->sqd[a], &f->tE[a], &f->tN[a]})
      FK(falloc(f, (void**)p, fb));
    for (int b = a + 1; b < L; ++b) {
      FK(falloc(f, (void**)&f->qs[a][b], fb));
      f->qs[b][a] = f->qs[a][b];
    }
  }
  *out = f;
  // coefficients (also redone by mc_frac_set_well)
  mc_status s = mc_frac_set_well(f, nullptr, nullptr);
  if (s != MC_OK) {
    *out = nullptr;
    ffree(f);
    delete f;
    return s;
  }
#undef FK
  return MC_OK;
}

mc_status mc_frac_set_well(mc_frac* f, const double* Wf, const double* pwf) {
  if (!f) return MC_E_ARG;
  mc_ctx* ctx = f->ctx;
  cudaStream_t st = ctx->stream;
  const int P = f->P, L = f->L;
  const size_t pb = (size_t)P * sizeof(double);
  if (Wf) {
    if (!pwf) return ferr(f, MC_E_ARG, "pwf is NULL");
    for (int l = 0; l < P; ++l)
      if (!(Wf[l] >= 0.0) || !isfinite(Wf[l]) || !isfinite(pwf[l]))
        return ferr(f, MC_E_ARG, "fracture wells must be finite, W >= 0");
    std::vector<double> fw(P);
    for (int l = 0; l < P; ++l) fw[l] = pwf[l];
    if (cudaMemcpyAsync(f->Wf, Wf, pb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(f->FWf, fw.data(), pb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ferr(f, MC_E_CUDA, "fracture wells upload");
    frac_wp_kernel<<<grid256(P), 256, 0, st>>>(P, f->Wf, f->FWf);  // FWf = W p_w
    if (cudaGetLastError() != cudaSuccess) return ferr(f, MC_E_CUDA, "fracture wells");
  } else if (cudaMemsetAsync(f->Wf, 0, pb, st) != cudaSuccess ||
             cudaMemsetAsync(f->FWf, 0, pb, st) != cudaSuccess) {
    return ferr(f, MC_E_CUDA, "fracture wells clear");
  }
  // coefficients
  if (f->NJ > 0) {
    frac_jsum_kernel<<<grid256(f->NJ), 256, 0, st>>>(f->NJ, f->jptr, f->jmem, f->len_d, f->kf, f->jsum);
    if (cudaGetLastError() != cudaSuccess) return ferr(f, MC_E_CUDA, "jsum");
  }
  FracCoef g{};
  g.P = P;
  g.L = L;
  g.kf = f->kf;
  g.cf = f->cf;
  g.tau = ctx->tau;
  g.h = ctx->h;
  for (int a = 0; a < L; ++a) {
    g.sigma[a] = f->sigma_f[a];
    g.q[a] = f->q[a];
  }
  g.rowptr = f->rowptr;
  g.col = f->col;
  g.ejct = f->ejct;
  g.len = f->len_d;
  g.jsum = f->jsum;
  g.Wf = f->Wf;
  g.T = f->T;
  g.mf = f->mf;
  g.dcf = f->dcf;
  g.invdf = f->invdf;
  frac_coef_kernel<<<grid256(P), 256, 0, st>>>(g);
  if (cudaGetLastError() != cudaSuccess) return ferr(f, MC_E_CUDA, "fracture coefficients");
  frac_line_factor_kernel<<<grid256(f->NS), 256, 0, st>>>(f->NS, f->segptr, f->rowptr, f->col, f->T,
                                                          f->invdf, f->llo, f->lcp, f->ldinv);
  if (cudaGetLastError() != cudaSuccess) return ferr(f, MC_E_CUDA, "fracture line factors");
  // matrix side: W = user wells + hosted exchange; FW starts as the user's W p_w
  for (int a = 0; a < L; ++a) {
    if (ctx->W[a]) {
      if (cudaMemcpyAsync(f->Wm[a], ctx->W[a], ctx->Np * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(f->FWm[a], ctx->FW[a], ctx->Np * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
              cudaSuccess)
        return ferr(f, MC_E_CUDA, "matrix wells copy");
    } else if (cudaMemsetAsync(f->Wm[a], 0, ctx->Np * sizeof(double), st) != cudaSuccess ||
               cudaMemsetAsync(f->FWm[a], 0, ctx->Np * sizeof(double), st) != cudaSuccess) {
      return ferr(f, MC_E_CUDA, "matrix wells clear");
    }
  }
  const double* base[MCL] = {};
  for (int a = 0; a < L; ++a) base[a] = ctx->W[a];
  if (launch_host(f, base, nullptr, f->Wm) != cudaSuccess) return ferr(f, MC_E_CUDA, "hosted exchange");
  for (int a = 0; a < L; ++a)
    if (mc_launch_diag_into(ctx, a, f->Wm[a], f->diagc[a], f->invd[a], f->sqd[a], f->tE[a], f->tN[a]) !=
        cudaSuccess)
      return ferr(f, MC_E_CUDA, "matrix diagonal");
  if (mc_launch_pairs_into(ctx, f->sqd, f->qs) != cudaSuccess) return ferr(f, MC_E_CUDA, "matrix pairs");
  if (cudaStreamSynchronize(st) != cudaSuccess) return ferr(f, MC_E_CUDA, "fracture set-up");
  return MC_OK;
}

mc_status mc_frac_info(const mc_frac* f, int64_t* info) {
  if (!f || !info) return MC_E_ARG;
  info[0] = f->P;
  info[1] = f->NJ;
  info[2] = f->nnz;
  info[3] = f->NH;
  info[4] = f->bytes;
  return MC_OK;
}

mc_status mc_frac_pieces(const mc_frac* f, double* len, double* mid, int32_t* host) {
  if (!f) return MC_E_ARG;
  for (int l = 0; l < f->P; ++l) {
    if (len) len[l] = f->len[l];
    if (mid) {
      mid[2 * l] = f->mid[2 * l];
      mid[2 * l + 1] = f->mid[2 * l + 1];
    }
    if (host) host[l] = f->host[l];
  }
  return MC_OK;
}

mc_status mc_frac_set_source(mc_frac* f, const double* Ff) {
  if (!f || !Ff) return MC_E_ARG;
  for (int l = 0; l < f->P; ++l)
    if (!isfinite(Ff[l])) return ferr(f, MC_E_ARG, "fracture sources must be finite");
  cudaStream_t st = f->ctx->stream;
  if (cudaMemcpyAsync(f->Ff, Ff, (size_t)f->P * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ferr(f, MC_E_CUDA, "fracture source upload");
  return MC_OK;
}

mc_status mc_frac_set_state(mc_frac* f, const double* const* pm, const double* pf) {
  if (!f) return MC_E_ARG;
  if (pm) {
    const mc_status s = mc_set_state(f->ctx, pm);
    if (s != MC_OK) return s;
  }
  if (pf) {
    cudaStream_t st = f->ctx->stream;
    if (cudaMemcpyAsync(f->pf, pf, (size_t)f->P * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ferr(f, MC_E_CUDA, "fracture state upload");
  }
  return MC_OK;
}

mc_status mc_frac_get_state(mc_frac* f, double* const* pm, double* pf) {
  if (!f) return MC_E_ARG;
  if (pm) {
    const mc_status s = mc_get_state(f->ctx, pm);
    if (s != MC_OK) return s;
  }
  if (pf) {
    cudaStream_t st = f->ctx->stream;
    if (cudaMemcpyAsync(pf, f->pf, (size_t)f->P * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return ferr(f, MC_E_CUDA, "fracture state download");
  }
  return MC_OK;
}

mc_status mc_frac_step(mc_frac* f, int32_t scheme, int32_t nsteps, mc_stats* stats) {
  mc_stats st;
  memset(&st, 0, sizeof(st));
  if (stats) memset(stats, 0, sizeof(*stats));
  if (!f) return MC_E_ARG;
  if (scheme != MC_SCHEME_COUPLED && scheme != MC_SCHEME_D && scheme != MC_SCHEME_L &&
      scheme != MC_SCHEME_U)
    return ferr(f, MC_E_ARG, "bad scheme");
  if (nsteps < 0) return MC_E_ARG;
  mc_ctx* ctx = f->ctx;
  cudaStream_t s = ctx->stream;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MC_E_CUDA;
  const int L = f->L;
  const size_t pb = (size_t)f->P * sizeof(double);
  const double* base[MCL] = {};
  for (int a = 0; a < L; ++a) base[a] = ctx->FW[a];
  mc_status rs = MC_OK;
  for (int n = 0; n < nsteps && rs == MC_OK; ++n) {
    // snapshot of the step's start (p^{n-1}) for the exchange and for rollback
    if (cudaMemcpyAsync(f->pf_prev, f->pf, pb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      rs = ferr(f, MC_E_CUDA, "fracture snapshot");
      break;
    }
    for (int a = 0; a < L; ++a)
      if (cudaMemcpyAsync(ctx->pprev[a], ctx->p[a], ctx->Np * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
        rs = ferr(f, MC_E_CUDA, "matrix snapshot");
    if (rs != MC_OK) break;
    if (scheme == MC_SCHEME_COUPLED) {
      rs = coupled_step(f, &st);
    } else if (scheme == MC_SCHEME_U) {
      // fracture first from p_m^{n-1}, then the matrix from p_f^n
      rs = frac_solve(f, ctx->p, &st);
      if (rs == MC_OK && launch_host(f, base, f->pf, f->FWm) != cudaSuccess) rs = ferr(f, MC_E_CUDA, "exchange");
      if (rs == MC_OK) rs = matrix_step(f, MC_SCHEME_U, &st);
    } else {
      if (launch_host(f, base, f->pf_prev, f->FWm) != cudaSuccess) rs = ferr(f, MC_E_CUDA, "exchange");
      if (rs == MC_OK) rs = matrix_step(f, scheme, &st);
      if (rs == MC_OK) rs = frac_solve(f, scheme == MC_SCHEME_D ? ctx->pprev : ctx->p, &st);
    }
    if (rs == MC_OK) ++st.steps_done;
  }
  if (rs != MC_OK) {
    // back to the start of the failed step
    for (int a = 0; a < L; ++a)
      cudaMemcpyAsync(ctx->p[a], ctx->pprev[a], ctx->Np * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(f->pf, f->pf_prev, pb, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    st.status = rs;
  }
  if (stats) *stats = st;
  return rs;
}

void mc_frac_destroy(mc_frac* f) {
  if (!f) return;
  cudaSetDevice(f->ctx->device);
  cudaStreamSynchronize(f->ctx->stream);
  ffree(f);
  delete f;
}

}  // extern "C"

namespace {

// ------------------------------------------------ coupled scheme (Eq. ct-mc) ---
// One cooperative launch per time step: Jacobi PCG on the whole system (every
// matrix continuum's cells and every piece), flux-form operator
//   matrix a, cell i: (m/tau + W) x + sum_faces T (x - x_n)
//                     + sum_b q_ab (x_a - x_b) + sum_hosted q_al (x_a - x_f,l)
//   piece l:          (m_f/tau + W_f) x + sum_n T_ln (x_l - x_n)
//                     + sum_a q_al (x_l - x_a,host)
// with P_new = z + beta P_old formed on the fly at every point the operator
// reads (two grid reductions per iteration), then the constant-mode
// correction per continuum (an (L+1) x (L+1) Galerkin system, as in the
// co-located coupled kernel).

constexpr int CT = 256;
constexpr int CQ = 4 * MCL + 8;   // partial-sum quantities per slot

struct CoupledArgs {
  StepParams sp;                  // matrix continua (TE, TN, F, p, pprev, r, z, P, q, W, FW, ...)
  int P, NH, NS;
  const int* segptr;              // fracture line blocks (as the decoupled fracture solve)
  const double* llo;
  const double* lcp;
  const double* ldinv;
  const int* rowptr;
  const int* col;
  const double* T;
  const double* mf;
  const double* dcf;              // m_f/tau + sum_a q + W_f
  const double* invdf;
  const double* Ff;
  const double* FWf;
  const double* Wf;
  const double* q[MCL];
  const int* hostp;
  const int* hidx;                // per pitched matrix cell: hosting-cell list index or -1
  const int* hptr;
  const int* hpiece;
  const double* hsum[MCL];        // per pitched matrix cell: sum of hosted q_al
  const double* invdm[MCL];       // Jacobi inverse of the coupled matrix rows
  double* xf;
  const double* xf_prev;
  double* rf;
  double* zf;
  double* Pf[2];
  double* qf;
  double* partials;               // [2][CQ][gridDim.x]
  GridBar bar;
  int* stat;                      // [0] status, [2] iterations
  double* relres;
};

__device__ __forceinline__ double cq(const StepParams& sp, int a, int b, long long i) {
  const double* c = sp.qcell[a][b];
  return c ? __ldg(c + i) : sp.qconst[a][b];
}

// store this CTA's NQ sums (deterministic CTA reduction) into slot s
template <int NQ>
__device__ void cstore(double (&v)[NQ], double* part, int slot) {
  __shared__ double s_red[(CT / 32) * NQ];
  __shared__ double s_res[NQ];
  cta_sum<NQ>(v, s_red, s_res);
  if (threadIdx.x < NQ) part[((size_t)slot * CQ + threadIdx.x) * gridDim.x + blockIdx.x] = v[threadIdx.x];
}

template <int NQ>
__device__ void ctotal(const double* part, int slot, double (&out)[NQ]) {
  __shared__ double s_tot[NQ];
  if (threadIdx.x < NQ) {
    double s = 0.0;
    const double* src = part + ((size_t)slot * CQ + threadIdx.x) * gridDim.x;
    for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(src + b);
    s_tot[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NQ; ++k) out[k] = s_tot[k];
  __syncthreads();
}

// P value of a matrix point / piece on the fly: z + beta P_old
__device__ __forceinline__ double pm_of(const CoupledArgs& A, int cur, int a, long long i, double bt) {
  return fma(bt, __ldcg(A.sp.P[cur][a] + i), __ldcg(A.sp.z[a] + i));
}
__device__ __forceinline__ double pf_of(const CoupledArgs& A, int cur, int l, double bt) {
  return fma(bt, __ldcg(A.Pf[cur] + l), __ldcg(A.zf + l));
}

// row of the operator at matrix point (a, i) applied to v (a function of (b, i)
// and the pieces)
template <int L, typename FM, typename FF>
__device__ __forceinline__ double mrow(const CoupledArgs& A, int a, long long i, int gx, int gy, double xc,
                                       FM vm, FF vf) {
  const StepParams& sp = A.sp;
  const int pitch = sp.pitch;
  double s = sp.mtau[a] * xc;
  if (sp.W[a]) s += __ldg(sp.W[a] + i) * xc;
  if (gx + 1 < sp.nx) s += __ldg(sp.TE[a] + i) * (xc - vm(a, i + 1));
  if (gx > 0) s += __ldg(sp.TE[a] + i - 1) * (xc - vm(a, i - 1));
  if (gy + 1 < sp.ny) s += __ldg(sp.TN[a] + i) * (xc - vm(a, i + pitch));
  if (gy > 0) s += __ldg(sp.TN[a] + i - pitch) * (xc - vm(a, i - pitch));
#pragma unroll
  for (int b = 0; b < L; ++b)
    if (b != a) s += cq(sp, a, b, i) * (xc - vm(b, i));
  const int c = __ldg(A.hidx + i);
  if (c >= 0)
    for (int e = A.hptr[c]; e < A.hptr[c + 1]; ++e) {
      const int l = A.hpiece[e];
      s += A.q[a][l] * (xc - vf(l));
    }
  return s;
}

template <int L, typename FM, typename FF>
__device__ __forceinline__ double frow(const CoupledArgs& A, int l, double xl, FM vm, FF vf) {
  double s = (A.mf[l] / A.sp.tau + A.Wf[l]) * xl;
  for (int e = A.rowptr[l]; e < A.rowptr[l + 1]; ++e) s += A.T[e] * (xl - vf(A.col[e]));
#pragma unroll
  for (int a = 0; a < L; ++a) s += A.q[a][l] * (xl - vm(a, (long long)A.hostp[l]));
  return s;
}

template <int L>
__global__ void __launch_bounds__(CT) frac_coupled_kernel(const __grid_constant__ CoupledArgs A) {
  const StepParams& sp = A.sp;
  const int nx = sp.nx, pitch = sp.pitch;
  const long long Np = sp.Np;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  const int P = A.P;
  // ---- right-hand side and initial residual (flux form): bb, rr, rz -------
  double acc[3] = {0.0, 0.0, 0.0};
  auto xm = [&](int b, long long i) { return __ldcg(sp.p[b] + i); };
  auto xfv = [&](int l) { return __ldcg(A.xf + l); };
  for (int a = 0; a < L; ++a)
    for (long long i = gt; i < Np; i += gs) {
      const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
      if (gx >= nx) continue;
      const double xc = xm(a, i);
      double b = sp.mtau[a] * __ldcg(sp.pprev[a] + i) + __ldg(sp.F[a] + i);
      if (sp.FW[a]) b += __ldg(sp.FW[a] + i);
      const double rv = b - mrow<L>(A, a, i, gx, gy, xc, xm, xfv);
      const double zv = A.invdm[a][i] * rv;
      sp.r[a][i] = rv;
      sp.z[a][i] = zv;
      sp.P[0][a][i] = 0.0;
      acc[0] += b * b;
      acc[1] += rv * rv;
      acc[2] += rv * zv;
    }
  // fracture rows by segment (one warp each): residual, then the line block
  const int lane = threadIdx.x & 31;
  const long long gwarp = gt >> 5, nwarp = gs >> 5;
  for (long long s = gwarp; s < A.NS; s += nwarp) {
    const int l0 = A.segptr[s], l1 = A.segptr[s + 1];
    for (int l = l0 + lane; l < l1; l += 32) {
      const double xl = xfv(l);
      const double b = A.mf[l] / sp.tau * A.xf_prev[l] + A.Ff[l] + A.FWf[l];
      const double rv = b - frow<L>(A, l, xl, xm, xfv);
      A.rf[l] = rv;
      A.Pf[0][l] = 0.0;
      acc[0] += b * b;
      acc[1] += rv * rv;
    }
    __syncwarp();
    line_apply_warp(l0, l1, A.llo, A.lcp, A.ldinv, A.rf, A.zf);
    for (int l = l0 + lane; l < l1; l += 32) acc[2] += A.rf[l] * A.zf[l];
  }
  cstore<3>(acc, A.partials, 0);
  if (!grid_barrier(A.bar)) return;
  double tot3[3];
  ctotal<3>(A.partials, 0, tot3);
  const double bb = tot3[0];
  double rr = tot3[1], rz = tot3[2];
  const double tol2 = sp.rtol * sp.rtol;
  double beta = 0.0;
  int it = 0, cur = 0, slot = 1, status = 0;
  while (rr > tol2 * bb) {
    if (it >= sp.max_iter) { status = MC_E_NOCONV; break; }
    // ---- P_new = z + beta P_old (stored), q = A P_new, <P_new, q> ----------
    const double bt = beta;
    auto pmv = [&](int b, long long i) { return pm_of(A, cur, b, i, bt); };
    auto pfv = [&](int l) { return pf_of(A, cur, l, bt); };
    double pq[1] = {0.0};
    for (int a = 0; a < L; ++a)
      for (long long i = gt; i < Np; i += gs) {
        const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
        if (gx >= nx) continue;
        const double pc = pmv(a, i);
        const double qv = mrow<L>(A, a, i, gx, gy, pc, pmv, pfv);
        sp.P[cur ^ 1][a][i] = pc;
        sp.q[a][i] = qv;
        pq[0] = fma(pc, qv, pq[0]);
      }
    for (long long l = gt; l < P; l += gs) {
      const double pc = pfv((int)l);
      const double qv = frow<L>(A, (int)l, pc, pmv, pfv);
      A.Pf[cur ^ 1][l] = pc;
      A.qf[l] = qv;
      pq[0] = fma(pc, qv, pq[0]);
    }
    cstore<1>(pq, A.partials, slot);
    if (!grid_barrier(A.bar)) return;
    double pqt[1];
    ctotal<1>(A.partials, slot, pqt);
    slot ^= 1;
    if (!(pqt[0] > 0.0) || !isfinite(pqt[0])) { status = MC_E_BREAKDOWN; break; }
    const double al = rz / pqt[0];
    // ---- x += al P, r -= al q, z = M^-1 r, (r, r), (r, z) --------------------
    double d2[2] = {0.0, 0.0};
    for (int a = 0; a < L; ++a)
      for (long long i = gt; i < Np; i += gs) {
        const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
        if (gx >= nx) continue;
        sp.p[a][i] = __ldcg(sp.p[a] + i) + al * __ldcg(sp.P[cur ^ 1][a] + i);
        const double rv = __ldcg(sp.r[a] + i) - al * __ldcg(sp.q[a] + i);
        const double zv = A.invdm[a][i] * rv;
        sp.r[a][i] = rv;
        sp.z[a][i] = zv;
        d2[0] += rv * rv;
        d2[1] += rv * zv;
      }
    for (long long s = gwarp; s < A.NS; s += nwarp) {
      const int l0 = A.segptr[s], l1 = A.segptr[s + 1];
      for (int l = l0 + lane; l < l1; l += 32) {
        A.xf[l] = __ldcg(A.xf + l) + al * __ldcg(A.Pf[cur ^ 1] + l);
        const double rv = __ldcg(A.rf + l) - al * __ldcg(A.qf + l);
        A.rf[l] = rv;
        d2[0] += rv * rv;
      }
      __syncwarp();
      line_apply_warp(l0, l1, A.llo, A.lcp, A.ldinv, A.rf, A.zf);
      for (int l = l0 + lane; l < l1; l += 32) d2[1] += A.rf[l] * A.zf[l];
    }
    cstore<2>(d2, A.partials, slot);
    if (!grid_barrier(A.bar)) return;
    double t2[2];
    ctotal<2>(A.partials, slot, t2);
    slot ^= 1;
    ++it;
    rr = t2[0];
    if (!isfinite(rr)) { status = MC_E_BREAKDOWN; break; }
    beta = t2[1] / rz;
    rz = t2[1];
    cur ^= 1;
  }
  // ---- constant-mode correction: one constant per continuum ----------------
  // G_aa = 1^T (M_a/tau + W_a) 1 + sum of the exchange of a, G_ab = -(exchange
  // sums of the pair); c_a = 1_a^T (b - A x) from the non-diffusive terms.
  constexpr int NL = L + 1;
  constexpr int NP2 = NL * NL;
  double cs[NL + NP2];
#pragma unroll
  for (int k = 0; k < NL + NP2; ++k) cs[k] = 0.0;
  if (status == 0) {
    for (long long i = gt; i < Np; i += gs) {
      const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
      if (gx >= nx) continue;
      const int c = __ldg(A.hidx + i);
#pragma unroll
      for (int a = 0; a < L; ++a) {
        const double xa = __ldcg(sp.p[a] + i);
        double d = sp.mtau[a];
        double tv = sp.mtau[a] * (__ldcg(sp.pprev[a] + i) - xa) + __ldg(sp.F[a] + i);
        if (sp.W[a]) {
          const double wv = __ldg(sp.W[a] + i);
          tv += __ldg(sp.FW[a] + i) - wv * xa;
          d += wv;
        }
#pragma unroll
        for (int b = 0; b < L; ++b) {
          if (b == a) continue;
          const double qv = cq(sp, a, b, i);
          tv += qv * (__ldcg(sp.p[b] + i) - xa);
          cs[NL + a * NL + b] -= qv;
          d += qv;
        }
        if (c >= 0)
          for (int e = A.hptr[c]; e < A.hptr[c + 1]; ++e) {
            const int l = A.hpiece[e];
            const double qv = A.q[a][l];
            tv += qv * (__ldcg(A.xf + l) - xa);
            cs[NL + a * NL + L] -= qv;
            d += qv;
          }
        cs[a] += tv;
        cs[NL + a * NL + a] += d;
      }
    }
    for (long long l = gt; l < P; l += gs) {
      const double xl = __ldcg(A.xf + l);
      double tv = A.mf[l] / sp.tau * (A.xf_prev[l] - xl) + A.Ff[l] + A.FWf[l] - A.Wf[l] * xl;
      double d = A.mf[l] / sp.tau + A.Wf[l];
#pragma unroll
      for (int a = 0; a < L; ++a) {
        const double qv = A.q[a][l];
        tv += qv * (__ldcg(sp.p[a] + A.hostp[l]) - xl);
        cs[NL + L * NL + a] -= qv;
        d += qv;
      }
      cs[L] += tv;
      cs[NL + L * NL + L] += d;
    }
  }
  cstore<NL + NP2>(cs, A.partials, slot);
  if (!grid_barrier(A.bar)) return;
  double ct[NL + NP2];
  ctotal<NL + NP2>(A.partials, slot, ct);
  if (status == 0) {
    double G[NL][NL], c[NL], sh[NL];
#pragma unroll
    for (int a = 0; a < NL; ++a) {
      c[a] = ct[a];
#pragma unroll
      for (int b = 0; b < NL; ++b) G[a][b] = ct[NL + a * NL + b];
    }
#pragma unroll
    for (int k = 0; k < NL; ++k)
#pragma unroll
      for (int r = k + 1; r < NL; ++r) {
        const double fct = G[r][k] / G[k][k];
#pragma unroll
        for (int cc = k; cc < NL; ++cc) G[r][cc] -= fct * G[k][cc];
        c[r] -= fct * c[k];
      }
#pragma unroll
    for (int r = NL - 1; r >= 0; --r) {
      double v = c[r];
#pragma unroll
      for (int cc = r + 1; cc < NL; ++cc) v -= G[r][cc] * sh[cc];
      sh[r] = v / G[r][r];
    }
    for (int a = 0; a < L; ++a) {
      const double s = isfinite(sh[a]) ? sh[a] : 0.0;
      for (long long i = gt; i < Np; i += gs) {
        const int gy = (int)(i / pitch), gx = (int)(i - (long long)gy * pitch);
        if (gx >= nx) continue;
        sp.p[a][i] = __ldcg(sp.p[a] + i) + s;
      }
    }
    const double s = isfinite(sh[L]) ? sh[L] : 0.0;
    for (long long l = gt; l < P; l += gs) A.xf[l] = __ldcg(A.xf + l) + s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (status) atomicCAS(A.stat, 0, status);
    A.stat[2] += it;
    *A.relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
  }
}

template <int L>
void* coupled_fn() { return (void*)frac_coupled_kernel<L>; }

void* coupled_pick(int L) {
  switch (L) {
    case 1: return coupled_fn<1>();
    case 2: return coupled_fn<2>();
    default: return coupled_fn<3>();
  }
}

// Jacobi inverse of the coupled rows (matrix: 1 / (d of the decoupled block,
// which has the same diagonal)), hosting-cell index per matrix cell.
__global__ void frac_hidx_kernel(int NH, const int* hcell, int* hidx) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < NH; c += gridDim.x * blockDim.x)
    hidx[hcell[c]] = c;
}

mc_status coupled_step(mc_frac* f, mc_stats* st) {
  mc_ctx* ctx = f->ctx;
  cudaStream_t s = ctx->stream;
  const int L = f->L;
  if (!f->cpart) {
    void* fn = coupled_pick(L);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, CT, 0) != cudaSuccess || per < 1)
      return ferr(f, MC_E_CUDA, "coupled fracture kernel occupancy");
    f->cblocks = per * ctx->num_sms;
    if (falloc(f, (void**)&f->cpart, (size_t)2 * CQ * f->cblocks * sizeof(double)) != cudaSuccess ||
        falloc(f, (void**)&f->cbar, 96 * sizeof(unsigned)) != cudaSuccess ||
        falloc(f, (void**)&f->hidx, (size_t)ctx->Np * sizeof(int)) != cudaSuccess ||
        (!f->Pf2 && falloc(f, (void**)&f->Pf2, (size_t)f->P * sizeof(double)) != cudaSuccess))
      return ferr(f, MC_E_ALLOC, "coupled fracture buffers");
    if (cudaMemsetAsync(f->hidx, 0xff, (size_t)ctx->Np * sizeof(int), s) != cudaSuccess)
      return ferr(f, MC_E_CUDA, "hidx");
    if (f->NH > 0) {
      frac_hidx_kernel<<<grid256(f->NH), 256, 0, s>>>(f->NH, f->hcell, f->hidx);
      if (cudaGetLastError() != cudaSuccess) return ferr(f, MC_E_CUDA, "hidx kernel");
    }
  }
  CoupledArgs A{};
  mc_fill_params(ctx, &A.sp, MC_SCHEME_COUPLED, 1);
  for (int a = 0; a < L; ++a) {
    A.sp.W[a] = ctx->W[a];
    A.sp.FW[a] = ctx->FW[a];
    A.q[a] = f->q[a];
    A.invdm[a] = f->invd[a];   // same diagonal as the decoupled block with the exchange
  }
  A.P = f->P;
  A.NH = f->NH;
  A.NS = f->NS;
  A.segptr = f->segptr;
  A.llo = f->llo;
  A.lcp = f->lcp;
  A.ldinv = f->ldinv;
  A.rowptr = f->rowptr;
  A.col = f->col;
  A.T = f->T;
  A.mf = f->mf;
  A.dcf = f->dcf;
  A.invdf = f->invdf;
  A.Ff = f->Ff;
  A.FWf = f->FWf;
  A.Wf = f->Wf;
  A.hostp = f->hostp;
  A.hidx = f->hidx;
  A.hptr = f->hptr;
  A.hpiece = f->hpiece;
  A.xf = f->pf;
  A.xf_prev = f->pf_prev;
  A.rf = f->r;
  A.zf = f->z;
  A.Pf[0] = f->pp;
  A.Pf[1] = f->Pf2;
  A.qf = f->qq;
  A.partials = f->cpart;
  A.bar.count = reinterpret_cast<unsigned long long*>(f->cbar);
  A.bar.abort_word = f->cbar + 64;
  A.bar.status = f->dstat;
  A.bar.spin_limit = ctx->opts.spin_limit;
  A.stat = f->dstat;
  A.relres = f->drel + 1;
  if (cudaMemsetAsync(f->cbar, 0, 96 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(f->dstat, 0, 4 * sizeof(int), s) != cudaSuccess)
    return ferr(f, MC_E_CUDA, "memset");
  void* args[] = {&A};
  if (cudaLaunchCooperativeKernel(coupled_pick(L), dim3(f->cblocks), dim3(CT), args, 0, s) != cudaSuccess)
    return ferr(f, MC_E_CUDA, "coupled fracture launch");
  int ss[4] = {0, 0, 0, 0};
  double rel = 0.0;
  if (cudaMemcpyAsync(ss, f->dstat, sizeof(ss), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&rel, f->drel + 1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ferr(f, MC_E_CUDA, "coupled fracture status");
  st->iters[0] += ss[2];
  if (ss[2] > st->max_iters[0]) st->max_iters[0] = ss[2];
  st->rel_residual[0] = rel;
  if (ss[0] != 0)
    return ferr(f, (mc_status)ss[0], std::string("coupled fracture solve: ") + mc_status_string((mc_status)ss[0]));
  return MC_OK;
}


// ------------------------------------------ fracture solve over the grid ---
// The fracture system of the decoupled schemes (Eq. app-md's fracture rows,
// the matrix state lagged or current as the scheme says) for large networks:
// the same line-preconditioned PCG as frac_solve_kernel (operator, line
// blocks, stopping test, constant-mode correction), spread over a cooperative
// grid. Pieces are grid-strided for the operator; segments go one per warp
// for the line blocks, together with the x and r updates of their pieces, so
// that each warp's line solve reads only the residuals it wrote. P_new = z +
// beta P_old is formed on the fly where the operator reads it (two P
// buffers): two grid reductions per iteration, summed in a fixed CTA order.
struct FracGridArgs {
  FracSolve S;
  double* P2;        // second search-direction buffer
  double* partials;  // [2][CQ][gridDim.x]
  GridBar bar;
};

__global__ void __launch_bounds__(CT) frac_solve_grid_kernel(const __grid_constant__ FracGridArgs G) {
  const FracSolve& A = G.S;
  const int P = A.P;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const long long gwarp = gt >> 5, nwarp = gs >> 5;
  // b and r = b - A x (flux form) by segment, then z = M^-1 r of the segment;
  // b kept in xb for the constant-mode correction
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long sg = gwarp; sg < A.NS; sg += nwarp) {
    const int l0 = A.segptr[sg], l1 = A.segptr[sg + 1];
    for (int l = l0 + lane; l < l1; l += 32) {
      double b = A.mf[l] / A.tau * A.xprev[l] + A.Ff[l] + A.FWf[l];
      for (int a = 0; a < A.L; ++a) b += A.q[a][l] * A.pm[a][A.hostp[l]];
      const double rv = b - frac_flux(A, A.x, l, A.x[l]);
      A.r[l] = rv;
      A.xb[l] = b;
      A.p[l] = 0.0;
      acc[0] += b * b;
      acc[1] += rv * rv;
    }
    __syncwarp();
    line_apply_warp(l0, l1, A.llo, A.lcp, A.ldinv, A.r, A.z);
    for (int l = l0 + lane; l < l1; l += 32) acc[2] += __ldcg(A.r + l) * __ldcg(A.z + l);
  }
  cstore<3>(acc, G.partials, 0);
  if (!grid_barrier(G.bar)) return;
  double t3[3];
  ctotal<3>(G.partials, 0, t3);
  const double bb = t3[0];
  double rr = t3[1], rz = t3[2];
  const double tol2 = A.rtol * A.rtol;
  double beta = 0.0;
  int it = 0, cur = 0, slot = 1, status = 0;
  while (rr > tol2 * bb) {
    if (it >= A.max_iter) { status = MC_E_NOCONV; break; }
    // ---- P_new = z + beta P_old (stored), q = A P_new, <P_new, q> ----------
    const double bt = beta;
    const double* Po = cur ? G.P2 : A.p;
    double* Pn = cur ? A.p : G.P2;
    double pq[1] = {0.0};
    for (long long l = gt; l < P; l += gs) {
      const double pc = fma(bt, __ldcg(Po + l), __ldcg(A.z + l));
      double v = A.dcf[l] * pc;
      for (int e = A.rowptr[l]; e < A.rowptr[l + 1]; ++e) {
        const int nb = A.col[e];
        v += A.T[e] * (pc - fma(bt, __ldcg(Po + nb), __ldcg(A.z + nb)));
      }
      Pn[l] = pc;
      A.qv[l] = v;
      pq[0] = fma(pc, v, pq[0]);
    }
    cstore<1>(pq, G.partials, slot);
    if (!grid_barrier(G.bar)) return;
    double pqt[1];
    ctotal<1>(G.partials, slot, pqt);
    slot ^= 1;
    if (!(pqt[0] > 0.0) || !isfinite(pqt[0])) { status = MC_E_BREAKDOWN; break; }
    const double al = rz / pqt[0];
    // ---- x += al P, r -= al q, z = M^-1 r by segment, (r, r), (r, z) ---------
    double d2[2] = {0.0, 0.0};
    for (long long sg = gwarp; sg < A.NS; sg += nwarp) {
      const int l0 = A.segptr[sg], l1 = A.segptr[sg + 1];
      for (int l = l0 + lane; l < l1; l += 32) {
        A.x[l] = __ldcg(A.x + l) + al * __ldcg(Pn + l);
        const double rv = __ldcg(A.r + l) - al * __ldcg(A.qv + l);
        A.r[l] = rv;
        d2[0] += rv * rv;
      }
      __syncwarp();
      line_apply_warp(l0, l1, A.llo, A.lcp, A.ldinv, A.r, A.z);
      for (int l = l0 + lane; l < l1; l += 32) d2[1] += __ldcg(A.r + l) * __ldcg(A.z + l);
    }
    cstore<2>(d2, G.partials, slot);
    if (!grid_barrier(G.bar)) return;
    double t2[2];
    ctotal<2>(G.partials, slot, t2);
    slot ^= 1;
    ++it;
    rr = t2[0];
    if (!isfinite(rr)) { status = MC_E_BREAKDOWN; break; }
    beta = t2[1] / rz;
    rz = t2[1];
    cur ^= 1;
  }
  // ---- constant-mode correction: c = 1^T (b - A x) / 1^T dcf ---------------
  double cs[2] = {0.0, 0.0};
  if (status == 0)
    for (long long l = gt; l < P; l += gs) {
      cs[0] += __ldcg(A.xb + l) - A.dcf[l] * __ldcg(A.x + l);
      cs[1] += A.dcf[l];
    }
  cstore<2>(cs, G.partials, slot);
  if (!grid_barrier(G.bar)) return;
  double ct[2];
  ctotal<2>(G.partials, slot, ct);
  if (status == 0) {
    const double c = ct[1] > 0.0 ? ct[0] / ct[1] : 0.0;
    if (isfinite(c))
      for (long long l = gt; l < P; l += gs) A.x[l] = __ldcg(A.x + l) + c;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (status) atomicCAS(A.stat, 0, status);
    A.stat[1] += it;
    *A.relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
  }
}

// Launch of the grid fracture solve: CTAs enough for one segment per warp and
// about eight pieces per thread, at most the co-resident count.
mc_status frac_solve_grid(mc_frac* f, const FracSolve& S) {
  mc_ctx* ctx = f->ctx;
  cudaStream_t s = ctx->stream;
  if (!f->gpart) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (void*)frac_solve_grid_kernel, CT, 0) !=
            cudaSuccess ||
        per < 1)
      return ferr(f, MC_E_CUDA, "grid fracture kernel occupancy");
    f->gcap = per * ctx->num_sms;
    const long long want = std::max<long long>((f->NS + CT / 32 - 1) / (CT / 32), ((long long)f->P + 8 * CT - 1) / (8 * CT));
    f->gblocks = (int)std::max<long long>(1, std::min<long long>(want, f->gcap));
    if (falloc(f, (void**)&f->gpart, (size_t)2 * CQ * f->gblocks * sizeof(double)) != cudaSuccess ||
        falloc(f, (void**)&f->gbar, 96 * sizeof(unsigned)) != cudaSuccess)
      return ferr(f, MC_E_ALLOC, "grid fracture buffers");
    if (!f->Pf2 && falloc(f, (void**)&f->Pf2, (size_t)f->P * sizeof(double)) != cudaSuccess)
      return ferr(f, MC_E_ALLOC, "grid fracture buffers");
  }
  FracGridArgs G{};
  G.S = S;
  G.P2 = f->Pf2;
  G.partials = f->gpart;
  G.bar.count = reinterpret_cast<unsigned long long*>(f->gbar);
  G.bar.abort_word = f->gbar + 64;
  G.bar.status = f->dstat;
  G.bar.spin_limit = ctx->opts.spin_limit;
  if (cudaMemsetAsync(f->gbar, 0, 96 * sizeof(unsigned), s) != cudaSuccess)
    return ferr(f, MC_E_CUDA, "memset");
  void* args[] = {&G};
  if (cudaLaunchCooperativeKernel((void*)frac_solve_grid_kernel, dim3(f->gblocks), dim3(CT), args, 0, s) !=
      cudaSuccess)
    return ferr(f, MC_E_CUDA, "grid fracture launch");
  return MC_OK;
}

}  // namespace
