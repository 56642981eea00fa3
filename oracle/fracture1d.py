"""Lower-dimensional fracture continuum on its own 1-D mesh (Section 2,
Eqs. mm-md and mm-tc; Section 3.1, Eqs. app-md and app-tc).

TEST INFRASTRUCTURE ONLY (see the package header). Plain definitions:
the 1-D mesh is built from the segment list, the block matrices are
assembled entry by entry as scipy sparse matrices, and every time step is
solved with a sparse direct factorisation plus extended-precision refinement.

Mesh of the fracture network gamma (readings of Section 3.1):
  * every segment is clipped to the unit square and split at the grid lines
    it crosses and at its intersections with the other segments; each piece
    iota_l is one fracture cell, of length |iota_l|, hosted by the matrix
    cell that holds its midpoint;
  * a junction is a point where pieces meet (a split point, an intersection,
    or both at once). Fracture-fracture transmissibility (Eq. app-md,
    T_f = k_f |E| / d with the point facet |E| = 1): every piece l at a
    junction has the half-transmissibility t_l = k_f / d_l, d_l = |iota_l| / 2
    the distance from its midpoint to the junction, and each pair (l, n) at
    the junction gets T_ln = t_l t_n / sum_m t_m (the flux balance of a
    junction without storage; two pieces give the two-point value
    k_f / (d_l + d_n)). Segment ends that meet nothing carry no flux;
  * fracture-matrix exchange (Eq. app-md, sigma_il = sigma |E_l^i| / d_l^i):
    the interface is the piece itself, |E| = |iota_l|, and d is taken as h/4
    (the mean distance from the points of an h x h cell to a line through its
    centre), so q_al = 4 sigma_af |iota_l| / h for every matrix continuum a;
  * mass c_f |iota_l|, sources F_f given per piece (already integrated),
    wells W_l = q_w |iota_l| on pieces, read like the matrix wells as the
    implicit relaxation W (p_w - p).

Unknown order: the L matrix continua (nx*ny cells each, continuum-major),
then the fracture (P pieces). The continua are in ascending permeability with
the fracture last, so the L-scheme solves the matrix continua first and the
fracture last, the U-scheme the reverse.
"""

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import splu


def clip_segment(x0, y0, x1, y1):
    """Parameter range [t0, t1] of the segment inside the unit square
    (Liang-Barsky), or None."""
    dx, dy = x1 - x0, y1 - y0
    t0, t1 = 0.0, 1.0
    for p, q in ((-dx, x0), (dx, 1.0 - x0), (-dy, y0), (dy, 1.0 - y0)):
        if p == 0.0:
            if q < 0.0:
                return None
            continue
        t = q / p
        if p < 0.0:
            t0 = max(t0, t)
        else:
            t1 = min(t1, t)
        if t0 >= t1:
            return None
    return t0, t1


def _intersect(a, b):
    """Parameters (s, u) on clipped segments a, b (each (x0, y0, x1, y1)) of
    their crossing point, or None (parallel or no crossing)."""
    ax, ay, bx, by = a[2] - a[0], a[3] - a[1], b[2] - b[0], b[3] - b[1]
    den = ax * by - ay * bx
    if den == 0.0:
        return None
    cx, cy = b[0] - a[0], b[1] - a[1]
    s = (cx * by - cy * bx) / den
    u = (cx * ay - cy * ax) / den
    if 0.0 <= s <= 1.0 and 0.0 <= u <= 1.0:
        return s, u
    return None


class FractureMesh:
    """Pieces and junctions of the fracture network on an nx x ny grid.

    Attributes: length (P,), mid (P, 2), host (P,) matrix cell index
    j * nx + i, seg (P,), junctions: list of lists of piece indices.
    """

    def __init__(self, segments, nx, ny, tol=1e-12):
        h = 1.0 / nx
        clipped = []
        for s in np.asarray(segments, dtype=np.float64).reshape(-1, 4):
            c = clip_segment(*s)
            if c is None:
                continue
            t0, t1 = c
            x0, y0, x1, y1 = s
            e = (x0 + t0 * (x1 - x0), y0 + t0 * (y1 - y0),
                 x0 + t1 * (x1 - x0), y0 + t1 * (y1 - y0))
            if np.hypot(e[2] - e[0], e[3] - e[1]) > tol:
                clipped.append(e)
        S = len(clipped)
        # break parameters of every segment: ends, grid lines, intersections
        brk = [[0.0, 1.0] for _ in range(S)]
        crossings = []
        for k, (x0, y0, x1, y1) in enumerate(clipped):
            for (lo, hi, d0, dd, ncell) in ((x0, x1, x0, x1 - x0, nx), (y0, y1, y0, y1 - y0, ny)):
                if dd == 0.0:
                    continue
                a, b = sorted((lo, hi))
                for g in range(int(np.ceil(a / h)), int(np.floor(b / h)) + 1):
                    t = (g * h - d0) / dd
                    if 0.0 < t < 1.0:
                        brk[k].append(t)
        for a in range(S):
            for b in range(a + 1, S):
                hit = _intersect(clipped[a], clipped[b])
                if hit is not None:
                    brk[a].append(hit[0])
                    brk[b].append(hit[1])
                    crossings.append((a, hit[0], b, hit[1]))
        # merge breaks closer than tol (in length) and cut the pieces
        lengths, mids, hosts, segs = [], [], [], []
        point_of = []   # per segment: sorted unique break parameters
        first = []      # per segment: index of its first piece
        for k, (x0, y0, x1, y1) in enumerate(clipped):
            L = np.hypot(x1 - x0, y1 - y0)
            ts = np.sort(np.asarray(brk[k]))
            keep = [ts[0]]
            for t in ts[1:]:
                if (t - keep[-1]) * L > tol:
                    keep.append(t)
            keep[-1] = 1.0
            ts = np.asarray(keep)
            point_of.append(ts)
            first.append(len(lengths))
            for t0, t1 in zip(ts[:-1], ts[1:]):
                tm = 0.5 * (t0 + t1)
                mx, my = x0 + tm * (x1 - x0), y0 + tm * (y1 - y0)
                i = min(max(int(np.floor(mx / h)), 0), nx - 1)
                j = min(max(int(np.floor(my / h)), 0), ny - 1)
                lengths.append((t1 - t0) * L)
                mids.append((mx, my))
                hosts.append(j * nx + i)
                segs.append(k)
        self.length = np.asarray(lengths)
        self.mid = np.asarray(mids).reshape(-1, 2)
        self.host = np.asarray(hosts, dtype=np.int64)
        self.seg = np.asarray(segs, dtype=np.int64)
        self.P = self.length.size
        # junctions: one per break point of every segment, merged at crossings
        parent = {}

        def find(x):
            while parent.setdefault(x, x) != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        def near(k, t):
            ts = point_of[k]
            return int(np.argmin(np.abs(ts - t)))

        for (a, s, b, u) in crossings:
            ra, rb = find((a, near(a, s))), find((b, near(b, u)))
            if ra != rb:
                parent[ra] = rb
        groups = {}
        for k in range(S):
            m = len(point_of[k]) - 1   # pieces of segment k
            for q in range(m + 1):
                pcs = []
                if q >= 1:
                    pcs.append(first[k] + q - 1)
                if q <= m - 1:
                    pcs.append(first[k] + q)
                groups.setdefault(find((k, q)), []).extend(pcs)
        self.junctions = [sorted(set(g)) for g in groups.values() if len(set(g)) >= 2]

    def transmissibility(self, kf):
        """Fracture-fracture T_ln (star-delta at each junction), as a
        symmetric sparse P x P matrix of the pair values (zero diagonal)."""
        rows, cols, vals = [], [], []
        for g in self.junctions:
            t = np.array([kf / (0.5 * self.length[l]) for l in g])
            s = t.sum()
            for x in range(len(g)):
                for y in range(x + 1, len(g)):
                    v = t[x] * t[y] / s
                    rows += [g[x], g[y]]
                    cols += [g[y], g[x]]
                    vals += [v, v]
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.P, self.P))


class MixedSystem:
    """Block system of L co-located matrix continua (an oracle FVSystem) and
    one fracture continuum on a FractureMesh (Eq. app-md / app-tc):

      M dp/dt + A p = F,  blocks a, b in 0..L (L = the fracture),
      A_aa = D_a + sum_b Q_ab + diag(sum over hosted pieces of q_al)  (matrix)
      A_af = -Q_af  (N x P: -q_al at (host(l), l)),  A_fa = A_af^T
      A_ff = D_f + diag(sum_a q_al)
    with fracture wells W_f (implicit) and sources F_f per piece.
    """

    def __init__(self, fv, mesh, kf, cf, sigma_f, Ff=None, Wf=None, pwf=None):
        self.fv, self.mesh = fv, mesh
        self.L = fv.L
        self.kf, self.cf = float(kf), float(cf)
        self.sigma_f = np.asarray(sigma_f, dtype=np.float64).reshape(self.L)
        P, N, h = mesh.P, fv.N, fv.h
        self.P, self.N = P, N
        self.Tf = mesh.transmissibility(kf)
        self.mf = cf * mesh.length
        # q_al = sigma_af |iota_l| / (h / 4)
        self.q = [4.0 * self.sigma_f[a] * mesh.length / h for a in range(self.L)]
        self.Ff = np.zeros(P) if Ff is None else np.asarray(Ff, dtype=np.float64).copy()
        self.Wf = np.zeros(P) if Wf is None else np.asarray(Wf, dtype=np.float64).copy()
        self.pwf = np.zeros(P) if pwf is None else np.broadcast_to(
            np.asarray(pwf, dtype=np.float64), (P,)).copy()

    def hosted_sum(self, a, dtype=np.float64):
        """sum of q_al over the pieces hosted by each matrix cell, in dtype."""
        out = np.zeros(self.N, dtype=dtype)
        np.add.at(out, self.mesh.host, self.q[a].astype(dtype))
        return out

    def Q_mf(self, a):
        """N x P exchange matrix of matrix continuum a (entries q_al)."""
        return sp.csr_matrix((self.q[a], (self.mesh.host, np.arange(self.P))),
                             shape=(self.N, self.P))

    def block(self, a, b, dtype=np.float64):
        """Block (a, b) of A (no mass, no wells); index L is the fracture."""
        L = self.L
        if a < L and b < L:
            blk = self.fv.A_block(a, b, dtype)
            if a == b:
                blk = (blk + sp.diags(self.hosted_sum(a, dtype))).tocsr()
            return blk
        if a < L:   # matrix a <- fracture
            return (-self.Q_mf(a)).astype(dtype).tocsr()
        if b < L:   # fracture <- matrix b
            return (-self.Q_mf(b).T).astype(dtype).tocsr()
        # the diagonal summed in dtype: extended precision keeps 1^T D_f = 0
        # (an FP64 sum of T ~ 1e7 breaks it by eps * sum T per row)
        Te = self.Tf.astype(dtype)
        d = np.asarray(Te.sum(axis=1)).ravel()
        for c in range(L):
            d = d + self.q[c].astype(dtype)
        return (sp.diags(d) - Te).tocsr()

    def mass(self, a):
        return self.fv.m[a] if a < self.L else self.mf

    def well(self, a):
        """(W, W p_w) of continuum a."""
        if a < self.L:
            return self.fv.W[a], self.fv.well_rhs(a)
        return self.Wf, self.Wf * self.pwf

    def source(self, a, F):
        return np.ravel(F[a]) if a < self.L else self.Ff

    def size(self, a):
        return self.N if a < self.L else self.P


class MixedOracle:
    """Coupled backward Euler (Eq. ct-mc) and the D-, L-, U-schemes (Eq.
    si-mc) on a MixedSystem; every step an exact (factorised) solve."""

    def __init__(self, ms, tau, refine=3):
        self.ms, self.tau, self.refine = ms, float(tau), int(refine)
        self._fact = {}

    def _matrix(self, key, dtype):
        ms, L = self.ms, self.ms.L
        idx = list(range(L + 1)) if key == "coupled" else [key]
        blocks = []
        for a in idx:
            row = []
            for b in idx:
                blk = ms.block(a, b, dtype)
                if a == b:
                    W, _ = ms.well(a)
                    blk = (blk + sp.diags((ms.mass(a) / self.tau + W).astype(dtype))).tocsr()
                row.append(blk)
            blocks.append(row)
        return sp.bmat(blocks, format="csc")

    def _solve(self, key, b):
        if key not in self._fact:
            A = self._matrix(key, np.float64)
            self._fact[key] = (self._matrix(key, np.longdouble).tocsr(), splu(A))
        Ae, lu = self._fact[key]
        x = lu.solve(b)
        be = np.asarray(b, dtype=np.float64).astype(np.longdouble)
        for _ in range(self.refine):
            r = be - Ae @ x.astype(np.longdouble)
            x = x + lu.solve(np.asarray(r, dtype=np.float64))
        return x

    def step(self, p, F, scheme="D"):
        """One step from p (list of L + 1 arrays; the last is the fracture);
        F: L matrix source fields (the fracture sources are in the system)."""
        ms, L, tau = self.ms, self.ms.L, self.tau
        rhs0 = []
        for a in range(L + 1):
            _, wp = ms.well(a)
            rhs0.append(ms.mass(a) / tau * p[a] + ms.source(a, F) + wp)
        if scheme == "coupled":
            x = self._solve("coupled", np.concatenate(rhs0))
            out, o = [], 0
            for a in range(L + 1):
                n = ms.size(a)
                out.append(x[o:o + n].copy())
                o += n
            return out
        order = list(range(L + 1)) if scheme in ("D", "L") else list(range(L, -1, -1))
        if scheme not in ("D", "L", "U"):
            raise ValueError(scheme)
        new = [None] * (L + 1)
        for a in order:
            r = rhs0[a].copy()
            for b in range(L + 1):
                if b == a:
                    continue
                src = new[b] if (scheme != "D" and new[b] is not None) else p[b]
                r = r - ms.block(a, b) @ src
            new[a] = self._solve(a, r)
        return new

    def run(self, p0, F, nsteps, scheme="D", keep=False):
        p = [np.asarray(x, dtype=np.float64).ravel().copy() for x in p0]
        hist = [p]
        for _ in range(nsteps):
            p = self.step(p, F, scheme)
            if keep:
                hist.append(p)
        return hist if keep else p


def piece_data(mesh, fr):
    """Per-piece sources, well indices and well pressures of a workload's
    fracture description: a point source goes to the piece whose midpoint is
    nearest to the point; wells W = q_w |iota| on the pieces whose midpoints
    lie in a well box."""
    Ff = np.zeros(mesh.P)
    for (x, y, v) in fr.sources:
        k = int(np.argmin((mesh.mid[:, 0] - x) ** 2 + (mesh.mid[:, 1] - y) ** 2))
        Ff[k] += v
    Wf = np.zeros(mesh.P)
    for (x0, x1, y0, y1) in fr.well_boxes:
        inb = ((mesh.mid[:, 0] >= x0) & (mesh.mid[:, 0] <= x1) &
               (mesh.mid[:, 1] >= y0) & (mesh.mid[:, 1] <= y1))
        Wf[inb] = fr.qw * mesh.length[inb]
    return Ff, Wf, np.full(mesh.P, fr.pw)


def from_workload(w, refine=3):
    """(MixedOracle, initial state list) of a workload with `w.frac`."""
    from .fv import FVSystem
    fv = FVSystem(w.nx, w.ny, w.L, w.k, w.c, w.sigma, w.sigma_cell,
                  wells=getattr(w, "wells", None))
    fr = w.frac
    mesh = FractureMesh(fr.segments, w.nx, w.ny)
    Ff, Wf, pwf = piece_data(mesh, fr)
    ms = MixedSystem(fv, mesh, fr.kf, fr.cf, fr.sigma_f, Ff, Wf, pwf)
    p0 = [np.ravel(x).astype(np.float64) for x in w.p0] + [np.full(mesh.P, fr.p0)]
    return MixedOracle(ms, w.tau, refine=refine), p0
