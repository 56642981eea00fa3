"""Nonlocal multicontinuum (NLMC) coarse model, Section 4.

For every coarse block K_i (bx x by fine cells) and continuum beta, the basis
function psi^{i,beta} = (psi_1, ..., psi_L) lives on the oversampled region
K_i^+ (K_i enlarged by `layers` coarse layers, clipped to the domain). It
solves the constrained energy minimisation of Eq. eq:basis: the coupled fine
operator D + Q restricted to K_i^+ with zero Dirichlet data on the region's
boundary, plus Lagrange multipliers that impose

    mean of psi_alpha over K_j = delta_ij delta_alpha,beta

for every coarse block K_j inside K_i^+ and every continuum alpha (co-located
continua: K_j^alpha = K_j). The KKT matrix is factorised directly.

R stacks the basis functions: row (beta, i) = psi^{i,beta}, columns in the
fine continuum-major order. The coarse operator is A_bar = R A R^T with A the
steady fine operator D + Q (Section 4.1).

Readings:
  * Zero Dirichlet on the part of the region boundary inside the domain,
    through a ghost value at distance h/2 (T = k |E| / (h/2) = 2 k); the part
    on the physical boundary keeps the zero-flux condition of Eq. mm-bc.
    `dirichlet_on_domain=True` applies the Dirichlet condition literally on
    the whole region boundary.
  * M_bar and F_bar are the coarse finite-volume forms the paper gives for
    piecewise-constant data: M_bar_alpha = diag(c_alpha |K_i|), F_bar = sums
    of the fine cell-integrated sources over each block.
  * Coarse schemes (Section 4.2-4.3): coupled Eq. is-nlmc; D-scheme with
    A0_bar = blockdiag(A_bar_aa); L/U schemes with the lower / upper block
    triangle of A_bar, continua in ascending / descending index order.

Parity pinned by: one-cell blocks reproduce the fine scheme exactly (R = I),
constraints to roundoff, symmetry and semi-definiteness of A_bar, and the
decay factor of the constant mode.
"""

import numpy as np
import scipy.linalg as la
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from .fv import diffusion_matrix


class NLMC:
    def __init__(self, fv, tau, ncx, ncy, layers, dirichlet_on_domain=False):
        nx, ny, L = fv.nx, fv.ny, fv.L
        if nx % ncx or ny % ncy:
            raise ValueError("coarse grid must divide the fine grid")
        self.fv, self.tau = fv, float(tau)
        self.ncx, self.ncy, self.layers = ncx, ncy, layers
        self.bx, self.by = nx // ncx, ny // ncy
        self.Nc = ncx * ncy
        self.dirichlet_on_domain = dirichlet_on_domain
        rr, cc, vv = [], [], []
        self.constraint_residual = 0.0
        for J in range(ncy):
            for I in range(ncx):
                psis, cres = self.local_basis(I, J)
                self.constraint_residual = max(self.constraint_residual, cres)
                for beta in range(L):
                    cols, vals = psis[beta]
                    rr.append(np.full(cols.size, beta * self.Nc + J * ncx + I))
                    cc.append(cols)
                    vv.append(vals)
        self.R = sp.csr_matrix((np.concatenate(vv), (np.concatenate(rr), np.concatenate(cc))),
                               shape=(L * self.Nc, L * fv.N))
        A = fv.A()
        self.Abar = (self.R @ A @ self.R.T).toarray()
        area = self.bx * self.by * fv.area
        self.mbar = np.concatenate([np.full(self.Nc, fv.c[a] * area) for a in range(L)])
        self._fact = {}

    # -- region geometry ---------------------------------------------------
    def region(self, I, J):
        l = self.layers
        I0, I1 = max(0, I - l), min(self.ncx, I + l + 1)
        J0, J1 = max(0, J - l), min(self.ncy, J + l + 1)
        return I0, I1, J0, J1

    def local_operator(self, I0, I1, J0, J1):
        """D + Q restricted to the region, with the Dirichlet ghost terms."""
        fv, L = self.fv, self.fv.L
        x0, x1, y0, y1 = I0 * self.bx, I1 * self.bx, J0 * self.by, J1 * self.by
        lnx, lny = x1 - x0, y1 - y0
        nloc = lnx * lny
        dom = self.dirichlet_on_domain
        blocks = [[None] * L for _ in range(L)]
        for a in range(L):
            TE = fv.TE[a][y0:y1, x0:x1 - 1]
            TN = fv.TN[a][y0:y1 - 1, x0:x1]
            D = diffusion_matrix(TE, TN, lnx, lny)
            k = fv.k[a][y0:y1, x0:x1]
            ghost = np.zeros((lny, lnx))
            if x0 > 0 or dom:
                ghost[:, 0] += 2.0 * k[:, 0]
            if x1 < fv.nx or dom:
                ghost[:, -1] += 2.0 * k[:, -1]
            if y0 > 0 or dom:
                ghost[0, :] += 2.0 * k[0, :]
            if y1 < fv.ny or dom:
                ghost[-1, :] += 2.0 * k[-1, :]
            ex = np.zeros(nloc)
            for b in range(L):
                if b != a:
                    qab = fv.q[(a, b)].reshape(fv.ny, fv.nx)[y0:y1, x0:x1].ravel()
                    ex += qab
                    blocks[a][b] = sp.diags(-qab)
            blocks[a][a] = D + sp.diags(ghost.ravel() + ex)
        return sp.bmat(blocks, format="csc"), lnx, lny

    def constraints(self, I0, I1, J0, J1):
        """C: one row per (alpha, coarse block in the region), the block mean."""
        L = self.fv.L
        lnx = (I1 - I0) * self.bx
        lny = (J1 - J0) * self.by
        nloc = lnx * lny
        nb = (I1 - I0) * (J1 - J0)
        inv = 1.0 / (self.bx * self.by)
        rows, cols = [], []
        lj, li = np.divmod(np.arange(nloc), lnx)
        blk = (lj // self.by) * (I1 - I0) + (li // self.bx)
        for a in range(L):
            rows.append(a * nb + blk)
            cols.append(a * nloc + np.arange(nloc))
        C = sp.csr_matrix((np.full(L * nloc, inv), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(L * nb, L * nloc))
        return C, nb

    def local_basis(self, I, J):
        """psi^{i,beta} for beta = 0..L-1 by a direct KKT solve (Eq. eq:basis).
        Returns ([(global columns, values)] per beta, constraint residual)."""
        fv, L = self.fv, self.fv.L
        I0, I1, J0, J1 = self.region(I, J)
        A, lnx, lny = self.local_operator(I0, I1, J0, J1)
        C, nb = self.constraints(I0, I1, J0, J1)
        nloc = lnx * lny
        K = sp.bmat([[A, C.T], [C, None]], format="csc")
        lu = splu(K)
        centre = (J - J0) * (I1 - I0) + (I - I0)
        x0, y0 = I0 * self.bx, J0 * self.by
        lj, li = np.divmod(np.arange(nloc), lnx)
        gcell = (y0 + lj) * fv.nx + (x0 + li)
        out = []
        cres = 0.0
        for beta in range(L):
            rhs = np.zeros(L * nloc + L * nb)
            rhs[L * nloc + beta * nb + centre] = 1.0
            sol = lu.solve(rhs)
            for _ in range(2):
                sol = sol + lu.solve(rhs - K @ sol)
            psi = sol[:L * nloc]
            target = rhs[L * nloc:]
            cres = max(cres, float(np.max(np.abs(C @ psi - target))))
            cols = np.concatenate([a * fv.N + gcell for a in range(L)])
            out.append((cols, psi))
        return out, cres

    # -- coarse data ---------------------------------------------------------
    def coarse_source(self, F):
        fv = self.fv
        return np.concatenate([
            np.asarray(F[a]).reshape(fv.ny, fv.nx)
            .reshape(self.ncy, self.by, self.ncx, self.bx).sum(axis=(1, 3)).ravel()
            for a in range(fv.L)])

    def coarse_mean(self, p):
        fv = self.fv
        return np.concatenate([
            np.asarray(p[a]).reshape(fv.ny, fv.nx)
            .reshape(self.ncy, self.by, self.ncx, self.bx).mean(axis=(1, 3)).ravel()
            for a in range(fv.L)])

    def block(self, a, b):
        n = self.Nc
        return self.Abar[a * n:(a + 1) * n, b * n:(b + 1) * n]

    # -- coarse time schemes ---------------------------------------------------
    def _lu(self, key):
        if key not in self._fact:
            n = self.Nc
            if key == "coupled":
                Mt = np.diag(self.mbar / self.tau) + self.Abar
            else:
                a = key
                Mt = np.diag(self.mbar[a * n:(a + 1) * n] / self.tau) + self.block(a, a)
            self._fact[key] = (Mt, la.lu_factor(Mt))
        return self._fact[key]

    def _solve(self, key, b):
        """Dense LU plus two refinement sweeps with an extended-precision
        residual (same reason as the fine-grid solves)."""
        Mt, f = self._lu(key)
        Me = Mt.astype(np.longdouble)
        be = np.asarray(b, dtype=np.float64).astype(np.longdouble)
        x = la.lu_solve(f, b)
        for _ in range(2):
            r = be - Me @ x.astype(np.longdouble)
            x = x + la.lu_solve(f, np.asarray(r, dtype=np.float64))
        return x

    def step(self, pbar, Fbar, scheme="D"):
        n, L = self.Nc, self.fv.L
        if scheme == "coupled":
            return self._solve("coupled", self.mbar / self.tau * pbar + Fbar)
        if scheme in ("D", "L"):
            order = list(range(L))
        elif scheme == "U":
            order = list(range(L - 1, -1, -1))
        else:
            raise ValueError(scheme)
        new = [None] * L
        for a in order:
            sl = slice(a * n, (a + 1) * n)
            rhs = self.mbar[sl] / self.tau * pbar[sl] + Fbar[sl]
            for b in range(L):
                if b == a:
                    continue
                src = new[b] if (scheme != "D" and new[b] is not None) else pbar[b * n:(b + 1) * n]
                rhs = rhs - self.block(a, b) @ src
            new[a] = self._solve(a, rhs)
        return np.concatenate(new)

    def run(self, p0, F, nsteps, scheme="D", keep=False):
        pbar = self.coarse_mean(p0)
        Fbar = self.coarse_source(F)
        hist = [pbar]
        for _ in range(nsteps):
            pbar = self.step(pbar, Fbar, scheme)
            if keep:
                hist.append(pbar)
        return hist if keep else pbar
