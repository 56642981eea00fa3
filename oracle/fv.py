"""Two-point flux finite-volume assembly on the structured h x h grid
(Section 3.1, Eqs. app-md, app, app-mc).

Conventions: cell (i, j), i along x, j along y, 0-based, global index
j * nx + i; field arrays are (ny, nx). Square cells, h = 1/nx.

Readings of the paper used here:
  * T_ij = k |E_ij| / d_ij (Eq. app-md). With square cells |E| = d = h, so
    T = k_face. The face value of a cell-wise k is not stated; the harmonic
    mean 2 k_a k_b / (k_a + k_b) is used (0 when both are 0).
  * Zero-flux boundaries (Eq. mm-bc) mean boundary faces carry no
    transmissibility.
  * m_alpha,i = c_alpha |cell| (Eq. app-mc), |cell| = h^2.
  * Co-located continua overlap cell by cell, so Q_alpha_beta is diagonal
    with q_alpha_beta,i = sigma_alpha_beta,i |cell| (sigma given per unit
    area; the cell-integrated exchange mirrors the mass and source terms).
  * F_alpha is given already cell-integrated (F = f |cell|).
  * Well term (Section 5: f_f = q_w (p - p_w) in the well regions). Read as
    the relaxation q_w (p_w - p) toward the well pressure -- the sign that
    keeps the problem dissipative -- taken implicitly in p: it adds
    W = q_w |cell| to the diagonal of the continuum's own block and W p_w to
    its right-hand side. It is a continuum-local diagonal term, so it sits in
    A0 of every decoupled scheme. W and p_w are given per cell (W = 0 outside
    the wells).
"""

import numpy as np
import scipy.sparse as sp


def harmonic_face(ka, kb):
    """Harmonic mean of the two cell permeabilities sharing a face."""
    ka = np.asarray(ka, dtype=np.float64)
    kb = np.asarray(kb, dtype=np.float64)
    s = ka + kb
    out = np.zeros(np.broadcast(ka, kb).shape)
    nz = s > 0.0
    out[nz] = (2.0 * ka * kb)[nz] / s[nz]
    return out


def diffusion_matrix(TE, TN, nx, ny, dtype=np.float64):
    """D_alpha: a_ii = sum_n T_in, a_ij = -T_ij (Section 3.1, entries a).

    TE[j, i] is the face between (i, j) and (i+1, j); TN[j, i] the face
    between (i, j) and (i, j+1). The diagonal is the sum of the duplicate
    (i, i) entries, formed in `dtype`.
    """
    N = nx * ny
    idx = np.arange(N).reshape(ny, nx)
    rows, cols, vals = [], [], []
    for T, a, b in ((TE, idx[:, :-1], idx[:, 1:]), (TN, idx[:-1, :], idx[1:, :])):
        t = T.ravel()
        a = a.ravel()
        b = b.ravel()
        rows += [a, b, a, b]
        cols += [a, b, b, a]
        vals += [t, t, -t, -t]
    return sp.csr_matrix((np.concatenate(vals).astype(dtype),
                          (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N), dtype=dtype)


class FVSystem:
    """Semi-discrete system M dp/dt + (D + Q) p = F of Eq. app-mc.

    Parity pinned by: cosine eigenmodes of D (closed form), dense brute force
    on tiny grids, row sums of D + Q (mass conservation), symmetry.
    """

    def __init__(self, nx, ny, L, k, c, sigma=None, sigma_cell=None, wells=None):
        self.nx, self.ny, self.L = int(nx), int(ny), int(L)
        self.N = self.nx * self.ny
        self.h = 1.0 / self.nx
        area = self.h * self.h
        self.area = area
        self.k = [np.asarray(ka, dtype=np.float64).reshape(ny, nx) for ka in k]
        self.c = np.asarray(c, dtype=np.float64)
        sigma = np.zeros((L, L)) if sigma is None else np.asarray(sigma, dtype=np.float64)
        sigma_cell = {} if sigma_cell is None else sigma_cell
        self.TE = [harmonic_face(ka[:, :-1], ka[:, 1:]) for ka in self.k]
        self.TN = [harmonic_face(ka[:-1, :], ka[1:, :]) for ka in self.k]
        self.m = [np.full(self.N, self.c[a] * area) for a in range(L)]
        self.D = [diffusion_matrix(self.TE[a], self.TN[a], nx, ny) for a in range(L)]
        # q[(a, b)] for a != b, per cell, symmetric in (a, b).
        self.q = {}
        for a in range(L):
            for b in range(a + 1, L):
                if (a, b) in sigma_cell and sigma_cell[(a, b)] is not None:
                    s = np.asarray(sigma_cell[(a, b)], dtype=np.float64).ravel()
                else:
                    s = np.full(self.N, sigma[a, b])
                self.q[(a, b)] = s * area
                self.q[(b, a)] = self.q[(a, b)]
        # wells: W[a] = q_w |cell| per cell and the well pressure pw[a]
        self.W = [np.zeros(self.N) for _ in range(L)]
        self.pw = [np.zeros(self.N) for _ in range(L)]
        for a, (Wa, pwa) in (wells or {}).items():
            self.W[a] = np.asarray(Wa, dtype=np.float64).ravel().copy()
            pwa = np.asarray(pwa, dtype=np.float64)
            self.pw[a] = (pwa.ravel().copy() if pwa.size == self.N
                          else np.full(self.N, float(pwa)))

    def well_rhs(self, a):
        """W_a p_w,a: the well term's right-hand side (zero without wells)."""
        return self.W[a] * self.pw[a]

    def exchange_sum(self, a):
        """Diagonal of sum_{beta != a} Q_a,beta."""
        out = np.zeros(self.N)
        for b in range(self.L):
            if b != a:
                out += self.q[(a, b)]
        return out

    def A_block(self, a, b, dtype=np.float64):
        """Block (a, b) of A = D + Q (Section 3.1, matrix Q), its entries
        summed in `dtype` (longdouble keeps 1^T D = 0 to extended precision:
        an FP64 diagonal sum of T breaks it by eps * sum T per row)."""
        if a == b:
            D = self.D[a] if dtype == np.float64 else diffusion_matrix(
                self.TE[a], self.TN[a], self.nx, self.ny, dtype)
            ex = np.zeros(self.N, dtype=dtype)
            for c in range(self.L):
                if c != a:
                    ex += self.q[(a, c)].astype(dtype)
            return (D + sp.diags(ex)).tocsr()
        return sp.diags(-self.q[(a, b)].astype(dtype)).tocsr()

    def A(self, dtype=np.float64):
        """The full coupled operator A = D + Q, continuum-major ordering."""
        L = self.L
        return sp.bmat([[self.A_block(a, b, dtype) for b in range(L)] for a in range(L)],
                       format="csr")

    def M(self, dtype=np.float64):
        return sp.diags(np.concatenate(self.m).astype(dtype)).tocsr()

    def apply_A(self, p):
        """A p for a list of L flat state vectors (a plain matrix product)."""
        return [sum(self.A_block(a, b) @ p[b] for b in range(self.L))
                for a in range(self.L)]
