"""Time schemes on the fine grid, each step solved exactly.

  coupled   -- backward Euler, Eq. ct-mc:  (M/tau + A) p^n = M/tau p^{n-1} + F.
  (With wells, every scheme's own diagonal blocks gain W_a and its
  right-hand sides W_a p_w,a: the implicit well term, see `fv`.)
  D-scheme  -- Eq. si-mc with A0 = blockdiag(D_a + sum_b Q_ab), A1 = A - A0
               (Section 3.3): every continuum solves
               (M_a/tau + D_a + sum_b Q_ab) p_a^n
                   = M_a/tau p_a^{n-1} + F_a + sum_b Q_ab p_b^{n-1}.
  L-scheme  -- A0 lower block triangular: continua solved in index order
               (ascending permeability); continuum a uses p_b^n of the
               continua b < a already solved and p_b^{n-1} of the others.
  U-scheme  -- A0 upper block triangular: solved in reverse index order,
               continuum a uses p_b^n for b > a.

Each linear system is factorised once (tau is fixed) with SuperLU and every
solve gets `refine` sweeps of iterative refinement whose residual b - A x is
formed in extended precision (numpy longdouble), with A assembled in extended
precision from the FP64 coefficients. The systems have a near-null constant
mode held only by the mass and exchange terms; an FP64 residual, or an FP64
sum a_ii = m/tau + sum q + sum T (which breaks 1^T D = 0 by eps * sum T per
row), shifts that mode by ~1e-11 (128 x 128) to ~1e-10 (1024 x 1024)
relative. Parity pinned by the closed-form uniform recurrence, the
cosine-mode decay factor, sigma = 0 reduction, mass and energy identities and
dense brute force (see the CPU tests).
"""

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import splu

SCHEMES = ("coupled", "D", "L", "U")


class Oracle:
    def __init__(self, fv, tau, refine=3, permc_spec="COLAMD"):
        self.fv = fv
        self.tau = float(tau)
        self.refine = int(refine)
        self.permc_spec = permc_spec
        self._fact = {}

    # -- matrices ---------------------------------------------------------
    def coupled_matrix(self, dtype=np.float64):
        """M/tau + D + Q (+ W, the implicit well term) over all continua
        (Eq. ct-mc)."""
        fv = self.fv
        mt = (np.concatenate(fv.m) / self.tau).astype(dtype) + np.concatenate(fv.W).astype(dtype)
        return (sp.diags(mt) + fv.A(dtype)).tocsc()

    def split_matrix(self, a, dtype=np.float64):
        """M_a/tau + D_a + sum_b Q_ab (+ W_a): the diagonal block of
        M/tau + A0."""
        fv = self.fv
        d = (fv.m[a] / self.tau).astype(dtype) + fv.W[a].astype(dtype)
        return (sp.diags(d) + fv.A_block(a, a, dtype)).tocsc()

    # -- direct solves ----------------------------------------------------
    def _factor(self, key):
        if key not in self._fact:
            if key == "coupled":
                A, Ae = self.coupled_matrix(), self.coupled_matrix(np.longdouble)
            else:
                A, Ae = self.split_matrix(key), self.split_matrix(key, np.longdouble)
            self._fact[key] = (Ae.tocsr(), splu(A, permc_spec=self.permc_spec))
        return self._fact[key]

    def solve(self, key, b):
        Ae, lu = self._factor(key)
        b = np.asarray(b, dtype=np.float64)
        be = b.astype(np.longdouble)
        x = lu.solve(b)
        for _ in range(self.refine):
            r = be - Ae @ x.astype(np.longdouble)
            x = x + lu.solve(np.asarray(r, dtype=np.float64))
        return x

    # -- one step of each scheme -------------------------------------------
    def rhs_coupled(self, p_prev, F):
        fv = self.fv
        return np.concatenate([fv.m[a] / self.tau * p_prev[a] + F[a] + fv.well_rhs(a)
                               for a in range(fv.L)])

    def step_coupled(self, p_prev, F):
        fv = self.fv
        x = self.solve("coupled", self.rhs_coupled(p_prev, F))
        return [x[a * fv.N:(a + 1) * fv.N].copy() for a in range(fv.L)]

    def rhs_split(self, a, p_prev, p_new, F):
        """Right-hand side of continuum a: mass term, source and the exchange
        with the other continua, at the newest layer already available."""
        fv = self.fv
        rhs = fv.m[a] / self.tau * p_prev[a] + F[a] + fv.well_rhs(a)
        for b in range(fv.L):
            if b == a:
                continue
            src = p_new[b] if p_new[b] is not None else p_prev[b]
            rhs = rhs + fv.q[(a, b)] * src
        return rhs

    def order(self, scheme):
        L = self.fv.L
        if scheme in ("D", "L"):
            return list(range(L))
        if scheme == "U":
            return list(range(L - 1, -1, -1))
        raise ValueError(scheme)

    def step_split(self, p_prev, F, scheme="D"):
        L = self.fv.L
        p_new = [None] * L
        for a in self.order(scheme):
            view = [None] * L if scheme == "D" else p_new
            p_new[a] = self.solve(a, self.rhs_split(a, p_prev, view, F))
        return p_new

    def step(self, p_prev, F, scheme="D"):
        if scheme == "coupled":
            return self.step_coupled(p_prev, F)
        return self.step_split(p_prev, F, scheme)

    def run(self, p0, F, nsteps, scheme="D", keep=False):
        """nsteps steps from p0 with a constant source F. Returns the final
        state (list of L flat arrays) or, with keep=True, every layer."""
        fv = self.fv
        p = [np.asarray(x, dtype=np.float64).ravel().copy() for x in p0]
        F = [np.asarray(x, dtype=np.float64).ravel() for x in F]
        hist = [p]
        for _ in range(nsteps):
            p = self.step(p, F, scheme)
            if keep:
                hist.append(p)
        return hist if keep else p


def from_workload(w, refine=3):
    """Oracle and FV system for an `mc_inputs.Workload`."""
    from .fv import FVSystem
    fv = FVSystem(w.nx, w.ny, w.L, w.k, w.c, w.sigma, w.sigma_cell,
                  wells=getattr(w, "wells", None))
    return Oracle(fv, w.tau, refine=refine)
