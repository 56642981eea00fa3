"""Error measures and the conserved / dissipated quantities.

  rel_l2       -- ||p - p~|| / ||p|| over all continuum cells jointly
                  (Section 5, e_h and e_H without the factor 100).
  mass_*       -- the mass identities that follow from 1^T D = 0 (every
                  TPFA flux leaves one cell and enters another).
  energy       -- ||p||_A^2 = (A p, p) of Theorems 2 and 3.
  block_mean   -- coarse-cell averages of a fine field (reference for e_H).
"""

import numpy as np


def rel_l2(ref, p):
    num = sum(float(np.sum((np.ravel(r) - np.ravel(x)) ** 2)) for r, x in zip(ref, p))
    den = sum(float(np.sum(np.ravel(r) ** 2)) for r in ref)
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


def rel_l2_each(ref, p):
    return [float(np.linalg.norm(np.ravel(r) - np.ravel(x)) /
                  max(np.linalg.norm(np.ravel(r)), 1e-300)) for r, x in zip(ref, p)]


def mass_change(fv, p_new, p_old):
    """sum_a sum_i m_a,i (p_a^n - p_a^{n-1})."""
    return sum(float(np.dot(fv.m[a], np.ravel(p_new[a]) - np.ravel(p_old[a])))
               for a in range(fv.L))


def exchange_change(fv, p_new, p_old):
    """sum over pairs a < b of sum_i q_ab,i (dp_a,i + dp_b,i): the part of the
    D-scheme mass balance carried by the lagged exchange (Section 3.3)."""
    s = 0.0
    for a in range(fv.L):
        for b in range(a + 1, fv.L):
            da = np.ravel(p_new[a]) - np.ravel(p_old[a])
            db = np.ravel(p_new[b]) - np.ravel(p_old[b])
            s += float(np.dot(fv.q[(a, b)], da + db))
    return s


def total_source(F):
    return float(sum(np.sum(f) for f in F))


def energy(fv, p):
    Ap = fv.apply_A([np.ravel(x) for x in p])
    return float(sum(np.dot(Ap[a], np.ravel(p[a])) for a in range(fv.L)))


def block_mean(field, nx, ny, bx, by):
    f = np.asarray(field).reshape(ny, nx)
    return f.reshape(ny // by, by, nx // bx, bx).mean(axis=(1, 3)).ravel()
