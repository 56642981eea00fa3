"""The five synthetic workloads, each a seeded recipe.

Every workload lives on the unit square with nx = ny = n square cells of side
h = 1/n. Continua are ordered by ascending permeability (the ordering the L-
and U-schemes of Section 3.3 assume). Sources are cell-integrated rates F
(Eq. app-mc: F = f |cell|), given directly: +1 in cell (n/8, n/8) and -1 in
cell (7n/8, 7n/8) of the most permeable continuum.

Exchange coefficients are given per unit area (sigma of Eq. mm); a constant
L x L matrix `sigma` and, for cells where the exchange varies, per-pair arrays
`sigma_cell[(a, b)]` (a < b) that replace the constant for that pair.
"""

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from .fields import correlated_lognormal, random_segments, segment_lengths


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    L: int
    k: List[np.ndarray]                     # L arrays (ny, nx)
    c: np.ndarray                           # (L,)
    sigma: np.ndarray                       # (L, L) symmetric, zero diagonal
    tau: float
    nsteps: int
    F: List[np.ndarray]                     # L arrays (ny, nx)
    p0: List[np.ndarray]                    # L arrays (ny, nx)
    sigma_cell: Dict[Tuple[int, int], np.ndarray] = field(default_factory=dict)
    # implicit wells: continuum -> (W = q_w |cell| per cell, p_w per cell)
    wells: Dict[int, Tuple[np.ndarray, np.ndarray]] = field(default_factory=dict)
    coarse: Optional[Tuple[int, int, int]] = None   # (ncx, ncy, layers)
    frac: Optional["Fracture1D"] = None             # lower-dimensional fracture continuum
    seed: Optional[int] = None
    # continuum -> boolean (ny, nx) cells where the continuum physically lives
    # (an embedded fracture continuum: the cells its segments cross); absent
    # continua cover the whole domain
    support: Dict[int, np.ndarray] = field(default_factory=dict)

    @property
    def h(self):
        return 1.0 / self.nx

    @property
    def cells(self):
        return self.nx * self.ny

    @property
    def continuum_cells(self):
        return self.L * self.nx * self.ny


def _sym(L, pairs):
    s = np.zeros((L, L))
    for (a, b), v in pairs.items():
        s[a, b] = s[b, a] = v
    return s


def _point_sources(n, L, alpha):
    F = [np.zeros((n, n)) for _ in range(L)]
    a, b = n // 8, (7 * n) // 8
    F[alpha][a, a] += 1.0
    F[alpha][b, b] -= 1.0
    return F


def dual_64(n=64, seed=1):
    """Dual-continuum matrix/fracture problem: k1 = exp(N(0,1)) per cell,
    k2 = 1e3 exp(0.5 N(0,1)) (drawn in that order from one generator),
    c = (1, 0.1), sigma_12 = 10, tau = 1/50, 50 steps from p = 0."""
    rng = np.random.default_rng(seed)
    k1 = np.exp(rng.standard_normal((n, n)))
    k2 = 1e3 * np.exp(0.5 * rng.standard_normal((n, n)))
    return Workload("dual_%d" % n, n, n, 2, [k1, k2], np.array([1.0, 0.1]),
                    _sym(2, {(0, 1): 10.0}), 1.0 / 50, 50,
                    _point_sources(n, 2, 1), [np.zeros((n, n))] * 2, seed=seed)


def triple_1024(n=1024, seeds=(21, 22, 23), nsteps=200):
    """Three continua with correlated log-normal k (correlation length 16
    cells, geometric means 1, 1e2, 1e4), c = (1, 0.2, 0.05),
    sigma = (12: 5, 13: 1, 23: 20), tau = 1/200."""
    k = [correlated_lognormal(np.random.default_rng(s), n, n, 16.0, m)
         for s, m in zip(seeds, (1.0, 1e2, 1e4))]
    return Workload("triple_%d" % n, n, n, 3, k, np.array([1.0, 0.2, 0.05]),
                    _sym(3, {(0, 1): 5.0, (0, 2): 1.0, (1, 2): 20.0}),
                    1.0 / 200, nsteps, _point_sources(n, 3, 2),
                    [np.zeros((n, n))] * 3, seed=seeds[0])


def precision_4096(n=4096, seed=3, nsteps=100):
    """Dual continuum as dual_64 but k2 = 1e5 exp(0.5 N(0,1)), tau = 1/50."""
    rng = np.random.default_rng(seed)
    k1 = np.exp(rng.standard_normal((n, n)))
    k2 = 1e5 * np.exp(0.5 * rng.standard_normal((n, n)))
    return Workload("precision_%d" % n, n, n, 2, [k1, k2],
                    np.array([1.0, 0.1]), _sym(2, {(0, 1): 10.0}), 1.0 / 50,
                    nsteps, _point_sources(n, 2, 1), [np.zeros((n, n))] * 2,
                    seed=seed)


def _fracture_sources(ell, n, L):
    """+1 / -1 in the fracture continuum at the fracture cells nearest to
    (n/8, n/8) and (7n/8, 7n/8): the wells sit in fractures, as in the
    paper's experiments (Section 5)."""
    F = [np.zeros((n, n)) for _ in range(L)]
    jj, ii = np.nonzero(ell > 0.0)
    for (t, v) in ((n // 8, 1.0), ((7 * n) // 8, -1.0)):
        if jj.size:
            d = (ii - t) ** 2 + (jj - t) ** 2
            k = int(np.argmin(d))
            F[L - 1][jj[k], ii[k]] += v
        else:
            F[L - 1][t, t] += v
    return F


def fracture_instance(seed, n=None, L=None, tau=1.0 / 100, nsteps=100,
                      sizes=(128, 256, 512, 1024)):
    """One realisation with an embedded fracture continuum (the last one).

    L in {2, 3} (p = 1/2) and n from `sizes` are drawn first unless given;
    then the matrix field (log-normal, mean 1), for L = 3 a natural-fracture
    field (log-normal, mean 1e2), then 20..200 random segments. Cells crossed
    by a segment get k = 1e4 in the fracture continuum, all others 1e-2; the
    fracture exchanges with every other continuum through
    sigma_i = 10 * l_i / h, l_i the segment length inside cell i. The sources
    are in the fracture cells nearest to (n/8, n/8) and (7n/8, 7n/8).
    """
    rng = np.random.default_rng(seed)
    if L is None:
        L = int(rng.integers(2, 4))
    else:
        rng.integers(2, 4)
    if n is None:
        n = int(sizes[int(rng.integers(0, len(sizes)))])
    else:
        rng.integers(0, len(sizes))
    k = [correlated_lognormal(rng, n, n, 16.0, 1.0)]
    if L == 3:
        k.append(correlated_lognormal(rng, n, n, 16.0, 1e2))
    ell = segment_lengths(random_segments(rng), n, n)
    k.append(np.where(ell > 0.0, 1e4, 1e-2))
    sig_f = 10.0 * ell * n
    if L == 2:
        c = np.array([1.0, 0.1])
        sigma = np.zeros((2, 2))
        sc = {(0, 1): sig_f}
    else:
        c = np.array([1.0, 0.2, 0.05])
        sigma = _sym(3, {(0, 1): 5.0})
        sc = {(0, 2): sig_f, (1, 2): sig_f.copy()}
    return Workload("fracture_%d_L%d_s%d" % (n, L, seed), n, n, L, k, c, sigma,
                    tau, nsteps, _fracture_sources(ell, n, L),
                    [np.zeros((n, n))] * L, sigma_cell=sc, seed=seed,
                    support={L - 1: ell > 0.0})


def batched_instances(count=256, base_seed=4000, sizes=(128, 256, 512, 1024),
                      nsteps=100):
    """Independent instances, instance b drawn with seed base_seed + b."""
    return [fracture_instance(base_seed + b, sizes=sizes, nsteps=nsteps)
            for b in range(count)]


def nlmc_1024(n=1024, seed=5000, ncoarse=32, layers=2, nsteps=200):
    """Dual-continuum fracture field at n^2, coarse grid ncoarse^2 with
    `layers` oversampling layers, tau = 1/200."""
    w = fracture_instance(seed, n=n, L=2, tau=1.0 / 200, nsteps=nsteps)
    w.name = "nlmc_%d_c%d" % (n, ncoarse)
    w.coarse = (ncoarse, ncoarse, layers)
    return w


def _box_cells(n, x0, x1, y0, y1):
    """Cells whose centres lie in [x0, x1] x [y0, y1] (boolean (n, n))."""
    c = (np.arange(n) + 0.5) / n
    return (((c[None, :] >= x0) & (c[None, :] <= x1)) &
            ((c[:, None] >= y0) & (c[:, None] <= y1)))


def paper_wells(L=2, n=200, seed=None, nsteps=50, qw=1e5, pw=1.2):
    """A workload shaped like the paper's 2C / 3C experiments (Section 5):
    p^0 = 1 in every continuum, T = 0.002 in 50 steps (tau = 4e-5), wells of
    index q_w = 1e5 and pressure p_w = 1.2 in the fracture cells of the boxes
    [0.1, 0.15]^2 and [0.6, 0.65] x [0.85, 0.9], no other source.

    2C: matrix c = 0.1, k = 1; fracture c = 1, k = 1e6.
    3C: matrix c = 0.05, k = 1e-3; natural fractures c = 0.1, k = 1;
        hydraulic fractures c = 1, k = 1e6.
    The paper's 25-line geometry exists only as a figure: 25 seeded random
    segments stand in for it (centre U[0,1]^2, length U[0.05, 0.5], angle
    U[0, pi)), rasterised as in `fracture_instance` (crossed cells get the
    fracture k, the others 1e-2; fracture exchange sigma_i = 10 l_i / h with
    every other continuum; matrix / natural-fracture exchange 5). A box with
    no fracture cell gets its well at the fracture cell nearest its centre.
    W = q_w |cell| in the well cells.
    """
    if L not in (2, 3):
        raise ValueError("L must be 2 or 3")
    seed = 6000 + L if seed is None else seed
    rng = np.random.default_rng(seed)
    ell = segment_lengths(random_segments(rng, 25, 25), n, n)
    frac = np.where(ell > 0.0, 1e6, 1e-2)
    sig_f = 10.0 * ell * n
    if L == 2:
        k = [np.ones((n, n)), frac]
        c = np.array([0.1, 1.0])
        sigma = np.zeros((2, 2))
        sc = {(0, 1): sig_f}
    else:
        k = [np.full((n, n), 1e-3), np.ones((n, n)), frac]
        c = np.array([0.05, 0.1, 1.0])
        sigma = _sym(3, {(0, 1): 5.0})
        sc = {(0, 2): sig_f, (1, 2): sig_f.copy()}
    W = np.zeros((n, n))
    jj, ii = np.nonzero(ell > 0.0)
    for (x0, x1, y0, y1) in ((0.1, 0.15, 0.1, 0.15), (0.6, 0.65, 0.85, 0.9)):
        box = _box_cells(n, x0, x1, y0, y1) & (ell > 0.0)
        if not box.any() and jj.size:
            cx, cy = 0.5 * (x0 + x1) * n - 0.5, 0.5 * (y0 + y1) * n - 0.5
            m = int(np.argmin((ii - cx) ** 2 + (jj - cy) ** 2))
            box = np.zeros((n, n), dtype=bool)
            box[jj[m], ii[m]] = True
        W[box] = qw / (n * n)
    tau = 0.002 / nsteps
    w = Workload("paper%dC_%d" % (L, n), n, n, L, k, c, sigma, tau, nsteps,
                 [np.zeros((n, n)) for _ in range(L)], [np.ones((n, n)) for _ in range(L)],
                 sigma_cell=sc, seed=seed, support={L - 1: ell > 0.0})
    w.wells = {L - 1: (W, np.full((n, n), pw))}
    return w


@dataclass
class Fracture1D:
    """The lower-dimensional fracture continuum of a workload (inputs only):
    segments (S, 4) as (x0, y0, x1, y1), not clipped; fracture permeability
    kf and capacity cf of the 1-D mesh; matrix-fracture exchange sigma_f per
    matrix continuum; point sources (x, y, value) put on the fracture piece
    nearest to the point; wells q_w (p_w - p) on the pieces whose midpoints
    lie in the boxes (x0, x1, y0, y1), of index q_w per unit length."""
    segments: np.ndarray
    kf: float
    cf: float
    sigma_f: np.ndarray
    sources: List[Tuple[float, float, float]] = field(default_factory=list)
    well_boxes: List[Tuple[float, float, float, float]] = field(default_factory=list)
    qw: float = 0.0
    pw: float = 0.0
    p0: float = 0.0


def fracture1d(L=1, n=200, seed=None, nsteps=50, nseg=(25, 25), tau=None, p0=1.0, wells=True):
    """Matrix continua on the n x n grid plus a fracture continuum on its own
    1-D mesh: the shape of the paper's 2C (L = 1 matrix continuum) and 3C
    (L = 2: matrix and natural fractures) problems (Section 5), with seeded
    segments (centre U[0,1]^2, length U[0.05, 0.5], angle U[0, pi)) standing
    in for its 25-line geometry.

    2C: matrix c = 0.1, k = 1; fracture c_f = 1, k_f = 1e6.
    3C: matrix c = 0.05, k = 1e-3; natural fractures c = 0.1, k = 1
        (exchange 5 with the matrix); fracture as in 2C.
    Fracture-matrix exchange sigma_f = 1 for every matrix continuum.
    p^0 = p0 everywhere; wells q_w = 1e5 per unit length at p_w = 1.2 on the
    pieces in [0.1, 0.15]^2 and [0.6, 0.65] x [0.85, 0.9] (wells=True);
    T = 0.002 in `nsteps` steps unless tau is given.
    """
    if L not in (1, 2):
        raise ValueError("L (matrix continua) must be 1 or 2")
    seed = 7000 + L if seed is None else seed
    rng = np.random.default_rng(seed)
    segs = random_segments(rng, nseg[0], nseg[1])
    if L == 1:
        k = [np.ones((n, n))]
        c = np.array([0.1])
        sigma = np.zeros((1, 1))
    else:
        k = [np.full((n, n), 1e-3), np.ones((n, n))]
        c = np.array([0.05, 0.1])
        sigma = _sym(2, {(0, 1): 5.0})
    tau = 0.002 / nsteps if tau is None else tau
    w = Workload("frac1d_%dC_%d" % (L + 1, n), n, n, L, k, c, sigma, tau, nsteps,
                 [np.zeros((n, n)) for _ in range(L)], [np.full((n, n), p0) for _ in range(L)],
                 seed=seed)
    w.frac = Fracture1D(segs, 1e6, 1.0, np.ones(L),
                        well_boxes=[(0.1, 0.15, 0.1, 0.15), (0.6, 0.65, 0.85, 0.9)] if wells else [],
                        qw=1e5 if wells else 0.0, pw=1.2, p0=p0)
    return w


def fracture1d_sources(L=1, n=1024, seed=None, nsteps=10, tau=1.0 / 100):
    """The 1-D fracture model on the fracture recipe's field (log-normal
    matrix k, mean 1; for L = 2 natural fractures, mean 1e2) with 20..200
    seeded segments, p^0 = 0 and point sources +1 / -1 on the pieces nearest
    to (1/8, 1/8) and (7/8, 7/8); no wells."""
    seed = 7100 + L if seed is None else seed
    rng = np.random.default_rng(seed)
    k = [correlated_lognormal(rng, n, n, 16.0, 1.0)]
    if L == 2:
        k.append(correlated_lognormal(rng, n, n, 16.0, 1e2))
    segs = random_segments(rng)
    c = np.array([1.0]) if L == 1 else np.array([1.0, 0.2])
    sigma = np.zeros((1, 1)) if L == 1 else _sym(2, {(0, 1): 5.0})
    w = Workload("frac1d_src_L%d_%d" % (L, n), n, n, L, k, c, sigma, tau, nsteps,
                 [np.zeros((n, n)) for _ in range(L)], [np.zeros((n, n)) for _ in range(L)],
                 seed=seed)
    w.frac = Fracture1D(segs, 1e4, 0.1, np.full(L, 10.0),
                        sources=[(0.125, 0.125, 1.0), (0.875, 0.875, -1.0)], p0=0.0)
    return w


def scaled(fn, n, **kw):
    """The recipe of `fn` at another grid size (small parity cases)."""
    return fn(n=n, **kw)


def by_name(name):
    table = {
        "dual_64": dual_64,
        "triple_1024": triple_1024,
        "precision_4096": precision_4096,
        "nlmc_1024": nlmc_1024,
        "paper_2c": lambda: paper_wells(2),
        "paper_3c": lambda: paper_wells(3),
    }
    return table[name]()
