"""Algorithm 1 (partition planning, hole filling) and Algorithm 2 (combine), plain Python.

Algorithm 1 chooses, for p windows, the request n_r,j and shift E_S,j from the
total request n_r, the extremal real parts E_min, E_max and the dimension N
(Section 2.2.1 and Algorithm 1).  Readings where the paper is silent:

* E_S,0 = E_min and n_r,0 = 0, so the first shift sits half a window above
  E_min.
* Odd p: the test ``j <= p/2`` is taken literally (real division).
* The hole-filling request n_r,j' is rounded up, minimum 1.

Algorithm 2 walks all computed pairs in order; a pair whose eigenvalue equals
that of an earlier kept pair (within a tolerance) is projected against it with
the unconjugated (bilinear) product, since the eigenvectors are bi-orthogonal
(Section 1); if what remains is small the pair is a duplicate and is removed,
and the interface it straddles is marked as having redundancy (no hole).
"""
from __future__ import annotations

import math

import numpy as np


def paper_round(x: float) -> int:
    """round() of Algorithm 1: halves round away from zero."""
    return int(math.floor(x + 0.5)) if x >= 0 else -int(math.floor(-x + 0.5))


def window_counts(n_r: int, p: int):
    """n_r,j of Algorithm 1 for j = 1..p."""
    n = [0] * (p + 1)  # 1-based
    for j in range(1, p + 1):
        if j <= p / 2:
            n[j] = paper_round(2.0 / (1.5 + (j - 1) / p) * n_r / p)
        else:
            n[j] = math.ceil(2 * n_r / p) - n[p - j + 1]
    return n[1:]


def window_shifts(counts, e_min: float, e_max: float, N: int):
    """E_S,j = E_S,j-1 + ((E_max - E_min)/N) (n_r,j + n_r,j-1)/2 with E_S,0 = E_min, n_r,0 = 0."""
    step = (e_max - e_min) / N
    shifts = []
    prev_s, prev_n = e_min, 0
    for c in counts:
        s = prev_s + step * (c + prev_n) / 2.0
        shifts.append(s)
        prev_s, prev_n = s, c
    return np.array(shifts)


def uniform_interval(r_min: float, r_max: float, n_r: int, N: int):
    """Interval of the lowest n_r eigenvalues assuming uniform density (Section 2.2.1)."""
    return r_min, r_min + (n_r / N) * (r_max - r_min)


def hole_window(eps_lower_window, eps_upper_window, e_min: float, e_max: float, N: int):
    """New window between two windows that show no redundancy (Algorithm 1, hole filling).

    Shift at the middle of the gap between the highest real part of the lower
    window and the lowest of the upper one; request 3/2 of the uniform-density
    count of the gap.
    """
    top = float(np.max(np.real(eps_lower_window)))
    bot = float(np.min(np.real(eps_upper_window)))
    shift = 0.5 * (top + bot)
    n_req = max(1, math.ceil(1.5 * (bot - top) / ((e_max - e_min) / N)))
    return shift, n_req


def hole_window_local(eps_lower_window, eps_upper_window, e_min: float, e_max: float, N: int, cap: int = 300):
    """Hole window with the request taken from the local spacing (a reading).

    Algorithm 1 sizes the request from the uniform spacing (E_max - E_min)/N;
    Section 2.2.1 suggests sampling the local density instead.  Reading: the
    mean spacing of the real parts the two neighbouring windows delivered
    (when they hold at least 4), 3/2 of the gap's count at that spacing plus 4
    (the new window must reach past both edges of the gap to overlap its
    neighbours), at most ``cap``; with fewer than 4 values, Algorithm 1's
    request (``hole_window``).  The shift is the same: the middle of the gap.
    """
    lo_re = np.real(np.asarray(eps_lower_window))
    hi_re = np.real(np.asarray(eps_upper_window))
    top, bot = float(np.max(lo_re)), float(np.min(hi_re))
    shift = 0.5 * (top + bot)
    both = np.concatenate([lo_re, hi_re])
    if len(both) >= 4 and both.max() > both.min():
        spacing = (both.max() - both.min()) / (len(both) - 1)
        n_req = math.ceil(1.5 * (bot - top) / spacing) + 4
    else:
        n_req = math.ceil(1.5 * (bot - top) / ((e_max - e_min) / N))
    return shift, int(min(cap, max(1, n_req)))


def merge_samples(spectrum, sample, prev_top: float, tol: float):
    """Add a sampling window's real parts to the sampled spectrum, with multiplicity (a reading).

    Section 2.2.1: a few eigenpairs at sample points estimate the density.
    Consecutive sample windows overlap, so a value found twice must count
    once; a twofold eigenvalue found twice in one sample must count twice.
    Values within tau = max(1e-7, 100 tol) max(1, |x|) of each other are one
    value up to multiplicity: a value of the sample is added when its rank
    among the sample's copies exceeds the copies already in the spectrum;
    values below prev_top - tau are already covered.
    """
    have = list(spectrum)
    out = list(spectrum)
    r = sorted(float(x) for x in sample)
    tau_rel = max(1e-7, 100.0 * tol)
    for i, x in enumerate(r):
        tau = tau_rel * max(1.0, abs(x))
        if x < prev_top - tau:
            continue
        rank = sum(1 for k in range(i + 1) if abs(r[k] - x) <= tau)
        old = sum(1 for y in have if abs(y - x) <= tau)
        if rank > old:
            out.append(x)
    return out


def complex_shift_window(eps, sigma: complex, n_req: int):
    """Indices of the eigenvalues a window with a complex shift delivers.

    Section 2 (after Eq. 5) extends the partition to strongly non-Hermitian
    problems with complex shifts on a two-dimensional grid; each window keeps
    the SM rule of Eq. 3 on A - sigma: the n_req eigenvalues nearest sigma in
    the complex plane, ties broken by (Re, Im) as for real shifts.
    """
    e = np.asarray(eps, dtype=np.complex128)
    d = np.abs(e - complex(sigma))
    order = np.lexsort((e.imag, e.real, d))
    return order[:n_req]


def combine(eps_list, U_list, eq_rtol: float = 1e-8, drop_tol: float = 1e-6):
    """Algorithm 2 over windows given in shift order.

    eps_list[j], U_list[j]: the pairs of window j (columns of U_list[j]).
    Returns (eps, U, window_of, holes) where holes[i] is True when the
    interface between windows i and i+1 showed no redundancy.  Surviving
    vectors are scaled to v^T v = 1.
    """
    p = len(eps_list)
    lam, vec, win = [], [], []
    for j in range(p):
        for k in range(len(eps_list[j])):
            lam.append(complex(eps_list[j][k]))
            vec.append(np.array(U_list[j][:, k], dtype=np.complex128))
            win.append(j)
    holes = [True] * max(0, p - 1)
    kept = []
    for k in range(len(lam)):
        v = vec[k].copy()
        n0 = np.linalg.norm(v)
        partner = None
        for m in kept:
            if abs(lam[m] - lam[k]) <= eq_rtol * max(1.0, abs(lam[k])):
                vm = vec[m]
                v = v - vm * ((vm @ v) / (vm @ vm))
                partner = m
        a = np.linalg.norm(v) / n0
        if a < drop_tol:
            if partner is not None and win[partner] != win[k]:
                lo, hi = sorted((win[partner], win[k]))
                for i in range(lo, hi):
                    holes[i] = False
            continue
        vec[k] = v / np.sqrt(v @ v)
        kept.append(k)
    eps = np.array([lam[k] for k in kept])
    U = np.stack([vec[k] for k in kept], axis=1) if kept else np.zeros((len(vec[0]) if vec else 0, 0))
    return eps, U, np.array([win[k] for k in kept]), holes
