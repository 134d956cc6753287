"""Pins for Algorithm 1 (planning, hole filling) and Algorithm 2 (combine)."""
import numpy as np

from oracle import partition
from conftest import golden_path


def _golden_counts():
    rows = []
    with open(golden_path("algorithm1_counts.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split(":")
            n_r, p = (int(x) for x in lhs.split())
            rows.append((n_r, p, [int(x) for x in rhs.split()]))
    return rows


def test_window_counts_worked_by_hand():
    for n_r, p, expect in _golden_counts():
        assert partition.window_counts(n_r, p) == expect, (n_r, p)


def test_coverage_constraint_eq4():
    # Eq. (4): sum_j n_r,j >= n_r for every plan.
    for n_r in (1, 7, 48, 100, 401, 2000, 3209):
        for p in range(1, 33):
            assert sum(partition.window_counts(n_r, p)) >= n_r


def test_odd_p_literal_reading():
    # p = 3, n_r = 30: j=1 -> round(2/1.5 * 10) = 13; j=2 (> 1.5) -> ceil(20) - n_2 = 20 - 0
    # (n_2 not yet set: literal reading); j=3 -> 20 - 13 = 7.
    assert partition.window_counts(30, 3) == [13, 20, 7]


def test_shift_placement_by_hand():
    # E_min = 0, E_max = N -> unit spacing; counts (16, 14, 10, 8):
    # 8, 8 + 15 = 23, 23 + 12 = 35, 35 + 9 = 44.
    s = partition.window_shifts([16, 14, 10, 8], 0.0, 1000.0, 1000)
    np.testing.assert_allclose(s, [8.0, 23.0, 35.0, 44.0])


def test_uniform_interval():
    assert partition.uniform_interval(-1.0, 3.0, 10, 40) == (-1.0, 0.0)


def test_hole_window_by_hand():
    # gap between 1.0 and 1.5 with spacing (2-0)/64 = 1/32: 16 states -> request 24.
    s, n = partition.hole_window([0.25, 1.0 - 0.01j], [1.5, 1.75], 0.0, 2.0, 64)
    assert s == 1.25 and n == 24


def _bilinear_unit(v):
    return v / np.sqrt(v @ v)


def test_hole_window_local_by_hand():
    # lower window real parts 0.0, 0.1, 0.2, 0.3; upper 0.9, 1.0: 6 values over
    # [0, 1], mean spacing 1/5 = 0.2; gap 0.3 .. 0.9 = 0.6, 3/2 x 0.6/0.2 = 4.5
    # -> 5, plus 4 = 9; shift at 0.6
    s, n = partition.hole_window_local([0.0, 0.1, 0.2 - 0.01j, 0.3], [0.9, 1.0], 0.0, 2.0, 64)
    assert abs(s - 0.6) < 1e-15 and n == 9
    # fewer than 4 values: Algorithm 1's uniform request (as hole_window)
    assert partition.hole_window_local([0.25, 1.0], [1.5], 0.0, 2.0, 64) == \
        partition.hole_window([0.25, 1.0], [1.5], 0.0, 2.0, 64)
    # the cap
    _, n = partition.hole_window_local([0.0, 0.1, 0.2, 0.3], [0.9, 1.0], 0.0, 2.0, 64, cap=5)
    assert n == 5


def test_merge_samples_counts_with_multiplicity():
    tol = 1e-8  # tau = 1e-6 max(1, |x|)
    spec = [0.1, 0.2, 0.3]
    # a repeat of values already sampled (overlapping windows) counts once;
    # values below the previous top are covered; a new value is added
    out = partition.merge_samples(spec, [0.2 + 1e-9, 0.3 - 1e-9, 0.4], prev_top=0.3, tol=tol)
    assert out == [0.1, 0.2, 0.3, 0.4]
    # a twofold value at the previous top: the earlier sample held one copy,
    # this one holds both -> one more copy
    out = partition.merge_samples(spec, [0.3, 0.3 + 2e-9, 0.5], prev_top=0.3, tol=tol)
    assert sorted(out) == [0.1, 0.2, 0.3, 0.3 + 2e-9, 0.5]
    # a new twofold value above counts twice
    out = partition.merge_samples(spec, [0.6, 0.6], prev_top=0.3, tol=tol)
    assert out == [0.1, 0.2, 0.3, 0.6, 0.6]
    # distinct values farther apart than tau are separate
    out = partition.merge_samples([], [1.0, 1.0 + 1e-5], prev_top=-np.inf, tol=tol)
    assert out == [1.0, 1.0 + 1e-5]


def test_combine_removes_duplicates_and_keeps_degenerate_partners():
    rng = np.random.default_rng(0)
    N = 50
    basis = [rng.standard_normal(N) + 0.1j * rng.standard_normal(N) for _ in range(6)]
    # Make 6 bilinear-orthonormal vectors by Gram-Schmidt (test's own, plain loop).
    vs = []
    for v in basis:
        for u in vs:
            v = v - u * (u @ v)
        vs.append(_bilinear_unit(v))
    lam = np.array([0.1, 0.2, 0.3, 0.3, 0.4, 0.5]) - 0.01j  # 0.3 is a degenerate pair
    # window 0 has pairs 0..3, window 1 has 2..5 (2, 3 duplicated, with noise).
    noise = 1e-12
    w0_e = lam[:4]
    w0_u = np.stack(vs[:4], 1)
    mix = (vs[2] + 0.5 * vs[3])  # a different basis of the degenerate space
    w1_e = np.array([lam[2] + 1e-13, lam[2], lam[4], lam[5]])
    w1_u = np.stack([mix + noise * basis[0], vs[3] - noise * basis[1], vs[4], vs[5]], 1)
    e, U, win, holes = partition.combine([w0_e, w1_e], [w0_u, w1_u])
    assert len(e) == 6
    np.testing.assert_allclose(np.sort(e.real), np.sort(lam.real), atol=1e-12)
    assert holes == [False]
    np.testing.assert_allclose(U.T @ U, np.eye(6), atol=1e-9)


def test_combine_gap_leaves_hole_flag():
    rng = np.random.default_rng(1)
    N = 30
    vs = []
    for _ in range(4):
        v = rng.standard_normal(N) + 0j
        for u in vs:
            v = v - u * (u @ v)
        vs.append(_bilinear_unit(v))
    e, U, win, holes = partition.combine([np.array([0.1, 0.2]), np.array([0.5, 0.6])],
                                         [np.stack(vs[:2], 1), np.stack(vs[2:], 1)])
    assert len(e) == 4 and holes == [True]


def test_complex_shift_window_by_hand():
    # distances to sigma = 0.5 - 0.5i: 0 -> 0.707, 1 -> 0.707, -i -> 0.707,
    # 2 - 0.5i -> 1.5, -1 -> 1.58; the three-way tie is broken by (Re, Im):
    # -i (Re 0, Im -1), then 0 (Re 0, Im 0), then 1
    eps = np.array([0.0, 1.0, -1j, 2.0 - 0.5j, -1.0])
    assert list(partition.complex_shift_window(eps, 0.5 - 0.5j, 2)) == [2, 0]
    assert list(partition.complex_shift_window(eps, 0.5 - 0.5j, 3)) == [2, 0, 1]
    assert list(partition.complex_shift_window(eps, 2.0 - 0.6j, 1)) == [3]
    # a real shift: the eigenvalues nearest it on the real axis
    assert sorted(partition.complex_shift_window(eps, -0.9, 2)) == [0, 4]
