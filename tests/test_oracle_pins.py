"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, LAPACK, closed forms, invariants the paper proves, or a
second formula for the same quantity.  None of them retypes the formula under
test.  All run on the CPU in a few seconds.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1602_01768_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _spd(n, kappa, seed):
    A, U, lam = wl.spd_spectrum(n, kappa, seed)
    return A, U, lam


def _sqrt_spd(U, lam):
    return (U * np.sqrt(lam)[None, :]) @ U.T


def _fa_err(Ahalf, X):
    """||A^{1/2} X A^{1/2} - I||_F = ||X - A^{-1}||_{F(A)} (notation, Sec. 1.2)."""
    n = X.shape[0]
    return np.linalg.norm(Ahalf @ X @ Ahalf - np.eye(n))


# --------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_gauss_sketch_moments_and_determinism():
    n, q = 4096, 64
    S = orc.gauss_sketch(7, 3, 11, n, q)
    z = S.ravel()
    N = z.size
    assert abs(z.mean()) < 5.0 / math.sqrt(N)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / N)
    assert abs(np.mean(z ** 4) - 3.0) < 5.0 * math.sqrt(96.0 / N)
    # columns nearly orthogonal: S^T S / n -> I
    G = S.T @ S / n
    assert np.max(np.abs(G - np.eye(q))) < 6.0 / math.sqrt(n)
    # same (seed, stream, k) -> same draw; any change -> a different draw
    assert np.array_equal(S, orc.gauss_sketch(7, 3, 11, n, q))
    for args in [(8, 3, 11), (7, 4, 11), (7, 3, 12)]:
        T = orc.gauss_sketch(*args, n, q)
        assert abs(np.corrcoef(S.ravel(), T.ravel())[0, 1]) < 0.01
    # a ragged n keeps the prefix of a longer draw (rows are a function of (row, col))
    S5 = orc.gauss_sketch(7, 3, 11, 4093, q)
    assert np.array_equal(S5, S[:4093])


def test_sketch_logf32_matches_libm():
    # the generator's binary32 ln against the platform's binary64 log, on the
    # 24-bit uniform grid it is used on (both ends included)
    xs = np.unique(np.concatenate([np.arange(0, 1 << 24, 977, dtype=np.int64),
                                   np.arange(0, 64), np.arange((1 << 24) - 64, 1 << 24)]))
    for x in xs:
        u = float(np.float32((x + 0.5) / 16777216.0))  # the binary32 uniform the generator uses
        got = float(orc.logf32(u))
        ref = math.log(u)
        ulp = float(np.spacing(np.float32(abs(ref)))) if ref != 0.0 else 0.0
        # a few roundings (divide, polynomial) on top of the series; a wrong
        # coefficient would be off by hundreds of ulps
        assert abs(got - ref) <= 8.0 * ulp, (u, got, ref)


def test_sketch_sincospif32_matches_libm():
    xs = np.concatenate([np.linspace(0.0, 2.0, 20001), [0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.75]])
    for x in xs:
        x = float(np.float32(x))
        s, c = orc.sincospif32(x)
        assert abs(float(s) - math.sin(math.pi * x)) <= 2.0 ** -22, x
        assert abs(float(c) - math.cos(math.pi * x)) <= 2.0 ** -22, x


def test_gauss_sketch_is_tf32_box_muller_of_the_philox_words():
    # every entry is the TF32 value nearest the binary64 Box-Muller normal of
    # its Philox words (computed here with numpy from the KAT-pinned Philox),
    # so a wrong word pairing, index or sign fails
    seed, stream, k, n, q = 0x1234_5678_9ABC_DEF0, 5, 9, 203, 7
    S = orc.gauss_sketch(seed, stream, k, n, q)
    f = S.astype(np.float32)
    assert np.array_equal(f.astype(np.float64), S)
    assert np.all((f.view(np.uint32) & 0x1FFF) == 0)  # 11 significant bits
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(q):
        for r in range((n + 3) // 4):
            w = orc.philox([r, j, k, stream], key)
            u = [float(np.float32(((int(x) >> 8) + 0.5) / 16777216.0)) for x in w]  # binary32 uniforms
            z = []
            for p in range(2):
                rad = math.sqrt(-2.0 * math.log(u[2 * p])) if u[2 * p] < 1.0 else 0.0
                z += [rad * math.cos(2 * math.pi * u[2 * p + 1]), rad * math.sin(2 * math.pi * u[2 * p + 1])]
            for t in range(4):
                if 4 * r + t < n:
                    v = S[4 * r + t, j]
                    assert abs(v - z[t]) <= 2.0 ** -11 * abs(z[t]) + 1e-6, (r, j, t, v, z[t])


def test_round_tf32_is_nearest_even():
    one = 1.0
    ulp = 2.0 ** -10
    assert float(orc.round_tf32(one + 0.49 * ulp)) == one
    assert float(orc.round_tf32(one + 0.51 * ulp)) == one + ulp
    assert float(orc.round_tf32(one + 0.5 * ulp)) == one                # tie -> even
    assert float(orc.round_tf32(one + 1.5 * ulp)) == one + 2 * ulp      # tie -> even
    assert float(orc.round_tf32(-(one + 0.51 * ulp))) == -(one + ulp)
    assert float(orc.round_tf32(2.0 - 0.4 * ulp)) == 2.0                # carries into the exponent


def test_floyd_sample_is_uniform_without_replacement():
    n, m, trials = 20, 5, 20000
    counts = np.zeros(n)
    for k in range(trials):
        s = orc.floyd_sample(1, 2, k, orc.TAG_COORD, n, m)
        assert len(set(s.tolist())) == m
        assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < n
        counts[s] += 1
    expect = trials * m / n
    chi2 = np.sum((counts - expect) ** 2 / expect)
    assert chi2 < 50.0  # 19 dof, p ~ 1e-4
    full = orc.floyd_sample(3, 0, 0, orc.TAG_COLS, 37, 37)
    assert np.array_equal(full, np.arange(37))


def test_coord_trace_block_frequencies_follow_diagonal():
    # blocks of q=3 over n=10 (last block ragged, size 1)
    d = np.array([1.0, 2.0, 3.0, 0.5, 0.5, 0.5, 4.0, 1.0, 1.0, 2.5])
    A = np.diag(d)
    q, nb = 3, 4
    w = np.array([d[0:3].sum(), d[3:6].sum(), d[6:9].sum(), d[9:].sum()])
    p = w / w.sum()
    trials = 20000
    counts = np.zeros(nb)
    for k in range(trials):
        b, first, size = orc.coord_trace_block(A, q, 5, 0, k)
        assert first == 3 * b and size == (1 if b == 3 else 3)
        counts[b] += 1
    chi2 = np.sum((counts - trials * p) ** 2 / (trials * p))
    assert chi2 < 25.0  # 3 dof


# --------------------------------------------------------------------------
# Small dense kernels
# --------------------------------------------------------------------------
@pytest.mark.parametrize("q", [1, 4, 7, 33])
def test_cholesky_matches_lapack(q):
    rng = np.random.default_rng(q)
    B = rng.standard_normal((q, q + 3))
    M = B @ B.T + 0.1 * np.eye(q)
    rc, C = orc.cholesky(M)
    assert rc == 0
    assert np.allclose(C, np.linalg.cholesky(M), rtol=1e-12, atol=1e-12)
    assert np.allclose(np.triu(C, 1), 0.0)


def test_cholesky_reports_indefinite():
    M = np.diag([1.0, -1.0, 2.0])
    rc, _ = orc.cholesky(M)
    assert rc == -1
    rc, _ = orc.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert rc == -1


@pytest.mark.parametrize("n", [1, 5, 64])
def test_gauss_jordan_matches_lapack(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    assert np.allclose(orc.gauss_jordan(A), np.linalg.inv(A), rtol=1e-11, atol=1e-12)


# --------------------------------------------------------------------------
# RBFGS (Eq. (qunac), Algorithm 3 with W = A^-1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("form", [0, 1])
def test_rbfgs_step_invariants(form):
    n, q = 40, 6
    A, U, lam = _spd(n, 50.0, 3)
    Ainv = np.linalg.inv(A)
    rng = np.random.default_rng(0)
    B = rng.standard_normal((n, n))
    X = B @ B.T / n + np.eye(n)  # symmetric positive definite start
    S = orc.gauss_sketch(1, 0, 0, n, q)
    rc, Xp = orc.rbfgs_step(A, X, S, form)
    assert rc == 0
    # sketch equation S^T A X+ = S^T (constraint of Eq. (NFsym)), i.e. X+ A S = S
    assert np.linalg.norm(Xp @ A @ S - S) / np.linalg.norm(S) < 1e-12
    # symmetry and positive definiteness preserved (Sec. 8.8)
    assert np.linalg.norm(Xp - Xp.T) / np.linalg.norm(Xp) < 1e-13
    assert np.linalg.eigvalsh(0.5 * (Xp + Xp.T)).min() > 0
    # error recursion Eq. (XZupdatesym) with W = A^-1:
    # X+ - A^-1 = (I - P A)(X - A^-1)(I - A P),  P = S (S^T A S)^-1 S^T
    P = S @ np.linalg.solve(S.T @ A @ S, S.T)
    I = np.eye(n)
    E = (I - P @ A) @ (X - Ainv) @ (I - A @ P)
    assert np.linalg.norm((Xp - Ainv) - E) / np.linalg.norm(E) < 1e-10


def test_rbfgs_literal_and_expanded_forms_agree():
    n, q = 32, 5
    A, _, _ = _spd(n, 100.0, 9)
    X = np.eye(n)
    for k in range(5):
        S = orc.gauss_sketch(2, 1, k, n, q)
        rc0, X0 = orc.rbfgs_step(A, X, S, 0)
        rc1, X1 = orc.rbfgs_step(A, X, S, 1)
        assert rc0 == rc1 == 0
        assert np.linalg.norm(X0 - X1) / np.linalg.norm(X1) < 1e-12
        X = X1


def test_rbfgs_one_step_with_invertible_sketch():
    # Sec. 8.1: S invertible (q = n) gives X1 = A^-1 in one step
    n = 24
    A, _, _ = _spd(n, 1e3, 4)
    S = np.eye(n)
    rc, X1 = orc.rbfgs_step(A, np.eye(n), S, 1)
    assert rc == 0
    Ainv = orc.gauss_jordan(A)
    assert np.linalg.norm(X1 - Ainv) / np.linalg.norm(Ainv) < 1e-11
    S = orc.gauss_sketch(3, 0, 0, n, n)
    rc, X1 = orc.rbfgs_step(A, np.eye(n), S, 0)
    assert np.linalg.norm(X1 - Ainv) / np.linalg.norm(Ainv) < 1e-9


def test_rbfgs_fixed_point():
    n, q = 30, 4
    A, _, _ = _spd(n, 20.0, 5)
    Ainv = np.linalg.inv(A)
    S = orc.gauss_sketch(4, 0, 0, n, q)
    rc, X1 = orc.rbfgs_step(A, Ainv, S, 1)
    assert np.linalg.norm(X1 - Ainv) / np.linalg.norm(Ainv) < 1e-12


def test_rbfgs_error_never_increases_in_FA_norm():
    # proof of Thm 6.2: ||R_{k+1}||_F <= ||R_k||_F for every sample (I - Z^ a projection)
    n, q = 48, 4
    A, U, lam = _spd(n, 100.0, 6)
    Ah = _sqrt_spd(U, lam)
    X = np.eye(n)
    prev = _fa_err(Ah, X)
    for k in range(40):
        S = orc.gauss_sketch(5, 0, k, n, q)
        rc, X = orc.rbfgs_step(A, X, S, 1)
        cur = _fa_err(Ah, X)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_rbfgs_coordinate_rate_bound():
    # Prop. 7.2 / Eq. (convqunac): with S a block of coordinates drawn with
    # p_b proportional to the block trace, E||X_k - A^-1||^2_{F(A)} <= rho^k ||X_0 - A^-1||^2_{F(A)},
    # rho = 1 - lambda_min(A) / Tr(A) (the stacked sketch is a permutation).
    n, q, k, seeds = 12, 3, 30, 300
    A, U, lam = _spd(n, 8.0, 7)
    Ah = _sqrt_spd(U, lam)
    rho = 1.0 - lam.min() / lam.sum()
    e0 = _fa_err(Ah, np.eye(n)) ** 2
    errs = []
    for s in range(seeds):
        done, X = orc.rbfgs_run(A, np.eye(n), q, orc.SKETCH_COORD_TRACE, s, 0, 0, k)
        assert done == k
        errs.append(_fa_err(Ah, X) ** 2)
    assert np.mean(errs) <= rho ** k * e0
    # coordinate steps change only rows/columns of the drawn block
    b, first, size = orc.coord_trace_block(A, q, 99, 0, 0)
    X0 = np.eye(n) * 2.0
    _, X1 = orc.rbfgs_run(A, X0, q, orc.SKETCH_COORD_TRACE, 99, 0, 0, 1)
    mask = np.ones(n, bool)
    mask[first:first + size] = False
    assert np.array_equal(X1[np.ix_(mask, mask)], X0[np.ix_(mask, mask)])


# --------------------------------------------------------------------------
# Approximate inverse preconditioning, Eq. (BFGSas) (Sec. 8, Algorithm 1 with W = A^-1)
# --------------------------------------------------------------------------
def test_aip_sketch_equation_and_nonsymmetric_iterate():
    # S^T A X+ = S^T (the row variant's constraint), and X+ is not symmetric in general
    n, q = 40, 6
    A, _, _ = _spd(n, 50.0, 31)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((n, n)) * 0.05
    S = orc.gauss_sketch(11, 0, 0, n, q)
    rc, X1 = orc.aip_step(A, X, S)
    assert rc == 0
    assert np.allclose(S.T @ A @ X1, S.T, atol=1e-10)
    assert np.max(np.abs(X1 - X1.T)) > 1e-3


def test_aip_is_the_constrain_and_approximate_minimiser():
    # Sec. 8: X+ = argmin ||A^{1/2} X A^{1/2} - I||_F over X = X_k + S Y^T.  Brute force: with
    # B = A^{1/2} S and Z = Y^T A^{1/2} (any q x n), minimise ||E0 + B Z||_F by least squares.
    n, q = 24, 5
    A, U, lam = _spd(n, 30.0, 32)
    Ah = _sqrt_spd(U, lam)
    Ahinv = (U / np.sqrt(lam)[None, :]) @ U.T
    rng = np.random.default_rng(5)
    X = rng.standard_normal((n, n)) * 0.1
    S = rng.standard_normal((n, q))
    E0 = Ah @ X @ Ah - np.eye(n)
    Bm = Ah @ S
    Z, *_ = np.linalg.lstsq(Bm, -E0, rcond=None)
    Xstar = X + S @ Z @ Ahinv
    rc, X1 = orc.aip_step(A, X, S)
    assert rc == 0
    assert np.max(np.abs(X1 - Xstar)) <= 1e-9 * max(1.0, np.max(np.abs(Xstar)))


def test_aip_error_never_increases_and_one_step_inverse():
    # E+ = (I - P) E with P = A^{1/2} S (S^T A S)^-1 S^T A^{1/2} an orthogonal projection
    n, q = 30, 4
    A, U, lam = _spd(n, 100.0, 33)
    Ah = _sqrt_spd(U, lam)
    X = np.eye(n)
    for k in range(25):
        S = orc.gauss_sketch(12, 0, k, n, q)
        before = _fa_err(Ah, X)
        rc, X = orc.aip_step(A, X, S)
        assert rc == 0
        assert _fa_err(Ah, X) <= before * (1 + 1e-12)
    # q = n with an invertible sketch: X_1 = A^-1 from any X_0 (Gauss-Jordan brute force)
    Ainv = orc.gauss_jordan(A)
    rc, X1 = orc.aip_step(A, np.ones((n, n)), orc.gauss_sketch(13, 0, 0, n, n))
    assert rc == 0 and np.allclose(X1, Ainv, rtol=1e-8, atol=1e-8 * np.abs(Ainv).max())
    # the inverse is a fixed point
    rc, X2 = orc.aip_step(A, Ainv, orc.gauss_sketch(14, 0, 0, n, q))
    assert np.allclose(X2, Ainv, atol=1e-10 * np.abs(Ainv).max())


def test_aip_coordinate_rate_bound():
    # Eq. (BBonv): block coordinates with p_b = block trace / Tr A (the stacked sketch is a
    # permutation) give E||A^{1/2} X_k A^{1/2} - I||^2_F <= (1 - lambda_min(A)/Tr(A))^k ||..X_0..||^2
    n, q, k, seeds = 12, 3, 30, 300
    A, U, lam = _spd(n, 8.0, 34)
    Ah = _sqrt_spd(U, lam)
    rho = 1.0 - lam.min() / lam.sum()
    e0 = _fa_err(Ah, np.eye(n)) ** 2
    errs = []
    for s in range(seeds):
        done, X = orc.aip_run(A, np.eye(n), q, orc.SKETCH_COORD_TRACE, s, 0, 0, k)
        assert done == k
        errs.append(_fa_err(Ah, X) ** 2)
    assert np.mean(errs) <= rho ** k * e0
    # a coordinate step changes only the rows of the drawn block
    b, first, size = orc.coord_trace_block(A, q, 99, 0, 0)
    X0 = np.eye(n) * 2.0
    _, X1 = orc.aip_run(A, X0, q, orc.SKETCH_COORD_TRACE, 99, 0, 0, 1)
    mask = np.ones(n, bool)
    mask[first:first + size] = False
    assert np.array_equal(X1[mask], X0[mask])


# --------------------------------------------------------------------------
# AdaRBFGS (Eq. (Cholimprov), Algorithm 4)
# --------------------------------------------------------------------------
def test_adarbfgs_factor_reproduces_rbfgs_iterate():
    # Eq. (Chol)/(Cholimprov): L+ L+^T equals the BFGS update of X = L L^T with S = L S~
    n, q = 36, 5
    A, _, _ = _spd(n, 200.0, 8)
    rng = np.random.default_rng(1)
    L = np.eye(n) + 0.2 * rng.standard_normal((n, n))
    St = orc.gauss_sketch(6, 0, 0, n, q)
    rc, Lp = orc.adarbfgs_step(A, L, St)
    assert rc == 0
    rc, Xp = orc.rbfgs_step(A, L @ L.T, L @ St, 0)
    assert np.linalg.norm(Lp @ Lp.T - Xp) / np.linalg.norm(Xp) < 1e-11
    # sketch equation on the factored iterate
    S = L @ St
    assert np.linalg.norm(Lp @ Lp.T @ A @ S - S) / np.linalg.norm(S) < 1e-11


def test_adarbfgs_cols_sketch_is_the_rbfgs_step_on_columns_of_L():
    n, q = 30, 4
    A, _, _ = _spd(n, 50.0, 10)
    rng = np.random.default_rng(2)
    L = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    C = orc.floyd_sample(3, 0, 0, orc.TAG_COORD, n, q)
    St = np.zeros((n, q))
    St[C, np.arange(q)] = 1.0
    rc, Lp = orc.adarbfgs_step(A, L, St)
    rc2, Xp = orc.rbfgs_step(A, L @ L.T, L[:, C], 1)
    assert rc == rc2 == 0
    assert np.linalg.norm(Lp @ Lp.T - Xp) / np.linalg.norm(Xp) < 1e-11
    done, Lr = orc.adarbfgs_run(A, L, q, orc.SKETCH_COORD_UNIFORM, 3, 0, 0, 1)
    assert done == 1 and np.allclose(Lr, Lp, rtol=0, atol=1e-14)


def test_adarbfgs_one_step_and_fixed_point():
    n = 20
    A, _, _ = _spd(n, 1e2, 11)
    Ainv = orc.gauss_jordan(A)
    rc, L1 = orc.adarbfgs_step(A, np.eye(n), np.eye(n))  # S~ = I: S invertible
    assert rc == 0
    assert np.linalg.norm(L1 @ L1.T - Ainv) / np.linalg.norm(Ainv) < 1e-11
    # at L with L L^T = A^-1, V = 0 and L is unchanged
    Lstar = np.linalg.cholesky(Ainv)
    St = orc.gauss_sketch(1, 0, 0, n, 3)
    rc, L2 = orc.adarbfgs_step(A, Lstar, St)
    assert np.linalg.norm(L2 - Lstar) / np.linalg.norm(Lstar) < 1e-11


def test_adarbfgs_gauss_converges_monotonically():
    n, q = 64, 8
    A, U, lam = _spd(n, 100.0, 12)
    Ah = _sqrt_spd(U, lam)
    L = np.eye(n)
    prev = _fa_err(Ah, L @ L.T)
    for k in range(120):
        St = orc.gauss_sketch(9, 0, k, n, q)
        rc, L = orc.adarbfgs_step(A, L, St)
        assert rc == 0
        cur = _fa_err(Ah, L @ L.T)
        assert cur <= prev * (1 + 1e-10)
        prev = cur
    assert orc.residual_factored(A, L) < 1e-4
    # the same 120 steps through the run driver
    done, L2 = orc.adarbfgs_run(A, np.eye(n), q, orc.SKETCH_GAUSS, 9, 0, 0, 120)
    assert done == 120 and np.allclose(L2, L, rtol=0, atol=1e-13)


def test_adarbfgs_adaptive_partition_step_meets_theorem_9_1():
    # Thm 9.1: with S = L_k I_{:C_i} for a partition {C_i} of [n], drawn with p_i proportional
    # to Tr(S_i^T A S_i), one AdaRBFGS step satisfies
    #   E[||X+ - A^-1||^2_F(A) | X_k] <= (1 - lambda_min(A X_k) / Tr(A X_k)) ||X_k - A^-1||^2_F(A).
    # The conditional expectation is taken exactly, by enumerating every block of the partition.
    n, q = 24, 4
    A, U, lam = _spd(n, 40.0, 15)
    Ah = _sqrt_spd(U, lam)
    for seed in range(4):
        rng = np.random.default_rng(100 + seed)
        L = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
        X = L @ L.T
        blocks = [np.arange(b, min(n, b + q)) for b in range(0, n, q)]
        w = np.array([np.trace(L[:, C].T @ A @ L[:, C]) for C in blocks])
        p = w / w.sum()
        e_next = 0.0
        for C, pi in zip(blocks, p):
            St = np.zeros((n, len(C)))
            St[C, np.arange(len(C))] = 1.0
            rc, Lp = orc.adarbfgs_step(A, L, St)
            assert rc == 0
            e_next += pi * _fa_err(Ah, Lp @ Lp.T) ** 2
        ax = np.linalg.eigvals(A @ X).real
        bound = (1.0 - ax.min() / np.trace(A @ X)) * _fa_err(Ah, X) ** 2
        assert e_next <= bound * (1 + 1e-10), (seed, e_next, bound)


def test_rbfgs_rate_lower_bound_rholower():
    # Eq. (rholower): rho >= 1 - q/n.  Each Z^ = A^{1/2} S (S^T A S)^-1 S^T A^{1/2} is a rank-q
    # projection (Lemma of Sec. 6), so Tr E[Z^] = q and lambda_min(E[Z^]) <= q/n.  The bound is
    # attained from X_0 = 0: there R_0 = -I and R_1 = -(I - Z^) for every sketch, so one RBFGS
    # step contracts ||X - A^-1||^2_F(A) by exactly 1 - q/n.
    n, q = 30, 5
    A, U, lam = _spd(n, 60.0, 16)
    Ah = _sqrt_spd(U, lam)
    Zsum = np.zeros((n, n))
    for k in range(200):
        S = orc.gauss_sketch(21, 0, k, n, q)
        rc, X1 = orc.rbfgs_step(A, np.zeros((n, n)), S, 1)
        assert rc == 0
        Zh = Ah @ X1 @ Ah  # X1 = S (S^T A S)^-1 S^T from X_0 = 0
        assert np.linalg.norm(Zh @ Zh - Zh) < 1e-10 * n
        assert abs(np.trace(Zh) - q) < 1e-10 * n
        ratio = _fa_err(Ah, X1) ** 2 / _fa_err(Ah, np.zeros((n, n))) ** 2
        assert abs(ratio - (1.0 - q / n)) < 1e-10
        Zsum += Zh
    rho_hat = 1.0 - np.linalg.eigvalsh(Zsum / 200).min()
    assert rho_hat >= 1.0 - q / n - 1e-12


def test_adarbfgs_reports_rank_deficient_sketch():
    n = 10
    A, _, _ = _spd(n, 10.0, 13)
    St = np.zeros((n, 2))
    St[0, 0] = 1.0  # a zero column: S^T A S has an exactly zero pivot
    rc, L = orc.adarbfgs_step(A, np.eye(n), St)
    assert rc == -1
    assert np.array_equal(L, np.eye(n))
    # an indefinite "A" breaks the same Cholesky
    rc, L = orc.adarbfgs_step(-A, np.eye(n), orc.gauss_sketch(1, 0, 0, n, 3))
    assert rc == -1


# --------------------------------------------------------------------------
# Newton-Schulz, MR and the residual monitor (Sec. 10)
# --------------------------------------------------------------------------
def test_power_norm_matches_lapack():
    A, _, lam = _spd(50, 30.0, 14)
    # gap lambda_2/lambda_1 = 0.988 here: 3000 iterations leave ~1e-30
    assert abs(orc.power_norm(A, 3000) - lam.max()) / lam.max() < 1e-12


def test_newton_schulz_squares_the_error():
    n = 32
    A, _, lam = _spd(n, 50.0, 15)
    X = orc.ns_init(A, lam.max())
    I = np.eye(n)
    # ||I - X0 A||_2 = 1 - 0.99/kappa^2 ~ 0.9996: about 17 squarings to converge
    for _ in range(22):
        E = I - X @ A
        X = orc.ns_step(A, X)
        E1 = I - X @ A
        assert np.linalg.norm(E1 - E @ E) <= 1e-12 * max(1.0, np.linalg.norm(E))
    assert np.linalg.norm(X - orc.gauss_jordan(A)) / np.linalg.norm(X) < 1e-10


def test_mr_step_length_is_optimal():
    n = 24
    A, _, _ = _spd(n, 40.0, 16)
    X = orc.mr_init(A)
    assert np.allclose(np.diag(X), np.trace(A) / np.sum(A * A))
    I = np.eye(n)
    for _ in range(3):
        alpha, X1 = orc.mr_step(A, X)
        D = X1 - X  # = alpha * X R
        f = lambda a: np.linalg.norm(I - A @ (X + a * D / alpha)) ** 2
        for da in (1e-3, -1e-3):
            assert f(alpha) <= f(alpha * (1 + da))
        assert np.linalg.norm(I - A @ X1) < np.linalg.norm(I - A @ X)
        X = X1


def test_residuals_closed_forms():
    n = 40
    A, _, _ = _spd(n, 10.0, 17)
    Ainv = np.linalg.inv(A)
    assert orc.residual(A, Ainv) < 1e-13
    assert abs(orc.residual(A, np.zeros((n, n))) - 1.0) < 1e-15
    # alpha I: ||I - alpha A||_F / sqrt(n) from the spectrum
    lam = np.linalg.eigvalsh(A)
    a = 0.7
    assert abs(orc.residual(A, a * np.eye(n)) - np.sqrt(np.mean((1 - a * lam) ** 2))) < 1e-13
    rng = np.random.default_rng(3)
    L = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    X = L @ L.T
    exact = orc.residual(A, X)
    assert abs(orc.residual_factored(A, L) - exact) < 1e-13
    assert abs(orc.residual_sampled(A, n, 5, X=X) - exact) < 1e-13
    assert abs(orc.residual_sampled(A, n, 5, L=L) - exact) < 1e-13
    est = np.mean([orc.residual_sampled(A, 8, s, X=X) ** 2 for s in range(400)])
    assert abs(est - exact ** 2) / exact ** 2 < 0.1
