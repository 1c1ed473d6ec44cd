"""Pins of the oracle's block COCG (the block variant of COCG, Section "Implementation"): one
column against the C COCG, the block solution against a dense solve, finite termination of the
block Krylov method on a small operator, and the two orthogonality relations that define block
conjugate gradients (a transposed or misplaced s x s factor breaks them)."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import brute


@pytest.fixture(scope="module")
def small():
    return synth.small_system((7, 6, 5), h=0.55, n_s=2, n_wells=2, seed=5)


def _rhs(n_d, s, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((s, n_d)) + 1j * rng.standard_normal((s, n_d))


def test_one_column_is_cocg(small):
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    b = _rhs(g.n_d, 1, 1)
    sig = -small.eps[0] + 0.2j
    xb, itb, stb = oracle.block_cocg(g, small.vloc, sig, b, 1e-10, 5000)
    xc, itc, stc = oracle.cocg(g, small.vloc, np.array([sig]), b, 1e-10, 5000)
    assert stb == oracle.OK and stc[0] == oracle.OK
    assert itb == itc[0]
    assert np.max(np.abs(xb - xc)) < 1e-10 * np.max(np.abs(xc))


@pytest.mark.parametrize("s", [2, 3, 5])
def test_matches_dense_solve(small, s):
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    H = brute.dense_h(small)
    b = _rhs(g.n_d, s, 2 + s)
    sig = -small.eps[1] + 0.1j
    x, it, st = oracle.block_cocg(g, small.vloc, sig, b, 1e-12, 5000)
    assert st == oracle.OK
    ref = np.linalg.solve(H + sig * np.eye(g.n_d), b.T).T
    # ||x - x*|| <= cond(A) ||r|| / ||A||-scale: with tol 1e-12 and cond ~ 1e3 well below 1e-8
    assert np.max(np.abs(x - ref)) < 1e-8 * np.max(np.abs(ref))
    # every column meets the stopping rule with the true residual
    A = H + sig * np.eye(g.n_d)
    res = np.linalg.norm(b.T - A @ x.T, axis=0) / np.linalg.norm(b.T, axis=0)
    assert np.all(res < 1e-11)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 6])
def test_finite_termination(s):
    """On an operator with N distinct eigenvalues the block Krylov space of s generic columns
    reaches the whole space after ceil(N / s) steps, so block COCG ends there (single-column COCG
    needs N); one step earlier the residuals are still above 1e-7 of the right-hand sides."""
    n = 12
    rng = np.random.default_rng(7)
    d = rng.uniform(1.0, 4.0, n) + 1j * rng.uniform(0.2, 1.0, n)     # complex symmetric (diagonal)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))                 # real orthogonal: A = Q D Q^T
    A = Qm @ np.diag(d) @ Qm.T
    b = _rhs(n, s, 8)
    steps = math.ceil(n / s)
    x, it, st = oracle.block_cocg_generic(lambda P: P @ A.T, b, 1e-9, steps)
    assert st == oracle.OK and it == steps
    ref = np.linalg.solve(A, b.T).T
    assert np.max(np.abs(x - ref)) < 1e-7 * np.max(np.abs(ref))
    _, it2, st2 = oracle.block_cocg_generic(lambda P: P @ A.T, b, 1e-7, steps - 1)
    assert st2 == oracle.NOT_CONVERGED


def test_block_orthogonality_and_conjugacy(small):
    """R_k^T R_l = 0 and P_k^T A P_l = 0 for k != l (unconjugated), the Galerkin conditions of
    block COCG, over the first iterations."""
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    sig = -small.eps[0] + 0.3j
    b = _rhs(g.n_d, 3, 11)
    hist = []
    oracle.block_cocg_generic(lambda P: np.array([oracle.apply_h(g, small.vloc, p, sig) for p in P]),
                              b, 1e-14, 6, history=hist)
    assert len(hist) == 6
    for k in range(6):
        for l in range(k):
            Rk, Pk, Qk = hist[k]
            Rl, Pl, Ql = hist[l]
            scale_r = np.linalg.norm(Rk) * np.linalg.norm(Rl)
            assert np.max(np.abs(Rk.T @ Rl)) < 1e-9 * scale_r
            scale_p = np.linalg.norm(Pk) * np.linalg.norm(Ql)
            assert np.max(np.abs(Pk.T @ Ql)) < 1e-9 * scale_p


@pytest.mark.parametrize("periodic", [False, True])
def test_chi0_by_blocks_matches_plain(small, periodic):
    s = small if not periodic else synth.small_system((8, 7, 6), h=0.5, n_s=2, n_wells=2, seed=6, periodic=True)
    o = oracle.Oracle.from_system(s)
    rng = np.random.default_rng(12)
    dv = rng.standard_normal((5, o.grid.n_d))          # blocks of 2: two full and a ragged one
    st_b = oracle.SolveStats()
    ref = o.chi0(dv, 0.4, 1e-11)
    got = o.chi0(dv, 0.4, 1e-11, block=2, stats=st_b)
    assert np.max(np.abs(got - ref)) < 1e-8 * np.max(np.abs(ref))
    assert st_b.n_solves() == 5 * o.n_s and st_b.worst_status() == oracle.OK
