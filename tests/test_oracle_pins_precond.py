"""Pins of the oracle's Laplacian-preconditioned COCG (Section "Implementation": Laplacian-based
preconditioning through the Kronecker product formalism): the preconditioner against a dense
inverse, the solver against a dense solve, the identity preconditioner against plain COCG."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import brute


@pytest.fixture(scope="module")
def small():
    return synth.small_system((7, 6, 5), h=0.55, n_s=2, n_wells=2, seed=5)


@pytest.mark.parametrize("periodic", [False, True])
def test_preconditioner_is_the_dense_inverse(periodic):
    g = oracle.Grid(8, 7, 6, 0.5, periodic=periodic)
    C = oracle.Coulomb(g)
    shift = -0.8 + 0.3j
    m = oracle.laplacian_preconditioner(C, shift)
    A = 0.5 * brute.dense_minus_laplacian(g.nx, g.ny, g.nz, g.h, periodic) + shift * np.eye(g.n_d)
    rng = np.random.default_rng(3)
    R = rng.standard_normal((2, g.n_d)) + 1j * rng.standard_normal((2, g.n_d))
    ref = np.linalg.solve(A, R.T).T
    assert np.max(np.abs(m(R) - ref)) < 1e-11 * np.max(np.abs(ref))


def test_pcocg_matches_dense_solve(small):
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    H = brute.dense_h(small)
    rng = np.random.default_rng(4)
    b = rng.standard_normal((2, g.n_d)) + 1j * rng.standard_normal((2, g.n_d))
    sig = -small.eps[1] + 0.1j
    m = oracle.laplacian_preconditioner(oracle.Coulomb(g), float(np.mean(small.vloc)) + sig)
    x, it, st = oracle.pcocg(g, small.vloc, sig, b, 1e-12, 5000, m)
    assert np.all(st == oracle.OK)
    A = H + sig * np.eye(g.n_d)
    for s in range(2):
        assert np.linalg.norm(b[s] - A @ x[s]) <= 1e-12 * np.linalg.norm(b[s]) * 1.01
        ref = np.linalg.solve(A, b[s])
        assert np.linalg.norm(x[s] - ref) <= 1e-12 * np.linalg.cond(A) * np.linalg.norm(ref)


def test_pcocg_with_identity_is_cocg(small):
    """M = c I gives COCG's iterates exactly (rho and beta scale by c, alpha does not)."""
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    b = np.random.default_rng(5).standard_normal((1, g.n_d)).astype(complex)
    sig = -small.eps[0] + 0.7j
    x1, it1, _ = oracle.pcocg(g, small.vloc, sig, b, 1e-10, 5000, lambda r: 2.0 * r)
    x0, it0, _ = oracle.cocg(g, small.vloc, np.array([sig]), b, 1e-10, 5000)
    assert it1[0] == it0[0]
    assert np.max(np.abs(x1 - x0)) < 1e-12 * np.max(np.abs(x0))


def test_preconditioning_cuts_iterations_at_small_omega():
    s = synth.small_system((12, 12, 12), h=0.4, n_s=2, n_wells=2, seed=6)
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h)
    b = np.random.default_rng(6).standard_normal((2, g.n_d)).astype(complex)
    b = b - (b @ s.psi.T) @ s.psi
    sig = -s.eps[1] + 0.05j
    m = oracle.laplacian_preconditioner(oracle.Coulomb(g), float(np.mean(s.vloc)) + sig)
    _, itp, stp = oracle.pcocg(g, s.vloc, sig, b, 1e-10, 20000, m)
    _, itc, stc = oracle.cocg(g, s.vloc, np.full(2, sig), b, 1e-10, 20000)
    assert np.all(stp == 0) and np.all(stc == 0)
    assert np.all(itp < itc), (itp, itc)


def test_chi0_preconditioned_equals_chi0():
    s = synth.small_system((8, 8, 8), h=0.5, n_s=3, n_wells=3, seed=7)
    o = oracle.Oracle.from_system(s)
    dv = synth.random_block(4, 2, s.n_d)
    a = o.chi0(dv, 0.3, tol=1e-13, maxit=20000)
    b = o.chi0(dv, 0.3, tol=1e-13, maxit=20000, precondition=True)
    assert np.max(np.abs(a - b)) < 1e-9 * np.max(np.abs(a))
