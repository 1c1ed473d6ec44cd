"""Pins of the oracle's periodic boundary conditions (the bulk cells of the paper's Section
"Results"): closed-form spectra of the circulant finite-difference operators, plane waves,
dense LAPACK routes assembled independently (synth's Fornberg-weight circulant matrices),
and the brute-force sum over states of Eq. 2 on a periodic cell."""
import math

import numpy as np
import pytest

import oracle
from oracle import rpa_oracle as ro
import synth
from tests import brute


def symbol(n, h, m):
    """Eigenvalue of the periodic 1D second difference on the Fourier mode exp(2 pi i m j / n):
    (w0 + 2 sum_k wk cos(2 pi k m / n)) / h^2 (the stencil's symbol)."""
    w = oracle.fd_weights(6)
    th = 2 * math.pi * m / n
    return (w[0] + 2 * sum(w[k] * math.cos(k * th) for k in range(1, 7))) / h ** 2


@pytest.fixture(scope="module")
def pcube():
    return synth.small_system((8, 8, 8), h=0.5, n_s=3, n_wells=3, seed=31, periodic=True)


@pytest.fixture(scope="module")
def psmall():
    return synth.small_system((9, 8, 7), h=0.55, n_s=2, n_wells=2, seed=32, periodic=True)


@pytest.mark.parametrize("n", [5, 9, 13, 24])
def test_periodic_second_difference_has_the_stencil_symbol(n):
    h = 0.4
    D = ro.second_difference_1d(n, h, periodic=True)
    ref = np.sort([symbol(n, h, m) for m in range(n)])
    assert np.max(np.abs(np.sort(np.linalg.eigvalsh(D)) - ref)) < 1e-11 * np.max(np.abs(ref))
    j = np.arange(n)
    for m in range(n):   # the Fourier modes are its eigenvectors (n < 13: wrapped taps add up)
        e = np.exp(2j * math.pi * m * j / n)
        assert np.max(np.abs(D @ e - symbol(n, h, m) * e)) < 1e-11 * np.max(np.abs(ref))


def test_apply_h_periodic_on_plane_waves():
    nx, ny, nz, h = 9, 8, 7, 0.5                   # all below the stencil width: taps wrap twice
    g = oracle.Grid(nx, ny, nz, h, periodic=True)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sigma = 0.2 + 0.9j
    for (a, b, c) in [(1, 0, 0), (0, 3, 0), (0, 0, 2), (4, 5, 6), (8, 7, 6)]:
        f = np.exp(2j * math.pi * (a * i / nx + b * j / ny + c * k / nz)).reshape(-1)
        lam = -0.5 * (symbol(nx, h, a) + symbol(ny, h, b) + symbol(nz, h, c)) + sigma
        out = oracle.apply_h(g, np.zeros(g.n_d), f, sigma)
        assert np.max(np.abs(out - lam * f)) < 1e-11 * abs(lam)


def test_apply_h_periodic_matches_independent_assembly(psmall):
    g = oracle.Grid(psmall.nx, psmall.ny, psmall.nz, psmall.h, periodic=True)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(psmall.n_d) + 1j * rng.standard_normal(psmall.n_d)
    out = oracle.apply_h(g, psmall.vloc, v, -0.4 + 0.3j)
    ref = synth.hamiltonian_matrix(psmall) @ v + (-0.4 + 0.3j) * v
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)


def test_periodic_orbitals_are_eigenvectors_of_oracle_h(pcube):
    g = oracle.Grid(pcube.nx, pcube.ny, pcube.nz, pcube.h, periodic=True)
    for n in range(pcube.n_s):
        r = oracle.apply_h(g, pcube.vloc, pcube.psi[n].astype(complex)) - pcube.eps[n] * pcube.psi[n]
        assert np.linalg.norm(r) < 1e-10


def test_coulomb_periodic_plane_waves_and_the_g0_mode():
    nx, ny, nz, h = 10, 8, 12, 0.45
    g = oracle.Grid(nx, ny, nz, h, periodic=True)
    C = oracle.Coulomb(g)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for (a, b, c) in [(1, 0, 0), (0, 2, 5), (3, 3, 3), (5, 4, 6)]:
        f = np.cos(2 * math.pi * (a * i / nx + b * j / ny + c * k / nz)).reshape(1, -1)
        lam = -(symbol(nx, h, a) + symbol(ny, h, b) + symbol(nz, h, c))     # -L_h on the mode
        for p in (1.0, 0.5):
            out = C.apply(f, p)
            assert np.max(np.abs(out - (4 * math.pi / lam) ** p * f)) < 1e-11 * (4 * math.pi / lam) ** p
    one = np.ones((1, g.n_d))
    assert np.max(np.abs(C.apply(one, 1.0))) < 1e-12 and np.max(np.abs(C.apply(one, 0.5))) < 1e-12


def test_coulomb_periodic_matches_dense_pseudo_inverse(psmall):
    g = oracle.Grid(psmall.nx, psmall.ny, psmall.nz, psmall.h, periodic=True)
    C = oracle.Coulomb(g)
    X = synth.random_block(12, 3, g.n_d)
    for p in (1.0, 0.5):
        ref = X @ brute.nu_power_dense(g.nx, g.ny, g.nz, g.h, p, periodic=True).T
        assert np.max(np.abs(C.apply(X, p) - ref)) < 1e-11 * np.max(np.abs(ref))
    # Poisson's equation for a neutral charge (zero mean): -L phi = 4 pi rho, phi of zero mean
    rho = X - X.mean(axis=1, keepdims=True)
    A = brute.dense_minus_laplacian(g.nx, g.ny, g.nz, g.h, periodic=True)
    phi = C.apply(rho, 1.0)
    assert np.max(np.abs(phi @ A.T - 4 * math.pi * rho)) < 1e-10 * np.max(np.abs(4 * math.pi * rho))
    assert np.max(np.abs(phi.mean(axis=1))) < 1e-12 * np.max(np.abs(phi))


def test_cocg_periodic_matches_dense_solve(psmall):
    g = oracle.Grid(psmall.nx, psmall.ny, psmall.nz, psmall.h, periodic=True)
    H = brute.dense_h(psmall)
    rng = np.random.default_rng(13)
    b = rng.standard_normal((2, g.n_d)) + 1j * rng.standard_normal((2, g.n_d))
    sig = np.array([-psmall.eps[1] + 0.3j, 0.5 - 1.5j])
    x, it, st = oracle.cocg(g, psmall.vloc, sig, b, tol=1e-12, maxit=5000)
    assert np.all(st == oracle.OK)
    for s in range(2):
        A = H + sig[s] * np.eye(g.n_d)
        assert np.linalg.norm(b[s] - A @ x[s]) <= 1e-12 * np.linalg.norm(b[s]) * 1.01
        ref = np.linalg.solve(A, b[s])
        assert np.linalg.norm(x[s] - ref) <= 1e-12 * np.linalg.cond(A) * np.linalg.norm(ref)


@pytest.mark.parametrize("omega", [0.1, 2.0])
def test_chi0_periodic_matches_sum_over_states(pcube, omega):
    o = oracle.Oracle.from_system(pcube)
    assert o.grid.periodic
    dv = synth.random_block(14, 3, pcube.n_d)
    got = o.chi0(dv, omega, tol=1e-13, maxit=20000)
    ref = dv @ brute.chi0_sum_over_states(pcube, omega).T
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_rayleigh_ritz_full_rank_periodic_gives_dense_eigenvalues(pcube):
    o = oracle.Oracle.from_system(pcube)
    R = o.chi_tilde(np.eye(pcube.n_d), 0.9, tol=1e-13)
    lam = np.linalg.eigvalsh(0.5 * (R + R.T))
    ref = np.linalg.eigvalsh(brute.chi_tilde_dense(pcube, 0.9))
    assert np.max(np.abs(lam - ref)) < 1e-10
    assert ref.max() < 1e-10
