"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something other than itself: textbook weights,
closed forms, dense LAPACK routes assembled independently, the brute-force sum over
states of Eq. 2, or invariants of chi0 stated in the Formulation.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.integrate as si

import oracle
import synth
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def small():
    return synth.small_system((7, 6, 5), h=0.55, n_s=2, n_wells=2, seed=5)


@pytest.fixture(scope="module")
def cube():
    return synth.small_system((8, 8, 8), h=0.5, n_s=3, n_wells=3, seed=7)


# ------------------------------------------------------------------ finite differences
def test_fd_weights_match_textbook_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fd_weights_order12.txt"))
            if l.strip() and not l.startswith("#")]
    ref = np.array([float(Fraction(int(n), int(d))) for _, n, d in rows])
    assert np.max(np.abs(oracle.fd_weights(6) - ref)) < 1e-15


def test_fd_weights_polynomial_exactness():
    w = oracle.fd_weights(6)
    for m in range(0, 16):
        val = (w[0] if m == 0 else 0.0) + sum(w[k] * (k ** m + (-k) ** m) for k in range(1, 7))
        exact = 2.0 if m == 2 else 0.0
        if m <= 13:
            assert abs(val - exact) < 1e-9 * max(1, 6 ** m), m
        elif m == 14:
            assert abs(val - exact) > 1.0  # order is exactly 12


def test_fd_weights_agree_with_fornberg_recursion():
    assert np.max(np.abs(oracle.fd_weights(6) - synth.fornberg_second_derivative(6))) < 1e-13


# ------------------------------------------------------------------ Hamiltonian
def test_apply_h_matches_independent_assembly(small):
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(small.n_d) + 1j * rng.standard_normal(small.n_d)
    sigma = 0.3 - 0.7j
    out = oracle.apply_h(g, small.vloc, v, sigma)
    ref = synth.hamiltonian_matrix(small) @ v + sigma * v
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)


def test_apply_h_polynomial_interior():
    n, h = 20, 0.3
    g = oracle.Grid(n, n, n, h)
    c = (np.arange(n) + 1.0) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = X ** 5 * Y ** 3 - 2 * Z ** 6 + X * Y * Z ** 4
    lap = 20 * X ** 3 * Y ** 3 + 6 * X ** 5 * Y - 60 * Z ** 4 + 12 * X * Y * Z ** 2
    out = oracle.apply_h(g, np.zeros(g.n_d), f.reshape(-1).astype(complex)).reshape(f.shape)
    inner = (slice(6, n - 6),) * 3
    assert np.max(np.abs(out[inner] - (-0.5 * lap[inner]))) < 1e-8 * np.max(np.abs(lap))


def test_orbitals_are_eigenvectors_of_oracle_h():
    s = synth.workload("tiny15").system
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h)
    assert np.max(np.abs(s.psi @ s.psi.T - np.eye(s.n_s))) < 1e-12
    for n in range(s.n_s):
        r = oracle.apply_h(g, s.vloc, s.psi[n].astype(complex)) - s.eps[n] * s.psi[n]
        assert np.linalg.norm(r) < 1e-10


# ------------------------------------------------------------------ Coulomb operator
def test_coulomb_matches_dense_inverse(small):
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    C = oracle.Coulomb(g)
    X = synth.random_block(3, 4, g.n_d)
    for p in (1.0, 0.5):
        ref = X @ brute.nu_power_dense(g.nx, g.ny, g.nz, g.h, p).T
        assert np.max(np.abs(C.apply(X, p) - ref)) < 1e-11 * np.max(np.abs(ref))
    # nu^1 against a plain linear solve of the Poisson equation (Eq. 5): -L phi = 4 pi rho
    A = brute.dense_minus_laplacian(g.nx, g.ny, g.nz, g.h)
    phi = np.linalg.solve(A, 4 * math.pi * X.T).T
    assert np.max(np.abs(C.apply(X, 1.0) - phi)) < 1e-11 * np.max(np.abs(phi))
    # nu^1/2 nu^1/2 = nu and nu^-1 = -L/(4 pi)
    assert np.max(np.abs(C.apply(C.apply(X, 0.5), 0.5) - phi)) < 1e-11 * np.max(np.abs(phi))
    assert np.max(np.abs(C.apply(X, -1.0) - X @ A.T / (4 * math.pi))) < 1e-9 * np.max(np.abs(X @ A.T))


# ------------------------------------------------------------------ COCG
def test_cocg_matches_dense_solve(small):
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    H = brute.dense_h(small)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((3, g.n_d)) + 1j * rng.standard_normal((3, g.n_d))
    sig = np.array([-small.eps[0] + 0.05j, -small.eps[1] + 1.0j, 0.4 - 2.0j])
    x, it, st = oracle.cocg(g, small.vloc, sig, b, tol=1e-12, maxit=5000)
    assert np.all(st == oracle.OK)
    for s in range(3):
        A = H + sig[s] * np.eye(g.n_d)
        ref = np.linalg.solve(A, b[s])
        cond = np.linalg.cond(A)
        assert np.linalg.norm(x[s] - ref) <= 1e-12 * cond * np.linalg.norm(ref)
        assert np.linalg.norm(b[s] - A @ x[s]) <= 1e-12 * np.linalg.norm(b[s]) * 1.01


def test_cocg_status_codes(small):
    g = oracle.Grid(small.nx, small.ny, small.nz, small.h)
    rng = np.random.default_rng(3)
    b = np.vstack([rng.standard_normal(g.n_d) + 0j, np.zeros(g.n_d, dtype=complex)])
    x, it, st = oracle.cocg(g, small.vloc, np.array([0.2j, 0.2j]), b, tol=1e-12, maxit=1)
    assert st[0] == oracle.NOT_CONVERGED and it[0] == 1
    assert st[1] == oracle.OK and it[1] == 0 and not np.any(x[1])


# ------------------------------------------------------------------ chi0 (Eqs. 2, 7-9)
@pytest.mark.parametrize("omega", [0.07, 0.8, 6.0])
def test_chi0_matches_sum_over_states(cube, omega):
    o = oracle.Oracle.from_system(cube)
    dv = synth.random_block(4, 3, cube.n_d)
    got = o.chi0(dv, omega, tol=1e-13, maxit=20000)
    ref = dv @ brute.chi0_sum_over_states(cube, omega).T
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_chi0_invariants(cube):
    o = oracle.Oracle.from_system(cube)
    a, b = synth.random_block(5, 2, cube.n_d)
    omega = 0.3
    ca, cb = o.chi0(np.vstack([a, b]), omega, tol=1e-13, maxit=20000)
    one = o.chi0(np.ones(cube.n_d), omega, tol=1e-13, maxit=20000)[0]
    scale = np.max(np.abs(ca))
    assert np.max(np.abs(one)) < 1e-10 * scale             # chi0 1 = 0 (charge conservation)
    assert abs(a @ cb - b @ ca) < 1e-10 * abs(a @ ca)      # symmetric
    assert a @ ca < 0 and b @ cb < 0                        # negative definite (Formulation)


def test_galerkin_initial_guess_equals_projection(cube):
    o = oracle.Oracle.from_system(cube)
    dv = synth.random_block(6, 2, cube.n_d)
    proj, xs = o.chi0(dv, 0.2, tol=1e-13, maxit=20000, return_x=True)
    gal = o.chi0(dv, 0.2, tol=1e-13, maxit=20000, galerkin=True)
    assert np.max(np.abs(proj - gal)) < 1e-9 * np.max(np.abs(proj))
    for n, _, x in xs:   # projected solves carry no occupied component
        assert np.max(np.abs(x @ cube.psi.T)) < 1e-9 * np.max(np.abs(x))


def test_sign_of_omega_gives_conjugate_solution(cube):
    o = oracle.Oracle.from_system(cube)
    dv = synth.random_block(7, 1, cube.n_d)
    rp, xp = o.chi0(dv, 0.5, tol=1e-13, maxit=20000, return_x=True, sign=+1)
    rm, xm = o.chi0(dv, 0.5, tol=1e-13, maxit=20000, return_x=True, sign=-1)
    assert np.max(np.abs(rp - rm)) < 1e-10 * np.max(np.abs(rp))
    for (_, _, a), (_, _, b) in zip(xp, xm):
        assert np.max(np.abs(a - np.conj(b))) < 1e-9 * np.max(np.abs(a))


def test_chi_tilde_and_nu_chi0_share_eigenvalues(cube):
    o = oracle.Oracle.from_system(cube)
    n = cube.n_d
    I = np.eye(n)
    A = o.chi_tilde(I, 0.4, tol=1e-13)        # rows: chi~0 e_k = column k (symmetric)
    B = o.nu_chi0(I, 0.4, tol=1e-13)          # rows: nu chi0 e_k
    la = np.sort(np.linalg.eigvalsh(0.5 * (A + A.T)))
    lb = np.sort(np.linalg.eigvals(B.T).real)
    ref = np.sort(np.linalg.eigvalsh(brute.chi_tilde_dense(cube, 0.4)))
    assert np.max(np.abs(la - ref)) < 1e-9
    assert np.max(np.abs(lb - ref)) < 1e-8
    assert ref.max() < 1e-10                     # all eigenvalues <= 0


# ------------------------------------------------------------------ frequency quadrature
@pytest.mark.parametrize("n_omega", [1, 4, 8, 12])
def test_frequency_quadrature_closed_forms(n_omega):
    w_nodes, w = oracle.frequency_quadrature(n_omega)
    # int_0^inf (1+w)^-2 = 1 and int_0^inf (1+w)^-3 = 1/2 are integrated exactly by the map
    assert abs(np.sum(w / (1 + w_nodes) ** 2) - 1.0) < 1e-13
    assert abs(np.sum(w / (1 + w_nodes) ** 3) - 0.5) < 1e-13
    assert np.all(np.diff(w_nodes) > 0) and np.all(w > 0)


def test_frequency_quadrature_converges_on_lorentzian():
    errs = []
    for n in (8, 16, 32):
        x, w = oracle.frequency_quadrature(n)
        errs.append(abs(np.sum(w / (1 + x * x)) - math.pi / 2))
    assert errs[2] < 1e-12 and errs[1] < errs[0]


# ------------------------------------------------------------------ subspace iteration, E_c
def test_rayleigh_ritz_full_rank_gives_dense_eigenvalues(cube):
    """With V = I (N_r = N_d) the projected matrix C = V^T chi~0 V is chi~0 itself."""
    o = oracle.Oracle.from_system(cube)
    R = o.chi_tilde(np.eye(cube.n_d), 1.3, tol=1e-13)
    lam = np.linalg.eigvalsh(0.5 * (R + R.T))
    ref = np.linalg.eigvalsh(brute.chi_tilde_dense(cube, 1.3))
    assert np.max(np.abs(lam - ref)) < 1e-10


def test_subspace_iteration_converges_to_lowest_eigenvalues():
    s = synth.small_system((6, 6, 6), h=0.6, n_s=2, n_wells=2, seed=9)
    o = oracle.Oracle.from_system(s)
    n_r = 5
    V0 = synth.trial_vectors(9, n_r, s.n_d)
    res = oracle.rpa_ec(o, V0, n_omega=2, tol=1e-12, eps_c=1e-14, max_subspace_iters=400)
    for m, om in enumerate(res.omegas):
        ref = np.linalg.eigvalsh(brute.chi_tilde_dense(s, om))[:n_r]
        assert np.max(np.abs(res.lambdas[m] - ref)) < 1e-7, (om, res.lambdas[m], ref)
        ref_e = res.weights[m] / (2 * math.pi) * np.sum(np.log1p(-ref) + ref)
        assert abs(res.e_c_per_omega[m] - ref_e) < 1e-9
    assert res.e_c < 0


def test_ec_quadrature_against_adaptive_integral():
    """E_c of the dense full-spectrum integrand (Eq. 6) by the oracle's frequency rule against
    adaptive quadrature on [0, inf)."""
    s = synth.small_system((5, 5, 5), h=0.6, n_s=2, n_wells=2, seed=4)

    def F(om):
        lam = np.linalg.eigvalsh(brute.chi_tilde_dense(s, om))
        return float(np.sum(oracle.g_rpa(lam)))

    ref = si.quad(F, 0, np.inf, epsabs=1e-11, epsrel=1e-10, limit=200)[0] / (2 * math.pi)
    x, w = oracle.frequency_quadrature(24)
    val = sum(wi * F(xi) for xi, wi in zip(x, w)) / (2 * math.pi)
    assert abs(val - ref) < 1e-7 * abs(ref)
    x8, w8 = oracle.frequency_quadrature(8)
    val8 = sum(wi * F(xi) for xi, wi in zip(x8, w8)) / (2 * math.pi)
    assert abs(val8 - ref) < 1e-2 * abs(ref)


# ------------------------------------------------------------------ adjoint dE_c/dV_loc
def test_projected_sos_reduces_to_sum_over_states(cube):
    """At the potential the orbitals belong to, the fixed-orbital response equals Eq. 2."""
    a = brute.chi0_projected_sos(cube, cube.vloc, 0.6)
    b = brute.chi0_sum_over_states(cube, 0.6)
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(b))


def test_ec_gradient_matches_finite_differences_of_dense_sos():
    s = synth.small_system((6, 5, 5), h=0.6, n_s=2, n_wells=2, seed=23)
    o = oracle.Oracle.from_system(s)
    n_r, n_omega = 3, 2
    V0 = synth.trial_vectors(23, n_r, s.n_d)
    res, grad = oracle.rpa_ec_gradient(o, V0, n_omega, tol=1e-13, eps_c=1e-15, max_subspace_iters=600)
    # the oracle's E_c is the dense projected-SOS E_c of the same n_r eigenvalues
    ref = brute.ec_projected_dense(s, s.vloc, n_r, res.omegas, res.weights)
    assert abs(res.e_c - ref) < 1e-10 * abs(ref)
    rng = np.random.default_rng(0)
    pts = rng.choice(s.n_d, 6, replace=False)
    d = 1e-4
    for r in pts:
        vp, vm = s.vloc.copy(), s.vloc.copy()
        vp[r] += d
        vm[r] -= d
        fd = (brute.ec_projected_dense(s, vp, n_r, res.omegas, res.weights)
              - brute.ec_projected_dense(s, vm, n_r, res.omegas, res.weights)) / (2 * d)
        assert abs(grad[r] - fd) < 1e-6 * np.max(np.abs(grad)), (r, grad[r], fd)


def test_frozen_subspace_gradient_is_exact_derivative():
    """With every frequency starting from the same fixed subspace and one Rayleigh-Ritz step
    (independent_frequencies), E_c is a smooth function of V_loc whose derivative is exactly the
    Hellmann-Feynman gradient; finite differences of the oracle's own E_c must agree."""
    s = synth.small_system((7, 6, 6), h=0.55, n_s=2, n_wells=2, seed=29)
    o = oracle.Oracle.from_system(s)
    V0 = synth.trial_vectors(29, 4, s.n_d)
    kw = dict(n_omega=2, tol=1e-13, eps_c=0.0, fixed_iters=1, independent_frequencies=True)
    res, grad = oracle.rpa_ec_gradient(o, V0, **kw)
    d = 1e-4
    for r in np.random.default_rng(1).choice(s.n_d, 4, replace=False):
        e = []
        for sgn in (1, -1):
            v = s.vloc.copy()
            v[r] += sgn * d
            o2 = oracle.Oracle(s.nx, s.ny, s.nz, s.h, v, s.psi, s.eps, s.n_atoms)
            e.append(oracle.rpa_ec(o2, V0, 2, 1e-13, 0.0, fixed_iters=1, project_solution=True,
                                   independent_frequencies=True).e_c)
        fd = (e[0] - e[1]) / (2 * d)
        assert abs(grad[r] - fd) < 1e-6 * np.max(np.abs(grad)), (r, grad[r], fd)


# ------------------------------------------------------------------ Gauss spectral quadrature
def _random_symmetric(n, seed, shift=0.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return 0.5 * (A + A.T) / math.sqrt(n) + shift * np.eye(n)


@pytest.mark.parametrize("n_o", [1, 2, 3, 4])
def test_gauss_sq_is_exact_for_polynomials_up_to_degree_2n_minus_1(n_o):
    """An N_o-node Gauss rule integrates polynomials of degree <= 2 N_o - 1 exactly, so the SQ
    trace of C^k equals Tr C^k (computed by matrix powers) for k <= 2 N_o - 1, and not beyond."""
    C = _random_symmetric(12, 5)
    for k in range(0, 2 * n_o):
        exact = float(np.trace(np.linalg.matrix_power(C, k)))
        sq = oracle.gauss_sq_trace(C, n_o, lambda x, k=k: x ** k)
        assert abs(sq - exact) <= 1e-11 * max(1.0, abs(exact)), (n_o, k)
    k = 2 * n_o
    exact = float(np.trace(np.linalg.matrix_power(C, k)))
    assert abs(oracle.gauss_sq_trace(C, n_o, lambda x: x ** k) - exact) > 1e-8 * abs(exact)


def test_gauss_sq_order_one_is_the_diagonal():
    C = _random_symmetric(9, 6, shift=-1.5)
    f = lambda x: np.log1p(-x) + x  # noqa: E731
    assert abs(oracle.gauss_sq_trace(C, 1, f) - float(np.sum(f(np.diag(C))))) < 1e-13


def test_gauss_sq_of_full_order_is_the_trace_by_eigenvalues():
    """With N_o >= n the Lanczos runs exhaust their Krylov spaces: the rule is exact for g."""
    C = -0.4 * np.abs(_random_symmetric(10, 7)) - 0.2 * np.eye(10)
    lam = np.linalg.eigvalsh(C)
    exact = float(np.sum(np.log1p(-lam) + lam))
    assert abs(oracle.gauss_sq_trace(C, 10, oracle.g_rpa) - exact) < 1e-11 * abs(exact)
    # and a modest order is already close for the smooth g (the paper's N_o = 3..7)
    assert abs(oracle.gauss_sq_trace(C, 4, oracle.g_rpa) - exact) < 1e-3 * abs(exact)


def test_rpa_ec_with_full_order_sq_equals_rayleigh_ritz():
    s = synth.workload("tiny15").system
    o = oracle.Oracle.from_system(s)
    V0 = synth.trial_vectors(0, 8, s.n_d)
    rr = oracle.rpa_ec(o, V0, 2, tol=1e-10, eps_c=0.0, fixed_iters=1)
    sq = oracle.rpa_ec(o, V0, 2, tol=1e-10, eps_c=0.0, fixed_iters=1, sq_order=8)
    sq3 = oracle.rpa_ec(o, V0, 2, tol=1e-10, eps_c=0.0, fixed_iters=1, sq_order=3)
    assert np.allclose(sq.e_c_per_omega, rr.e_c_per_omega, rtol=1e-11, atol=0)
    assert abs(sq3.e_c - rr.e_c) < 1e-3 * abs(rr.e_c)
