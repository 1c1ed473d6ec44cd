"""Dense brute-force references used to pin the oracle (tiny grids only).

Everything here is assembled from the model problem's sparse matrices (``synth``)
and dense LAPACK routines: a route independent of the oracle's matrix-free
stencil, Kronecker Coulomb operator and COCG.
"""
import math

import numpy as np
import scipy.linalg as sla

import synth


def dense_h(system):
    return synth.hamiltonian_matrix(system).toarray()


def dense_minus_laplacian(nx, ny, nz, h, periodic=False):
    return -synth.laplacian_matrix(nx, ny, nz, h, periodic).toarray()


def full_spectrum(system):
    """All eigenpairs of the model Hamiltonian; rows of the vector array are u_k."""
    vals, vecs = np.linalg.eigh(dense_h(system))
    return vals, vecs.T.copy()


def chi0_sum_over_states(system, omega):
    """chi0(i omega) as an N_d x N_d matrix on grid values, from the sum over occupied i and
    unoccupied a (Eq. 2 with f in {0,1}, both orderings of each pair combined):
        chi0 = (4/h^3) sum_{i,a} (u_i u_a)(u_i u_a)^T (e_i - e_a) / ((e_i - e_a)^2 + omega^2)."""
    vals, U = full_spectrum(system)
    n_s = system.n_s
    occ, un = U[:n_s], U[n_s:]
    X = np.zeros((system.n_d, system.n_d))
    for i in range(n_s):
        d = vals[i] - vals[n_s:]
        f = d / (d * d + omega * omega)
        P = occ[i][None, :] * un                        # (N_un, N_d)
        X += (P.T * f) @ P
    return (4.0 / system.h ** 3) * X


def nu_power_dense(nx, ny, nz, h, power, periodic=False):
    """(4 pi)^p (-L_h)^{-p} by a dense symmetric eigendecomposition; on a periodic grid the
    pseudo-inverse power (the null space of -L_h, the constant function, maps to zero)."""
    mu, Q = np.linalg.eigh(dense_minus_laplacian(nx, ny, nz, h, periodic))
    keep = mu > 1e-9 * mu.max() if periodic else np.ones(mu.shape, bool)
    f = np.zeros_like(mu)
    f[keep] = (4.0 * math.pi) ** power * mu[keep] ** (-power)
    return (Q * f) @ Q.T


def chi_tilde_dense(system, omega):
    nh = nu_power_dense(system.nx, system.ny, system.nz, system.h, 0.5, system.periodic)
    return nh @ chi0_sum_over_states(system, omega) @ nh


def chi0_projected_sos(system, vloc, omega):
    """chi0(i omega) at fixed occupied orbitals u_i and eigenvalues eps_i for the potential vloc:
    the unoccupied states are the eigenpairs (phi_a, e_a) of the Hamiltonian H(vloc) restricted
    to the orthogonal complement of span{u_i}; then
        chi0 = (4/h^3) sum_{i,a} (u_i phi_a)(u_i phi_a)^T (eps_i - e_a) / ((eps_i - e_a)^2 + omega^2).
    At the potential the orbitals belong to, this is the sum over states of Eq. 2."""
    import scipy.linalg as sla
    s2 = synth.System(system.name, system.nx, system.ny, system.nz, system.h, np.asarray(vloc),
                      system.psi, system.eps, system.n_atoms, system.periodic)
    H = dense_h(s2)
    Q = sla.null_space(system.psi)
    e, Z = np.linalg.eigh(Q.T @ H @ Q)
    Phi = (Q @ Z).T
    X = np.zeros((system.n_d, system.n_d))
    for i in range(system.n_s):
        d = system.eps[i] - e
        f = d / (d * d + omega * omega)
        P = system.psi[i][None, :] * Phi
        X += (P.T * f) @ P
    return (4.0 / system.h ** 3) * X


def ec_projected_dense(system, vloc, n_r, omegas, weights):
    """E_c = (1/2pi) sum_m w_m sum_{i < n_r} g(lambda_i) over the n_r lowest eigenvalues of
    nu^1/2 chi0 nu^1/2, chi0 from chi0_projected_sos."""
    nh = nu_power_dense(system.nx, system.ny, system.nz, system.h, 0.5, system.periodic)
    e = 0.0
    for om, w in zip(omegas, weights):
        lam = np.linalg.eigvalsh(nh @ chi0_projected_sos(system, vloc, om) @ nh)[:n_r]
        e += w / (2.0 * math.pi) * float(np.sum(np.log1p(-lam) + lam))
    return e
