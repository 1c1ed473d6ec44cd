"""Plain FP64 CPU oracle of the real-space RPA correlation-energy method
(B. Zhang, S. Shah, J. E. Pask, E. Chow, P. Suryanarayana, arXiv 2504.01816).

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA library.  Only
the test-suite, the smoke check (``__graft_entry__.smoke``) and the timed CPU
baseline of ``bench.py`` may import it.  It shares no code with the CUDA library:
it has its own finite-difference weights, Hamiltonian, Coulomb operator, COCG
(``cocg_oracle.c``), projections, eigensolver calls and frequency quadrature.

Every function follows the paper's steps in the paper's order, in FP64, with no
blocking, fusion or reordering beyond what the definition states.  Library
routines (numpy matmul, eigh, cholesky, Gauss-Legendre nodes) serve as single
steps.

Discrete conventions (the paper says only "high-order centred finite differences"
and "trapezoidal rule", Section "Implementation"; these are the readings):

* grid functions are vectors of length N_d = nx*ny*nz, point (i,j,k) at
  i + nx*(j + ny*k); a block of K of them is an array (K, N_d);
* orbitals u_n are l2-orthonormal (u = psi h^{3/2});
* L_h is the 12th-order centred Laplacian with zero values outside the box
  (Dirichlet) or, for a periodic grid, the values of the periodic continuation
  (the bulk cells of Section "Results"); H = -1/2 L_h + diag(V_loc);
* nu = 4 pi (-L_h)^{-1} (Poisson equation, Eq. 5); nu^p is applied through the
  eigendecompositions of the three 1D second-difference matrices (Kronecker
  product formalism, Section "Implementation"); on a periodic grid -L_h is
  singular on the constant function (the G = 0 mode), which nu^p maps to zero
  (the neutralising background of a periodic cell);
* chi0 dV = drho = (4/h^3) Re sum_n u_n (.) x_n with
  (H - eps_n + i omega) x_n = -P_c(u_n (.) dV),  P_c = I - U U^T   (Eqs. 7-9);
* the correlation energy is E_c = (1/2pi) int_0^inf sum_i [log(1-lambda_i) +
  lambda_i] d omega over the lowest N_r eigenvalues of nu^1/2 chi0 nu^1/2
  (Eq. 10), by subspace iteration with Rayleigh-Ritz on the projected matrix
  (Algorithm 1 with subspace diagonalisation in place of spectral quadrature).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import scipy.linalg as sla

from . import build as _build

RADIUS = 6  # 12th-order centred differences

OK, NOT_CONVERGED, BREAKDOWN, NOT_SPD = 0, 4, 5, 6

_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        lib = ctypes.CDLL(_build.build())
        d, i = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        lib.oracle_apply_h.argtypes = [ctypes.c_int] * 4 + [d, ctypes.c_int, d, ctypes.c_double, ctypes.c_double,
                                                             d, d]
        lib.oracle_apply_h.restype = None
        lib.oracle_cocg_batch.argtypes = ([ctypes.c_int] * 4 + [d, ctypes.c_int, d, ctypes.c_int, d, d, d, d,
                                          ctypes.c_double, ctypes.c_int, i, i])
        lib.oracle_cocg_batch.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib_handle = lib
    return _lib_handle


def num_threads() -> int:
    return _lib().oracle_num_threads()


def set_threads(n: int) -> None:
    _lib().oracle_set_threads(int(n))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ------------------------------------------------------------------------------------
# Finite differences and the Hamiltonian (Section "Implementation", Eq. 4 local part)
# ------------------------------------------------------------------------------------
def fd_weights(radius: int = RADIUS) -> np.ndarray:
    """Centred second-derivative weights of order 2*radius on a unit grid.

    f'' ~ w0 f(0) + sum_k wk (f(k) + f(-k)),
    wk = 2 (-1)^(k+1) (p!)^2 / (k^2 (p-k)! (p+k)!),  w0 = -2 sum_k 1/k^2.
    """
    p = radius
    w = np.zeros(p + 1)
    for k in range(1, p + 1):
        w[k] = 2.0 * (-1) ** (k + 1) * math.factorial(p) ** 2 / (
            k * k * math.factorial(p - k) * math.factorial(p + k))
    w[0] = -2.0 * sum(1.0 / (k * k) for k in range(1, p + 1))
    return w


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    h: float
    periodic: bool = False      # periodic continuation instead of zero values outside the box

    @property
    def n_d(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def apply_h(grid: Grid, vloc: np.ndarray, vec: np.ndarray, sigma: complex = 0.0) -> np.ndarray:
    """(H + sigma) vec for one complex grid function (matrix-free)."""
    w = fd_weights() / grid.h ** 2
    v = np.ascontiguousarray(vec, dtype=np.complex128)
    out = np.empty_like(v)
    _lib().oracle_apply_h(grid.nx, grid.ny, grid.nz, RADIUS, _dp(w), int(grid.periodic),
                          _dp(np.ascontiguousarray(vloc)),
                          float(np.real(sigma)), float(np.imag(sigma)),
                          _dp(v.view(np.float64)), _dp(out.view(np.float64)))
    return out


def cocg(grid: Grid, vloc: np.ndarray, sigma: np.ndarray, b: np.ndarray, tol: float, maxit: int):
    """Solve (H + sigma_s) x_s = b_s for every row s of b by COCG (Section
    "Implementation"; complex-symmetric Sternheimer operator of Eq. 9).

    Returns (x, iterations, status); status 0 converged, 4 not converged, 5 breakdown.
    """
    b = np.ascontiguousarray(b, dtype=np.complex128)
    nsys = b.shape[0]
    sigma = np.asarray(sigma, dtype=np.complex128).reshape(nsys)
    x = np.zeros_like(b)
    it = np.zeros(nsys, dtype=np.int32)
    st = np.zeros(nsys, dtype=np.int32)
    w = fd_weights() / grid.h ** 2
    sre = np.ascontiguousarray(sigma.real)
    sim = np.ascontiguousarray(sigma.imag)
    _lib().oracle_cocg_batch(grid.nx, grid.ny, grid.nz, RADIUS, _dp(w), int(grid.periodic),
                             _dp(np.ascontiguousarray(vloc)), nsys,
                             _dp(sre), _dp(sim), _dp(b.view(np.float64)), _dp(x.view(np.float64)),
                             float(tol), int(maxit), _ip(it), _ip(st))
    return x, it, st


# ------------------------------------------------------------------------------------
# Coulomb operator by the Kronecker-product formalism (Section "Implementation")
# ------------------------------------------------------------------------------------
# (The preconditioned COCG, which uses the same eigendecomposition of -L_h, follows the Coulomb
# operator below.)
def second_difference_1d(n: int, h: float, periodic: bool = False) -> np.ndarray:
    """Dense 1D second-derivative matrix: zero boundary values (Toeplitz), or the periodic
    continuation (circulant: every tap i +- k taken modulo n, so taps that wrap onto the same
    point add up)."""
    w = fd_weights()
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] += w[0] / h ** 2
        for k in range(1, RADIUS + 1):
            for j in (i - k, i + k):
                if periodic:
                    D[i, j % n] += w[k] / h ** 2
                elif 0 <= j < n:
                    D[i, j] += w[k] / h ** 2
    return D


class Coulomb:
    """nu^p = (4 pi)^p (-L_h)^(-p) through -L_h = (Q_z x Q_y x Q_x) diag(mu_x+mu_y+mu_z) (...)^T,
    with K_a = -D_a = Q_a diag(mu_a) Q_a^T the 1D eigendecompositions.  On a periodic grid the
    one zero eigenvalue of -L_h (all three 1D constant modes) gets the factor 0."""

    def __init__(self, grid: Grid):
        self.grid = grid
        self.mu, self.Q = [], []
        for n in (grid.nx, grid.ny, grid.nz):
            mu, Q = np.linalg.eigh(-second_difference_1d(n, grid.h, grid.periodic))
            self.mu.append(mu)
            self.Q.append(Q)
        mx, my, mz = self.mu
        self.lam = mz[:, None, None] + my[None, :, None] + mx[None, None, :]
        # the G = 0 mode: eigh returns the constant modes' zero eigenvalues to rounding
        self.zero = self.lam <= 1e-9 * self.lam.max() if grid.periodic else np.zeros(self.lam.shape, bool)

    def apply(self, X: np.ndarray, power: float) -> np.ndarray:
        """nu^power applied to every row of X (K, N_d)."""
        g = self.grid
        Qx, Qy, Qz = self.Q
        Y = np.asarray(X, dtype=np.float64).reshape(-1, g.nz, g.ny, g.nx)
        # to the eigenbasis: multiply by Q_a^T along each axis
        Y = np.einsum("ia,kzyi->kzya", Qx, Y)
        Y = np.einsum("ja,kzjx->kzax", Qy, Y)
        Y = np.einsum("la,klyx->kayx", Qz, Y)
        lam = np.where(self.zero, 1.0, self.lam)
        Y = Y * np.where(self.zero, 0.0, (4.0 * math.pi) ** power * lam ** (-power))[None]
        # back: multiply by Q_a along each axis
        Y = np.einsum("ia,kzya->kzyi", Qx, Y)
        Y = np.einsum("ja,kzax->kzjx", Qy, Y)
        Y = np.einsum("la,kayx->klyx", Qz, Y)
        return Y.reshape(np.shape(X))


# ------------------------------------------------------------------------------------
# Laplacian-preconditioned COCG (Section "Implementation": Laplacian-based preconditioning
# through the Kronecker product formalism)
# ------------------------------------------------------------------------------------
def laplacian_preconditioner(coulomb: "Coulomb", shift: complex):
    """M = (-1/2 L_h + shift)^(-1) applied to rows of a complex block, through the Kronecker
    eigendecomposition -L_h = (Q_z x Q_y x Q_x) diag(lam) (...)^T: the Sternheimer operator
    H - eps_n + i omega with V_loc replaced by a constant (the paper names the preconditioner and
    the formalism, not the shift; reading: shift = mean(V_loc) - eps_n + i omega)."""
    g = coulomb.grid
    Qx, Qy, Qz = coulomb.Q
    d = 1.0 / (0.5 * coulomb.lam + shift)

    def apply(R):
        Y = np.asarray(R, dtype=np.complex128).reshape(-1, g.nz, g.ny, g.nx)
        Y = np.einsum("ia,kzyi->kzya", Qx, Y)
        Y = np.einsum("ja,kzjx->kzax", Qy, Y)
        Y = np.einsum("la,klyx->kayx", Qz, Y)
        Y = Y * d[None]
        Y = np.einsum("ia,kzya->kzyi", Qx, Y)
        Y = np.einsum("ja,kzax->kzjx", Qy, Y)
        Y = np.einsum("la,kayx->klyx", Qz, Y)
        return Y.reshape(np.shape(R))
    return apply


def pcocg(grid: Grid, vloc: np.ndarray, sigma: complex, b: np.ndarray, tol: float, maxit: int, apply_m):
    """Preconditioned COCG for (H + sigma) x = b, every row of b, with the complex-symmetric
    preconditioner apply_m (van der Vorst & Melissen's COCG with M; unconjugated r^T z):
        r = b, z = M r, p = z, rho = r^T z;  repeat: q = A p, alpha = rho / p^T q, x += alpha p,
        r -= alpha q, z = M r, rho' = r^T z, p = z + (rho'/rho) p;
    stop when ||r||_2 <= tol ||b||_2 (checked before each iteration).  Returns (x, iterations,
    status) like cocg; status 5 where p^T q or r^T z vanishes."""
    b = np.atleast_2d(np.asarray(b, dtype=np.complex128))
    ns = b.shape[0]
    x = np.zeros_like(b)
    its = np.zeros(ns, dtype=np.int32)
    st = np.zeros(ns, dtype=np.int32)
    for s in range(ns):
        r = b[s].copy()
        bn = np.linalg.norm(b[s])
        z = apply_m(r[None])[0]
        p = z.copy()
        rho = r @ z
        k = 0
        while True:
            if np.linalg.norm(r) <= tol * bn:
                break
            if k >= maxit:
                st[s] = NOT_CONVERGED
                break
            q = apply_h(grid, vloc, p, sigma)
            pq = p @ q
            if pq == 0 or rho == 0:
                st[s] = BREAKDOWN
                break
            alpha = rho / pq
            x[s] += alpha * p
            r -= alpha * q
            z = apply_m(r[None])[0]
            rho_new = r @ z
            p = z + (rho_new / rho) * p
            rho = rho_new
            k += 1
        its[s] = k
    return x, its, st


def block_cocg_generic(apply_a, B: np.ndarray, tol: float, maxit: int, history: Optional[list] = None):
    """Block COCG for A X = B, every row of B a right-hand side of the same complex-symmetric A
    (the block variant of COCG named in Section "Implementation" as the paper's preliminary
    alternative).  Block conjugate gradients (O'Leary's block CG) with the unconjugated form
    x^T y in place of the inner product, as COCG is to CG; with the s right-hand sides as the
    columns of B:
        X = 0, R = B, P = R, rho = R^T R                           (s x s)
        repeat:  Q = A P, alpha = (P^T Q)^-1 rho, X += P alpha, R -= Q alpha,
                 rho' = R^T R, beta = rho^-1 rho', P = R + P beta, rho = rho'
    stopping when every column has ||r_j||_2 <= tol ||b_j||_2 (checked before each iteration).
    apply_a maps an (s, N) block of rows to A applied to each row.  Returns (X as rows,
    iterations, status): status 5 where P^T Q or rho is singular to working precision.
    history, if a list, receives (R, P, Q) of every iteration as columns (the pins check the
    block orthogonality of the residuals and the block A-conjugacy of the directions)."""
    Bc = np.asarray(B, dtype=np.complex128).T.copy()        # (N, s)
    X = np.zeros_like(Bc)
    R = Bc.copy()
    P = R.copy()
    rho = R.T @ R
    bn = np.linalg.norm(Bc, axis=0)
    k, status = 0, OK
    while True:
        if np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            break
        if k >= maxit:
            status = NOT_CONVERGED
            break
        Q = apply_a(P.T).T
        if history is not None:
            history.append((R.copy(), P.copy(), Q.copy()))
        G = P.T @ Q
        if not np.all(np.isfinite(G)) or np.linalg.cond(G) > 1e14 or np.linalg.cond(rho) > 1e14:
            status = BREAKDOWN
            break
        alpha = np.linalg.solve(G, rho)
        X += P @ alpha
        R -= Q @ alpha
        rho_new = R.T @ R
        beta = np.linalg.solve(rho, rho_new)
        P = R + P @ beta
        rho = rho_new
        k += 1
    return X.T.copy(), k, status


def block_cocg(grid: Grid, vloc: np.ndarray, sigma: complex, B: np.ndarray, tol: float, maxit: int):
    """Block COCG (block_cocg_generic) for (H + sigma) X = B, the rows of B sharing one shift."""
    def apply_a(P):
        return np.array([apply_h(grid, vloc, p, sigma) for p in P])
    return block_cocg_generic(apply_a, np.atleast_2d(B), tol, maxit)


# ------------------------------------------------------------------------------------
# chi0 by density functional perturbation theory (Eqs. 7-9, Algorithm 1 inner loop)
# ------------------------------------------------------------------------------------
@dataclass
class SolveStats:
    iterations: List[np.ndarray] = field(default_factory=list)
    status: List[np.ndarray] = field(default_factory=list)

    def total_iterations(self) -> int:
        return int(sum(int(a.sum()) for a in self.iterations))

    def n_solves(self) -> int:
        return int(sum(a.size for a in self.iterations))

    def worst_status(self) -> int:
        return int(max((int(a.max()) for a in self.status if a.size), default=0))


class Oracle:
    """One model system (grid, V_loc, occupied u_n and eps_n) and the method on it."""

    def __init__(self, nx, ny, nz, h, vloc, psi, eps, n_atoms=1, periodic=False):
        self.grid = Grid(int(nx), int(ny), int(nz), float(h), bool(periodic))
        self.vloc = np.ascontiguousarray(vloc, dtype=np.float64)
        self.psi = np.ascontiguousarray(psi, dtype=np.float64)   # (N_s, N_d)
        self.eps = np.asarray(eps, dtype=np.float64)
        self.n_atoms = int(n_atoms)
        self.coulomb = Coulomb(self.grid)

    @classmethod
    def from_system(cls, s):
        return cls(s.nx, s.ny, s.nz, s.h, s.vloc, s.psi, s.eps, s.n_atoms, getattr(s, "periodic", False))

    @property
    def n_s(self):
        return self.psi.shape[0]

    def sternheimer_rhs(self, n: int, dv: np.ndarray) -> np.ndarray:
        """b = -P_c(u_n (.) dV) for every row of dv: the Sternheimer right-hand side (Eq. 9)
        with the occupied components removed (P_c = I - U U^T)."""
        u = self.psi
        pair = u[n][None, :] * dv
        return -(pair - (pair @ u.T) @ u)

    def chi0(self, dv: np.ndarray, omega: float, tol: float, maxit: int = 100000, sign: int = +1,
             stats: Optional[SolveStats] = None, max_chunk_bytes: float = 2.5e8,
             galerkin: bool = False, return_x: bool = False, project_solution: bool = False,
             precondition: bool = False, block: int = 0):
        """drho = chi0(i omega) dV for every row of dv (Eqs. 7-9).

        For each occupied n and each dV: solve (H - eps_n + sign*i*omega) x = b by COCG, then
        drho = (4/h^3) Re sum_n u_n (.) x_n.  galerkin=True takes the paper's Galerkin
        initial guess instead of projecting the right-hand side (Section "Implementation").
        project_solution=True also removes the occupied components of x (x <- P_c x): the same
        operator when the orbitals are exact eigenvectors of H, and the first-order-consistent
        response of the fixed occupied space when V_loc moves away from them.  precondition=True
        solves by the Laplacian-preconditioned COCG (pcocg) instead.  block=s > 0 solves the
        right-hand sides of each orbital s at a time by block COCG (block_cocg; every column of a
        block reports the block's iteration count).
        """
        g = self.grid
        dv = np.atleast_2d(np.asarray(dv, dtype=np.float64))
        k = dv.shape[0]
        drho = np.zeros((k, g.n_d))
        xs = [] if return_x else None
        per_row = 16.0 * 2 * g.n_d
        chunk = max(1, int(max_chunk_bytes // per_row))
        if block > 0:
            chunk = block
        for n in range(self.n_s):
            sigma = -self.eps[n] + sign * 1j * omega
            for j0 in range(0, k, chunk):
                blk = dv[j0:j0 + chunk]
                if galerkin:
                    x = self._galerkin_solve(n, blk, sigma, tol, maxit, stats)
                else:
                    b = self.sternheimer_rhs(n, blk).astype(np.complex128)
                    if block > 0:
                        x, it1, st1 = block_cocg(g, self.vloc, sigma, b, tol, maxit)
                        it = np.full(len(blk), it1, dtype=np.int32)
                        st = np.full(len(blk), st1, dtype=np.int32)
                    elif precondition:
                        m = laplacian_preconditioner(self.coulomb, float(np.mean(self.vloc)) + sigma)
                        x, it, st = pcocg(g, self.vloc, sigma, b, tol, maxit, m)
                    else:
                        x, it, st = cocg(g, self.vloc, np.full(len(blk), sigma), b, tol, maxit)
                    if stats is not None:
                        stats.iterations.append(it)
                        stats.status.append(st)
                if project_solution:
                    x = x - (x @ self.psi.T) @ self.psi
                drho[j0:j0 + chunk] += (4.0 / g.h ** 3) * np.real(self.psi[n][None, :] * x)
                if return_x:
                    xs.append((n, j0, x))
        return (drho, xs) if return_x else drho

    def _galerkin_solve(self, n, blk, sigma, tol, maxit, stats):
        """Unprojected b = -u_n (.) dV; initial guess x0 = U y with (U^T A U) y = U^T b, which
        removes the occupied components from the initial residual; COCG then solves for the
        correction."""
        g = self.grid
        u = self.psi
        b = -(u[n][None, :] * blk).astype(np.complex128)
        UtAU = np.empty((self.n_s, self.n_s), dtype=np.complex128)
        AU = np.array([apply_h(g, self.vloc, u[m].astype(np.complex128), sigma) for m in range(self.n_s)])
        UtAU[:, :] = u @ AU.T
        y = np.linalg.solve(UtAU, (b @ u.T).T).T          # (len(blk), N_s)
        x0 = y @ u
        r0 = b - np.array([apply_h(g, self.vloc, xi, sigma) for xi in x0])
        d, it, st = cocg(g, self.vloc, np.full(len(blk), sigma), r0, tol, maxit)
        if stats is not None:
            stats.iterations.append(it)
            stats.status.append(st)
        return x0 + d

    def chi_tilde(self, V: np.ndarray, omega: float, tol: float, maxit: int = 100000,
                  stats: Optional[SolveStats] = None, project_solution: bool = False) -> np.ndarray:
        """R = nu^1/2 chi0(i omega) nu^1/2 V for every row of V (Algorithm 1: V_j = N V_j,
        Sternheimer loop over n, R_j = N R_j)."""
        vt = self.coulomb.apply(V, 0.5)
        drho = self.chi0(vt, omega, tol, maxit, stats=stats, project_solution=project_solution)
        return self.coulomb.apply(drho, 0.5)

    def response_square(self, Y: np.ndarray, omega: float, coef: np.ndarray, tol: float,
                        maxit: int = 100000) -> np.ndarray:
        """sum_i coef_i (4/h^3) Re sum_n x_{n,i}(r)^2 with x_{n,i} the projected Sternheimer
        solutions for dV = nu^1/2 y_i (rows of Y): the derivative of y_i^T chi~0 y_i with respect to
        V_loc(r) at fixed orbitals (the adjoint solve is the forward solve, A being complex
        symmetric)."""
        g = self.grid
        vt = self.coulomb.apply(Y, 0.5)
        out = np.zeros(g.n_d)
        for n in range(self.n_s):
            sigma = -self.eps[n] + 1j * omega
            b = self.sternheimer_rhs(n, vt).astype(np.complex128)
            x, it, st = cocg(g, self.vloc, np.full(len(vt), sigma), b, tol, maxit)
            x = x - (x @ self.psi.T) @ self.psi
            out += (4.0 / g.h ** 3) * (coef[:, None] * np.real(x * x)).sum(axis=0)
        return out

    def nu_chi0(self, V: np.ndarray, omega: float, tol: float, maxit: int = 100000,
                stats: Optional[SolveStats] = None) -> np.ndarray:
        """nu chi0(i omega) V (same eigenvalues as nu^1/2 chi0 nu^1/2, Formulation)."""
        return self.coulomb.apply(self.chi0(V, omega, tol, maxit, stats=stats), 1.0)


# ------------------------------------------------------------------------------------
# Subspace iteration, Rayleigh-Ritz and the frequency integral (Algorithm 1, Eq. 10)
# ------------------------------------------------------------------------------------
def frequency_quadrature(n_omega: int, omega0: float = 1.0):
    """Gauss-Legendre nodes x_k, weights w_k on (-1,1) mapped to [0, inf):
    omega = omega0 (1+x)/(1-x), weight = 2 omega0 w / (1-x)^2.  Ascending omega."""
    x, w = np.polynomial.legendre.leggauss(n_omega)
    return omega0 * (1.0 + x) / (1.0 - x), 2.0 * omega0 * w / (1.0 - x) ** 2


def g_rpa(lam: np.ndarray) -> np.ndarray:
    """g(x) = log(1 - x) + x."""
    lam = np.asarray(lam, dtype=np.float64)
    return np.log1p(-lam) + lam


class NotSPD(RuntimeError):
    pass


def orthonormalize_cholesky(R: np.ndarray) -> np.ndarray:
    """V = R L^{-T} with L L^T = R^T R (rows of R are the vectors): Algorithm 1 overlap,
    Cholesky and orthonormalisation."""
    M = R @ R.T
    try:
        L = np.linalg.cholesky(M)
    except np.linalg.LinAlgError as e:
        raise NotSPD(str(e))
    return sla.solve_triangular(L, R, lower=True)


@dataclass
class EcResult:
    e_c: float                        # Hartree
    e_c_per_atom: float
    e_c_per_omega: np.ndarray         # weighted contribution (w_m / 2 pi) sum_i g(lambda_i), ascending omega
    lambdas: np.ndarray               # (N_omega, N_r) Ritz values of the last iteration, ascending omega
    omegas: np.ndarray
    weights: np.ndarray
    subspace_iterations: np.ndarray   # per frequency
    sternheimer_solves: int = 0
    cocg_iterations: int = 0
    V_final: Optional[np.ndarray] = None
    ritz_vectors: Optional[List[np.ndarray]] = None   # per frequency (ascending omega), rows y_i


def gauss_sq_trace(C: np.ndarray, n_o: int, f) -> float:
    """Tr f(C) of a symmetric matrix by Gauss spectral quadrature (Section "Implementation",
    Algorithm 1): for each standard basis vector e_r, n_o steps of the Lanczos iteration with C
    started from e_r give a tridiagonal matrix J (diagonal alpha, off-diagonal beta); the
    eigenvalues of J are the quadrature nodes and the squares of the first components of its
    eigenvectors the weights, e_r^T f(C) e_r ~ sum_j Q_1j^2 f(theta_j).  A Lanczos run that
    exhausts its Krylov space (beta = 0) stops early; its rule is then exact."""
    n = C.shape[0]
    scale = max(float(np.max(np.abs(C))), 1e-300)
    total = 0.0
    for r in range(n):
        q_prev = np.zeros(n)
        q = np.zeros(n)
        q[r] = 1.0
        alpha, beta = [], []
        b = 0.0
        for k in range(n_o):
            w = C @ q - b * q_prev
            a = float(q @ w)
            w = w - a * q
            alpha.append(a)
            if k == n_o - 1:
                break
            b = float(np.linalg.norm(w))
            if b <= 1e-13 * scale:
                break
            beta.append(b)
            q_prev, q = q, w / b
        J = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        theta, Q = np.linalg.eigh(J)
        total += float(np.sum(Q[0, :] ** 2 * f(theta)))
    return total


def rpa_ec(o: Oracle, V0: np.ndarray, n_omega: int, tol: float, eps_c: float, omega0: float = 1.0,
           max_subspace_iters: int = 100, fixed_iters: Optional[int] = None, maxit: int = 100000,
           verbose: bool = False, project_solution: bool = False, keep_ritz: bool = False,
           independent_frequencies: bool = False, sq_order: int = 0,
           omega_subset: Optional[Sequence[int]] = None) -> EcResult:
    """E_c by Algorithm 1 with Rayleigh-Ritz: frequencies from highest to lowest, the subspace
    carried over from each frequency to the next; at each frequency iterate
    R = chi~0 V, C = V^T R, lambda = eig(C), E_cm = (w_m/2pi) sum g(lambda), M = R^T R = L L^T,
    V = R L^{-T} while |E_cm - E_cm_old| > eps_c * N_atoms / N_omega (eps_c in Ha/atom), at least
    two iterations (E_cm starts at 0).  fixed_iters runs exactly that many iterations instead.
    sq_order > 0 evaluates E_cm = (w_m/2pi) Tr g(C) by Gauss spectral quadrature of that order
    (gauss_sq_trace), the paper's choice; lambda are still the Ritz values.
    omega_subset (indices into the ascending frequencies) evaluates only those frequencies and
    leaves zeros for the others; the first one evaluated starts from V0."""
    omegas, weights = frequency_quadrature(n_omega, omega0)
    V = orthonormalize_cholesky(np.asarray(V0, dtype=np.float64))
    n_r = V.shape[0]
    lambdas = np.zeros((n_omega, n_r))
    e_m = np.zeros(n_omega)
    iters = np.zeros(n_omega, dtype=np.int64)
    stats = SolveStats()
    thr = eps_c * o.n_atoms / n_omega
    ritz = [None] * n_omega
    V_start = V
    selected = set(range(n_omega)) if omega_subset is None else set(int(m) for m in omega_subset)
    for m in range(n_omega - 1, -1, -1):
        if m not in selected:
            continue
        if independent_frequencies:
            V = V_start
        ecm = 0.0
        it = 0
        while True:
            ecm_old = ecm
            R = o.chi_tilde(V, omegas[m], tol, maxit, stats=stats, project_solution=project_solution)
            C = V @ R.T
            C = 0.5 * (C + C.T)
            lam, Qc = np.linalg.eigh(C)
            if keep_ritz:
                ritz[m] = Qc.T @ V
            tr = gauss_sq_trace(C, sq_order, g_rpa) if sq_order > 0 else float(np.sum(g_rpa(lam)))
            ecm = weights[m] / (2.0 * math.pi) * tr
            V = orthonormalize_cholesky(R)
            it += 1
            if verbose:
                print(f"  omega={omegas[m]:.5f} it={it} E_cm={ecm:.12f}")
            if fixed_iters is not None:
                if it >= fixed_iters:
                    break
            elif abs(ecm - ecm_old) <= thr or it >= max_subspace_iters:
                break
        lambdas[m] = lam
        e_m[m] = ecm
        iters[m] = it
    e_c = float(np.sum(e_m))
    return EcResult(e_c, e_c / o.n_atoms, e_m, lambdas, omegas, weights, iters,
                    stats.n_solves(), stats.total_iterations(), V, ritz if keep_ritz else None)


def rpa_ec_gradient(o: Oracle, V0: np.ndarray, n_omega: int, tol: float, eps_c: float, omega0: float = 1.0,
                    max_subspace_iters: int = 100, fixed_iters: Optional[int] = None, maxit: int = 100000,
                    independent_frequencies: bool = False):
    """dE_c/dV_loc(r) at fixed occupied orbitals and eigenvalues, by Hellmann-Feynman on the Ritz
    pairs of the last subspace iteration at each frequency:
        dE_c/dV(r) = (1/2pi) sum_m w_m sum_i g'(lambda_i) d lambda_i/dV(r),  g'(x) = -x/(1-x),
        d lambda_i/dV(r) = (4/h^3) Re sum_n x_{n,i}(r)^2
    where x_{n,i} solves the projected Sternheimer system for dV = nu^1/2 y_i.  E_c is evaluated
    with the projected response (project_solution).  Returns (EcResult, gradient)."""
    res = rpa_ec(o, V0, n_omega, tol, eps_c, omega0, max_subspace_iters, fixed_iters, maxit,
                 project_solution=True, keep_ritz=True, independent_frequencies=independent_frequencies)
    grad = np.zeros(o.grid.n_d)
    for m in range(n_omega):
        lam = res.lambdas[m]
        coef = res.weights[m] / (2.0 * math.pi) * (-lam / (1.0 - lam))
        grad += o.response_square(res.ritz_vectors[m], res.omegas[m], coef, tol, maxit)
    return res, grad
