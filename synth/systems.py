"""Seeded synthetic model systems for the real-space RPA correlation-energy method.

This module is the ONE piece shared by the CUDA library's callers and the FP64
oracle: it produces *inputs* only — the grid, a Gaussian-well local potential,
the occupied ground-state orbitals and eigenvalues of that model Hamiltonian,
and random starting trial vectors.  It contains none of the RPA method's
arithmetic (no response function, no Sternheimer solver, no Coulomb operator,
no subspace iteration, no frequency quadrature).

The paper computes its ground state with a full Kohn-Sham SCF (Section
"Implementation": orbitals and eigenvalues are computed by the ground-state code,
written to files and read back).  Pseudopotentials and SCF are outside the hot
path, so the ground state here is the exact lowest eigenpairs of a model
Hamiltonian  H = -1/2 L_h + diag(V_loc)  with Dirichlet (zero) boundary values, or
periodic ones for a bulk cell, and a 12th-order central finite-difference Laplacian L_h.  The finite-difference
weights are generated here by Fornberg's recursion (B. Fornberg, Math. Comp. 51
(1988) 699), which is a different derivation from the closed form the oracle and
the library use; a test checks that the orbitals produced here are eigenvectors
of the oracle's Hamiltonian.

Layouts: a grid function is a float64 vector of length N_d = nx*ny*nz with
point (i, j, k) at index i + nx*(j + ny*k) (x fastest).  A block of K grid
functions is a C-contiguous array of shape (K, N_d): row c is column c of the
N_d x K column-major matrix the C interface takes.
"""
from __future__ import annotations

import dataclasses
import hashlib
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np
import scipy.sparse as sp

__all__ = [
    "System", "Workload", "fornberg_second_derivative", "make_system", "workload",
    "trial_vectors", "WORKLOADS", "hamiltonian_matrix", "laplacian_matrix", "small_system", "random_block",
]


# --------------------------------------------------------------------------------------
# Finite-difference weights (Fornberg's recursion; independent of the closed form)
# --------------------------------------------------------------------------------------
def fornberg_second_derivative(radius: int) -> np.ndarray:
    """Weights w[0..radius] of the centred second-derivative stencil on a unit grid.

    f''(0) ~ w[0] f(0) + sum_k w[k] (f(k) + f(-k)).  Computed with Fornberg's
    generic recursion over the node list 0, 1, -1, 2, -2, ... and then read back
    by node position.
    """
    nodes = [0.0]
    for k in range(1, radius + 1):
        nodes += [float(k), float(-k)]
    m_max = 2
    n = len(nodes)
    delta = np.zeros((m_max + 1, n, n))
    delta[0, 0, 0] = 1.0
    c1 = 1.0
    for i in range(1, n):
        c2 = 1.0
        for j in range(i):
            c3 = nodes[i] - nodes[j]
            c2 *= c3
            for m in range(min(i, m_max) + 1):
                prev = delta[m - 1, i - 1, j] if m > 0 else 0.0
                delta[m, i, j] = (nodes[i] * delta[m, i - 1, j] - m * prev) / c3
        for m in range(min(i, m_max) + 1):
            prev = delta[m - 1, i - 1, i - 1] if m > 0 else 0.0
            delta[m, i, i] = c1 / c2 * (m * prev - nodes[i - 1] * delta[m, i - 1, i - 1])
        c1 = c2
    w_nodes = delta[2, n - 1, :]
    w = np.zeros(radius + 1)
    w[0] = w_nodes[0]
    for k in range(1, radius + 1):
        w[k] = w_nodes[2 * k - 1]
    return w


def _second_derivative_1d(n: int, h: float, w: np.ndarray, periodic: bool = False) -> sp.csr_matrix:
    radius = len(w) - 1
    if periodic:
        # circulant: entry (i, (i + o) mod n) for every offset o; wrapped taps that land on the
        # same point are summed by the COO -> CSR conversion
        rows, cols, vals = [], [], []
        for o in range(-radius, radius + 1):
            rows.append(np.arange(n))
            cols.append((np.arange(n) + o) % n)
            vals.append(np.full(n, w[abs(o)] / h ** 2))
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, n)).tocsr()
    offsets = [o for o in range(-radius, radius + 1) if abs(o) < n]
    diags = [np.full(n - abs(o), w[abs(o)] / h ** 2) for o in offsets]
    return sp.diags(diags, offsets, shape=(n, n), format="csr")


def _hamiltonian_sparse(nx: int, ny: int, nz: int, h: float, vloc: np.ndarray,
                        periodic: bool = False) -> sp.csr_matrix:
    w = fornberg_second_derivative(6)
    dx = _second_derivative_1d(nx, h, w, periodic)
    dy = _second_derivative_1d(ny, h, w, periodic)
    dz = _second_derivative_1d(nz, h, w, periodic)
    ix, iy, iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    lap = (sp.kron(iz, sp.kron(iy, dx)) + sp.kron(iz, sp.kron(dy, ix))
           + sp.kron(dz, sp.kron(iy, ix)))
    return (-0.5 * lap + sp.diags(vloc)).tocsr()


# --------------------------------------------------------------------------------------
# Gaussian-well potentials
# --------------------------------------------------------------------------------------
def _grid_coords(n: int, h: float, periodic: bool = False) -> np.ndarray:
    # Dirichlet: interior points of the box [0, (n+1) h], the walls carry the zero boundary
    # values; periodic: the points of the cell [0, n h).
    return np.arange(n) * h if periodic else (np.arange(n) + 1.0) * h


def _potential(nx, ny, nz, h, centres, depths, widths, periodic: bool = False) -> np.ndarray:
    x, y, z = (_grid_coords(n, h, periodic) for n in (nx, ny, nz))
    cell = (nx * h, ny * h, nz * h)
    images = (-1, 0, 1) if periodic else (0,)

    def gauss(t, c, s, length):
        # a periodic cell sums the well's nearest images along the axis
        return sum(np.exp(-((t - c - m * length) ** 2) / (2 * s * s)) for m in images)

    v = np.zeros((nz, ny, nx))
    for (cx, cy, cz), d, s in zip(centres, depths, widths):
        gx, gy, gz = gauss(x, cx, s, cell[0]), gauss(y, cy, s, cell[1]), gauss(z, cz, s, cell[2])
        v -= d * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return v.reshape(-1)


def _random_wells(rng, n_wells, box, periodic: bool = False):
    depths = rng.uniform(1.0, 3.0, n_wells)
    widths = rng.uniform(0.8, 1.5, n_wells)
    centres = []
    for s in widths:
        if periodic:
            centres.append([rng.uniform(0.0, b) for b in box])
        else:
            centres.append([rng.uniform(min(2.0 * s, 0.3 * b), b - min(2.0 * s, 0.3 * b)) for b in box])
    return np.array(centres), depths, widths


def _rocksalt_wells(rng, box, a=7.6, cells=2, jitter=0.1):
    """Rock-salt lattice of Li-like (deep) and H-like (shallow) wells, centred in the box."""
    fcc = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    li, hy = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                base = np.array([i, j, k], dtype=float)
                for f in fcc:
                    li.append((base + f) * a)
                    hy.append((base + f + np.array([0.5, 0.0, 0.0])) * a)
    li, hy = np.array(li), np.array(hy)
    extent = cells * a
    shift = (np.asarray(box) - extent) / 2.0 + a / 4.0
    centres = np.concatenate([li, hy]) + shift
    centres += rng.uniform(-jitter, jitter, centres.shape)
    depths = np.concatenate([np.full(len(li), 3.0), np.full(len(hy), 1.5)])
    widths = np.concatenate([np.full(len(li), 1.2), np.full(len(hy), 0.9)])
    return centres, depths, widths


# --------------------------------------------------------------------------------------
# Ground state: dense eigensolver or Chebyshev-filtered subspace iteration
# --------------------------------------------------------------------------------------
def _dense_ground_state(H: sp.csr_matrix, n_s: int):
    import scipy.linalg as sla
    vals, vecs = sla.eigh(H.toarray(), subset_by_index=[0, n_s])
    return vals[:n_s], vecs[:, :n_s].T.copy(), float(vals[n_s] - vals[n_s - 1])


def _chefsi_ground_state(H: sp.csr_matrix, n_s: int, rng, upper: float, lower: float,
                         tol: float = 1e-8, degree: int = 24, max_outer: int = 400):
    """Lowest n_s eigenpairs of the sparse symmetric H by Chebyshev-filtered subspace
    iteration (Y. Zhou, Y. Saad, M. Tiago, J. Chelikowsky, J. Comput. Phys. 219 (2006)
    172).  Runs on the GPU through torch when one is present, else on the host."""
    import torch
    dev = torch.device("cuda") if torch.cuda.is_available() else None
    n = H.shape[0]
    m = n_s + max(8, n_s // 2)
    if dev is not None:
        Ht = torch.sparse_csr_tensor(torch.from_numpy(H.indptr.astype(np.int64)),
                                     torch.from_numpy(H.indices.astype(np.int64)),
                                     torch.from_numpy(H.data), size=H.shape, device=dev)
        mv = lambda X: Ht @ X  # noqa: E731
        X = torch.from_numpy(rng.standard_normal((n, m))).to(dev)
        qr = lambda A: torch.linalg.qr(A)[0]  # noqa: E731
        eigh = torch.linalg.eigh
        norm = lambda A: torch.linalg.norm(A, dim=0)  # noqa: E731
        to_np = lambda A: A.cpu().numpy()  # noqa: E731
    else:
        mv = lambda X: H @ X  # noqa: E731
        X = rng.standard_normal((n, m))
        qr = lambda A: np.linalg.qr(A)[0]  # noqa: E731
        eigh = np.linalg.eigh
        norm = lambda A: np.linalg.norm(A, axis=0)  # noqa: E731
        to_np = lambda A: A  # noqa: E731

    X = qr(X)
    HX = mv(X)
    theta, Q = eigh(X.T @ HX)
    X, HX = X @ Q, HX @ Q
    a0 = float(lower)
    for _ in range(max_outer):
        res = norm(HX - X * theta[None, :])
        if float(res[:n_s].max()) <= tol:
            break
        cut = float(theta[-1])
        e, c = (upper - cut) / 2.0, (upper + cut) / 2.0
        sigma = e / (a0 - c)
        tau = 2.0 / sigma
        Y0 = X
        Y = (mv(X) - c * X) * (sigma / e)
        for _k in range(2, degree + 1):
            sigma_new = 1.0 / (tau - sigma)
            Y1 = (mv(Y) - c * Y) * (2.0 * sigma_new / e) - (sigma * sigma_new) * Y0
            Y0, Y, sigma = Y, Y1, sigma_new
        X = qr(Y)
        HX = mv(X)
        G = X.T @ HX
        theta, Q = eigh(0.5 * (G + G.T))
        X, HX = X @ Q, HX @ Q
        a0 = min(a0, float(theta[0]))
    else:
        raise RuntimeError("ground-state iteration did not reach the residual tolerance")
    vals = to_np(theta[:n_s]).copy()
    vecs = to_np(X[:, :n_s]).T.copy()
    return vals, vecs, float(theta[n_s] - theta[n_s - 1])


# --------------------------------------------------------------------------------------
# Public containers
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class System:
    """One isolated model system: grid, local potential, occupied orbitals, eigenvalues."""
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    vloc: np.ndarray          # (N_d,) float64, Hartree
    psi: np.ndarray           # (N_s, N_d) float64, l2-orthonormal rows (u = psi_continuum h^{3/2})
    eps: np.ndarray           # (N_s,) float64, ascending, Hartree
    n_atoms: int
    periodic: bool = False    # periodic cell (bulk) instead of zero boundary values

    @property
    def n_d(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_s(self) -> int:
        return self.psi.shape[0]


@dataclasses.dataclass
class Workload:
    """A system plus the method's run parameters (not the method itself)."""
    system: System
    n_r: int
    n_omega: int
    tol: float
    eps_c: float              # subspace-iteration energy threshold, Ha/atom
    seed: int


def _cache_dir() -> Optional[str]:
    d = os.environ.get("RPA_SYNTH_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "rpa_synth"))
    try:
        os.makedirs(d, exist_ok=True)
        return d
    except OSError:
        return None


_GEN_VERSION = "v2"


def make_system(name: str, n: Sequence[int], h: float, n_s: int, seed: int, wells: str = "random",
                n_wells: int = 4, gs_tol: float = 1e-8, periodic: bool = False) -> System:
    """Build (or load from the on-disk cache) a seeded Gaussian-well system.

    wells="random": n_wells wells with depth U[1,3] Ha, width U[0.8,1.5] bohr and
    centres uniform in the box at least 2 widths from every wall.
    wells="rocksalt": 32 Li-like (3 Ha, 1.2 bohr) + 32 H-like (1.5 Ha, 0.9 bohr)
    wells on a 2x2x2 rock-salt lattice of constant 7.6 bohr, jittered by U[-0.1,0.1].
    periodic: a periodic cell of n h per axis (wells summed over their nearest images, centres
    uniform in the cell) instead of a box with zero boundary values.
    """
    nx, ny, nz = (int(v) for v in n)
    key = f"{_GEN_VERSION}|{name}|{nx},{ny},{nz}|{h!r}|{n_s}|{seed}|{wells}|{n_wells}|{gs_tol!r}"
    if periodic:
        key += "|periodic"
    digest = hashlib.sha1(key.encode()).hexdigest()[:16]
    cdir = _cache_dir()
    path = os.path.join(cdir, f"{name}_{digest}.npz") if cdir else None
    if path and os.path.exists(path):
        z = np.load(path)
        return System(name, nx, ny, nz, h, z["vloc"], z["psi"], z["eps"], int(z["n_atoms"]), periodic)

    rng = np.random.default_rng(np.random.SeedSequence([seed, 0]))
    box = [nx * h, ny * h, nz * h] if periodic else [(nx + 1) * h, (ny + 1) * h, (nz + 1) * h]
    if wells == "random":
        centres, depths, widths = _random_wells(rng, n_wells, box, periodic)
    elif wells == "rocksalt":
        centres, depths, widths = _rocksalt_wells(rng, box)
    else:
        raise ValueError(wells)
    vloc = _potential(nx, ny, nz, h, centres, depths, widths, periodic)
    H = _hamiltonian_sparse(nx, ny, nz, h, vloc, periodic)
    if H.shape[0] <= 4096:
        eps, psi, gap = _dense_ground_state(H, n_s)
    else:
        w = fornberg_second_derivative(6)
        upper = 1.5 * (abs(w[0]) + 2.0 * np.abs(w[1:]).sum()) / h ** 2 + max(0.0, float(vloc.max()))
        gs_rng = np.random.default_rng(np.random.SeedSequence([seed, 1]))
        eps, psi, gap = _chefsi_ground_state(H, n_s, gs_rng, upper, float(vloc.min()), tol=gs_tol)
    if gap < 1e-4:
        raise ValueError(f"{name}: no gap between occupied and unoccupied levels ({gap:.2e} Ha)")
    # fix the sign of each orbital so that the result does not depend on the eigensolver
    for i in range(n_s):
        k = int(np.argmax(np.abs(psi[i])))
        if psi[i, k] < 0:
            psi[i] = -psi[i]
    system = System(name, nx, ny, nz, h, vloc, np.ascontiguousarray(psi), np.asarray(eps, dtype=np.float64),
                    len(depths), periodic)
    if path:
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "wb") as f:
            np.savez(f, vloc=vloc, psi=system.psi, eps=system.eps, n_atoms=system.n_atoms)
        os.replace(tmp, path)
    return system


def hamiltonian_matrix(system: System) -> sp.csr_matrix:
    """The model Hamiltonian that defines the ground-state problem, as a sparse matrix
    (assembled from Kronecker sums of 1D Fornberg-weight matrices)."""
    return _hamiltonian_sparse(system.nx, system.ny, system.nz, system.h, system.vloc, system.periodic)


def laplacian_matrix(nx: int, ny: int, nz: int, h: float, periodic: bool = False) -> sp.csr_matrix:
    """The finite-difference Laplacian of the model problem (Dirichlet or periodic), as a sparse
    matrix."""
    return -2.0 * _hamiltonian_sparse(nx, ny, nz, h, np.zeros(nx * ny * nz), periodic)


def trial_vectors(seed: int, n_r: int, n_d: int) -> np.ndarray:
    """Starting trial vectors V0: i.i.d. N(0,1), shape (n_r, n_d), not orthonormalised."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 2]))
    return rng.standard_normal((n_r, n_d))


def random_block(seed: int, k: int, n_d: int, stream: int = 3) -> np.ndarray:
    """Generic seeded N(0,1) block (k, n_d) for operator tests."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, stream]))
    return rng.standard_normal((k, n_d))


# --------------------------------------------------------------------------------------
# The model workloads (sizes follow the paper's cells: h 0.3-0.5 bohr, N_s = N_e/2)
# --------------------------------------------------------------------------------------
WORKLOADS = {
    # 15^3, h=0.5, 4 wells, 4 orbitals, N_r=8, N_omega=4, COCG tol 1e-8, plain FP64
    "tiny15": dict(n=(15, 15, 15), h=0.5, n_s=4, n_wells=4, wells="random", n_r=8, n_omega=4,
                   tol=1e-8, eps_c=1e-8, seed=0),
    # 40^3, h=0.4, 16 wells, 16 orbitals, N_r=64, N_omega=8 (plain vs mixed)
    "mixed40": dict(n=(40, 40, 40), h=0.4, n_s=16, n_wells=16, wells="random", n_r=64, n_omega=8,
                    tol=1e-8, eps_c=1e-6, seed=1),
    # 72^3, h=0.3, rock-salt LiH-shaped cell, 64 orbitals, N_r=256, N_omega=12
    "lih72": dict(n=(72, 72, 72), h=0.3, n_s=64, n_wells=64, wells="rocksalt", n_r=256, n_omega=12,
                  tol=1e-8, eps_c=1e-6, seed=2),
    # 32^3, h=0.45, 8 wells, 8 orbitals, N_r=32, N_omega=6 (adjoint)
    "adjoint32": dict(n=(32, 32, 32), h=0.45, n_s=8, n_wells=8, wells="random", n_r=32, n_omega=6,
                      tol=1e-8, eps_c=1e-7, seed=3),
    # periodic 40^3 cell, h=0.4, 16 wells, 16 orbitals, N_r=64, N_omega=8 (mixed40's sizes, bulk
    # boundary conditions)
    "bulk40": dict(n=(40, 40, 40), h=0.4, n_s=16, n_wells=16, wells="random", n_r=64, n_omega=8,
                   tol=1e-8, eps_c=1e-6, seed=4, periodic=True),
}


def workload(name: str, **overrides) -> Workload:
    p = dict(WORKLOADS[name])
    p.update(overrides)
    sys_ = make_system(name, p["n"], p["h"], p["n_s"], p["seed"], wells=p["wells"], n_wells=p["n_wells"],
                       periodic=p.get("periodic", False))
    return Workload(sys_, p["n_r"], p["n_omega"], p["tol"], p["eps_c"], p["seed"])


def small_system(n: Tuple[int, int, int] = (8, 8, 8), h: float = 0.5, n_s: int = 2, n_wells: int = 2,
                 seed: int = 11, periodic: bool = False) -> System:
    """Tiny system for brute-force checks (dense diagonalisation is cheap)."""
    return make_system(f"small{n[0]}x{n[1]}x{n[2]}", n, h, n_s, seed, wells="random", n_wells=n_wells,
                       periodic=periodic)
