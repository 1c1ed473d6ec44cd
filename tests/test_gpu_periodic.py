"""Periodic boundary conditions (the paper's bulk cells, Section "Results") in the CUDA library
against the FP64 oracle's periodic operators, which tests/test_oracle_pins_periodic.py pins to
closed-form spectra and independent dense assemblies.

Grids: (16, 14, 12) runs the fused kernel (even nx: point pairs wrap onto point pairs);
(15, 13, 11) an odd nx, which runs the split kernels; (14, 8, 5) fewer planes than the stencil's
reach, so the wrapped z neighbours of a plane repeat.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRIDS = [(16, 14, 12), (15, 13, 11), (14, 8, 5)]


@pytest.fixture(scope="module")
def rpa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_01816_gb300 as m
    return m


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def opts(rpa, **kw):
    o = rpa.default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def system(grid, seed=41, n_s=2):
    return synth.small_system(grid, h=0.5, n_s=n_s, n_wells=2, seed=seed, periodic=True)


@pytest.mark.parametrize("grid", GRIDS)
def test_periodic_coulomb_matches_oracle(rpa, grid):
    s = system(grid)
    o = oracle.Oracle.from_system(s)
    assert o.grid.periodic
    X = synth.random_block(2, 4, s.n_d)
    with rpa.Context.from_system(s) as ctx:
        assert ctx.options.periodic == 1
        for p in (0.5, 1.0, -1.0):
            got = ctx.coulomb_apply(p, cuda(X)).cpu().numpy()
            assert relerr(got, o.coulomb.apply(X, p)) < 1e-12, p
        # the G = 0 mode: nu^p of a constant is zero
        one = ctx.coulomb_apply(0.5, cuda(np.ones((1, s.n_d)))).cpu().numpy()
        assert np.max(np.abs(one)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("grid", GRIDS)
def test_periodic_sternheimer_matches_oracle(rpa, prec, grid):
    s = system(grid)
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h, periodic=True)
    rng = np.random.default_rng(5)
    nsys = 5
    orbs = np.arange(nsys) % s.n_s
    b = rng.standard_normal((nsys, s.n_d))
    omega, tol = 0.3, 1e-11
    p = rpa.RPA_MIXED if prec == "mixed" else rpa.RPA_FP64
    with rpa.Context.from_system(s, opts(rpa, tol=tol, prec=p)) as ctx:
        x, it, st, code = ctx.sternheimer_solve(omega, orbs, cuda(b), project=True)
        x = x.cpu().numpy()
    assert code == rpa.RPA_OK and np.all(st.cpu().numpy() == 0)
    sig = -s.eps[orbs] + 1j * omega
    bp = b - (b @ s.psi.T) @ s.psi
    ref, _, rst = oracle.cocg(g, s.vloc, sig, bp.astype(complex), tol, 100000)
    assert np.all(rst == 0)
    assert relerr(x, ref) < 1e-8
    for k in range(nsys):     # true residual of the GPU solution under the oracle's periodic operator
        r = bp[k] - oracle.apply_h(g, s.vloc, x[k], sig[k])
        assert np.linalg.norm(r) <= 1.5 * tol * np.linalg.norm(bp[k])


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5])
def test_periodic_stencil_variants_match_oracle(rpa, shape):
    """Every stencil_shape on a periodic grid: the fused kernel (4), the split kernels (1, 2); the
    two-column split kernel (3) and the warp-specialised fused kernel (5) are Dirichlet only and
    stand in with the first split variant and the fused kernel."""
    s = system((16, 14, 12))
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h, periodic=True)
    b = np.random.default_rng(6).standard_normal((3, s.n_d))
    orbs = np.array([0, 1, 1])
    omega, tol = 0.4, 1e-11
    with rpa.Context.from_system(s, opts(rpa, tol=tol, prec=rpa.RPA_MIXED, stencil_shape=shape)) as ctx:
        x, _, st, code = ctx.sternheimer_solve(omega, orbs, cuda(b), project=False)
    assert code == rpa.RPA_OK
    sig = -s.eps[orbs] + 1j * omega
    ref, _, rst = oracle.cocg(g, s.vloc, sig, b.astype(complex), tol, 100000)
    assert np.all(rst == 0)
    assert relerr(x.cpu().numpy(), ref) < 1e-8


@pytest.mark.parametrize("zc", [2, 3])
def test_periodic_z_chunks_match_oracle(rpa, zc):
    s = system((15, 13, 11))
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h, periodic=True)
    b = np.random.default_rng(7).standard_normal((2, s.n_d))
    orbs = np.array([0, 1])
    omega, tol = 0.7, 1e-11
    for prec in (rpa.RPA_FP64, rpa.RPA_MIXED):
        with rpa.Context.from_system(s, opts(rpa, tol=tol, prec=prec, stencil_shape=1, z_chunks=zc)) as ctx:
            x, _, _, code = ctx.sternheimer_solve(omega, orbs, cuda(b), project=False)
        assert code == rpa.RPA_OK
        ref, _, _ = oracle.cocg(g, s.vloc, -s.eps[orbs] + 1j * omega, b.astype(complex), tol, 100000)
        assert relerr(x.cpu().numpy(), ref) < 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("grid", [(16, 14, 12), (15, 13, 11)])
def test_periodic_ec_matches_oracle_fixed_iterations(rpa, prec, grid):
    s = system(grid, seed=43, n_s=3)
    n_r, n_omega, iters, tol = 6, 3, 2, 1e-10
    V0 = synth.trial_vectors(43, n_r, s.n_d)
    p = rpa.RPA_MIXED if prec == "mixed" else rpa.RPA_FP64
    o = opts(rpa, tol=tol, prec=p, n_omega=n_omega, fixed_subspace_iters=iters, n_atoms=s.n_atoms, contractions=1)
    with rpa.Context.from_system(s, o) as ctx:
        res = ctx.ec(cuda(V0))
    ref = oracle.rpa_ec(oracle.Oracle.from_system(s), V0, n_omega, tol=tol, eps_c=0.0, fixed_iters=iters)
    lam_tol = 1e-8 if prec == "fp64" else 1e-7
    assert np.max(np.abs(res.lambdas - ref.lambdas)) < lam_tol
    assert abs(res.e_c - ref.e_c) < 1e-8
    assert np.all(res.lambdas <= 1e-12) and res.e_c < 0


def test_periodic_tensor_core_ec_meets_the_method_target(rpa):
    s = system((16, 14, 12), seed=43, n_s=3)
    n_r, n_omega, iters, tol = 6, 3, 2, 1e-10
    V0 = synth.trial_vectors(43, n_r, s.n_d)
    o = opts(rpa, tol=tol, prec=rpa.RPA_MIXED, n_omega=n_omega, fixed_subspace_iters=iters, n_atoms=s.n_atoms,
             contractions=2)
    with rpa.Context.from_system(s, o) as ctx:
        res = ctx.ec(cuda(V0))
    ref = oracle.rpa_ec(oracle.Oracle.from_system(s), V0, n_omega, tol=tol, eps_c=0.0, fixed_iters=iters)
    assert np.max(np.abs(res.lambdas - ref.lambdas)) < 1e-6
    assert abs(res.e_c - ref.e_c) / s.n_atoms < 1e-6


def test_periodic_is_fixed_at_setup(rpa):
    s = system((16, 14, 12))
    with rpa.Context.from_system(s) as ctx:
        o = opts(rpa, periodic=0)
        with pytest.raises(rpa.RpaError):
            ctx.set_options(o)
