"""Laplacian-preconditioned COCG (rpa_options.precondition; the paper's Section "Implementation":
Laplacian-based preconditioning through the Kronecker product formalism) in the CUDA library,
against the FP64 oracle (whose preconditioner and solver tests/test_oracle_pins_precond.py pins).
The preconditioner changes the iteration, not the solution: solutions are held to the bounds of
test_gpu_parity.py, and the FP64 form's iteration counts to those of the oracle's pcocg."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


CASES = [((16, 14, 12), False), ((15, 13, 11), False), ((16, 14, 12), True), ((14, 8, 5), True)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("grid,periodic", CASES)
def test_preconditioned_sternheimer_matches_oracle(rpa, prec, grid, periodic):
    s = synth.small_system(grid, h=0.5, n_s=2, n_wells=2, seed=47, periodic=periodic)
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h, periodic=periodic)
    rng = np.random.default_rng(8)
    nsys = 4
    orbs = np.arange(nsys) % s.n_s
    b = rng.standard_normal((nsys, s.n_d))
    omega, tol = 0.2, 1e-11
    p = rpa.RPA_MIXED if prec == "mixed" else rpa.RPA_FP64
    with rpa.Context.from_system(s, opts(rpa, tol=tol, prec=p, precondition=1)) as ctx:
        x, it, st, code = ctx.sternheimer_solve(omega, orbs, cuda(b), project=True)
        x, it = x.cpu().numpy(), it.cpu().numpy()
    assert code == rpa.RPA_OK and np.all(st.cpu().numpy() == 0)
    sig = -s.eps[orbs] + 1j * omega
    bp = b - (b @ s.psi.T) @ s.psi
    ref, rit, rst = oracle.cocg(g, s.vloc, sig, bp.astype(complex), tol, 100000)
    assert np.all(rst == 0)
    assert relerr(x, ref) < 1e-8
    for k in range(nsys):
        r = bp[k] - oracle.apply_h(g, s.vloc, x[k], sig[k])
        assert np.linalg.norm(r) <= 1.5 * tol * np.linalg.norm(bp[k])
    if prec == "fp64":
        o = oracle.Oracle.from_system(s)
        pit = []
        for k in range(nsys):
            m = oracle.laplacian_preconditioner(o.coulomb, float(np.mean(s.vloc)) + sig[k])
            _, itk, stk = oracle.pcocg(g, s.vloc, sig[k], bp[k:k + 1].astype(complex), tol, 100000, m)
            assert stk[0] == 0
            pit.append(itk[0])
        pit = np.array(pit)
        # same algorithm, different summation order: counts agree up to the last few iterations,
        # and the preconditioner needs fewer than the plain solver
        assert np.all(np.abs(it - pit) <= np.maximum(3, 0.1 * pit)), (it, pit)
        assert np.all(pit < rit), (pit, rit)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_preconditioned_ec_matches_oracle(rpa, prec):
    s = synth.small_system((16, 14, 12), h=0.5, n_s=3, n_wells=2, seed=43)
    n_r, n_omega, iters, tol = 6, 3, 2, 1e-10
    V0 = synth.trial_vectors(43, n_r, s.n_d)
    p = rpa.RPA_MIXED if prec == "mixed" else rpa.RPA_FP64
    o = opts(rpa, tol=tol, prec=p, n_omega=n_omega, fixed_subspace_iters=iters, n_atoms=s.n_atoms, contractions=1,
             precondition=1)
    with rpa.Context.from_system(s, o) as ctx:
        res = ctx.ec(cuda(V0))
        o.precondition = 0
        ctx.set_options(o)
        plain = ctx.ec(cuda(V0))
    ref = oracle.rpa_ec(oracle.Oracle.from_system(s), V0, n_omega, tol=tol, eps_c=0.0, fixed_iters=iters)
    lam_tol = 1e-8 if prec == "fp64" else 1e-7
    assert np.max(np.abs(res.lambdas - ref.lambdas)) < lam_tol
    assert abs(res.e_c - ref.e_c) < 1e-8
    # the same systems in fewer COCG iterations
    assert res.stats["cocg_iterations"] < plain.stats["cocg_iterations"], (res.stats["cocg_iterations"],
                                                                           plain.stats["cocg_iterations"])


def test_preconditioned_split_variants_and_z_chunks(rpa):
    s = synth.small_system((16, 14, 12), h=0.5, n_s=2, n_wells=2, seed=47)
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h)
    b = np.random.default_rng(9).standard_normal((3, s.n_d))
    orbs = np.array([0, 1, 1])
    omega, tol = 0.5, 1e-11
    ref, _, _ = oracle.cocg(g, s.vloc, -s.eps[orbs] + 1j * omega, b.astype(complex), tol, 100000)
    for shape, zc in ((1, 1), (2, 2), (3, 1), (4, 1), (6, 1)):
        o = opts(rpa, tol=tol, prec=rpa.RPA_MIXED, precondition=1, stencil_shape=shape, z_chunks=zc)
        with rpa.Context.from_system(s, o) as ctx:
            x, _, _, code = ctx.sternheimer_solve(omega, orbs, cuda(b), project=False)
        assert code == rpa.RPA_OK
        assert relerr(x.cpu().numpy(), ref) < 1e-8, (shape, zc)
