"""Block COCG (rpa_options.block_cocg: the systems of one orbital solved s at a time by the block
variant of COCG, Section "Implementation") in the CUDA library, against the FP64 oracle (whose
block_cocg tests/test_oracle_pins_block.py pins).  Blocks change the iteration, not the
solution: solutions are held to the bounds of test_gpu_parity.py, and the FP64 form's block
iteration counts to those of the oracle's block_cocg on the same groups."""
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


def groups(orbs, s):
    """The library's grouping: runs of consecutive systems with the same orbital, s at most."""
    out, i = [], 0
    while i < len(orbs):
        e = i + 1
        while e < len(orbs) and e - i < s and orbs[e] == orbs[i]:
            e += 1
        out.append((i, e))
        i = e
    return out


CASES = [((16, 14, 12), False), ((15, 13, 11), False), ((14, 8, 5), True)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("s_blk", [1, 3, 4])
@pytest.mark.parametrize("grid,periodic", CASES)
def test_block_sternheimer_matches_oracle(rpa, prec, s_blk, grid, periodic):
    s = synth.small_system(grid, h=0.5, n_s=2, n_wells=2, seed=47, periodic=periodic)
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h, periodic=periodic)
    rng = np.random.default_rng(8)
    orbs = np.array([0, 0, 0, 0, 0, 1, 1])
    nsys = len(orbs)
    b = rng.standard_normal((nsys, s.n_d))
    omega, tol = 0.2, 1e-11
    p = rpa.RPA_MIXED if prec == "mixed" else rpa.RPA_FP64
    with rpa.Context.from_system(s, opts(rpa, tol=tol, prec=p, block_cocg=s_blk)) as ctx:
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
        for i, e in groups(orbs, s_blk):
            _, bit, bst = oracle.block_cocg(g, s.vloc, sig[i], bp[i:e].astype(complex), tol, 100000)
            assert bst == oracle.OK
            # same algorithm, different summation order: counts agree up to the last few iterations
            # (a column whose true residual ends just above tol takes a short second solve alone)
            assert abs(int(it[i:e].min()) - bit) <= max(3, 0.1 * bit), (i, e, it[i:e], bit)
            if e - i == 1:
                assert abs(int(it[i]) - rit[i]) <= max(3, 0.1 * rit[i])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_block_chi0_matches_oracle(rpa, prec):
    s = synth.small_system((12, 11, 10), h=0.5, n_s=3, n_wells=2, seed=21)
    o = oracle.Oracle.from_system(s)
    V = synth.random_block(8, 6, s.n_d)                # blocks of 4: one full and one of 2
    tol = 1e-11
    p = rpa.RPA_MIXED if prec == "mixed" else rpa.RPA_FP64
    with rpa.Context.from_system(s, opts(rpa, tol=tol, prec=p, contractions=1, block_cocg=4)) as ctx:
        for omega in (0.05, 1.7):
            R, code = ctx.apply_nuchi0(omega, cuda(V), symmetric=True)
            assert code == rpa.RPA_OK
            assert relerr(R.cpu().numpy(), o.chi_tilde(V, omega, tol)) < 1e-8
        R2, code = ctx.apply_nuchi0(0.4, cuda(V), symmetric=False)
        assert relerr(R2.cpu().numpy(), o.nu_chi0(V, 0.4, tol)) < 1e-8


def test_block_chi0_deterministic_and_block_sizes_agree(rpa):
    s = synth.small_system((13, 11, 9), h=0.5, n_s=3, n_wells=3, seed=33)
    V = synth.random_block(9, 7, s.n_d)
    out = {}
    with rpa.Context.from_system(s, opts(rpa, tol=1e-12, prec=rpa.RPA_MIXED)) as ctx:
        for blk in (0, 2, 7, 16):
            ctx.set_options(opts(rpa, tol=1e-12, prec=rpa.RPA_MIXED, block_cocg=blk))
            out[blk] = ctx.apply_nuchi0(0.6, cuda(V))[0].cpu().numpy()
        again = ctx.apply_nuchi0(0.6, cuda(V))[0].cpu().numpy()
        # waves of two groups of 2 (the 3 orbitals x 4 groups in six waves): the same sums in order
        ctx.set_options(opts(rpa, tol=1e-12, prec=rpa.RPA_MIXED, block_cocg=2, batch_systems=4))
        waves = ctx.apply_nuchi0(0.6, cuda(V))[0].cpu().numpy()
    assert np.array_equal(again, out[16])
    assert np.array_equal(waves, out[2])
    for blk in (2, 7, 16):
        assert relerr(out[blk], out[0]) < 1e-9, blk


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_block_ec_matches_oracle(rpa, prec):
    s = synth.small_system((16, 14, 12), h=0.5, n_s=3, n_wells=2, seed=43)
    n_r, n_omega, iters, tol = 8, 3, 2, 1e-10
    V0 = synth.trial_vectors(43, n_r, s.n_d)
    p = rpa.RPA_MIXED if prec == "mixed" else rpa.RPA_FP64
    o = opts(rpa, tol=tol, prec=p, n_omega=n_omega, fixed_subspace_iters=iters, n_atoms=s.n_atoms, contractions=1,
             block_cocg=8)
    with rpa.Context.from_system(s, o) as ctx:
        res = ctx.ec(cuda(V0))
    ref = oracle.rpa_ec(oracle.Oracle.from_system(s), V0, n_omega, tol=tol, eps_c=0.0, fixed_iters=iters)
    lam_tol = 1e-8 if prec == "fp64" else 1e-7
    assert res.status == rpa.RPA_OK
    assert np.max(np.abs(res.lambdas - ref.lambdas)) < lam_tol
    assert abs(res.e_c - ref.e_c) < 1e-8
    assert res.stats["sternheimer_solves"] == n_omega * iters * n_r * s.n_s


def test_block_sizes_past_a_tile_and_a_wave(rpa):
    """A grid of several Gram tiles with a ragged last tile, groups of 16 and of 5 in waves of one
    group (batch_systems = 16): the mixed form against the oracle's solutions."""
    s = synth.small_system((20, 18, 15), h=0.5, n_s=2, n_wells=3, seed=61)
    g = oracle.Grid(s.nx, s.ny, s.nz, s.h)
    rng = np.random.default_rng(62)
    orbs = np.array([1] * 16 + [0] * 5)
    b = rng.standard_normal((len(orbs), s.n_d))
    omega, tol = 0.8, 1e-10
    with rpa.Context.from_system(s, opts(rpa, tol=tol, prec=rpa.RPA_MIXED, block_cocg=16, batch_systems=16)) as ctx:
        x, it, st, code = ctx.sternheimer_solve(omega, orbs, cuda(b), project=False)
    assert code == rpa.RPA_OK
    sig = -s.eps[orbs] + 1j * omega
    ref, _, _ = oracle.cocg(g, s.vloc, sig, b.astype(complex), tol, 100000)
    assert relerr(x.cpu().numpy(), ref) < 1e-7
