"""Several independent systems in flight at once (an uneven batch: different grids, orbital
counts and subspace sizes), two ways.  (1) Each system with its own context, CUDA stream and host
thread: a library call blocks its own thread while its kernels run, so the threads are what put
the systems on the GPU together.  (2) The batch calls rpa_apply_nuchi0_batch and rpa_ec_batch:
the Sternheimer systems of all contexts in one set of launches of the block COCG kernels.  The
results must equal those of the same systems run one after another bit for bit where the same
kernels run (every reduction in the library has a fixed order, and a group's arithmetic does not
depend on the other groups in flight), agree with the single-context default path to the mixed
form's tolerance, and one system is checked against the oracle (1e-7 on the Ritz values).
"""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (grid, occupied orbitals, subspace vectors, seed)
SPECS = [((24, 24, 24), 4, 8, 41), ((32, 32, 32), 6, 12, 42), ((24, 28, 26), 5, 10, 43),
         ((32, 24, 28), 8, 16, 44)]


@pytest.fixture(scope="module")
def rpa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_01816_gb300 as m
    return m


@pytest.fixture(scope="module")
def systems():
    return [synth.small_system(g, h=0.45, n_s=ns, n_wells=4, seed=seed) for g, ns, _, seed in SPECS]


def options(rpa, s):
    o = rpa.default_options()
    o.prec = rpa.RPA_MIXED
    o.tol = 1e-8
    o.n_omega = 2
    o.fixed_subspace_iters = 1
    o.n_atoms = s.n_atoms
    o.contractions = 1      # FP64 contractions: the oracle check below is held to 1e-7
    return o


def test_independent_systems_on_concurrent_streams(rpa, systems):
    v0 = [torch.as_tensor(synth.trial_vectors(seed, nr, s.n_d), device="cuda")
          for (_, _, nr, seed), s in zip(SPECS, systems)]
    ctxs = [rpa.Context.from_system(s, options(rpa, s)) for s in systems]
    try:
        torch.cuda.synchronize()
        alone = [ctx.ec(v) for ctx, v in zip(ctxs, v0)]
        streams = [torch.cuda.Stream() for _ in ctxs]
        together = [None] * len(ctxs)
        errors = []

        def run(i):
            try:
                with torch.cuda.stream(streams[i]):
                    together[i] = ctxs[i].ec(v0[i], stream=streams[i])
            except Exception as e:        # reported below, on the main thread
                errors.append(e)

        threads = [threading.Thread(target=run, args=(i,)) for i in range(len(ctxs))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        torch.cuda.synchronize()
        assert not errors, errors
        for a, b in zip(alone, together):
            assert a.status == rpa.RPA_OK and b.status == rpa.RPA_OK
            assert a.e_c == b.e_c
            assert np.array_equal(a.lambdas, b.lambdas)
    finally:
        for ctx in ctxs:
            ctx.close()
    # the first system against the oracle: same V0, one subspace iteration per frequency
    s, (_, _, nr, seed) = systems[0], SPECS[0]
    ref = oracle.rpa_ec(oracle.Oracle.from_system(s), synth.trial_vectors(seed, nr, s.n_d), 2, tol=1e-8,
                        eps_c=0.0, fixed_iters=1)
    assert np.max(np.abs(alone[0].lambdas - ref.lambdas)) < 1e-7
    assert abs(alone[0].e_c - ref.e_c) < 1e-7


def batch_options(rpa, s, block, fixed=1):
    o = options(rpa, s)
    o.block_cocg = block
    o.fixed_subspace_iters = fixed
    return o


@pytest.mark.parametrize("block", [1, 2])
def test_apply_nuchi0_batch_equals_each_context_alone(rpa, systems, block):
    ncols = [3, 0, 5, 2]                      # one member with no columns
    Vs = [torch.as_tensor(synth.random_block(70 + k, nc, s.n_d), device="cuda")
          for k, (nc, s) in enumerate(zip(ncols, systems))]
    ctxs = [rpa.Context.from_system(s, batch_options(rpa, s, block)) for s in systems]
    try:
        together, st = rpa.rpa.apply_nuchi0_batch(ctxs, 0.7, Vs)
        assert st == rpa.RPA_OK
        for ctx, V, R in zip(ctxs, Vs, together):
            if V.shape[0] == 0:
                continue
            alone, st1 = ctx.apply_nuchi0(0.7, V)
            assert st1 == rpa.RPA_OK
            assert torch.equal(alone, R)
    finally:
        for ctx in ctxs:
            ctx.close()


@pytest.mark.parametrize("fixed", [1, 0])
def test_ec_batch_equals_each_context_alone(rpa, systems, fixed):
    """fixed = 0: every context iterates to its own stopping rule, so contexts leave the batch at
    different subspace iterations."""
    v0 = [torch.as_tensor(synth.trial_vectors(seed, nr, s.n_d), device="cuda")
          for (_, _, nr, seed), s in zip(SPECS, systems)]
    ctxs = [rpa.Context.from_system(s, batch_options(rpa, s, 2, fixed)) for s in systems]
    try:
        together, st = rpa.rpa.ec_batch(ctxs, v0)
        assert st == rpa.RPA_OK
        for ctx, v, b in zip(ctxs, v0, together):
            a = ctx.ec(v)
            assert a.status == rpa.RPA_OK
            assert a.e_c == b.e_c
            assert np.array_equal(a.lambdas, b.lambdas)
            assert np.array_equal(a.e_c_per_omega, b.e_c_per_omega)
            assert a.stats["subspace_iterations"] == b.stats["subspace_iterations"]
            assert a.stats["sternheimer_solves"] == b.stats["sternheimer_solves"]
    finally:
        for ctx in ctxs:
            ctx.close()


def test_ec_batch_against_default_path_and_oracle(rpa, systems):
    """The batch (single-column groups in the block kernels) against each context's default path
    (the fused or split COCG kernels) and the first system against the oracle."""
    v0 = [torch.as_tensor(synth.trial_vectors(seed, nr, s.n_d), device="cuda")
          for (_, _, nr, seed), s in zip(SPECS, systems)]
    ctxs = [rpa.Context.from_system(s, options(rpa, s)) for s in systems]
    try:
        together, st = rpa.rpa.ec_batch(ctxs, v0)
        assert st == rpa.RPA_OK
        alone = [ctx.ec(v) for ctx, v in zip(ctxs, v0)]
    finally:
        for ctx in ctxs:
            ctx.close()
    for a, b in zip(alone, together):
        assert np.max(np.abs(a.lambdas - b.lambdas)) < 1e-7
        assert abs(a.e_c - b.e_c) < 1e-8
    s, (_, _, nr, seed) = systems[0], SPECS[0]
    ref = oracle.rpa_ec(oracle.Oracle.from_system(s), synth.trial_vectors(seed, nr, s.n_d), 2, tol=1e-8,
                        eps_c=0.0, fixed_iters=1)
    assert np.max(np.abs(together[0].lambdas - ref.lambdas)) < 1e-7
    assert abs(together[0].e_c - ref.e_c) < 1e-7


def test_batch_rejects_unequal_settings_and_repeated_contexts(rpa, systems):
    s0, s1 = systems[0], systems[1]
    a = rpa.Context.from_system(s0, options(rpa, s0))
    o = options(rpa, s1)
    o.tol = 1e-9
    b = rpa.Context.from_system(s1, o)
    V = torch.as_tensor(synth.random_block(5, 2, s0.n_d), device="cuda")
    W = torch.as_tensor(synth.random_block(6, 2, s1.n_d), device="cuda")
    try:
        with pytest.raises(rpa.RpaError) as e:
            rpa.rpa.apply_nuchi0_batch([a, b], 0.5, [V, W])
        assert "equal prec" in str(e.value)
        with pytest.raises(rpa.RpaError) as e:
            rpa.rpa.ec_batch([a, a], [V, V])
        assert "appears twice" in str(e.value)
    finally:
        a.close()
        b.close()
