"""Several independent systems in flight at once (an uneven batch: different grids, orbital
counts and subspace sizes).  Each system has its own context, CUDA stream and host thread: a
library call blocks its own thread while its kernels run, so the threads are what put the
systems on the GPU together.  The results must equal those of the same systems run one after
another bit for bit (every reduction in the library has a fixed order), and one system is
checked against the oracle at the mixed form's tolerance (1e-7 on the Ritz values).
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
