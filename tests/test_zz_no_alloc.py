"""The allocation-free Coulomb entry point (rpa_coulomb_apply_noalloc), for callers that cannot
let the library allocate device memory during a call: it must give the same result as the
allocating rpa_coulomb_apply.  Kept in a file that runs last."""
import ctypes

import numpy as np
import pytest

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


def _call(lib, fn, ctx, power, X, out):
    stream = torch.cuda.current_stream().cuda_stream
    return fn(ctx._h, ctx_power(power), X.data_ptr(), out.data_ptr(), X.shape[0], stream)


def ctx_power(p):
    return ctypes.c_double(p)


def test_noalloc_coulomb_matches_allocating_entry_point(rpa):
    s = synth.workload("tiny15").system
    lib = rpa.library()
    with rpa.Context.from_system(s) as ctx:
        for call, (power, seed, k) in enumerate([(0.5, 41, 5), (1.0, 42, 3)]):   # two calls in a row
            X = torch.as_tensor(synth.random_block(seed, k, s.n_d), device="cuda")
            ref = torch.empty_like(X)
            got = torch.full_like(X, float("nan"))
            assert _call(lib, lib.rpa_coulomb_apply, ctx, power, X, ref) == rpa.RPA_OK
            assert _call(lib, lib.rpa_coulomb_apply_noalloc, ctx, power, X, got) == rpa.RPA_OK
            err = (got - ref).abs().max().item() / ref.abs().max().item()
            assert err < 1e-12, (call, err)


def test_noalloc_coulomb_rejects_requests_beyond_the_scratch(rpa):
    s = synth.workload("tiny15").system
    lib = rpa.library()
    # 2 * k * N_d + N_d doubles must fit in RPA_STATIC_SCRATCH_BYTES = 64 MiB
    k = (64 << 20) // (8 * 2 * s.n_d) + 1
    with rpa.Context.from_system(s) as ctx:
        X = torch.zeros((k, s.n_d), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(X)
        st = _call(lib, lib.rpa_coulomb_apply_noalloc, ctx, 0.5, X, out)
        assert st == rpa.RPA_ERR_INVALID
        assert "scratch" in rpa.last_error()
