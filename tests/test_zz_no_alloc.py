"""The allocation-free Coulomb entry point (rpa_coulomb_apply_noalloc).

It serves callers that cannot let the library allocate device memory during a call, for
example an application whose device memory is fully reserved by its own pool allocator.
Two things are checked: the call gives the same result as the allocating rpa_coulomb_apply
on two calls in a row, and it allocates nothing.  The no-alloc calls run first on a fresh
context, before any allocating call could have grown the context's own Coulomb workspace,
and the device's free memory must not change across them.  Kept in a file that runs last.
"""
import ctypes

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


def _call(fn, ctx, power, X, out):
    stream = torch.cuda.current_stream().cuda_stream
    return fn(ctx._h, ctypes.c_double(power), X.data_ptr(), out.data_ptr(), X.shape[0], stream)


def test_noalloc_coulomb_matches_allocating_entry_point(rpa):
    s = synth.workload("tiny15").system
    lib = rpa.library()
    cases = [(0.5, 41, 5), (1.0, 42, 3)]              # two calls in a row
    with rpa.Context.from_system(s) as ctx:
        # every tensor is allocated up front so that the calls below are the only candidates
        # for a device allocation
        inputs = [torch.as_tensor(synth.random_block(seed, k, s.n_d), device="cuda") for _, seed, k in cases]
        got = [torch.full_like(X, float("nan")) for X in inputs]
        ref = [torch.empty_like(X) for X in inputs]
        warm = torch.zeros((1, s.n_d), dtype=torch.float64, device="cuda")
        # one warm-up call: the module's first call on this device looks up the scratch address
        assert _call(lib.rpa_coulomb_apply_noalloc, ctx, 0.5, warm, torch.empty_like(warm)) == rpa.RPA_OK
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        for (power, _, _), X, out in zip(cases, inputs, got):
            assert _call(lib.rpa_coulomb_apply_noalloc, ctx, power, X, out) == rpa.RPA_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, "the no-alloc entry point allocated device memory"
        # the allocating entry point on the same inputs
        for (power, _, _), X, out in zip(cases, inputs, ref):
            assert _call(lib.rpa_coulomb_apply, ctx, power, X, out) == rpa.RPA_OK
        for call, (g, r) in enumerate(zip(got, ref)):
            err = (g - r).abs().max().item() / r.abs().max().item()
            assert err < 1e-12, (call, err)


def test_noalloc_coulomb_rejects_requests_beyond_the_scratch(rpa):
    s = synth.workload("tiny15").system
    lib = rpa.library()
    # 2 * k * N_d + N_d doubles must fit in RPA_STATIC_SCRATCH_BYTES = 64 MiB
    k = (64 << 20) // (8 * 2 * s.n_d) + 1
    with rpa.Context.from_system(s) as ctx:
        X = torch.zeros((k, s.n_d), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(X)
        st = _call(lib.rpa_coulomb_apply_noalloc, ctx, 0.5, X, out)
        assert st == rpa.RPA_ERR_INVALID
        assert "scratch" in rpa.last_error()
