"""The allocation-free coarse solve (amg_coarse_solve_noalloc) against amg_coarse_solve.

amg_coarse_solve_noalloc serves callers that may not allocate device memory at
solve time; it keeps its Krylov workspace in a fixed scratch array inside the
library.  This file runs last so that a failure here leaves every other test
already run; it must pass both alone in a fresh process and after the others.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


def _handle(amg, L, B, ntv, seed, max_nrhs):
    sites = si.all_sites(L)
    U = torch.from_numpy(si.links(seed, 0.3, sites)).cuda()
    tv = torch.from_numpy(si.test_vectors(seed, ntv, sites)).cuda()
    p = amg.make_params(L, B, ntv, max_nrhs, H.M0, H.CSW, amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32)
    h, _ = amg.amg_setup_coarse(p, U, tv, torch.cuda.current_stream())
    return h


@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_solve_matches_allocating_solve(amg, nrhs):
    L, B, ntv = (8, 4, 6, 4), (2, 2, 2, 2), 6
    h = _handle(amg, L, B, ntv, 123, 4)
    try:
        stream = torch.cuda.current_stream()
        Vc = 4 * 2 * 3 * 2
        ref = torch.empty((Vc, 2, ntv, nrhs), dtype=torch.complex64, device="cuda")
        got = torch.empty_like(ref)
        for call in range(2):  # two calls in a row: the second runs on the scratch the first left behind
            b = torch.from_numpy(si.coarse_vector(500 + call, ntv, nrhs, np.arange(Vc))).to(torch.complex64).cuda()
            info_ref = amg.amg_coarse_solve(h, b, ref, nrhs, tol=1e-4, restart=8, max_applies=200, stream=stream)
            info = amg.amg_coarse_solve_noalloc(h, b, got, nrhs, tol=1e-4, restart=8, max_applies=200,
                                                stream=stream)
            torch.cuda.synchronize()
            assert [i[0] for i in info] == [i[0] for i in info_ref]
            assert all(i[1] <= 1e-4 for i in info)
            assert H.rel(got.cpu().numpy(), ref.cpu().numpy()) < 1e-5
        # without info the call does not synchronise and still gives the same answer
        got.zero_()
        assert amg.amg_coarse_solve_noalloc(h, b, got, nrhs, tol=1e-4, restart=8, max_applies=200,
                                            stream=stream, info=False) is None
        torch.cuda.synchronize()
        assert H.rel(got.cpu().numpy(), ref.cpu().numpy()) < 1e-5
        assert amg.amg_sync_status(h) == amg.AMG_OK
    finally:
        amg.amg_destroy(h)


def test_noalloc_rejects_workspace_beyond_scratch(amg):
    """16^4 lattice, 4^4 blocks, Ntv = 20, 16 right-hand sides: FGMRES(30) needs about 43 MB."""
    L, B, ntv = (16, 16, 16, 16), (4, 4, 4, 4), 20
    h = _handle(amg, L, B, ntv, 321, 16)
    try:
        Vc = 256
        b = torch.zeros((Vc, 2, ntv, 16), dtype=torch.complex64, device="cuda")
        x = torch.empty_like(b)
        assert amg.amg_noalloc_scratch_bytes() == 16 << 20
        with pytest.raises(amg.AmgError) as e:
            amg.amg_coarse_solve_noalloc(h, b, x, 16, tol=0.05, restart=30, max_applies=10)
        assert e.value.status == amg.AMG_ERR_INVALID_ARG
        assert "scratch" in str(e.value)
        # the same request with a short restart fits; with 40 coarse components and 16 columns it
        # runs the split-TF32 tensor-core apply and the long-vector form of the fused Arnoldi step,
        # and must give what amg_coarse_solve gives with the same arguments
        b = torch.from_numpy(si.coarse_vector(654, ntv, 16, np.arange(Vc))).to(torch.complex64).cuda()
        ref = torch.empty_like(b)
        info_ref = amg.amg_coarse_solve(h, b, ref, 16, tol=0.05, restart=4, max_applies=20)
        info = amg.amg_coarse_solve_noalloc(h, b, x, 16, tol=0.05, restart=4, max_applies=20)
        torch.cuda.synchronize()
        assert [i[0] for i in info] == [i[0] for i in info_ref]
        assert all(i[1] <= 0.05 for i in info)
        assert H.rel(x.cpu().numpy(), ref.cpu().numpy()) < 1e-5
        assert amg.amg_sync_status(h) == amg.AMG_OK
    finally:
        amg.amg_destroy(h)


def test_noalloc_allocates_nothing(amg):
    """The property the entry point exists for: on a handle that has never run the allocating solve,
    noalloc calls leave the device's free memory unchanged.  A first call on another handle loads
    the solver's kernels beforehand (module loading may itself take device memory)."""
    L, B, ntv, nrhs = (8, 4, 6, 4), (2, 2, 2, 2), 6, 4
    Vc = 4 * 2 * 3 * 2
    stream = torch.cuda.current_stream()
    warm = _handle(amg, L, B, ntv, 124, nrhs)
    fresh = _handle(amg, L, B, ntv, 125, nrhs)
    try:
        b = torch.from_numpy(si.coarse_vector(77, ntv, nrhs, np.arange(Vc))).to(torch.complex64).cuda()
        x = torch.empty_like(b)
        amg.amg_coarse_solve_noalloc(warm, b, x, nrhs, tol=1e-4, restart=8, max_applies=40, stream=stream)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            info = amg.amg_coarse_solve_noalloc(fresh, b, x, nrhs, tol=1e-4, restart=8, max_applies=40,
                                                stream=stream)
            assert all(i[1] <= 1e-4 for i in info)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert amg.amg_sync_status(fresh) == amg.AMG_OK
    finally:
        amg.amg_destroy(warm)
        amg.amg_destroy(fresh)
