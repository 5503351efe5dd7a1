"""The fused persistent batch x_k = P_k D_ck R_k y_k over lattices of different size.

Checked against the FP64 oracle's composition P D_c R y per lattice (FP32
tolerance), against the composition of the three single calls, after CUDA-graph
capture and replay, after autotuning, and through the bounded-wait test hook.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coarse, dirac, lattice as lat  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu

# (L, B, ntv, eps, nrhs): uneven sizes, right-hand-side counts that exercise the 4 + 1 chunking
BATCH = [((8, 8, 8, 8), (4, 4, 4, 4), 8, 0.2, 1),
         ((8, 8, 4, 12), (4, 4, 2, 4), 12, 0.3, 4),
         ((12, 8, 8, 8), (4, 4, 4, 4), 16, 0.4, 6)]


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


@pytest.fixture(scope="module")
def batch(amg):
    st = torch.cuda.current_stream()
    lats = []
    for k, (L, B, ntv, eps, nrhs) in enumerate(BATCH):
        seed = 800 + k
        sites = si.all_sites(L)
        Uh = si.links(seed, eps, sites)
        tvh = si.test_vectors(seed, ntv, sites)
        U = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
        Q = coarse.orthonormalize(tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
        Dc = coarse.coarse_operator(U, dirac.clover_field(U, H.CSW), H.M0, Q, L, B)
        p = amg.make_params(L, B, ntv, nrhs, H.M0, H.CSW, amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32)
        h, _ = amg.amg_setup_coarse(p, torch.from_numpy(Uh).cuda(), torch.from_numpy(tvh).cuda(), st)
        y = si.fine_rhs(seed + 50, nrhs, sites).astype(np.complex64)
        yf = y.astype(np.complex128).reshape(H.field_shape(L) + (4, 3, nrhs))
        ref = coarse.prolong(Q, coarse.coarse_apply(Dc, coarse.restrict(Q, yf, B), lat.coarse_dims(L, B)), L, B)
        lats.append(dict(h=h, L=L, nrhs=nrhs, y=torch.from_numpy(y).cuda(), ref=ref.reshape(y.shape),
                         x=torch.empty(y.shape, dtype=torch.complex64, device="cuda"),
                         Vc=int(np.prod(lat.coarse_dims(L, B))), ntv=ntv))
    yield lats
    for c in lats:
        amg.amg_destroy(c["h"])


def _run(amg, lats):
    amg.amg_batch_cgc([c["h"] for c in lats], [c["y"] for c in lats], [c["x"] for c in lats],
                      [c["nrhs"] for c in lats], torch.cuda.current_stream())


def _check(lats, tol=1e-5):
    torch.cuda.synchronize()
    for c in lats:
        assert H.rel(c["x"].cpu().numpy().astype(np.complex128), c["ref"]) < tol


def test_batch_matches_oracle(amg, batch):
    _run(amg, batch)
    _check(batch)
    assert amg.amg_sync_status(batch[0]["h"]) == amg.AMG_OK


def test_batch_matches_single_calls(amg, batch):
    _run(amg, batch)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    for c in batch:
        yc = torch.empty((c["Vc"], 2, c["ntv"], c["nrhs"]), dtype=torch.complex64, device="cuda")
        zc = torch.empty_like(yc)
        x = torch.empty_like(c["x"])
        amg.amg_restrict(c["h"], c["y"], yc, c["nrhs"], st)
        amg.amg_coarse_apply(c["h"], yc, zc, c["nrhs"], st)
        amg.amg_prolong(c["h"], zc, x, c["nrhs"], st)
        torch.cuda.synchronize()
        assert H.rel(c["x"].cpu().numpy(), x.cpu().numpy()) < 1e-5


def test_batch_graph_capture_and_replay(amg, batch):
    _run(amg, batch)  # the first call builds the job list; later calls only launch
    torch.cuda.synchronize()
    for c in batch:
        c["x"].zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            amg.amg_batch_cgc([c["h"] for c in batch], [c["y"] for c in batch], [c["x"] for c in batch],
                              [c["nrhs"] for c in batch], s)
    torch.cuda.current_stream().wait_stream(s)
    for c in batch:
        c["x"].zero_()
    g.replay()
    _check(batch)
    for c in batch:
        c["x"].zero_()
    g.replay()
    _check(batch)


def test_batch_autotune(amg, batch):
    best = amg.amg_batch_autotune([c["h"] for c in batch], [c["y"] for c in batch], [c["x"] for c in batch],
                                  [c["nrhs"] for c in batch], torch.cuda.current_stream())
    assert best > 0
    _run(amg, batch)
    _check(batch)


def test_batch_bounded_wait_reports_timeout(amg, batch):
    """Phase-1 count of lattice 0 that can never be reached: the coarse-operator jobs give up after
    their limit, the launch ends, the status says so, and the context stays usable."""
    h0 = batch[0]["h"]
    amg.amg_batch_test_hook(h0, 1)
    try:
        _run(amg, batch)
        assert amg.amg_sync_status(h0) == amg.AMG_ERR_TIMEOUT
    finally:
        amg.amg_batch_test_hook(h0, 0)
    # the status was reported once and cleared; the context and the handles stay usable
    _run(amg, batch)
    _check(batch)
    assert amg.amg_sync_status(h0) == amg.AMG_OK
    a = torch.ones(1000, device="cuda")
    assert float(a.sum()) == 1000.0
    st = torch.cuda.current_stream()
    c = batch[1]
    yc = torch.empty((c["Vc"], 2, c["ntv"], c["nrhs"]), dtype=torch.complex64, device="cuda")
    amg.amg_restrict(c["h"], c["y"], yc, c["nrhs"], st)
    assert amg.amg_sync_status(c["h"]) == amg.AMG_OK
