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


# A batch mixing precisions: an FP32 lattice with one right-hand side and two BF16 lattices that
# run on the tensor cores (R, D_c and fine vectors BF16; 4 and 12 right-hand sides).
MIXED = [((8, 8, 8, 8), (4, 4, 4, 4), 8, 0.2, 1, "fp32"),
         ((8, 8, 8, 8), (4, 4, 4, 4), 20, 0.3, 4, "bf16"),
         ((8, 8, 8, 12), (4, 4, 4, 4), 24, 0.4, 12, "bf16")]
U_BF16 = 2.0 ** -8


def _to_bf16_pairs(z):
    f = torch.from_numpy(np.ascontiguousarray(np.stack([z.real, z.imag], -1)).astype(np.float32))
    return f.to(torch.bfloat16)


def _from_bf16_pairs(t):
    f = t.float().cpu().numpy().astype(np.float64)
    return f[..., 0] + 1j * f[..., 1]


@pytest.fixture(scope="module")
def mixed(amg):
    st = torch.cuda.current_stream()
    lats = []
    for k, (L, B, ntv, eps, nrhs, prec) in enumerate(MIXED):
        seed = 860 + k
        sites = si.all_sites(L)
        Uh = si.links(seed, eps, sites)
        tvh = si.test_vectors(seed, ntv, sites)
        U = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
        Q = coarse.orthonormalize(tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
        Dc = coarse.coarse_operator(U, dirac.clover_field(U, H.CSW), H.M0, Q, L, B)
        pr = amg.AMG_FP32 if prec == "fp32" else amg.AMG_BF16
        p = amg.make_params(L, B, ntv, max(nrhs, 4), H.M0, H.CSW, pr, pr, pr)
        h, _ = amg.amg_setup_coarse(p, torch.from_numpy(Uh).cuda(), torch.from_numpy(tvh).cuda(), st)
        y = si.fine_rhs(seed + 50, nrhs, sites)
        if prec == "fp32":
            y = y.astype(np.complex64)
            yd = torch.from_numpy(y).cuda()
            x = torch.empty(y.shape, dtype=torch.complex64, device="cuda")
            yv = y.astype(np.complex128)
        else:
            yd = _to_bf16_pairs(y).cuda()
            x = torch.empty(yd.shape, dtype=torch.bfloat16, device="cuda")
            yv = _from_bf16_pairs(yd)  # the values the library sees
        Lc = lat.coarse_dims(L, B)
        yf = yv.reshape(H.field_shape(L) + (4, 3, nrhs))
        ref = coarse.prolong(Q, coarse.coarse_apply(Dc, coarse.restrict(Q, yf, B), Lc), L, B)
        aQ, aD = np.abs(Q).astype(np.complex128), np.abs(Dc).astype(np.complex128)
        absref = coarse.prolong(aQ, coarse.coarse_apply(aD, coarse.restrict(aQ, np.abs(yf).astype(np.complex128), B),
                                                        Lc), L, B)
        lats.append(dict(h=h, L=L, nrhs=nrhs, prec=prec, y=yd, x=x, ref=ref.reshape(yv.shape),
                         absref=absref.reshape(yv.shape).real, Vc=int(np.prod(Lc)), ntv=ntv))
    yield lats
    for c in lats:
        amg.amg_destroy(c["h"])


def _run_mixed(amg, lats, stream=None):
    amg.amg_batch_cgc([c["h"] for c in lats], [c["y"] for c in lats], [c["x"] for c in lats],
                      [c["nrhs"] for c in lats], stream or torch.cuda.current_stream())


def _result(c):
    return c["x"].cpu().numpy().astype(np.complex128) if c["prec"] == "fp32" else _from_bf16_pairs(c["x"])


def test_mixed_batch_matches_oracle(amg, mixed):
    """FP32 lattice within 1e-5; BF16 lattices within the stated bound: six BF16 roundings
    (R, y_c, D_c, D_c y_c, R again, x) of at most 2^-8 each, times || |P||D_c||R||y| || / ||P D_c R y||,
    plus the FP32 accumulation."""
    _run_mixed(amg, mixed)
    torch.cuda.synchronize()
    assert amg.amg_sync_status(mixed[0]["h"]) == amg.AMG_OK
    for c in mixed:
        got = _result(c)
        err = H.rel(got, c["ref"])
        if c["prec"] == "fp32":
            assert err < 1e-5
        else:
            ratio = np.linalg.norm(c["absref"]) / np.linalg.norm(c["ref"])
            assert err <= (6 * U_BF16 + 1e-4) * ratio, (err, ratio)
            assert err < 2e-2


def test_mixed_batch_equals_single_calls(amg, mixed):
    """The tensor-core lattices of the batch give exactly the bits of the single calls (same
    kernels, same rounding of y_c to BF16); the FP32 lattice agrees to 1e-5."""
    _run_mixed(amg, mixed)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    for c in mixed:
        yc = torch.empty((c["Vc"], 2, c["ntv"], c["nrhs"]), dtype=torch.complex64, device="cuda")
        zc = torch.empty_like(yc)
        x = torch.empty_like(c["x"])
        amg.amg_restrict(c["h"], c["y"], yc, c["nrhs"], st)
        amg.amg_coarse_apply(c["h"], yc, zc, c["nrhs"], st)
        amg.amg_prolong(c["h"], zc, x, c["nrhs"], st)
        torch.cuda.synchronize()
        if c["prec"] == "fp32":
            assert H.rel(c["x"].cpu().numpy(), x.cpu().numpy()) < 1e-5
        else:
            assert torch.equal(c["x"].view(torch.int16), x.view(torch.int16))


def test_mixed_batch_graph_and_autotune(amg, mixed):
    best = amg.amg_batch_autotune([c["h"] for c in mixed], [c["y"] for c in mixed], [c["x"] for c in mixed],
                                  [c["nrhs"] for c in mixed], torch.cuda.current_stream())
    assert best > 0
    _run_mixed(amg, mixed)
    torch.cuda.synchronize()
    want = [c["x"].clone() for c in mixed]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            _run_mixed(amg, mixed, s)
    torch.cuda.current_stream().wait_stream(s)
    for c in mixed:
        c["x"].zero_()
    g.replay()
    torch.cuda.synchronize()
    for c, w in zip(mixed, want):
        assert torch.equal(c["x"], w)
    assert amg.amg_sync_status(mixed[0]["h"]) == amg.AMG_OK
