"""Edge cases of the coarse-operator kernels: the largest supported Ntv (32, so 2 Ntv = 64: four
m-tiles, 16-piece row rotation) and the smallest (4, so 2 Ntv = 8: one half tile, one k-step),
with every column count the one-pass kernels specialise (1, 2, 3, 4, 8, 16), for FP32 storage
(SIMT and split-TF32 tensor cores), FP16-scaled storage and BF16 tensor-core storage.  Each result
is compared with the FP64 oracle: FP32 to 1e-5, FP16 / BF16 within the stated bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coarse, dirac, lattice as lat  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu

L, B = (8, 8, 8, 8), (4, 4, 4, 4)  # coarse 2^4: every direction aliases its opposite face


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


@pytest.fixture(scope="module", params=[32, 4], ids=["ntv32", "ntv4"])
def system(request):
    ntv = request.param
    sites = si.all_sites(L)
    Uh = si.links(717, 0.3, sites)
    tvh = si.test_vectors(717, ntv, sites)
    U = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
    Q = coarse.orthonormalize(tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
    Dc = coarse.coarse_operator(U, dirac.clover_field(U, H.CSW), H.M0, Q, L, B)
    return dict(ntv=ntv, Uh=Uh, tvh=tvh, Dc=Dc, Lc=lat.coarse_dims(L, B))


def _handle(amg, c, link):
    p = amg.make_params(L, B, c["ntv"], 16, H.M0, H.CSW, link, amg.AMG_FP32, amg.AMG_FP32)
    h, _ = amg.amg_setup_coarse(p, torch.from_numpy(c["Uh"]).cuda(), torch.from_numpy(c["tvh"]).cuda(),
                                torch.cuda.current_stream())
    return h


def _apply(amg, h, c, nrhs, seed):
    Vc = int(np.prod(c["Lc"]))
    xc = si.coarse_vector(seed, c["ntv"], nrhs, np.arange(Vc)).astype(np.complex64)
    y = torch.empty(xc.shape, dtype=torch.complex64, device="cuda")
    amg.amg_coarse_apply(h, torch.from_numpy(xc).cuda(), y, nrhs, torch.cuda.current_stream())
    got = y.cpu().numpy().astype(np.complex128)
    x64 = xc.astype(np.complex128)
    return got, coarse.coarse_apply(c["Dc"], x64, c["Lc"]), x64


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 8, 16])
def test_fp32_apply_edges(amg, system, nrhs):
    h = _handle(amg, system, amg.AMG_FP32)
    try:
        got, ref, _ = _apply(amg, h, system, nrhs, 40 + nrhs)
        assert H.rel(got, ref) < 1e-5
        assert amg.amg_sync_status(h) == amg.AMG_OK
    finally:
        amg.amg_destroy(h)


@pytest.mark.parametrize("nrhs", [1, 3, 4, 16])
def test_fp16_apply_edges(amg, system, nrhs):
    h = _handle(amg, system, amg.AMG_FP16_SCALED)
    try:
        got, ref, x64 = _apply(amg, h, system, nrhs, 50 + nrhs)
        bound = coarse.reduced_precision_bound(system["Dc"], x64, system["Lc"], 2.0 ** -11)
        assert H.rel(got, ref) <= bound
        assert amg.amg_sync_status(h) == amg.AMG_OK
    finally:
        amg.amg_destroy(h)


@pytest.mark.parametrize("nrhs", [4, 16])
def test_bf16_apply_edges(amg, system, nrhs):
    h = _handle(amg, system, amg.AMG_BF16)
    try:
        got, ref, x64 = _apply(amg, h, system, nrhs, 60 + nrhs)
        # BF16 storage of D_c and BF16 rounding of the input (2 u), FP32 accumulation
        bound = coarse.reduced_precision_bound(system["Dc"], x64, system["Lc"], 2 * 2.0 ** -8)
        assert H.rel(got, ref) <= bound
        assert amg.amg_sync_status(h) == amg.AMG_OK
    finally:
        amg.amg_destroy(h)


def test_bf16_restrict_prolong_edges(amg, system):
    """Tensor-core R and P with Ntv = 32 (four n-tiles, two k-steps in the prolongation) and
    Ntv = 4 (one half n-tile; the prolongation's k-step mostly padding)."""
    c = system
    ntv, nrhs = c["ntv"], 4
    p = amg.make_params(L, B, ntv, nrhs, H.M0, H.CSW, amg.AMG_BF16, amg.AMG_BF16, amg.AMG_BF16)
    st = torch.cuda.current_stream()
    h, _ = amg.amg_setup_coarse(p, torch.from_numpy(c["Uh"]).cuda(), torch.from_numpy(c["tvh"]).cuda(), st)
    try:
        Q = coarse.orthonormalize(c["tvh"].reshape(H.field_shape(L) + (4, 3, ntv)), B)
        y = si.fine_rhs(71, nrhs, si.all_sites(L))
        yb = torch.from_numpy(np.ascontiguousarray(np.stack([y.real, y.imag], -1)).astype(np.float32)).to(
            torch.bfloat16)
        yv = yb.float().numpy().astype(np.float64)
        yv = yv[..., 0] + 1j * yv[..., 1]
        Vc = int(np.prod(c["Lc"]))
        yc = torch.empty((Vc, 2, ntv, nrhs), dtype=torch.complex64, device="cuda")
        amg.amg_restrict(h, yb.cuda(), yc, nrhs, st)
        ref = coarse.restrict(Q, yv.reshape(H.field_shape(L) + (4, 3, nrhs)), B)
        assert H.rel(yc.cpu().numpy().astype(np.complex128), ref) < 1e-2
        x = torch.empty(yb.shape, dtype=torch.bfloat16, device="cuda")
        amg.amg_prolong(h, yc, x, nrhs, st)
        xf = x.float().cpu().numpy().astype(np.float64)
        got = xf[..., 0] + 1j * xf[..., 1]
        refx = coarse.prolong(Q, yc.cpu().numpy().astype(np.complex128), L, B).reshape(got.shape)
        assert H.rel(got, refx) < 1e-2
        assert amg.amg_sync_status(h) == amg.AMG_OK
    finally:
        amg.amg_destroy(h)
