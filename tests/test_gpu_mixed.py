"""GPU tests of the mixed-precision coarse solve (FP16 / BF16 inner FGMRES, FP32 refinement).

The check is the one that matters to a user: the true relative residual
|b - D_c x| / |b| of the returned x, computed by the FP64 oracle with the FP64
D_c, is at most the requested tolerance (plus the FP32 operator's own error).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coarse, dirac, lattice as lat  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


@pytest.fixture(scope="module")
def lattice3(amg):
    L, B, ntv, seed = (8, 8, 8, 8), (4, 4, 4, 4), 24, 303
    sites = si.all_sites(L)
    Uh = si.links(seed, 0.3, sites)
    tvh = si.test_vectors(seed, ntv, sites)
    U = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
    Q = coarse.orthonormalize(tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
    Dc = coarse.coarse_operator(U, dirac.clover_field(U, H.CSW), H.M0, Q, L, B)
    st = torch.cuda.current_stream()
    Ud, tvd = torch.from_numpy(Uh).cuda(), torch.from_numpy(tvh).cuda()
    hs = {}
    for name, link, r, v in (("fp32", amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32),
                             ("fp16", amg.AMG_FP16_SCALED, amg.AMG_FP32, amg.AMG_FP32),
                             ("bf16", amg.AMG_BF16, amg.AMG_FP32, amg.AMG_FP32)):
        p = amg.make_params(L, B, ntv, 16, H.M0, H.CSW, link, r, v)
        hs[name], _ = amg.amg_setup_coarse(p, Ud, tvd, st)
    yield dict(L=L, B=B, ntv=ntv, Lc=lat.coarse_dims(L, B), Dc=Dc, h=hs, seed=seed)
    for h in hs.values():
        amg.amg_destroy(h)


@pytest.mark.parametrize("inner,nrhs", [("fp16", 4), ("bf16", 16), ("bf16", 4)])
def test_mixed_solve_reaches_true_tolerance(amg, lattice3, inner, nrhs):
    c = lattice3
    Vc = int(np.prod(c["Lc"]))
    b = si.coarse_vector(c["seed"] + 7, c["ntv"], nrhs, np.arange(Vc)).astype(np.complex64)
    x = torch.empty((Vc, 2, c["ntv"], nrhs), dtype=torch.complex64, device="cuda")
    tol = 1e-4
    info = amg.amg_coarse_solve_mixed(c["h"]["fp32"], c["h"][inner], torch.from_numpy(b).cuda(), x, nrhs,
                                      tol=tol, inner_tol=0.05, restart=20, max_inner_applies=200, max_outer=20,
                                      stream=torch.cuda.current_stream())
    xs = x.cpu().numpy().astype(np.complex128)
    for r in range(nrhs):
        inner_applies, passes, rel = info[r]
        assert rel <= tol and passes >= 2 and inner_applies >= passes
        true = H.rel(coarse.coarse_apply(c["Dc"], xs[..., r], c["Lc"]), b[..., r].astype(np.complex128))
        assert true <= tol * 1.05 + 1e-6
        assert abs(true - rel) <= 2e-6


def test_mixed_rejects_mismatched_handles(amg, lattice3):
    c = lattice3
    b = torch.zeros((16 * 48, 4), dtype=torch.complex64, device="cuda")
    x = torch.empty_like(b)
    with pytest.raises(amg.AmgError):
        amg.amg_coarse_solve_mixed(c["h"]["fp32"], c["h"]["fp16"], b, x, 17)
