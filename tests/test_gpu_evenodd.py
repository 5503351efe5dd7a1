"""GPU parity of the even/odd-reduced coarse solve (Alg. 2's even/odd-preconditioned FGMRES).

The self-block inverses, the Schur-complement application and the reduced solve are compared with
the oracle (oracle/evenodd.py, pinned against the dense Schur complement): FP64 to 1e-12 (fixed
FGMRES steps to 1e-10), FP32 to 1e-5; converged solves by the oracle's true residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coarse, dirac, evenodd as eo, lattice as lat  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


class EoCase:
    def __init__(self, amg, L, B, ntv, prec, seed, max_nrhs=4):
        self.amg, self.L, self.B, self.ntv = amg, L, B, ntv
        self.Lc = lat.coarse_dims(L, B)
        self.Vc = int(np.prod(self.Lc))
        self.nc = 2 * ntv
        sites = si.all_sites(L)
        Uh = si.links(seed, 0.3, sites)
        tvh = si.test_vectors(seed, ntv, sites)
        U = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
        self.Q = coarse.orthonormalize(tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
        self.Dc = coarse.coarse_operator(U, dirac.clover_field(U, H.CSW), H.M0, self.Q, L, B)
        pr = amg.AMG_FP64 if prec == "fp64" else amg.AMG_FP32
        self.ctype = torch.complex128 if prec == "fp64" else torch.complex64
        self.np_ctype = np.complex128 if prec == "fp64" else np.complex64
        p = amg.make_params(L, B, ntv, max_nrhs, H.M0, H.CSW, pr, pr, pr)
        self.stream = torch.cuda.current_stream()
        self.h, _ = amg.amg_setup_coarse(p, torch.from_numpy(Uh).cuda(), torch.from_numpy(tvh).cuda(), self.stream)
        amg.amg_setup_evenodd(self.h, self.stream)

    def dev(self, a):
        return torch.from_numpy(np.ascontiguousarray(a.astype(self.np_ctype))).cuda()

    def close(self):
        self.amg.amg_destroy(self.h)


@pytest.fixture(scope="module")
def fp64(amg):
    c = EoCase(amg, (8, 4, 4, 8), (2, 2, 2, 2), 6, "fp64", 515)  # coarse 4 x 2 x 2 x 4 (extent 2 aliasing)
    yield c
    c.close()


@pytest.fixture(scope="module")
def fp32(amg):
    c = EoCase(amg, (16, 8, 8, 16), (4, 4, 4, 4), 12, "fp32", 516)  # coarse 4 x 2 x 2 x 4, nc = 24
    yield c
    c.close()


def _half(c, seed, nrhs):
    v = si.coarse_vector(seed, c.ntv, nrhs, np.arange(c.Vc // 2))
    return v.reshape(c.Vc // 2, c.nc, nrhs)


def test_self_inverses_match_oracle(amg, fp64):
    c = fp64
    out = torch.empty((c.Vc // 2, c.nc, c.nc), dtype=torch.complex128, device="cuda")
    amg.amg_export_Dinv(c.h, out)
    got = out.cpu().numpy()
    want = eo.self_inverses(c.Dc, c.Lc)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("nrhs", [1, 3])
def test_schur_apply_fp64(amg, fp64, nrhs):
    c = fp64
    xe = _half(c, 70 + nrhs, nrhs)
    ye = torch.empty((c.Vc // 2, c.nc, nrhs), dtype=c.ctype, device="cuda")
    amg.amg_schur_apply(c.h, c.dev(xe), ye, nrhs, c.stream)
    want = eo.schur_apply(c.Dc, xe, c.Lc)
    assert H.rel(ye.cpu().numpy(), want) < 1e-12
    assert amg.amg_sync_status(c.h) == amg.AMG_OK


@pytest.mark.parametrize("nrhs", [1, 4])
def test_schur_apply_fp32(amg, fp32, nrhs):
    c = fp32
    xe = _half(c, 80 + nrhs, nrhs).astype(np.complex64)
    ye = torch.empty((c.Vc // 2, c.nc, nrhs), dtype=c.ctype, device="cuda")
    amg.amg_schur_apply(c.h, c.dev(xe), ye, nrhs, c.stream)
    want = eo.schur_apply(c.Dc, xe.astype(np.complex128), c.Lc)
    assert H.rel(ye.cpu().numpy().astype(np.complex128), want) < 1e-5


def test_eo_solve_fixed_steps_fp64(amg, fp64):
    """tol = 0: both run exactly 7 applications of S with restart 4 (one restart residual)."""
    c = fp64
    b = si.coarse_vector(91, c.ntv, 1, np.arange(c.Vc)).reshape(c.Vc, c.nc)
    x = torch.empty((c.Vc, c.nc, 1), dtype=c.ctype, device="cuda")
    info = amg.amg_coarse_solve_eo(c.h, c.dev(b[..., None]), x, 1, tol=0.0, restart=4, max_applies=7,
                                   stream=c.stream)
    xo, hist, n = eo.eo_solve(c.Dc, b, c.Lc, tol=0.0, restart=4, max_applies=7)
    assert info[0][0] == n == 7
    assert H.rel(x.cpu().numpy()[..., 0], xo) < 1e-10


def test_eo_solve_converged_fp32(amg, fp32):
    c = fp32
    nrhs, tol = 2, 1e-3
    b = si.coarse_vector(92, c.ntv, nrhs, np.arange(c.Vc)).reshape(c.Vc, c.nc, nrhs).astype(np.complex64)
    x = torch.empty((c.Vc, c.nc, nrhs), dtype=c.ctype, device="cuda")
    info = amg.amg_coarse_solve_eo(c.h, c.dev(b), x, nrhs, tol=tol, restart=30, max_applies=200, stream=c.stream)
    xs = x.cpu().numpy().astype(np.complex128)
    for r in range(nrhs):
        br = b[..., r].astype(np.complex128)
        rhs, _ = eo.reduced_rhs(c.Dc, br, c.Lc)
        res = br - coarse.coarse_apply(c.Dc, xs[..., r].reshape(c.Vc, 2, c.ntv), c.Lc).reshape(c.Vc, c.nc)
        assert info[r][1] <= tol
        assert np.linalg.norm(res) <= 1.05 * tol * np.linalg.norm(rhs) + 1e-5 * np.linalg.norm(br)


def test_cgc_eo_fp64(amg, fp64):
    """x = P x_c with x_c the reduced solve of R y to 1e-12 equals P D_c^-1 R y (dense solve)."""
    c = fp64
    y = si.fine_rhs(93, 1, si.all_sites(c.L))
    x = torch.empty(y.shape, dtype=torch.complex128, device="cuda")
    amg.amg_cgc_eo(c.h, torch.from_numpy(y).cuda(), x, 1, tol=1e-12, restart=64, max_applies=2000, stream=c.stream)
    yc = coarse.restrict(c.Q, y.reshape(H.field_shape(c.L) + (4, 3, 1)), c.B).reshape(c.Vc * c.nc)
    xc = np.linalg.solve(coarse.dense_coarse(c.Dc, c.Lc), yc).reshape(c.Vc, 2, c.ntv, 1)
    want = coarse.prolong(c.Q, xc, c.L, c.B).reshape(y.shape)
    assert H.rel(x.cpu().numpy(), want) < 1e-9


def test_rejections(amg, fp64):
    c = fp64
    # odd coarse extent: 12 / 4 = 3
    L, B = (12, 8, 8, 8), (4, 4, 4, 4)
    sites = si.all_sites(L)
    p = amg.make_params(L, B, 4, 1, H.M0, H.CSW, amg.AMG_FP64, amg.AMG_FP64, amg.AMG_FP64)
    h, _ = amg.amg_setup_coarse(p, torch.from_numpy(si.links(5, 0.3, sites)).cuda(),
                                torch.from_numpy(si.test_vectors(5, 4, sites)).cuda(), c.stream)
    try:
        with pytest.raises(amg.AmgError) as e:
            amg.amg_setup_evenodd(h, c.stream)
        assert e.value.status == amg.AMG_ERR_UNSUPPORTED
        b = torch.zeros((24, 8, 1), dtype=torch.complex128, device="cuda")
        with pytest.raises(amg.AmgError):  # no even/odd setup on this handle
            amg.amg_coarse_solve_eo(h, b, torch.empty_like(b), 1)
    finally:
        amg.amg_destroy(h)
    xe = torch.zeros((c.Vc // 2, c.nc, 17), dtype=torch.complex128, device="cuda")
    with pytest.raises(amg.AmgError):  # more right-hand sides than max_nrhs
        amg.amg_schur_apply(c.h, xe, torch.empty_like(xe), 17, c.stream)
