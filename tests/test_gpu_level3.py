"""GPU parity of the third level (amg_setup_level2, amg_restrict2 / amg_prolong2, amg_two_grid,
amg_attach_level2 with amg_vcycle and amg_solve) against oracle/mg3.py.

* R2 and D_cc against the oracle's Q2 and R2 D_c P2: 1e-12 (FP64 setup on both sides);
* the level-1 / level-2 transfers: 1e-13;
* one two-grid cycle on level 1 and the three-level V-cycle with fixed work (MR steps, level-2
  FGMRES at tolerance 0 with a fixed number of applications, SAP cycles), so that both sides take
  the same steps: 1e-10;
* the outer FGMRES with the three-level V-cycle to convergence, by the oracle's true residual;
* detaching (explicitly or by destroying the level-2 handle) gives back the two-level V-cycle.
The level-2 lattices include an extent-3 direction (its +mu and -mu neighbours differ) and
blocks of extent 1 and 3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dirac, lattice as lat, mg, mg3  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


class Three:
    def __init__(self, amg, L, B, ntv, B2, ntv2, seed, prec="fp64", eps=0.3, max_nrhs=4):
        self.amg, self.L, self.B, self.ntv, self.B2, self.ntv2 = amg, L, B, ntv, B2, ntv2
        self.V = int(np.prod(L))
        self.Lc = lat.coarse_dims(L, B)
        self.Vc = int(np.prod(self.Lc))
        self.Lc2 = lat.coarse_dims(self.Lc, B2)
        self.seed = seed
        sites = si.all_sites(L)
        Uh = si.links(seed, eps, sites)
        self.tvh = si.test_vectors(seed, ntv, sites)
        self.U = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
        self.C = dirac.clover_field(self.U, H.CSW)
        self.tv2 = si.coarse_vector(seed + 1, ntv, ntv2, np.arange(self.Vc))
        pr = amg.AMG_FP64 if prec == "fp64" else amg.AMG_FP32
        self.ctype = torch.complex128 if prec == "fp64" else torch.complex64
        self.np_ctype = np.complex128 if prec == "fp64" else np.complex64
        self.stream = torch.cuda.current_stream()
        p = amg.make_params(L, B, ntv, max_nrhs, H.M0, H.CSW, pr, pr, pr)
        Ud = torch.from_numpy(Uh).cuda()
        self.h1, _ = amg.amg_setup_coarse(p, Ud, torch.from_numpy(self.tvh).cuda(), self.stream)
        amg.amg_setup_fine(self.h1, Ud, self.stream)
        p2 = amg.make_params(self.Lc, B2, ntv2, max_nrhs, H.M0, H.CSW, pr, pr, pr)
        self.h2, _ = amg.amg_setup_level2(self.h1, p2, torch.from_numpy(self.tv2).cuda(), self.stream)

    def hierarchy(self, **kw):
        hh = mg.Hierarchy(self.U, self.C, H.M0, self.L, self.B, **kw)
        hh.build_coarse(self.tvh.reshape(H.field_shape(self.L) + (4, 3, self.ntv)))
        return hh

    def level2(self, Dc, **kw):
        return mg3.Level2(Dc, self.Lc, self.B2, self.tv2, **kw)

    def dev(self, a):
        return torch.from_numpy(np.ascontiguousarray(a.astype(self.np_ctype))).cuda()

    def field(self, v):
        return v.reshape(H.field_shape(self.L) + (4, 3))

    def close(self):
        if self.h2 is not None:
            self.amg.amg_destroy(self.h2)
        self.amg.amg_destroy(self.h1)


CASES = [((12, 4, 4, 8), (2, 2, 2, 2), 6, (2, 1, 1, 2), 4),   # level-2 lattice 3x2x2x2
         ((8, 4, 4, 8), (2, 2, 2, 2), 5, (1, 1, 1, 2), 3)]    # B2 extents 1; odd ntv1


@pytest.fixture(scope="module", params=CASES, ids=["12x4x4x8_b2_b2112", "8x4x4x8_b2_b1112"])
def three(amg, request):
    L, B, ntv, B2, ntv2 = request.param
    c = Three(amg, L, B, ntv, B2, ntv2, 811)
    c.hh = c.hierarchy(n_smoother=2, n_mr=3, coarse_tol=0.0, coarse_restart=30, coarse_max_applies=5)
    yield c
    c.close()


def test_level2_setup_matches_oracle(amg, three):
    c = three
    l2 = c.level2(c.hh.Dc)
    Vc2 = int(np.prod(c.Lc2))
    nagg2 = int(np.prod(c.B2)) * c.ntv
    R = torch.empty((Vc2, 2, c.ntv2, nagg2), dtype=torch.complex128, device="cuda")
    amg.amg_export_R(c.h2, R)
    nc2 = 2 * c.ntv2
    D = torch.empty((Vc2, 9, nc2, nc2), dtype=torch.complex128, device="cuda")
    amg.amg_export_Dc(c.h2, D)
    torch.cuda.synchronize()
    assert H.rel(R.cpu().numpy(), H.q_to_lib_R(l2.Q2)) < 1e-12
    got = D.cpu().numpy()
    for d in range(9):
        assert H.rel(got[:, d], l2.Dcc[:, d]) < 1e-12, d
    assert amg.amg_sync_status(c.h2) == amg.AMG_OK


def test_transfers_match_oracle(amg, three):
    c = three
    l2 = c.level2(c.hh.Dc)
    Vc2 = int(np.prod(c.Lc2))
    yc = si.coarse_vector(c.seed + 5, c.ntv, 3, np.arange(c.Vc))
    ycc = torch.empty((Vc2, 2, c.ntv2, 3), dtype=c.ctype, device="cuda")
    amg.amg_restrict2(c.h2, c.dev(yc), ycc, 3, c.stream)
    assert H.rel(ycc.cpu().numpy(), mg3.restrict2(l2.Q2, yc, c.Lc, c.B2)) < 1e-13
    xcc = si.coarse_vector(c.seed + 6, c.ntv2, 3, np.arange(Vc2))
    xc = torch.empty((c.Vc, 2, c.ntv, 3), dtype=c.ctype, device="cuda")
    amg.amg_prolong2(c.h2, c.dev(xcc), xc, 3, c.stream)
    assert H.rel(xc.cpu().numpy(), mg3.prolong2(l2.Q2, xcc, c.Lc, c.B2)) < 1e-13


def test_two_grid_cycle_fixed_steps(amg, three):
    """Two MR steps on D_c before and after, the level-2 FGMRES(6) at tolerance 0 for 6
    applications of D_cc: the same steps on both sides, two independent columns."""
    c = three
    l2 = c.level2(c.hh.Dc, n_mr=2, tol=0.0, restart=6, max_applies=6)
    amg.amg_attach_level2(c.h1, c.h2, amg.make_level2_params(n_mr=2, restart=6, max_applies=6, tol=0.0))
    try:
        yc = si.coarse_vector(c.seed + 7, c.ntv, 2, np.arange(c.Vc))
        xc = torch.empty((c.Vc, 2, c.ntv, 2), dtype=c.ctype, device="cuda")
        amg.amg_two_grid(c.h1, c.dev(yc), xc, 2, c.stream)
        assert H.rel(xc.cpu().numpy(), l2.two_grid(yc)) < 1e-10
        assert amg.amg_sync_status(c.h1) == amg.AMG_OK
    finally:
        amg.amg_attach_level2(c.h1, None)


def test_three_level_vcycle_fixed_steps_and_detach(amg, three):
    c = three
    vp = amg.make_vcycle_params(coarse_tol=0.0, coarse_restart=30, coarse_max_applies=5, n_smoother=2, n_mr=3)
    l2 = c.level2(c.hh.Dc, n_mr=1, tol=0.0, restart=4, max_applies=4)
    y = si.fine_rhs(c.seed + 8, 1, si.all_sites(c.L))
    x = torch.empty((c.V, 4, 3, 1), dtype=c.ctype, device="cuda")
    amg.amg_attach_level2(c.h1, c.h2, amg.make_level2_params(n_mr=1, restart=4, max_applies=4, tol=0.0))
    amg.amg_vcycle(c.h1, vp, c.dev(y), x, 1, c.stream)
    ref3 = mg3.vcycle3(c.hh, l2, c.field(y[..., 0])).reshape(c.V, 4, 3)
    assert H.rel(x.cpu().numpy()[..., 0], ref3) < 1e-10
    amg.amg_attach_level2(c.h1, None)
    amg.amg_vcycle(c.h1, vp, c.dev(y), x, 1, c.stream)
    ref2 = c.hh.vcycle(c.field(y[..., 0])).reshape(c.V, 4, 3)
    assert H.rel(x.cpu().numpy()[..., 0], ref2) < 1e-10
    assert amg.amg_sync_status(c.h1) == amg.AMG_OK


def _dirac(c, psi):
    return dirac.apply_dirac(c.U, c.C, H.M0, c.field(psi.astype(np.complex128))).reshape(c.V, 4, 3)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_three_level_outer_solve_converges(amg, prec):
    """FGMRES on D preconditioned with the three-level V-cycle to 1e-8 (FP64) or 1e-5 (FP32), by
    the oracle's true residual; destroying the level-2 handle first detaches it."""
    c = Three(amg, (8, 8, 8, 8), (2, 2, 2, 2), 8, (2, 2, 2, 2), 6, 812, prec=prec)
    try:
        tol = 1e-8 if prec == "fp64" else 1e-5
        vp = amg.make_vcycle_params(n_smoother=4, n_mr=4)
        amg.amg_attach_level2(c.h1, c.h2, amg.make_level2_params(n_mr=2, restart=30, max_applies=200, tol=0.05))
        f = si.fine_rhs(c.seed + 9, 2, si.all_sites(c.L))
        u = torch.empty((c.V, 4, 3, 2), dtype=c.ctype, device="cuda")
        info = amg.amg_solve(c.h1, vp, c.dev(f), u, 2, tol=tol, restart=30, max_applies=300, stream=c.stream)
        got = u.cpu().numpy()
        for r in range(2):
            true = np.linalg.norm(f[..., r] - _dirac(c, got[..., r])) / np.linalg.norm(f[..., r])
            assert info[r][1] <= tol
            assert true < 10 * tol
        amg.amg_destroy(c.h2)
        c.h2 = None
        info2 = amg.amg_solve(c.h1, vp, c.dev(f), u, 2, tol=tol, restart=30, max_applies=300, stream=c.stream)
        assert all(i[1] <= tol for i in info2)
        assert amg.amg_sync_status(c.h1) == amg.AMG_OK
    finally:
        c.close()


def test_adaptive_setup_refuses_with_level2_attached(amg, three):
    """The adaptive setup rebuilds D_c, which would leave an attached D_cc stale: it refuses
    until the level 2 is detached."""
    c = three
    vp = amg.make_vcycle_params(n_smoother=1, n_mr=2)
    amg.amg_attach_level2(c.h1, c.h2, amg.make_level2_params())
    try:
        U = torch.from_numpy(si.links(c.seed, 0.3, si.all_sites(c.L))).cuda()
        tv = torch.from_numpy(c.tvh.copy()).cuda()
        with pytest.raises(amg.AmgError) as e:
            amg.amg_adaptive_setup(c.h1, vp, U, tv, n_setup=0, stream=c.stream)
        assert e.value.status == amg.AMG_ERR_INVALID_ARG
    finally:
        amg.amg_attach_level2(c.h1, None)
    assert amg.amg_sync_status(c.h1) == amg.AMG_OK
