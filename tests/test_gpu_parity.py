"""GPU parity: the CUDA library through its C ABI against the FP64 oracle.

Tolerances (relative L2): FP64 setup and applies 1e-12; FP32 applies 1e-5;
FP16 / BF16 applies within the stated bound of oracle.coarse.reduced_precision_bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coarse, dirac, krylov, lattice as lat  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


class Case:
    """Host inputs, oracle results and a library handle for one lattice."""

    def __init__(self, amg, L, B, ntv, eps, seed, link_prec, vec_prec, r_prec=None, max_nrhs=8):
        self.amg, self.L, self.B, self.ntv, self.eps, self.seed = amg, L, B, ntv, eps, seed
        self.Lc = lat.coarse_dims(L, B)
        self.Vc = int(np.prod(self.Lc))
        self.V = int(np.prod(L))
        sites = si.all_sites(L)
        self.Uh = si.links(seed, eps, sites)
        self.tvh = si.test_vectors(seed, ntv, sites)
        self.U = np.moveaxis(self.Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
        self.C = dirac.clover_field(self.U, H.CSW)
        self.Q = coarse.orthonormalize(self.tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
        self.Dc = coarse.coarse_operator(self.U, self.C, H.M0, self.Q, L, B)
        self.vec_prec = vec_prec
        self.cdt = torch.complex128 if vec_prec == amg.AMG_FP64 else torch.complex64
        r_prec = r_prec if r_prec is not None else (amg.AMG_FP64 if vec_prec == amg.AMG_FP64 else amg.AMG_FP32)
        p = amg.make_params(L, B, ntv, max_nrhs, H.M0, H.CSW, link_prec, r_prec, vec_prec)
        self.stream = torch.cuda.current_stream()
        self.h, _ = amg.amg_setup_coarse(p, torch.from_numpy(self.Uh).cuda(),
                                         torch.from_numpy(self.tvh).cuda(), self.stream)

    def close(self):
        self.amg.amg_destroy(self.h)

    def fine(self, nrhs, seed_off=0):
        return si.fine_rhs(self.seed + seed_off, nrhs, si.all_sites(self.L))

    def coarse_vec(self, nrhs, seed_off=0):
        return si.coarse_vector(self.seed + seed_off, self.ntv, nrhs, np.arange(self.Vc))

    def dev(self, a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(self.cdt).cuda()


def _export(amg, fn, h, shape):
    out = torch.empty(shape, dtype=torch.complex128, device="cuda")
    fn(h, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def tiny64(amg):
    L, B, ntv, eps, off = H.WORKLOADS["tiny_4^4_b2_ntv8"]
    c = Case(amg, L, B, ntv, eps, si.SEED_BASE + off, amg.AMG_FP64, amg.AMG_FP64)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ragged32(amg):
    # coarse extents 4, 2, 3, 2 and ntv = 6: nothing is a power of two or a tile multiple
    c = Case(amg, (8, 4, 6, 4), (2, 2, 2, 2), 6, 0.4, 99, amg.AMG_FP32, amg.AMG_FP32)
    yield c
    c.close()


def test_setup_fp64_matches_oracle(amg, tiny64):
    c = tiny64
    C = _export(amg, amg.amg_export_clover, c.h, (c.V, 2, 6, 6))
    assert H.rel(C, H.clover_to_lib(c.C)) < 1e-12
    R = _export(amg, amg.amg_export_R, c.h, (c.Vc, 2, c.ntv, 6 * 16))
    assert H.rel(R, H.q_to_lib_R(c.Q)) < 1e-12
    Dc = _export(amg, amg.amg_export_Dc, c.h, (c.Vc, 9, 2 * c.ntv, 2 * c.ntv))
    assert H.rel(Dc, c.Dc) < 1e-12
    for d in range(9):
        assert H.rel(Dc[:, d], c.Dc[:, d]) < 1e-12
    # Eq. dagger holds exactly in the stored operator (backward blocks are filled from it)
    s = coarse.gamma5_coarse(c.ntv)
    nbr = lat.coarse_neighbours(c.Lc)
    for i in range(c.Vc):
        for mu in range(4):
            j = nbr[i, 1 + 2 * mu]
            assert np.array_equal(Dc[j, 2 + 2 * mu], s[:, None] * Dc[i, 1 + 2 * mu].conj().T * s[None, :])
    stored = _export(amg, amg.amg_export_Dc_stored, c.h, Dc.shape)
    assert np.array_equal(stored, Dc)


@pytest.mark.parametrize("nrhs", [1, 3, 4])
def test_applies_fp64(amg, tiny64, nrhs):
    c = tiny64
    y = c.fine(nrhs)
    yc = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=c.cdt, device="cuda")
    amg.amg_restrict(c.h, c.dev(y), yc, nrhs, c.stream)
    ref = coarse.restrict(c.Q, y.reshape(H.field_shape(c.L) + (4, 3, nrhs)), c.B)
    assert H.rel(yc.cpu().numpy(), ref) < 1e-12
    xc = c.coarse_vec(nrhs)
    zc = torch.empty_like(yc)
    amg.amg_coarse_apply(c.h, c.dev(xc), zc, nrhs, c.stream)
    assert H.rel(zc.cpu().numpy(), coarse.coarse_apply(c.Dc, xc, c.Lc)) < 1e-12
    x = torch.empty((c.V, 4, 3, nrhs), dtype=c.cdt, device="cuda")
    amg.amg_prolong(c.h, c.dev(xc), x, nrhs, c.stream)
    refx = coarse.prolong(c.Q, xc, c.L, c.B).reshape(c.V, 4, 3, nrhs)
    assert H.rel(x.cpu().numpy(), refx) < 1e-12
    assert amg.amg_sync_status(c.h) == amg.AMG_OK


def test_setup_ragged_matches_oracle(amg, ragged32):
    c = ragged32
    Dc = _export(amg, amg.amg_export_Dc, c.h, (c.Vc, 9, 2 * c.ntv, 2 * c.ntv))
    assert H.rel(Dc, c.Dc) < 1e-12
    R = _export(amg, amg.amg_export_R, c.h, (c.Vc, 2, c.ntv, 6 * 16))
    assert H.rel(R, H.q_to_lib_R(c.Q)) < 1e-12
    stored = _export(amg, amg.amg_export_Dc_stored, c.h, Dc.shape)
    assert H.rel(stored, Dc) < 1e-7


@pytest.mark.parametrize("nrhs", [1, 2, 5])
def test_applies_fp32_ragged(amg, ragged32, nrhs):
    c = ragged32
    y = c.fine(nrhs, 3)
    yc = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=c.cdt, device="cuda")
    amg.amg_restrict(c.h, c.dev(y), yc, nrhs, c.stream)
    ref = coarse.restrict(c.Q, y.reshape(H.field_shape(c.L) + (4, 3, nrhs)), c.B)
    assert H.rel(yc.cpu().numpy(), ref) < 1e-5
    xc = c.coarse_vec(nrhs, 5)
    zc = torch.empty_like(yc)
    amg.amg_coarse_apply(c.h, c.dev(xc), zc, nrhs, c.stream)
    assert H.rel(zc.cpu().numpy(), coarse.coarse_apply(c.Dc, xc, c.Lc)) < 1e-5
    x = torch.empty((c.V, 4, 3, nrhs), dtype=c.cdt, device="cuda")
    amg.amg_prolong(c.h, c.dev(xc), x, nrhs, c.stream)
    refx = coarse.prolong(c.Q, xc, c.L, c.B).reshape(c.V, 4, 3, nrhs)
    assert H.rel(x.cpu().numpy(), refx) < 1e-5
    # every coarse site and every fine site individually, not just in norm
    err = np.abs(zc.cpu().numpy() - coarse.coarse_apply(c.Dc, xc, c.Lc)).max()
    assert err < 1e-5 * np.abs(coarse.coarse_apply(c.Dc, xc, c.Lc)).max()


def test_fp16_scaled_within_bound(amg):
    L, B, ntv = (8, 8, 8, 8), (4, 4, 4, 4), 24
    c = Case(amg, L, B, ntv, 0.3, 7, amg.AMG_FP16_SCALED, amg.AMG_FP32, max_nrhs=16)
    try:
        stored = _export(amg, amg.amg_export_Dc_stored, c.h, (c.Vc, 9, 48, 48))
        # element-wise quantisation error: |re|, |im| each within 2^-11 relative (or subnormal step)
        scale = np.abs(np.stack([c.Dc.real, c.Dc.imag])).max(axis=(0, 3, 4)) / 2 ** 15
        tol = 2.0 ** -11 * np.maximum(np.abs(c.Dc.real), np.abs(c.Dc.imag)) + 2.0 ** -24 * scale[..., None, None]
        assert np.all(np.abs(stored.real - c.Dc.real) <= tol * 1.0001)
        assert np.all(np.abs(stored.imag - c.Dc.imag) <= tol * 1.0001)
        for nrhs in (1, 4, 8, 12, 16):  # 8 .. 16 columns take the one-pass multi-column kernel
            xc = c.coarse_vec(nrhs, 11)
            zc = torch.empty((c.Vc, 2, ntv, nrhs), dtype=torch.complex64, device="cuda")
            amg.amg_coarse_apply(c.h, c.dev(xc), zc, nrhs, c.stream)
            got = zc.cpu().numpy()
            # against the stored (dequantised) operator: only FP32 arithmetic remains
            assert H.rel(got, coarse.coarse_apply(stored, xc, c.Lc)) < 1e-5
            # against the FP64 operator: the stated bound
            bound = coarse.reduced_precision_bound(c.Dc, xc, c.Lc, 2.0 ** -11)
            err = H.rel(got, coarse.coarse_apply(c.Dc, xc, c.Lc))
            assert err <= bound, (err, bound)
    finally:
        c.close()


def test_coarse_solve_fp64_matches_oracle_fgmres(amg, tiny64):
    """A fixed number of FGMRES steps (one restart included) gives the oracle's iterate; a converged
    solve reaches the tolerance in the true residual with the oracle's number of applications."""
    c = tiny64
    b = c.coarse_vec(1, 21)
    x = torch.empty((c.Vc, 2, c.ntv, 1), dtype=c.cdt, device="cuda")
    for applies in (4, 9):
        info = amg.amg_coarse_solve(c.h, c.dev(b), x, 1, tol=1e-12, restart=6, max_applies=applies,
                                    stream=c.stream)
        ref, hist, n = krylov.fgmres(lambda v: coarse.coarse_apply(c.Dc, v, c.Lc), b, tol=1e-12, restart=6,
                                     max_applies=applies)
        assert info[0][0] == n == applies
        assert abs(info[0][1] - hist[-1]) <= 1e-9 * hist[-1]
        assert H.rel(x.cpu().numpy(), ref) < 1e-10
    info = amg.amg_coarse_solve(c.h, c.dev(b), x, 1, tol=1e-9, restart=6, max_applies=400, stream=c.stream)
    ref, hist, n = krylov.fgmres(lambda v: coarse.coarse_apply(c.Dc, v, c.Lc), b, tol=1e-9, restart=6,
                                 max_applies=400)
    assert abs(info[0][0] - n) <= 2 and info[0][1] <= 1e-9
    true = H.rel(coarse.coarse_apply(c.Dc, x.cpu().numpy(), c.Lc), b)
    assert true <= 1.05e-9


def test_arnoldi_bounded_barrier_reports_timeout(amg, tiny64):
    """The fused Arnoldi step's grid barrier expects one more arrival than there are CTAs: every
    CTA's wait runs out (about one second), the step ends early, the status says so once, and the
    handle and the context stay usable (the next solve gives the oracle's iterate)."""
    c = tiny64
    b = c.coarse_vec(1, 23)
    x = torch.empty((c.Vc, 2, c.ntv, 1), dtype=c.cdt, device="cuda")
    amg.amg_solve_test_hook(c.h, 1)
    try:
        amg.amg_coarse_solve(c.h, c.dev(b), x, 1, tol=0.0, restart=4, max_applies=1, stream=c.stream, info=False)
        assert amg.amg_sync_status(c.h) == amg.AMG_ERR_TIMEOUT
    finally:
        amg.amg_solve_test_hook(c.h, 0)
    info = amg.amg_coarse_solve(c.h, c.dev(b), x, 1, tol=1e-12, restart=6, max_applies=4, stream=c.stream)
    ref, hist, n = krylov.fgmres(lambda v: coarse.coarse_apply(c.Dc, v, c.Lc), b, tol=1e-12, restart=6,
                                 max_applies=4)
    assert info[0][0] == n == 4
    assert H.rel(x.cpu().numpy(), ref) < 1e-10
    assert amg.amg_sync_status(c.h) == amg.AMG_OK
    a = torch.ones(1000, device="cuda")
    assert float(a.sum()) == 1000.0
    with pytest.raises(amg.AmgError):
        amg.amg_solve_test_hook(c.h, -1)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_coarse_solve_fp32_reaches_tolerance(amg, ragged32, nrhs):
    c = ragged32
    b = c.coarse_vec(nrhs, 31)
    x = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=c.cdt, device="cuda")
    info = amg.amg_coarse_solve(c.h, c.dev(b), x, nrhs, tol=1e-4, restart=10, max_applies=300, stream=c.stream)
    xs = x.cpu().numpy().astype(np.complex128)
    for r in range(nrhs):
        ref, hist, n = krylov.fgmres(lambda v: coarse.coarse_apply(c.Dc, v, c.Lc), b[..., r], tol=1e-4,
                                     restart=10, max_applies=300)
        assert abs(info[r][0] - n) <= 2
        true = H.rel(coarse.coarse_apply(c.Dc, xs[..., r], c.Lc), b[..., r])
        assert true <= 1e-4 * 1.05
        assert H.rel(xs[..., r], ref) < 1e-3


def test_cgc_composition(amg, ragged32):
    c = ragged32
    y = c.fine(2, 41)
    x = torch.empty((c.V, 4, 3, 2), dtype=c.cdt, device="cuda")
    info = amg.amg_cgc(c.h, c.dev(y), x, 2, tol=1e-5, restart=12, max_applies=400, stream=c.stream)
    assert all(i[1] <= 1e-5 for i in info)
    yc = coarse.restrict(c.Q, y.reshape(H.field_shape(c.L) + (4, 3, 2)), c.B)
    xg = x.cpu().numpy().astype(np.complex128).reshape(H.field_shape(c.L) + (4, 3, 2))
    # R x = x_c solves D_c x_c = R y to the tolerance (R P = I)
    xc = coarse.restrict(c.Q, xg, c.B)
    for r in range(2):
        assert H.rel(coarse.coarse_apply(c.Dc, xc[..., r], c.Lc), yc[..., r]) < 1.2e-5


@pytest.mark.parametrize("arith", [0, 1], ids=["fp64", "f32pair"])
def test_rank_deficient_test_vectors_reported(amg, arith):
    L, B, ntv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    sites = si.all_sites(L)
    U = torch.from_numpy(si.links(5, 0.3, sites)).cuda()
    tvh = si.test_vectors(5, ntv, sites)
    tvh[..., 3] = tvh[..., 0] * (1 - 2j) + tvh[..., 1]
    p = amg.make_params(L, B, ntv, 1, H.M0, H.CSW, amg.AMG_FP64, amg.AMG_FP64, amg.AMG_FP64, setup_arith=arith)
    h, st = amg.amg_setup_coarse(p, U, torch.from_numpy(tvh).cuda(), torch.cuda.current_stream(),
                                 allow_rank_deficient=True)
    assert st == amg.AMG_ERR_RANK_DEFICIENT
    amg.amg_destroy(h)


def test_invalid_calls_rejected(amg, tiny64):
    c = tiny64
    a = torch.empty((c.Vc, 2, c.ntv, 1), dtype=c.cdt, device="cuda")
    with pytest.raises(amg.AmgError) as e:
        amg.amg_coarse_apply(c.h, a, a, 1)
    assert e.value.status == amg.AMG_ERR_INVALID_ARG
    with pytest.raises(amg.AmgError):
        amg.amg_coarse_apply(c.h, a, a.data_ptr() + 8, 1)
    with pytest.raises(amg.AmgError):
        amg.amg_restrict(c.h, a, a, 9)
