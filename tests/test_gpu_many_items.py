"""Whole-array parity when every CTA of a persistent grid-stride kernel runs many items.

The bulk-copy and tensor-core kernels walk the coarse sites (or blocks) with a stride of the
grid, carrying their copy ring's stage and phase from one item to the next, and the fused batch
hands out jobs from a queue.  On the full-size lattices each CTA runs several to tens of items.
Here amg_grid_cap_test_hook lowers the grid to a few CTAs on lattices the oracle computes whole,
so that each CTA runs 6-60 items and its ring wraps many times, and every output element is
compared with the oracle (Alg. 2: y_c = R y, D_c x_c, x = P x_c):

* FP64: relative L2 1e-12; FP32: 1e-5 and every element within 1e-5 of the largest;
* BF16 (tensor cores): every element within its own bound
  (u_store + u_in + 4 (K + 2) u_fp32) (|A| |x|)_e, the FP32 term counting the real products of
  a complex sum of K terms, and relative L2 1e-5 against the oracle applied to the stored
  operator and the rounded input;
* the capped grid gives bit for bit the uncapped result (each item's arithmetic does not depend
  on which CTA runs it).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coarse, dirac, evenodd as eo, lattice as lat  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu

CAP = 5  # CTAs: does not divide the item counts, so CTAs run uneven numbers of items


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


class Lattice:
    """Inputs and oracle results (Q, D_c) for one small lattice, and library handles on it."""

    def __init__(self, amg, L, B, ntv, seed, eps=0.3):
        self.amg, self.L, self.B, self.ntv, self.seed = amg, L, B, ntv, seed
        self.Lc = lat.coarse_dims(L, B)
        self.Vc = int(np.prod(self.Lc))
        self.V = int(np.prod(L))
        self.nc = 2 * ntv
        sites = si.all_sites(L)
        self.Uh = si.links(seed, eps, sites)
        self.tvh = si.test_vectors(seed, ntv, sites)
        U = np.moveaxis(self.Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
        self.Q = coarse.orthonormalize(self.tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
        self.Dc = coarse.coarse_operator(U, dirac.clover_field(U, H.CSW), H.M0, self.Q, L, B)
        self.stream = torch.cuda.current_stream()
        self.handles = []

    def handle(self, link, r, vec, max_nrhs=16):
        p = self.amg.make_params(self.L, self.B, self.ntv, max_nrhs, H.M0, H.CSW, link, r, vec)
        h, _ = self.amg.amg_setup_coarse(p, torch.from_numpy(self.Uh).cuda(), torch.from_numpy(self.tvh).cuda(),
                                         self.stream)
        self.handles.append(h)
        return h

    def close(self):
        for h in self.handles:
            self.amg.amg_destroy(h)

    def fine(self, nrhs, off):
        return si.fine_rhs(self.seed + off, nrhs, si.all_sites(self.L))

    def coarse_vec(self, nrhs, off):
        return si.coarse_vector(self.seed + off, self.ntv, nrhs, np.arange(self.Vc))


def _both(amg, h, fn):
    """fn() with the grid capped at CAP CTAs, then with the full grid; returns both results."""
    amg.amg_grid_cap_test_hook(h, CAP)
    try:
        capped = fn()
    finally:
        amg.amg_grid_cap_test_hook(h, 0)
    full = fn()
    torch.cuda.synchronize()
    assert amg.amg_sync_status(h) == amg.AMG_OK
    return capped, full


def _to_bf16_dev(z):
    f = torch.from_numpy(np.ascontiguousarray(np.stack([z.real, z.imag], -1)).astype(np.float32))
    return f.to(torch.bfloat16).cuda()


def _from_bf16_dev(t):
    f = t.float().cpu().numpy().astype(np.float64)
    return f[..., 0] + 1j * f[..., 1]


# 8^4 with 2^4 blocks: 256 coarse sites / blocks of two 8-site chunks (about 51 items per CTA);
# 16 x 8 x 8 x 8 with 4^4 blocks: 32 blocks of 32 chunks (6 or 7 blocks per CTA, 200+ chunks)
@pytest.fixture(scope="module", params=[((8, 8, 8, 8), (2, 2, 2, 2), 24), ((16, 8, 8, 8), (4, 4, 4, 4), 24),
                                        ((8, 8, 8, 8), (2, 2, 2, 2), 20)],
                ids=["8^4_b2_ntv24", "16x8^3_b4_ntv24", "8^4_b2_ntv20"])
def bf16(amg, request):
    L, B, ntv = request.param
    c = Lattice(amg, L, B, ntv, 911)
    c.h = c.handle(amg.AMG_BF16, amg.AMG_BF16, amg.AMG_BF16)
    st = torch.empty((c.Vc, 9, c.nc, c.nc), dtype=torch.complex128, device="cuda")
    amg.amg_export_Dc_stored(c.h, st)
    c.stored = st.cpu().numpy()
    del st
    yield c
    c.close()


@pytest.mark.parametrize("nrhs", [4, 16])
def test_bf16_apply_every_site(amg, bf16, nrhs):
    c = bf16
    x32 = c.coarse_vec(nrhs, 1).astype(np.complex64)
    xd = torch.from_numpy(x32).cuda()

    def run():
        y = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=torch.complex64, device="cuda")
        amg.amg_coarse_apply(c.h, xd, y, nrhs, c.stream)
        return y

    capped, full = _both(amg, c.h, run)
    assert torch.equal(capped, full)
    got = capped.cpu().numpy().astype(np.complex128)
    x64 = x32.astype(np.complex128)
    assert H.rel(got, coarse.coarse_apply(c.stored, H.bf16_round(x64), c.Lc)) < 1e-5
    ref = coarse.coarse_apply(c.Dc, x64, c.Lc)
    absref = coarse.abs_apply(c.Dc, x64, c.Lc)
    K = 9 * c.nc
    assert H.worst_ratio(got, ref, absref, 2 * H.U_BF16 + 4 * (K + 2) * H.U_FP32) <= 1.0


@pytest.mark.parametrize("nrhs", [4, 16])
def test_bf16_restrict_prolong_every_block(amg, bf16, nrhs):
    c = bf16
    y = H.bf16_round(c.fine(nrhs, 2))  # BF16-valued fine vectors: the library and the oracle see the same values
    yd = _to_bf16_dev(y)

    def run_r():
        yc = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=torch.complex64, device="cuda")
        amg.amg_restrict(c.h, yd, yc, nrhs, c.stream)
        return yc

    capped, full = _both(amg, c.h, run_r)
    assert torch.equal(capped, full)
    got = capped.cpu().numpy().astype(np.complex128)
    yf = y.reshape(H.field_shape(c.L) + (4, 3, nrhs))
    ref = coarse.restrict(c.Q, yf, c.B)
    absref = coarse.restrict(np.abs(c.Q).astype(np.complex128), np.abs(yf).astype(np.complex128), c.B).real
    K = 6 * int(np.prod(c.B))
    assert H.worst_ratio(got, ref, absref, H.U_BF16 + 4 * (K + 2) * H.U_FP32) <= 1.0
    assert H.rel(got, ref) < 4e-3

    xc = c.coarse_vec(nrhs, 3).astype(np.complex64)
    xd = torch.from_numpy(xc).cuda()

    def run_p():
        x = torch.empty((c.V, 4, 3, nrhs, 2), dtype=torch.bfloat16, device="cuda")
        amg.amg_prolong(c.h, xd, x, nrhs, c.stream)
        return x

    capped, full = _both(amg, c.h, run_p)
    assert torch.equal(capped, full)
    gotx = _from_bf16_dev(capped)
    xc64 = xc.astype(np.complex128)
    refx = coarse.prolong(c.Q, xc64, c.L, c.B).reshape(c.V, 4, 3, nrhs)
    absx = coarse.prolong(np.abs(c.Q).astype(np.complex128), np.abs(xc64).astype(np.complex128),
                          c.L, c.B).reshape(c.V, 4, 3, nrhs).real
    assert H.worst_ratio(gotx, refx, absx, 3 * H.U_BF16 + 4 * (c.ntv + 2) * H.U_FP32) <= 1.0


@pytest.fixture(scope="module")
def small32(amg):
    """8^4, 2^4 blocks, Ntv = 24: FP32 (split-TF32 tensor cores for 4-16 columns, one-pass SIMT for
    1-3), FP16 with block scales (one-pass SIMT), FP64 (bulk-copy apply and prolongation)."""
    c = Lattice(amg, (8, 8, 8, 8), (2, 2, 2, 2), 24, 912)
    c.h32 = c.handle(amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32)
    c.h16 = c.handle(amg.AMG_FP16_SCALED, amg.AMG_FP32, amg.AMG_FP32)
    c.h64 = c.handle(amg.AMG_FP64, amg.AMG_FP64, amg.AMG_FP64, max_nrhs=4)
    yield c
    c.close()


def _apply(amg, c, h, x, nrhs, dtype):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()

    def run():
        y = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=dtype, device="cuda")
        amg.amg_coarse_apply(h, xd, y, nrhs, c.stream)
        return y

    capped, full = _both(amg, h, run)
    assert torch.equal(capped, full)
    return capped.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("nrhs", [1, 3, 4, 16])
def test_fp32_apply_every_site(amg, small32, nrhs):
    c = small32
    x = c.coarse_vec(nrhs, 4).astype(np.complex64)
    got = _apply(amg, c, c.h32, x, nrhs, torch.complex64)
    ref = coarse.coarse_apply(c.Dc, x.astype(np.complex128), c.Lc)
    assert H.rel(got, ref) < 1e-5
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("nrhs", [1, 4, 16])
def test_fp16_apply_every_site(amg, small32, nrhs):
    c = small32
    x = c.coarse_vec(nrhs, 5).astype(np.complex64)
    got = _apply(amg, c, c.h16, x, nrhs, torch.complex64)
    x64 = x.astype(np.complex128)
    ref = coarse.coarse_apply(c.Dc, x64, c.Lc)
    # the stored value's error is <= 2^-11 of the larger of |Re|, |Im| (<= 2^-11 |D|) or, below the
    # normal range, one subnormal step of the block's scale (2^-24 s <= 2^-39 max|D| per entry)
    absref = coarse.abs_apply(c.Dc, x64, c.Lc)
    K = 9 * c.nc
    floor = 2.0 ** -39 * np.abs(c.Dc).max() * K * np.abs(x64).max()
    assert H.worst_ratio(got, ref, absref, H.U_FP16 + 4 * (K + 2) * H.U_FP32, floor) <= 1.0


@pytest.mark.parametrize("nrhs", [1, 3])
def test_fp64_apply_prolong_every_site(amg, small32, nrhs):
    c = small32
    x = c.coarse_vec(nrhs, 6)
    got = _apply(amg, c, c.h64, x, nrhs, torch.complex128)
    assert H.rel(got, coarse.coarse_apply(c.Dc, x, c.Lc)) < 1e-12
    xd = torch.from_numpy(x).cuda()

    def run():
        out = torch.empty((c.V, 4, 3, nrhs), dtype=torch.complex128, device="cuda")
        amg.amg_prolong(c.h64, xd, out, nrhs, c.stream)
        return out

    capped, full = _both(amg, c.h64, run)
    assert torch.equal(capped, full)
    ref = coarse.prolong(c.Q, x, c.L, c.B).reshape(c.V, 4, 3, nrhs)
    assert H.rel(capped.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("nrhs", [1, 4])
def test_fp32_schur_apply_every_site(amg, nrhs):
    """The even/odd passes (one-pass kernel for FP32) over 128 sites of one parity on 5 CTAs."""
    c = Lattice(amg, (8, 8, 8, 8), (2, 2, 2, 2), 12, 913)
    try:
        h = c.handle(amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32, max_nrhs=4)
        amg.amg_setup_evenodd(h, c.stream)
        xe = si.coarse_vector(914 + nrhs, c.ntv, nrhs, np.arange(c.Vc // 2)).reshape(c.Vc // 2, c.nc, nrhs)
        xe = xe.astype(np.complex64)
        xd = torch.from_numpy(xe).cuda()

        def run():
            ye = torch.empty((c.Vc // 2, c.nc, nrhs), dtype=torch.complex64, device="cuda")
            amg.amg_schur_apply(h, xd, ye, nrhs, c.stream)
            return ye

        capped, full = _both(amg, h, run)
        assert torch.equal(capped, full)
        got = capped.cpu().numpy().astype(np.complex128)
        want = eo.schur_apply(c.Dc, xe.astype(np.complex128), c.Lc)
        assert H.rel(got, want) < 1e-5
        assert np.abs(got - want).max() < 1e-5 * np.abs(want).max()
    finally:
        c.close()


# Fused batch: an FP32 lattice with one right-hand side and two BF16 tensor-core lattices; with
# the grid capped, three CTAs take all jobs of all phases from the queue in order.
BATCH = [((8, 8, 8, 8), (2, 2, 2, 2), 8, 0.2, 1, "fp32"),
         ((8, 8, 8, 8), (2, 2, 2, 2), 20, 0.3, 4, "bf16"),
         ((16, 8, 8, 8), (4, 4, 4, 4), 24, 0.4, 12, "bf16")]


def test_batch_few_ctas_every_site(amg):
    lats = []
    try:
        for k, (L, B, ntv, eps, nrhs, prec) in enumerate(BATCH):
            c = Lattice(amg, L, B, ntv, 920 + k, eps)
            pr = amg.AMG_FP32 if prec == "fp32" else amg.AMG_BF16
            c.h = c.handle(pr, pr, pr, max_nrhs=max(nrhs, 4))
            c.nrhs, c.prec = nrhs, prec
            y = c.fine(nrhs, 50)
            if prec == "fp32":
                y = y.astype(np.complex64)
                c.y = torch.from_numpy(y).cuda()
                c.yv = y.astype(np.complex128)
            else:
                c.y = _to_bf16_dev(y)
                c.yv = _from_bf16_dev(c.y)
            lats.append(c)
        hs = [c.h for c in lats]

        def run():
            xs = [torch.empty(c.y.shape, dtype=c.y.dtype, device="cuda") for c in lats]
            amg.amg_batch_cgc(hs, [c.y for c in lats], xs, [c.nrhs for c in lats], torch.cuda.current_stream())
            return xs

        amg.amg_grid_cap_test_hook(hs[0], 3)
        try:
            capped = run()
        finally:
            amg.amg_grid_cap_test_hook(hs[0], 0)
        full = run()
        torch.cuda.synchronize()
        assert amg.amg_sync_status(hs[0]) == amg.AMG_OK
        for c, a, b in zip(lats, capped, full):
            assert torch.equal(a, b)
            yf = c.yv.reshape(H.field_shape(c.L) + (4, 3, c.nrhs))
            ref = coarse.prolong(c.Q, coarse.coarse_apply(c.Dc, coarse.restrict(c.Q, yf, c.B), c.Lc), c.L, c.B)
            ref = ref.reshape(c.yv.shape)
            if c.prec == "fp32":
                got = a.cpu().numpy().astype(np.complex128)
                assert H.rel(got, ref) < 1e-5
                assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()
            else:
                got = _from_bf16_dev(a)
                aQ, aD = np.abs(c.Q).astype(np.complex128), np.abs(c.Dc).astype(np.complex128)
                absref = coarse.prolong(aQ, coarse.coarse_apply(
                    aD, coarse.restrict(aQ, np.abs(yf).astype(np.complex128), c.B), c.Lc), c.L, c.B)
                absref = absref.reshape(c.yv.shape).real
                # six BF16 roundings (R, y_c, D_c, D_c y_c, R again, x) and the FP32 sums
                K = 6 * int(np.prod(c.B)) + 9 * c.nc + c.ntv
                assert H.worst_ratio(got, ref, absref, 6 * H.U_BF16 + 4 * (K + 6) * H.U_FP32) <= 1.0
    finally:
        for c in lats:
            c.close()
