"""GPU parity at the full sizes of the mixed-precision, tensor-core and batch workloads.

* FP16 D_c with per-block scales: 32^3 x 64, 4^4 blocks (8^3 x 16 coarse sites), Ntv = 24;
* BF16 tensor cores: 48^3 x 96, 4^4 blocks (12^3 x 24 coarse sites), Ntv = 24, 16 right-hand sides;
* the uneven batch in one persistent launch: 16^4 (Ntv 16, 1 RHS, FP32), 24^3 x 48 (Ntv 20,
  4 RHS, BF16), 32^3 x 64 (Ntv 24, 12 RHS, BF16), 4^4 blocks, eps 0.2 / 0.3 / 0.4.

Inputs are generated on the device (synth.device).  For 8 sampled blocks per lattice the oracle
regenerates the inputs of the 3x3x3x3-block box around the block on the host (same counter-based
generator) and computes the block's R rows, its D_c row and its neighbours' R rows; the library's
outputs on those blocks are compared element by element.  The samples are the first and last
blocks and blocks spread over the whole range: the persistent kernels run at most
(resident CTAs per SM) x SMs ~ 450-900 CTAs over 8,192-41,472 items, so all but the first sample
fall in the second or later pass of a CTA's loop.  The box computations run in a process pool
(started with 'spawn', before any GPU work of this module) while the GPU work runs.

Bounds, element by element: (sum of the unit roundoffs of every rounding on the path, with
4 (K + 2) u_fp32 for FP32 sums of K complex terms) x (the same product of absolute values).
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lattice as lat  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

# a stalled oracle pool or launch fails its test instead of holding the GPU (pytest-timeout)
pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

B4 = (4, 4, 4, 4)
FP16_CASE = ((32, 32, 32, 64), 24, 0.3, si.SEED_BASE + 3)
TC16_CASE = ((48, 48, 48, 96), 24, 0.3, si.SEED_BASE + 4)
BATCH_CASE = [((16, 16, 16, 16), 16, 1, 0.2, "fp32"), ((24, 24, 24, 48), 20, 4, 0.3, "bf16"),
              ((32, 32, 32, 64), 24, 12, 0.4, "bf16")]


def _batch_seed(k):
    return si.SEED_BASE + 5 + 10 * k


def sample_sites(Vc):
    """8 coarse sites: the first, the last and six spread over the range."""
    s = [0, 1 + Vc // 7, Vc // 3, Vc // 2 + 1, (2 * Vc) // 3 + 5, (5 * Vc) // 6, Vc - 2, Vc - 1]
    return sorted(set(int(v) for v in s))


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


@pytest.fixture(scope="module")
def patches():
    """Every oracle box of this module, submitted at once to a spawn-started process pool."""
    jobs = []
    L, ntv, eps, seed = FP16_CASE
    jobs += [("fp16", i, (seed, eps, L, ntv)) for i in sample_sites(int(np.prod(lat.coarse_dims(L, B4))))]
    L, ntv, eps, seed = TC16_CASE
    jobs += [("tc16", i, (seed, eps, L, ntv)) for i in sample_sites(int(np.prod(lat.coarse_dims(L, B4))))]
    for k, (L, ntv, _, eps, _) in enumerate(BATCH_CASE):
        jobs += [("batch%d" % k, i, (_batch_seed(k), eps, L, ntv))
                 for i in sample_sites(int(np.prod(lat.coarse_dims(L, B4))))]
    workers = max(1, min(12, (os.cpu_count() or 2) - 2))
    # one BLAS / OpenMP thread per worker: the workers already fill the cores, and numpy's own
    # threads on top of them (workers x cores threads) made the boxes about 8 times slower
    saved = {k: os.environ.get(k) for k in THREAD_VARS}
    os.environ.update({k: "1" for k in THREAD_VARS})
    try:
        ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
        fut = {}
        for name, i, (seed, eps, L, ntv) in jobs:
            X = H.coarse_coords(lat.coarse_dims(L, B4), i)
            fut[(name, i)] = ex.submit(H.patch_neighbourhood, seed, eps, L, B4, ntv, X)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    yield lambda name, i: fut[(name, i)].result()
    ex.shutdown(cancel_futures=True)


def _nbr_sites(L, i):
    return lat.coarse_neighbours(lat.coarse_dims(L, B4))[i]


def _bf16_dev(t32):
    return torch.view_as_real(t32).to(torch.bfloat16)


def _from_bf16(t):
    f = t.float().cpu().numpy().astype(np.float64)
    return f[..., 0] + 1j * f[..., 1]


# ------------------------------------------------------------------ BF16 tensor cores, 48^3 x 96
def test_tc16_full_size_sampled(amg, patches):
    from synth import device as sd
    L, ntv, eps, seed = TC16_CASE
    nrhs, nc = 16, 2 * ntv
    Lc = lat.coarse_dims(L, B4)
    Vc = int(np.prod(Lc))
    st = torch.cuda.current_stream()
    U = sd.links(seed, eps, L)
    tv = sd.test_vectors(seed, ntv, L)
    p = amg.make_params(L, B4, ntv, nrhs, H.M0, H.CSW, amg.AMG_BF16, amg.AMG_BF16, amg.AMG_BF16)
    h, _ = amg.amg_setup_coarse(p, U, tv, st)
    del U, tv
    torch.cuda.empty_cache()
    try:
        y32 = sd.fine_rhs(seed, nrhs, L, torch.complex64)
        y = _bf16_dev(y32)
        del y32
        yc = torch.empty((Vc, 2, ntv, nrhs), dtype=torch.complex64, device="cuda")
        amg.amg_restrict(h, y, yc, nrhs, st)
        del y
        xc = sd.coarse_vector(seed + 1, ntv, nrhs, Vc, torch.complex64)
        zc = torch.empty_like(xc)
        amg.amg_coarse_apply(h, xc, zc, nrhs, st)
        x = torch.empty((int(np.prod(L)), 4, 3, nrhs, 2), dtype=torch.bfloat16, device="cuda")
        amg.amg_prolong(h, xc, x, nrhs, st)
        torch.cuda.empty_cache()
        Dc = torch.empty((Vc, 9, nc, nc), dtype=torch.complex128, device="cuda")
        amg.amg_export_Dc(h, Dc)
        torch.cuda.synchronize()
        assert amg.amg_sync_status(h) == amg.AMG_OK
        K_r, K_a, K_p = 6 * 256, 9 * nc, ntv
        for i in sample_sites(Vc):
            Qn, Dref = patches("tc16", i)
            Qi = Qn[0]
            assert H.rel(Dc[i].cpu().numpy(), Dref) < 1e-12
            X = H.coarse_coords(Lc, i)
            bs = H.block_sites(L, B4, X)
            # restriction of the 16 BF16 right-hand sides on block i
            yb = H.bf16_round(si.fine_rhs(seed, nrhs, bs).astype(np.complex64).astype(np.complex128))
            ya = H.to_aggregates_block(yb)                                        # (2, n, k)
            ref = np.einsum("hnj,hnk->hjk", Qi.conj(), ya)
            absref = np.einsum("hnj,hnk->hjk", np.abs(Qi), np.abs(ya))
            got = yc[i].cpu().numpy().astype(np.complex128)
            assert H.worst_ratio(got, ref, absref, H.U_BF16 + 4 * (K_r + 2) * H.U_FP32) <= 1.0, i
            # coarse apply at site i (FP32 input rounded to BF16 inside)
            xh = si.coarse_vector(seed + 1, ntv, nrhs, _nbr_sites(L, i)).astype(np.complex64)
            xh = xh.astype(np.complex128).reshape(9, nc, nrhs)
            refz = sum(Dref[d] @ xh[d] for d in range(9))
            absz = sum(np.abs(Dref[d]) @ np.abs(xh[d]) for d in range(9))
            gotz = zc[i].reshape(nc, nrhs).cpu().numpy().astype(np.complex128)
            assert H.worst_ratio(gotz, refz, absz, 2 * H.U_BF16 + 4 * (K_a + 2) * H.U_FP32) <= 1.0, i
            # prolongation onto block i (x_c rounded to BF16, the output rounded to BF16)
            xci = xh[0].reshape(2, ntv, nrhs)
            refx = H.from_aggregates_block(np.einsum("hnj,hjk->hnk", Qi, xci))
            absx = H.from_aggregates_block(np.einsum("hnj,hjk->hnk", np.abs(Qi), np.abs(xci)))
            gotx = _from_bf16(x[torch.from_numpy(bs).cuda()])
            assert H.worst_ratio(gotx, refx, absx, 3 * H.U_BF16 + 4 * (K_p + 2) * H.U_FP32) <= 1.0, i
    finally:
        amg.amg_destroy(h)
        torch.cuda.empty_cache()


# ------------------------------------------------------------------ FP16 D_c, 32^3 x 64
def test_fp16_full_size_sampled(amg, patches):
    from synth import device as sd
    L, ntv, eps, seed = FP16_CASE
    nc = 2 * ntv
    Lc = lat.coarse_dims(L, B4)
    Vc = int(np.prod(Lc))
    st = torch.cuda.current_stream()
    U = sd.links(seed, eps, L)
    tv = sd.test_vectors(seed, ntv, L)
    p = amg.make_params(L, B4, ntv, 16, H.M0, H.CSW, amg.AMG_FP16_SCALED, amg.AMG_FP32, amg.AMG_FP32)
    h, _ = amg.amg_setup_coarse(p, U, tv, st)
    del U, tv
    torch.cuda.empty_cache()
    try:
        Dc = torch.empty((Vc, 9, nc, nc), dtype=torch.complex128, device="cuda")
        amg.amg_export_Dc(h, Dc)
        Ds = torch.empty_like(Dc)
        amg.amg_export_Dc_stored(h, Ds)
        R = torch.empty((Vc, 2, ntv, 6 * 256), dtype=torch.complex128, device="cuda")
        amg.amg_export_R(h, R)
        y = sd.fine_rhs(seed, 1, L, torch.complex64)
        yc = torch.empty((Vc, 2, ntv, 1), dtype=torch.complex64, device="cuda")
        amg.amg_restrict(h, y, yc, 1, st)
        out = {}
        for nrhs in (1, 4, 16):
            xc = sd.coarse_vector(seed + nrhs, ntv, nrhs, Vc, torch.complex64)
            zc = torch.empty_like(xc)
            amg.amg_coarse_apply(h, xc, zc, nrhs, st)
            out[nrhs] = zc
        xc1 = sd.coarse_vector(seed + 1, ntv, 1, Vc, torch.complex64)
        x = torch.empty_like(y)
        amg.amg_prolong(h, xc1, x, 1, st)
        torch.cuda.synchronize()
        assert amg.amg_sync_status(h) == amg.AMG_OK
        K = 9 * nc
        for i in sample_sites(Vc):
            Qn, Dref = patches("fp16", i)
            Qi = Qn[0]
            assert H.rel(Dc[i].cpu().numpy(), Dref) < 1e-12
            assert H.rel(R[i].cpu().numpy(), H.q_to_lib_R(Qi)) < 1e-12
            # stored FP16 entries: within 2^-11 of each part, or one subnormal step of the block scale
            st_i = Ds[i].cpu().numpy()
            scale = np.abs(np.stack([Dref.real, Dref.imag])).max(axis=(0, 2, 3)) / 2 ** 15
            tol = H.U_FP16 * np.maximum(np.abs(Dref.real), np.abs(Dref.imag)) + 2.0 ** -24 * scale[:, None, None]
            assert np.all(np.abs(st_i.real - Dref.real) <= tol * 1.0001), i
            assert np.all(np.abs(st_i.imag - Dref.imag) <= tol * 1.0001), i
            X = H.coarse_coords(Lc, i)
            bs = H.block_sites(L, B4, X)
            yb = si.fine_rhs(seed, 1, bs).astype(np.complex64).astype(np.complex128)
            ref = np.einsum("hnj,hnk->hjk", Qi.conj(), H.to_aggregates_block(yb))
            got = yc[i].cpu().numpy().astype(np.complex128)
            assert H.rel(got, ref) < 1e-5 and np.abs(got - ref).max() < 1e-5 * np.abs(ref).max(), i
            for nrhs, zc in out.items():
                xh = si.coarse_vector(seed + nrhs, ntv, nrhs, _nbr_sites(L, i)).astype(np.complex64)
                xh = xh.astype(np.complex128).reshape(9, nc, nrhs)
                refz = sum(Dref[d] @ xh[d] for d in range(9))
                absz = sum(np.abs(Dref[d]) @ np.abs(xh[d]) for d in range(9))
                floor = 2.0 ** -39 * np.abs(Dref).max() * K * np.abs(xh).max()
                gotz = zc[i].reshape(nc, nrhs).cpu().numpy().astype(np.complex128)
                assert H.worst_ratio(gotz, refz, absz, H.U_FP16 + 4 * (K + 2) * H.U_FP32, floor) <= 1.0, (i, nrhs)
            xci = si.coarse_vector(seed + 1, ntv, 1, [i]).astype(np.complex64).astype(np.complex128)[0]
            refx = H.from_aggregates_block(np.einsum("hnj,hjk->hnk", Qi, xci))
            gotx = x[torch.from_numpy(bs).cuda()].cpu().numpy().astype(np.complex128)
            assert H.rel(gotx, refx) < 1e-5 and np.abs(gotx - refx).max() < 1e-5 * np.abs(refx).max(), i
    finally:
        amg.amg_destroy(h)
        torch.cuda.empty_cache()


# ------------------------------------------------------------------ the uneven batch at full size
def test_batch_full_size_sampled(amg, patches):
    from synth import device as sd
    st = torch.cuda.current_stream()
    hs, ys, xs, nr = [], [], [], []
    try:
        for k, (L, ntv, nrhs, eps, prec) in enumerate(BATCH_CASE):
            seed = _batch_seed(k)
            U = sd.links(seed, eps, L)
            tv = sd.test_vectors(seed, ntv, L)
            pr = amg.AMG_BF16 if prec == "bf16" else amg.AMG_FP32
            h, _ = amg.amg_setup_coarse(amg.make_params(L, B4, ntv, nrhs, H.M0, H.CSW, pr, pr, pr), U, tv, st)
            hs.append(h)
            del U, tv
            y = sd.fine_rhs(seed, nrhs, L, torch.complex64)
            if prec == "bf16":
                y = _bf16_dev(y)
            ys.append(y)
            xs.append(torch.empty_like(y))
            nr.append(nrhs)
        torch.cuda.empty_cache()
        amg.amg_batch_cgc(hs, ys, xs, nr, st)
        torch.cuda.synchronize()
        assert amg.amg_sync_status(hs[0]) == amg.AMG_OK
        for k, (L, ntv, nrhs, eps, prec) in enumerate(BATCH_CASE):
            seed = _batch_seed(k)
            nc = 2 * ntv
            Lc = lat.coarse_dims(L, B4)
            Vc = int(np.prod(Lc))
            for i in sample_sites(Vc):
                Qn, Dref = patches("batch%d" % k, i)
                nb = _nbr_sites(L, i)
                z = np.zeros((nc, nrhs), dtype=np.complex128)
                az = np.zeros((nc, nrhs))
                for d in range(9):
                    bs = H.block_sites(L, B4, H.coarse_coords(Lc, int(nb[d])))
                    yb = si.fine_rhs(seed, nrhs, bs).astype(np.complex64).astype(np.complex128)
                    if prec == "bf16":
                        yb = H.bf16_round(yb)
                    ya = H.to_aggregates_block(yb)
                    ycd = np.einsum("hnj,hnk->hjk", Qn[d].conj(), ya).reshape(nc, nrhs)
                    acd = np.einsum("hnj,hnk->hjk", np.abs(Qn[d]), np.abs(ya)).reshape(nc, nrhs)
                    z += Dref[d] @ ycd
                    az += np.abs(Dref[d]) @ acd
                refx = H.from_aggregates_block(np.einsum("hnj,hjk->hnk", Qn[0], z.reshape(2, ntv, nrhs)))
                absx = H.from_aggregates_block(np.einsum("hnj,hjk->hnk", np.abs(Qn[0]), az.reshape(2, ntv, nrhs)))
                bs = torch.from_numpy(H.block_sites(L, B4, H.coarse_coords(Lc, i))).cuda()
                if prec == "fp32":
                    got = xs[k][bs].cpu().numpy().astype(np.complex128)
                    assert H.rel(got, refx) < 1e-5 and np.abs(got - refx).max() < 1e-5 * np.abs(refx).max(), (k, i)
                else:
                    got = _from_bf16(xs[k][bs])
                    Ksum = 6 * 256 + 9 * nc + ntv
                    assert H.worst_ratio(got, refx, absx, 6 * H.U_BF16 + 4 * (Ksum + 6) * H.U_FP32) <= 1.0, (k, i)
    finally:
        for h in hs:
            amg.amg_destroy(h)
        torch.cuda.empty_cache()
