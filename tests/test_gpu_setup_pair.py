"""GPU parity of the setup in pairs of FP32 numbers (setup_arith = AMG_SETUP_F32PAIR: the
Gram-Schmidt and the D_c assembly).

Every case runs the setup twice on the same inputs, once per arithmetic, and checks the pair
results (R and D_c) against the FP64 oracle (1e-12 relative L2, per stencil direction for D_c:
the FP64 setup's bar) and against the library's own FP64 setup (1e-13: the two differ by the
pairs' 47-bit rounding).  The cases cover both tilings (2x2 tiles up to nc = 44, 2x4 beyond),
the widest of each, padded tile columns, an odd Ntv (tiles across the chirality boundary, which
the self job's quadrant skip must not drop), a block extent of 1 (every link of that direction
leaves the block) and blocks whose +mu face does not start on a chunk of 8 sites.
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


def _setup(amg, L, B, ntv, U, tv, arith):
    p = amg.make_params(L, B, ntv, 1, H.M0, H.CSW, amg.AMG_FP64, amg.AMG_FP64, amg.AMG_FP64, setup_arith=arith)
    stream = torch.cuda.current_stream()
    h, _ = amg.amg_setup_coarse(p, U, tv, stream)
    return h


def _export_dc(amg, h, Vc, nc):
    out = torch.empty((Vc, 9, nc, nc), dtype=torch.complex128, device="cuda")
    amg.amg_export_Dc(h, out)
    torch.cuda.synchronize()
    return out


CASES = [
    # L, B, ntv, eps, seed
    ((4, 4, 4, 4), (2, 2, 2, 2), 8, 0.3, 11),     # nc 16, 2x2 tiles
    ((8, 4, 6, 4), (2, 2, 2, 2), 6, 0.4, 12),     # ragged coarse extents 4, 2, 3, 2
    ((4, 4, 4, 4), (2, 2, 2, 2), 5, 0.3, 13),     # odd Ntv: tiles straddle the chirality boundary
    ((4, 4, 4, 4), (1, 2, 2, 2), 8, 0.3, 14),     # B_x = 1: every x-link leaves its block
    ((6, 6, 6, 6), (3, 3, 3, 3), 12, 0.3, 15),    # Vb 81: the +mu face starts inside a chunk
    ((8, 8, 8, 8), (4, 4, 4, 4), 22, 0.3, 16),    # nc 44: widest 2x2 tiling, 484 threads
    ((8, 8, 8, 8), (4, 4, 2, 2), 23, 0.3, 17),    # nc 46: 2x4 tiles, a padded column, odd Ntv
    ((8, 8, 8, 8), (2, 2, 2, 2), 32, 0.3, 18),    # nc 64: 512 threads
]


@pytest.mark.parametrize("L,B,ntv,eps,seed", CASES, ids=["%s_b%s_ntv%d" % ("x".join(map(str, c[0])), "".join(map(str, c[1])), c[2]) for c in CASES])
def test_pair_assembly_matches_oracle_and_fp64(amg, L, B, ntv, eps, seed):
    sites = si.all_sites(L)
    Uh = si.links(seed, eps, sites)
    tvh = si.test_vectors(seed, ntv, sites)
    Uf = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
    Cf = dirac.clover_field(Uf, H.CSW)
    Q = coarse.orthonormalize(tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
    ref = coarse.coarse_operator(Uf, Cf, H.M0, Q, L, B)
    Lc = lat.coarse_dims(L, B)
    Vc, nc = int(np.prod(Lc)), 2 * ntv
    U, tv = torch.from_numpy(Uh).cuda(), torch.from_numpy(tvh).cuda()
    h64 = _setup(amg, L, B, ntv, U, tv, amg.AMG_SETUP_FP64)
    hp = _setup(amg, L, B, ntv, U, tv, amg.AMG_SETUP_F32PAIR)
    try:
        nagg = 6 * int(np.prod(B))
        R64 = torch.empty((Vc, 2, ntv, nagg), dtype=torch.complex128, device="cuda")
        Rp = torch.empty_like(R64)
        amg.amg_export_R(h64, R64)
        amg.amg_export_R(hp, Rp)
        torch.cuda.synchronize()
        assert H.rel(Rp.cpu().numpy(), H.q_to_lib_R(Q)) < 1e-12
        assert H.rel(Rp.cpu().numpy(), R64.cpu().numpy()) < 1e-13
        D64 = _export_dc(amg, h64, Vc, nc)
        Dp = _export_dc(amg, hp, Vc, nc)
        got = Dp.cpu().numpy()
        for d in range(9):
            assert H.rel(got[:, d], ref[:, d]) < 1e-12, d
            assert H.rel(got[:, d], D64[:, d].cpu().numpy()) < 1e-13, d
        # largest entry error of the self blocks (a dropped quadrant could hide in a norm)
        assert np.abs(got[:, 0] - ref[:, 0]).max() <= 1e-12 * np.abs(ref[:, 0]).max()
        assert amg.amg_sync_status(hp) == amg.AMG_OK
    finally:
        amg.amg_destroy(h64)
        amg.amg_destroy(hp)


def test_pair_assembly_full_size_32x4(amg):
    """32^4, 4^4 blocks, Ntv = 20 (the benchmark's lattice): the whole D_c against the library's
    FP64 assembly, and sampled D_c rows against the oracle (first, last, a t-wrapping and interior
    blocks); the pair assembly must also be the faster one."""
    from synth import device as sd
    L, B, ntv, eps, off = H.WORKLOADS["fp32_32^4_b4_ntv20"]
    seed = si.SEED_BASE + off
    Lc = tuple(L[m] // B[m] for m in range(4))
    Vc, nc = int(np.prod(Lc)), 2 * ntv
    U = sd.links(seed, eps, L)
    tv = sd.test_vectors(seed, ntv, L)
    h64 = _setup(amg, L, B, ntv, U, tv, amg.AMG_SETUP_FP64)
    hp = _setup(amg, L, B, ntv, U, tv, amg.AMG_SETUP_F32PAIR)
    del U, tv
    torch.cuda.empty_cache()
    try:
        t64 = amg.amg_setup_timings(h64)
        tp = amg.amg_setup_timings(hp)
        D64 = _export_dc(amg, h64, Vc, nc)
        Dp = _export_dc(amg, hp, Vc, nc)
        for d in range(9):
            num = torch.linalg.vector_norm(Dp[:, d] - D64[:, d]).item()
            den = torch.linalg.vector_norm(D64[:, d]).item()
            assert num <= 1e-13 * den, d
        samples = [(0, 0, 0, 0), (7, 7, 7, 7), (3, 5, 1, 7), (7, 0, 6, 2), (2, 7, 4, 0), (5, 2, 3, 4),
                   (1, 6, 0, 5), (6, 3, 7, 1)]
        for X in samples:
            i = int(lat.coarse_index(np.array(X), Lc))
            _, Dref, _, _ = H.patch_reference(seed, eps, L, B, ntv, X)
            assert H.rel(Dp[i].cpu().numpy(), Dref) < 1e-12, X
        assert tp[1] < t64[1] and tp[2] < t64[2], (tp, t64)
    finally:
        amg.amg_destroy(h64)
        amg.amg_destroy(hp)
