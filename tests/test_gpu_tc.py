"""GPU parity of the tensor-core (BF16 planes, FP32 accumulation) multi-RHS forms.

The BF16 storage of D_c and R rounds each real and imaginary part to nearest
even (relative error <= 2^-8); BF16 fine vectors are given to the library and
to the oracle as the same values.  Each result is checked
  (a) against the oracle applied to the dequantised stored operator (only FP32
      accumulation and the BF16 rounding of the other operand remain), and
  (b) against the FP64 oracle within the stated bound
      (sum of unit roundoffs) * || |A| |x| || / || A x ||.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coarse, dirac, lattice as lat  # noqa: E402
from synth import inputs as si  # noqa: E402

import helpers as H  # noqa: E402

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def amg():
    import paper_1512_04506_gb300 as m
    return m


def bf16_round(z):
    """Complex array -> the nearest BF16 Re/Im values (torch's round-to-nearest-even), as complex128."""
    f = torch.from_numpy(np.ascontiguousarray(np.stack([z.real, z.imag], -1)).astype(np.float32))
    b = f.to(torch.bfloat16).to(torch.float64).numpy()
    return b[..., 0] + 1j * b[..., 1]


def to_bf16_dev(z):
    """Complex array -> device tensor of interleaved BF16 (re, im) pairs."""
    f = torch.from_numpy(np.ascontiguousarray(np.stack([z.real, z.imag], -1)).astype(np.float32))
    return f.to(torch.bfloat16).cuda()


def from_bf16_dev(t):
    f = t.float().cpu().numpy().astype(np.float64)
    return f[..., 0] + 1j * f[..., 1]


class TcCase:
    def __init__(self, amg, L, B, ntv, seed):
        self.amg, self.L, self.B, self.ntv, self.seed = amg, L, B, ntv, seed
        self.Lc = lat.coarse_dims(L, B)
        self.Vc = int(np.prod(self.Lc))
        self.V = int(np.prod(L))
        sites = si.all_sites(L)
        Uh = si.links(seed, 0.3, sites)
        tvh = si.test_vectors(seed, ntv, sites)
        U = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
        C = dirac.clover_field(U, H.CSW)
        self.Q = coarse.orthonormalize(tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
        self.Dc = coarse.coarse_operator(U, C, H.M0, self.Q, L, B)
        p = amg.make_params(L, B, ntv, 16, H.M0, H.CSW, amg.AMG_BF16, amg.AMG_BF16, amg.AMG_BF16)
        self.stream = torch.cuda.current_stream()
        self.h, _ = amg.amg_setup_coarse(p, torch.from_numpy(Uh).cuda(), torch.from_numpy(tvh).cuda(), self.stream)

    def close(self):
        self.amg.amg_destroy(self.h)


@pytest.fixture(scope="module", params=[((8, 8, 8, 8), (4, 4, 4, 4), 24), ((8, 4, 8, 12), (4, 2, 4, 4), 16),
                                        ((8, 8, 8, 8), (4, 4, 4, 4), 20)],
                ids=["8^4_b4_ntv24", "8x4x8x12_b4x2x4x4_ntv16", "8^4_b4_ntv20_half_tiles"])
def case(amg, request):
    L, B, ntv = request.param
    c = TcCase(amg, L, B, ntv, 404)
    yield c
    c.close()


def test_bf16_storage_of_dc(amg, case):
    c = case
    stored = torch.empty((c.Vc, 9, 2 * c.ntv, 2 * c.ntv), dtype=torch.complex128, device="cuda")
    amg.amg_export_Dc_stored(c.h, stored)
    st = stored.cpu().numpy()
    # entries that are rounding noise of an exact zero (~1e-17) differ between the two FP64
    # assemblies; they get an absolute floor of 1e-13 of the largest entry
    floor = 1e-13 * np.abs(c.Dc).max()
    assert np.all(np.abs(st.real - c.Dc.real) <= U_BF16 * np.abs(c.Dc.real) + floor)
    assert np.all(np.abs(st.imag - c.Dc.imag) <= U_BF16 * np.abs(c.Dc.imag) + floor)
    # nearly every entry is exactly the BF16 rounding (direct double->BF16 may differ from the
    # double->float->BF16 path of the test in rare ties, and noise entries differ)
    assert np.mean(st == bf16_round(c.Dc)) > 0.99


@pytest.mark.parametrize("nrhs", [4, 8, 12, 16])
def test_tc_coarse_apply(amg, case, nrhs):
    c = case
    xc = si.coarse_vector(c.seed + 1, c.ntv, nrhs, np.arange(c.Vc))
    x32 = xc.astype(np.complex64)
    y = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=torch.complex64, device="cuda")
    amg.amg_coarse_apply(c.h, torch.from_numpy(x32).cuda(), y, nrhs, c.stream)
    got = y.cpu().numpy().astype(np.complex128)
    stored = torch.empty((c.Vc, 9, 2 * c.ntv, 2 * c.ntv), dtype=torch.complex128, device="cuda")
    amg.amg_export_Dc_stored(c.h, stored)
    ref_stored = coarse.coarse_apply(stored.cpu().numpy(), bf16_round(x32.astype(np.complex128)), c.Lc)
    assert H.rel(got, ref_stored) < 1e-5
    ref = coarse.coarse_apply(c.Dc, x32.astype(np.complex128), c.Lc)
    bound = coarse.reduced_precision_bound(c.Dc, x32.astype(np.complex128), c.Lc, 2 * U_BF16)
    assert H.rel(got, ref) <= bound


@pytest.mark.parametrize("nrhs", [4, 8, 12, 16])
def test_tc_restrict_prolong(amg, case, nrhs):
    c = case
    y = bf16_round(si.fine_rhs(c.seed + 2, nrhs, si.all_sites(c.L)))        # (V, 4, 3, nrhs)
    yc = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=torch.complex64, device="cuda")
    amg.amg_restrict(c.h, to_bf16_dev(y), yc, nrhs, c.stream)
    got = yc.cpu().numpy().astype(np.complex128)
    yf = y.reshape(H.field_shape(c.L) + (4, 3, nrhs))
    ref = coarse.restrict(c.Q, yf, c.B)
    absref = coarse.restrict(np.abs(c.Q).astype(np.complex128), np.abs(yf).astype(np.complex128), c.B).real
    K = 2 * 6 * int(np.prod(c.B))
    bound = (U_BF16 + (K + 2) * 2.0 ** -24) * np.linalg.norm(absref) / np.linalg.norm(ref)
    assert H.rel(got, ref) <= bound
    assert H.rel(got, ref) < 4e-3
    # prolongation of an FP32 coarse vector to BF16 fine vectors
    xc = si.coarse_vector(c.seed + 3, c.ntv, nrhs, np.arange(c.Vc)).astype(np.complex64)
    x = torch.empty((c.V, 4, 3, nrhs, 2), dtype=torch.bfloat16, device="cuda")
    amg.amg_prolong(c.h, torch.from_numpy(xc).cuda(), x, nrhs, c.stream)
    gotx = from_bf16_dev(x)
    xc64 = xc.astype(np.complex128)
    refx = coarse.prolong(c.Q, xc64, c.L, c.B).reshape(c.V, 4, 3, nrhs)
    absx = coarse.prolong(np.abs(c.Q).astype(np.complex128), np.abs(xc64).astype(np.complex128),
                          c.L, c.B).reshape(c.V, 4, 3, nrhs).real
    boundx = (3 * U_BF16 + (2 * c.ntv + 2) * 2.0 ** -24) * np.linalg.norm(absx) / np.linalg.norm(refx)
    assert H.rel(gotx, refx) <= boundx
    assert amg.amg_sync_status(c.h) == amg.AMG_OK


def test_tc_solver_runs_on_bf16_links(amg, case):
    """FGMRES on the BF16 operator with 16 right-hand sides reaches its tolerance in the true
    residual of the stored (BF16) operator."""
    c = case
    nrhs = 16
    b = si.coarse_vector(c.seed + 4, c.ntv, nrhs, np.arange(c.Vc)).astype(np.complex64)
    x = torch.empty((c.Vc, 2, c.ntv, nrhs), dtype=torch.complex64, device="cuda")
    info = amg.amg_coarse_solve(c.h, torch.from_numpy(b).cuda(), x, nrhs, tol=1e-2, restart=10,
                                max_applies=100, stream=c.stream)
    stored = torch.empty((c.Vc, 9, 2 * c.ntv, 2 * c.ntv), dtype=torch.complex128, device="cuda")
    amg.amg_export_Dc_stored(c.h, stored)
    xs = x.cpu().numpy().astype(np.complex128)
    for r in range(nrhs):
        assert info[r][1] <= 1e-2
        true = H.rel(coarse.coarse_apply(stored.cpu().numpy(), xs[..., r], c.Lc), b[..., r].astype(np.complex128))
        assert true < 2e-2


@pytest.fixture(scope="module", params=[((8, 8, 8, 8), (4, 4, 4, 4), 24), ((8, 8, 8, 8), (4, 4, 4, 4), 20)],
                ids=["ntv24", "ntv20_half_tiles"])
def fp32case(amg, request):
    """FP32 storage with max_nrhs 16: applies with 4, 8, 12 or 16 columns take the tensor-core path
    with split TF32 operands."""
    L, B, ntv = request.param
    sites = si.all_sites(L)
    Uh = si.links(505, 0.3, sites)
    tvh = si.test_vectors(505, ntv, sites)
    U = np.moveaxis(Uh.reshape(H.field_shape(L) + (4, 3, 3)), 4, 0)
    Q = coarse.orthonormalize(tvh.reshape(H.field_shape(L) + (4, 3, ntv)), B)
    Dc = coarse.coarse_operator(U, dirac.clover_field(U, H.CSW), H.M0, Q, L, B)
    p = amg.make_params(L, B, ntv, 16, H.M0, H.CSW, amg.AMG_FP32, amg.AMG_FP32, amg.AMG_FP32)
    st = torch.cuda.current_stream()
    h, _ = amg.amg_setup_coarse(p, torch.from_numpy(Uh).cuda(), torch.from_numpy(tvh).cuda(), st)
    yield dict(h=h, Dc=Dc, Lc=lat.coarse_dims(L, B), ntv=ntv, st=st)
    amg.amg_destroy(h)


@pytest.mark.parametrize("nrhs", [4, 8, 12, 16])
def test_fp32_multi_rhs_apply_tf32x3(amg, fp32case, nrhs):
    """The FP32 apply tolerance (1e-5 against FP64) although the products run on TF32 tensor cores
    (three split products: each term carries about 2^-21 relative error, which the cancellation in
    D_c x amplifies to a few 1e-6), and the one-column SIMT FP32 path agrees to 1e-5."""
    c = fp32case
    Vc = int(np.prod(c["Lc"]))
    xc = si.coarse_vector(606 + nrhs, c["ntv"], nrhs, np.arange(Vc)).astype(np.complex64)
    xd = torch.from_numpy(xc).cuda()
    y = torch.empty_like(xd)
    amg.amg_coarse_apply(c["h"], xd, y, nrhs, c["st"])
    got = y.cpu().numpy().astype(np.complex128)
    ref = coarse.coarse_apply(c["Dc"], xc.astype(np.complex128), c["Lc"])
    assert H.rel(got, ref) < 1e-5
    cols = []
    for r in range(nrhs):
        x1 = xd[..., r:r + 1].contiguous()
        y1 = torch.empty_like(x1)
        amg.amg_coarse_apply(c["h"], x1, y1, 1, c["st"])
        cols.append(y1.cpu().numpy())
    simt = np.concatenate(cols, axis=-1).astype(np.complex128)
    assert H.rel(got, simt) < 1e-5
    assert amg.amg_sync_status(c["h"]) == amg.AMG_OK
