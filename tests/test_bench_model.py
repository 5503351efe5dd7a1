"""Host-side arithmetic of the benchmark: the algorithmic bytes of one coarse-grid correction on
the default workload (32^4 lattice, 4^4 blocks, Ntv = 20, FP32 = 8 bytes per complex value), the
Arnoldi step indices of FGMRES(30) for a given number of applications, and the whole-job rate.
Expected values are written out from the byte counts of each kernel, not taken from bench.py.
"""
import bench


def test_default_workload_bytes():
    V, Vb, Vc, nc, ntv = 32 ** 4, 4 ** 4, 8 ** 4, 40, 20
    c8 = 8
    R = Vc * 2 * ntv * 6 * Vb * c8        # R streamed once by restriction and once by prolongation
    fine = V * 12 * c8                     # y read / x written
    coarse = Vc * nc * c8                  # one coarse vector
    restrict = R + fine + coarse
    apply_ = Vc * 9 * nc * nc * c8 + 2 * coarse
    # Arnoldi steps j = 0, 1: dots read w and V_0..V_j, the update reads them again and writes w,
    # plus the scaled read and the V_j write of the application (2 (j + 1) + 4 vectors)
    gs = (2 * 1 + 4) * coarse + (2 * 2 + 4) * coarse
    total = 2 * restrict + 2 * apply_ + gs
    got, parts = bench.bytes_model(2, bench.arnoldi_iterations(2))
    assert got == total == 5197791232
    assert parts["restrict"] == parts["prolong"] == restrict == 2115239936
    assert parts["apply"] == apply_ == 474480640


def test_arnoldi_iterations():
    assert bench.RESTART == 30
    assert bench.arnoldi_iterations(1) == [0]
    assert bench.arnoldi_iterations(2) == [0, 1]
    # 200 applications: cycles of 30 Arnoldi steps, each followed by one residual application
    its = bench.arnoldi_iterations(200)
    cycles = 200 // 31
    assert its[:30] == list(range(30))
    assert len(its) == 30 * cycles + (200 - 31 * cycles)
    assert max(its) == 29 and its.count(0) == cycles + 1


def test_whole_job_rate_is_per_rank_bytes_times_ranks():
    one = bench.whole_job_gbs(1, 5e9, 10, 0.01)
    assert one == 5e9 * 10 / 0.01 / 1e9
    assert bench.whole_job_gbs(4, 5e9, 10, 0.01) == 4 * one
