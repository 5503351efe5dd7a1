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


def test_reference_arm_runs_the_gpu_arms_step_on_every_core(monkeypatch):
    """--impl reference: the oracle on every host core (one single-threaded process each), the
    same step mix as the GPU arm (R, FGMRES with the workload's 2 applications, P) and the same
    config; the sample's bytes are the workload's FP32 byte model scaled to the 16^4 volume."""
    import os
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    cfg = bench.workload_config(bench.APPLIES_PER_STEP)
    assert bench.APPLIES_PER_STEP == 2
    assert cfg["applies_per_step"] == 2 and cfg["bytes_per_step"] == 5197791232
    assert bench.sample_step_bytes(2) == 5197791232 / 16
    res, rank = bench.run_reference(type("A", (), {"warmup": 0, "steps": 1})())
    assert rank == 0 and res["impl"] == "reference"
    assert res["config"] == cfg
    cores = len(os.sched_getaffinity(0))
    assert res["cpu_baseline"]["cores"] == res["cpu_baseline"]["threads"] == cores
    assert res["value"] > 0 and res["e2e"]["h2d_bytes_per_step"] == 0


def test_setup_report_counts_the_rank6_sums():
    # 48^3 x 96, Ntv = 24: per fine site four hop jobs over all (2 Ntv)^2 entries and the self job
    # over its two chirality-diagonal quadrants, six rows each, 8 flops per complex multiply-add
    V, ntv = 48 ** 3 * 96, 24
    per_site = 6 * (4 * (2 * ntv) ** 2 + 2 * ntv ** 2)
    flop = 8 * V * per_site
    rep = bench.setup_report([150.0, 860.0, 1742.0, 25.0], V, ntv)
    assert rep["assembly_tflop"] == round(flop / 1e12, 3) == 5.284
    assert abs(rep["assembly_fp64_equiv_tflops"] - flop / 1.742 / 1e12) < 1e-3
    assert rep["assembly"] == 1742.0 and rep["gram_schmidt"] == 860.0
    assert rep["fp64_peak_tflops"] == 1.25 and rep["assembly_arith"] == "f32pair"


def test_fine_grid_byte_models():
    # FP32 complex = 8 bytes: D reads 4 links (4 x 9), the clover as two Hermitian upper triangles
    # (2 x 21), psi (12) and writes out (12); a SAP half sweep per site of its colour reads the
    # links, the clover, y and x and writes x, and reads the other colour's x once
    c8 = 8
    d = (4 * 9 + 2 * 21 + 12 + 12) * c8
    sap_colour_site = (4 * 9 + 2 * 21 + 3 * 12) * c8
    assert d == 816
    assert (sap_colour_site + 12 * c8) // 2 == 504
    import inspect
    src = inspect.getsource(bench.run_vcycle)
    assert "d_bytes = V * 816" in src and "half_bytes = V * 504" in src
