"""The autotuner's selection and its record, on the CPU with a stand-in
measurement (the real one runs the batch on the GPU): the fastest candidate
per kernel is chosen from the stages of the workload asked for, and the
choice round-trips through the JSON record keyed by device, precision and
workload."""
from paper_2311_01135_gb300 import RKS_FP64, RKS_MIXED, tune


def _fake(best_grid, best_jk, grid_key, jk_key):
    def measure(mols, precision, grid_chunks, jk_chunks):
        return {grid_key: 10.0 + abs(grid_chunks - best_grid), jk_key: 5.0 + abs(jk_chunks - best_jk),
                "scf_step": 1.0}
    return measure


def test_picks_the_fastest_per_kernel():
    r = tune.tune([], RKS_MIXED, measure=_fake(8, 4, "grid_xc_tc", "jk"))
    assert (r["grid_chunks"], r["jk_chunks"]) == (8, 4)
    r = tune.tune([], RKS_FP64, measure=_fake(32, 16, "grid_xc", "jk"))
    assert (r["grid_chunks"], r["jk_chunks"]) == (32, 16)


def test_large_workload_reads_the_global_memory_kernels():
    r = tune.tune([], RKS_MIXED, workload="large", measure=_fake(16, 2, "grid_large", "jk_large"))
    assert (r["grid_chunks"], r["jk_chunks"]) == (16, 2)


def test_record_round_trip(tmp_path):
    p = str(tmp_path / "tuned.json")
    assert tune.load_choice(p, "GB300", RKS_MIXED) == {}
    tune.save_choice(p, "GB300", RKS_MIXED, "small", {"grid_chunks": 16, "jk_chunks": 8})
    tune.save_choice(p, "GB300", RKS_MIXED, "large", {"grid_chunks": 32, "jk_chunks": 4})
    assert tune.load_choice(p, "GB300", RKS_MIXED) == {"grid_chunks": 16, "jk_chunks": 8}
    assert tune.load_choice(p, "GB300", RKS_MIXED, "large") == {"grid_chunks": 32, "jk_chunks": 4}
    assert tune.load_choice(p, "GB300", RKS_FP64) == {}
