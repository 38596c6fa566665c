"""Autotuner host logic (no GPU): candidate generation, memory estimates, cache keys and files."""
import json

from paper_2103_14921_gb300 import tune


def test_candidates_cover_core_sizes_and_overlaps():
    c = tune.candidates(256, 256, 96)
    parts = {p for p, _ in c}
    assert (16, 16, 6) in parts and (11, 11, 4) in parts and (13, 13, 5) in parts
    assert {ov for _, ov in c} == {2, 3, 4}
    assert len(c) == len(set(c))
    # tiny grids never ask for zero boxes
    assert all(min(p) >= 1 for p, _ in tune.candidates(10, 10, 8))


def test_problem_key_rounds_rhs_up():
    assert tune.problem_key(112, 112, 112, 5.0, 16, 2) == tune.problem_key(112, 112, 112, 5.0, 9, 2)
    assert tune.problem_key(112, 112, 112, 5.0, 17, 2) != tune.problem_key(112, 112, 112, 5.0, 16, 2)


def test_krylov_bytes_matches_basis_count():
    assert tune.krylov_bytes(1000, 2, 30) == 1000 * 2 * (63 * 8 + 48)


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    assert tune.load_cache(p) == {}
    tune.save_cache(p, {"k": {"parts": [2, 2, 2], "overlap": 2}})
    assert json.load(open(p))["k"]["overlap"] == 2
    assert tune.load_cache(p)["k"]["parts"] == [2, 2, 2]


def test_library_memory_estimate_grows_with_boxes_and_rhs():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    import ctypes as C
    g = helm.GridDesc(64, 64, 64, 25.0, 5.0, 8, 1e-3, 0, (C.c_double * 7)(1, 0, 0, 1, 0, 0, 0))
    small = helm.estimate_bytes(g, helm.OrasDesc(2, 2, 2, 2, 4, 0, helm.PREC_TF32), 1)
    more_rhs = helm.estimate_bytes(g, helm.OrasDesc(2, 2, 2, 2, 4, 0, helm.PREC_TF32), 64)
    fp64 = helm.estimate_bytes(g, helm.OrasDesc(2, 2, 2, 2, 4, 0, helm.PREC_FP64), 1)
    assert 0 < small < more_rhs and small < fp64
    # factors of 8 boxes of 34 x 34 x 34 nodes, padded rows of 1168 complex64: about 3 GB
    assert 2.5e9 < small < 6e9


def test_package_cache_holds_the_benched_problem_classes():
    """The tuning cache shipped in the package holds the autotuner's choices for the two benched workloads that
    use it (thrust-fold 256 x 256 x 96 at 5 Hz in batches of 32, attenuating 160 x 160 x 80 tuned at 6 Hz for 128
    columns), each among the decompositions that workload lets the tuner time, with its timed trials."""
    import os

    import bench
    cache = tune.load_cache(bench.TUNE_CACHE)
    assert os.path.dirname(bench.TUNE_CACHE).endswith("paper_2103_14921_gb300")
    tf = cache[tune.problem_key(256, 256, 96, 5.0, 32, 2)]
    assert (tuple(tf["parts"]), tf["overlap"]) in set(tune.candidates(256, 256, 96))
    assert tf["coarse_iters"] in (0, 10) and tf["knobs"]["tc_flow"] in (0, 1)
    at = cache[tune.problem_key(160, 160, 80, 6.0, 128, 2)]
    assert (tuple(at["parts"]), at["overlap"]) in {(tuple(p), ov) for p, ov in bench.ATTEN_CANDS}
    for entry in (tf, at):
        good = [t for t in entry["trials"] if t.get("converged")]
        assert good and entry["rhs_per_s"] == max(t["rhs_per_s"] for t in good)
