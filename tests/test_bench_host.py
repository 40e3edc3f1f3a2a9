"""Host logic of bench.py: the recorded ncu traffic is used only while the
dominant kernel's sources hash to the value recorded with it."""
import os

import bench


def test_recorded_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    h = bench.source_hash("gemm_simt")
    f = tmp_path / "summary.md"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # source_hash reads the sources relative to ROOT: give it copies
    for src in bench.KERNEL_SOURCES["gemm_simt"]:
        dst = tmp_path / src
        dst.parent.mkdir(parents=True, exist_ok=True)
        with open(os.path.join(os.path.dirname(bench.__file__), src), "rb") as fh:
            dst.write_bytes(fh.read())
    monkeypatch.setattr(bench, "TRAFFIC_FILES", {("gemm_simt", "w"): "summary.md"})
    f.write_text(f"text\ntraffic_bytes_per_launch: 1234 sources_sha256: {h}\n")
    assert bench.recorded_traffic("gemm_simt", "w") == 1234.0
    f.write_text("traffic_bytes_per_launch: 1234 sources_sha256: 0000000000000000\n")
    assert bench.recorded_traffic("gemm_simt", "w") is None        # kernel changed since
    assert bench.recorded_traffic("gemm_simt", "other") is None    # no summary
    assert bench.recorded_traffic("gemm_tc", "w") is None          # kernel not tracked


def test_committed_summary_parses():
    with open(os.path.join(os.path.dirname(bench.__file__),
                           bench.TRAFFIC_FILES[("gemm_simt", "direct_gemm_64")])) as fh:
        line = [l for l in fh if l.startswith("traffic_bytes_per_launch:")]
    assert len(line) == 1
    w = line[0].split()
    assert float(w[1]) > 0 and w[2] == "sources_sha256:" and len(w[3]) == 16


def test_cpu_recipe_baseline_matches_the_oracle():
    """The paper's method on the host (recipe slicing over host BLAS), which
    bench.py times as a CPU baseline, computes the contraction: random
    descriptors of every class and storage order, against the oracle."""
    import numpy as np

    import oracle
    import tcsynth as ts
    rng = np.random.Generator(np.random.PCG64(20131))
    probs = [ts.slice_gemm_48(), ts.direct_gemm_64(n=7), ts.fused_permute_48(n=6)]
    probs += [ts.random_problem(rng, max_order=4, max_ext=5) for _ in range(60)]
    for p in probs:
        ref = oracle.contract_problem(p)
        got = bench.recipe_cpu(p, 2)
        assert oracle.rel_fro(got, ref) <= 1e-13, p.name
