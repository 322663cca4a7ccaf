"""The bench's reference arm (the FP64 oracle on the host cores) runs without a GPU: its one JSON
line carries the keys the benchmark contract names, with the oracle's own sample and no host-device
traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--workload", "walker_2d"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "walker_2d"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["nproc"] >= 1 and "cpu_model" in cb
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_default_workload_is_the_largest_single_gpu_scene():
    """With no flags the bench times the 1M-particle 3D cluster under its 4 GiB checkpoint budget."""
    sys.path.insert(0, ROOT)
    import bench
    old = sys.argv
    sys.argv = ["bench.py"]
    try:
        args = bench.parse()
    finally:
        sys.argv = old
    assert args.workload == "box_cluster_3d" and args.gpus == 1
    spec = bench.workload(args.workload)
    assert spec.n_particles == 1_000_000 and spec.n_steps == 200
    assert bench.budget_of(spec) == 4 << 30


def test_committed_traffic_matches_the_kernel_sources_and_algorithmic_bytes():
    """profiles/traffic.json holds ncu DRAM bytes per particle of the roofline kernels, keyed to a
    hash of the kernel sources; the bench reports them only while the sources still match.  Each
    entry names its committed summary, and DRAM traffic stays within a factor of the algorithmic
    bytes (no kernel re-reads its inputs many times)."""
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    dims = {"walker_2d": 0, "box_cluster_3d": 1}
    for wl, kernels in rec.items():
        for kern, e in kernels.items():
            assert os.path.exists(os.path.join(ROOT, e["capture"])), e["capture"]
            assert len(e["kernel_hash"]) == 12
            algo = bench.ALGO_BYTES[kern][dims[wl]]
            assert 0.5 * algo <= e["dram_bytes_per_particle"] <= 2.0 * algo, (wl, kern)
            if e["kernel_hash"] == bench.kernel_source_hash():
                assert bench.measured_traffic(kern, wl, 1000) == e["dram_bytes_per_particle"] * 1000
