"""The oracle arm of bench.py (`--impl reference`) on the host cores: one JSON line with the
metric, unit and workload of the GPU arm, and the oracle described as the CPU baseline."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == "fwd+adjoint particle-substeps/s (batched)" and d["unit"] == "particle-substeps/s"
    assert d["config"]["workload"] == "fluid-1024env-8192p-64grid-16x25-fwd+adjoint"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_roofline_traffic_belongs_to_these_kernel_sources():
    """The DRAM traffic bench.py reports beside the roofline comes from an ncu capture of the
    kernel sources as they are now; a kernel change must be recaptured before it is reported
    (bench.py then prints null), and the profile summary names the same source hash."""
    sys.path.insert(0, ROOT)
    import bench

    h = bench.kernel_source_hash()
    for kernel, (per_particle, src_hash) in bench.MEASURED_TRAFFIC.items():
        assert src_hash == h, (kernel, src_hash, h)
        assert 0 < per_particle < 1000
    with open(os.path.join(ROOT, "profiles", "dram_traffic_fluid256_1x5.md")) as fh:
        assert h in fh.read()
