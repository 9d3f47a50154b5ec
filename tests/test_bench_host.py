"""bench.py's host-side measurement logic, without a GPU: the DRAM traffic read from a committed ncu
summary only while the kernel sources hash to the captured ones, scaled by the events of a launch;
the workload table and the per-rank bookkeeping."""
import hashlib

import bench


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)


def test_profiled_traffic_follows_the_source_hash(tmp_path):
    src = tmp_path / "k.cuh"
    _write(src, "kernel v1\n")
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    md = tmp_path / "p.md"
    _write(md, "# k\n\nsource_sha256_16: %s   (k.cuh)\ntraffic_bytes_per_event: 1000  (per event)\n" % sha)
    assert bench.profiled_traffic([str(src)], str(md), 524288) == 1000.0 * 524288
    _write(src, "kernel v2\n")   # the kernel changed since the capture: no traffic figure
    assert bench.profiled_traffic([str(src)], str(md), 524288) is None
    assert bench.profiled_traffic([str(src)], str(tmp_path / "missing.md"), 1) is None


def test_workloads_and_rank_bookkeeping():
    assert {w["nevt"] for w in bench.WORKLOADS.values()} == {16384, 524288, 262144, 65536}
    assert bench.rank_first_event(3, 1000) == 3000
    assert bench.aggregate_rate(2, 1000, 10.0) == 2000 / 10e-3


def test_clock_records_that_disqualify_a_timed_region():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    assert not bench.rejected_clocks(ok)
    assert not bench.rejected_clocks(None)
    assert not bench.rejected_clocks(dict(ok, reasons=["sw_power_cap"], sm_mhz=1500.0))   # kept, noted
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.rejected_clocks(dict(ok, reasons=[r]))
    assert bench.rejected_clocks(dict(ok, sm_mhz=1000.0))   # well below max with no reason: a clock lock


def test_clock_sampler_names_the_gpu_by_uuid():
    """nvidia-smi numbers GPUs physically and ignores CUDA_VISIBLE_DEVICES: the sampler is given the
    device's UUID, as torch reports it, in nvidia-smi's "GPU-<uuid>" form."""
    class Props:
        def __init__(self, uuid):
            self.uuid = uuid

    u = "6b1c0e52-7a3d-4f0e-9c1a-2b3c4d5e6f70"
    assert bench.nvsmi_gpu_id(Props(u)) == "GPU-" + u
    assert bench.nvsmi_gpu_id(Props("GPU-" + u)) == "GPU-" + u
    assert bench.nvsmi_gpu_id(Props("")) is None
    assert bench.nvsmi_gpu_id(object()) is None
