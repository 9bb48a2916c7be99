"""The ncu records under profiles/ that bench.py reads for its roofline (L1 wavefronts and DRAM bytes of the
propagation) are keyed by the SHA-256 of csrc/propagate.cu; a record taken on another version of the kernel is
ignored by the benchmark.  This checks that every record describes the current source, so a change to the kernel
cannot silently drop the roofline's measured denominators from the benchmark line."""
import hashlib
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RECORDS = ("propagate_l1_kitti_1242x375.json", "propagate_traffic_kitti_1242x375.json",
           "propagate_traffic_batch8_kitti_1242x375.json")


def test_roofline_records_match_the_propagation_source():
    with open(os.path.join(ROOT, "paper_1805_03517_gb300", "csrc", "propagate.cu"), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    with open(os.path.join(ROOT, "paper_1805_03517_gb300", "tuned.json")) as f:
        table = json.load(f)["kitti_1242x375"]
    for name in RECORDS:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            rec = json.load(f)
        assert rec["propagate_cu_sha256"] == sha, f"{name} was captured on another version of propagate.cu"
        assert [list(c) for c in rec["tiles_per_level"]] == [list(c) for c in table], name
        assert "ncu" in rec["capture"] and "--clock-control none" in rec["capture"], name
