"""bench.py's stored DRAM traffic: the figure of an ncu capture is used only
while the kernel's source file still has the hash recorded with it."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_committed_entry_matches_its_source():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        entry = json.load(f)["pcg_batched_persistent"]
    with open(os.path.join(ROOT, entry["source"]), "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    assert digest == entry["sha256"], "kernel source changed since the ncu capture"
    import bench
    assert bench.stored_traffic("pcg_batched_persistent", 1000, entry["instances"]) == \
        int(entry["bytes_per_unit"] * 1000)
    # another instance count, or an unknown kernel: no figure
    assert bench.stored_traffic("pcg_batched_persistent", 1000, entry["instances"] * 2) is None
    assert bench.stored_traffic("no_such_kernel", 1000, 8) is None
