"""Host logic of bench.py on CPU: the algorithmic byte count of the roofline
kernel and the ncu traffic record it reports beside it."""
import glob
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_fused_operator_byte_count():
    """The roofline's algorithmic bytes of the fused CG operator: z, p and six
    factors read, p and w written (ten values per point)."""
    import bench
    assert bench.ka_bytes_per_point("mixed") == 40
    assert bench.ka_bytes_per_point("gmres") == 40
    assert bench.ka_bytes_per_point("fp64") == 80


def test_traffic_record_follows_the_kernel_source():
    """roofline.traffic comes from the committed ncu summary only while the
    kernel's source file is unchanged since the capture."""
    import hashlib
    import re
    import bench
    rec = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path).read().splitlines():
            line = line.strip().strip("`")
            if line.startswith("traffic-record:"):
                rec = dict(kv.split("=", 1) for kv in line[len("traffic-record:"):].split())
    assert rec is not None
    src_sha = hashlib.sha256(open(os.path.join(ROOT, rec["source"]), "rb").read()).hexdigest()[:16]
    got = bench._traffic_for(rec["kernel"], rec["workload"])
    if src_sha == rec["source_sha"]:
        assert got == float(rec["bytes_per_launch"])
    else:
        assert got is None
    assert bench._traffic_for("no_such_kernel<float>", rec["workload"]) is None
    assert re.fullmatch(r"[0-9a-f]{16}", rec["source_sha"])
