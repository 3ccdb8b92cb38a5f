"""The DRAM-traffic records under profiles/ that bench.py reads for the
roofline's `traffic` key: each parses, names sources that exist, carries a
sha256 digest and a byte count, and the recorded bytes of one launch are
within 10% of the algorithmic bytes bench.py divides by (no capture shows
wasted re-reads).  A record whose sources changed after the
capture makes bench.py report null; that is allowed and not checked here."""
import glob
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

RECORDS = sorted(glob.glob(os.path.join(ROOT, "profiles", "dram_traffic_*.txt")))


def _parse(path):
    kv, comments = {}, []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                comments.append(line)
                continue
            key, _, val = line.partition(" ")
            kv[key] = val.strip()
    return kv, comments


def test_there_are_records():
    assert len(RECORDS) >= 4


@pytest.mark.parametrize("path", RECORDS, ids=[os.path.basename(p) for p in RECORDS])
def test_record_is_well_formed(path):
    kv, comments = _parse(path)
    for key in ("kernel", "sources", "sha256", "rows", "dram_bytes"):
        assert key in kv, key
    assert os.path.basename(path) == f"dram_traffic_{kv['kernel']}.txt"
    for rel in kv["sources"].split():
        assert os.path.isfile(os.path.join(ROOT, rel)), rel
    assert re.fullmatch(r"[0-9a-f]{64}", kv["sha256"])
    rows, total = int(kv["rows"]), int(kv["dram_bytes"])
    assert rows > 0 and total > 0
    # the comment block gives the command that made the record and the two
    # counters whose sum is dram_bytes
    text = "\n".join(comments)
    assert "--clock-control none" in text
    m = re.search(r"dram__bytes_read\.sum (\d+), dram__bytes_write\.sum (\d+)", text)
    assert m and int(m.group(1)) + int(m.group(2)) == total


@pytest.mark.parametrize("path", RECORDS, ids=[os.path.basename(p) for p in RECORDS])
def test_recorded_traffic_is_close_to_the_algorithmic_bytes(path):
    """Scaled to the bench's rows the way bench.py scales it, the recorded
    traffic of one launch is within 10% of bench.py's algorithmic bytes."""
    import bench
    kv, _ = _parse(path)
    work = bench.algorithmic_work(kv["kernel"])
    assert "bytes" in work
    total = float(kv["dram_bytes"]) * bench.N_ROWS / float(kv["rows"])
    alg = float(work["bytes"])
    assert alg <= 1.10 * total and total <= 1.10 * alg, (total, alg)
