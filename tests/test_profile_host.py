"""Host logic of the measurement: the ncu summary (units, grouping of the
launches, DRAM bytes per row), the source-digest gate on the committed
summary, and the bench's algorithmic bytes of a sub-query.
No GPU."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1901_01488_gb300 import ncu_profile  # noqa: E402


def _csv(path, launches):
    """An ncu --csv log: launches = [(id, kernel, {metric: (value, unit)})]."""
    head = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",' \
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    with open(path, "w") as f:
        f.write("==PROF== Connected to process\n")
        f.write(head)
        for lid, name, metrics in launches:
            for m, (v, u) in metrics.items():
                f.write(f'"{lid}","1","python","box","{name}","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3",'
                        f'"Command line profiler metrics","{m}","{u}","{v}"\n')


def test_summary_units_grouping_and_bytes_per_row(tmp_path):
    rows = 1_000_000
    launches = []
    lid = 0
    # two count scans, then two materialising calls (scan + write); mixed units
    for t_ns, rd_mb in ((2000, 19.0), (4000, 21.0)):
        launches.append((lid, "void esc::scan_kernel<19, 0, 2>(esc::Launch)",
                         {"gpu__time_duration.sum": (f"{t_ns:,}", "ns"), "dram__bytes_read.sum": (rd_mb, "Mbyte"),
                          "dram__bytes_write.sum": (0, "byte")}))
        lid += 1
    for t_us, rd_mb, w_kb in ((3.0, 19.5, 125.0), (5.0, 21.5, 125.0)):
        launches.append((lid, "void esc::scan_kernel<23, 0, 1>(esc::Launch)",
                         {"gpu__time_duration.sum": (t_us, "us"), "dram__bytes_read.sum": (rd_mb, "Mbyte"),
                          "dram__bytes_write.sum": (w_kb, "Kbyte")}))
        lid += 1
        launches.append((lid, "esc::write_kernel(esc::Launch)",
                         {"gpu__time_duration.sum": (1.0, "us"), "dram__bytes_read.sum": (4.0, "Mbyte"),
                          "dram__bytes_write.sum": (1.0, "Mbyte")}))
        lid += 1
    path = tmp_path / "launches.csv"
    _csv(path, launches)
    out = ncu_profile.summarise(str(path), rows, str(tmp_path / "s.json"), "ncu ...")
    k = out["kernels"]
    assert k["scan_kernel (count)"]["launches"] == 2
    assert k["scan_kernel (count)"]["time_us_mean"] == pytest.approx(3.0)           # ns -> us
    assert k["scan_kernel (count)"]["dram_bytes_per_row"] == pytest.approx(20.0)    # (19 + 21) MB / 2 / 1M rows
    assert k["scan_kernel (materialise)"]["dram_bytes_per_row"] == pytest.approx(20.625)
    assert k["write_kernel"]["dram_bytes_per_row"] == pytest.approx(5.0)
    call = out["materialising_call"]
    assert call["dram_bytes_per_row"] == pytest.approx(25.625)
    assert call["shares"]["scan_kernel"] == pytest.approx(8.0 / 10.0)
    assert json.load(open(tmp_path / "s.json"))["source_digest"] == ncu_profile.source_digest()


def test_digest_gate(tmp_path, monkeypatch):
    good = {"source_digest": ncu_profile.source_digest(),
            "kernels": {"scan_kernel (count)": {"dram_bytes_per_row": 19.07}},
            "materialising_call": {"dram_bytes_per_row": 24.14}}
    p = tmp_path / "summary.json"
    p.write_text(json.dumps(good))
    monkeypatch.setattr(ncu_profile, "SUMMARY", str(p))
    assert ncu_profile.traffic_per_row("count") == pytest.approx(19.07)
    assert ncu_profile.traffic_per_row("call") == pytest.approx(24.14)
    p.write_text(json.dumps(dict(good, source_digest="0" * 16)))          # kernels changed since
    assert ncu_profile.traffic_per_row("count") is None
    monkeypatch.setattr(ncu_profile, "SUMMARY", str(tmp_path / "missing.json"))
    assert ncu_profile.traffic_per_row("call") is None


def test_digest_ignores_comments_only(tmp_path, monkeypatch):
    """A comment or whitespace edit keeps the digest (and the committed
    figures valid); a code edit changes it."""
    src = os.path.join(ROOT, "paper_1901_01488_gb300", "csrc")
    os.makedirs(tmp_path / "csrc")
    for f in ("esc_scan.cu", "esc_internal.h"):
        (tmp_path / "csrc" / f).write_text(open(os.path.join(src, f)).read())
    monkeypatch.setattr(ncu_profile, "HERE", str(tmp_path))
    d0 = ncu_profile.source_digest()
    scan = tmp_path / "csrc" / "esc_scan.cu"
    scan.write_text(scan.read_text() + "\n// a note\n/* another\n note */\n\n")
    assert ncu_profile.source_digest() == d0
    scan.write_text(scan.read_text() + "static int esc_extra_symbol;\n")
    assert ncu_profile.source_digest() != d0


def test_algorithmic_bytes_of_a_sub_query():
    import bench
    proj = [("key", "i32"), ("day", "i32"), ("price", "i64")]
    # reads price and code7: 9 B/row; gathers key and day (8 B) per selected row; writes 4 + 16 B
    refs = [("price", "i64"), ("code7", "u8")]
    assert bench.algorithmic_bytes(1000, refs, proj, 10) == 1000 * 9 + 10 * 8 + 10 * 20
    # a count-only call reads the columns alone
    assert bench.algorithmic_bytes(1000, refs, proj, 0) == 9000
