"""Small-case ncu captures of the scan and write kernels, and their summary.

The counters that need more than one profiler pass (DRAM bytes) are taken
on a small case of the headline workload: its 200 predicates on an 8M-row
skewed table (256 MB of columns, larger than L2), each counted once, then
materialised once (scan + write), so that a capture is a few hundred short
launches that ends by itself.  The summary is a small JSON file that
bench.py reads: per kernel and mode, launches, mean duration and mean DRAM
bytes per launch and per table row, with the digest of the kernel source
measured (a figure is used only while the source is unchanged); DRAM bytes
per row scale linearly with the table size (the same generator and the same
selectivities at every size).

    python -m paper_1901_01488_gb300.ncu_profile workload --rows 8000000
    ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum \\
        --clock-control none -k regex:'scan_kernel|write_kernel' --csv \\
        --log-file scan_8m.csv \\
        python -m paper_1901_01488_gb300.ncu_profile workload --rows 8000000
    python -m paper_1901_01488_gb300.ncu_profile summarise scan_8m.csv \\
        --rows 8000000 --out profiles/scan_kernel.skewed_8m_200preds.json
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
import sys
from collections import defaultdict

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SUMMARY = os.path.join(ROOT, "profiles", "scan_kernel.skewed_8m_200preds.json")


def source_digest() -> str:
    """Digest of the scan and write kernels' code: comments removed and
    whitespace collapsed, so that a comment edit keeps a profile valid."""
    h = hashlib.sha256()
    for p in (os.path.join(HERE, "csrc", "esc_scan.cu"), os.path.join(HERE, "csrc", "esc_internal.h")):
        with open(p) as f:
            code = re.sub(r"/\*.*?\*/", " ", f.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def workload(rows: int, preds: int = 200) -> None:
    """The launches a capture sees: `preds` count calls, then `preds`
    materialising calls (capacity = the count)."""
    import torch
    sys.path.insert(0, ROOT)
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import datagen, esc
    t = datagen.skewed_table(rows, seed=2, device="cuda")
    tbl = esc.Table.from_datagen(t)
    ps = [esc.Predicate(tbl, p.text, datagen.SKEWED_PROJECTION) for p in datagen.skewed_predicates(preds)]
    counts = [esc.count(tbl, p) for p in ps]
    for p, c in zip(ps, counts):
        esc.esc_selectivity(tbl.handle, p.handle, p.alloc_rows(max(1, c)))
    torch.cuda.synchronize()
    print("launches: %d count, %d materialising" % (len(ps), len(ps)))


def mlp_workload(samples: int) -> None:
    """The surrogate's kernels for a capture: one forward pass over `samples`
    rows of 64 bfloat16 features (128 bytes a row), then one gradient pass
    over the same rows and one Adam step."""
    import torch
    sys.path.insert(0, ROOT)
    from paper_1901_01488_gb300 import build
    build.build()
    from paper_1901_01488_gb300 import esc, surrogate
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(samples, surrogate.NFEAT, device="cuda", generator=g).to(torch.bfloat16).view(torch.int16)
    y = torch.randn(samples, device="cuda", generator=g)
    m = surrogate.Surrogate(esc, seed=3)
    m.predict(x)
    grad = torch.zeros_like(m.params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    esc.esc_mlp_grad(x, y, m.wbf, m.params, grad, loss)
    esc.esc_mlp_adam(m.params, m.wbf, grad, m.m, m.v, 1e-3, 1)
    torch.cuda.synchronize()
    print("mlp launches: forward, gradient, adam over %d samples" % samples)


def _read_ncu_csv(path: str):
    """Rows of ncu --csv output: (launch id, kernel name, metric, value)."""
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    out = []
    for r in csv.DictReader(lines):
        try:
            v = float(r["Metric Value"].replace(",", ""))
        except (KeyError, ValueError):
            continue
        unit = r.get("Metric Unit", "")
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9,
                 "ns": 1e-3, "nsecond": 1e-3, "us": 1, "usecond": 1, "ms": 1e3, "msecond": 1e3,
                 "s": 1e6, "second": 1e6}.get(unit, 1)   # durations in microseconds
        out.append((int(r["ID"]), r["Kernel Name"], r["Metric Name"], v * scale))
    return out


def summarise(csv_path: str, rows: int, out_path: str, command: str) -> dict:
    per = defaultdict(dict)
    names = {}
    for lid, name, metric, value in _read_ncu_csv(csv_path):
        per[lid][metric] = value
        names[lid] = name
    scans = [i for i in sorted(per) if "scan_kernel" in names[i]]
    writes = [i for i in sorted(per) if "write_kernel" in names[i]]
    npred = len(writes)
    groups = {"scan_kernel (count)": scans[:len(scans) - npred], "scan_kernel (materialise)": scans[len(scans) - npred:],
              "write_kernel": writes}

    def stats(ids):
        if not ids:
            return None
        dram = [per[i].get("dram__bytes_read.sum", 0) + per[i].get("dram__bytes_write.sum", 0) for i in ids]
        t = [per[i].get("gpu__time_duration.sum", 0) for i in ids]
        return {"launches": len(ids), "time_us_mean": sum(t) / len(ids), "time_us_total": sum(t),
                "dram_bytes_per_launch": sum(dram) / len(ids), "dram_bytes_per_row": sum(dram) / len(ids) / rows}

    kern = {k: stats(v) for k, v in groups.items()}
    sel = kern["scan_kernel (materialise)"]
    wr = kern["write_kernel"]
    call = None
    if sel and wr:
        call = {"dram_bytes_per_row": sel["dram_bytes_per_row"] + wr["dram_bytes_per_row"],
                "time_us_mean": sel["time_us_mean"] + wr["time_us_mean"],
                "shares": {"scan_kernel": sel["time_us_total"] / (sel["time_us_total"] + wr["time_us_total"]),
                           "write_kernel": wr["time_us_total"] / (sel["time_us_total"] + wr["time_us_total"])}}
    out = {"what": "ncu DRAM bytes and durations (cold cache, serialised launches) of the headline's 200 "
                   "predicates on a %d-row skewed table: count calls, then materialising calls" % rows,
           "command": command, "rows": rows, "source_digest": source_digest(), "kernels": kern,
           "materialising_call": call}
    with open(out_path, "w") as f:
        json.dump(out, f, indent=1)
    return out


def traffic_per_row(key: str):
    """DRAM bytes per table row from the committed summary: key "count" (the
    scan kernel of a count call) or "call" (scan + write of a materialising
    call); None when the summary is missing or the kernel source changed."""
    try:
        with open(SUMMARY) as f:
            s = json.load(f)
    except (OSError, ValueError):
        return None
    if s.get("source_digest") != source_digest():
        return None
    if key == "count":
        k = s["kernels"].get("scan_kernel (count)")
        return k and k["dram_bytes_per_row"]
    c = s.get("materialising_call")
    return c and c["dram_bytes_per_row"]


def main() -> None:
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    w = sub.add_parser("workload")
    w.add_argument("--rows", type=int, default=8_000_000)
    w.add_argument("--preds", type=int, default=200)
    mw = sub.add_parser("mlp")
    mw.add_argument("--samples", type=int, default=1_000_000)
    s = sub.add_parser("summarise")
    s.add_argument("csv")
    s.add_argument("--rows", type=int, default=8_000_000)
    s.add_argument("--out", default=SUMMARY)
    s.add_argument("--command", default="")
    a = ap.parse_args()
    if a.cmd == "workload":
        workload(a.rows, a.preds)
    elif a.cmd == "mlp":
        mlp_workload(a.samples)
    else:
        print(json.dumps(summarise(a.csv, a.rows, a.out, a.command), indent=1))


if __name__ == "__main__":
    main()
