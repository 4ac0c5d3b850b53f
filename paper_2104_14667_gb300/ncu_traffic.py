"""DRAM traffic per launch of the accumulation kernel, from an ncu metrics
capture, written as a small JSON record that bench.py reports as
roofline.traffic.

The capture is taken on a small case of the same kernel (ncu replays a
launch once per pass and saves device memory around the passes, so the full
workload is not captured).  Member bytes grow with the member count, the
composite plane's bytes do not, so the full-size traffic is

    captured bytes - captured members x raster bytes + full members x raster bytes

Usage (after a capture with --csv --log-file of dram__bytes_read.sum,
dram__bytes_write.sum and gpu__time_duration.sum):

    python -m paper_2104_14667_gb300.ncu_traffic CSV --kernel count_linear \\
        --width 4096 --height 4096 --captured-members 64 --members 1024 \\
        --command "the ncu command line" --out profiles/FILE.json
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# the sources the linear count kernel is built from
KERNEL_SOURCES = ("count_kernels.cu", "device_common.cuh")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2104_14667_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def read_metrics(path: str, kernel: str) -> dict:
    """Metric name -> value (float) of the first launch whose kernel name
    contains `kernel`, from ncu's CSV log (one row per metric)."""
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    rows = list(csv.DictReader(lines))
    out: dict = {}
    first_id = None
    for r in rows:
        if kernel not in r.get("Kernel Name", ""):
            continue
        if first_id is None:
            first_id = r["ID"]
        if r["ID"] != first_id:
            break
        unit = r.get("Metric Unit", "")
        v = float(r["Metric Value"].replace(",", ""))
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-3, "ns": 1e-3,
                 "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3}.get(unit, 1.0)
        out[r["Metric Name"]] = v * scale
    if not out:
        raise ValueError(f"no launch of a kernel matching {kernel!r} in {path}")
    return out


def summarize(path: str, kernel: str, width: int, height: int, captured_members: int, members: int,
              command: str) -> dict:
    m = read_metrics(path, kernel)
    captured = m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"]
    raster = width * height
    full = captured - captured_members * raster + members * raster
    return {"kernel": kernel, "workload": f"{width}x{height}x{members}",
            "kernel_source_sha256_16": kernel_source_hash(),
            "captured_members": captured_members, "captured_dram_bytes": captured,
            "captured_duration_us": m.get("gpu__time_duration.sum"),
            "dram_bytes_per_launch": full, "command": command}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("csv")
    ap.add_argument("--kernel", default="count_linear")
    ap.add_argument("--width", type=int, default=4096)
    ap.add_argument("--height", type=int, default=4096)
    ap.add_argument("--captured-members", type=int, required=True)
    ap.add_argument("--members", type=int, required=True)
    ap.add_argument("--command", default="")
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    rec = summarize(a.csv, a.kernel, a.width, a.height, a.captured_members, a.members, a.command)
    with open(a.out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
