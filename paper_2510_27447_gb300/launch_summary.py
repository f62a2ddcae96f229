"""Summarise an `ncu --metrics gpu__time_duration.sum --csv` launch list:
per kernel (demangled short name) its launches, total time and share.

usage: python -m paper_2510_27447_gb300.launch_summary <launches.csv> [--markdown]
"""
import csv
import re
import sys
from collections import defaultdict


def short(name: str) -> str:
    m = re.search(r"bd::\(anonymous namespace\)::(\w+)", name)
    if m:
        base = m.group(1)
        for tag in ("TP06", "LR91"):
            if tag in name:
                base += f"<{tag}"
                base += ",float" if "float" in name else ",double"
                mode = re.search(r", \(int\)(\d)>", name) or re.search(r", (\d)>", name)
                if mode and base.startswith("ionic_kernel"):
                    base += f",mode{mode.group(1)}"
                base += ">"
                break
        return base
    if "at::" in name or "at_cuda" in name:
        return "torch:" + re.sub(r"<.*", "", name.split("at::")[-1])[:40]
    return name[:60]


def main(path, markdown=False):
    tot = defaultdict(float)
    cnt = defaultdict(int)
    with open(path) as fh:
        lines = [l for l in fh if l.startswith('"')]
    for row in csv.DictReader(lines):
        if row.get("Metric Name") != "gpu__time_duration.sum":
            continue
        k = short(row["Kernel Name"])
        v = float(row["Metric Value"].replace(",", ""))
        unit = row.get("Metric Unit", "ns")
        scale = {"ns": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3, "nsecond": 1e-3}.get(unit, 1e-3)
        tot[k] += v * scale
        cnt[k] += 1
    all_us = sum(tot.values())
    order = sorted(tot, key=lambda x: -tot[x])
    if markdown:
        print("| kernel | launches | total us | share |")
        print("|---|---|---|---|")
        for k in order:
            print(f"| `{k}` | {cnt[k]} | {tot[k]:.1f} | {100 * tot[k] / all_us:.2f}% |")
        print(f"| TOTAL | {sum(cnt.values())} | {all_us:.1f} | |")
        return
    print(f"{'kernel':52s} {'launches':>8s} {'total us':>12s} {'share':>7s}")
    for k in order:
        print(f"{k:52s} {cnt[k]:8d} {tot[k]:12.1f} {100 * tot[k] / all_us:6.2f}%")
    print(f"{'TOTAL':52s} {sum(cnt.values()):8d} {all_us:12.1f}")


if __name__ == "__main__":
    main(sys.argv[1], markdown="--markdown" in sys.argv[2:])
