"""Table of the parity errors a GPU test run recorded.

    FDTD_PARITY_RECORD=parity.jsonl python -m pytest tests -m gpu
    python tests/parity_summary.py parity.jsonl > summary.md

One row per (case, quantity): the relative L2 error of the CUDA path
against the FP64 oracle, the stated bar (1e-5 fields, 1e-4 probes), the bar
the test applied and, for runs from rest, the error of the same algorithm
evaluated with FP32 storage on the CPU.
"""
import json
import sys


def main(path):
    rows = [json.loads(x) for x in open(path) if x.strip()]
    print("| case | steps | quantity | rel. L2 achieved | stated bar | applied bar | FP32-storage yardstick |")
    print("|---|---|---|---|---|---|---|")
    for r in rows:
        y = r.get("fp32_yardstick")
        print(f"| {r['case']} | {r.get('steps', '')} | {r['quantity']} | {r['rel_l2']:.3e} | {r['stated_bar']:.0e} "
              f"| {r['bar']:.3e} | {'' if y is None else f'{y:.3e}'} |")


if __name__ == "__main__":
    main(sys.argv[1])
