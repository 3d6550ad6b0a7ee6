import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: large CPU case")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Parity summary: for the A/b checks of this run, the worst cancellation-aware error (the
    asserted quantity), the worst plain relative error |gpu - oracle| / |oracle|, that error over
    the entries whose contributions cancel by at most 10x (scale <= 10 |oracle|), and the
    share of entries that cancel more. EEC_PARITY_LOG=<path> also writes the records as JSON."""
    try:
        from helpers import PARITY_LOG
    except Exception:  # pragma: no cover
        return
    if not PARITY_LOG:
        return
    import json
    by = {}
    for r in PARITY_LOG:
        a = by.setdefault(r["test"], dict(checks=0, entries=0, max_err=0.0, max_plain=0.0,
                                          max_plain_well=0.0, p99_ratio=0.0, max_ratio=0.0,
                                          frac_ratio_gt10=0.0))
        a["checks"] += 1
        a["entries"] += r["n"]
        for k in ("max_err", "max_plain", "max_plain_well", "p99_ratio", "max_ratio",
                  "frac_ratio_gt10"):
            a[k] = max(a[k], r.get(k, 0.0))
    tr = terminalreporter
    tr.write_sep("-", "parity summary (A, b entries against the oracle)")
    tr.write_line(f"{'max err':>9} {'max plain':>9} {'plain|<=10':>10} {'p99 S/|e|':>9} "
                  f"{'>10 share':>9}  test")
    for t, a in sorted(by.items()):
        tr.write_line(f"{a['max_err']:9.1e} {a['max_plain']:9.1e} {a['max_plain_well']:10.1e} "
                      f"{a['p99_ratio']:9.2f} {a['frac_ratio_gt10']:9.2e}  {t}")
    path = os.environ.get("EEC_PARITY_LOG")
    if path:
        with open(path, "w") as f:
            json.dump(by, f, indent=1, sort_keys=True)
