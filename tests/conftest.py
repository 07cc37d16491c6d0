import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def _worst(records):
    """Largest error per (test, quantity, precision), with the step it came from."""
    worst = {}
    for r in records:
        key = (r["test"], r["quantity"], r.get("prec", ""))
        if key not in worst or r["err"] > worst[key]["err"]:
            worst[key] = r
    return worst


def pytest_terminal_summary(terminalreporter):
    from parity import RECORDS
    if not RECORDS:
        return
    tr = terminalreporter
    tr.section("measured errors against the FP64 oracle (largest per test and quantity)")
    for (test, q, prec), r in sorted(_worst(RECORDS).items()):
        step = f" step {r['step']}" if "step" in r else ""
        tr.write_line(f"{r['err']:.3e} <= {r['bound']:.1e}  {prec:5s} {q:24s} {test}{step}")


def pytest_sessionfinish(session):
    from parity import RECORDS
    path = os.environ.get("DNNMG_PARITY_LOG")
    if not path or not RECORDS:
        return
    with open(path, "a") as f:
        for r in RECORDS:
            f.write(json.dumps(r) + "\n")
