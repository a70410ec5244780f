import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libbm.so")


def pytest_terminal_summary(terminalreporter):
    """Parity figures recorded by the GPU tests (flip counts inside and
    outside the 1e-6 window, hard-gate mismatches, round-off margins)."""
    import json

    try:
        from _util import PARITY_RECORDS
    except ImportError:
        return
    if not PARITY_RECORDS:
        return
    terminalreporter.write_sep("-", "parity records")
    for r in PARITY_RECORDS:
        terminalreporter.write_line(json.dumps(r, sort_keys=True))
    path = os.environ.get("BM_PARITY_LOG")
    if path:
        with open(path, "w") as f:
            json.dump(PARITY_RECORDS, f, indent=1, sort_keys=True)
