import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size parity case")


def golden_rows(name):
    """Non-comment rows of a golden fixture, split on whitespace."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def golden_directives(name, tag):
    """Rows of the form '#<tag> a b c' in a golden fixture."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#" + tag + " "):
                rows.append(line[len(tag) + 1:].split())
    return rows


# Numbers the parity tests measure (error against the FP64 oracle per result, near-ties
# followed in lock step), printed at the end of the run.
PARITY_REPORT = {}


def report(key, value):
    PARITY_REPORT[key] = value


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    if not PARITY_REPORT:
        return
    terminalreporter.section("parity report (error against the FP64 oracle)")
    for k in sorted(PARITY_REPORT):
        terminalreporter.write_line(f"{k}: {PARITY_REPORT[k]}")
