import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: long-running case")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    """Parse a hand-derived fixture: n, events (u v t), expected out-components
    (``oc``) and optionally expected in-components (``rows``)."""
    n, events, oc, rows, section = None, [], {}, {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("n "):
                n = int(line.split()[1])
            elif line in ("events", "oc", "rows"):
                section = line
            elif section == "events":
                a, b, t = line.split()
                events.append((int(a), int(b), int(t)))
            else:
                key, vals = line.split(":")
                target = oc if section == "oc" else rows
                target[int(key)] = sorted(int(x) for x in vals.split())
    return n, events, oc, rows


def golden_names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
