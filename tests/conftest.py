import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: full-size workloads (minutes of CPU time)")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Parse a golden fixture: '# ...' comments, 'key: value' headers, then a 'trace:' block."""
    hdr, trace, in_trace = {}, [], False
    with open(os.path.join(GOLDEN, name), encoding="latin-1") as f:
        for line in f:
            line = line.rstrip("\n")
            if line.startswith("#") or (not line and not in_trace):
                continue
            if in_trace:
                trace.append(line)
            elif line == "trace:":
                in_trace = True
            else:
                k, v = line.split(":", 1)
                hdr[k.strip()] = v.strip()
    return hdr, trace
