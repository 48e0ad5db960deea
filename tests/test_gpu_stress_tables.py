"""The paths for full shared-memory tables give the oracle's results.

The defaults size the kernels' tables so that these paths are rare: k_tile
merges an edge in place when its hash is crowded, k_repair repairs a branch
minimum from an overflow bitmap when its list is full and chases a target without a copy
slot along the global chain, k_labels lets a vertex whose chain start found
no slot chase the chain itself. A library built with MT_STRESS_TABLES
shrinks those tables (and nothing else); stress_cases.py runs the parity
cases against it in a child process (MT_LIBRARY) so that these paths carry
most of the work.
"""

from __future__ import annotations

import os
import subprocess
import sys

import pytest

from paper_2301_10838_gb300 import build

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(os.path.abspath(__file__))


def test_stress_tables_equal_oracle():
    lib = build.build(variant="stress", defines=("MT_STRESS_TABLES",))
    env = dict(os.environ, MT_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "stress_cases.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "all cases equal the oracle" in r.stdout
