"""The KADABRA_CHECKED build (GPU only, slow): the library compiled with an
index check at every list, frontier-array, level-bound, adjacency and
hit-counter access of the sampler runs the forced-tier parity cases of
checked_cases.py in a child process; no check may fail and every result must
equal the oracle's.  It stands in for a memory checker, which this GPU pool
does not offer."""

import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_finds_no_bad_index():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1604_08553_gb300 import _build
    lib = _build.build_checked()
    out = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), lib], capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "checked build:" in out.stdout
