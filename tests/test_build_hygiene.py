"""Build hygiene of the CUDA library (no GPU needed).

nvcc silently replaces a kernel launch in host template code by an ``exit(1)``
stub when the launch expression calls a device-only helper; the library must
therefore never import ``exit``.
"""
import os
import shutil
import subprocess

import pytest


def test_library_never_calls_exit():
    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    from paper_2501_03245_gb300 import build

    path = build.build()
    out = subprocess.run(["nm", "-D", "--undefined-only", path], capture_output=True, text=True).stdout
    undefined = {line.split()[-1].split("@")[0] for line in out.splitlines() if line.strip()}
    assert "exit" not in undefined and "_exit" not in undefined
