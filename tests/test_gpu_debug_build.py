"""The debug build of the library (-DLDPC_DEBUG: every edge offset a kernel
reads is checked against the posterior region and a bad one is reported
through ldpc_sync) decodes bit-exactly with no check firing."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu


def test_debug_build_decodes_clean():
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, os.path.join(here, "debug_build_check.py")],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug build ok" in r.stdout
