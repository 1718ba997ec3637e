"""Host arithmetic of the CRT residue products (the library's crt.h) against exact 128-bit integer
products, compiled with the host C++ compiler: no GPU needed."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_crt_arithmetic_exact():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "crt_check")
        subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "native", "crt_check.cpp"), "-o", exe],
                       check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails 0" in r.stdout
