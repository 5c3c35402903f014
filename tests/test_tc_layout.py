"""The tensor-core convolution's shared-memory matrix descriptors, checked on
the host: tests/tc_layout_check.cpp decodes every descriptor the kernel
issues and compares each element an MMA reads with where the kernel's
staging loop stored it (and that it lies inside the staged buffer)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_conv_descriptors_address_the_staged_elements(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "tc_layout_check"
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-o", str(exe), os.path.join(HERE, "tc_layout_check.cpp")])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip().endswith("ok"), out.stdout
