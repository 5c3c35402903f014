"""The tensor-core kernels' shared-memory matrix descriptors, checked on the
host.  tests/tc_layout_check.cpp decodes every descriptor the convolution
issues and compares each element an MMA reads with where the kernel's
staging loop stored it (and that it lies inside the staged buffer).
tests/wgrad_layout_check.cpp simulates one weight-gradient CTA on a small
ragged image with the kernel's staging offsets, copy split and descriptor
builders, and compares the accumulators, read back with the kernel's row
map, with the weight and bias gradients summed from their definition.
tests/row_plan_check.cpp checks the work plan both persistent kernels use:
every image row of every column band in exactly one item, every item in
exactly one CTA, one pass of the CTAs whenever the items could grow."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _run_check(tmp_path, name):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / name
    subprocess.check_call([cxx, "-std=c++17", "-O2", "-o", str(exe), os.path.join(HERE, name + ".cpp")])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip().endswith("ok"), out.stdout


def test_conv_descriptors_address_the_staged_elements(tmp_path):
    _run_check(tmp_path, "tc_layout_check")


def test_weight_gradient_layout_reproduces_the_gradient(tmp_path):
    _run_check(tmp_path, "wgrad_layout_check")


def test_row_plan_covers_every_row_once(tmp_path):
    _run_check(tmp_path, "row_plan_check")
