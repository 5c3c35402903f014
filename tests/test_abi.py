"""The C-ABI library loads and exports every entry point include/swe.h
declares, and the Python binding's structures have the header's layout.
No compute call is made (this runs without a GPU)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1705_00614_gb300 import build as B
from paper_1705_00614_gb300 import swe

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "swe.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return swe.load()


def declared():
    txt = open(HDR).read()
    return sorted(set(re.findall(r"SWE_API\s+[\w\s\*]*?\b(swe_\w+)\s*\(", txt)))


def test_header_declares_the_api():
    names = declared()
    assert set(names) == set(swe.API), names
    # the entry points the method's problem statement names
    for n in ("swe_create", "swe_set_terrain", "swe_set_sources", "swe_step", "swe_get_state"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (swe_\w+)", out))
    assert set(declared()) <= exported


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(f'''#include <stdio.h>
#include <stddef.h>
#include "{HDR}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(swe_params), offsetof(swe_params, dx),
         offsetof(swe_params, cuda_stream), offsetof(swe_params, seg_h), offsetof(swe_params, skip_dry),
         offsetof(swe_params, ghost_ring), offsetof(swe_params, infil_rate),
         sizeof(swe_step_info),
         offsetof(swe_step_info, wet_cells));
  return 0;
}}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(src)])
    vals = list(map(int, subprocess.check_output([str(exe)]).split()))
    assert vals == [ctypes.sizeof(swe.Params), swe.Params.dx.offset, swe.Params.cuda_stream.offset,
                    swe.Params.seg_h.offset, swe.Params.skip_dry.offset, swe.Params.ghost_ring.offset,
                    swe.Params.infil_rate.offset,
                    ctypes.sizeof(swe.StepInfo),
                    swe.StepInfo.wet_cells.offset]


def test_status_strings_and_defaults(lib):
    assert lib.swe_status_str(0) == b"ok"
    assert lib.swe_status_str(-6) == b"device wait timed out"
    p = swe.Params()
    lib.swe_params_default(ctypes.byref(p))
    assert p.g == 9.81 and p.cfl == 0.3 and p.eps_dry == 1e-4 and p.precision == 0 and p.mode == 0


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    p = swe.Params()
    lib.swe_params_default(ctypes.byref(p))
    h = ctypes.c_void_p()
    for bad in ({"nx": 0, "ny": 4, "dx": 1.0}, {"nx": 4, "ny": 4, "dx": -1.0},
                {"nx": 4, "ny": 4, "dx": 1.0, "cfl": 1.5}, {"nx": 4, "ny": 4, "dx": 1.0, "precision": 7},
                {"nx": 4, "ny": 4, "dx": 1.0, "skip_dry": 2},
                {"nx": 4, "ny": 4, "dx": 1.0, "skip_dry": 1, "mode": swe.SWE_STAGED},
                {"nx": 4, "ny": 4, "dx": 1.0, "ghost_ring": 1, "mode": swe.SWE_STAGED},
                {"nx": 4, "ny": 4, "dx": 1.0, "ghost_ring": 1, "skip_dry": 1},
                {"nx": 4, "ny": 4, "dx": 1.0, "rain_rate": -1e-3}):
        q = swe.Params()
        lib.swe_params_default(ctypes.byref(q))
        for k, v in bad.items():
            setattr(q, k, v)
        assert lib.swe_create(ctypes.byref(q), ctypes.byref(h)) == -1
        assert lib.swe_last_error()


def test_state_calls_reject_null_arguments_before_touching_the_device(lib):
    z = ctypes.c_void_p()
    buf = (ctypes.c_double * 4)()
    t = ctypes.c_double()
    for rc in (lib.swe_set_state_native(None, buf, buf, buf, 0.0),
               lib.swe_set_state_native(z, None, buf, buf, 0.0),
               lib.swe_get_state_native(None, buf, buf, buf, ctypes.byref(t)),
               lib.swe_set_state(None, ctypes.cast(buf, swe._dp), ctypes.cast(buf, swe._dp),
                                 ctypes.cast(buf, swe._dp), 0.0),
               lib.swe_get_state(None, None, None, None, None)):
        assert rc == -1


def test_bounded_wait_check_rejects_bad_limits_before_touching_the_device(lib):
    for bad in (0, -3, 2001):
        assert lib.swe_check_bounded_wait(bad) == -1
