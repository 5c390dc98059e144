"""The C ABI library loads, exports every function include/fricp.h declares, and
the Python binding's ctypes structures match the header's layout (CPU only: no
compute call is made)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fricp.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(fricp_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def libfricp():
    from paper_2007_07627_gb300 import build
    build.build()
    import paper_2007_07627_gb300 as fr
    return fr.lib()


def test_every_declared_symbol_is_exported(libfricp):
    names = _declared()
    assert "fricp_register" in names and "fricp_target_create" in names
    missing = [n for n in names if not hasattr(libfricp, n)]
    assert not missing, missing


def test_struct_layout_matches_header():
    import paper_2007_07627_gb300 as fr
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "fricp.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(fricp_params), sizeof(fricp_result),
         offsetof(fricp_params, timeout_s), offsetof(fricp_result, wall_ms),
         offsetof(fricp_result, status), offsetof(fricp_result, nu_max),
         sizeof(fricp_step_record), offsetof(fricp_step_record, T), offsetof(fricp_step_record, result));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(fr.Params)
    assert vals[1] == ctypes.sizeof(fr.Result)
    assert vals[2] == fr.Params.timeout_s.offset
    assert vals[3] == fr.Result.wall_ms.offset
    assert vals[4] == fr.Result.status.offset
    assert vals[6] == ctypes.sizeof(fr.StepRecord)
    assert vals[7] == fr.StepRecord.T.offset and vals[8] == fr.StepRecord.result.offset
    assert vals[5] == fr.Result.nu_max.offset


def test_defaults_and_argument_errors_without_gpu(libfricp):
    """Calls that validate arguments before touching the device."""
    import paper_2007_07627_gb300 as fr
    p = fr.params_default("p2pl_welsch")
    assert (p.anderson_m, p.max_iters, p.p2pl_iters_first, p.p2pl_iters_cap, p.eps) == (5, 1000, 6, 10, 1e-5)
    with pytest.raises(fr.FricpError) as e:
        fr.params_default(7)
    assert e.value.status == 1
    out = ctypes.c_void_p()
    assert libfricp.fricp_target_create(None, None, 10, 0, None, ctypes.byref(out)) == 1
    assert b"NULL" in libfricp.fricp_last_error()
    assert libfricp.fricp_target_destroy(None) == 0


def test_batch_shape_override_argument_checks(libfricp):
    import paper_2007_07627_gb300 as fr
    for bad in ((3, 1, 0), (512, 1, 0), (2, 0, 0), (2, 1, 3), (2, 1, -1), (-1, 1, 0)):
        assert libfricp.fricp_batch_set_shape(*bad) == 1   # FRICP_EINVAL
    fr.batch_set_shape(4, 2, True)
    fr.batch_set_shape(8, 2, 2)   # query tiles
    fr.batch_set_shape(0)   # back to autotuning
