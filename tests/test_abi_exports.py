"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import glob
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pd_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for n in ["pd_plan_create", "pd_kernel_spectrum", "pd_force", "pd_step_verlet", "pd_solve_static",
              "pd_force_adjoint", "pd_plan_destroy", "pd_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2105_06055_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for name in sorted(_declared()):
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert _declared() <= exported
    # pure host calls work without a GPU
    lib.pd_status_string.restype = ctypes.c_char_p
    assert lib.pd_status_string(0) == b"ok"
    assert lib.pd_status_string(-5) == b"not converged"


def test_binding_names_match_header():
    from paper_2105_06055_gb300 import pd
    assert set(pd.EXPORTS) == _declared()
