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


def test_problem_struct_layout_matches_header(tmp_path):
    """The binding's ctypes pd_problem has the size and field offsets that a C
    compiler gives the header's struct (the struct crosses the ABI by pointer)."""
    from paper_2105_06055_gb300 import pd
    fields = [f[0] for f in pd._Problem._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"pd.h\"\nint main(void){\n"
                   + 'printf("%zu\\n", sizeof(pd_problem));\n'
                   + "".join(f'printf("%zu\\n", offsetof(pd_problem, {f}));\n' for f in fields)
                   + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(pd._Problem)
    assert got[1:] == [getattr(pd._Problem, f).offset for f in fields]


def test_volume_rule_arguments_are_checked_on_the_host():
    """The quadrature-rule and cell-shape checks return PD_ERR_ARG before any
    device work, so they run without a GPU."""
    from paper_2105_06055_gb300 import build, pd
    build.build()
    lib = pd.load()
    buf = (ctypes.c_uint8 * 64)()
    ptr = ctypes.cast(buf, ctypes.c_void_p)

    def create(**kw):
        prob = pd.Problem(shape=(64, 64), delta=3.0, **kw).to_c()
        h = ctypes.c_void_p()
        st = lib.pd_plan_create(ctypes.byref(prob), ptr, None, None, ctypes.byref(h))
        return st, lib.pd_last_error_detail().decode()

    st, msg = create(volume_rule=2)
    assert st == -1 and "volume_rule" in msg
    st, msg = create(volume_rule=1, dx=(1.0, 1.1))
    assert st == -1 and "cubic cells" in msg
    prob = pd.Problem(shape=(64, 64), delta=3.0, volume_rule=1).to_c()
    st = lib.pd_force2d_noalloc(ctypes.byref(prob), ptr, ptr, ptr, None)
    assert st == -1 and "volume_rule" in lib.pd_last_error_detail().decode()


def test_tuning_widths_are_checked_on_the_host():
    """pd_plan_set_tuning refuses a column-tile width of 1 (and other bad values)
    before it touches the plan: a one-column tile would start tensor copies off
    a 16-byte boundary."""
    from paper_2105_06055_gb300 import build, pd
    build.build()
    lib = pd.load()
    dummy = (ctypes.c_uint8 * 4096)()  # never read: the arguments are refused first
    for bad in [(0, 1, 0, 0, 0, 0), (0, 0, 1, 0, 0, 0), (0, 64, 0, 0, 0, 0), (3, 0, 0, 0, 0, 0),
                (0, 0, 0, 2, 0, 0), (0, 0, 0, 0, 3, 0)]:
        arr = (ctypes.c_int * 6)(*bad)
        assert lib.pd_plan_set_tuning(ctypes.cast(dummy, ctypes.c_void_p), arr) == -1, bad
    assert "widths 2..32" in lib.pd_last_error_detail().decode()
    assert not any(dummy)


def test_binding_plan_queries_are_properties():
    """Plan queries that the tests and the bench read as attributes stay properties."""
    from paper_2105_06055_gb300 import pd
    for name in ("stable_dt", "critical_energy", "boundary_nodes", "launch_count", "workspace_bytes", "tuning"):
        assert isinstance(getattr(pd.Plan, name), property), name
