"""CPU checks of the C ABI library: it builds, loads and exports every symbol of include/pm.h."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pm.h")


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(pm_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1207_0486_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("pm_assemble_operator", "pm_pcg_solve", "pm_project_step"):
        assert required in names


def test_library_exports_every_header_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(pm_[a-z0-9_]+)", out))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    import paper_1207_0486_gb300.api as api
    lib = api.load()
    assert set(header_functions()) == set(api.SIGNATURES), set(header_functions()) ^ set(api.SIGNATURES)
    assert lib.pm_kernel_launch_count() == 0
    assert lib.pm_status_string(api.PM_BREAKDOWN) == b"breakdown"


def test_host_side_validation_without_gpu(lib_path):
    """Argument checks run on the host and return PM_EINVAL without touching a GPU."""
    import ctypes

    import numpy as np

    import paper_1207_0486_gb300.api as api
    lib = api.load()
    h = ctypes.c_void_p()
    depth = np.ones((4, 4))
    d = api.MeshDesc(1, 4, 4, 0, 1.0, 1.0, None, depth.ctypes.data)
    ph = api.Physics((ctypes.c_double * 3)(1, 1, 1), 1.0, None)
    assert lib.pm_assemble_operator(ctypes.byref(d), ctypes.byref(ph), ctypes.byref(h), None) == api.PM_EINVAL
    buf = ctypes.create_string_buffer(256)
    lib.pm_last_error(buf, 256)
    assert b">= 2" in buf.value
    # two separate ocean patches -> PM_DISCONNECTED
    mask = np.zeros((6, 9), dtype=np.uint8)
    mask[:, 0:3] = 1
    mask[:, 6:9] = 1
    depth = np.ones((6, 9))
    d = api.MeshDesc(9, 6, 3, 0, 1.0, 1.0, mask.ctypes.data, depth.ctypes.data)
    assert lib.pm_assemble_operator(ctypes.byref(d), ctypes.byref(ph), ctypes.byref(h), None) == api.PM_DISCONNECTED
    # non-positive depth on an ocean column
    mask = np.ones((4, 4), dtype=np.uint8)
    depth = np.ones((4, 4))
    depth[2, 2] = 0.0
    d = api.MeshDesc(4, 4, 3, 0, 1.0, 1.0, mask.ctypes.data, depth.ctypes.data)
    assert lib.pm_assemble_operator(ctypes.byref(d), ctypes.byref(ph), ctypes.byref(h), None) == api.PM_EINVAL
    ph_bad = api.Physics((ctypes.c_double * 3)(1, 1, 1), 0.0, None)
    depth[2, 2] = 1.0
    assert lib.pm_assemble_operator(ctypes.byref(d), ctypes.byref(ph_bad), ctypes.byref(h), None) == api.PM_EINVAL
    # solves and residuals with a null operator or vector
    nb = (ctypes.c_double * 3)()
    assert lib.pm_residual(None, api.OP_PRESSURE, None, None, None, nb, None) == api.PM_EINVAL
    o = api.SolveOpts(1e-8, 100, api.PREC_JACOBI, api.FP64, 0, 3, 0.0)
    assert lib.pm_pcg_solve_noalloc(None, api.OP_PRESSURE, None, None, ctypes.byref(o), None, None) == api.PM_EINVAL
    assert lib.pm_pcg_solve(None, api.OP_PRESSURE, None, None, ctypes.byref(o), None, None) == api.PM_EINVAL
    # state fields, checkpoints and diagnostics without a state
    assert lib.pm_state_field(None, api.FIELD_U1, None, None) == api.PM_EINVAL
    assert lib.pm_state_set_field(None, api.FIELD_U1, None, None) == api.PM_EINVAL
    assert lib.pm_state_set_step_index(None, 3) == api.PM_EINVAL
    assert lib.pm_state_save(None, b"/nonexistent/x.pmck", None) == api.PM_EINVAL
    assert lib.pm_state_load(None, b"/nonexistent/x.pmck", None) == api.PM_EINVAL
    assert lib.pm_state_diagnostics(None, None, nb, None) == api.PM_EINVAL


def test_operator_bytes_scales(lib_path):
    import paper_1207_0486_gb300.api as api
    from workloads import box_basin
    b1 = api.operator_bytes(box_basin(nh=16, nz=8))
    b2 = api.operator_bytes(box_basin(nh=32, nz=8))
    assert b1 > 0 and 3.5 < b2 / b1 < 4.5


def test_server_and_batch_validation_without_gpu(lib_path):
    """The batch and server entry points reject bad arguments on the host, before any CUDA call."""
    import ctypes

    import paper_1207_0486_gb300.api as api
    lib = api.load()
    out = ctypes.c_void_p()

    def opts(**kw):
        return ctypes.byref(api.Options(**{"rtol": 1e-8, "prec": api.PREC_LINE, **kw}).c())

    good = dict(slots=8, nz_cap=32, tile_cols=64, block=128, bps=0)
    bad = [dict(slots=0), dict(slots=5000), dict(nz_cap=1), dict(tile_cols=48), dict(tile_cols=16, block=512),
           dict(bps=-1)]
    for b in bad:
        a = {**good, **b}
        assert lib.pm_server_create(a["slots"], a["nz_cap"], opts(), a["tile_cols"], a["block"], a["bps"],
                                    ctypes.byref(out), None) == api.PM_EINVAL, b
    for o in (opts(prec=7), opts(prec=-1), opts(precision=3), opts(rtol=0.0)):
        assert lib.pm_server_create(8, 32, o, 64, 128, 0, ctypes.byref(out), None) == api.PM_EINVAL
    assert lib.pm_server_create(8, 32, None, 64, 128, 0, ctypes.byref(out), None) == api.PM_EINVAL
    assert lib.pm_server_workspace_bytes(None, api.FP64) == 0
    slot = ctypes.c_int32()
    assert lib.pm_server_admit(None, None, 0, api.PREC_DEFAULT, None, None, None, 0, ctypes.byref(slot),
                               None) == api.PM_EINVAL
    act = ctypes.c_int32()
    assert lib.pm_server_run(None, 16, ctypes.byref(act), None) == api.PM_EINVAL
    n = ctypes.c_int32()
    assert lib.pm_server_poll(None, None, None, 0, ctypes.byref(n)) == api.PM_EINVAL
    assert lib.pm_server_info(None, None, None, None, None, None) == api.PM_EINVAL
    lib.pm_server_destroy(None)
    assert lib.pm_status_string(api.PM_EBUSY).decode() == "no free server slot"

    ops = (ctypes.c_void_p * 2)(None, None)
    which = (ctypes.c_int * 2)(0, 3)
    for count, o in ((0, opts()), (5000, opts()), (2, opts(prec=7)), (2, opts(precision=3)),
                     (2, opts(rtol=-1.0))):
        assert lib.pm_batch_create(ops, which, None, count, o, 0, ctypes.byref(out), None) == api.PM_EINVAL
    for bad in ((0, 9), (0, -2)):    # unknown per-entry preconditioners
        pr = (ctypes.c_int32 * 2)(*bad)
        assert lib.pm_batch_create(ops, which, pr, 2, opts(), 0, ctypes.byref(out), None) == api.PM_EINVAL
    assert lib.pm_batch_solve(None, None, None, None, None) == api.PM_EINVAL
    assert lib.pm_batch_info(None, None, None, None, None) == api.PM_EINVAL
    lib.pm_batch_destroy(None)


def test_log_file_and_build_flags_without_gpu(lib_path, tmp_path):
    """pm_set_log opens (append) and closes the per-solve log on the host; an unopenable path is
    PM_EINVAL and leaves logging off. The default build is not the checked one."""
    import paper_1207_0486_gb300.api as api
    lib = api.load()
    path = tmp_path / "solves.jsonl"
    assert lib.pm_set_log(str(path).encode(), 6800.0) == api.PM_OK
    assert path.exists() and path.read_text() == ""
    assert lib.pm_set_log(None, 0.0) == api.PM_OK
    assert lib.pm_set_log(str(tmp_path / "missing" / "x.jsonl").encode(), 0.0) == api.PM_EINVAL
    assert lib.pm_build_flags() == 0
    assert lib.pm_status_string(api.PM_EBOUNDS) == b"bad index caught by a checked build"
