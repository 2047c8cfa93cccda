"""The C-ABI library builds for sm_103a and exports every function include/rt.h declares.

No compute calls are made (no GPU is needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_0908_2654_gb300 import _rt
    if not os.path.exists(_rt.LIB_PATH):
        import importlib
        importlib.import_module("paper_0908_2654_gb300.build").build()
    return _rt.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rt_init_grid", "rt_implicit_step", "rt_adjoint_step", "rt_destroy_grid", "rt_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rt_[a-z_0-9]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_error_strings(libpath):
    from paper_0908_2654_gb300 import _rt
    try:
        L = _rt.lib()
    except OSError as e:   # the CUDA runtime may be absent on a machine without a driver
        pytest.skip(f"library not loadable here: {e}")
    for name in declared_functions():
        assert hasattr(L, name)
    assert L.rt_error_string(_rt.RT_ENOCONV).decode().startswith("Newton")
    assert _rt.GridDesc in (type(_rt.GridDesc()),)
    # the ctypes mirrors have the field order of the header structs
    hdr = open(HEADER).read()
    for field in ("newton_tol", "lin_rtol", "mg_nu1", "stream"):
        assert field in hdr and field in [f for f, _ in _rt.GridDesc._fields_]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built library the binding raises instead of computing."""
    from paper_0908_2654_gb300 import _rt
    monkeypatch.setattr(_rt, "LIB_PATH", str(tmp_path / "librtfld.so"))
    monkeypatch.setattr(_rt, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _rt.lib()


def test_solver_without_a_gpu_raises():
    """On a machine without a GPU the solver refuses to run (no CPU path exists)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import workloads as W
    from paper_0908_2654_gb300.solver import Solver
    with pytest.raises(Exception):
        Solver(W.stromgren_static(n=8), precision="fp64")


def test_ctypes_mirrors_match_the_c_struct_layouts(tmp_path):
    """Every struct of include/rt.h has, in the Python binding, the same size and the same
    offset for every field (compiled with the host C compiler)."""
    import json
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_layout")
    subprocess.run([cc, "-std=c99", "-o", exe, os.path.join(ROOT, "tests", "host", "abi_layout.c")], check=True)
    layout = json.loads(subprocess.run([exe], capture_output=True, text=True, check=True).stdout)
    from paper_0908_2654_gb300 import _rt
    mirrors = {"rt_grid_desc": _rt.GridDesc, "rt_step_inputs": _rt.StepInputs, "rt_state": _rt.State,
               "rt_step_stats": _rt.StepStats, "rt_kernel_profile": _rt.KernelProfile}
    for cname, py in mirrors.items():
        c = layout[cname]
        assert ctypes.sizeof(py) == c["__size__"], cname
        fields = [f for f, _ in py._fields_]
        assert sorted(fields) == sorted(k for k in c if not k.startswith("__")), cname
        for f in fields:
            assert getattr(py, f).offset == c[f], (cname, f)
