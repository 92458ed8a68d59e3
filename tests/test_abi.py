"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol
declared in include/*.h; the binding refuses to run without it (no CPU fallback)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(csp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for f in ("csp_create_lattice", "csp_destroy_lattice", "csp_solve", "csp_solve_async", "csp_status_string"):
        assert f in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1511_06441_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_symbols() - exported
    assert not missing, missing
    import ctypes
    lib = ctypes.CDLL(path)  # loads on a machine without a GPU
    for name in declared_symbols():
        assert hasattr(lib, name)
    lib.csp_status_string.restype = ctypes.c_char_p
    assert lib.csp_status_string(4) == b"flow pool capacity exceeded"


def test_binding_has_no_fallback(monkeypatch, tmp_path):
    from paper_1511_06441_gb300 import csp
    monkeypatch.setattr(csp, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(csp, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        csp.lib()


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1511_06441_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "csp_oracle" not in text, path


def test_product_is_not_imported_by_the_oracle():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if path.endswith((".py", ".c", ".h")):
            text = open(path).read()
            assert "import paper_1511_06441_gb300" not in text and "from paper_1511_06441_gb300" not in text, path
            assert "csp_device" not in text and '#include "csp' not in text and "libcsp" not in text, path


def test_shape_flags_from_the_cached_choice(tmp_path, monkeypatch):
    from paper_1511_06441_gb300 import build
    assert build.shape_flags({}) == ["-DCSP_TPB=512", "-DCSP_IPT=4", "-DCSP_NSTAGE=3", "-DCSP_MIN_CTAS_PER_SM=2",
                                     "-DCSP_BATCH_MIN_CTAS_PER_SM=1"]
    f = tmp_path / "shape.json"
    f.write_text('{"chosen": {"tpb": 256, "ipt": 8, "nstage": 2, "min_ctas_per_sm": 4, "batch_min_ctas_per_sm": 2}}')
    monkeypatch.setattr(build, "SHAPE_JSON", str(f))
    assert build.shape_flags() == ["-DCSP_TPB=256", "-DCSP_IPT=8", "-DCSP_NSTAGE=2", "-DCSP_MIN_CTAS_PER_SM=4",
                                   "-DCSP_BATCH_MIN_CTAS_PER_SM=2"]
    with pytest.raises(ValueError):
        build.shape_flags({"tpb": 0})


def test_library_reports_its_build_shape():
    import ctypes
    from paper_1511_06441_gb300 import build
    lib = ctypes.CDLL(build.build())
    out = (ctypes.c_int32 * 5)()
    lib.csp_build_shape(out)
    assert [f"-D{m}={v}" for (m, _), v in zip(build.SHAPE_KEYS.values(), out)] == build.shape_flags()
