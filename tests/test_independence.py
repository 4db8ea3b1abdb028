"""The oracle and the CUDA path share nothing (CPU): no module or source of the package imports
or includes the oracle, the oracle imports or includes nothing of the package, the shared input
generators import only numpy, scipy and the standard library, and the binding refuses to load
without the compiled library instead of falling back to anything."""
import ast
import glob
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1603_03590_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            mods.add((node.module or "").split(".")[0] if node.level == 0 else ".")
    return mods


def includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), re.M)


def test_package_never_imports_the_oracle():
    files = glob.glob(os.path.join(PKG, "*.py"))
    assert files
    for f in files:
        assert "oracle" not in imported_modules(f), f


def test_cuda_sources_include_nothing_of_the_oracle():
    files = glob.glob(os.path.join(PKG, "csrc", "*.cu")) + glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + \
        glob.glob(os.path.join(PKG, "csrc", "*.h"))
    assert files
    for f in files:
        for inc in includes(f):
            assert "oracle" not in inc, (f, inc)


def test_oracle_uses_nothing_of_the_package():
    for f in glob.glob(os.path.join(ORACLE, "*.py")):
        assert "paper_1603_03590_gb300" not in imported_modules(f), f
    for f in glob.glob(os.path.join(ORACLE, "*.c")) + glob.glob(os.path.join(ORACLE, "*.h")):
        for inc in includes(f):
            assert "/" not in inc and not inc.startswith("dis"), (f, inc)


def test_input_generators_hold_only_library_imports():
    mods = imported_modules(os.path.join(PKG, "synth.py"))
    assert mods <= {"math", "numpy", "scipy"}, mods


def test_binding_refuses_to_load_without_the_library(tmp_path):
    """A copy of the binding next to no libdis.so raises ImportError on import."""
    pkg = tmp_path / "pkgcopy"
    pkg.mkdir()
    shutil.copy(os.path.join(PKG, "dis.py"), pkg / "dis.py")
    (pkg / "__init__.py").write_text("")
    r = subprocess.run([sys.executable, "-c", "import pkgcopy.dis"], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0 and "ImportError" in r.stderr and "libdis.so" in r.stderr, r.stderr


@pytest.mark.parametrize("name", ["bench.py", "__graft_entry__.py"])
def test_oracle_imports_stay_in_the_allowed_places(name):
    """bench.py imports the oracle only inside its CPU legs (the CPU baseline, the reference arm,
    the CPU report and their worker);
    __graft_entry__ only inside build() and smoke()."""
    path = os.path.join(ROOT, name)
    tree = ast.parse(open(path).read(), path)
    allowed = {"bench.py": {"cpu_baseline", "run_reference", "cpu_report", "_oracle_job"},
               "__graft_entry__.py": {"build", "smoke"}}[name]
    for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        for node in ast.walk(fn):
            if isinstance(node, (ast.Import, ast.ImportFrom)):
                mods = {a.name.split(".")[0] for a in node.names} if isinstance(node, ast.Import) \
                    else {(node.module or "").split(".")[0]}
                if "oracle" in mods:
                    assert fn.name in allowed, (name, fn.name)
    top = {a.name.split(".")[0] for n in tree.body if isinstance(n, ast.Import) for a in n.names}
    top |= {(n.module or "").split(".")[0] for n in tree.body if isinstance(n, ast.ImportFrom)}
    assert "oracle" not in top, name
