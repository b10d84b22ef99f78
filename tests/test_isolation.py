"""The oracle and the CUDA path share no code.

The oracle (`oracle/`) is test infrastructure: only the tests, the smoke
check and the benchmark's CPU baseline may use it.  The library (the package,
its native sources and the C headers) never names it, and the oracle never
imports the library or reads its sources, so a parity test compares two
independent implementations.
"""
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent
PRODUCT_SUFFIXES = {".py", ".cpp", ".cu", ".cuh", ".h"}


def _files(folder, suffixes):
    return sorted(p for p in (ROOT / folder).rglob("*") if p.is_file() and p.suffix in suffixes
                  and "__pycache__" not in p.parts and "_build" not in p.parts)


def test_library_never_names_the_oracle():
    files = _files("paper_2106_15740_gb300", PRODUCT_SUFFIXES) + _files("include", {".h"})
    assert files
    for f in files:
        assert not re.search(r"\boracle\b", f.read_text()), f


def test_oracle_never_uses_the_library():
    files = _files("oracle", {".py", ".c", ".h"})
    assert files
    for f in files:
        text = f.read_text()
        assert "paper_2106_15740_gb300" not in text, f
        assert "csrc" not in text and "qtensor" not in text, f


def test_only_tests_smoke_and_baseline_import_the_oracle():
    """Outside tests/ and oracle/, only __graft_entry__.py (the smoke check)
    and bench.py (the CPU baseline and the reference arm) import it."""
    importers = set()
    for f in ROOT.glob("*.py"):
        if re.search(r"^\s*(from|import)\s+oracle\b", f.read_text(), flags=re.M):
            importers.add(f.name)
    assert importers <= {"__graft_entry__.py", "bench.py"}


def test_bench_uses_the_oracle_only_for_its_cpu_arms():
    """In bench.py the oracle is imported by one helper, which only the CPU
    baseline and the reference arm call."""
    import ast
    tree = ast.parse((ROOT / "bench.py").read_text())
    funcs = {n.name: n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)}
    importers = {name for name, fn in funcs.items() for sub in ast.walk(fn)
                 if isinstance(sub, (ast.Import, ast.ImportFrom))
                 and any((getattr(sub, "module", None) or a.name).split(".")[0] == "oracle" for a in sub.names)}
    assert importers == {"_oracle_eval"}
    assert not any(isinstance(n, (ast.Import, ast.ImportFrom)) and "oracle" in ast.dump(n) for n in tree.body)
    callers = {name for name, fn in funcs.items() for sub in ast.walk(fn)
               if isinstance(sub, ast.Name) and sub.id == "_oracle_eval"}
    assert callers <= {"cpu_baseline", "run_reference"}


def test_binding_fails_loudly_without_the_library(tmp_path):
    """A copy of the binding whose shared library is not built raises on
    first use: there is no pure-Python or CPU path behind it."""
    import importlib.util
    import shutil
    import pytest
    pkg = tmp_path / "unbuilt"
    pkg.mkdir()
    shutil.copy(ROOT / "paper_2106_15740_gb300" / "binding.py", pkg / "binding.py")
    spec = importlib.util.spec_from_file_location("unbuilt_binding", pkg / "binding.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with pytest.raises(ImportError, match="not built"):
        mod.lib()


def test_no_cpu_fallback_without_a_gpu(qtlib):
    """On a host without a usable CUDA device an evaluation reports
    QT_ECUDA instead of computing anywhere else.  (Skipped where a device
    exists: the call is given placeholder device pointers.)"""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2106_15740_gb300 import binding as qb
    from workloads import random_regular_graph
    opt = qb.qt_plan_options_default()
    opt.mode = qb.QT_MODE_PERSISTENT
    plan = qb.qt_plan_create(8, random_regular_graph(8, 3, 39), 1, opt)
    try:
        with pytest.raises(qb.QTError) as ei:
            qb.qt_plan_energy_static(plan, 8, 8, 8, 0, 0)
        assert ei.value.status == qb.QT_ECUDA
    finally:
        qb.qt_plan_free(plan)
