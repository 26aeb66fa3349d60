"""The oracle and the CUDA path share nothing, and the product never reaches the oracle.

Checked on the sources: no file of the package (Python, CUDA, C++ or headers) imports, includes,
loads or names the oracle; no oracle file imports the package or includes the library's headers;
outside the tests, only the smoke check and the benchmark's CPU-baseline / reference code load
the oracle.  And the binding refuses to run without its compiled library (no CPU fallback)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1305_6861_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or os.sep + "lib" in d[len(top):]:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _code(path):
    src = open(path, encoding="utf-8").read()
    if path.endswith(".py"):  # drop docstrings and comments, keep code
        tree = ast.parse(src)
        for node in ast.walk(tree):
            body = getattr(node, "body", None)
            if isinstance(body, list) and body and isinstance(body[0], ast.Expr) \
                    and isinstance(getattr(body[0], "value", None), ast.Constant) and isinstance(body[0].value.value, str):
                body[0] = ast.Pass()
        return ast.unparse(tree)
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    return re.sub(r"//[^\n]*", " ", src)


def test_package_never_reaches_the_oracle():
    bad = []
    for f in _files(PKG, (".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
        code = _code(f)
        if re.search(r"\boracle\b", code):
            bad.append(os.path.relpath(f, ROOT))
    assert not bad, bad


def test_oracle_does_not_use_the_library():
    bad = []
    for f in _files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        code = _code(f)
        if re.search(r"paper_1305_6861_gb300|mrsim\.h|libmrsim|csrc", code):
            bad.append(os.path.relpath(f, ROOT))
    assert not bad, bad


def test_oracle_users_outside_tests():
    """__graft_entry__ loads it in build() (to compile it) and smoke(); bench.py only inside its
    CPU-baseline legs (the timed sample, the oracle-parity sample) and reference-arm code."""
    allowed = {"__graft_entry__.py": {"build", "smoke"},
               "bench.py": {"cpu_baseline", "cpu_baseline_parity_run", "cpu_baseline_fields", "run_adjoint", "run_kt"}}
    for name, funcs in allowed.items():
        tree = ast.parse(open(os.path.join(ROOT, name), encoding="utf-8").read())
        users = set()
        for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                    users.add(fn.name)
                if isinstance(node, ast.ImportFrom) and (node.module or "").split(".")[0] == "oracle":
                    users.add(fn.name)
        top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
        assert not any((isinstance(n, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in n.names))
                       or (isinstance(n, ast.ImportFrom) and (n.module or "").split(".")[0] == "oracle")
                       for n in top), name
        assert users <= funcs, (name, users)
    # in run_adjoint / run_kt the import sits under the `not args.no_cpu_baseline` branch
    tree = ast.parse(open(os.path.join(ROOT, "bench.py"), encoding="utf-8").read())
    for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef) and n.name in ("run_adjoint", "run_kt")]:
        guarded = set()
        for br in [n for n in ast.walk(fn) if isinstance(n, ast.If) and "no_cpu_baseline" in ast.unparse(n.test)]:
            guarded |= {id(x) for x in ast.walk(br)}
        for node in ast.walk(fn):
            if isinstance(node, (ast.Import, ast.ImportFrom)) and "oracle" in ast.unparse(node):
                assert id(node) in guarded, fn.name


def test_binding_has_no_fallback(monkeypatch, tmp_path):
    from paper_1305_6861_gb300 import mrsim as M

    monkeypatch.setattr(M, "_lib", None)
    monkeypatch.setattr(M, "LIB_PATH", str(tmp_path / "libmrsim.so"))
    with pytest.raises(RuntimeError, match="missing"):
        M.lib()
