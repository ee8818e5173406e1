"""Static checks of the boundary between the library and its test oracle (CPU, no GPU).

The oracle exists only to check the library: the library never imports, links or includes
it, and the oracle never touches the library.  Outside the tests, only the smoke check and
build step of __graft_entry__.py and the CPU-baseline / reference legs of bench.py may load
it, and those load it inside the functions that need it, never at module level.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1703_03637_gb300")


def _files(top, exts):
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if d not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def _imported_modules(tree):
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield node, a.name.split(".")[0]
        elif isinstance(node, ast.ImportFrom) and node.module:
            yield node, node.module.split(".")[0]


def test_library_never_loads_the_oracle():
    for path in _files(PKG, (".py",)):
        mods = {m for _, m in _imported_modules(ast.parse(open(path).read()))}
        assert "oracle" not in mods, path
    for path in list(_files(PKG, (".cu", ".cuh", ".h", ".cpp"))) + list(_files(os.path.join(ROOT, "include"), (".h",))):
        text = open(path).read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', text), path
        assert "hphi_oracle" not in text and "liboracle" not in text, path


def test_oracle_never_loads_the_library():
    py = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    mods = {m for _, m in _imported_modules(ast.parse(py))}
    assert not mods & {"paper_1703_03637_gb300", "torch"}, mods
    cpp = open(os.path.join(ROOT, "oracle", "hphi_oracle.cpp")).read()
    for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', cpp):
        assert "/" not in inc and not inc.endswith((".cuh", ".cu")) and "hphi_gpu" not in inc, inc


def _functions_loading_oracle(path):
    tree = ast.parse(open(path).read())
    top_level = [m for node, m in _imported_modules(tree) if m == "oracle" and node in tree.body]
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, (ast.FunctionDef, ast.AsyncFunctionDef)):
            if any(m == "oracle" for _, m in _imported_modules(fn)):
                users.add(fn.name)
    return top_level, users


def test_bench_loads_the_oracle_only_in_its_baseline_legs():
    top, users = _functions_loading_oracle(os.path.join(ROOT, "bench.py"))
    assert not top, "bench.py imports the oracle at module level"
    assert users <= {"oracle_rows_per_s", "oracle_sampled_rows_per_s", "oracle_baseline", "run_reference"}, users


def test_entry_loads_the_oracle_only_to_build_and_smoke_check():
    top, users = _functions_loading_oracle(os.path.join(ROOT, "__graft_entry__.py"))
    assert not top and users <= {"build", "smoke"}, (top, users)
