"""Static checks that the oracle and the CUDA path stay independent.

The oracle is test infrastructure: the tests, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` (the CPU baseline and the reference arm) are the
only code that may import it.  The library must neither load nor include
anything of it, and the oracle must share no header or helper with the
library.  The input generators serve both sides and must hold none of the
filter's arithmetic."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(sub, exts):
    out = []
    for ext in exts:
        out += glob.glob(os.path.join(ROOT, sub, "**", "*" + ext), recursive=True)
    return sorted(out)


def test_library_never_touches_the_oracle():
    src = _files("paper_cs_0610046_gb300", (".py", ".cu", ".cuh", ".h", ".c")) + _files("include", (".h",))
    assert src
    for path in src:
        text = open(path).read()
        assert not re.search(r"\boracle\b", text), f"{path} mentions the oracle"
        assert "liboracle" not in text and "mmf_oracle" not in text, path


def test_oracle_shares_no_code_with_the_library():
    c = open(os.path.join(ROOT, "oracle", "mmf_oracle.c")).read()
    includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', c)
    # Only the C standard library.
    assert includes and all(re.fullmatch(r"std\w*\.h|math\.h|string\.h|limits\.h", h) for h in includes), includes
    py = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    tree = ast.parse(py)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names = [a.name for a in node.names]
        elif isinstance(node, ast.ImportFrom):
            names = [node.module or ""]
        else:
            continue
        for name in names:
            assert not name.startswith("paper_cs_0610046_gb300"), name
            assert not name.startswith("torch"), name


def _oracle_imports(path):
    """(enclosing function name or None, line) of every import of the oracle."""
    tree = ast.parse(open(path).read())
    found = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.append((func, child.lineno))
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                found.append((func, child.lineno))
            visit(child, f)

    visit(tree, None)
    return found


def test_bench_imports_the_oracle_only_in_its_cpu_legs():
    found = _oracle_imports(os.path.join(ROOT, "bench.py"))
    assert found, "the CPU baseline and the reference arm time the oracle"
    assert {f for f, _ in found} <= {"cpu_baseline", "run_reference"}, found


def test_entry_point_imports_the_oracle_only_to_build_and_smoke():
    found = _oracle_imports(os.path.join(ROOT, "__graft_entry__.py"))
    assert {f for f, _ in found} <= {"build", "smoke"}, found


def test_generators_hold_no_filter_arithmetic():
    """The shared input generators draw numbers; they compute no window
    maximum or minimum and import neither side."""
    src = open(os.path.join(ROOT, "synth", "__init__.py")).read()
    for node in ast.walk(ast.parse(src)):
        if isinstance(node, ast.Import):
            names = [a.name for a in node.names]
        elif isinstance(node, ast.ImportFrom):
            names = [node.module or ""]
        else:
            continue
        assert not any(n.split(".")[0] in ("oracle", "paper_cs_0610046_gb300") for n in names), names
    for banned in ("maximum.accumulate", "minimum.accumulate", "sliding_window_view", "max_pool", "cummax",
                   "cummin"):
        assert banned not in src, banned
