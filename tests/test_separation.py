"""The oracle and the CUDA path stay independent.

The FP64 oracle is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it, and it imports nothing of the CUDA
library.  The input generators (workloads/) import neither.  The library's
sources include only their own headers and system headers.  Checked on the
source text (AST for Python), so no import side effects run here.
"""

import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2607_00488_gb300"


def _imports(path):
    """(module name, enclosing top-level function or None) for every import."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = func
            if func is None and isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)):
                f = child.name
            if isinstance(child, ast.Import):
                out.extend((a.name, f) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = ("." * child.level) + (child.module or "")
                out.append((mod, f))
            visit(child, f)

    visit(tree, None)
    return out


def _top(mod):
    return mod.lstrip(".").split(".")[0] if not mod.startswith(".") else "."


def _py(pattern):
    files = sorted(glob.glob(os.path.join(ROOT, pattern)))
    assert files, pattern
    return files


def test_library_binding_never_imports_the_oracle():
    for path in _py(PKG + "/*.py"):
        for mod, _ in _imports(path):
            assert _top(mod) != "oracle", (path, mod)


def test_oracle_never_touches_the_cuda_library():
    for path in _py("oracle/*.py"):
        for mod, _ in _imports(path):
            assert _top(mod) not in (PKG, "ctypes"), (path, mod)
        text = open(path).read()
        assert "libsrw" not in text and ".cuda" not in text, path


def test_inputs_import_neither_side():
    for path in _py("workloads/*.py"):
        for mod, _ in _imports(path):
            assert _top(mod) not in ("oracle", PKG), (path, mod)


def test_oracle_only_in_the_allowed_legs():
    allowed = {
        "__graft_entry__.py": {"smoke"},
        "bench.py": {"_oracle_sample", "_oracle_share"},  # the CPU-baseline / reference legs
    }
    for name, funcs in allowed.items():
        for mod, func in _imports(os.path.join(ROOT, name)):
            if _top(mod) == "oracle":
                assert func in funcs, (name, mod, func)


def test_cuda_sources_include_only_their_own_headers():
    csrc = os.path.join(ROOT, PKG, "csrc")
    own = {os.path.join(csrc, f) for f in os.listdir(csrc)} | {os.path.join(ROOT, "include", "srw.h")}
    for path in sorted(glob.glob(os.path.join(csrc, "*"))):
        for m in re.finditer(r'^\s*#\s*include\s*([<"])([^>"]+)[>"]', open(path).read(), re.M):
            kind, inc = m.groups()
            if kind == '"':
                # the library's own sources and its public header, nothing else
                assert os.path.normpath(os.path.join(csrc, inc)) in own, (path, inc)
            assert "oracle" not in inc, (path, inc)
