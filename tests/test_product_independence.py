"""The product path never reaches the oracle, and the oracle never reaches the product.

The oracle (oracle/) is test infrastructure: only the tests, the smoke entry
point and bench.py's CPU-baseline and reference legs may use it.  Checked
statically on the sources:
  * no module of the package paper_1508_02599_gb300 and no CUDA/C++ source
    imports, includes or names the oracle;
  * the oracle and the shared input generators import nothing of the package
    or of the CUDA sources;
  * in bench.py the oracle is imported only inside cpu_baseline and
    run_reference, in __graft_entry__.py only inside smoke.
"""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1508_02599_gb300")


def _py_files(d):
    for base, _, files in os.walk(d):
        if "_build" in base or "__pycache__" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def _imports(tree):
    """(module name, enclosing function name or None) of every import."""
    out = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import):
                out.extend((a.name, func) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                out.append((child.module or "", func))
            visit(child, f)

    visit(tree, None)
    return out


def test_package_does_not_import_the_oracle():
    for path in _py_files(PKG):
        tree = ast.parse(open(path).read())
        for mod, _ in _imports(tree):
            assert not mod.split(".")[0] == "oracle", (path, mod)


def test_cuda_sources_do_not_name_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cpp", ".h")):
            text = open(os.path.join(csrc, f)).read()
            assert "oracle" not in text.lower(), f
    for f in os.listdir(os.path.join(ROOT, "include")):
        assert "oracle" not in open(os.path.join(ROOT, "include", f)).read().lower(), f


def test_oracle_and_inputs_do_not_import_the_package():
    for d in ("oracle", "feti_inputs"):
        for path in _py_files(os.path.join(ROOT, d)):
            for mod, _ in _imports(ast.parse(open(path).read())):
                top = mod.split(".")[0]
                assert top not in ("paper_1508_02599_gb300", "torch", "__graft_entry__"), (path, mod)


def test_oracle_use_is_confined():
    allowed = {"bench.py": {"cpu_baseline", "run_reference"}, "__graft_entry__.py": {"smoke"}}
    for name, funcs in allowed.items():
        tree = ast.parse(open(os.path.join(ROOT, name)).read())
        for mod, func in _imports(tree):
            if mod.split(".")[0] == "oracle":
                assert func in funcs, (name, func)
