"""The oracle and the CUDA path share no code: the oracle imports only the
seeded input module of the package, and no product module imports the oracle."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.add(node.module)
    return out


def _py_files(d):
    for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def test_oracle_imports_only_inputs_from_package():
    for f in _py_files("oracle"):
        for mod in _imports(f):
            if mod.startswith("paper_2605_14526_b300"):
                assert mod == "paper_2605_14526_b300.inputs", (f, mod)


def test_package_never_imports_oracle():
    for f in _py_files("paper_2605_14526_b300"):
        for mod in _imports(f):
            assert not mod.startswith("oracle"), (f, mod)


def test_inputs_module_has_no_method_arithmetic():
    src = open(os.path.join(ROOT, "paper_2605_14526_b300", "inputs.py")).read()
    for word in ("svd", "gradN", "Dm_inv", "lame(", "linalg.eig", "prox", "density *", "density*"):
        assert word not in src, word
