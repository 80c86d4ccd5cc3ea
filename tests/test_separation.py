"""The oracle and the product share no code (static check, no GPU): the
oracle imports nothing from the product package, the product imports
nothing from the oracle, and bench.py touches the oracle only in its CPU
legs."""
import ast
import os

import pytest

ROOT = os.path.join(os.path.dirname(__file__), "..")


def imports(path):
    tree = ast.parse(open(path).read())
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append((node.module, node))
    return tree, out


def py_files(sub):
    d = os.path.join(ROOT, sub)
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


@pytest.mark.parametrize("path", py_files("oracle"))
def test_oracle_imports_nothing_from_the_product(path):
    _, imps = imports(path)
    assert not [m for m, _ in imps if m.split(".")[0] == "paper_2204_01117_gb300"], path


@pytest.mark.parametrize("path", py_files("paper_2204_01117_gb300"))
def test_product_imports_nothing_from_the_oracle(path):
    _, imps = imports(path)
    assert not [m for m, _ in imps if m.split(".")[0] == "oracle"], path


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    tree, _ = imports(os.path.join(ROOT, "bench.py"))
    allowed = {"oracle_sample", "oracle_single_box_run"}
    for fn in (n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)):
        for node in ast.walk(fn):
            if isinstance(node, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in node.names):
                assert fn.name in allowed, fn.name


def test_product_sources_never_name_the_oracle():
    csrc = os.path.join(ROOT, "paper_2204_01117_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle.cpp" not in text and "liboracle" not in text, f
