"""The oracle and the CUDA path share nothing, and only the allowed places use
the oracle: the package (binding, inputs, workload, build) never imports it,
the CUDA and C sources include nothing across the boundary, the oracle never
imports the package, and bench.py reaches it only in the reference arm and in
the CPU-baseline leg."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1607_06303_gb300")


def _imported_modules(path):
    tree = ast.parse(open(path).read(), path)
    mods = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods += [(a.name.split(".")[0], node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            mods.append((node.module.split(".")[0], node))
    return tree, mods


def test_package_never_imports_the_oracle():
    for name in sorted(os.listdir(PKG)):
        if name.endswith(".py"):
            _, mods = _imported_modules(os.path.join(PKG, name))
            assert "oracle" not in [m for m, _ in mods], name


def test_sources_do_not_cross():
    csrc = os.path.join(PKG, "csrc")
    for name in sorted(os.listdir(csrc)):
        text = open(os.path.join(csrc, name)).read()
        for inc in re.findall(r'#include\s*"([^"]+)"', text):
            assert "oracle" not in inc, (name, inc)
    oracle_dir = os.path.join(ROOT, "oracle")
    for name in sorted(os.listdir(oracle_dir)):
        path = os.path.join(oracle_dir, name)
        if name.endswith(".py"):
            _, mods = _imported_modules(path)
            assert "paper_1607_06303_gb300" not in [m for m, _ in mods], name
        elif name.endswith(".c"):
            for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(path).read()):
                assert "csrc" not in inc and "signtri" not in inc, (name, inc)


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    tree, mods = _imported_modules(os.path.join(ROOT, "bench.py"))
    parents = {}
    for node in ast.walk(tree):
        for child in ast.iter_child_nodes(node):
            parents[child] = node
    sites = [node for m, node in mods if m == "oracle"]
    assert sites, "bench.py no longer times the oracle"
    for node in sites:
        allowed = False
        p = parents.get(node)
        while p is not None:
            if isinstance(p, ast.FunctionDef) and p.name == "run_reference":
                allowed = True
            if isinstance(p, ast.If) and "no_cpu_baseline" in ast.unparse(p.test):
                allowed = True
            p = parents.get(p)
        assert allowed, "oracle imported at line %d outside the CPU legs" % node.lineno
