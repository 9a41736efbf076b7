"""Structure of the repository that the parity claims rest on (CPU only).

The oracle and the CUDA path share no code: nothing under `oracle/` imports
the package, the package neither imports nor includes anything of `oracle/`,
and `workloads/` (the seeded input generators both sides use) imports
neither.  Outside the tests, only `__graft_entry__.smoke()` and the CPU
baseline / reference arm of `bench.py` may call the oracle, from inside
those functions.
"""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom):
            mod = ("." * node.level) + (node.module or "")
            out.append((mod, node))
    return tree, out


def _py_files(sub):
    d = os.path.join(ROOT, sub)
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def test_oracle_does_not_import_the_package():
    for path in _py_files("oracle"):
        for mod, _ in _imports(path)[1]:
            assert not mod.startswith("paper_1501_06211_gb300"), (path, mod)


def test_package_does_not_use_the_oracle():
    for path in _py_files("paper_1501_06211_gb300"):
        for mod, _ in _imports(path)[1]:
            assert not mod.split(".")[0] == "oracle", (path, mod)
    csrc = os.path.join(ROOT, "paper_1501_06211_gb300", "csrc")
    for name in os.listdir(csrc):
        text = open(os.path.join(csrc, name), errors="replace").read()
        assert "oracle" not in text.lower(), name


def test_workloads_import_neither_side():
    for path in _py_files("workloads"):
        for mod, _ in _imports(path)[1]:
            top = mod.split(".")[0]
            assert top not in ("oracle", "paper_1501_06211_gb300"), (path, mod)


def test_oracle_calls_outside_tests_sit_in_the_allowed_functions():
    allowed = {"__graft_entry__.py": {"smoke"}, "bench.py": {"oracle_solve_ms", "run_reference",
                                                             "cpu_baseline_and_errors"}}
    for fname, funcs in allowed.items():
        tree, imps = _imports(os.path.join(ROOT, fname))
        parents = {}
        for node in ast.walk(tree):
            for child in ast.iter_child_nodes(node):
                parents[child] = node
        for mod, node in imps:
            if mod.split(".")[0] != "oracle":
                continue
            p = parents.get(node)
            while p is not None and not isinstance(p, ast.FunctionDef):
                p = parents.get(p)
            assert p is not None and p.name in funcs, (fname, mod, getattr(p, "name", None))
