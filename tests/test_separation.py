"""The product and the oracle share no code: the library package never imports the oracle,
the oracle never imports the library, and synth (the one module both take inputs from) holds
no solver.  In bench.py the oracle is reached only from the CPU-baseline / reference legs."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imports(path):
    tree = ast.parse(open(path).read())
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name.split(".")[0], node) for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append((node.module.split(".")[0], node))
    return out, tree


def _py_files(d):
    for base, _, files in os.walk(os.path.join(ROOT, d)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_library_never_imports_the_oracle():
    for f in _py_files("paper_0707_3405_gb300"):
        mods = {m for m, _ in _imports(f)[0]}
        assert "oracle" not in mods, f
    for base, _, files in os.walk(os.path.join(ROOT, "paper_0707_3405_gb300", "csrc")):
        for f in files:
            assert "oracle" not in open(os.path.join(base, f)).read().lower(), f


def test_oracle_and_synth_never_import_the_library():
    for d in ("oracle", "synth"):
        for f in _py_files(d):
            mods = {m for m, _ in _imports(f)[0]}
            assert "paper_0707_3405_gb300" not in mods, f
            assert "torch" not in mods, f
    for f in _py_files("synth"):
        assert "oracle" not in {m for m, _ in _imports(f)[0]}, f


def test_bench_reaches_the_oracle_only_from_its_cpu_legs():
    imps, tree = _imports(os.path.join(ROOT, "bench.py"))
    parents = {}
    for node in ast.walk(tree):
        for ch in ast.iter_child_nodes(node):
            parents[ch] = node
    for mod, node in imps:
        if mod != "oracle":
            continue
        fn = node
        while fn is not None and not isinstance(fn, ast.FunctionDef):
            fn = parents.get(fn)
        assert fn is not None and fn.name in ("oracle_sample", "oracle_setup"), mod
    callers = {}
    for node in ast.walk(tree):
        name = getattr(node.func, "id", None) if isinstance(node, ast.Call) else None
        if name in ("oracle_sample", "oracle_setup"):
            fn = node
            while fn is not None and not isinstance(fn, ast.FunctionDef):
                fn = parents.get(fn)
            callers.setdefault(name, set()).add(fn.name)
    assert callers["oracle_sample"] == {"run_reference", "main"}
    assert callers["oracle_setup"] <= {"run_reference", "oracle_sample"}
