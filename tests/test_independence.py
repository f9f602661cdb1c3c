"""The CPU oracle and the CUDA path share no code: the product package never imports,
loads or includes anything under oracle/, and the oracle never includes or imports the
product's sources (the seeded input module is the one thing both sides read)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2603_22902_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def sources(top, exts):
    for d, _, files in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_does_not_use_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#\s*include\s*[<\"][^>\"]*lbo\.h)", re.M)
    for p in sources(PKG, (".py", ".cu", ".cuh", ".hpp", ".h")):
        with open(p) as fh:
            text = fh.read()
        assert not pat.search(text), p
        assert "liblbo" not in text, p


def test_oracle_does_not_use_the_product():
    pat = re.compile(r"(csrc|lbm_step|lbm_device|lbm_df64|lbm_lattice|liblbm_gb300|include/lbm\.h|#\s*include\s*\"lbm)")
    for p in sources(ORACLE, (".c", ".h", ".py")):
        with open(p) as fh:
            text = fh.read()
        assert not pat.search(text), p
        assert "import paper_2603_22902_gb300" not in text and "from paper_2603_22902_gb300" not in text, p


def _functions_importing_oracle(path):
    import ast
    with open(path) as fh:
        tree = ast.parse(fh.read())
    found = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.append(func)
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                found.append(func)
            visit(child, name)

    visit(tree, None)
    return found


def test_bench_and_entry_use_the_oracle_only_where_allowed():
    # bench.py: only the CPU-baseline / reference timing; __graft_entry__: smoke() checks
    # against it, build() compiles it (building the checker is not using it)
    assert _functions_importing_oracle(os.path.join(ROOT, "bench.py")) == ["time_oracle"]
    assert set(_functions_importing_oracle(os.path.join(ROOT, "__graft_entry__.py"))) <= {"build", "smoke"}
