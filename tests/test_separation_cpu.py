"""The CUDA path and the oracle stay apart, and the product path has no
fallback: the package never imports the oracle, the oracle never imports the
package, no CUDA or header source includes anything of the oracle, and
loading the library from a missing path raises instead of degrading.
"""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2208_12187_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def imported_modules(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def py_files(d):
    return [os.path.join(d, f) for f in sorted(os.listdir(d)) if f.endswith(".py")]


def test_package_never_imports_the_oracle():
    for f in py_files(PKG):
        assert "oracle" not in imported_modules(f), f


def test_oracle_never_imports_the_package():
    for f in py_files(ORACLE):
        assert "paper_2208_12187_gb300" not in imported_modules(f), f


def test_native_sources_include_nothing_of_the_oracle():
    dirs = [os.path.join(PKG, "csrc"), os.path.join(ROOT, "include")]
    for d in dirs:
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                for line in open(os.path.join(d, f)):
                    if line.lstrip().startswith("#include"):
                        assert "oracle" not in line, (f, line)


def test_missing_library_fails_loudly():
    code = ("import sys\n"
            "from paper_2208_12187_gb300 import gbfit\n"
            "try:\n"
            "    gbfit.load('/nonexistent/libgbfit.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "raised:" in r.stdout
