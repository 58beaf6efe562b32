"""The product and the oracle stay apart, and the product has no fallback:

- no module of the package imports the oracle or reads a file under oracle/, and no CUDA
  source includes one; the oracle imports nothing of the package and its C source
  includes nothing of the CUDA library;
- importing every module of the package leaves the oracle unimported;
- without libpget.so the binding raises instead of computing anything.
"""
import ast
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2604_26745_gb300")
CSRC = os.path.join(PKG, "csrc")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield ("." * node.level) + (node.module or "")


def _py(d):
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith(".py"))


def _includes(path):
    return re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read())


def test_package_does_not_reach_the_oracle():
    for f in _py(PKG):
        for m in _imports(f):
            assert not m.split(".")[0] == "oracle", (f, m)
        src = open(f).read()
        assert not re.search(r"""["'][^"'\n]*oracle/""", src), f  # no path into oracle/
    for f in os.listdir(CSRC):
        for inc in _includes(os.path.join(CSRC, f)):
            assert "oracle" not in inc, (f, inc)


def test_oracle_does_not_reach_the_package():
    for f in _py(ORACLE):
        for m in _imports(f):
            assert not m.split(".")[0] in ("paper_2604_26745_gb300", "bench"), (f, m)
        assert "csrc" not in open(f).read(), f
    local = set(os.listdir(CSRC)) | {"pget.h"}
    for inc in _includes(os.path.join(ORACLE, "pget_oracle.c")):
        assert os.path.basename(inc) not in local, inc


def test_importing_the_package_leaves_the_oracle_out():
    mods = [os.path.splitext(os.path.basename(f))[0] for f in _py(PKG) if not f.endswith("__init__.py")]
    code = ("import sys\n"
            + "".join(f"import paper_2604_26745_gb300.{m}\n" for m in mods)
            + "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]\n"
            + "assert not bad, bad\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]


def test_missing_library_raises():
    code = ("from paper_2604_26745_gb300 import pget\n"
            "pget._lib = None\n"
            "try:\n"
            "    pget.load('/nonexistent/libpget.so')\n"
            "except RuntimeError as e:\n"
            "    assert 'missing' in str(e)\n"
            "else:\n"
            "    raise SystemExit('load() returned without a library')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
