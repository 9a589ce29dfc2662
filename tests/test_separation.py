"""The product path and the oracle stay apart, and the product fails loudly
without its CUDA library (no CPU fallback)."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1605_01799_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                assert "oracle" not in _imports(os.path.join(dirpath, f)), f


def test_oracle_never_imports_the_package():
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith(".py"):
            assert "paper_1605_01799_gb300" not in _imports(os.path.join(odir, f)), f


def test_cuda_sources_share_nothing_with_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        src = open(os.path.join(csrc, f), errors="replace").read()
        assert "hopf_oracle" not in src and "oracle/" not in src, f
    osrc = open(os.path.join(ROOT, "oracle", "hopf_oracle.c")).read()
    assert "#include \"" not in osrc  # only system headers


def test_missing_library_raises():
    """With the library path pointing nowhere, the first call raises instead of
    computing anything on the host."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_1605_01799_gb300 as hg\n"
            "hg.LIB_PATH = '/nonexistent/libhopf_gb300.so'\n"
            "try:\n"
            "    hg.version()\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "else:\n"
            "    print('no error')\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.startswith("raised:") and "not built" in r.stdout, r.stdout
