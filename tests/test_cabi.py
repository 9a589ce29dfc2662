"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/hopf.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hg():
    from paper_1605_01799_gb300 import build
    build.build()
    import paper_1605_01799_gb300 as pkg
    pkg.lib()
    return pkg


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(hopf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(hg):
    names = declared_functions()
    assert len(names) >= 10
    L = hg.lib()
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(hg.EXPORTS), set(names) ^ set(hg.EXPORTS)


def test_version(hg):
    assert "sm_103a" in hg.version()


def _desc(hg, **kw):
    A = kw.pop("A", np.ones(4))
    d = dict(n=4, a_kind=0, A=None if A is None else A.ctypes.data, centre=None, c0=0.5, h_kind=0, w=None, lam=1.0, tol=1e-10,
             max_iter=10, precision=1, stop_rule=0)
    d.update(kw)
    return hg.hopf_desc(**d), A


@pytest.mark.parametrize("field,value", [("n", 0), ("n", 9000), ("a_kind", 7), ("h_kind", 9), ("lam", 0.0),
                                         ("lam", -1.0), ("tol", 0.0), ("max_iter", 0), ("precision", 42),
                                         ("stop_rule", 5)])
def test_create_rejects_bad_arguments(hg, field, value):
    d, keep = _desc(hg, **{field: value})
    h = ctypes.c_void_p()
    st = hg.lib().hopf_create(ctypes.byref(d), ctypes.byref(h), None)
    assert st == hg.HOPF_EINVAL
    assert not h.value
    assert hg.lib().hopf_last_error().decode()


def test_create_rejects_weighted_without_weights(hg):
    d, keep = _desc(hg, h_kind=1)
    h = ctypes.c_void_p()
    assert hg.lib().hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EINVAL


def test_create_rejects_nonpositive_diagonal(hg):
    d, keep = _desc(hg, A=np.array([1.0, 0.0, 2.0, 3.0]))
    h = ctypes.c_void_p()
    assert hg.lib().hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_ENOTSPD


def test_unsupported_combinations(hg):
    A = np.eye(4)
    d, keep = _desc(hg, A=A, a_kind=1, precision=0)
    h = ctypes.c_void_p()
    assert hg.lib().hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EUNSUPPORTED
    d, keep = _desc(hg, A=A, a_kind=1, precision=1, stop_rule=0)
    assert hg.lib().hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EUNSUPPORTED


def test_new_kinds_argument_checks(hg):
    """l_inf and sqrt(sum w p^2) Hamiltonians and the norm initial data:
    weights required and positive for sqrt(sum w p^2), l_inf and
    sqrt(sum w p^2) refused on the dense path, a norm J needs no A but still a
    valid n."""
    L = hg.lib()
    h = ctypes.c_void_p()
    d, keep = _desc(hg, h_kind=hg.H_DNORM)
    assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EINVAL
    w = np.array([1.0, 2.0, -1.0, 1.0])
    d, keep = _desc(hg, h_kind=hg.H_DNORM, w=w.ctypes.data)
    assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EINVAL
    A = np.eye(4)
    for hk in (hg.H_LINF, hg.H_DNORM):
        wv = np.ones(4)
        d, keep = _desc(hg, A=A, a_kind=hg.A_DENSE, h_kind=hk, w=wv.ctypes.data, precision=hg.P_MIXED,
                        stop_rule=hg.STOP_UREL)
        assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EUNSUPPORTED
    for jk in (hg.J_L1SQ, hg.J_LINFSQ):
        d, keep = _desc(hg, a_kind=jk, A=None, n=0)
        assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EINVAL
        d, keep = _desc(hg, a_kind=jk, A=None, n=9000)
        assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EINVAL
    assert not h.value


def test_anorm_argument_checks(hg):
    """H = sqrt(<p, M p>): M required, symmetric, positive definite (the
    host eigendecomposition finds a non-positive eigenvalue), n <= 512, and
    the diagonal path only.  All refused before any device work."""
    L = hg.lib()
    h = ctypes.c_void_p()
    d, keep = _desc(hg, h_kind=hg.H_ANORM)
    assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EINVAL
    M = np.eye(4)
    M[0, 1] = 0.5
    d, keep = _desc(hg, h_kind=hg.H_ANORM, w=M.ctypes.data)
    assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EINVAL
    M = np.ones((4, 4)) + np.diag([1.0, 1.0, 1.0, -3.9])  # eigenvalue below 0
    assert np.linalg.eigvalsh(M).min() < 0
    d, keep = _desc(hg, h_kind=hg.H_ANORM, w=M.ctypes.data)
    assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_ENOTSPD
    big = np.eye(600)
    a = np.ones(600)
    d, keep = _desc(hg, A=a, n=600, h_kind=hg.H_ANORM, w=big.ctypes.data)
    assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EUNSUPPORTED
    I4 = np.eye(4)
    d, keep = _desc(hg, A=np.eye(4), a_kind=hg.A_DENSE, h_kind=hg.H_ANORM, w=I4.ctypes.data,
                    precision=hg.P_MIXED, stop_rule=hg.STOP_UREL)
    assert L.hopf_create(ctypes.byref(d), ctypes.byref(h), None) == hg.HOPF_EUNSUPPORTED
    assert not h.value


def test_null_arguments(hg):
    L = hg.lib()
    assert L.hopf_create(None, None, None) == hg.HOPF_EINVAL
    assert L.hopf_eval(None, 4, None, None, None, None, None, None, None, None, 0, None) == hg.HOPF_EINVAL
    assert L.hopf_eval_f64(None, 4, None, None, None, None, None, None, None, None, 0, None) == hg.HOPF_EINVAL
    b = ctypes.c_size_t()
    assert L.hopf_workspace_size(None, 4, ctypes.byref(b)) == hg.HOPF_EINVAL
    assert L.hopf_union_eval(None, 0, 4, None, None, None, None, None, None, None, None, 0, None) == hg.HOPF_EINVAL
    assert L.hopf_backward(None, 4, None, None, None, None, None, None) == hg.HOPF_EINVAL
    L.hopf_destroy(None)


def test_batch_rejects_bad_arguments(hg):
    L = hg.lib()
    out = ctypes.c_void_p()
    assert L.hopf_batch_create(None, 1, ctypes.byref(out), None) == hg.HOPF_EINVAL
    d, keep = _desc(hg)
    descs = (hg.hopf_desc * 2)(d, d)
    assert L.hopf_batch_create(descs, 0, ctypes.byref(out), None) == hg.HOPF_EINVAL
    # an FP64 instance is refused, and a bad instance is named in the message
    descs[1].precision = hg.P_FP64
    assert L.hopf_batch_create(descs, 2, ctypes.byref(out), None) == hg.HOPF_EUNSUPPORTED
    assert not out.value
    descs[1].precision = hg.P_FP32
    descs[0].n = 0
    assert L.hopf_batch_create(descs, 2, ctypes.byref(out), None) == hg.HOPF_EINVAL
    assert "instance 0" in L.hopf_last_error().decode()
    b = ctypes.c_size_t()
    cnt = np.zeros(2, np.int64)
    assert L.hopf_batch_workspace_size(None, cnt.ctypes.data, ctypes.byref(b)) == hg.HOPF_EINVAL
    assert L.hopf_batch_eval(None, cnt.ctypes.data, None, None, None, None, None, None, None, None, 0,
                             None) == hg.HOPF_EINVAL
    assert L.hopf_batch_info(None, None, None, None) == hg.HOPF_EINVAL
    L.hopf_batch_destroy(None)


def test_control_and_maxH_reject_bad_arguments(hg):
    L = hg.lib()
    assert L.hopf_eval_control(None, 4, None, None, None, None, None, None, None, None, None, None, 0,
                               None) == hg.HOPF_EINVAL
    assert L.hopf_maxH_eval(None, 0, 4, None, None, None, None, None, None, None, None, 0, None) == hg.HOPF_EINVAL


def test_figure_grid_and_level_lines():
    """Host side of the 2-D slices: the paper's grid x_i = -20 + 40 k / 99 in
    the first two coordinates (the rest 0), and level lines where phi crosses a
    multiple of the step."""
    from paper_1605_01799_gb300 import figures as F
    X = F.grid_points()
    assert X.shape == (10000, 8) and (X[:, 2:] == 0).all()
    assert X[0, 0] == -20.0 and X[-1, 0] == 20.0 and abs(X[1, 1] - (-20.0 + 40.0 / 99)) < 1e-12
    assert (X[:100, 0] == -20.0).all()  # x2 runs fastest
    phi = np.add.outer(np.arange(10.0), np.zeros(4))  # phi = row index
    img = F.to_pgm(phi, 5.0)
    assert (img[4] == 0).all() and (img[3] != 0).all()  # 4 -> 5 crosses a multiple of 5


def test_allocator_and_wait_limit_arguments(hg):
    """One allocator function without the other, a null handle or a negative
    limit: refused before anything touches the device."""
    import ctypes
    L = hg.lib()
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    fa = ALLOC(lambda n, c: None)
    assert L.hopf_set_allocator(ctypes.cast(fa, ctypes.c_void_p), None, None) == hg.HOPF_EINVAL
    assert b"both" in L.hopf_last_error()
    assert L.hopf_set_allocator(None, None, None) == hg.HOPF_OK
    assert L.hopf_set_wait_limit(None, 100) == hg.HOPF_EINVAL
    assert L.hopf_set_tc_pairs(None, 1) == hg.HOPF_EINVAL
    assert b"hopf_set_tc_pairs" in L.hopf_last_error()
    assert L.hopf_set_split_start(None, 1e-12) == hg.HOPF_EINVAL
    assert b"hopf_set_split_start" in L.hopf_last_error()


def test_backward_params_null_handle(hg):
    L = hg.lib()
    assert L.hopf_backward_params(None, 4, None, None, None, None, None, None, None, None) == hg.HOPF_EINVAL


def test_header_is_plain_c_and_links(hg, tmp_path):
    """The boundary is usable from C: a C99 program that includes hopf.h and
    takes the address of every declared entry point compiles with gcc and
    links against the library (C linkage, no C++ types in the signatures)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not on PATH")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    names = declared_functions()
    src = tmp_path / "use_hopf.c"
    src.write_text('#include "hopf.h"\n#include <stdio.h>\ntypedef void (*fn)(void);\n'
                   "static const fn entry[] = {\n" + ",\n".join("    (fn)%s" % n for n in names) + "\n};\n"
                   "int main(void) {\n"
                   "    printf(\"%d entry points\\n\", (int)(sizeof(entry) / sizeof(entry[0])));\n"
                   "    return 0;\n}\n")
    lib = hg.LIB_PATH
    exe = tmp_path / "use_hopf"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"),
                        "-I" + cuda_inc, str(src), lib, "-Wl,--allow-shlib-undefined", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    env = dict(os.environ, LD_LIBRARY_PATH=os.pathsep.join(
        [os.path.dirname(lib), os.environ.get("LD_LIBRARY_PATH", "")]))
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "%d entry points" % len(names), (r.stdout, r.stderr)


_OPAQUE = {"hopf_handle", "hopf_batch", "cudaStream_t", "cudaEvent_t", "hopf_alloc_fn", "hopf_free_fn"}
_SCALAR = {"int64_t": "i64", "int32_t": "i32", "float": "f32", "double": "f64", "size_t": "sz",
           "hopf_status": "i32", "void": None}


def _c_kind(decl):
    """Argument or return category of a C declaration (without its name)."""
    decl = decl.replace("const", " ").strip()
    if "*" in decl:
        return "ptr"
    base = decl.split()[0]
    if base in _OPAQUE:
        return "ptr"
    return _SCALAR[base]


def _ctypes_kind(t):
    if t is None:
        return None
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    return {ctypes.c_int64: "i64", ctypes.c_int32: "i32", ctypes.c_float: "f32", ctypes.c_double: "f64",
            ctypes.c_size_t: "sz"}[t]


def declared_prototypes():
    src = open(os.path.join(ROOT, "include", "hopf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"([A-Za-z_][\w \*]*?)\s*\b(hopf_\w+)\s*\(([^)]*)\)\s*;", src):
        ret, name, args = m.group(1).strip(), m.group(2), " ".join(m.group(3).split())
        kinds = []
        if args != "void":
            for a in args.split(","):
                a = a.strip()
                # drop the parameter name (the last identifier), keep the type and any '*'
                kinds.append(_c_kind(re.sub(r"\b\w+$", "", a)))
        out[name] = (_c_kind(ret), kinds)
    return out


def test_binding_signatures_match_the_header(hg):
    """Every entry point's ctypes signature in the binding has the header's
    arity and, argument by argument, the same width and kind (pointer,
    int32, int64, size_t, float, double), and the same return type: a
    mismatch would pass wrong values across the boundary without an error."""
    protos = declared_prototypes()
    assert set(protos) == set(hg.EXPORTS)
    L = hg.lib()
    for name, (ret, kinds) in protos.items():
        f = getattr(L, name)
        got = [_ctypes_kind(t) for t in f.argtypes]
        assert got == kinds, (name, got, kinds)
        r = _ctypes_kind(f.restype)
        if name in ("hopf_last_error", "hopf_version"):
            assert f.restype is ctypes.c_char_p, name
        elif ret == "i32":
            assert f.restype is ctypes.c_int, name
        else:
            assert r == ret, (name, r, ret)


def test_descriptor_layout_matches_c(hg, tmp_path):
    """hopf_desc has the same size and field offsets in the binding as in C
    (compiled from the header with gcc)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not on PATH")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    c_names = ["n", "a_kind", "A", "centre", "c0", "h_kind", "w", "lambda", "tol", "max_iter", "precision",
               "stop_rule"]
    py_names = [f[0] for f in hg.hopf_desc._fields_]
    assert len(py_names) == len(c_names)
    src = tmp_path / "layout.c"
    src.write_text('#include "hopf.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void) {\n'
                   '    printf("%zu", sizeof(hopf_desc));\n' +
                   "".join('    printf(" %%zu", offsetof(hopf_desc, %s));\n' % c for c in c_names) +
                   '    printf("\\n");\n    return 0;\n}\n')
    exe = tmp_path / "layout"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"), "-I" + cuda_inc,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.split()]
    assert vals[0] == ctypes.sizeof(hg.hopf_desc)
    assert vals[1:] == [getattr(hg.hopf_desc, p).offset for p in py_names]
