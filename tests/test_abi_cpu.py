"""The C-ABI library loads, exports every declared entry point, and rejects
bad arguments before touching a GPU.  No compute calls here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2603_24920_gb300 import build_ext
from paper_2603_24920_gb300 import detlsh as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return D.lib()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "detlsh.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(detlsh_[a-z_]+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(n for n, _, _ in D.SIGNATURES) == names


def test_status_strings(lib):
    for s, name in D.STATUS.items():
        assert isinstance(D.status_string(s), str) and D.status_string(s)
    assert D.status_string(12345) == "unknown status"


def test_default_params(lib):
    p = D.detlsh_default_build_params()
    assert (p.L, p.K, p.N_r, p.max_size) == (4, 16, 256, 64)
    assert p.sample_frac == pytest.approx(0.1)
    assert p.tree_group == 0
    q = D.detlsh_default_query_params()
    assert (q.beta, q.c, q.precision, q.rerank_mult) == (pytest.approx(0.1), 1.5, 0, 0)


@pytest.mark.parametrize("kw", [dict(L=0), dict(L=17), dict(K=0), dict(K=17), dict(N_r=3),
                                dict(N_r=512), dict(N_r=1), dict(max_size=0),
                                dict(sample_frac=0.0), dict(sample_frac=1.5), dict(box_mode=2),
                                dict(L=16, K=17), dict(tree_group=-1), dict(L=2, tree_group=3)])
def test_build_rejects_bad_parameters(lib, kw):
    X = np.zeros((10, 4), np.float32)
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_build(X, **kw)
    assert e.value.status == -1


def test_build_rejects_bad_sizes(lib):
    p = D.detlsh_default_build_params()
    h = C.c_void_p()
    X = np.zeros((4, 4), np.float32)
    assert lib.detlsh_build_ex(D._ptr(X), 0, 4, C.byref(p), None, C.byref(h)) == -1
    assert lib.detlsh_build_ex(D._ptr(X), 4, 0, C.byref(p), None, C.byref(h)) == -1
    assert lib.detlsh_build_ex(None, 4, 4, C.byref(p), None, C.byref(h)) == -1
    assert lib.detlsh_build_ex(D._ptr(X), 4, 4, None, None, C.byref(h)) == -1


def test_query_and_accessors_reject_null_index(lib):
    Q = np.zeros((2, 4), np.float32)
    ids = np.zeros((2, 3), np.int64)
    dd = np.zeros((2, 3), np.float32)
    assert lib.detlsh_query(None, D._ptr(Q), 2, 3, 1.5, D._ptr(ids), D._ptr(dd)) == -1
    assert lib.detlsh_get_info(None, None) == -1
    assert lib.detlsh_get_tree(None, 0, None, None, None, None, None, None) == -1
    assert lib.detlsh_free(None) == 0
    t = D.Tuning(0, 4, 512, 1024, 0, 0)
    assert lib.detlsh_get_tuning(None, C.byref(t)) == -1
    assert lib.detlsh_set_tuning(None, C.byref(t)) == -1
    assert lib.detlsh_autotune(None, D._ptr(Q), 2, 3, None, None, None, None, None) == -1


def test_no_device_is_reported(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(D.DetlshError) as e:
        D.detlsh_build(np.random.rand(100, 8).astype(np.float32), L=2, K=4, N_r=16)
    assert e.value.status == -6


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes mirrors have the header's sizes and field offsets
    (checked by compiling the header with the host C compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = [("detlsh_build_params", D.BuildParams), ("detlsh_query_params", D.QueryParams),
             ("detlsh_info", D.Info), ("detlsh_timings", D.Timings), ("detlsh_tuning", D.Tuning)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "detlsh.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append('  printf("%%s size %%zu\\n", "%s", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('  printf("%%s %s %%zu\\n", "%s", offsetof(%s, %s));' % (f, cname, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in pairs:
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
