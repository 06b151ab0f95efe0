"""C-ABI checks that need no GPU: the library builds, loads and exports every
symbol the headers declare; the binding's structures match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:[a-z_0-9]+\s*\*?\s+)+\*?(rsvd_[a-z_0-9]+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2307_15572_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "rsvd_plan" in declared and "rsvd_decompose_batched" in declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu():
    from paper_2307_15572_gb300 import rsvd
    lib = rsvd.load()
    assert lib.rsvd_version() >= 100
    assert isinstance(lib.rsvd_last_error_string(), bytes)


def test_struct_layout_matches_header(tmp_path):
    """Compile a C probe against include/rsvd.h and compare every field offset."""
    import shutil
    import subprocess
    from paper_2307_15572_gb300 import rsvd
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"rsvd_opts": rsvd.Opts, "rsvd_matrix": rsvd.Matrix, "rsvd_factors": rsvd.Factors,
               "rsvd_profile": rsvd.Profile, "rsvd_tune_record": rsvd.TuneRecord}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rsvd.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, v = line.split()
            got[(a, b)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_plan_rejects_bad_options_before_touching_the_device():
    from paper_2307_15572_gb300 import rsvd
    bad = [dict(n_max=0, k=4), dict(n_max=10, k=0), dict(n_max=10, k=4, p=-1),
           dict(n_max=10, k=4, q=-1), dict(n_max=10, k=4, precision=7),
           dict(n_max=10, k=4, policy="tol", tol=0.0), dict(n_max=10, k=4, slices=5)]
    for kw in bad:
        with pytest.raises(rsvd.RsvdError) as e:
            rsvd.rsvd_plan(rsvd.make_opts(**kw))
        assert e.value.status == rsvd.RSVD_ERR_INVALID_ARG
