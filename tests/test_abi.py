"""The C ABI library builds, loads and exports every function include/mvp.h
declares; host-only calls (no GPU needed) behave as documented; without the library
the Python entry points raise instead of falling back."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from paper_2103_01954_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "mvp.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(mvp_\w+)\s*\(", hdr, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mvp_build_bvh", "mvp_raymarch_fwd", "mvp_raymarch_bwd", "mvp_hitlists",
                     "mvp_ctx_create", "mvp_pack_payload"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = B.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mvp_\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = B.lib()
    for n in declared_functions():
        assert getattr(L, n) is not None
    # the binding declares a signature for every symbol
    assert set(n for n, _, _ in B._SIGS) == set(declared_functions())


def test_host_only_calls():
    L = B.lib()
    assert b"sm_103a" in L.mvp_version()
    assert L.mvp_status_string(B.MVP_ERR_CAPACITY) == b"MVP_ERR_CAPACITY"
    assert L.mvp_num_steps(1.0, 5.0, 0.01) == 400
    assert L.mvp_num_steps(1.0, 5.0, 0.005) == 800
    assert L.mvp_num_steps(1.0, 1.0, 0.01) == 0
    assert L.mvp_saved_bytes(10) == 320
    assert L.mvp_saved_bytes(0) == 0


def test_num_steps_matches_input_generator():
    import synthetic
    for t0, t1, dt in [(1.0, 5.0, 0.01), (1.0, 5.0, 0.005), (0.5, 2.25, 0.0025), (0.0, 6.0, 0.01), (2.0, 2.0005, 1e-3)]:
        r = synthetic.Rays(o=None, d=None, t_near=t0, t_far=t1, dt=dt)
        assert B.lib().mvp_num_steps(t0, t1, dt) == r.n_steps


def test_ctx_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = B.lib().mvp_ctx_create(0, ctypes.byref(h))
    assert st in (B.MVP_ERR_CUDA, B.MVP_ERR_INVALID_ARG)
    assert B.lib().mvp_last_error() != b""
    with pytest.raises(B.MVPError):
        B.check(st, "ctx")


def test_invalid_arguments_rejected_on_host():
    # a NULL context is rejected before anything touches the device
    L = B.lib()
    pr = B.mvp_prims(n=1, M=1, dtype=0)
    assert L.mvp_build_bvh(None, ctypes.byref(pr), None, None) == B.MVP_ERR_INVALID_ARG
    assert L.mvp_raymarch_fwd(None, ctypes.byref(pr), None, None, None, None, None) == B.MVP_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path):
    """With no built library and no compiler, the binding and the torch entry points raise;
    nothing falls back to another implementation."""
    script = f"""
import sys
sys.path.insert(0, {ROOT!r})
import paper_2103_01954_gb300.build as Bd
Bd.BUILD = {str(tmp_path)!r}
def _no_nvcc():
    raise RuntimeError("nvcc not found")
Bd._nvcc = _no_nvcc
from paper_2103_01954_gb300 import binding as B
try:
    B.lib()
    print("LOADED")
except RuntimeError as e:
    print("RAISED", e)
from paper_2103_01954_gb300 import torch_ops as T
try:
    T.Context(0)
    print("CONTEXT")
except Exception as e:
    print("RAISED", type(e).__name__)
"""
    out = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=300)
    lines = out.stdout.strip().splitlines()
    assert len(lines) == 2, (out.stdout, out.stderr[-2000:])
    assert lines[0].startswith("RAISED") and "nvcc not found" in lines[0]
    assert lines[1].startswith("RAISED")


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (a C
    program compiled against include/mvp.h prints them)."""
    structs = [B.mvp_prims, B.mvp_rays, B.mvp_request, B.mvp_serve_info]
    lines = ['#include <stdio.h>', '#include "mvp.h"', "int main(void) {"]
    for S in structs:
        n = S.__name__
        lines.append(f'  printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in S._fields_:
            lines.append(f'  printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for S in structs:
        n = S.__name__
        assert got[(n, "size")] == ctypes.sizeof(S), n
        for f, _ in S._fields_:
            assert got[(n, f)] == getattr(S, f).offset, (n, f)


def test_binding_signatures_match_the_prototypes():
    """Each function's ctypes signature has the prototype's argument count, a pointer
    wherever the prototype takes one, and the same scalar type otherwise (a mismatch
    would pass garbage through the ABI without an error)."""
    hdr = open(os.path.join(ROOT, "include", "mvp.h")).read()
    hdr = re.sub(r"\s+", " ", re.sub(r"/\*.*?\*/", "", hdr, flags=re.S))
    protos = {m.group(2): (m.group(1), m.group(3).strip())
              for m in re.finditer(r"([\w\s\*]*?)\b(mvp_\w+)\s*\(([^;{)]*)\)\s*;", hdr)}
    scalar = {"int": ctypes.c_int32, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
              "uint64_t": ctypes.c_uint64, "size_t": ctypes.c_size_t, "float": ctypes.c_float,
              "double": ctypes.c_double}
    returns = {"const char *": ctypes.c_char_p, "mvp_status": ctypes.c_int32, "void": None,
               "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "size_t": ctypes.c_size_t}

    def is_pointer(t):
        return t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer)

    for name, res, args in B._SIGS:
        ret, params = protos[name]
        ret = ret.split("MVP_API")[-1].strip()
        assert returns[ret] is res, (name, ret, res)
        params = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        assert len(params) == len(args), (name, params)
        for p, a in zip(params, args):
            ptype = " ".join(p.split()[:-1])
            if "*" in p or ptype == "mvp_stream":
                assert is_pointer(a), (name, p, a)
            else:
                assert scalar[ptype] is a, (name, p, a)


def test_binding_constants_match_the_header():
    """Status codes, payload types and ray flags: every name the binding defines has the
    header's value (from the enums and #defines, read as text and evaluated by a C
    program compiled against the header)."""
    names = [n for n in dir(B) if n.startswith("MVP_") and isinstance(getattr(B, n), int)]
    assert {"MVP_OK", "MVP_ERR_CAPACITY", "MVP_BF16", "MVP_BLEND_SEQUENTIAL"} <= set(names)
    import tempfile

    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "consts.c")
        with open(src, "w") as f:
            f.write('#include <stdio.h>\n#include "mvp.h"\nint main(void) {\n')
            for n in names:
                f.write(f'  printf("{n} %lld\\n", (long long)({n}));\n')
            f.write("  return 0;\n}\n")
        exe = os.path.join(d, "consts")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = {a: int(b) for a, b in (ln.split() for ln in out.splitlines())}
    for n in names:
        assert got[n] == getattr(B, n), n
