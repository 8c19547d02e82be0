"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, and
exports exactly the entry points the public header declares; context
creation without a GPU fails with a status instead of crashing."""

import ctypes
import glob
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"^ssl_status\s+(ssl_\w+)\s*\(", txt, flags=re.M))
    return names


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_03373_gb300.build import build
    return build()


def test_header_declares_the_boundary():
    names = _header_functions()
    for required in ("ssl_create", "ssl_destroy", "ssl_correlate", "ssl_gsvd",
                     "ssl_music_spectrum", "ssl_localize", "ssl_peaks", "ssl_noise_inverse"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(ssl_\w+)$", out, flags=re.M))
    declared = _header_functions()
    assert declared <= exported, declared - exported
    assert exported <= declared, exported - declared


def test_binding_covers_header(libpath):
    from paper_2504_03373_gb300 import binding
    assert set(binding.SIGNATURES) == _header_functions()
    lib = binding.load(libpath)
    for name in binding.SIGNATURES:
        assert getattr(lib, name) is not None


def test_create_without_gpu_returns_status(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2504_03373_gb300 import binding
    lib = binding.load(libpath)
    h = ctypes.c_void_p()
    st = lib.ssl_create(ctypes.byref(h), 0)
    assert st != 0 and not h.value
    # NULL handles are rejected synchronously.
    assert lib.ssl_correlate(None, None, 1, 1, 1, 1, None, None) == 1
    assert lib.ssl_destroy(None) == 0


def test_sources_are_sm103a_only():
    from paper_2504_03373_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_every_entry_point_rejects_null_arguments(libpath):
    """Argument errors come back synchronously as a status (the header's error
    convention): every entry point called with NULL pointers and zero sizes
    returns SSL_E_INVALID_ARG, and the destroy calls accept NULL.  Run in a
    child process so that a crash names the call instead of ending the run."""
    code = (
        "import ctypes, sys\n"
        "from paper_2504_03373_gb300 import binding\n"
        f"lib = binding.load({libpath!r})\n"
        "for name, argt in binding.SIGNATURES.items():\n"
        "    args = [None if (t in (ctypes.c_void_p, ctypes.c_char_p) or\n"
        "                     (isinstance(t, type) and issubclass(t, ctypes._Pointer))) else 0\n"
        "            for t in argt]\n"
        "    print(name, end=' ', flush=True)\n"
        "    print(getattr(lib, name)(*args), flush=True)\n")
    r = subprocess.run([os.sys.executable, "-c", code], capture_output=True, text=True,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stdout[-400:] + r.stderr[-400:]
    got = dict(line.split() for line in r.stdout.splitlines() if line.strip())
    from paper_2504_03373_gb300 import binding
    assert set(got) == set(binding.SIGNATURES)
    for name, st in got.items():
        want = "0" if name.endswith("_destroy") else "1"
        assert st == want, (name, st)


# C struct -> binding class; the field names are the same on both sides
_STRUCTS = {"ssl_jacobi_opts": "JacobiOpts", "ssl_config": "Config",
            "ssl_array_desc": "ArrayDesc", "ssl_result": "Result", "ssl_stats": "Stats",
            "ssl_batch_item": "BatchItem", "ssl_plan_info": "PlanInfo"}


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """Compile a probe against the public header (plain C) and compare every
    struct's size and field offsets, and the header's constants, with what the
    ctypes binding marshals."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2504_03373_gb300 import binding
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ssl_gsvd_music.h"',
             "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        cls = getattr(binding, pyname)
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    consts = ["SSL_OK", "SSL_E_INVALID_ARG", "SSL_E_NOT_PD", "SSL_E_NO_CONVERGENCE",
              "SSL_E_NONFINITE", "SSL_E_OOM", "SSL_E_ADMISSION", "SSL_E_TIMEOUT", "SSL_E_CUDA",
              "SSL_E_UNSUPPORTED", "SSL_E_CAPACITY", "SSL_FLAG_NOT_PD", "SSL_FLAG_NO_CONVERGENCE",
              "SSL_FLAG_NONFINITE", "SSL_FLAG_TIMEOUT", "SSL_FLAG_BOUNDS", "SSL_FORM_ABS",
              "SSL_FORM_SQ",
              "SSL_PREC_FP32", "SSL_PREC_TF32", "SSL_PREC_BF16", "SSL_PREC_TF32X3", "SSL_ANGLES_F64",
              "SSL_ANGLES_F32", "SSL_SVD_JACOBI", "SSL_SVD_BIDIAG", "SSL_SVD_SPLIT", "SSL_MAX_M",
              "SSL_MAX_NS",
              "SSL_PLAN_GRAPH", "SSL_PLAN_AUTOTUNE"]
    for c in consts:
        lines.append(f'  printf("const {c} %lld\\n", (long long)({c}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi_probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi_probe"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    c = {}
    for ln in out.splitlines():
        a, b, v = ln.split()
        c[(a, b)] = int(v)
    for cname, pyname in _STRUCTS.items():
        cls = getattr(binding, pyname)
        assert c[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert c[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
    k = {b: v for (a, b), v in c.items() if a == "const"}
    assert {v: n for v, n in binding.STATUS_NAMES.items()} == {
        k[n]: n for n in consts if n == "SSL_OK" or n.startswith("SSL_E_")}
    assert (binding.FLAG_NOT_PD, binding.FLAG_NO_CONVERGENCE, binding.FLAG_NONFINITE,
            binding.FLAG_TIMEOUT, binding.FLAG_BOUNDS) == (
        k["SSL_FLAG_NOT_PD"], k["SSL_FLAG_NO_CONVERGENCE"], k["SSL_FLAG_NONFINITE"],
        k["SSL_FLAG_TIMEOUT"], k["SSL_FLAG_BOUNDS"])
    assert binding.FORM == {"abs": k["SSL_FORM_ABS"], "sq": k["SSL_FORM_SQ"]}
    assert binding.PRECISION == {"fp32": k["SSL_PREC_FP32"], "tf32": k["SSL_PREC_TF32"],
                                 "bf16": k["SSL_PREC_BF16"], "tf32x3": k["SSL_PREC_TF32X3"]}
    assert binding.ANGLES == {"f64": k["SSL_ANGLES_F64"], "f32": k["SSL_ANGLES_F32"]}
    assert binding.METHOD == {"jacobi": k["SSL_SVD_JACOBI"], "bidiag": k["SSL_SVD_BIDIAG"],
                              "split": k["SSL_SVD_SPLIT"]}
    assert (binding.MAX_M, binding.MAX_NS) == (k["SSL_MAX_M"], k["SSL_MAX_NS"])
    assert (binding.PLAN_GRAPH, binding.PLAN_AUTOTUNE) == (k["SSL_PLAN_GRAPH"],
                                                          k["SSL_PLAN_AUTOTUNE"])


def test_bounds_checked_debug_build(libpath):
    """The bounds-checked debug build (-DSSL_DEBUG_BOUNDS) compiles for
    sm_103a and exports exactly the public header's entry points."""
    from paper_2504_03373_gb300.build import build
    dbg = build(debug_bounds=True)
    assert dbg != libpath and os.path.exists(dbg)
    out = subprocess.run(["nm", "-D", "--defined-only", dbg], capture_output=True, text=True,
                         check=True).stdout
    assert set(re.findall(r"\bT\s+(ssl_\w+)$", out, flags=re.M)) == _header_functions()
