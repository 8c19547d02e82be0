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
