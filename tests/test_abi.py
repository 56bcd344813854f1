"""C-ABI checks that need no GPU: the library loads, exports every symbol the header
declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import numpy as np

import pytest

from paper_2405_16267_b300 import bicadmm as bc
from paper_2405_16267_b300 import build_lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "bicadmm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bicadmm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return bc.lib()


def test_header_declares_expected_api():
    names = declared_functions()
    for required in ["bicadmm_create", "bicadmm_setup", "bicadmm_solve", "bicadmm_step",
                     "bicadmm_get_x", "bicadmm_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    cdll = ctypes.CDLL(build_lib.LIB)
    missing = [n for n in declared_functions() if not hasattr(cdll, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in bc.SIGNATURES}
    assert set(declared_functions()) <= bound


def _c_layout(struct, fields):
    """sizeof and offsetof of a header struct, from a C program compiled against the header."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    body = "".join('  printf("%%s %%zu\\n", "%s", offsetof(%s, %s));\n' % (f, struct, f) for f in fields)
    src = ("#include <stddef.h>\n#include <stdio.h>\n#include \"bicadmm.h\"\nint main(void) {\n"
           '  printf("sizeof %%zu\\n", sizeof(%s));\n%s  return 0;\n}\n' % (struct, body))
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(c, "w") as f:
            f.write(src)
        subprocess.run([cc, "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("struct,cls", [("bicadmm_params", "Params"), ("bicadmm_info", "Info"),
                                        ("bicadmm_server_params", "ServerParams")])
def test_struct_layouts_match_header(lib, struct, cls):
    """Every field of the ctypes mirror sits at the offset the C header gives it."""
    py = getattr(bc, cls)
    names = [name for name, _ in py._fields_]
    want = _c_layout(struct, names)
    assert ctypes.sizeof(py) == want["sizeof"]
    for name in names:
        assert getattr(py, name).offset == want[name], name
    p = bc.default_params()
    assert p.gamma == 10.0 and p.rho_c == 1.0 and p.inner_iters == 1 and p.K == 1


@pytest.mark.parametrize("field,value,code", [
    ("m", 0, -1), ("n", 0, -1), ("kappa", 0, -1), ("kappa", 101, -1), ("N_shards", 0, -1),
    ("N_shards", 51, -1), ("M_blocks", 101, -1), ("gamma", 0.0, -1), ("rho_c", -1.0, -1),
    ("inner_iters", 0, -1), ("K", 2, -1), ("loss", 2, -1), ("loss", 9, -1), ("precision", 5, -1),
    ("pass_rows", 3, -1), ("n", 40000, -7),
])
def test_create_rejects_bad_arguments_without_gpu(lib, field, value, code):
    p = bc.default_params(m=50, n=100, N_shards=2, M_blocks=2, kappa=5)
    if field == "n" and value == 40000:
        p.kappa = 5
    setattr(p, field, value)
    h = ctypes.c_void_p()
    rc = lib.bicadmm_create(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == code
    assert not h.value
    assert len(bc.last_error(None)) > 0


@pytest.mark.parametrize("K,n,kappa,code", [(17, 100, 5, -1), (10, 4000, 5, -7), (10, 100, 1001, -1)])
def test_softmax_create_checks_without_gpu(lib, K, n, kappa, code):
    """Softmax: 2 <= K <= 16, n K <= 32768, kappa <= n K (entrywise)."""
    p = bc.default_params(m=50, n=n, N_shards=2, M_blocks=2, kappa=kappa, loss=bc.LOSS_SOFTMAX, K=K)
    h = ctypes.c_void_p()
    assert lib.bicadmm_create(ctypes.byref(p), None, ctypes.byref(h)) == code
    assert not h.value


@pytest.mark.parametrize("kappas,loss,K,n,code", [
    ([3], 0, 1, 100, -1),              # a path holds 2..16 instances
    ([3] * 17, 0, 1, 100, -1),
    ([0, 3], 0, 1, 100, -1),           # 1 <= kappa <= n for every instance
    ([3, 101], 0, 1, 100, -1),
    ([3, 4], 2, 3, 100, -1),           # one-column losses only (2: softmax)
    ([3, 4], 0, 1, 20000, -7),         # n times the instance count <= 32768
])
def test_path_create_checks_without_gpu(lib, kappas, loss, K, n, code):
    p = bc.default_params(m=50, n=n, N_shards=2, M_blocks=2, kappa=3, loss=loss, K=K)
    k = (ctypes.c_int64 * len(kappas))(*kappas)
    h = ctypes.c_void_p()
    assert lib.bicadmm_create_path(ctypes.byref(p), len(kappas), k, None, ctypes.byref(h)) == code
    assert not h.value
    assert len(bc.last_error(None)) > 0


def test_null_handle_calls_are_safe(lib):
    assert lib.bicadmm_destroy(None) == 0
    assert lib.bicadmm_step(None, 1, None) == -1
    assert lib.bicadmm_default_params(None) == -1


def test_noalloc_binding_rejects_bad_tensors_before_launch():
    """The allocation-free entry point indexes w, z, s (n doubles) and tvt (4 doubles) on the
    device; the binding rejects every argument that would make it read or write outside them,
    on the host, before any launch (CPU tensors here, so no launch is even possible)."""
    import torch
    n = 16
    ok = lambda k=n: torch.zeros(k, dtype=torch.float64)
    tvt = ok(4)
    bad_cases = [
        ("float64", (ok().float(), ok(), ok(), tvt)),
        ("float64", (ok(), ok(), ok(), tvt.float())),
        ("contiguous", (ok(2 * n)[::2], ok(), ok(), tvt)),
        ("same length", (ok(), ok(n - 1), ok(), tvt)),
        ("same length", (ok(), ok(), ok(n + 1), tvt)),
        ("at least 4", (ok(), ok(), ok(), ok(3))),
        ("torch tensor", (np.zeros(n), ok(), ok(), tvt)),
        ("CUDA tensor", (ok(), ok(), ok(), tvt)),
    ]
    for what, args in bad_cases:
        with pytest.raises(ValueError, match=what):
            bc.consensus_step_noalloc(*args, kappa=2, N_shards=1, rho_c=1.0, rho_b=0.5)
