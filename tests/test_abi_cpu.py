"""The C-ABI library without a GPU: it loads, exports every entry point that
include/nf.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2110_11398_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_11398_gb300 import build
    build.build()
    return N.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nf.h")).read()
    return sorted(set(re.findall(r"NF_API\s+[\w\s\*]*?\b(nf_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("nf_init", "nf_bin_particles", "nf_compute_accel", "nf_compute_accel_vjp", "nf_free"):
        assert name in syms
    assert sorted(N.EXPORTS) == syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    # and nothing but the ABI is exported
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert exported == declared_symbols()


def test_status_strings(lib):
    assert lib.nf_status_string(0) == b"NF_OK"
    assert lib.nf_status_string(-2) == b"NF_ERANGE"
    assert lib.nf_status_string(-99) == b"NF_UNKNOWN"


def _init(lib, n_boxes=1, L=(1.0,), cpd=(9,), R=2, eps=(1e-3,), soft=0, prec=0, cap=1000, dev=0):
    ctx = ctypes.c_void_p()
    Ls = (ctypes.c_double * len(L))(*L)
    Cs = (ctypes.c_int * len(cpd))(*cpd)
    Es = (ctypes.c_double * len(eps))(*eps)
    rc = lib.nf_init(ctypes.byref(ctx), dev, n_boxes, Ls, Cs, R, Es, soft, prec, cap)
    return rc, ctx


@pytest.mark.parametrize("kw,frag", [
    (dict(cpd=(4,)), "cpd"),                 # CPD < 2R+1
    (dict(eps=(0.0,)), "eps"),
    (dict(eps=(-1.0,)), "eps"),
    (dict(L=(0.0,)), "box_size"),
    (dict(L=(float("nan"),)), "box_size"),
    (dict(R=0), "radius"),
    (dict(R=4, cpd=(9,)), "radius"),
    (dict(prec=7), "precision"),
    (dict(soft=3), "softening"),
    (dict(cap=-1), "capacity"),
    (dict(cap=2 ** 31), "capacity"),
    (dict(n_boxes=0), "n_boxes"),
    (dict(cpd=(2000,)), "cpd"),
])
def test_init_rejects_bad_arguments(lib, kw, frag):
    rc, ctx = _init(lib, **kw)
    assert rc == N.NF_EINVAL
    assert ctx.value is None
    assert frag in lib.nf_last_error(None).decode()


def test_init_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, ctx = _init(lib)
    assert rc == N.NF_ECUDA
    assert ctx.value is None
    assert "device" in lib.nf_last_error(None).decode()


def test_null_context_calls(lib):
    lib.nf_free(None)                        # no-op
    assert lib.nf_compute_accel(None, None, None) == N.NF_EINVAL
    assert lib.nf_bin_particles(None, None, None, 0.0, 0, None, None) == N.NF_EINVAL
    assert lib.nf_compute_accel_vjp(None, None, None, None) == N.NF_EINVAL
    assert lib.nf_get_stats(None, None) == N.NF_EINVAL
    assert lib.nf_copy_binning(None, None, None, None, None) == N.NF_EINVAL
    assert lib.nf_compute_accel_f64(None, None, None) == N.NF_EINVAL
    assert lib.nf_compute_accel_density(None, None, None, None, None) == N.NF_EINVAL
    assert lib.nf_set_box_masses(None, None) == N.NF_EINVAL
    assert lib.nf_far_init(None, 8, None) == N.NF_EINVAL
    assert "nf_far_init" in lib.nf_last_error(None).decode()
    assert lib.nf_compute_far(None, None, 0, None) == N.NF_EINVAL
    assert lib.nf_kick(None, None, None, 0.1, None) == N.NF_EINVAL
    assert lib.nf_drift(None, None, None, 0.1, None) == N.NF_EINVAL
    assert lib.nf_timestep(None, None, None, 0.25, None, None) == N.NF_EINVAL
    assert lib.nf_kdk_step(None, None, None, None, None, 0.0, 0.1, None, None) == N.NF_EINVAL
    assert lib.nf_accel_host(None, None, None, 0.0, 0, None, None, None) == N.NF_EINVAL
    assert lib.nf_set_tuning(None, None) == N.NF_EINVAL
    assert lib.nf_get_tuning(None, None) == N.NF_EINVAL
    assert lib.nf_autotune(None, 1, None, None) == N.NF_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        N._lib_saved = N._lib
        try:
            N._lib = None
            N.load(str(tmp_path / "nope.so"))
        finally:
            N._lib = N._lib_saved


@pytest.mark.parametrize("name", ["nf_stats", "nf_tuning"])
def test_binding_structs_match_the_header(name, tmp_path):
    """The ctypes structures of the binding have the header's size and field
    offsets (a C program compiled against include/nf.h prints them)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    st = getattr(N, name)
    fields = [f[0] for f in st._fields_]
    prog = ['#include <stddef.h>', '#include <stdio.h>', '#include "nf.h"', "int main(void) {",
            f'  printf("%zu\\n", sizeof({name}));']
    prog += [f'  printf("%zu\\n", offsetof({name}, {f}));' for f in fields]
    prog += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(st)] + [getattr(st, f).offset for f in fields]
    assert got == want, (name, got, want)
