"""C-ABI checks that need no GPU: the library loads, exports every entry point
include/nv.h declares, and rejects bad arguments on the host before any launch."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "nv.h")).read()
    return sorted(set(re.findall(r"^\s*(?:nv_status|const char \*)\s*(nv_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def nvmod():
    import torch  # noqa: F401  (loads the CUDA runtime libnv.so links against)
    from paper_2207_11620_gb300 import build, nv
    build.build()
    return nv


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("nv_create", "nv_encode", "nv_infer", "nv_backward", "nv_train_step", "nv_render",
                 "nv_macrocells_build", "nv_sample", "nv_volume_mse", "nv_image_mse", "nv_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(nvmod):
    lib = nvmod.lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) == set(nvmod.EXPORTS)


def _prototypes():
    """name -> number of parameters of every entry point declared in nv.h."""
    txt = open(os.path.join(ROOT, "include", "nv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"(?:nv_status|const char \*)\s*(nv_\w+)\s*\(([^;{]*?)\)\s*;", txt, re.S):
        args = " ".join(m.group(2).split())
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(nvmod):
    """The ctypes table of the binding has one argument type per declared
    parameter, so a changed signature cannot be marshalled with a stale one."""
    protos = _prototypes()
    table = nvmod.EXPORTS
    assert set(protos) == set(table)
    bad = {n: (protos[n], len(table[n][0])) for n in protos if protos[n] != len(table[n][0])}
    assert not bad, bad


def _enum_values():
    """NAME -> value of every enumerator in nv.h (explicit values only)."""
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "nv.h")).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(NV_[A-Z0-9_]+)\s*=\s*(\d+)", txt)}


def test_binding_constants_match_the_header_enums(nvmod):
    ev = _enum_values()
    assert nvmod.PREC == {"fp32": ev["NV_FP32"], "fp16": ev["NV_FP16"], "bf16": ev["NV_BF16"]}
    assert nvmod.BUF == {"params": ev["NV_BUF_PARAMS"], "grads": ev["NV_BUF_GRADS"],
                         "adam_m": ev["NV_BUF_ADAM_M"], "adam_v": ev["NV_BUF_ADAM_V"]}
    for name, v in nvmod.KCLASS.items():
        assert ev["NV_K_" + name.upper()] == v, name


def test_binding_structs_have_the_header_layout():
    """Every argument struct the binding builds has the C struct's size and
    field offsets (a C program compiled against nv.h prints them)."""
    import shutil
    import subprocess
    from paper_2207_11620_gb300 import nv as binding
    pairs = [(binding.Volume, "nv_volume"), (binding.Camera, "nv_camera"), (binding.RenderOpts, "nv_render_opts"),
             (binding.PtOpts, "nv_pt_opts"), (binding.Macrocells, "nv_macrocells"),
             (binding.AdamCfg, "nv_adam_cfg")]
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "nv.h"', "int main(void) {"]
    for cls, cname in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    src, exe = os.path.join(out_dir, "layout.c"), os.path.join(out_dir, "layout")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    got = {}
    for ln in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for cls, cname in pairs:
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def _create(nvmod, L=8, F=2, log2T=14, Nmin=16, b=1.5, dims=(16, 64, 64, 1), prec=0):
    arr = (C.c_int * len(dims))(*dims)
    h = C.c_void_p()
    st = nvmod.lib().nv_create(L, F, log2T, Nmin, b, arr, len(dims), prec, None, C.byref(h))
    return st, h, nvmod.lib().nv_last_error().decode()


@pytest.mark.parametrize("kw,frag", [
    (dict(L=0), "L=0"), (dict(F=3), "F=3"), (dict(log2T=0), "log2T"), (dict(b=0.5), "b=0.5"),
    (dict(dims=(15, 64, 64, 1)), "mlp_dims[0]"), (dict(dims=(16, 64, 64, 2)), "output width"),
    (dict(prec=7), "prec=7"), (dict(dims=(16,)), "n_dims"),
])
def test_create_rejects_bad_arguments(nvmod, kw, frag):
    st, h, msg = _create(nvmod, **kw)
    assert st == 1 and not h.value and frag in msg


def test_entry_points_reject_null_context(nvmod):
    lib = nvmod.lib()
    assert lib.nv_infer(None, None, 0, None) == 1
    assert lib.nv_train_step(None, None, None, 1, None, 0, None) == 1
    assert lib.nv_sync(None) == 1
    assert lib.nv_destroy(None) == 0
    assert "ctx is NULL" in lib.nv_last_error().decode()


def test_renderer_rejects_bad_arguments(nvmod):
    lib = nvmod.lib()
    h = C.c_void_p()
    assert lib.nv_renderer_create(0, 8, None, C.byref(h)) == 1
    assert lib.nv_renderer_create(16, 0, None, C.byref(h)) == 1
    assert lib.nv_render(None, None, None, None, None, None, None, None) == 1


def test_sample_rejects_missing_volume(nvmod):
    lib = nvmod.lib()
    assert lib.nv_sample(None, 10, 0, 0, None, None, None) == 1
    v = nvmod.Volume(None, 4, 4, 4)
    assert lib.nv_sample(C.byref(v), 10, 0, 0, None, None, None) == 1
    v = nvmod.Volume(1234, 0, 4, 4)
    assert lib.nv_macrocells_build(C.byref(v), 16, None, None, None, None) == 1
