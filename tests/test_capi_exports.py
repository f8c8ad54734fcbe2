"""The C-ABI library loads and exports every symbol include/ags.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2503_01471_gb300 as ags
from paper_2503_01471_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(ags_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ags.lib()


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(ags.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def header_constants():
    """Integer constants of include/ags.h: object-like #defines and enum members."""
    text = open(os.path.join(ROOT, "include", "ags.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for name, expr in re.findall(r"^#define\s+(AGS_[A-Z0-9_]+)\s+([^\n(][^\n]*|\([^\n]*\))$", text, flags=re.M):
        expr = re.sub(r"(\d+)u\b", r"\1", expr.strip())
        if re.fullmatch(r"[\d\s()<x|a-fA-F]+", expr):
            out[name] = eval(expr)  # noqa: S307 (digits, shifts and or only)
    for name, val in re.findall(r"\b(AGS_[A-Z0-9_]+)\s*=\s*(\d+)", text):
        out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    consts = header_constants()
    assert len(consts) >= 20
    for name, val in consts.items():
        assert getattr(ags, name) == val, name
    assert ags.AGS_LEAF_SIZE(3) == 3 << 8 and ags.AGS_SPLIT_CELLS(64) == 64 << 12
    assert [ags.AGS_CLUSTER_RADIUS(r) for r in (16, 32, 64, 128)] == [0, 1 << 23, 2 << 23, 3 << 23]


def test_struct_layouts_match_the_header():
    assert ctypes.sizeof(ags.ags_submesh) == 32
    assert ctypes.sizeof(ags.ags_env_mesh) == 16
    assert ctypes.sizeof(ags.ags_sensor_spec) == 40
    assert ctypes.sizeof(ags.ags_hit_channels) == 32
    assert ctypes.sizeof(ags.ags_stereo) == 16
    assert ctypes.sizeof(ags.ags_render_options) == 24
    assert ctypes.sizeof(ags.ags_launch_config) == 20
    assert ctypes.sizeof(ags.ags_server_config) == 40


def test_null_arguments_are_rejected_without_a_device(lib):
    spec = ags.ags_sensor_spec(0, 4, 4, 1.0, 0, 0, 0.1, 10.0, 0, 0)
    assert lib.ags_render(None, None, ctypes.byref(spec), None, None, None, None) == ags.AGS_ERR_INVALID_ARG
    assert "NULL" in ags.ags_last_error()
    h = ctypes.c_void_p()
    assert lib.ags_scene_build(None, None, 1, None, 0, ctypes.byref(h)) == ags.AGS_ERR_INVALID_ARG
    assert lib.ags_scene_n_envs(None) == -1


def test_context_on_a_missing_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.ags_context_create(0, ctypes.byref(h))
    assert st in (ags.AGS_ERR_CUDA, ags.AGS_ERR_INVALID_ARG)
    assert h.value is None
    assert ags.ags_last_error() != ""


def test_header_compiles_as_c_and_links(tmp_path, lib):
    """include/ags.h is plain C: a C99 program that takes the address of every declared function compiles
    with warnings as errors and links against the library; creating a context without a device fails with
    a status, not a crash."""
    names = declared_functions()
    src = tmp_path / "use_ags.c"
    body = "\n".join(f"  (void (*)(void))&{n}," for n in names)
    src.write_text(f"""#include <stdio.h>
#include "ags.h"
static void (*const table[])(void) = {{
{body}
}};
int main(void) {{
  ags_context *ctx = 0;
  ags_status st = ags_context_create(0, &ctx);
  if (st == AGS_OK) ags_context_destroy(ctx);
  printf("%d %d\\n", (int)(sizeof table / sizeof table[0]), (int)st);
  printf("%d %d %d %d %d %d %d %d\\n", (int)sizeof(ags_submesh), (int)sizeof(ags_env_mesh),
         (int)sizeof(ags_sensor_spec), (int)sizeof(ags_hit_channels), (int)sizeof(ags_stereo),
         (int)sizeof(ags_render_options), (int)sizeof(ags_launch_config), (int)sizeof(ags_server_config));
  printf("%u %u %u %u\\n", (unsigned)AGS_CLUSTER_RADIUS(16), (unsigned)AGS_CLUSTER_RADIUS(32),
         (unsigned)AGS_CLUSTER_RADIUS(64), (unsigned)AGS_CLUSTER_RADIUS(128));
  return 0;
}}
""")
    import subprocess
    exe = tmp_path / "use_ags"
    so = B.LIB if hasattr(B, "LIB") else None
    libdir = os.path.dirname(so) if so else os.path.join(ROOT, "paper_2503_01471_gb300", "_build")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lags", f"-Wl,-rpath,{libdir}"], check=True)
    import torch
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == len(names)
    # the C compiler's struct sizes equal the binding's
    assert [int(x) for x in out[2:10]] == [ctypes.sizeof(t) for t in (
        ags.ags_submesh, ags.ags_env_mesh, ags.ags_sensor_spec, ags.ags_hit_channels, ags.ags_stereo,
        ags.ags_render_options, ags.ags_launch_config, ags.ags_server_config)]
    # the header's macros encode as the binding's helpers do
    assert [int(x) for x in out[10:14]] == [ags.AGS_CLUSTER_RADIUS(r) for r in (16, 32, 64, 128)]
    if not torch.cuda.is_available():
        assert int(out[1]) != 0  # no device here: an error status


def test_render_wrappers_refuse_host_buffers_before_any_call():
    """A kernel would write through a host array's address: the binding refuses host arrays and CPU tensors as
    device buffers, on the host, before the library is asked to launch anything."""
    import numpy as np
    import torch

    from paper_2503_01471_gb300 import scenes as S
    spec = S.pinhole(4, 4)
    dev_like = [np.zeros((1, 4, 4), np.float32), torch.zeros((1, 4, 4))]
    for bad in dev_like:
        with pytest.raises(ValueError):
            ags.ags_render(0, None, spec, None, bad, None)
    with pytest.raises(ValueError):
        ags.ags_render_ex(0, None, spec, None, None, None, normal=np.zeros(3, np.float32))
    with pytest.raises(ValueError):
        ags.ags_render_envs(0, None, spec, np.zeros(1, np.int32), None, None, None)
