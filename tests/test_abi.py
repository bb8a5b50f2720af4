"""CPU checks of the C ABI: the library builds, loads, exports every symbol
include/rll.h declares, and its host-side argument checks answer without a
GPU (no compute is launched here)."""
import ctypes
import os
import subprocess
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "rll.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rll_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1911_10217_gb300 import build, rll
    build.build()
    return rll.load(build_if_missing=False)


def test_every_declared_symbol_is_exported(lib):
    from paper_1911_10217_gb300 import rll
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(rll.EXPORTS) == names


def test_null_arguments_are_rejected(lib):
    P = ctypes.c_void_p
    assert lib.rll_build_light_tree(None, None, None, 0, None) == 1
    assert lib.rll_learn_update(None, None, None, None, 0) == 1
    assert lib.rll_split_collapse(None, None, None) == 1
    assert lib.rll_sample_and_shade(None, None, None, None, None, None, 0, None, 0, 0, 0, 1, None,
                                    None, None) == 1
    assert lib.rll_ctx_create(None, 0, None) == 1
    assert lib.rll_ctx_destroy(None) == 0
    assert lib.rll_tree_destroy(None) == 0
    assert lib.rll_grid_destroy(None) == 0
    assert lib.rll_tree_num_lights(None) == 0
    assert lib.rll_grid_cut_len(None) == 0
    assert lib.rll_last_error(None) == b"no context"
    assert lib.rll_grid_touched_cells(None, None, None) == 1
    assert lib.rll_bounce_vertices(None, None, None, 0, None, 0, None, 0, 0, 1.0, None, None, None) == 1
    del P


def test_context_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    rc = lib.rll_ctx_create(ctypes.byref(h), 0, None)
    assert rc == 3 and not h.value  # RLL_E_CUDA, no handle


def test_grid_params_layout_matches_header(lib, tmp_path):
    from paper_1911_10217_gb300 import rll
    # 2 u32 + 3 f32 + f32 + 5 u32 + 4 f32 + 2 u32 = 17 words
    assert ctypes.sizeof(rll.GridParams) == 68
    assert ctypes.sizeof(rll.SampleDebug) == 3 * ctypes.sizeof(ctypes.c_void_p)
    # the C compiler's view of the header agrees, field by field
    prog = tmp_path / "layout.c"
    fields = [f for f, _ in rll.GridParams._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rll.h"', "int main(void) {",
             'printf("%zu\\n", sizeof(rll_grid_params));']
    lines += [f'printf("%zu\\n", offsetof(rll_grid_params, {f}));' for f in fields]
    lines += ["return 0; }"]
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert out[0] == ctypes.sizeof(rll.GridParams)
    assert out[1:] == [getattr(rll.GridParams, f).offset for f in fields]


def test_oracle_builds_independently():
    """The oracle is a separate C file: it includes no header of the CUDA
    library and the library includes nothing from it."""
    src = open(os.path.join(ROOT, "oracle", "rll_oracle.c")).read()
    assert "#include \"" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_1911_10217_gb300", "csrc")):
        text = open(os.path.join(ROOT, "paper_1911_10217_gb300", "csrc", f)).read()
        assert "oracle" not in text.lower(), f
