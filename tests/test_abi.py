"""The C ABI without a GPU: the library builds, loads, exports every function
declared in include/slpic.h, and the ctypes structures match the C layout."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1511_08225_gb300 import binding
from paper_1511_08225_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "slpic.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(slpic_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return ctypes.CDLL(binding.LIB_PATH)


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == names


def test_binding_loads_and_sets_signatures(lib):
    L = binding.load_library()
    assert L.slpic_step.argtypes is not None


def test_struct_layout_matches_c(tmp_path):
    """Compile a host program against slpic.h and compare sizeof/offsetof
    with the ctypes mirror (a silent mismatch would scramble the config)."""
    prog = tmp_path / "layout.c"
    fields_cfg = [f for f, _ in binding.slpic_config._fields_]
    fields_sp = [f for f, _ in binding.slpic_species._fields_]
    fields_dg = [f for f, _ in binding.slpic_diag._fields_]
    fields_tu = [f for f, _ in binding.slpic_tuning._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "slpic.h"', 'int main(void){']
    for st, fl in (("slpic_config", fields_cfg), ("slpic_species", fields_sp),
                   ("slpic_diag", fields_dg), ("slpic_tuning", fields_tu)):
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fl:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    for line in out:
        if not line.strip():
            continue
        parts = line.split()
        cls = getattr(binding, parts[0])
        if parts[1] == "size":
            assert ctypes.sizeof(cls) == int(parts[2]), line
        else:
            assert getattr(cls, parts[1]).offset == int(parts[2]), line


def test_create_without_gpu_fails_cleanly(lib):
    """With no device, slpic_create returns an error code and a message
    instead of crashing (on a GPU machine this test is skipped)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1511_08225_gb300 import inputs
    cfg = binding.config_from_problem(inputs.periodic_problem(n_cells=16, ppc=2))
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_create(cfg)
    assert ei.value.code == binding.SLPIC_ERR_CUDA


def test_config_errors_need_no_device(lib):
    """Config validation runs before any device call: CFL violations and bad
    source bands are refused with their own codes on any machine."""
    from paper_1511_08225_gb300 import inputs
    prob = inputs.sheath_problem(n_cells=64, ppc=2, v0=0.1)
    prob["dt"] = 2 * prob["dx"] / 0.1
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_create(binding.config_from_problem(prob))
    assert ei.value.code == binding.SLPIC_ERR_CFL
    prob = inputs.sheath_problem(n_cells=64, ppc=2, v0=0.1)
    prob["source"]["len_cells"] = 64.0
    with pytest.raises(binding.SlpicError) as ei:
        binding.slpic_create(binding.config_from_problem(prob))
    assert ei.value.code == binding.SLPIC_ERR_INVALID


# ------------------------------------------------------------------ 2D entry points
HEADER2D = os.path.join(ROOT, "include", "slpic2d.h")


def test_every_2d_function_is_exported(lib):
    from paper_1511_08225_gb300 import binding2d
    src = re.sub(r"/\*.*?\*/", "", open(HEADER2D).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(slpic2d_[a-z0-9_]+)\s*\(", src)))
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding2d.EXPORTS2D) == names
    assert binding2d.load_library().slpic2d_step.argtypes is not None


def test_2d_struct_layout_matches_c(tmp_path):
    from paper_1511_08225_gb300 import binding2d
    prog = tmp_path / "layout2d.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "slpic2d.h"', 'int main(void){']
    for st in ("slpic2d_config", "slpic2d_diag"):
        cls = getattr(binding2d, st)
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout2d"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    for line in subprocess.check_output([str(exe)], text=True).split("\n"):
        if not line.strip():
            continue
        parts = line.split()
        cls = getattr(binding2d, parts[0])
        if parts[1] == "size":
            assert ctypes.sizeof(cls) == int(parts[2]), line
        else:
            assert getattr(cls, parts[1]).offset == int(parts[2]), line


def test_2d_config_errors_need_no_device(lib):
    from paper_1511_08225_gb300 import binding2d, inputs
    prob = inputs.plasma2d_problem(nx=16, ny=16, ppc=1)
    prob["dt"] = 2 * prob["dx"] / 0.1
    with pytest.raises(binding.SlpicError) as ei:
        binding2d.slpic2d_create(binding2d.config_from_problem(prob))
    assert ei.value.code == binding.SLPIC_ERR_CFL
    for key, val in (("cg_rtol", 0.0), ("cg_maxit", 0), ("nx", 1)):
        prob = inputs.plasma2d_problem(nx=16, ny=16, ppc=1)
        prob[key] = val
        with pytest.raises(binding.SlpicError) as ei:
            binding2d.slpic2d_create(binding2d.config_from_problem(prob))
        assert ei.value.code == binding.SLPIC_ERR_INVALID
    prob = inputs.plasma2d_problem(nx=16, ny=16, ppc=1)
    prob["source"]["len_cells"] = 16.0
    with pytest.raises(binding.SlpicError) as ei:
        binding2d.slpic2d_create(binding2d.config_from_problem(prob))
    assert ei.value.code == binding.SLPIC_ERR_INVALID


def test_every_fp64_function_is_exported(lib):
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "slpic_fp64.h")).read(),
                 flags=re.S)
    names = sorted(set(re.findall(r"\b(slpic_fp64_[a-z0-9_]+)\s*\(", src)))
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS_FP64) == names


# ------------------------------------------------------------------ U-Net entry points
def test_every_unet_function_is_exported(lib):
    from paper_1511_08225_gb300 import binding_unet
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "slpic_unet.h")).read(),
                 flags=re.S)
    names = sorted(set(re.findall(r"\b(slpic_unet_[a-z0-9_]+)\s*\(", src)))
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding_unet.EXPORTS_UNET) == names
    assert binding_unet.load_library().slpic_unet_forward.argtypes is not None


def test_unet_config_layout_matches_c(tmp_path):
    from paper_1511_08225_gb300 import binding_unet
    cls = binding_unet.slpic_unet_config
    prog = tmp_path / "layout_unet.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "slpic_unet.h"', 'int main(void){',
             'printf("size %zu\\n", sizeof(slpic_unet_config));']
    for f, _ in cls._fields_:
        lines.append(f'printf("{f} %zu\\n", offsetof(slpic_unet_config, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout_unet"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    for line in subprocess.check_output([str(exe)], text=True).split("\n"):
        if line.strip():
            name, val = line.split()
            want = ctypes.sizeof(cls) if name == "size" else getattr(cls, name).offset
            assert want == int(val), line


@pytest.mark.parametrize("bad", [dict(levels=0), dict(base=0), dict(height=30),
                                 dict(width=12, levels=4), dict(max_batch=0),
                                 dict(out_scale=0.0), dict(levels=13), dict(loss=2)])
def test_unet_config_errors_need_no_device(lib, bad):
    from paper_1511_08225_gb300 import binding_unet
    c = binding_unet.slpic_unet_config()
    c.levels, c.base, c.height, c.width, c.max_batch, c.out_scale = 3, 4, 32, 32, 1, 1.0
    for k, v in bad.items():
        setattr(c, k, v)
    with pytest.raises(binding.SlpicError) as ei:
        binding_unet.slpic_unet_create(c)
    assert ei.value.code == binding.SLPIC_ERR_INVALID


def test_unet_parameter_layout_round_trips():
    from oracle import unet as ounet
    from paper_1511_08225_gb300 import binding_unet
    assert binding_unet.layer_shapes(3, 4) == ounet.layer_shapes(3, 4)
    params = ounet.init_params(3, 4, seed=1)
    flat = binding_unet.join_params(params)
    back = binding_unet.split_params(flat, 3, 4)
    for (w, b), (w2, b2) in zip(params, back):
        assert np.array_equal(np.float32(w), w2) and np.array_equal(np.float32(b), b2)
