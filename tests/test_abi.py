"""The C ABI library loads and exports every declared entry point (no GPU).

No compute call is made here: only symbol lookup, struct layouts and
argument checks that fail before any device is touched.
"""

import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2405_14903_b300 import _lib
    return _lib.lib


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nf_create", "nf_destroy", "nf_episode_create", "nf_set_params",
                     "nf_set_velocity", "nf_step", "nf_backward_step", "nf_backward",
                     "nf_get_velocity", "nf_get_pressure", "nf_get_fractions", "nf_loss",
                     "nf_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_signatures_cover_the_header():
    from paper_2405_14903_b300 import _lib
    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_kernel_class_names_match_the_header():
    from paper_2405_14903_b300 import _lib
    src = open(HEADER).read()
    codes = dict(re.findall(r"#define NF_K_([A-Z0-9_]+) (\d+)", src))
    assert int(codes.pop("COUNT")) == len(_lib.KCLASS)
    for name, code in codes.items():
        assert _lib.KCLASS[int(code)] == name.lower()


def test_status_strings_and_defaults(lib):
    from paper_2405_14903_b300 import _lib
    for s in range(0, 9):
        assert lib.nf_status_string(s) != b"unknown status"
    cfg = _lib.Config()
    assert lib.nf_config_default(ctypes.byref(cfg)) == 0
    assert cfg.precision == _lib.PREC["mixed"] and cfg.solver == _lib.SOLVER["mgpcg"]
    assert cfg.checkpoint_every == 10 and abs(cfg.tol - 1e-6) < 1e-18
    assert cfg.mg_transfer == 1 and cfg.mg_persistent == 0 and cfg.residual_fp64 == 1 and cfg.mg_fused == 0 and cfg.recompute_overlap == 1
    assert cfg.mg_cluster == 0


def test_invalid_arguments_are_rejected_without_a_device(lib):
    from paper_2405_14903_b300 import _lib
    assert lib.nf_config_default(None) == _lib.NF_E_INVALID
    assert lib.nf_create(None, None) == _lib.NF_E_INVALID
    assert lib.nf_destroy(None) == _lib.NF_E_INVALID
    cfg = _lib.Config()
    lib.nf_config_default(ctypes.byref(cfg))
    cfg.tol = -1.0
    h = ctypes.c_void_p()
    assert lib.nf_create(ctypes.byref(h), ctypes.byref(cfg)) == _lib.NF_E_INVALID
    lib.nf_config_default(ctypes.byref(cfg))
    cfg.mg_persistent = 2
    assert lib.nf_create(ctypes.byref(h), ctypes.byref(cfg)) == _lib.NF_E_INVALID


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors must have the sizes the C compiler gives the header's
    # structs (compiled here with the host compiler)
    from paper_2405_14903_b300 import _lib
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "nf.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu %zu", '
                   'sizeof(nf_config), sizeof(nf_grid), sizeof(nf_scene), sizeof(nf_step_stats), '
                   'sizeof(nf_request), sizeof(nf_result), sizeof(nf_server_stats));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sizes = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert sizes == [ctypes.sizeof(_lib.Config), ctypes.sizeof(_lib.Grid),
                     ctypes.sizeof(_lib.Scene), ctypes.sizeof(_lib.StepStats),
                     ctypes.sizeof(_lib.Request), ctypes.sizeof(_lib.Result),
                     ctypes.sizeof(_lib.ServerStats)]


def test_server_rejects_bad_arguments_without_a_device(lib):
    from paper_2405_14903_b300 import _lib
    cfg = _lib.Config()
    lib.nf_config_default(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    assert lib.nf_server_create(None, 2, 0, ctypes.byref(h)) == _lib.NF_E_INVALID
    assert lib.nf_server_create(ctypes.byref(cfg), 0, 0, ctypes.byref(h)) == _lib.NF_E_INVALID
    assert lib.nf_server_create(ctypes.byref(cfg), 65, 0, ctypes.byref(h)) == _lib.NF_E_INVALID
    assert lib.nf_server_submit(None, None, None) == _lib.NF_E_INVALID
    r = _lib.Result()
    assert lib.nf_server_poll(None, 1, 0, ctypes.byref(r)) == _lib.NF_E_INVALID
    assert lib.nf_server_drain(None, 0) == _lib.NF_E_INVALID
    assert lib.nf_server_destroy(None) == _lib.NF_E_INVALID


def test_grid_marshalling_of_viscosity_and_fraction_rule():
    # host-side marshalling of nf_grid (no device): nu and the fraction rule
    # reach the struct with the header's codes; what the library cannot run
    # is refused before any call
    import nf_inputs as I
    from paper_2405_14903_b300 import _lib
    from paper_2405_14903_b300.api import grid_struct
    src = open(HEADER).read()
    codes = dict(re.findall(r"#define NF_FRACTIONS_([A-Z]+) (\d+)", src))
    assert {k.lower(): int(v) for k, v in codes.items()} == _lib.FRACTIONS
    g = grid_struct(dict(I.make_grid(8, 0.01, nu=0.03), fractions="corner"))
    assert g.nu == 0.03 and g.fractions == _lib.FRACTIONS["corner"]
    g = grid_struct(I.make_grid(8, 0.01))
    assert g.nu == 0.0 and g.fractions == _lib.FRACTIONS["supersample"]
    with pytest.raises(ValueError):
        grid_struct(dict(I.make_grid(8, 0.01), fractions="marching"))
    with pytest.raises(ValueError):
        grid_struct(I.make_grid(8, 0.01, periodic=True))
    g = grid_struct(I.make_grid(8, 0.01, inlet=I.centred_inlet(8, 2, 0.3)))
    assert (g.inlet, g.inlet_side, g.inlet_j0, g.inlet_k0, g.inlet_w, g.inlet_h) == \
        (1, -1, 3, 3, 2, 2) and g.inlet_speed == 0.3
    with pytest.raises(ValueError):
        grid_struct(I.make_grid(8, 0.01, inlet=dict(I.centred_inlet(8, 2, 0.3), axis=1)))


def test_struct_field_offsets_match_the_header(tmp_path):
    # every field of every ctypes mirror sits at the offset the C compiler
    # gives the header's field of the same name (catches reordered fields that
    # keep the total size)
    from paper_2405_14903_b300 import _lib
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no host C compiler")
    mirrors = {"nf_config": _lib.Config, "nf_grid": _lib.Grid, "nf_scene": _lib.Scene,
               "nf_step_stats": _lib.StepStats, "nf_request": _lib.Request,
               "nf_result": _lib.Result, "nf_server_stats": _lib.ServerStats}
    lines, want = [], []
    for cname, cls in mirrors.items():
        for fname, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {fname}));')
            want.append((cname, fname, getattr(cls, fname).offset))
    src = tmp_path / "off.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "nf.h"\nint main(void){'
                   + "".join(lines) + "return 0;}\n")
    exe = tmp_path / "off"
    subprocess.check_call([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert len(got) == len(want)
    for g, (cname, fname, off) in zip(got, want):
        assert g == off, (cname, fname, g, off)
