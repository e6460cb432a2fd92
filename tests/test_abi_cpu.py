"""The C-ABI library builds, loads and exports every entry point include/splatloam.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "splatloam.h")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SPLAT_API\s+[\w\s\*]+?\b(splat_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_17491_gb300 import _lib
    return _lib.load()


def test_header_declares_the_api():
    names = declared()
    for must in ("splat_render", "splat_render_backward", "splat_render_views",
                 "splat_render_views_backward", "splat_ctx_create", "splat_loss",
                 "splat_adam_step", "splat_refine_step", "splat_get_status"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2503_17491_gb300 import _lib
    so = _lib.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in declared():
        assert name in exported, name
        assert getattr(lib, name) is not None
    # the binding covers exactly the declared entry points
    assert sorted(_lib.SIGNATURES) == declared()


def test_host_only_calls(lib):
    from paper_2503_17491_gb300 import _lib
    assert lib.splat_version() >= 100
    assert lib.splat_error_string(0) == b"ok"
    assert lib.splat_error_string(3) == b"pair capacity exceeded"
    cfg = _lib.splat_render_config()
    lib.splat_default_config(ctypes.byref(cfg))
    assert (cfg.tile_h, cfg.tile_w, cfg.flip_normals) == (16, 16, 1)
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and abs(cfg.alpha_max - 0.99) < 1e-7
    # argument validation returns before touching the device
    out = ctypes.c_void_p()
    cap = _lib.splat_capacity(10, 1, 100, 100, 0)
    assert lib.splat_ctx_create(None, ctypes.byref(cap), ctypes.byref(out)) == 1
    bad = _lib.splat_render_config()
    lib.splat_default_config(ctypes.byref(bad))
    bad.tile_h, bad.tile_w = 12, 12
    assert lib.splat_ctx_create(ctypes.byref(bad), ctypes.byref(cap), ctypes.byref(out)) == 7
    assert lib.splat_render_views(None, None, None, None, None, None) == 1
    assert lib.splat_loss(None, None, None, None, None, 0, None, None, None, None, None,
                          None) == 1


def test_no_graphics_or_fallback_imports():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2503_17491_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def _prototypes():
    """name -> parameter count of every SPLAT_API prototype in the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"SPLAT_API\s+[\w\s\*]+?\b(splat_\w+)\s*\(([^)]*)\)\s*;", text):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_arity_matches_the_header():
    from paper_2503_17491_gb300 import _lib
    protos = _prototypes()
    assert sorted(protos) == declared()
    for name, (argtypes, _) in _lib.SIGNATURES.items():
        assert len(argtypes) == protos[name], (name, len(argtypes), protos[name])


def test_argument_checks_of_the_map_and_tracking_calls(lib):
    """splat_view_loss, splat_densify and splat_photometric reject null arguments before any
    device work (status 1 = INVALID_ARG)."""
    from paper_2503_17491_gb300 import _lib
    cfg = _lib.splat_loss_config(1.0, 0.0, 1e-6, 0.0, 0.5, 1, 0.0)
    assert lib.splat_view_loss(None, None, None, None, None, None, ctypes.byref(cfg), None, None,
                               None, None, None) == 1
    dcfg = _lib.splat_densify_config(0, 0.5, 0.1, 0.05, 2.0, 2.0, 0.5, 0)
    assert lib.splat_densify(None, None, None, None, ctypes.byref(dcfg), 10, None, None, None, 0,
                             10, None) == 1
    assert lib.splat_photometric(None, 0, None, None, None, None, 0.5, 0.2, None, None,
                                 None) == 1
    # the context-free loss has no view geometry for the range-map normal mode
    assert lib.splat_loss(None, None, None, None, None, 0, ctypes.byref(cfg), None, None, None,
                          None, None) == 1
