"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/fc.h declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "fc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:fc_status|size_t|const char\*)\s+(fc_\w+)\s*\(", src, re.M)))


def test_header_declares_entry_points():
    names = declared()
    for must in ("fc_setup", "fc_smooth", "fc_vcycle", "fc_solve", "fc_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2403_11636_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_2403_11636_gb300 import fc
    assert sorted(fc.EXPORTS) == declared()


def test_options_default_without_gpu():
    from paper_2403_11636_gb300 import fc
    lib = fc.load()
    o = fc.FcOptions()
    assert lib.fc_options_default(ctypes.byref(o)) == 0
    assert o.omega == 0.8 and o.eta == 1e-3 and o.fgmres_restart == 30
    # every default the header states
    assert (o.nu_pre, o.nu_post, o.quad_depth, o.cache, o.prec) == (2, 2, 4, 0, 0)
    assert (o.bc_preset, o.ubar, o.force_kind, tuple(o.force)) == (0, 0.3, 0, (0.0, 0.0, 0.0))
    assert o.nitsche_beta == 100.0 and o.dedup == 1 and o.tc == 0 and o.badcut_frac == 1e-3
    assert o.element == 0 and o.galerkin == 0
    assert lib.fc_setup(None, None, None, 1.0, 1, None, None) == fc.FC_ERR_INVALID


def test_footprint_estimate_scales():
    from paper_2403_11636_gb300 import fc, inputs
    small = fc.footprint_estimate(inputs.porous_3d(0, n=16, nspheres=2, nlevels=3))
    big = fc.footprint_estimate(inputs.porous_3d(0, n=32, nspheres=2, nlevels=4))
    assert 6 < big / small < 10
