"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares (no compute calls: those need a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"^MS2_API\s+[\w\s\*]+?\b(ms2_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1507_07548_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["ms2_create_system", "ms2_step", "ms2_energy_virial", "ms2_forces_torques", "ms2_ewald_params",
                     "ms2_get_state", "ms2_set_state", "ms2_rdf", "ms2_batch_create", "ms2_batch_step",
                     "ms2_serve_open", "ms2_serve_submit", "ms2_serve_poll", "ms2_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1507_07548_gb300 import ms2
    assert set(declared_symbols()) <= set(ms2.SIGNATURES)


def test_host_only_calls_work_without_gpu(lib):
    from paper_1507_07548_gb300 import ms2
    assert ms2.lib().ms2_version().startswith(b"ms2-gb300")
    o = ms2.ms2_options()
    assert ms2.lib().ms2_default_options(ctypes.byref(o)) == 0
    assert o.quat_iters == 3 and o.thermostat == 1 and o.lrc == 1
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert ms2.lib().ms2_create_system(None, None, 0, 10.0, 1.0, 0.0, 4.0, 0, None, ctypes.byref(h)) == 1
    assert b"n_models" in ms2.lib().ms2_last_error()
