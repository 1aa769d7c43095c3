"""CPU checks of the boundary: the C-ABI library builds for sm_103a, loads,
and exports every entry point include/adgi.h declares; the binding uses the
same names; the oracle and the CUDA path share no source."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "adgi.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(adgi_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2301_05125_gb300 import build

    return build.build()


def test_header_declares_the_five_core_calls():
    names = _declared()
    for n in ("adgi_create_volume", "adgi_set_scene", "adgi_update", "adgi_query_irradiance", "adgi_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath]).decode()
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_names_match(libpath):
    from paper_2301_05125_gb300 import adgi

    L = adgi.load(libpath)
    for n in _declared():
        assert hasattr(L, n)
        assert hasattr(adgi, n), "binding lacks %s" % n
    assert adgi.adgi_last_error() == ""


def test_library_is_sm_103a(libpath):
    out = subprocess.check_output(["cuobjdump", "--list-elf", libpath]).decode()
    assert "sm_103a" in out


def test_oracle_and_cuda_path_share_no_source():
    csrc = os.path.join(ROOT, "paper_2301_05125_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in re.findall(r'#include\s+"([^"]+)"', txt).__str__()
    otxt = open(os.path.join(ROOT, "oracle", "adgi_oracle.c")).read()
    for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', otxt):
        assert not inc.startswith("adgi") and "csrc" not in inc and "include/" not in inc
    for f in ("adgi.py", "build.py", "scenegen.py", "__init__.py"):
        txt = open(os.path.join(ROOT, "paper_2301_05125_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt


def test_errors_without_gpu_work():
    """Argument validation runs on the host and fails loudly."""
    from paper_2301_05125_gb300 import adgi

    d = adgi.make_desc((0, 0, 0), (1, 1, 1), (1, 4, 4))
    with pytest.raises(adgi.AdgiError) as e:
        adgi.adgi_create_volume(d)
    assert e.value.code == -1 and "dims" in str(e.value)
    d = adgi.make_desc((0, 0, 0), (1, 1, 1), (2, 2, 2), rays_avg=7)
    with pytest.raises(adgi.AdgiError):
        adgi.adgi_create_volume(d)


def test_tick_arguments_checked_on_the_host():
    """The persistent tick rejects bad arguments before any device work."""
    import ctypes as C

    from paper_2301_05125_gb300 import adgi

    L = adgi.load()
    out = C.c_void_p()
    assert L.adgi_tick_create(None, 1, None, C.byref(out)) == -1
    arr = (C.c_void_p * 1)(None)
    assert L.adgi_tick_create(arr, 1, None, C.byref(out)) == -1 and "NULL volume" in adgi.adgi_last_error()
    assert L.adgi_tick_create(arr, 0, None, C.byref(out)) == -1
    assert L.adgi_tick_update(None, None) == -1
    assert L.adgi_tick_sync(None) == -1
    assert L.adgi_tick_set_wait(None, 1000, -1) == -1
    assert L.adgi_tick_phase_ns(None, None, 0) == -1
    assert L.adgi_tick_destroy(None) == 0
