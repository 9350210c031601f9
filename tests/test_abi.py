"""The C-ABI library loads, exports every entry point include/*.h declares, and
rejects invalid descriptors on the host (no GPU needed for any of this)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1812_03358_b300 import build, inputs as I, lt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(testing=False):
    """lt_* entry points of include/*.h; the fault-injection header
    (lt_testing.h) only for the test build."""
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        if os.path.basename(h) == "lt_testing.h" and not testing:
            continue
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(lt_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def library():
    build.build()
    return lt.lib()


def test_every_declared_symbol_is_exported(library):
    names = declared_symbols()
    assert "lt_forward" in names and "lt_adjoint" in names and "lt_plan_create" in names
    missing = [n for n in names if not hasattr(library, n)]
    assert not missing, missing


def _exported(path):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    return {l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("lt_")}


def test_only_declared_symbols_are_exported(library):
    assert _exported(build.LIB) == set(declared_symbols())


def test_test_build_adds_only_the_fault_injection_entry_points(library):
    testing = set(declared_symbols(testing=True)) - set(declared_symbols())
    assert testing == {"lt_test_fail_allocation_after", "lt_nn_test_stall_tensor_core"}
    assert _exported(build.TEST_LIB) == set(declared_symbols(testing=True))


def test_invalid_descriptors_rejected_on_host(library):
    vol, cam = I.config_single_small()
    with pytest.raises(lt.LtError) as e:
        lt.lt_plan_create(I.Volume(0, 4, 4, 1, 1, 1), [cam])
    assert e.value.status == lt.LT_EINVAL and "positive" in str(e.value)
    bad = I.Camera(**{**cam.__dict__, "f_main": -1.0})
    with pytest.raises(lt.LtError) as e:
        lt.lt_plan_create(vol, [bad])
    assert e.value.status == lt.LT_EINVAL
    near = I.Camera(**{**cam.__dict__, "d_obj": 10.0})
    with pytest.raises(lt.LtError) as e:
        lt.lt_plan_create(vol, [near])
    assert e.value.status == lt.LT_EINVAL and "main lens" in str(e.value)
    _, pc = I.config_plenoptic()
    wide = I.Camera(**{**pc.__dict__, "mla_radius": pc.mla_pitch})
    with pytest.raises(lt.LtError) as e:
        lt.lt_plan_create(vol, [wide])
    assert e.value.status == lt.LT_EINVAL and "radius" in str(e.value)
    with pytest.raises(lt.LtError) as e:
        lt.lt_plan_create(vol, [cam], n_frames=0)
    assert e.value.status == lt.LT_EINVAL
    with pytest.raises(lt.LtError) as e:
        lt.lt_plan_sizes(None, 1)
    assert e.value.status == lt.LT_EINVAL


def test_orientation_and_mla_fields_validated_on_host(library):
    vol, cam = I.config_single_small()
    nan_pitch = I.Camera(**{**cam.__dict__, "pitch": float("nan")})
    with pytest.raises(lt.LtError) as e:
        lt.lt_plan_create(vol, [nan_pitch])
    assert e.value.status == lt.LT_EINVAL and "pitch" in str(e.value)
    _, pc = I.config_plenoptic()
    bad_layout = I.Camera(**{**pc.__dict__, "mla_layout": 7})
    with pytest.raises(lt.LtError) as e:
        lt.lt_plan_create(vol, [bad_layout])
    assert e.value.status == lt.LT_EINVAL and "mla_layout" in str(e.value)



def test_binding_refuses_to_run_without_the_library(monkeypatch):
    """No CPU fallback: with the library absent, the first call raises."""
    from paper_1812_03358_b300 import inputs as I
    from paper_1812_03358_b300 import lt as LT
    monkeypatch.setattr(LT, "_lib", None)
    monkeypatch.setattr(LT, "LIB_PATH", "/nonexistent/liblt.so")
    with pytest.raises(RuntimeError, match="missing"):
        LT.Plan(I.Volume(4, 4, 4, 1.0, 1.0, 1.0), [I.table_single_lens(8, 0.1)])
