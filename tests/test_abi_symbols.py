"""The CUDA library builds for sm_103a, loads without a GPU, and exports
every entry point declared in include/lbm_letkf.h. CPU only (no compute)."""
import ctypes
import os
import re

import pytest

from paper_2308_03972_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s*([a-z_][a-z_0-9]*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ("lbm_init", "lbm_forecast", "letkf_observe", "letkf_analyze", "lbm_moments"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert set(binding.SIGNATURES) == _declared()


def test_init_rejects_bad_arguments_without_touching_the_device(lib):
    binding.load()
    with pytest.raises(binding.LbmError) as e:
        binding.lbm_init(8, 8, 4, tau0=0.5, cs_smag=0.2, mu=0.0, stream=None)
    assert e.value.code == binding.LBM_EINVAL
    with pytest.raises(binding.LbmError) as e:
        binding.lbm_init(0, 8, 4, tau0=0.6, cs_smag=0.2, mu=0.0, stream=None)
    assert e.value.code == binding.LBM_EINVAL
    assert "nx" in binding.lbm_last_error(None)
