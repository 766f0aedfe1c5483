"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every symbol the
public header declares; argument checks that run before any device work."""
import ctypes
import os
import re

import pytest

from paper_2011_01207_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return ctypes.CDLL(build.LIB)


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                            txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "induced_dipoles_pcg" in names and "build_neighbour_blocks" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(binding.EXPORTS) <= set(names)


def test_create_rejects_bad_parameters_before_touching_a_device(lib):
    binding.load()
    p = binding.make_params(0, (20.0, 20.0, 20.0))
    with pytest.raises(binding.ApError, match="AP_ERR_ARG"):
        binding.ap_create(p)
    p = binding.make_params(100, (10.0, 10.0, 10.0), cutoff=7.0, buffer=2.0)
    with pytest.raises(binding.ApError, match="box"):
        binding.ap_create(p)
    p = binding.make_params(100, (30.0, 30.0, 30.0))
    p.pme_order = 4
    with pytest.raises(binding.ApError, match="pme_order"):
        binding.ap_create(p)


def test_null_context_calls_return_arg_error(lib):
    binding.load()
    L = binding.load()
    assert L.build_neighbour_blocks(None, None, None, None, 0) == -1
    assert L.permanent_field(None, None, None, None, None, None) == -1
    assert L.induced_dipoles_pcg(None, None, 1e-5, 10, None, None) == -1
    assert L.polarization_energy_forces(None, None, None, None, None) == -1
    assert L.induced_dipoles_diis(None, None, 1e-5, 10, 6, None, None) == -1
    assert L.set_scaled_pairs(None, 0, None, None) == -1
    assert L.permanent_field_dp(None, None, None, None, None, None, None) == -1
    assert L.induced_dipoles_pcg_dp(None, None, None, 1e-5, 10, None, None, None) == -1
    assert L.polarization_energy_forces_dp(None, None, None, None, None, None) == -1
