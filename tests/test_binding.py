"""Host-side checks of the Python binding that run without a GPU: argument marshalling
rejects host tensors, wrong dtypes and wrong shapes before any library call, and the
constants mirror the public header."""
import os
import re

import pytest

torch = pytest.importorskip("torch")

from paper_2011_01207_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ptr_rejects_host_tensors_and_missing_inputs():
    with pytest.raises(binding.ApError, match="CUDA tensor"):
        binding._ptr(torch.zeros((4, 3), dtype=torch.float64), torch.float64, (4, 3), "xyz")
    with pytest.raises(binding.ApError, match="required"):
        binding._ptr(None, torch.float64, (4, 3), "xyz")
    assert binding._ptr(None, torch.float64, (4, 3), "guess", allow_none=True) is None


def test_header_constants_match_the_binding():
    txt = open(os.path.join(ROOT, "include", "amoebapol.h")).read()
    consts = dict(re.findall(r"#define\s+(AP_[A-Z0-9_]+)\s+(-?\d+)", txt))
    assert int(consts["AP_MIXED"]) == binding.AP_MIXED
    assert int(consts["AP_FP64"]) == binding.AP_FP64
    assert int(consts["AP_FIXED"]) == binding.AP_FIXED
    assert int(consts["AP_ADAPTIVE_SCRATCH"]) == binding.AP_ADAPTIVE_SCRATCH
    assert int(consts["AP_NOT_CONVERGED"]) == binding.AP_NOT_CONVERGED
    kernels = {k: int(v) for k, v in consts.items() if k.startswith("AP_KERNEL_")}
    assert {("AP_KERNEL_" + k.upper()): v for k, v in binding.KERNELS.items()} == kernels


def test_batch_step_layout_matches_the_header():
    """The ctypes mirror of ap_batch_step lists the header's fields in the header's order."""
    txt = open(os.path.join(ROOT, "include", "amoebapol.h")).read()
    body = txt[txt.index("typedef struct {", txt.index("typedef struct ap_batch ap_batch;")):
               txt.index("} ap_batch_step;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"([A-Za-z_][A-Za-z0-9_]*)\s*;", body)
    assert fields == [name for name, _ in binding.ApBatchStep._fields_]
