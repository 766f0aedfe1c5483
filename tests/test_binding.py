"""Host-side checks of the Python binding that run without a GPU: argument marshalling
rejects host tensors, wrong dtypes and wrong shapes before any library call, the
constants mirror the public header, and learned-guess checkpoints are validated before
any device work."""
import os
import re

import numpy as np
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


def test_checkpoint_header_is_checked_before_any_device_work(tmp_path):
    import struct
    from paper_2011_01207_gb300 import learned
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"NOTMAGIC" + b"\0" * 16)
    with pytest.raises(ValueError, match="not an MLP checkpoint"):
        learned.Trainer.load(str(bad), device="cpu")
    short = tmp_path / "short.ckpt"
    short.write_bytes(learned.MAGIC + struct.pack("<qq", 10, 3) + b"\0" * (4 * 25))
    with pytest.raises(ValueError, match="does not match"):
        learned.Trainer.load(str(short), device="cpu")
    long_ = tmp_path / "long.ckpt"
    long_.write_bytes(learned.MAGIC + struct.pack("<qq", 10, 3) + b"\0" * (4 * 31))
    with pytest.raises(ValueError, match="does not match"):
        learned.Trainer.load(str(long_), device="cpu")
    head = tmp_path / "head.ckpt"
    head.write_bytes(learned.MAGIC + b"\0" * 5)
    with pytest.raises(ValueError, match="truncated"):
        learned.Trainer.load(str(head), device="cpu")


def test_initial_parameters_fit_the_network_shape():
    from paper_2011_01207_gb300 import learned
    p = learned.init_params(3)
    assert p.dtype == np.float32 and p.size == 16 * 128 + 128 + 128 * 128 + 128 + 128 * 3 + 3
    assert np.array_equal(p, learned.init_params(3)) and not np.array_equal(p, learned.init_params(4))
