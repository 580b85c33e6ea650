"""Checkpoint files (paper_2509_08971_gb300/checkpoint.py) on the host: the
round trip keeps every field bit for bit, an interrupted write leaves no
partial file under the checkpoint's name, and mismatched or foreign files
are refused."""
import os
import types

import pytest

torch = pytest.importorskip("torch")
from paper_2509_08971_gb300 import checkpoint  # noqa: E402


def _mesh(dtype=torch.float64):
    return types.SimpleNamespace(shape=(4, 3, 5), gamma=1.4, bc6=(0, 0, 2, 2, 1, 1),
                                 extent=(1.0, 0.6, 0.8), dtype=dtype, scheme=0)


def test_round_trip(tmp_path):
    m = _mesh()
    g = torch.Generator().manual_seed(0)
    U = torch.rand((5,) + m.shape, generator=g, dtype=torch.float64)
    dts = [1e-3, 1.5e-3, 2.0000000000000004e-3]
    path = os.path.join(tmp_path, "run.ckpt")
    checkpoint.save(path, m, U, 0.1 + 0.2, 3, dts)
    assert not os.path.exists(path + ".tmp")
    c = checkpoint.load(path, device="cpu")
    assert torch.equal(c.U, U) and c.U.dtype == torch.float64
    assert c.t == 0.1 + 0.2 and c.step == 3 and c.dts == dts
    assert c.mesh == {"shape": [4, 3, 5], "gamma": 1.4, "bc6": [0, 0, 2, 2, 1, 1],
                      "extent": [1.0, 0.6, 0.8], "dtype": "float64", "scheme": 0}


def test_refuses_mismatches(tmp_path):
    m = _mesh(torch.float32)
    U = torch.zeros((5,) + m.shape, dtype=torch.float32)
    path = os.path.join(tmp_path, "a.ckpt")
    with pytest.raises(ValueError):
        checkpoint.save(path, m, U[:, :2], 0.0, 0)               # wrong shape
    with pytest.raises(ValueError):
        checkpoint.save(path, m, U.double(), 0.0, 0)             # wrong element type
    with pytest.raises(ValueError):
        checkpoint.save(path, m, U, 0.0, 2, [1e-3])              # one dt per step
    torch.save({"something": 1}, path)
    with pytest.raises(ValueError):
        checkpoint.load(path, device="cpu")                     # not a checkpoint
