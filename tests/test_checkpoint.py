"""Checkpoint files round-trip bit for bit (host only)."""

import json
import os

import numpy as np
import pytest

from paper_2305_15661_gb300 import checkpoint as ck
from paper_2305_15661_gb300 import workloads as W


def test_roundtrip_exact(tmp_path):
    rng = np.random.default_rng(0)
    arrays = {"a": rng.normal(size=(7, 3)), "b": np.arange(11, dtype=np.int32), "c": np.float32([1.5, -2.0]),
              "empty": np.zeros((0, 4))}
    ck.save(str(tmp_path / "m"), arrays, {"note": "x", "k": 3})
    got, meta = ck.load(str(tmp_path / "m"))
    assert meta == {"note": "x", "k": 3}
    for k, v in arrays.items():
        assert got[k].dtype == v.dtype and got[k].shape == v.shape
        np.testing.assert_array_equal(got[k], v)
    # raw little-endian files of the expected size
    assert os.path.getsize(tmp_path / "m" / "a.bin") == 7 * 3 * 8
    head = json.load(open(tmp_path / "m" / "header.json"))
    assert head["arrays"]["b"] == {"file": "b.bin", "dtype": "int32", "shape": [11]}


def test_model_checkpoint(tmp_path):
    wl = W.euler_workload(n=4, p=1, k_u=3, k_x=2, seed=5)
    rho = (np.array([1, 4, 9], dtype=np.int32), np.array([0.5, 2.0, 3.0]))
    ck.save_model(str(tmp_path / "model"), wl, rho_set=rho, train_mu=np.ones((2, 2)), train_y=np.zeros((2, 5)))
    got, meta = ck.load(str(tmp_path / "model"))
    np.testing.assert_array_equal(got["Phi"], wl.Phi)
    np.testing.assert_array_equal(got["elem_verts"], wl.ev)
    np.testing.assert_array_equal(got["rho"], rho[1])
    assert meta["p"] == 1 and meta["problem"] == wl.problem


def test_rejects_other_formats(tmp_path):
    os.makedirs(tmp_path / "bad")
    json.dump({"format": "other"}, open(tmp_path / "bad" / "header.json", "w"))
    with pytest.raises(ValueError):
        ck.load(str(tmp_path / "bad"))
