"""Checkpoint and resume of a trained hyperreduced model.

A checkpoint is a directory with one raw little-endian binary per array and a
JSON header listing each array's file, dtype and shape plus free-form metadata,
so that training (bases, weights, the network and its training set) and serving
can restart without recomputing. Nothing here runs on the GPU; the network's
parameters go through the library's get/set calls.
"""

from __future__ import annotations

import json
import os

import numpy as np

HEADER = "header.json"
_DTYPES = {"float64": "<f8", "float32": "<f4", "int32": "<i4", "int64": "<i8", "int8": "<i1", "uint8": "<u1"}


def save(path: str, arrays: dict, meta: dict | None = None) -> None:
    """Write arrays (name -> ndarray) and meta (JSON-serialisable) under path."""
    os.makedirs(path, exist_ok=True)
    entries = {}
    for name, a in arrays.items():
        a = np.asarray(a)
        key = a.dtype.name
        if key not in _DTYPES:
            raise ValueError(f"unsupported dtype {key} for {name}")
        fn = f"{name}.bin"
        np.ascontiguousarray(a, dtype=np.dtype(_DTYPES[key])).tofile(os.path.join(path, fn))
        entries[name] = {"file": fn, "dtype": key, "shape": list(a.shape)}
    with open(os.path.join(path, HEADER), "w") as f:
        json.dump({"format": "ift-checkpoint-1", "arrays": entries, "meta": meta or {}}, f, indent=1)


def load(path: str):
    """Read a checkpoint written by save: (arrays, meta)."""
    with open(os.path.join(path, HEADER)) as f:
        head = json.load(f)
    if head.get("format") != "ift-checkpoint-1":
        raise ValueError("not a checkpoint of this format")
    arrays = {}
    for name, e in head["arrays"].items():
        a = np.fromfile(os.path.join(path, e["file"]), dtype=np.dtype(_DTYPES[e["dtype"]]))
        arrays[name] = a.reshape(e["shape"]).astype(np.dtype(e["dtype"]), copy=False)
    return arrays, head["meta"]


def save_model(path: str, wl, rho_set=None, mlp=None, train_mu=None, train_y=None, meta=None) -> None:
    """Mesh, bases, empirical-quadrature weights, and optionally the warm-start
    network (parameters, architecture) with its training set."""
    arrays = {"X": wl.X, "elem_verts": np.asarray(wl.ev, dtype=np.int32), "Phi": wl.Phi, "Psi": wl.Psi}
    m = {"problem": int(wl.problem), "p": int(wl.p), "gamma": float(wl.gamma), "kappa": float(wl.kappa)}
    if rho_set is not None:
        arrays["rho_elems"] = np.asarray(rho_set[0], dtype=np.int32)
        arrays["rho"] = np.asarray(rho_set[1], dtype=np.float64)
    if mlp is not None:
        arrays["mlp_params"] = mlp.get_params()
        for name, v in zip(("mlp_x_mean", "mlp_x_std", "mlp_t_mean", "mlp_t_std"), mlp.get_scaling()):
            arrays[name] = v
        m["mlp"] = {"n_in": mlp.n_in, "width": mlp.width, "depth": mlp.depth, "n_out": mlp.n_out}
    if train_mu is not None:
        arrays["train_mu"] = np.asarray(train_mu, dtype=np.float64)
        arrays["train_y"] = np.asarray(train_y, dtype=np.float64)
    m.update(meta or {})
    save(path, arrays, m)


def restore_mlp(arrays: dict, meta: dict, stream=None):
    """The warm-start network of a model checkpoint, on the current device."""
    from . import ift

    a = meta["mlp"]
    net = ift.MLP(a["n_in"], a["width"], a["depth"], a["n_out"], stream=stream)
    net.set_params(arrays["mlp_params"])
    net.set_scaling(arrays["mlp_x_mean"], arrays["mlp_x_std"], arrays["mlp_t_mean"], arrays["mlp_t_std"])
    return net
