"""JSON cache of launch shapes chosen by lbm_autotune, keyed by the problem
signature (lattice, collision, storage, sizes, obstacle mask) and the device
name, so a shape measured once is reused by later runs of the same problem."""
from __future__ import annotations

import json
import os
import tempfile


def device_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name()
    except Exception:
        pass
    return "unknown"


def signature(lat) -> str:
    lattice, coll, st, nx, ny, nz, mask = lat.signature_fields
    return f"{device_name()}|L{lattice}|C{coll}|S{st}|{nx}x{ny}x{nz}|mask{int(mask)}"


def lookup(path: str, key: str):
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def store(path: str, key: str, launch, ms: float) -> None:
    data = {}
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        pass
    data[key] = {"launch": list(launch), "ms": ms}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d)
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
