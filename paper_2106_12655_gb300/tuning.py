"""On-disk cache of the autotuner's table, keyed by GPU name.

lk_autotune measures the best work-item height per size class on the GPU at
hand; this module keeps those tables in a JSON file so that a later process
on the same kind of GPU can install them with lk_tune_set instead of tuning
again.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import lk


def _load(path):
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def save(ctx, device_name: str, path: str):
    """Store ctx's table for device_name in the JSON file at path."""
    data = _load(path)
    data[device_name] = lk.lk_tune_get(ctx).tolist()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def restore(ctx, device_name: str, path: str) -> bool:
    """Install the table stored for device_name, if any; returns whether one was found."""
    entries = _load(path).get(device_name)
    if not entries:
        return False
    lk.lk_tune_set(ctx, np.asarray(entries, np.int32))
    return True
