"""Autotuner cache: the fastest CTA shape of each pass per (grid, precision, device),
measured on the device by dirac_autotune and kept in a JSON file."""
from __future__ import annotations

import json
import os

from . import dirac_autotune, dirac_set_launch

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "dirac_gb300_autotune.json")


def _device_name():
    try:
        import torch

        return torch.cuda.get_device_name()
    except Exception:
        return "cuda"


def tune(sim, precision, cache_path: str = DEFAULT_CACHE, reps: int = 20, refresh: bool = False):
    """Apply the cached (or newly measured) launch shapes to a Simulation's context."""
    key = f"{_device_name()}|{sim.nx}x{sim.ny}|{'c64' if precision == 0 else 'c128'}"
    cache = {}
    if os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache and not refresh:
        tx, ty = cache[key]
        dirac_set_launch(sim.ctx, tx, ty)
        return tx, ty
    tx, ty = dirac_autotune(sim.ctx, reps)
    cache[key] = [tx, ty]
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return tx, ty
