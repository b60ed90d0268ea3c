"""Cache of autotuned launch shapes (chunks of samples per lane, per grid).

cmg_autotune times each candidate on the GPU; this module keeps the choices
in a JSON file keyed by GPU name, grid size, sample count and precision so
later runs can apply them with cmg_set_tuning instead of re-timing.
"""
from __future__ import annotations

import json
import os


def _key(gpu: str, n: int, N: int, precision: int) -> str:
    return f"{gpu}|n={n}|N={N}|prec={precision}"


def load(path: str) -> dict:
    if path and os.path.exists(path):
        try:
            with open(path) as fh:
                return json.load(fh)
        except (OSError, ValueError):
            return {}
    return {}


def apply_or_tune(H, precision: int, path: str | None = None) -> list:
    """Apply cached targets for this hierarchy, or autotune and store them."""
    import torch

    gpu = torch.cuda.get_device_name(H.device)
    key = _key(gpu, H.n, H.N, precision)
    cache = load(path) if path else {}
    if key in cache and len(cache[key]) == H.levels:
        H.set_tuning(precision, cache[key])
        return list(cache[key])
    chosen = H.autotune(precision)
    if path:
        cache[key] = chosen
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return chosen
