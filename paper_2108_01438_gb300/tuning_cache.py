"""Persistent cache of autotuned launch choices.

`Plan.autotune` (mbir_plan_autotune) times the candidate lateral tile widths,
lateral radix orders and row-adjoint kernels of a plan and keeps the fastest; the
library remembers the choice for the plan's shape class within one process.
This module keeps those choices across processes in a JSON file, keyed by the
shape class and the GPU, so that a service tunes each class once per device
type instead of once per start.

Key: "<gpu name>|<nx>x<nz>x<m>|J<kb width>|p<precision>".  A missing, unreadable
or malformed file starts an empty cache; writes go through a temporary file and
an atomic rename, so a reader never sees half a file.
"""
from __future__ import annotations

import json
import os
import tempfile

__all__ = ["class_key", "TuningCache"]

_FIELDS = ("tile_c", "lateral_order", "adjoint_kernel")


def class_key(plan, gpu_name: str) -> str:
    """The shape class of a plan on a GPU: sizes, KB width and precision."""
    g = plan.geometry
    return f"{gpu_name}|{int(g['nx'])}x{int(g['nz'])}x{int(g['m'])}|J{int(g.get('kb_width', 6))}|p{int(plan.precision)}"


class TuningCache:
    def __init__(self, path: str):
        self.path = path
        self.entries: dict[str, dict] = {}
        try:
            with open(path) as fh:
                data = json.load(fh)
            if isinstance(data, dict):
                self.entries = {k: v for k, v in data.items()
                                if isinstance(v, dict) and all(isinstance(v.get(f), int) for f in _FIELDS)}
        except (OSError, ValueError):
            self.entries = {}

    def get(self, key: str) -> dict | None:
        e = self.entries.get(key)
        return None if e is None else {f: e[f] for f in _FIELDS}

    def put(self, key: str, tuning: dict) -> None:
        self.entries[key] = {f: int(tuning[f]) for f in _FIELDS}
        if "pair_ms" in tuning:
            self.entries[key]["pair_ms"] = float(tuning["pair_ms"])

    def save(self) -> None:
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tuning-", suffix=".json")
        with os.fdopen(fd, "w") as fh:
            json.dump(self.entries, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def apply_or_tune(self, plan, gpu_name: str | None = None, reps: int = 5, save: bool = True) -> dict:
        """Apply the cached choice for the plan's class, or autotune the plan, record
        the result (and write the file when save).  Returns the choice and whether it
        came from the cache."""
        if gpu_name is None:
            import torch
            gpu_name = torch.cuda.get_device_name()
        key = class_key(plan, gpu_name)
        hit = self.get(key)
        if hit is not None:
            plan.set_tuning(hit["tile_c"], hit["lateral_order"], hit["adjoint_kernel"])
            return dict(hit, cached=True)
        t = plan.autotune(reps=reps)
        self.put(key, t)
        if save:
            self.save()
        return dict({f: t[f] for f in _FIELDS}, cached=False)
