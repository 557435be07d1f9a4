"""Moves a synthetic workload to the GPU and builds its fsqr_design.

Plumbing only (torch holds the device buffers); no solver arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import fsqr


@dataclass
class DeviceWorkload:
    design: fsqr.Design
    geno: torch.Tensor
    cov: torch.Tensor | None
    y: torch.Tensor
    omega: torch.Tensor
    n: int
    P: int
    block_ptr: np.ndarray


def upload(ctx: fsqr.Context, w, device="cuda", standardize=1, omega=None) -> DeviceWorkload:
    geno = torch.from_numpy(np.ascontiguousarray(w.geno).view(np.uint8)).to(device) if w.p else None
    if w.fmt == fsqr.DENSE_F64 and geno is not None:
        geno = torch.from_numpy(np.ascontiguousarray(w.geno, dtype=np.float64)).to(device)
    cov = torch.from_numpy(np.ascontiguousarray(w.cov, dtype=np.float64)).to(device) if w.c else None
    y = torch.from_numpy(np.ascontiguousarray(w.y, dtype=np.float64)).to(device)
    om = torch.from_numpy(np.ascontiguousarray(w.omega if omega is None else omega, dtype=np.float64)).to(device)
    d = ctx.design(w.n, w.p, w.c, w.fmt, geno, w.ld, cov=cov, standardize=standardize)
    return DeviceWorkload(d, geno, cov, y, om, w.n, w.P, w.block_ptr())


def zeros_state(n_fits: int, P: int, n: int, device="cuda"):
    t = lambda k: torch.zeros(k, dtype=torch.float64, device=device)
    return t(n_fits * P), t(n_fits * n), t(n_fits * n)
