"""Training data and training loop of the spectral neural operator (coarse propagator of Parareal).

Trajectories come from the plain GPU solver (the batched ETDRK2 executor): for trajectory i the
seeded u0 and D of the workload, `traj_steps` steps of size tau, and input/target pairs
(u(k w tau), u((k+1) w tau)) for k = 0 .. traj_steps / w - 1 (w = the window). Training steps,
gradients and Adam updates run in the library's kernels (Sno.train_step); this module only
orders the pairs (seeded shuffles) and gathers batches.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs
from .etd import Batch, _torch
from .sno import Sno


def make_pairs(w: inputs.SnoWorkload, indices, chunk: int = 500):
    """Input/target pairs of the trajectories `indices`: (u_in, u_out, D) with u_in, u_out CUDA
    float32 tensors of shape (P, N-1, N-1) and D a list of P floats."""
    torch = _torch()
    n = w.N - 1
    nwin = w.traj_steps // w.window
    ins, outs, Ds = [], [], []
    indices = list(indices)
    for c0 in range(0, len(indices), chunk):
        idx = indices[c0:c0 + chunk]
        D = [w.D(i) for i in idx]
        U = torch.from_numpy(np.stack([w.u0(i) for i in idx]).astype(np.float32)).cuda()
        with Batch([(w.N, w.N)] * len(idx), D, w.tau, scheme=2, dtype="f32") as b:
            snaps = [U.clone()]
            for _ in range(nwin):
                b.run([U[i] for i in range(len(idx))], w.window)
                snaps.append(U.clone())
        for k in range(nwin):
            ins.append(snaps[k])
            outs.append(snaps[k + 1])
            Ds.extend(D)
    u_in = torch.cat(ins).contiguous()
    u_out = torch.cat(outs).contiguous()
    assert u_in.shape[1:] == (n, n)
    return u_in, u_out, Ds


def train(sno: Sno, u_in, u_out, D, epochs: int, batch: int, lr: float = 1e-3, seed: int = 0,
          lr_final: float = 1e-4) -> list:
    """Adam over seeded shuffles of the pairs; learning rate decays geometrically from lr to
    lr_final over the run. Returns the mean loss of every epoch."""
    torch = _torch()
    P = u_in.shape[0]
    steps = epochs * (P // batch)
    decay = (lr_final / lr) ** (1.0 / max(1, steps - 1))
    rng = np.random.default_rng(seed)
    hist, it = [], 0
    Dn = np.asarray(D, dtype=np.float64)
    for _ in range(epochs):
        perm = rng.permutation(P)
        tot = 0.0
        for s in range(P // batch):
            sel = perm[s * batch:(s + 1) * batch]
            ix = torch.from_numpy(sel).cuda()
            x = u_in.index_select(0, ix).contiguous()
            y = u_out.index_select(0, ix).contiguous()
            tot += sno.train_step(x, Dn[sel].tolist(), y, lr * decay ** it)
            it += 1
        hist.append(tot / max(1, P // batch))
    return hist


def rel_error(sno: Sno, u_in, u_out, D, batch: int) -> float:
    """||sno(u_in) - u_out|| / ||u_out|| over all pairs together (fields that decay to near zero do
    not dominate, as they would in a mean of per-pair ratios)."""
    torch = _torch()
    num = den = 0.0
    for s in range(0, u_in.shape[0], batch):
        x = u_in[s:s + batch].contiguous()
        y = u_out[s:s + batch]
        p = sno.forward(x, D[s:s + batch])
        num += float(torch.sum((p - y) ** 2).item())
        den += float(torch.sum(y * y).item())
    return math.sqrt(num / den) if den > 0 else math.nan
