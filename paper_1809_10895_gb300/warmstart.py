"""Training driver of the learned warm start.

The plain solver generates the training data: before each accepted step the
state h^n is saved, and after it the library writes the step's features
(``rf_ws_features`` of h^n, its time and the step's dt) and its target
(``rf_ws_target``: (h^{n+1} - h^n) / (out_scale dt)).  The network is then
trained on random mini-batches of those snapshots by the library's own
forward / backward / Adam kernels (``rf_nn_train_step``).  Python here only
allocates tensors, picks snapshot indices and calls the library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rf


def _lnKs(case) -> np.ndarray:
    """ln Ks of the active cells of a workload case."""
    if case.Ks_cell is not None:
        Ks = np.asarray(case.Ks_cell, dtype=np.float64)
    else:
        zone = np.zeros(case.N, dtype=np.int64) if case.zone_of_cell is None else np.asarray(case.zone_of_cell)
        Ks = np.array([case.soils[z]["Ks"] for z in range(len(case.soils))])[zone]
    act = np.ones(case.N, bool) if case.active is None else np.asarray(case.active, bool)
    return np.log(Ks[act])


def scales_for(case, out_scale: float = 1.0, h_scale: float = 1.0, q_scale: float = 1e-6) -> rf.rf_ws_scales:
    """Feature scales from a case: ln Ks standardised over the active cells,
    the top flux in units of q_scale, dt in units of the case's dt_max."""
    l = _lnKs(case)
    std = float(np.std(l))
    return rf.rf_ws_scales(h_scale=h_scale, lnK_mean=float(np.mean(l)), lnK_std=std if std > 0 else 1.0,
                           q_scale=q_scale, t_scale=float(case.params.get("dt_max", 600.0)), out_scale=out_scale)


@dataclass
class Snapshots:
    """Features, targets and masks of accepted steps, stacked on the device."""
    x: object                      # (S, nz, ny, nx, 4) float32
    target: object                 # (S, nz, ny, nx) float32
    mask: object                   # (S, nz, ny, nx) float32
    dt: list = field(default_factory=list)
    picard: list = field(default_factory=list)

    def __len__(self):
        return len(self.dt)


def collect(solver: rf.Solver, case, scales: rf.rf_ws_scales, n_steps: int, t_end: float = None,
            stride: int = 1) -> Snapshots:
    """Step the solver (plain method, no network attached) and keep every
    stride-th accepted step as a snapshot, up to n_steps snapshots."""
    import torch
    nz, ny, nx = case.nz, case.ny, case.nx
    dev = solver.device
    S = Snapshots(torch.empty((n_steps, nz, ny, nx, 4), dtype=torch.float32, device=dev),
                  torch.empty((n_steps, nz, ny, nx), dtype=torch.float32, device=dev),
                  torch.empty((n_steps, nz, ny, nx), dtype=torch.float32, device=dev))
    h_old = torch.empty(case.N, dtype=torch.float64, device=dev)
    t_stop = case.t_end if t_end is None else t_end
    k, taken = 0, 0
    t = case.t0
    while taken < n_steps and t < t_stop * (1 - 1e-12):
        solver.get_state_device(h_old)
        info = solver.step()
        t_old, t = info.t - info.dt, info.t
        if k % stride == 0:
            solver.ws_features(scales, t_old, info.dt, S.x[taken], h=h_old)
            solver.ws_target(scales, h_old, info.dt, S.target[taken], S.mask[taken])
            S.dt.append(info.dt)
            S.picard.append(info.picard)
            taken += 1
        k += 1
    if taken < n_steps:
        S.x, S.target, S.mask = S.x[:taken], S.target[:taken], S.mask[:taken]
    return S


def target_rms(S: Snapshots) -> float:
    """Root mean square of the targets over the masked voxels (host)."""
    t = S.target.double().cpu().numpy()
    m = S.mask.double().cpu().numpy()
    n = max(m.sum(), 1.0)
    return float(np.sqrt(np.sum((t * m) ** 2) / n))


def train(net: rf.Network, S: Snapshots, steps: int, batch: int = 4, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0, lr_final: float = None):
    """Adam on random mini-batches of snapshots; the learning rate decays
    along a cosine from lr to lr_final (default lr / 10).  Returns the
    losses logged every log_every steps (and the last one)."""
    import torch
    rng = np.random.default_rng(seed)
    lr_final = lr / 10 if lr_final is None else lr_final
    losses = []
    n = len(S)
    for k in range(steps):
        idx = torch.as_tensor(rng.integers(0, n, size=min(batch, n)), device=S.x.device)
        xb, tb, mb = S.x[idx].contiguous(), S.target[idx].contiguous(), S.mask[idx].contiguous()
        lr_k = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * k / max(steps - 1, 1)))
        want = (log_every and k % log_every == 0) or k == steps - 1
        L = net.train_step(xb, tb, mb, lr=float(lr_k), want_loss=bool(want))
        if want:
            losses.append((k, L))
    return losses
