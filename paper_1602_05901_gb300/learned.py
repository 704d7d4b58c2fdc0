"""Training data and training loop of the learned pressure stage (orchestration of library calls).

The network imitates the CPR pressure stage: its samples are the restricted
residuals r_p that a plain FP64 FGMRES + CPR solve feeds to its pressure
solver (recorded on the device by ``rsv_solver_record_pressure``), and its
targets are one multigrid V-cycle applied to each (``rsv_cpr_vcycle``).
Every arithmetic step runs in librsv's kernels; this module only sequences
the calls and keeps the sample tensors.
"""
from __future__ import annotations

import numpy as np

from . import Matrix, Solver, Unet  # noqa: F401


def collect_samples(grid, vals, b, max_samples, restart=30):
    """Record up to ``max_samples`` pressure-stage inputs of a plain CPR solve of A x = b and their V-cycle targets.

    Returns (rp, target): CUDA float64 tensors [k][nb], k <= max_samples (the
    solve stops after max_samples iterations).
    """
    import torch
    A = Matrix(*grid)
    A.set_values(vals)
    nb = A.nb
    s = Solver(A, solver="fgmres", precision="fp64", rtol=1e-8, restart=restart, maxit=max_samples)
    s.setup("cpr")
    buf = torch.empty((max_samples, nb), dtype=torch.float64, device="cuda")
    s.record_pressure(buf, max_samples)
    x = np.zeros(3 * nb)
    s.solve(np.ascontiguousarray(b, dtype=np.float64), x, raise_on_error=False)
    k = s.recorded()
    s.record_pressure(None, 0)
    rp = buf[:k].clone()
    tgt = torch.empty_like(rp)
    for i in range(k):
        s.vcycle(rp[i], tgt[i])
    torch.cuda.synchronize()
    return rp, tgt


def train(net: Unet, samples, epochs, lr=3e-4, seed=0, chunk=64):
    """Adam over the samples [(rp, lnk, target) CUDA tensors], shuffled each epoch (seeded).

    Returns the mean loss of each epoch.
    """
    order_rng = np.random.default_rng(seed)
    means = []
    for _ in range(epochs):
        order = order_rng.permutation(len(samples))
        losses = []
        for c0 in range(0, len(order), chunk):
            idx = order[c0:c0 + chunk]
            losses.append(net.train_batch([samples[i][0] for i in idx], [samples[i][1] for i in idx],
                                          [samples[i][2] for i in idx], lr))
        means.append(float(np.mean(np.concatenate(losses))))
    return means


def imitation_error(net: Unet, rp, lnk, target):
    """Relative error ||N(r_p) - V(r_p)|| / ||V(r_p)|| of the network against the V-cycle, per sample."""
    import torch
    out = torch.empty_like(rp[0])
    errs = []
    for i in range(rp.shape[0]):
        net.apply(rp[i], lnk, out)
        errs.append(float(torch.linalg.norm(out - target[i]) / torch.linalg.norm(target[i])))
    return np.array(errs)
