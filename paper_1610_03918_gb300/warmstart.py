"""Learned warm start of the Poisson solve: data, training and inference
around the library's U-Net (all arithmetic in the CUDA kernels; this module
only moves tensors between the C ABI calls).

The network maps (rho / s, Dirichlet mask) to (phi - phi_L) / s, with
s = max |rho| and phi_L the potential of the empty box; the solve starts
from phi_L + s * U(...) and still runs to its tolerance.
"""
from __future__ import annotations

import numpy as np

from . import Unet


def padded_rows(nxn: int) -> int:
    return (nxn + 7) // 8 * 8


def dump_pairs(sim, steps: int, every: int):
    """Advance `sim` by `steps` steps; every `every` steps record a training
    pair (x [hpad, nyn, 2], target [hpad, nyn]) as torch CUDA tensors, both
    formed by the library's kernels."""
    hpad = padded_rows(sim.nxn)
    pairs = []
    for k in range(steps // every):
        sim.step(every)
        x, s = sim.learned_input(hpad)
        pairs.append((x[0], sim.learned_target(hpad, s)))
    return pairs


def train(net: Unet, pairs, epochs: int, lr: float, batch: int = 1, seed: int = 0, lr_end=None):
    """Adam on the MSE loss over the pairs (shuffled each epoch); the learning
    rate decays linearly to lr_end (default lr / 10)."""
    import torch
    rng = np.random.default_rng(seed)
    lr_end = lr / 10 if lr_end is None else lr_end
    n = len(pairs)
    total = max(1, epochs * (n // batch))
    k = 0
    for _ in range(epochs):
        order = rng.permutation(n)
        for b0 in range(0, n - batch + 1, batch):
            idx = order[b0:b0 + batch]
            x = torch.stack([pairs[i][0] for i in idx])
            t = torch.stack([pairs[i][1] for i in idx])
            net.train_step(x, t, lr + (lr_end - lr) * k / total)
            k += 1
    torch.cuda.synchronize()


class LearnedWarmStart:
    """Inference side: net is a batch-1 Unet of the context's padded grid."""

    def __init__(self, net: Unet):
        self.net = net

    def solve(self, sim):
        """Build the guess for the current rho and solve from it.  Returns
        (stats of pic_poisson, total device ms including the input and the
        network)."""
        import torch
        hpad = self.net.shape[1]
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record()
        x, s = sim.learned_input(hpad)
        y = self.net.forward(x)
        stats = sim.poisson(3, y, s)
        stop.record()
        torch.cuda.synchronize()
        return stats, start.elapsed_time(stop)
