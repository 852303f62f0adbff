"""Unrolled learned normalised min-sum and its training loss in plain PyTorch
on the CPU; autograd of this forward is the oracle's reference gradient.

TEST INFRASTRUCTURE ONLY: imported by tests/ and by the benchmark's CPU leg.
The CUDA library never uses it.

The forward is the layered single-scan min-sum of Section 4 (eq. 22: the
extrinsic input Q = Z_n - L_mn; eq. 23: the new check message from the
smallest and second smallest |Q| of the row and the product of the signs;
eq. 20 in single-scan form: Z_n = Q + L_mn), with the paper's plain eq. 23
magnitude multiplied by a learned factor w[t, b] chosen per iteration t and
per nonzero block b of the base matrix (blocks numbered row by row, columns
increasing).  Layers run in natural order; the Z rows of a layer touch
disjoint variables, so they are updated together.  There is no early stop:
every frame runs T iterations.

Training loss: the sum over iterations t = 1..T, frames f and bits n of the
binary cross-entropy of sigmoid(-Z_n^(t)) (the posterior probability that
bit n is 1) against the transmitted bit c_n, times `loss_scale`:
    BCE = softplus(-Z) + c Z,  softplus(x) = max(x, 0) + log1p(exp(-|x|)).

The derivative of |Q| is sign(Q); the signs themselves have derivative 0;
the minimum passes its gradient to the first edge attaining it and the
second minimum to the first attaining edge among the others.  At exact ties
these are one choice of subgradient.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np
import torch


def layer_tables(hbm: np.ndarray, z: int) -> List[Tuple[torch.Tensor, torch.Tensor]]:
    """Per block row l: (vars [Z, d] int64, blocks [d] int64).

    Row r of block row l with a block of shift s in column j has its edge at
    variable j Z + (r + s) mod Z (the circulant P_s); the blocks of a row are
    taken in increasing column order and numbered consecutively over rows.
    """
    hbm = np.asarray(hbm)
    mb, nb = hbm.shape
    out = []
    b = 0
    r = np.arange(z)
    for l in range(mb):
        cols = [j for j in range(nb) if hbm[l, j] >= 0]
        v = np.stack([j * z + (r + int(hbm[l, j])) % z for j in cols], axis=1)
        out.append((torch.from_numpy(v.astype(np.int64)),
                    torch.arange(b, b + len(cols), dtype=torch.int64)))
        b += len(cols)
    return out


def bce_posterior(Z: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
    """Elementwise BCE(sigmoid(-Z), c) in its overflow-free form."""
    x = -Z
    return torch.clamp(x, min=0) + torch.log1p(torch.exp(-x.abs())) - c * x


def unrolled_forward(hbm, z: int, llr: torch.Tensor, bits: torch.Tensor,
                     weights: torch.Tensor, loss_scale: float = 1.0):
    """Run T = weights.shape[0] iterations on frames llr [F, N].

    Computes in llr's dtype (float64 for the reference gradient; float32
    reproduces the GPU decoder's rounding, each operation rounded once).
    Returns (loss, loss_per_frame [F], posteriors [T, F, N], decisions), where
    decisions is a per-frame int64 signature of every discrete choice (argmin,
    second argmin, sign bits) for spotting a finite-difference step that
    crosses a kink.
    """
    tables = layer_tables(hbm, z)
    T = weights.shape[0]
    F, N = llr.shape
    dt = llr.dtype
    c = bits.to(dt)
    Zp = llr
    msgs = [torch.zeros((F, z, v.shape[1]), dtype=dt) for v, _ in tables]
    per_frame = torch.zeros(F, dtype=dt)
    posts = []
    sig = torch.zeros(F, dtype=torch.int64)
    for t in range(T):
        for l, (v, blocks) in enumerate(tables):
            d = v.shape[1]
            Q = Zp[:, v] - msgs[l]                          # eq. 22
            a = Q.abs()
            idx = a.argmin(dim=2, keepdim=True)             # first smallest
            m1 = a.gather(2, idx)
            rest = a.detach().scatter(2, idx, float("inf"))
            idx2 = rest.argmin(dim=2, keepdim=True)         # first of the others
            m2 = a.gather(2, idx2)
            neg = Q.detach() < 0
            parity = neg.sum(dim=2, keepdim=True) % 2
            sgn = 1.0 - 2.0 * (neg.to(torch.int64) ^ parity).to(dt)   # product of the others' signs
            at_min = torch.arange(d).view(1, 1, d) == idx
            mag = torch.where(at_min, m2, m1)
            L = (weights[t, blocks].view(1, 1, d) * mag) * sgn       # eq. 23, weighted
            msgs[l] = L
            Zp = Zp.index_copy(1, v.reshape(-1), (Q + L).reshape(F, -1))   # eq. 20
            code = (idx.squeeze(2) * 32 + idx2.squeeze(2)) * 2 + parity.squeeze(2)
            sig = (sig * 1000003 + code.sum(dim=1) * 7919
                   + (neg.to(torch.int64) * torch.arange(1, d + 1)).sum(dim=(1, 2))) % (1 << 61)
        posts.append(Zp)
        per_frame = per_frame + bce_posterior(Zp, c).sum(dim=1)
    loss = loss_scale * per_frame.sum()
    return loss, per_frame, torch.stack(posts), sig


def reference_gradient(hbm, z: int, llr: np.ndarray, bits: np.ndarray,
                       weights: np.ndarray, loss_scale: float = 1.0,
                       dtype=torch.float64):
    """(loss, loss_per_frame, d loss / d weights [T, E_b], d loss / d llr [F, N])
    by reverse-mode differentiation of `unrolled_forward` in `dtype`."""
    x = torch.tensor(np.asarray(llr), dtype=dtype, requires_grad=True)
    w = torch.tensor(np.asarray(weights), dtype=dtype, requires_grad=True)
    b = torch.tensor(np.asarray(bits))
    loss, per_frame, _, _ = unrolled_forward(hbm, z, x, b, w, loss_scale)
    loss.backward()
    return (loss.item(), per_frame.detach().numpy(), w.grad.numpy(), x.grad.numpy())
