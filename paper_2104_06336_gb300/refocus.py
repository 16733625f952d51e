"""Interactive refocusing (Sec. IV, Fig. 2: only Eq. 3 is redone when the
aberrations change) driven by the hand-written adjoint.

* ``sweep``: image variance for many aberration candidates in one batched
  launch of the fused trotter kernel (no phase images).
* ``fit``: gradient ascent on the variance with Adam over a chosen subset of
  (C1, C12a, C12b, C3, rot); each step is one pass over the resident G that
  returns V and dV/dtheta (``ssb_variance_grad``).  The five-number optimizer
  update is host-side glue; the objective and gradient run in the kernels.
* ``RefocusGraph``: the device-resident refocus step (``ssb_refocus_step``:
  V, gradient, phase image and a fixed-step ascent update of the aberrations in
  device memory; or ``ssb_refocus_step_adam`` with an Adam update whose
  moments also live in device memory) captured once as a CUDA graph and
  replayed.
"""

from __future__ import annotations

import torch

from . import _lib as L
from .pipeline import Reconstructor

SCALES = (100.0, 50.0, 50.0, 1.0e4, 0.1)  # typical magnitudes (A, A, A, A, rad)


def sweep(rec: Reconstructor, candidates: torch.Tensor) -> torch.Tensor:
    """V for each candidate row of ``candidates`` [n][5] (rotation shared)."""
    cand = candidates.to(rec.device, torch.float64).reshape(-1, 5).contiguous()
    n = cand.shape[0]
    if n > rec.n_cand:
        raise ValueError(f"{n} candidates; the Reconstructor was sized for {rec.n_cand}")
    var = torch.empty(n, dtype=torch.float64, device=rec.device)
    L.ssb_reconstruct(rec.plan, rec.G, cand, rec.scratch, None, var, status=rec.status)
    return var


def fit(rec: Reconstructor, theta0, steps: int = 30, lr: float = 0.05,
        mask=(1, 1, 1, 0, 0), scales=SCALES):
    """Adam ascent on V from ``theta0``; ``lr`` is in units of ``scales``.
    Returns (theta, list of V)."""
    dev = rec.device
    sc = torch.tensor(scales, dtype=torch.float64, device=dev)
    m = torch.tensor(mask, dtype=torch.float64, device=dev)
    x = (torch.as_tensor(theta0, dtype=torch.float64, device=dev) / sc).clone()
    m1 = torch.zeros(5, dtype=torch.float64, device=dev)
    m2 = torch.zeros(5, dtype=torch.float64, device=dev)
    b1, b2, eps = 0.9, 0.999, 1e-12
    hist = []
    for t in range(1, steps + 1):
        V, g, _ = rec.variance_grad(x * sc)
        hist.append(float(V.item()))
        gs = g * sc * m  # gradient with respect to the scaled parameters
        m1 = b1 * m1 + (1 - b1) * gs
        m2 = b2 * m2 + (1 - b2) * gs * gs
        mh = m1 / (1 - b1 ** t)
        vh = m2 / (1 - b2 ** t)
        x = x + lr * m * mh / (vh.sqrt() + eps)
    V, _, _ = rec.variance_grad(x * sc)
    hist.append(float(V.item()))
    return x * sc, hist


class RefocusGraph:
    """A captured CUDA graph of one ``ssb_refocus_step``: the aberrations,
    step sizes and outputs live in device memory, so every replay continues
    from the previous one's update.  With ``adam`` (a learning rate per
    parameter in units of ``scales``; 0 holds a parameter) each replay is an
    Adam step instead of a fixed one; ``reset`` restarts it."""

    def __init__(self, rec: Reconstructor, theta0, step=None, warmup: int = 2, adam=None,
                 scales=SCALES):
        dev = rec.device
        self.rec = rec
        self.theta = torch.as_tensor(theta0, dtype=torch.float64).to(dev).contiguous().clone()
        self.adam = adam is not None
        if self.adam:
            self.step = torch.tensor(list(adam) + list(scales), dtype=torch.float64, device=dev)
        else:
            self.step = torch.as_tensor(step, dtype=torch.float64).to(dev).contiguous().clone()
        self.state = torch.zeros(11, dtype=torch.float64, device=dev)
        self.theta0 = self.theta.clone()
        self.var = torch.empty(1, dtype=torch.float64, device=dev)
        self.grad = torch.empty(5, dtype=torch.float64, device=dev)
        self.phase = torch.empty(rec.Ny, rec.Nx, dtype=torch.float32, device=dev)
        th_save = self.theta.clone()
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # first calls set up kernel attributes outside capture
            for _ in range(warmup):
                self._call()
        torch.cuda.current_stream().wait_stream(s)
        self.theta.copy_(th_save)
        self.state.zero_()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._call()

    def _call(self):
        if self.adam:
            L.ssb_refocus_step_adam(self.rec.plan, self.rec.G, self.theta, self.step, self.state,
                                    self.rec.scratch, self.var, self.grad, self.phase,
                                    status=self.rec.status)
        else:
            L.ssb_refocus_step(self.rec.plan, self.rec.G, self.theta, self.step, self.rec.scratch,
                               self.var, self.grad, self.phase, status=self.rec.status)

    def reset(self, theta0=None):
        """Back to ``theta0`` (default: the start) with fresh Adam moments."""
        self.theta.copy_(self.theta0 if theta0 is None else
                         torch.as_tensor(theta0, dtype=torch.float64).to(self.theta.device))
        self.state.zero_()

    def replay(self, n: int = 1):
        for _ in range(n):
            self.graph.replay()
