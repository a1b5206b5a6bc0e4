"""Learning an orthogonal transform M that improves compressibility (an extension of the
paper's "learned transforms" of Sec. 2.2): M(A) = (I + W)^{-1} (I - W) M0 with
W = A^T - A, trained with Adam on the t-SVDM-I truncation loss
L = sqrt(sum of discarded sigma^2) / ||X||_F at rank k.

One training step, every part of it a libtsvdm kernel (torch only allocates):
  tsvdm_cayley          M = Cayley(A) M0 (Gauss-Jordan of I + W, two small GEMMs)
  tsvdm_fixed_rank      forward: Ahat = X x_3 M, batched Jacobi SVDs (optionally warm-started
                        from the previous step's right vectors), rank-k factors
  tsvdm_backward        residual R = Ahat - U_k S_k V_k^T, L, dL/dM (and dL/dX if asked)
  tsvdm_cayley_backward dL/dA from dL/dM
  tsvdm_adam            A <- Adam(A, dL/dA)
"""
from __future__ import annotations

import time

import torch

from . import native as N
from .tsvdm import Plan

_DT = {torch.float32: N.F32, torch.float64: N.F64}


class CayleyTrainer:
    """Holds the plan and every buffer of the training loop (allocated once)."""

    def __init__(self, X: torch.Tensor, M0: torch.Tensor, shape, k, lr=1e-3, betas=(0.9, 0.999),
                 eps=1e-8, want_dX=False, warm_start=False):
        """warm_start: every step's slice SVDs start from the previous step's right vectors
        (M moves by one Adam step at a time, so a few Jacobi sweeps suffice)."""
        n1, n2, n3 = shape
        self.shape, self.k, self.lr, self.betas, self.eps = shape, int(k), lr, betas, eps
        self.X = X
        self.M0 = M0
        self.dtype = X.dtype
        dev = X.device
        self.plan = Plan(n1, n2, n3, dtype=self.dtype, orthogonal=True)
        if warm_start:
            self.plan.set_warm_start(True)
        self.A = torch.zeros(n3, n3, dtype=self.dtype, device=dev)
        self.m1 = torch.zeros_like(self.A)
        self.m2 = torch.zeros_like(self.A)
        self.M = torch.empty_like(self.A)
        self.Z = torch.empty_like(self.A)
        self.Q = torch.empty_like(self.A)
        self.work = torch.empty(3 * n3 * n3, dtype=self.dtype, device=dev)
        self.U = torch.empty(n3, k, n1, dtype=self.dtype, device=dev)
        self.S = torch.empty(n3, k, dtype=self.dtype, device=dev)
        self.V = torch.empty(n3, k, n2, dtype=self.dtype, device=dev)
        self.dM = torch.empty_like(self.A)
        self.dA = torch.empty_like(self.A)
        self.dX = torch.empty_like(X) if want_dX else None
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.t = 0

    def step(self, events=None):
        """One training step.  events (optional list) receives a CUDA event before each part
        and one after the last, on the current stream (for a per-part time split)."""
        n3 = self.shape[2]
        dt = _DT[self.dtype]

        def mark():
            if events is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                events.append(e)

        mark()
        N.tsvdm_cayley(n3, dt, self.A, self.M0, self.M, self.Z, self.Q, self.work)
        mark()
        N.tsvdm_fixed_rank(self.plan.handle, self.X, self.M, self.k, self.U, self.S, self.V, 0,
                           want_rel_err=False)
        mark()
        N.tsvdm_backward(self.plan.handle, self.X, self.M, self.k, self.U, self.S, self.V, 1.0,
                         self.dX, self.dM, self.loss)
        mark()
        N.tsvdm_cayley_backward(n3, dt, self.M0, self.Z, self.Q, self.dM, self.dA, self.work)
        self.t += 1
        mark()
        N.tsvdm_adam(n3 * n3, dt, self.A, self.dA, self.m1, self.m2, self.t, self.lr,
                     self.betas[0], self.betas[1], self.eps)
        mark()
        return self.loss

    PARTS = ("cayley", "forward_fixed_rank", "backward", "cayley_backward", "adam")

    def part_split(self, steps=5):
        """Mean milliseconds of each part of a step over `steps` further steps."""
        acc = [0.0] * len(self.PARTS)
        for _ in range(steps):
            ev = []
            self.step(ev)
            torch.cuda.synchronize()
            for i in range(len(self.PARTS)):
                acc[i] += ev[i].elapsed_time(ev[i + 1]) / steps
        return dict(zip(self.PARTS, acc))

    def current_transform(self, out=None):
        """M = Cayley(A) M0 for the current parameters."""
        n3 = self.shape[2]
        out = out if out is not None else torch.empty_like(self.A)
        N.tsvdm_cayley(n3, _DT[self.dtype], self.A, self.M0, out, self.Z, self.Q, self.work)
        return out

    def train(self, steps, record=True):
        """Runs `steps` steps; returns (losses, ms_per_step) timed with CUDA events."""
        losses = []
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            self.step()
            if record:
                losses.append(self.loss.clone())
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(steps, 1)
        return [float(x.item()) for x in losses], ms
