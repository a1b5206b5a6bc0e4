"""PyTorch-facing wrappers over the C ABI: output allocation, streams and autograd.

Everything numerical happens inside libtsvdm's kernels; this module only allocates result
tensors with torch, passes pointers, and wires the hand-written adjoint into autograd.
Tensors follow the library layout: an (n1, n2, n3) tensor is stored column-major, i.e.
as a torch tensor whose memory is X[a + n1*b + n1*n2*t].  ``to_lib`` / ``from_lib``
convert between a row-major torch tensor of shape (n1, n2, n3) and that layout.
"""
from __future__ import annotations

import torch

from . import native as N

_DT = {torch.float32: N.F32, torch.float64: N.F64}


def to_lib(x: torch.Tensor) -> torch.Tensor:
    """(n1, n2, n3) tensor -> column-major storage (a contiguous tensor of shape
    (n3, n2, n1) whose flat memory is X[a + n1 b + n1 n2 t])."""
    return x.permute(*reversed(range(x.dim()))).contiguous()


def from_lib(x: torch.Tensor) -> torch.Tensor:
    """Inverse of to_lib: a (n3, n2, n1) contiguous buffer -> (n1, n2, n3) view."""
    return x.permute(*reversed(range(x.dim())))


class Plan:
    """A plan for n1 x n2 x n3 tensors (owns the device workspace)."""

    def __init__(self, n1, n2, n3, dtype=torch.float32, prec=None, orthogonal=True,
                 stream=None, device="cuda"):
        self.n1, self.n2, self.n3 = int(n1), int(n2), int(n3)
        self.dtype = dtype
        self.device = torch.device(device)
        if prec is None:
            prec = "fp64" if dtype == torch.float64 else "fp32"
        self.prec = prec
        self.orthogonal = bool(orthogonal)
        self.r = min(self.n1, self.n2)
        self.handle = N.tsvdm_plan_create(self.n1, self.n2, self.n3, _DT[dtype],
                                          N.PRECISIONS[prec], self.orthogonal, stream)

    @classmethod
    def dway(cls, dims, dtype=torch.float32, prec=None, orthogonal=True, stream=None,
             device="cuda"):
        """A plan for a d-way tensor of `dims` (n1, n2, n3, ..., nd): one transform matrix per
        mode >= 3, passed to every method as one buffer holding M_3, M_4, ... one after the
        other (see `concat`); the slices are the n3 ... nd trailing index combinations."""
        self = cls.__new__(cls)
        dims = [int(d) for d in dims]
        self.n1, self.n2 = dims[0], dims[1]
        self.n3 = 1
        for d in dims[2:]:
            self.n3 *= d
        self.dims = tuple(dims)
        self.dtype = dtype
        self.device = torch.device(device)
        if prec is None:
            prec = "fp64" if dtype == torch.float64 else "fp32"
        self.prec = prec
        self.orthogonal = bool(orthogonal)
        self.r = min(self.n1, self.n2)
        self.handle = N.tsvdm_plan_create_dway(dims, _DT[dtype], N.PRECISIONS[prec],
                                               self.orthogonal, stream)
        return self

    @staticmethod
    def concat(mats):
        """The per-mode matrices (library layout, i.e. torch tensors of to_lib) as one buffer."""
        return torch.cat([m.reshape(-1) for m in mats])

    def close(self):
        if getattr(self, "handle", None) is not None:
            N.tsvdm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, *shape, dtype=None):
        return torch.empty(*shape, dtype=dtype or self.dtype, device=self.device)

    def set_jacobi(self, tol=0.0, max_sweeps=0):
        N.tsvdm_plan_set_jacobi(self.handle, tol, max_sweeps)

    def data_transform(self, X, out=None):
        """The data-driven M (transposed left singular vectors of the mode-3 unfolding),
        an n3 x n3 buffer in library layout."""
        out = out if out is not None else self._empty(self.n3, self.n3)
        N.tsvdm_data_transform(self.handle, X, out)
        return out

    def set_warm_start(self, enable=True):
        """Start each decomposition's slice SVDs from the previous call's right vectors."""
        N.tsvdm_plan_set_warm_start(self.handle, enable)

    def set_engine(self, engine):
        """Engine of the Jacobi Gram / rotation products: "auto", "fma" or "tc"."""
        N.tsvdm_plan_set_engine(self.handle, engine)

    def set_angle_precision(self, angles):
        """Arithmetic of the slice SVDs' rotation test and angle: "fp64" (default) or "fp32"."""
        N.tsvdm_plan_set_angle_precision(self.handle, angles)

    def set_vectors(self, mode):
        """How singular vectors are formed: "accumulate" (one pass, default) or
        "second_pass" (singular values first, then the kept triplets' other side)."""
        N.tsvdm_plan_set_vectors(self.handle, mode)

    def set_transform(self, kind):
        """"dense" (the given M, default) or "dct2" (the orthonormal DCT-II by a fast kernel;
        M arguments are then not read)."""
        N.tsvdm_plan_set_transform(self.handle, kind)

    def set_wait_limit(self, polls):
        """Bound (polls) of the tensor-core slice-SVD kernel's scheduler waits; 0 = default."""
        N.tsvdm_plan_set_wait_limit(self.handle, polls)

    def transform(self, X, M, inverse=False, out=None):
        out = out if out is not None else torch.empty_like(X)
        N.tsvdm_transform(self.handle, X, M, int(inverse), out)
        return out

    def fixed_rank(self, X, M, k, original_domain=False, rel_err=True, raise_on_error=True):
        """t-SVDM-I.  X: library-layout buffer (n1 n2 n3 elements), M: n3 x n3 library
        layout.  Returns dict(U (k n3 n1 buffer), S, V, rel_err, status)."""
        U = self._empty(self.n3, k, self.n1)
        S = self._empty(self.n3, k)
        V = self._empty(self.n3, k, self.n2)
        err, st = N.tsvdm_fixed_rank(self.handle, X, M, k, U, S, V, int(original_domain),
                                     rel_err, raise_on_error)
        return dict(U=U, S=S, V=V, rel_err=err, status=st)

    def tolerance(self, X, M, eps, rel_err=True, raise_on_error=True):
        """t-SVDM-II; returns ranks, offsets and packed factors sized to the total rank."""
        ranks = self._empty(self.n3, dtype=torch.int32)
        offsets = self._empty(self.n3 + 1, dtype=torch.int64)
        tot, err, st = N.tsvdm_tolerance(self.handle, X, M, eps, ranks, offsets, None, None,
                                         None, 0, rel_err, raise_on_error)
        cap = max(tot, 1)
        U = self._empty(cap, self.n1)
        S = self._empty(cap)
        V = self._empty(cap, self.n2)
        if tot > 0:
            N.tsvdm_tolerance_pack(self.handle, U, S, V, cap)
        return dict(ranks=ranks, offsets=offsets, U=U, S=S, V=V, total_rank=tot, rel_err=err,
                    status=st)

    def reconstruct(self, U, S, V, M, k=None, offsets=None, out=None):
        out = out if out is not None else self._empty(self.n3, self.n2, self.n1)
        N.tsvdm_reconstruct(self.handle, U, S, V, offsets, 0 if k is None else k, M, out)
        return out

    def backward(self, X, M, k, U, S, V, dL=1.0, dX=None, dM=None, loss="host"):
        return N.tsvdm_backward(self.handle, X, M, k, U, S, V, dL, dX, dM, loss)

    def stats(self):
        return N.tsvdm_plan_stats(self.handle)

    def last_status(self):
        return N.tsvdm_last_status(self.handle)


class TruncationLoss(torch.autograd.Function):
    """L(X, M) = sqrt(sum of discarded sigma^2 of X x_3 M at rank k) / ||X||_F with the
    library's hand-written adjoint.  The forward pass runs t-SVDM-I and the residual
    adjoint once (dL = 1), forming only the gradients that are needed (none when neither X
    nor M requires one: the loss alone); backward scales them by the upstream grad."""

    @staticmethod
    def forward(ctx, X, M, plan, k):
        f = plan.fixed_rank(X, M, k, rel_err=False)
        need_x, need_m = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dX = torch.empty_like(X) if need_x else None
        dM = torch.empty_like(M) if need_m else None
        loss = torch.zeros(1, dtype=torch.float64, device=X.device)
        plan.backward(X, M, k, f["U"], f["S"], f["V"], 1.0, dX, dM, loss)
        ctx.need = (need_x, need_m)
        ctx.save_for_backward(*[t for t in (dX, dM) if t is not None])
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        saved = list(ctx.saved_tensors)
        dX = saved.pop(0) if ctx.need[0] else None
        dM = saved.pop(0) if ctx.need[1] else None
        return (dX * g.to(dX.dtype) if dX is not None else None,
                dM * g.to(dM.dtype) if dM is not None else None, None, None)


class CayleyTransform(torch.nn.Module):
    """Orthogonal M(A) = (I + W)^{-1} (I - W) M0, W = A^T - A, parameter A (n x n, library
    layout = column-major, i.e. stored transposed in torch), A = 0 gives M0."""

    def __init__(self, M0: torch.Tensor):
        super().__init__()
        n = M0.shape[0]
        self.n = n
        self.register_buffer("M0", M0.clone())
        self.A = torch.nn.Parameter(torch.zeros_like(M0))
        self.register_buffer("Z", torch.empty_like(M0))
        self.register_buffer("Q", torch.empty_like(M0))
        self.register_buffer("work", torch.empty(3 * n * n, dtype=M0.dtype, device=M0.device))

    def forward_matrix(self, out=None):
        out = out if out is not None else torch.empty_like(self.M0)
        N.tsvdm_cayley(self.n, _DT[self.M0.dtype], self.A.detach(), self.M0, out, self.Z, self.Q,
                       self.work)
        return out

    def grad_A(self, dM, out=None):
        out = out if out is not None else torch.empty_like(self.M0)
        N.tsvdm_cayley_backward(self.n, _DT[self.M0.dtype], self.M0, self.Z, self.Q, dM, out,
                                self.work)
        return out
