"""torch.autograd.Functions over the differentiation entry points of libevr.

PacketSolve: u_K = S(f, lambda; u0, p0, metric), K unrolled primal-dual iterations
(Eq. cont_iterates with Eq. update_rules), forward with (u, p) checkpoints every
`every` iterations and a hand-written adjoint kernel for the backward pass.
DataImage: f = u_prev exp(Delta+ n+ - Delta- n-) (Eq. intensity_update), whose
backward gives dL/du_prev and dL/dDelta+-; passing the same tensor for Delta+ and
Delta- differentiates a single contrast threshold C.

Argument marshalling only: PyTorch allocates the outputs and the workspace, every
computation runs in the library's kernels (evr_grad.cu).  Tensors are CUDA float32,
contiguous, images (H, W) with pitch W and dual variables (3, H, W); or a batch of n
independent packets of one sensor size, images (n, H, W) and dual variables
(n, 3, H, W), solved by one call (lambda shared, its gradient summed over the batch).
"""
from __future__ import annotations

import ctypes

import torch

from . import evr as E

_f = ctypes.c_float


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc, what):
    if rc != E.EVR_OK:
        raise E.EvrError(rc, what)


def _need(t, shape, dtype=torch.float32):
    if not (t.is_cuda and t.is_contiguous() and t.dtype == dtype and tuple(t.shape) == shape):
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor of shape {shape}")


class PacketSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, lam, u0, p0, tx, ty, iters: int, every: int, tau: float, sigma: float,
                u_min: float, u_max: float):
        batched = f.dim() == 3
        n, H, W = f.shape if batched else (1,) + tuple(f.shape)
        img = (n, H, W) if batched else (H, W)
        for t in (f, u0, tx, ty):
            _need(t, img)
        _need(p0, (n, 3, H, W) if batched else (3, H, W))
        # the library's dual layout is component-major: (3, n, H, W)
        p0c = p0.transpose(0, 1).contiguous() if batched else p0
        nbytes = E._lib.evr_unrolled_workspace_bytes(W, H, W, n, int(iters), int(every))
        if nbytes == 0:
            raise ValueError("bad sizes for the unrolled solve")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=f.device)
        u_out = torch.empty_like(u0)
        p_out = torch.empty_like(p0c)
        lam_v = float(lam)
        rc = E._lib.evr_unrolled_forward(
            _ptr(tx), _ptr(ty), _ptr(f), _ptr(u0), _ptr(p0c), W, H, W, n, _f(lam_v), _f(tau),
            _f(sigma), _f(u_min), _f(u_max), int(iters), int(every), _ptr(ws), _ptr(u_out),
            _ptr(p_out), _stream())
        _check(rc, "evr_unrolled_forward")
        ctx.save_for_backward(f, tx, ty, ws)
        ctx.cfg = (W, H, n, batched, lam_v, tau, sigma, u_min, u_max, int(iters), int(every))
        ctx.lam_shape = lam.shape if torch.is_tensor(lam) else None
        return u_out, (p_out.transpose(0, 1) if batched else p_out)

    @staticmethod
    def backward(ctx, gu, gp):
        f, tx, ty, ws = ctx.saved_tensors
        W, H, n, batched, lam, tau, sigma, u_min, u_max, iters, every = ctx.cfg
        gu = torch.zeros_like(f) if gu is None else gu.contiguous()
        if gp is not None:
            gp = gp.transpose(0, 1).contiguous() if batched else gp.contiguous()
        gf = torch.empty_like(f)
        gu0 = torch.empty_like(f)
        gp0 = torch.empty((3, n, H, W) if batched else (3, H, W), dtype=torch.float32,
                          device=f.device)
        gl = torch.empty((1,), dtype=torch.float64, device=f.device)
        rc = E._lib.evr_unrolled_backward(
            _ptr(tx), _ptr(ty), _ptr(f), W, H, W, n, _f(lam), _f(tau), _f(sigma), _f(u_min),
            _f(u_max), iters, every, _ptr(ws), _ptr(gu), _ptr(gp), _ptr(gu0), _ptr(gp0),
            _ptr(gf), _ptr(gl), _stream())
        _check(rc, "evr_unrolled_backward")
        glam = gl.to(torch.float32).reshape(ctx.lam_shape) if ctx.lam_shape is not None else None
        if batched:
            gp0 = gp0.transpose(0, 1)
        return gf, glam, gu0, gp0, None, None, None, None, None, None, None, None


class DataImage(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u_prev, npos, nneg, delta_pos, delta_neg):
        shape = tuple(u_prev.shape)
        _need(u_prev, shape)
        _need(npos, shape, torch.int32)
        _need(nneg, shape, torch.int32)
        W = shape[-1]
        H = u_prev.numel() // W  # a batch (n, H, W) is n*H rows of one plane
        f = torch.empty_like(u_prev)
        dp, dn = float(delta_pos), float(delta_neg)
        rc = E._lib.evr_data_image(_ptr(u_prev), _ptr(npos), _ptr(nneg), W, H, W, _f(dp), _f(dn),
                                   _ptr(f), _stream())
        _check(rc, "evr_data_image")
        ctx.save_for_backward(f, u_prev, npos, nneg)
        ctx.deltas = (dp, dn)
        ctx.shapes = tuple(d.shape if torch.is_tensor(d) else None
                           for d in (delta_pos, delta_neg))
        return f

    @staticmethod
    def backward(ctx, gf):
        f, u_prev, npos, nneg = ctx.saved_tensors
        W = f.shape[-1]
        H = f.numel() // W
        dp, dn = ctx.deltas
        gf = gf.contiguous()
        g_uprev = torch.empty_like(u_prev)
        scratch = torch.empty(2 * H * W + 1024, dtype=torch.float64, device=f.device)
        gd = torch.empty((2,), dtype=torch.float64, device=f.device)
        rc = E._lib.evr_data_image_backward(_ptr(f), _ptr(u_prev), _ptr(npos), _ptr(nneg), W, H,
                                            W, _f(dp), _f(dn), _ptr(gf), _ptr(g_uprev),
                                            _ptr(scratch), _ptr(gd), _stream())
        _check(rc, "evr_data_image_backward")
        outs = []
        for k, shp in enumerate(ctx.shapes):
            outs.append(gd[k].to(torch.float32).reshape(shp) if shp is not None else None)
        return g_uprev, None, None, outs[0], outs[1]


def packet_solve(f, lam, u0, p0, tx, ty, iters: int, every: int = 10, tau: float | None = None,
                 sigma: float | None = None, u_min: float | None = None,
                 u_max: float | None = None):
    """Differentiable K-iteration solve of one packet, or of a batch of packets
    ((n, H, W) images); returns (u_K, p_K)."""
    d = E.evr_default_params()
    return PacketSolve.apply(f, lam, u0, p0, tx, ty, iters, every,
                             d.tau if tau is None else tau, d.sigma if sigma is None else sigma,
                             d.u_min if u_min is None else u_min,
                             d.u_max if u_max is None else u_max)


def packet_solve_many(members, lam, iters: int, every: int = 10, **kw):
    """Differentiable solves of packets of different sensor sizes: `members` is a list of
    (f, u0, p0, tx, ty) tuples ((H, W) images, (3, H, W) dual variables).  Members of one
    size are stacked and solved by one library call per size (each member's result is
    that of its own call: the stacked images are independent); returns [(u_K, p_K)] in
    the members' order.  lambda is shared, so dL/dlambda sums over every member."""
    groups = {}
    for k, m in enumerate(members):
        groups.setdefault(tuple(m[0].shape), []).append(k)
    out = [None] * len(members)
    for idx in groups.values():
        stk = [torch.stack([members[k][j] for k in idx]) for j in range(5)]
        u, p = packet_solve(stk[0], lam, stk[1], stk[2], stk[3], stk[4], iters, every, **kw)
        for b, k in enumerate(idx):
            out[k] = (u[b], p[b])
    return out


def data_image(u_prev, npos, nneg, delta_pos, delta_neg):
    """Differentiable data image of one packet or a batch of packets."""
    return DataImage.apply(u_prev, npos, nneg, delta_pos, delta_neg)
