"""Differentiable entropy autofocus: a torch.autograd.Function over the C ABI.

Forward calls ``sar_autofocus_entropy`` (image entropy E(phi) of the
azimuth-compressed, phase-corrected data; the image is never stored).
Backward calls ``sar_autofocus_grad``, the hand-written adjoint, which
recomputes the forward transforms on the GPU instead of keeping them.  Only
argument marshalling happens here.
"""

from __future__ import annotations

import torch

from . import bfpfft as B


class Workspace:
    """Device scratch for the autofocus calls at one azimuth length, and the
    arithmetic they run in (BFPFFT_ARITH_F32, or ARITH_F16_MUL_F32_ACC for the
    tensor-core transforms at n_az = 4096)."""

    def __init__(self, n_az: int, device, arith: int = B.ARITH_F32):
        self.arith = arith
        self.bytes = B.sar_autofocus_workspace_bytes(n_az)
        if self.bytes == 0:
            raise ValueError(f"unsupported azimuth length {n_az}")
        self.buf = torch.empty(self.bytes, dtype=torch.uint8, device=device)
        self.stats = torch.empty(4, dtype=torch.float64, device=device)


class SarEntropy(torch.autograd.Function):
    """E = entropy(|A(rc . exp(-j phi))|^2); d E / d phi by the GPU adjoint.

    rc: device tensor [n_rg][n_az] in storage dtype rc_dtype (complex64 for
    BFPFFT_F32, float16 [n_rg][n_az][2] for BFPFFT_F16_BFP); ha: complex64
    [n_az]; phi: float32 [n_az] (requires grad).  Returns a float64 scalar.
    """

    @staticmethod
    def forward(ctx, phi, rc, ha, rc_dtype: int, ws: Workspace):
        n_rg, n_az = rc.shape[0], rc.shape[1]
        phi_c = phi.detach().contiguous()
        B.sar_autofocus_entropy(rc, rc_dtype, phi_c, ha, n_az, n_rg, ws.stats, ws.buf, ws.bytes, arith=ws.arith)
        ctx.save_for_backward(phi_c)
        ctx.rc, ctx.ha, ctx.rc_dtype, ctx.ws = rc, ha, rc_dtype, ws
        return ws.stats[2].clone()

    @staticmethod
    def backward(ctx, g_e):
        (phi_c,) = ctx.saved_tensors
        rc, ha, ws = ctx.rc, ctx.ha, ctx.ws
        n_rg, n_az = rc.shape[0], rc.shape[1]
        grad = torch.empty(n_az, dtype=torch.float32, device=phi_c.device)
        B.sar_autofocus_grad(rc, ctx.rc_dtype, phi_c, ha, n_az, n_rg, grad, ws.stats, ws.buf, ws.bytes,
                             arith=ws.arith)
        return (g_e.to(torch.float32) * grad), None, None, None, None


def entropy(phi, rc, ha, rc_dtype: int, ws: Workspace):
    return SarEntropy.apply(phi, rc, ha, rc_dtype, ws)
