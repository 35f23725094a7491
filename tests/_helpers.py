"""Test-side conversions between numpy complex arrays and device storage tensors."""

import numpy as np

from paper_2605_28451_gb300 import bfpfft as B


def to_device(x: np.ndarray, dtype: int, device="cuda:0"):
    """complex ndarray [..., n] -> device tensor in the storage format of `dtype`.

    F32 -> complex64; F16_* -> float16 [..., n, 2]; FP8 -> uint8 [..., n, 2]
    holding the bit patterns.  FP8 inputs must already be representable.
    """
    import torch
    x = np.asarray(x)
    if dtype == B.F32:
        return torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).to(device)
    pair = np.stack([x.real, x.imag], axis=-1)
    if dtype in (B.F16_BFP, B.F16_NAIVE):
        return torch.from_numpy(np.ascontiguousarray(pair.astype(np.float16))).to(device)
    if dtype == B.BF16:
        t = torch.from_numpy(np.ascontiguousarray(pair.astype(np.float32))).to(torch.bfloat16)
        assert np.array_equal(t.float().numpy(), pair.astype(np.float32)), "BF16 input not exactly representable"
        return t.to(device)
    f8 = torch.float8_e4m3fn if dtype == B.E4M3_BFP else torch.float8_e5m2
    t = torch.from_numpy(np.ascontiguousarray(pair.astype(np.float32))).to(f8)
    back = t.to(torch.float32).numpy()
    assert np.array_equal(back, pair.astype(np.float32)), "FP8 input not exactly representable"
    return t.view(torch.uint8).to(device)


def from_device(t, dtype: int) -> np.ndarray:
    import torch
    t = t.detach().cpu()
    if dtype == B.F32:
        return t.numpy().astype(np.complex128)
    if dtype in (B.F16_BFP, B.F16_NAIVE):
        a = t.numpy().astype(np.float64)
    elif dtype == B.BF16:
        a = t.float().numpy().astype(np.float64)
    else:
        f8 = torch.float8_e4m3fn if dtype == B.E4M3_BFP else torch.float8_e5m2
        a = t.view(f8).to(torch.float32).numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


def empty_like_storage(shape_pts, dtype: int, device="cuda:0"):
    import torch
    if dtype == B.F32:
        return torch.empty(shape_pts, dtype=torch.complex64, device=device)
    if dtype in (B.F16_BFP, B.F16_NAIVE):
        return torch.empty(tuple(shape_pts) + (2,), dtype=torch.float16, device=device)
    if dtype == B.BF16:
        return torch.empty(tuple(shape_pts) + (2,), dtype=torch.bfloat16, device=device)
    return torch.empty(tuple(shape_pts) + (2,), dtype=torch.uint8, device=device)


def storage_round(x: np.ndarray, dtype: int) -> np.ndarray:
    """The exact values a storage dtype holds for x (what the GPU receives)."""
    from oracle import quant
    if dtype == B.F32:
        return quant.round_binary32(x)
    if dtype in (B.F16_BFP, B.F16_NAIVE):
        return quant.round_binary16(x)
    if dtype == B.BF16:
        return quant.round_bfloat16(x)
    return quant.round_fp8(x, "e4m3" if dtype == B.E4M3_BFP else "e5m2")


def fp16_elementwise_ok(got: np.ndarray, ref: np.ndarray, fp32_rel: float = 1e-5):
    """FP16 output = RN-even rounding of an FP32-computed value.

    |got - ref| <= 2^-11 |ref| (half an FP16 ulp, normal range)
                 + fp32_rel * rms(ref) (FP32 arithmetic of the passes)
                 + 2^-25 (half the FP16 subnormal spacing), per component.
    Returns (ok, worst ratio of error to bound).
    """
    rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
    out = 1.0
    worst = 0.0
    for g, r in ((got.real, ref.real), (got.imag, ref.imag)):
        bound = 2.0 ** -11 * np.abs(r) * (1 + 1e-3) + fp32_rel * rms + 2.0 ** -25
        ratio = np.abs(g - r) / bound
        worst = max(worst, float(np.max(ratio)))
    return worst <= out, worst


def fp8_close(got, exact, fmt, max_frac=1e-3):
    """FP8 parity: every stored value equals the oracle's RN rounding of the
    exact FP64 value, except where the FP32 arithmetic of the GPU can put the
    value on the other side of a rounding boundary: within
    delta = 1e-5 |x| + 1e-6 rms(x) of it (relative FP32 error of the value plus
    the absolute error the passes leave on small outputs).  There one step
    either way is accepted, for at most max_frac of the points."""
    from oracle import quant
    rms = float(np.sqrt(np.mean(np.abs(exact) ** 2)))
    expect = quant.round_fp8(exact, fmt)
    for g, e, x in ((got.real, expect.real, exact.real), (got.imag, expect.imag, exact.imag)):
        bad = g != e
        if not bad.any():
            continue
        d = 1e-5 * np.abs(x[bad]) + 1e-6 * rms
        lo = quant.round_fp8(x[bad] - d, fmt)
        hi = quant.round_fp8(x[bad] + d, fmt)
        assert np.all((g[bad] == lo) | (g[bad] == hi)), (g[bad][:5], e[bad][:5], x[bad][:5])
        assert bad.mean() <= max_frac


def fp8_within(got, exact, fmt, rel, rms_frac):
    """FP8 parity of a path whose value before the final rounding may differ
    from the exact x by up to delta = rel |x| + rms_frac rms(x): rounding is
    monotonic, so every stored value lies between the oracle's roundings of
    x - delta and x + delta (equal to RN(x) unless that interval crosses a
    rounding boundary).  Returns the fraction of stored values that differ
    from RN(x)."""
    from oracle import quant
    rms = float(np.sqrt(np.mean(np.abs(exact) ** 2)))
    differ = 0
    for g, x in ((got.real, exact.real), (got.imag, exact.imag)):
        d = rel * np.abs(x) + rms_frac * rms
        lo = quant.round_fp8(x - d, fmt)
        hi = quant.round_fp8(x + d, fmt)
        assert np.all((g >= lo) & (g <= hi)), (g[(g < lo) | (g > hi)][:5], x[(g < lo) | (g > hi)][:5])
        differ += int(np.count_nonzero(g != quant.round_fp8(x, fmt)))
    return differ / (2 * got.size)
