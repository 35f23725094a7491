"""bfp_sqnr_sums_noalloc: the SQNR sums computed with the library's built-in
scratch array, for callers that cannot allocate device memory or lend the
library a workspace (for example a processing chain that fixes its device
memory at start-up).

Checked through the C ABI against bfp_sqnr_sums (the workspace version) on
two calls in a row with different inputs, so the second call also shows that
what the first left in the shared array does not leak into its result.  The
tolerance is the one the metric tests use (relative 1e-10 on each sum; the
two versions add the same terms in different groupings).  This file is named
to be collected last.
"""

import numpy as np
import pytest

from paper_2605_28451_gb300 import bfpfft as B
from paper_2605_28451_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib(cuda_ready):
    build.build()
    B.lib()


def _device_pair(count, seed, dtype16):
    import torch
    g = torch.Generator(device="cuda:0").manual_seed(seed)
    ref = torch.randn(count, dtype=torch.complex64, device="cuda:0", generator=g)
    noise = torch.randn(count, dtype=torch.complex64, device="cuda:0", generator=g)
    test = 0.8 * ref + 1e-3 * noise
    if dtype16:
        test = torch.view_as_real(test).to(torch.float16).contiguous()
    return ref, test


def _with_workspace(ref, test, test_dtype, count):
    import torch
    ws_bytes = B.bfp_sqnr_workspace_bytes()
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device="cuda:0")
    out = torch.empty(8, dtype=torch.float64, device="cuda:0")
    B.bfp_sqnr_sums(ref, B.F32, test, test_dtype, count, out, ws, ws_bytes)
    return out


def test_noalloc_matches_workspace_version_twice():
    import torch
    cases = [(B.F16_BFP, 4096 * 4096, 11), (B.F32, 300001, 12)]
    outs = torch.empty((2, 8), dtype=torch.float64, device="cuda:0")
    refs = []
    for i, (dtype, count, seed) in enumerate(cases):
        ref, test = _device_pair(count, seed, dtype == B.F16_BFP)
        B.bfp_sqnr_sums_noalloc(ref, B.F32, test, dtype, count, outs[i])
        refs.append(_with_workspace(ref, test, dtype, count))
    torch.cuda.synchronize()
    for i in range(2):
        got = outs[i, :5].cpu().numpy()
        want = refs[i][:5].cpu().numpy()
        assert np.allclose(got, want, rtol=1e-10, atol=0), (i, got, want)
        assert got[4] == 0
    assert not np.allclose(outs[0, :4].cpu().numpy(), outs[1, :4].cpu().numpy())


def test_noalloc_rejects_counts_beyond_its_scratch():
    import torch
    limit = B.bfp_sqnr_sums_noalloc_max_count()
    assert limit == 4096 * 4096
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda:0")
    out = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.BfpfftError) as e:
        B.bfp_sqnr_sums_noalloc(buf, B.F32, buf, B.F32, limit + 1, out)
    assert e.value.status == B.ERR_UNSUPPORTED
