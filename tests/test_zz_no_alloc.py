"""svgd_step_noalloc: the SVGD update for callers that cannot allocate GPU
memory (a plug-in handed device pointers but no allocator, a process whose
device memory is owned by another framework's pool, a loop that must not
call cudaMalloc/cudaFree). Its scratch is the library's fixed device array,
so this file checks, through the C ABI, that two calls in a row give the
results of svgd_step with a caller workspace (to the 1e-5 relative L2 used by
the other SVGD parity tests), and that a problem larger than the array is
refused without touching the GPU. The file name sorts last so that a run
stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2310_13325_gb300 as vg
from paper_2310_13325_gb300 import _lib

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _rel(a, b):
    return float((a - b).double().norm() / b.double().norm())


@pytest.fixture(scope="module")
def lib():
    from paper_2310_13325_gb300 import build
    build.build()
    return _lib.load()


@pytest.mark.parametrize("n,d,gp,bounded", [(40, 5000, vg.VIP_GRAM_BF16X3, False),
                                            (8, 4096, vg.VIP_GRAM_BF16X3, True),
                                            (33, 1003, vg.VIP_GRAM_FP32, False)])
def test_noalloc_matches_workspace_version_on_two_calls(lib, n, d, gp, bounded):
    g = torch.Generator(device=DEV).manual_seed(n * 7 + d)
    X = torch.randn((n, d), generator=g, device=DEV)
    G = torch.randn((n, d), generator=g, device=DEV)
    lo = hi = None
    if bounded:
        lo = torch.full((d,), -1.5, device=DEV)
        hi = torch.full((d,), 1.5, device=DEV)
    eps = 50.0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    X_ref = X.clone()
    X_new = X.clone()
    for call in range(2):
        h_ref = torch.empty(1, dtype=torch.float64, device=DEV)
        h_new = torch.empty(1, dtype=torch.float64, device=DEV)
        vg.svgd_step(X_ref, G, eps, lo=lo, hi=hi, gram_precision=gp, h2_used=h_ref,
                     gscale=-1.0)
        rc = lib.svgd_step_noalloc(_p(X_new), _p(G), -1.0, n, d, eps, 0.0, _p(lo), _p(hi),
                                   gp, _p(h_new), stream)
        assert rc == 0, lib.vip_strerror(rc)
        torch.cuda.synchronize()
        assert torch.isfinite(X_new).all()
        assert _rel(X_new, X_ref) <= 1e-5, (call, _rel(X_new, X_ref))
        assert abs(h_new.item() - h_ref.item()) <= 1e-12 * h_ref.item()


def test_noalloc_refuses_problems_larger_than_its_array(lib):
    # 600 x 36000 needs far more than the fixed array; refused before any
    # device call, so null pointers are never dereferenced
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.svgd_step_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 1.0, 600, 36000,
                               0.1, 0.0, None, None, vg.VIP_GRAM_BF16X3, None, stream)
    assert rc == -3
    assert lib.svgd_workspace_size(600, 36000, vg.VIP_GRAM_BF16X3, 0) > (64 << 20)
