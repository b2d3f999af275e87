"""The allocation-free entry point, mds_loglik_grad_noalloc.

It exists for callers that must not let a library allocate device memory
(a program that budgets all GPU memory itself, code inside an allocator
callback, a real-time loop past start-up).  Here it is called through the C
ABI on caller-owned device buffers, twice in a row.  Each result is checked
against the CPU oracle (L, dL/dX and dL/dsigma of Eq. (2) and (9), FP64)
with the FP64 tolerances of the parity tests, and against the library's
existing entry point (mds_gradient on an FP64 context); the second call
must reproduce the first bit for bit.  This file is collected last so that a
run stopping at the first failure has run everything else first.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300 import capi
from gpu_util import TOL, grad_check, scalar_check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _call(lib, n, d, y_dev, x_dev, sigma, g_dev):
    ll = ctypes.c_double()
    ds = ctypes.c_double()
    st = lib.mds_loglik_grad_noalloc(n, d, ctypes.c_void_p(y_dev.data_ptr()), n, ctypes.c_void_p(x_dev.data_ptr()),
                                     float(sigma), ctypes.c_void_p(g_dev.data_ptr()), ctypes.byref(ll),
                                     ctypes.byref(ds), None)
    assert st == capi.MDS_OK, lib.mds_last_error(None)
    return ll.value, ds.value


@pytest.mark.parametrize("n,d", [(700, 2), (257, 3)])
def test_noalloc_matches_context_path_twice(n, d):
    from paper_1905_04582_gb300.mds import MDS
    lib = capi.lib()
    wl = W.custom(n, d, sigma=0.5, seed=300 + n)
    x64 = wl.x_eval.astype(np.float64)
    with MDS(n, d, "fp64", strip=2) as m:
        m.set_data(wl.y_packed)
        m.set_locations(x64)
        m.set_sigma(wl.sigma)
        ll_ctx, g_ctx, ds_ctx = m.gradient()
    ll_ref, _ = oracle.loglik(wl.y_packed, x64, wl.sigma)
    g_ref, s_abs, s_sq = oracle.gradient(wl.y_packed, x64, wl.sigma, with_abs=True, with_sq=True)
    ds_ref = oracle.dsigma(wl.y_packed, x64, wl.sigma)
    y_dev = torch.from_numpy(W.packed_to_full(wl.y_packed, n)).cuda()
    x_dev = torch.from_numpy(x64).cuda()
    tol = TOL["fp64"]
    m_pairs = n * (n - 1) / 2
    results = []
    for _ in range(2):
        g_dev = torch.full((n, d), float("nan"), dtype=torch.float64, device="cuda")
        ll, ds = _call(lib, n, d, y_dev, x_dev, wl.sigma, g_dev)
        g = g_dev.cpu().numpy()
        for ref_ll, ref_g, ref_ds, who in ((ll_ref, g_ref, ds_ref, "oracle"), (ll_ctx, g_ctx, ds_ctx, "mds_gradient")):
            scalar_check(ll, ref_ll, tol["ll"], what=f"L vs {who}")
            scalar_check(ds, ref_ds, tol["g"], scale=abs(ref_ds) + 2 * m_pairs / wl.sigma,
                         what=f"dL/dsigma vs {who}")
            grad_check(g, ref_g, s_abs, tol["g"], what=f"gradient vs {who}", s_sq=s_sq, u=tol["u"])
        results.append((ll, ds, g))
    # the second call reuses the same scratch and reproduces the first bit for bit
    assert results[0][0] == results[1][0] and results[0][1] == results[1][1]
    assert np.array_equal(results[0][2], results[1][2])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = capi.lib()
    st = lib.mds_loglik_grad_noalloc(70000, 2, ctypes.c_void_p(16), 70000, ctypes.c_void_p(16), 1.0,
                                     ctypes.c_void_p(16), None, None, None)
    assert st == capi.MDS_ERR_INVALID_ARG
    assert b"exceeds the maximum" in lib.mds_last_error(None)
