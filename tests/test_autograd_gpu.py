"""torch.autograd.Function over (X, sigma) at the paper-scale size (N = 5392,
D = 2): forward value and backward adjoints against the FP64 oracle, and
against central finite differences (h = 1e-4) of the FP64 GPU path."""
import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import workloads as W
from gpu_util import TOL, grad_check, scalar_check

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autograd_matches_oracle_and_finite_differences():
    from paper_1905_04582_gb300.mds import MDS, mds_loglik
    wl = W.paper_scale()
    x = torch.from_numpy(wl.x_eval).cuda().requires_grad_(True)
    sigma = torch.tensor(wl.sigma, dtype=torch.float32, device="cuda", requires_grad=True)
    with MDS(wl.n, wl.d, "fp32c") as m:
        m.set_data(wl.y_packed)
        ll = mds_loglik(x, sigma, m)
        ll.backward()
    x64 = wl.x_eval.astype(np.float64)
    s32 = float(np.float32(wl.sigma))
    ll_ref, _ = oracle.loglik(wl.y_packed, x64, s32, nthreads=8)
    g_ref, s_abs, s_sq = oracle.gradient(wl.y_packed, x64, s32, nthreads=8, with_abs=True, with_sq=True)
    ds_ref = oracle.dsigma(wl.y_packed, x64, s32, nthreads=8)
    tol = TOL["fp32c"]
    scalar_check(float(ll.detach()), ll_ref, tol["ll"], what="L")
    assert x.grad.dtype == torch.float32
    info = grad_check(x.grad.double().cpu().numpy(), g_ref, s_abs, tol["g"], s_sq=s_sq, u=tol["u"])
    print("autograd grad vs oracle", info)
    m_pairs = wl.n * (wl.n - 1) / 2
    scalar_check(float(sigma.grad), ds_ref, tol["g"], scale=ds_ref + 2 * m_pairs / s32, what="dL/dsigma")

    # central differences of the FP64 GPU path, h = 1e-4, on a few coordinates
    with MDS(wl.n, wl.d, "fp64") as m64:
        m64.set_data(wl.y_packed)
        m64.set_sigma(s32)
        rng = np.random.default_rng(0)
        for i, k in zip(rng.choice(wl.n, 6, replace=False), rng.integers(0, wl.d, 6)):
            vals = []
            for h in (1e-4, -1e-4):
                xp = x64.copy()
                xp[i, k] += h
                m64.set_locations(xp)
                vals.append(m64.log_likelihood()[0])
            fd = (vals[0] - vals[1]) / 2e-4
            g = float(x.grad[i, k])
            # FD truncation error ~ h^2 |L'''| and the FP32 gradient's 1e-5
            assert abs(g - fd) <= 1e-4 * abs(fd) + 1e-5 * s_abs[i, k] + 1e-3, (i, k, g, fd)
