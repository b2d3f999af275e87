"""Checkpoint and resume (mds_get_state / mds_set_state): a chain saved after
some HMC iterations and restored into a fresh context continues with the same
Philox draws and, with the same strip length and order, bitwise the same
states as the uninterrupted chain; snapshots that do not fit are rejected."""
import numpy as np
import pytest

from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_INVALID_ARG

pytestmark = pytest.mark.gpu


def model(wl, prec):
    from paper_1905_04582_gb300.mds import MDS
    m = MDS(wl.n, wl.d, prec, strip=2)
    m.set_data(wl.y_packed)
    m.set_locations(wl.x_eval)
    m.set_sigma(wl.sigma)
    return m


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("reorder", [False, True])
def test_resume_continues_the_chain_bitwise(prec, reorder):
    wl = W.custom(300, 2, sigma=0.3, seed=81, mixture=(4, 0.3))
    with model(wl, prec) as a:
        if reorder:
            a.reorder()
        a.set_strip(2)
        a.hmc(3, 10, 2e-3, seed=9)
        state = a.get_state()
        acc_a, dh_a, _ = a.hmc(3, 10, 2e-3, seed=9)
        x_a = a.get_locations()
        p_a = a.get_momentum()
    with model(wl, prec) as b:
        b.set_state(state)
        b.set_strip(2)
        acc_b, dh_b, _ = b.hmc(3, 10, 2e-3, seed=9)
        x_b = b.get_locations()
        p_b = b.get_momentum()
    assert np.array_equal(acc_a, acc_b)
    if not reorder:
        # the same order and strips: bitwise the same chain
        assert np.array_equal(dh_a, dh_b)
        assert np.array_equal(x_a, x_b) and np.array_equal(p_a, p_b)
    else:
        # the strips of a reordered context are dispatched by measured cost,
        # so sums are taken in another order: the same chain within rounding
        np.testing.assert_allclose(x_b, x_a, rtol=0, atol=1e-5 * (1 + np.abs(x_a).max()))


def test_snapshots_that_do_not_fit_are_rejected():
    wl = W.custom(120, 2, seed=82)
    other = W.custom(121, 2, seed=83)
    with model(wl, "fp32c") as a, model(other, "fp32c") as b, model(wl, "fp64") as c:
        state = a.get_state()
        for ctx, blob in ((b, state), (c, state), (a, state[:50]), (a, b"\0" * len(state))):
            with pytest.raises(MDSError) as e:
                ctx.set_state(blob)
            assert e.value.status == MDS_ERR_INVALID_ARG
        a.set_state(state)  # its own snapshot fits
