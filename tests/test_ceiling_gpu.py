"""The measured ceiling of the FP32C pass's per-pair arithmetic
(mds_pair_body_ceiling): positive, the body without the Phi terms faster than
the full one, and above the rate of the pass itself (which adds loads, tile
epilogues and reductions to the same arithmetic); refused on an FP64
context and without sigma."""
import pytest

from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_STATE

pytestmark = pytest.mark.gpu


def test_ceiling_bounds_the_pass():
    from paper_1905_04582_gb300.mds import MDS
    wl = W.custom(3000, 2, sigma=0.3, seed=71, mixture=(6, 0.3))
    with MDS(wl.n, wl.d, "fp32c") as m:
        m.set_data(wl.y_packed)
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        near = m.pair_body_ceiling(far=False)
        far = m.pair_body_ceiling(far=True)
        ms = m.time_pass(10)  # caller's order: every pair takes the full body
        m_pairs = wl.n * (wl.n - 1) / 2
    print("ceiling near", near, "far", far, "pass", m_pairs / (ms / 1e3))
    assert far > near > 0
    assert m_pairs / (ms / 1e3) < near


def test_ceiling_needs_fp32c_and_sigma():
    from paper_1905_04582_gb300.mds import MDS
    with MDS(100, 2, "fp64") as m:
        m.set_sigma(0.5)
        with pytest.raises(MDSError) as e:
            m.pair_body_ceiling()
        assert e.value.status == MDS_ERR_STATE
    with MDS(100, 2, "fp32c") as m:
        with pytest.raises(MDSError) as e:
            m.pair_body_ceiling()
        assert e.value.status == MDS_ERR_STATE
