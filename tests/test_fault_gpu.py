"""Failure detection without a GPU fault.  Faults are injected from the
environment (MDS_FAULT): a failing device allocation (host side), a NaN in
the scalar partials of a pass, and a device-side wait that runs out (a probe
kernel waits on an mbarrier that nothing completes; the bounded wait gives up
after one second and sets the error word).  Each call reports its status
(MDS_ERR_OOM, MDS_ERR_NONFINITE, MDS_ERR_TIMEOUT) and the context stays
usable: the next call, with the variable unset, matches the oracle."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError, MDS_ERR_NONFINITE, MDS_ERR_OOM, MDS_ERR_TIMEOUT

pytestmark = pytest.mark.gpu


class fault:
    def __init__(self, kind):
        self.kind = kind

    def __enter__(self):
        os.environ["MDS_FAULT"] = self.kind

    def __exit__(self, *exc):
        os.environ.pop("MDS_FAULT", None)


def model(wl, prec="fp32c"):
    from paper_1905_04582_gb300.mds import MDS
    m = MDS(wl.n, wl.d, prec)
    m.set_data(wl.y_packed)
    m.set_locations(wl.x_eval)
    m.set_sigma(wl.sigma)
    return m


def check_usable(m, wl, prec):
    ll, _ = m.log_likelihood()
    ref, _ = oracle.loglik(wl.y_packed, m.get_locations(), wl.sigma)
    assert math.isclose(ll, ref, rel_tol=1e-6 if prec == "fp32c" else 1e-11)


def test_allocation_failure_is_reported():
    from paper_1905_04582_gb300.mds import MDS
    wl = W.custom(150, 2, seed=91)
    with fault("alloc"):
        with pytest.raises(MDSError) as e:
            MDS(wl.n, wl.d, "fp32c")
    assert e.value.status == MDS_ERR_OOM
    with model(wl) as m:
        check_usable(m, wl, "fp32c")


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_nonfinite_partial_is_reported(prec):
    wl = W.custom(150, 2, seed=92)
    with model(wl, prec) as m:
        with fault("nan"):
            with pytest.raises(MDSError) as e:
                m.gradient()
        assert e.value.status == MDS_ERR_NONFINITE
        check_usable(m, wl, prec)


def test_device_wait_that_runs_out_is_reported():
    wl = W.custom(150, 2, seed=93)
    with model(wl) as m:
        with fault("timeout"):
            with pytest.raises(MDSError) as e:
                m.gradient()
        assert e.value.status == MDS_ERR_TIMEOUT
        check_usable(m, wl, "fp32c")
