"""Sharded evaluation on one GPU, the ranks emulated by host threads of one
process (no kernel waits on another: each rank's kernels run to completion
and the exchange is a host barrier between launches).  Through the C ABI
(mds_set_shard with an all-gather among the threads), against the FP64
oracle and the unsharded library:

- every rank holds bitwise the same L, dL/dsigma and gradient after the
  exchange, within the stated tolerances of the oracle (Eq. (2), (9));
- HMC with injected draws stays identical on every rank (replicated
  updates from the combined gradient) and matches the oracle's chain;
- ranks with no tiles (more ranks than tiles), host and device exchange
  buffers, Y given on the host and on the device;
- the calls a sharded context refuses, and a failing exchange.
"""
import ctypes
import math
import threading

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import capi
from paper_1905_04582_gb300 import workloads as W
from paper_1905_04582_gb300.capi import MDSError
from test_parity_gpu import compare, oracle_ref
from test_hmc_gpu import dh_tol

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


class ThreadGather:
    """All-gather among `world` threads of this process (bounded waits)."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)
        self.slots = [None] * world

    def fn(self, rank):
        def allgather(send, recv, count, where):
            if where == capi.MDS_HOST:
                s = np.ctypeslib.as_array((ctypes.c_double * count).from_address(send)).copy()
            else:
                s = torch.as_tensor(_Dev(send, count), device="cuda").clone()
                torch.cuda.synchronize()
            self.slots[rank] = s
            self.bar.wait()
            if where == capi.MDS_HOST:
                r = np.ctypeslib.as_array((ctypes.c_double * (count * self.world)).from_address(recv))
                for k in range(self.world):
                    r[k * count:(k + 1) * count] = self.slots[k]
            else:
                r = torch.as_tensor(_Dev(recv, count * self.world), device="cuda")
                for k in range(self.world):
                    r[k * count:(k + 1) * count].copy_(self.slots[k])
                torch.cuda.synchronize()
            self.bar.wait()  # every rank has copied before the slots are reused
            return 0
        return allgather


class _Dev:
    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def sharded_model(wl, prec, world, rank, gather, where=capi.MDS_HOST, chunks=None, y_dev=None):
    from paper_1905_04582_gb300.mds import MDS
    m = MDS(wl.n, wl.d, prec, stream=torch.cuda.Stream())
    if chunks is not None:
        m.set_pass_shape(capi.MDS_PASS_CHUNK_COUNT, chunks)
    m.set_shard(world, rank, gather.fn(rank), where)
    m.set_data(y_dev if y_dev is not None else wl.y_packed)
    m.set_locations(wl.x_eval)
    m.set_sigma(wl.sigma)
    return m


def run_ranks(world, body):
    """body(rank) in one thread per rank; returns the results in rank order."""
    res, errs = [None] * world, []

    def worker(r):
        try:
            torch.cuda.set_device(0)
            res[r] = body(r)
        except BaseException as e:  # noqa: BLE001 - reported below
            errs.append(e)

    th = [threading.Thread(target=worker, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    return res


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("world,n,d,where,chunks", [(2, 700, 2, capi.MDS_HOST, None), (3, 1000, 3, capi.MDS_DEVICE, None),
                                                     (2, 333, 6, capi.MDS_HOST, 5), (5, 100, 2, capi.MDS_HOST, None)])
def test_sharded_evaluation_matches_oracle(prec, world, n, d, where, chunks):
    if prec == "fp64" and chunks is not None:
        pytest.skip("the FP64 path has the strip pass only")
    wl = W.custom(n, d, sigma=0.5, seed=700 + n + world)
    ref = oracle_ref(wl)
    gather = ThreadGather(world)

    def body(r):
        with sharded_model(wl, prec, world, r, gather, where, chunks) as m:
            info = compare(m, wl, prec, ref)
            ll, g, ds = m.gradient()
            _, yb = m.problem_size()
            return ll, g, ds, yb, info

    out = run_ranks(world, body)
    for ll, g, ds, _, _ in out[1:]:
        assert ll == out[0][0] and ds == out[0][2] and np.array_equal(g, out[0][1])
    # each rank holds about 1 / world of Y (tiles; a rank can hold none)
    tiles = ((n + 63) // 64) * ((n + 63) // 64 + 1) // 2
    assert sum(o[3] for o in out) == tiles * 16384
    print(prec, world, n, d, [o[4]["max_rel"] for o in out])


def test_sharded_y_on_device():
    wl = W.custom(600, 2, sigma=0.5, seed=9)
    ref = oracle_ref(wl)
    y_dev = torch.from_numpy(wl.y_packed).cuda()
    gather = ThreadGather(2)

    def body(r):
        with sharded_model(wl, "fp32c", 2, r, gather, y_dev=y_dev) as m:
            compare(m, wl, "fp32c", ref)
            return m.gradient()[1]

    g = run_ranks(2, body)
    assert np.array_equal(g[0], g[1])


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_sharded_hmc_replicated_and_matches_oracle(prec):
    wl = W.small()
    world, n_iter, n_steps, eps = 2, 6, 10, 1.5e-2
    p_all, u_all = W.momenta(22, n_iter, wl.n, wl.d)
    x64 = wl.x_eval.astype(np.float64)
    xr, acc_r, dh_r = oracle.hmc(wl.y_packed, x64, wl.sigma, eps, n_steps, p_all, u_all)
    gather = ThreadGather(world)

    def body(r):
        with sharded_model(wl, prec, world, r, gather) as m:
            ll0, _ = m.log_likelihood()
            acc, dh, st = m.hmc(n_iter, n_steps, eps, p_all=p_all, u_all=u_all)
            return ll0, acc, dh, m.get_locations(), m.get_momentum()

    out = run_ranks(world, body)
    for o in out[1:]:
        assert np.array_equal(o[1], out[0][1]) and np.array_equal(o[2], out[0][2])
        assert np.array_equal(o[3], out[0][3]) and np.array_equal(o[4], out[0][4])
    ll0, acc, dh, x, _ = out[0]
    tol = dh_tol(prec, ll0)
    for t in range(n_iter):
        if abs(math.log(u_all[t]) + dh_r[t]) <= 2 * tol:
            pytest.skip(f"iteration {t} falls in the tie zone")
        assert abs(dh[t] - dh_r[t]) <= tol, (t, dh[t], dh_r[t])
        assert acc[t] == acc_r[t]
    np.testing.assert_allclose(x, xr, rtol=0, atol=(2e-5 if prec == "fp32c" else 1e-11) * (1 + np.abs(xr).max()))


def test_sharded_context_refusals_and_failed_exchange():
    from paper_1905_04582_gb300.mds import MDS
    wl = W.custom(300, 2, seed=5)
    with MDS(wl.n, wl.d, "fp32c") as m:
        m.set_data(wl.y_packed)
        with pytest.raises(MDSError) as ei:
            m.set_shard(2, 0, lambda *a: 0)
        assert ei.value.status == capi.MDS_ERR_STATE  # after set_data
    with MDS(wl.n, wl.d, "fp32c") as m:
        with pytest.raises(MDSError) as ei:
            m.set_shard(2, 2, lambda *a: 0)
        assert ei.value.status == capi.MDS_ERR_INVALID_ARG
        m.set_shard(2, 1, lambda *a: 1)  # an exchange that fails
        m.set_data(wl.y_packed)
        m.set_locations(wl.x_eval)
        m.set_sigma(wl.sigma)
        with pytest.raises(MDSError) as ei:
            m.gradient()
        assert ei.value.status == capi.MDS_ERR_EXCHANGE
        with pytest.raises(MDSError) as ei:
            m.reorder()
        assert ei.value.status == capi.MDS_ERR_STATE
        with pytest.raises(MDSError) as ei:
            m.set_heldout([(0, 1)])
        assert ei.value.status == capi.MDS_ERR_STATE
