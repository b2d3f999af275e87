"""Sharded evaluation (section 2.5 of arXiv:1905.04582: the pairwise sum
split over workers, the partial sums reduced) on the CPU, without a GPU.

- The split (mds_shard_range): contiguous tile ranges that cover the tiles
  once, each holding M / n_ranks pairs to within one tile.
- The fixed-order combine (mds_shard_sum): rank 0 first, as a plain loop.
- Two gloo ranks: each computes the oracle's partials {L_r, dL/dsigma_r,
  sum r_r, dL/dX_r} over the pairs of its tile range, the partial vectors are
  all-gathered through the library's torch.distributed adapter
  (shard.torch_allgather, host buffers) and summed by mds_shard_sum.  Both
  ranks must hold bitwise the same totals, equal to the same sum formed in
  one process, and the totals must match the unsharded oracle.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1905_04582_gb300 import shard
from paper_1905_04582_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def tile_pairs(n):
    """Pairs in each tile (row-block order), from the tile geometry."""
    nt = (n + 63) // 64
    out = []
    for i in range(nt):
        r = min(64, n - 64 * i)
        for j in range(i, nt):
            c = min(64, n - 64 * j)
            out.append(r * (r - 1) // 2 if i == j else r * c)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("n", [2, 3, 65, 100, 300, 1000, 5392, 20000])
@pytest.mark.parametrize("g", [1, 2, 3, 4, 7, 16])
def test_split_covers_tiles_with_equal_pair_counts(n, g):
    tp = tile_pairs(n)
    m = n * (n - 1) // 2
    assert tp.sum() == m
    ranges = [shard.shard_range(n, g, r) for r in range(g)]
    assert ranges[0][0] == 0 and ranges[-1][1] == len(tp)
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0 and a0 <= a1
    counts = [int(tp[t0:t1].sum()) for t0, t1 in ranges]
    assert sum(counts) == m
    # every rank's share within one tile of M / g (the cut is at tile edges)
    for c in counts:
        assert abs(c - m / g) <= tp.max() + 1, (counts, m / g)


def test_fixed_order_sum():
    rng = np.random.default_rng(3)
    gathered = rng.standard_normal((5, 1000)) * np.logspace(-8, 8, 1000)
    want = gathered[0].copy()
    for r in range(1, 5):
        want += gathered[r]
    assert np.array_equal(shard.shard_sum(gathered), want)


def shard_keep(n, t0, t1):
    """Packed-pair mask of the pairs in tiles [t0, t1)."""
    nt = (n + 63) // 64
    iu, ju = np.triu_indices(n, 1)
    bi, bj = iu // 64, ju // 64
    t = bi * nt - bi * (bi - 1) // 2 + (bj - bi)
    return ((t >= t0) & (t < t1)).astype(np.uint8)


def oracle_partials(wl, keep):
    """{L_r, dL/dsigma_r, sum r_r, dL/dX_r} over the kept pairs (L_r with
    M_r = the kept count, as a shard's reduction forms it)."""
    x = wl.x_eval.astype(np.float64)
    ll, sr = oracle.loglik(wl.y_packed, x, wl.sigma, keep=keep)
    ds = oracle.dsigma(wl.y_packed, x, wl.sigma, keep=keep)
    g = oracle.gradient(wl.y_packed, x, wl.sigma, keep=keep)
    return np.concatenate([[ll, ds, sr], g.ravel()])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np
import torch.distributed as dist
from paper_1905_04582_gb300 import capi, shard
from paper_1905_04582_gb300 import workloads as W
import test_shard_cpu as T
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo")
wl = W.custom({n}, {d}, sigma=0.4, seed=41, mixture=(4, 0.3))
t0, t1 = shard.shard_range(wl.n, world, rank)
send = T.oracle_partials(wl, T.shard_keep(wl.n, t0, t1))
recv = np.zeros(world * send.size)
ag = shard.torch_allgather()
assert ag(send.ctypes.data, recv.ctypes.data, send.size, capi.MDS_HOST) == 0
total = shard.shard_sum(recv.reshape(world, -1))
np.save(os.path.join({tmp!r}, f"total{{rank}}.npy"), total)
np.save(os.path.join({tmp!r}, f"gathered{{rank}}.npy"), recv)
print("OUT " + json.dumps(dict(rank=rank, t0=t0, t1=t1)), flush=True)
dist.destroy_process_group()
"""


@pytest.mark.parametrize("world,n,d", [(2, 300, 2), (2, 257, 3), (3, 200, 2)])
def test_gloo_ranks_exchange_and_combine(tmp_path, world, n, d):
    port = _free_port()
    code = _WORKER.format(root=ROOT, tmp=str(tmp_path), n=n, d=d)
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True, env=env, cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=240)
        assert p.returncode == 0, e[-3000:]
        outs.append([json.loads(ln[4:]) for ln in o.splitlines() if ln.startswith("OUT ")][0])
    totals = [np.load(tmp_path / f"total{r}.npy") for r in range(world)]
    # every rank holds bitwise the same totals
    for t in totals[1:]:
        assert np.array_equal(t, totals[0])
    # the same partials and fixed-order sum formed in one process
    wl = W.custom(n, d, sigma=0.4, seed=41, mixture=(4, 0.3))
    parts = np.stack([oracle_partials(wl, shard_keep(n, o["t0"], o["t1"])) for o in sorted(outs, key=lambda o: o["rank"])])
    assert np.array_equal(np.load(tmp_path / "gathered0.npy").reshape(world, -1), parts)
    assert np.array_equal(totals[0], shard.shard_sum(parts))
    # and the totals are the unsharded evaluation (FP64, another summation order)
    x = wl.x_eval.astype(np.float64)
    ll, sr = oracle.loglik(wl.y_packed, x, wl.sigma)
    ds = oracle.dsigma(wl.y_packed, x, wl.sigma)
    g = oracle.gradient(wl.y_packed, x, wl.sigma)
    tot = totals[0]
    np.testing.assert_allclose(tot[0], ll, rtol=1e-12)
    np.testing.assert_allclose(tot[1], ds, rtol=1e-11, atol=1e-9 * n * n)
    np.testing.assert_allclose(tot[2], sr, rtol=1e-12)
    np.testing.assert_allclose(tot[3:].reshape(n, d), g, rtol=1e-10, atol=1e-10 * np.abs(g).max())
