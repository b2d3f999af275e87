"""Python front end of the C ABI: an ``MDS`` context object and a
``torch.autograd.Function`` over (X, sigma).

Arguments are marshalled to the C entry points (numpy arrays as host
pointers, CUDA torch tensors as device pointers); all arithmetic of the
likelihood, gradient and HMC runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi
from .capi import check

try:  # torch is plumbing (device memory, streams); the library works without it
    import torch
except ImportError:  # pragma: no cover
    torch = None


def _is_torch(a):
    return torch is not None and isinstance(a, torch.Tensor)


def _buf(a, writable=False):
    """(pointer, dtype code, where code, keepalive) for a numpy array or torch tensor."""
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if a.dtype == torch.float32:
            dt = capi.MDS_F32
        elif a.dtype == torch.float64:
            dt = capi.MDS_F64
        else:
            raise TypeError(f"unsupported dtype {a.dtype}")
        where = capi.MDS_DEVICE if a.is_cuda else capi.MDS_HOST
        return ctypes.c_void_p(a.data_ptr()), dt, where, a
    arr = np.asarray(a)
    if arr.dtype not in (np.float32, np.float64):
        arr = arr.astype(np.float64)
    if not arr.flags.c_contiguous:
        if writable:
            raise ValueError("output array must be C-contiguous")
        arr = np.ascontiguousarray(arr)
    dt = capi.MDS_F32 if arr.dtype == np.float32 else capi.MDS_F64
    return arr.ctypes.data_as(ctypes.c_void_p), dt, capi.MDS_HOST, arr


class MDS:
    """One MDS problem (N items, D latent dimensions) resident on the GPU."""

    def __init__(self, n, d, precision="fp32c", strip=None, stream=None, chunks=None):
        flags = {"fp32c": capi.MDS_PREC_FP32C, "fp64": capi.MDS_PREC_FP64}[precision]
        self._lib = capi.lib()
        h = ctypes.c_void_p()
        check(self._lib.mds_create(int(n), int(d), flags, ctypes.byref(h)), None)
        self._h = h
        self.n, self.d, self.precision = int(n), int(d), precision
        if strip is not None:
            self.set_strip(strip)
        if chunks is not None:
            # chunks per resident CTA slot, ("count", k) for exactly k chunks,
            # or ("sm", m) for m per slot in the one-CTA-per-SM grouped form
            if isinstance(chunks, tuple):
                kind = {"count": capi.MDS_PASS_CHUNK_COUNT, "sm": capi.MDS_PASS_SM_CHUNKS}[chunks[0]]
                self.set_pass_shape(kind, chunks[1])
            else:
                self.set_pass_shape(capi.MDS_PASS_CHUNKS, chunks)
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.mds_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        return check(st, self._h)

    # -- configuration
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        if stream is None:
            ptr = None
        elif torch is not None and isinstance(stream, torch.cuda.Stream):
            ptr = stream.cuda_stream
        else:
            ptr = int(stream)
        self._stream = stream  # the caller's stream object stays alive with the context
        self._check(self._lib.mds_set_stream(self._h, ctypes.c_void_p(ptr)))

    def set_data(self, y, layout="packed", ld=None):
        """y: packed strict upper triangle (M values) or full N x N matrix."""
        p, dt, where, keep = _buf(y)
        lay = {"packed": capi.MDS_Y_PACKED_UPPER, "full": capi.MDS_Y_FULL}[layout]
        if ld is None:
            ld = self.n
        self._check(self._lib.mds_set_data(self._h, p, dt, lay, int(ld), where))
        del keep

    def set_locations(self, x):
        p, dt, where, keep = _buf(x)
        self._check(self._lib.mds_set_locations(self._h, p, dt, where))

    def get_locations(self, out=None, dtype=np.float64):
        if out is None:
            out = np.empty((self.n, self.d), dtype=dtype)
        p, dt, where, keep = _buf(out, writable=True)
        self._check(self._lib.mds_get_locations(self._h, p, dt, where))
        return out

    def set_sigma(self, sigma):
        self._check(self._lib.mds_set_sigma(self._h, float(sigma)))

    def set_prior(self, lam):
        self._check(self._lib.mds_set_prior(self._h, float(lam)))

    def set_strip(self, strip):
        self._check(self._lib.mds_set_strip(self._h, int(strip)))

    def get_strip(self):
        s = ctypes.c_int32()
        self._check(self._lib.mds_get_strip(self._h, ctypes.byref(s)))
        return s.value

    def set_pass_shape(self, kind, param):
        """kind capi.MDS_PASS_STRIPS (param: tiles per strip),
        capi.MDS_PASS_CHUNKS (param: chunks per resident CTA slot),
        capi.MDS_PASS_CHUNK_COUNT (param: chunks) or capi.MDS_PASS_SM_CHUNKS
        (param: chunks per slot, one CTA per SM running its slots as groups);
        param 0 returns to the autotuner (mds_set_pass_shape)."""
        self._check(self._lib.mds_set_pass_shape(self._h, int(kind), int(param)))

    def get_pass_shape(self):
        """(kind, param, CTAs of the pass) in use."""
        k, p, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.mds_get_pass_shape(self._h, ctypes.byref(k), ctypes.byref(p), ctypes.byref(g)))
        return k.value, p.value, g.value

    def set_shard(self, n_ranks, rank, allgather, where=capi.MDS_HOST):
        """Make this context rank `rank` of `n_ranks` of a sharded evaluation
        (mds_set_shard; before set_data).  allgather(send, recv, count, where)
        gets raw addresses (ints) of the context's buffers: `count` doubles to
        send, n_ranks * count doubles to fill in rank order (host memory for
        MDS_HOST, device memory for MDS_DEVICE); it returns 0 on success."""
        def _cb(user, send, recv, count, wh):
            try:
                return int(allgather(send, recv, count, wh))
            except Exception:  # an exception must not cross the C boundary
                return -1
        self._shard_cb = capi.ALLGATHER_FN(_cb)  # kept alive with the context
        self._check(self._lib.mds_set_shard(self._h, int(n_ranks), int(rank), self._shard_cb, None, int(where)))

    def set_pass_stamps(self, on=True):
        self._check(self._lib.mds_set_pass_stamps(self._h, 1 if on else 0))

    def get_pass_span(self):
        """(passes, total milliseconds) of the pass spans since set_pass_stamps."""
        n, ms = ctypes.c_int64(), ctypes.c_double()
        self._check(self._lib.mds_get_pass_span(self._h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def reorder(self):
        """Arrange the tile layouts in the locality order of the current
        locations (mds_reorder); every array of the API keeps the item order."""
        self._check(self._lib.mds_reorder(self._h))

    def get_order(self):
        perm = np.empty(self.n, dtype=np.int32)
        self._check(self._lib.mds_get_order(self._h, perm.ctypes.data_as(ctypes.c_void_p)))
        return perm

    # -- checkpoint / resume
    def get_state(self):
        """A snapshot of the chain (bytes): locations, momenta, sigma, lambda,
        RNG counters, order (mds_get_state)."""
        n = ctypes.c_int64()
        self._check(self._lib.mds_get_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self._lib.mds_get_state(self._h, buf, ctypes.byref(n)))
        return buf.raw[:n.value]

    def set_state(self, state):
        """Restore a snapshot of get_state (mds_set_state)."""
        b = bytes(state)
        self._check(self._lib.mds_set_state(self._h, ctypes.c_char_p(b), len(b)))

    # -- single-item random-walk Metropolis (section 2.3's prior art)
    def rwmh(self, n_prop, step, seed=0, items=None, z_all=None, u_all=None):
        """n_prop single-item random-walk proposals (injected draws or
        Philox); returns (accepted[n_prop], dlogpi[n_prop])."""
        acc = np.zeros(int(n_prop), dtype=np.int32)
        dl = np.zeros(int(n_prop))
        vp = ctypes.c_void_p
        if items is not None:
            it = np.ascontiguousarray(items, dtype=np.int64)
            z = np.ascontiguousarray(z_all, dtype=np.float64)
            u = np.ascontiguousarray(u_all, dtype=np.float64)
            args = (it.ctypes.data_as(vp), z.ctypes.data_as(vp), u.ctypes.data_as(vp))
        else:
            args = (None, None, None)
        self._check(self._lib.mds_rwmh(self._h, int(n_prop), float(step), int(seed) & (2 ** 64 - 1), *args,
                                       acc.ctypes.data_as(vp), dl.ctypes.data_as(vp)))
        return acc, dl

    # -- phylogenetic Brownian-diffusion prior (section 2.2)
    def set_tree_prior(self, parent, length, sigma_mat, mu, tau0, tau_u):
        """Forest over the items (parent / length per node, -1 for roots) and
        the diffusion parameters; parent=None removes the prior."""
        if parent is None:
            self._check(self._lib.mds_set_tree_prior(self._h, 0, None, None, None, None, 1.0, 1.0))
            return
        par = np.ascontiguousarray(parent, dtype=np.int64)
        ln = np.ascontiguousarray(length, dtype=np.float64)
        sm = np.ascontiguousarray(sigma_mat, dtype=np.float64)
        mu_ = np.ascontiguousarray(mu, dtype=np.float64)
        vp = ctypes.c_void_p
        self._check(self._lib.mds_set_tree_prior(self._h, par.shape[0], par.ctypes.data_as(vp),
                                                 ln.ctypes.data_as(vp), sm.ctypes.data_as(vp),
                                                 mu_.ctypes.data_as(vp), float(tau0), float(tau_u)))

    def tree_prior(self, out=None, dtype=np.float64):
        """(log p(X), d log p / dX) of the tree prior at the current locations."""
        lp = ctypes.c_double()
        if out is None:
            out = np.empty((self.n, self.d), dtype=dtype)
        ptr, dt, where, keep = _buf(out, writable=True)
        self._check(self._lib.mds_tree_prior(self._h, ctypes.byref(lp), ptr, dt, where))
        return lp.value, out

    def pair_body_ceiling(self, far=False):
        """Pairs/s of the FP32C pass's per-pair body with its operands in
        registers (far: the body without the Phi terms); mds_pair_body_ceiling."""
        v = ctypes.c_double()
        self._check(self._lib.mds_pair_body_ceiling(self._h, 1 if far else 0, ctypes.byref(v)))
        return v.value

    def far_blocks(self):
        """(far, total) warp blocks of one evaluation pass (far: Phi terms skipped)."""
        f = ctypes.c_int64()
        t = ctypes.c_int64()
        self._check(self._lib.mds_far_blocks(self._h, ctypes.byref(f), ctypes.byref(t)))
        return f.value, t.value

    def set_tail_cutoff(self, z):
        """Phi-term cut-off z_c of the FP32C pass (0: off; else >= 8)."""
        self._check(self._lib.mds_set_tail_cutoff(self._h, float(z)))

    def problem_size(self):
        m = ctypes.c_int64()
        b = ctypes.c_int64()
        self._check(self._lib.mds_problem_size(self._h, ctypes.byref(m), ctypes.byref(b)))
        return m.value, b.value

    # -- evaluation
    def log_likelihood(self):
        """(L, sum_r) of Eq. (2) at the current locations."""
        ll = ctypes.c_double()
        sr = ctypes.c_double()
        self._check(self._lib.mds_log_likelihood(self._h, ctypes.byref(ll), ctypes.byref(sr)))
        return ll.value, sr.value

    def gradient(self, out=None, dtype=np.float64):
        """(L, dL/dX, dL/dsigma) from one fused pass.  `out` may be a numpy
        array or a (CUDA) torch tensor of shape N x D."""
        if out is None:
            out = np.empty((self.n, self.d), dtype=dtype)
        p, dt, where, keep = _buf(out, writable=True)
        ll = ctypes.c_double()
        ds = ctypes.c_double()
        self._check(self._lib.mds_gradient(self._h, ctypes.byref(ll), p, dt, where, ctypes.byref(ds)))
        return ll.value, out, ds.value

    def time_pass(self, reps=20):
        ms = ctypes.c_double()
        self._check(self._lib.mds_time_pass(self._h, int(reps), ctypes.byref(ms)))
        return ms.value

    def set_profiling(self, on=True):
        self._check(self._lib.mds_set_profiling(self._h, 1 if on else 0))

    def pass_time(self):
        """(number of timed pair-pass launches, their total ms) while profiling."""
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        self._check(self._lib.mds_get_pass_time(self._h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    # -- HMC
    def set_momentum(self, p):
        ptr, dt, where, keep = _buf(p)
        self._check(self._lib.mds_set_momentum(self._h, ptr, dt, where))

    def get_momentum(self, out=None, dtype=np.float64):
        if out is None:
            out = np.empty((self.n, self.d), dtype=dtype)
        p, dt, where, keep = _buf(out, writable=True)
        self._check(self._lib.mds_get_momentum(self._h, p, dt, where))
        return out

    def leapfrog(self, n_steps, eps, p0=None):
        """n_steps leapfrog steps in place; returns H(end) - H(start)."""
        dh = ctypes.c_double()
        if p0 is None:
            st = self._lib.mds_leapfrog(self._h, int(n_steps), float(eps), None, 0, 0, ctypes.byref(dh))
        else:
            ptr, dt, where, keep = _buf(p0)
            st = self._lib.mds_leapfrog(self._h, int(n_steps), float(eps), ptr, dt, where, ctypes.byref(dh))
        self._check(st)
        return dh.value

    def hmc(self, n_iter, n_steps, eps, seed=0, p_all=None, u_all=None):
        """n_iter HMC iterations; returns (accepted[n_iter], dH[n_iter], stats)."""
        acc = np.zeros(n_iter, dtype=np.int32)
        dh = np.zeros(n_iter, dtype=np.float64)
        stats = capi.mds_hmc_stats()
        pp = uu = None
        if p_all is not None:
            pp = np.ascontiguousarray(p_all, dtype=np.float64)
            uu = np.ascontiguousarray(u_all, dtype=np.float64)
            if pp.shape != (n_iter, self.n, self.d) or uu.shape != (n_iter,):
                raise ValueError("p_all must be n_iter x N x D and u_all n_iter")
        st = self._lib.mds_hmc(self._h, int(n_iter), int(n_steps), float(eps), int(seed) & (2**64 - 1),
                               None if pp is None else pp.ctypes.data_as(ctypes.c_void_p),
                               None if uu is None else uu.ctypes.data_as(ctypes.c_void_p),
                               acc.ctypes.data_as(ctypes.c_void_p), dh.ctypes.data_as(ctypes.c_void_p),
                               ctypes.byref(stats))
        self._check(st)
        return acc.astype(bool), dh, {"iterations": stats.iterations, "accepted": stats.accepted,
                                      "last_dh": stats.last_dh, "last_loglik": stats.last_loglik}

    # -- sigma update (random walk on log sigma, Gamma prior on sigma^-2)
    def get_sigma(self):
        v = ctypes.c_double()
        self._check(self._lib.mds_get_sigma(self._h, ctypes.byref(v)))
        return v.value

    def sigma_mh(self, n_iter, step, shape, rate, seed=0, z_all=None, u_all=None):
        """n_iter Metropolis updates of sigma given X; returns (accepted, sigma)."""
        acc = np.zeros(n_iter, dtype=np.int32)
        zz = uu = None
        if z_all is not None:
            zz = np.ascontiguousarray(z_all, dtype=np.float64)
            uu = np.ascontiguousarray(u_all, dtype=np.float64)
            if zz.shape != (n_iter,) or uu.shape != (n_iter,):
                raise ValueError("z_all and u_all must hold n_iter values each")
        self._check(self._lib.mds_sigma_mh(self._h, int(n_iter), float(step), float(shape), float(rate),
                                           int(seed) & (2**64 - 1),
                                           None if zz is None else zz.ctypes.data_as(ctypes.c_void_p),
                                           None if uu is None else uu.ctypes.data_as(ctypes.c_void_p),
                                           acc.ctypes.data_as(ctypes.c_void_p)))
        return acc.astype(bool), self.get_sigma()

    # -- cross-validation (section 2.4)
    def set_heldout(self, pairs):
        """Hold out the pairs (K x 2, any order within a pair); None or an
        empty list restores every pair."""
        if pairs is None or len(pairs) == 0:
            self._check(self._lib.mds_set_heldout(self._h, None, 0))
            return
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        self._check(self._lib.mds_set_heldout(self._h, pr.ctypes.data_as(ctypes.c_void_p), pr.shape[0]))

    def heldout_count(self):
        c = ctypes.c_int64()
        self._check(self._lib.mds_heldout_count(self._h, ctypes.byref(c)))
        return c.value

    def lpd_accumulate(self):
        """Score the current (X, sigma) as one posterior draw."""
        self._check(self._lib.mds_lpd_accumulate(self._h))

    def lpd(self):
        """(lpd-hat, draws) over the draws accumulated so far."""
        v = ctypes.c_double()
        s = ctypes.c_int64()
        self._check(self._lib.mds_lpd(self._h, ctypes.byref(v), ctypes.byref(s)))
        return v.value, s.value

    def lpd_reset(self):
        self._check(self._lib.mds_lpd_reset(self._h))

    def hmc_enqueue(self, n_iter, n_steps, eps, seed=0):
        """Queue n_iter HMC iterations on the context's stream; no waiting."""
        self._check(self._lib.mds_hmc_enqueue(self._h, int(n_iter), int(n_steps), float(eps),
                                              int(seed) & (2**64 - 1)))

    def hmc_collect(self, cap=1 << 16):
        """Wait for the queued iterations; returns (accepted, dH, stats) of
        all of them in queue order (at most `cap` entries)."""
        acc = np.zeros(cap, dtype=np.int32)
        dh = np.zeros(cap, dtype=np.float64)
        cnt = ctypes.c_int64()
        stats = capi.mds_hmc_stats()
        self._check(self._lib.mds_hmc_collect(self._h, int(cap), acc.ctypes.data_as(ctypes.c_void_p),
                                              dh.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt),
                                              ctypes.byref(stats)))
        k = min(cnt.value, cap)
        return acc[:k].astype(bool), dh[:k], {"iterations": stats.iterations, "accepted": stats.accepted,
                                              "last_dh": stats.last_dh, "last_loglik": stats.last_loglik}


def locality_order(x):
    """Locality-preserving order of the rows of x (N x D): perm[s] is the item
    at position s (mds_locality_order; host only)."""
    xa = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    n, d = xa.shape
    perm = np.empty(n, dtype=np.int32)
    capi.check(capi.lib().mds_locality_order(n, d, xa.ctypes.data_as(ctypes.c_void_p),
                                             perm.ctypes.data_as(ctypes.c_void_p)))
    return perm


def tree_plan_check(n, parent, length, d):
    """Check the per-cluster work split of the tree prior for this forest
    (mds_tree_plan_check; host only).  Returns its statistics as a dict."""
    par = np.ascontiguousarray(parent, dtype=np.int64)
    ln = np.ascontiguousarray(length, dtype=np.float64)
    st = np.zeros(8, dtype=np.int64)
    capi.check(capi.lib().mds_tree_plan_check(int(n), len(par), par.ctypes.data_as(ctypes.c_void_p),
                                              ln.ctypes.data_as(ctypes.c_void_p), int(d),
                                              st.ctypes.data_as(ctypes.c_void_p)))
    keys = ("cluster", "parts", "chain_levels", "smem_bytes", "block_roots", "max_top", "max_block_nodes", "trees")
    return dict(zip(keys, (int(v) for v in st)))


class Batch:
    """Several datasets (uneven N, same D), each with several HMC chains,
    advanced together: one batched pair pass per leapfrog step for all chains."""

    def __init__(self, ns, d, chains, stream=None, strip=None):
        self._lib = capi.lib()
        ns = np.ascontiguousarray(ns, dtype=np.int64)
        ch = np.ascontiguousarray(chains, dtype=np.int32)
        h = ctypes.c_void_p()
        st = self._lib.mds_batch_create(len(ns), ns.ctypes.data_as(ctypes.c_void_p), int(d),
                                        ch.ctypes.data_as(ctypes.c_void_p), capi.MDS_PREC_FP32C, ctypes.byref(h))
        if st != capi.MDS_OK:
            raise capi.MDSError(st, self._lib.mds_batch_last_error(None).decode(errors="replace"))
        self._h = h
        self.ns = [int(v) for v in ns]
        self.d = int(d)
        self.chains = [int(v) for v in ch]
        self.total = int(ch.sum())
        if stream is not None:
            ptr = stream.cuda_stream if (torch is not None and isinstance(stream, torch.cuda.Stream)) else int(stream)
            self._check(self._lib.mds_batch_set_stream(self._h, ctypes.c_void_p(ptr)))
        if strip is not None:
            self._check(self._lib.mds_batch_set_strip(self._h, int(strip)))

    def _check(self, st):
        if st != capi.MDS_OK:
            raise capi.MDSError(st, self._lib.mds_batch_last_error(self._h).decode(errors="replace"))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.mds_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_data(self, dataset, y, layout="packed", ld=None):
        p, dt, where, keep = _buf(y)
        lay = {"packed": capi.MDS_Y_PACKED_UPPER, "full": capi.MDS_Y_FULL}[layout]
        self._check(self._lib.mds_batch_set_data(self._h, int(dataset), p, dt, lay,
                                                 int(ld if ld is not None else self.ns[dataset]), where))

    def set_sigma(self, dataset, sigma):
        self._check(self._lib.mds_batch_set_sigma(self._h, int(dataset), float(sigma)))

    def set_locations(self, dataset, chain, x):
        p, dt, where, keep = _buf(x)
        self._check(self._lib.mds_batch_set_locations(self._h, int(dataset), int(chain), p, dt, where))

    def get_locations(self, dataset, chain, dtype=np.float64):
        out = np.empty((self.ns[dataset], self.d), dtype=dtype)
        p, dt, where, keep = _buf(out, writable=True)
        self._check(self._lib.mds_batch_get_locations(self._h, int(dataset), int(chain), p, dt, where))
        return out

    def get_gradient(self, dataset, chain, dtype=np.float64):
        out = np.empty((self.ns[dataset], self.d), dtype=dtype)
        p, dt, where, keep = _buf(out, writable=True)
        self._check(self._lib.mds_batch_get_gradient(self._h, int(dataset), int(chain), p, dt, where))
        return out

    def evaluate(self):
        """(L[g], dL/dsigma[g]) for every global chain g (dataset-major)."""
        ll = np.zeros(self.total)
        ds = np.zeros(self.total)
        self._check(self._lib.mds_batch_evaluate(self._h, ll.ctypes.data_as(ctypes.c_void_p),
                                                 ds.ctypes.data_as(ctypes.c_void_p)))
        return ll, ds

    def hmc(self, n_iter, n_steps, eps, seed=0):
        """n_iter HMC iterations for all chains; eps per dataset.  Returns
        (accepted[n_iter, total], dH[n_iter, total])."""
        e = np.ascontiguousarray(eps, dtype=np.float64)
        acc = np.zeros((n_iter, self.total), dtype=np.int32)
        dh = np.zeros((n_iter, self.total))
        self._check(self._lib.mds_batch_hmc(self._h, int(n_iter), int(n_steps), e.ctypes.data_as(ctypes.c_void_p),
                                            int(seed) & (2**64 - 1), acc.ctypes.data_as(ctypes.c_void_p),
                                            dh.ctypes.data_as(ctypes.c_void_p)))
        return acc.astype(bool), dh

    def reorder(self):
        """Locality order for every dataset (mds_batch_reorder); the arrays of
        the API stay in the caller's order."""
        self._check(self._lib.mds_batch_reorder(self._h))

    def get_strip(self):
        s = ctypes.c_int32()
        self._check(self._lib.mds_batch_get_strip(self._h, ctypes.byref(s)))
        return s.value

    def time_pass(self, reps=10):
        ms = ctypes.c_double()
        self._check(self._lib.mds_batch_time_pass(self._h, int(reps), ctypes.byref(ms)))
        return ms.value


if torch is not None:

    class MDSLogLik(torch.autograd.Function):
        """L(X, sigma) of Eq. (2) as a differentiable torch function.

        forward runs one fused pass of the library (likelihood, dL/dX and
        dL/dsigma together); backward scales the saved adjoints by the
        incoming gradient.  X: [N, D] CUDA tensor, sigma: 0-d tensor."""

        @staticmethod
        def forward(ctx, x, sigma, model):
            model.set_stream(torch.cuda.current_stream(x.device))
            model.set_locations(x.detach().contiguous())
            model.set_sigma(float(sigma))
            g = torch.empty((model.n, model.d), dtype=torch.float64, device=x.device)
            ll, _, ds = model.gradient(out=g)
            ctx.save_for_backward(g)
            ctx.ds = ds
            ctx.x_dtype = x.dtype
            ctx.s_dtype = sigma.dtype
            return torch.tensor(ll, dtype=torch.float64, device=x.device)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            gx = (gout * g).to(ctx.x_dtype)
            gs = (gout * ctx.ds).to(ctx.s_dtype)
            return gx, gs, None

    def mds_loglik(x, sigma, model):
        """Differentiable L(X, sigma); `model` is an MDS context holding Y."""
        if not torch.is_tensor(sigma):
            sigma = torch.tensor(float(sigma), dtype=torch.float64, device=x.device)
        return MDSLogLik.apply(x, sigma, model)
