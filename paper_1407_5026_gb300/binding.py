"""ctypes binding of libcg (include/cg.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method; all steps of the chain run in libcg's kernels.  If
the library is missing the import of this module still succeeds but every
call raises: there is no CPU fallback.

``System`` is a convenience wrapper that gives the handle a torch-allocated
device workspace and the current torch stream (PyTorch supplies device memory
and streams, nothing else).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcg.so")

CG_OK, CG_EINVAL, CG_ENOMEM, CG_ECUDA, CG_ETIMEOUT, CG_ESTUCK, CG_ESTATE = 0, -1, -2, -3, -4, -5, -6
CG_FP64, CG_FP32 = 0, 1
CG_TIME_DETERMINISTIC, CG_TIME_GAUSSIAN = 0, 1
CG_SITES_LATTICE, CG_SITES_RANDOM = 0, 1
CG_REFRESH_AUTO, CG_REFRESH_FP64, CG_REFRESH_BF16X2, CG_REFRESH_FFT = 0, 1, 2, 3

EXPORTED = [
    "cg_create", "cg_create_batch", "cg_workspace_bytes", "cg_create_batch_ws",
    "cg_destroy", "cg_last_error", "cg_num_replicas", "cg_num_sites", "cg_run",
    "cg_run_async", "cg_sync", "cg_run_logged", "cg_read_state", "cg_write_state",
    "cg_observables", "cg_refresh", "cg_refresh_async", "cg_microbench",
    "cg_set_toy_acceptance", "cg_debug_philox", "cg_debug_exp", "cg_debug_tower", "cg_version",
    "cg_group_replicas", "cg_read_group_state", "cg_write_group_state", "cg_debug_gauss",
    "cg_refresh_tc_noalloc", "cg_autotune", "cg_num_groups", "cg_group_shape",
    "cg_set_trace", "cg_read_trace", "cg_eps_histogram", "cg_site_positions",
]


class CgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libcg error {code}: {msg}")
        self.code = code


class cg_replica_desc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("r_max", ctypes.c_int32),
                ("nu", ctypes.c_double), ("W", ctypes.c_double),
                ("xi", ctypes.c_double), ("T", ctypes.c_double),
                ("E", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("replica", ctypes.c_uint32), ("dim", ctypes.c_int32),
                ("sites", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class cg_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("refresh_kind", ctypes.c_int32),
                ("refresh_every", ctypes.c_uint32), ("block_threads", ctypes.c_int32),
                ("max_rounds_per_hop", ctypes.c_uint64), ("device", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("hop_timeout_ms", ctypes.c_uint32), ("cluster_size", ctypes.c_int32),
                ("time_mode", ctypes.c_int32), ("pair_rmax", ctypes.c_int32),
                ("pair_frac", ctypes.c_double)]


class cg_counters(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint64), ("hops", ctypes.c_uint64),
                ("attempts", ctypes.c_uint64), ("evaluated", ctypes.c_uint64),
                ("P", ctypes.c_int64), ("energy", ctypes.c_double), ("time", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class cg_obs(ctypes.Structure):
    _fields_ = [("c", cg_counters), ("time", ctypes.c_double), ("Gamma", ctypes.c_double),
                ("acceptance", ctypes.c_double), ("energy_per_site", ctypes.c_double),
                ("max_eps_err_last_refresh", ctypes.c_double),
                ("refreshes", ctypes.c_uint64), ("cycles_reject", ctypes.c_uint64),
                ("cycles_update", ctypes.c_uint64)]

    def as_dict(self):
        # the counters first, then the observables: "time" is the observable
        # (attempts / Gamma, or the stochastic clock)
        d = self.c.as_dict()
        d.update({f: getattr(self, f) for f, _ in self._fields_ if f != "c"})
        return d


class cg_hop(ctypes.Structure):
    _fields_ = [("i", ctypes.c_uint32), ("j", ctypes.c_uint32), ("q", ctypes.c_uint32),
                ("p", ctypes.c_uint32), ("round", ctypes.c_uint64), ("dx", ctypes.c_int32),
                ("dy", ctypes.c_int32), ("dE", ctypes.c_double), ("k", ctypes.c_uint32),
                ("l", ctypes.c_uint32), ("dx2", ctypes.c_int32), ("dy2", ctypes.c_int32)]


HOP_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("q", "<u4"), ("p", "<u4"),
                      ("round", "<u8"), ("dx", "<i4"), ("dy", "<i4"), ("dE", "<f8"),
                      ("k", "<u4"), ("l", "<u4"), ("dx2", "<i4"), ("dy2", "<i4")])


class cg_trace_point(ctypes.Structure):
    _fields_ = [("attempts", ctypes.c_uint64), ("hops", ctypes.c_uint64),
                ("P", ctypes.c_int64), ("energy", ctypes.c_double), ("time", ctypes.c_double)]


TRACE_DTYPE = np.dtype([("attempts", "<u8"), ("hops", "<u8"), ("P", "<i8"), ("energy", "<f8"),
                        ("time", "<f8")])
# layout of cg_counters, for arrays of counter records
COUNTERS_DTYPE = np.dtype([("rounds", "<u8"), ("hops", "<u8"), ("attempts", "<u8"),
                           ("evaluated", "<u8"), ("P", "<i8"), ("energy", "<f8"),
                           ("time", "<f8")])

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libcg.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libcg.so not built ({p}); run __graft_entry__.build()")
        L = ctypes.CDLL(p)
        P = ctypes.POINTER
        vp, u8p, dp, u32p = ctypes.c_void_p, P(ctypes.c_uint8), P(ctypes.c_double), P(ctypes.c_uint32)
        sig = {
            "cg_create": (vp, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64]),
            "cg_create_batch": (vp, [ctypes.c_int, P(cg_replica_desc), P(cg_opts)]),
            "cg_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, P(cg_replica_desc), P(cg_opts)]),
            "cg_create_batch_ws": (vp, [ctypes.c_int, P(cg_replica_desc), P(cg_opts), vp,
                                        ctypes.c_size_t]),
            "cg_destroy": (None, [vp]),
            "cg_last_error": (ctypes.c_char_p, []),
            "cg_num_replicas": (ctypes.c_int, [vp]),
            "cg_num_sites": (ctypes.c_int, [vp, ctypes.c_int]),
            "cg_site_positions": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_double)]),
            "cg_run": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32]),
            "cg_run_async": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32]),
            "cg_sync": (ctypes.c_int, [vp]),
            "cg_run_logged": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint32, P(cg_hop)]),
            "cg_read_state": (ctypes.c_int, [vp, ctypes.c_int, u8p, dp, dp, P(cg_counters)]),
            "cg_write_state": (ctypes.c_int, [vp, ctypes.c_int, u8p, dp, dp, P(cg_counters)]),
            "cg_observables": (ctypes.c_int, [vp, ctypes.c_int, P(cg_obs)]),
            "cg_refresh": (ctypes.c_int, [vp]),
            "cg_refresh_async": (ctypes.c_int, [vp]),
            "cg_microbench": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, dp]),
            "cg_set_toy_acceptance": (ctypes.c_int, [vp, ctypes.c_double]),
            "cg_debug_philox": (ctypes.c_int, [u32p, u32p, u32p, ctypes.c_int]),
            "cg_debug_exp": (ctypes.c_int, [dp, dp, ctypes.c_int]),
            "cg_group_replicas": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_int)]),
            "cg_debug_gauss": (ctypes.c_int, [P(ctypes.c_uint64), u32p, P(ctypes.c_uint64), dp,
                                              ctypes.c_int]),
            "cg_read_group_state": (ctypes.c_int, [vp, ctypes.c_int, u32p, vp, vp]),
            "cg_write_group_state": (ctypes.c_int, [vp, ctypes.c_int, u32p, vp, vp]),
            "cg_debug_tower": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, u32p,
                                              ctypes.POINTER(ctypes.c_int32), ctypes.c_int]),
            "cg_version": (ctypes.c_char_p, []),
            "cg_eps_histogram": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, vp]),
            "cg_refresh_tc_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                     vp, vp, vp, vp, vp]),
            "cg_autotune": (ctypes.c_int, [vp, ctypes.c_uint32]),
            "cg_set_trace": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int]),
            "cg_read_trace": (ctypes.c_int, [vp, ctypes.c_int, P(cg_trace_point), ctypes.c_int]),
            "cg_num_groups": (ctypes.c_int, [vp]),
            "cg_group_shape": (ctypes.c_int, [vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
                                              P(ctypes.c_uint), P(ctypes.c_int)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


def _check(rc, allow=()):
    if rc != CG_OK and rc not in allow:
        raise CgError(rc, cg_last_error())
    return rc


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


def desc(L, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=0, replica=0, dim=0,
         sites=0):
    return cg_replica_desc(L=L, r_max=r_max, nu=nu, W=W, xi=xi, T=T, E=E, seed=seed,
                           replica=replica, dim=dim, sites=sites)


def opts(precision=CG_FP64, refresh_every=0, refresh_kind=CG_REFRESH_AUTO, block_threads=0,
         max_rounds_per_hop=0, device=0, use_graph=0, stream=None, hop_timeout_ms=0,
         cluster_size=0, time_mode=CG_TIME_DETERMINISTIC, pair_frac=0.0, pair_rmax=0):
    return cg_opts(precision=precision, refresh_kind=refresh_kind, refresh_every=refresh_every,
                   block_threads=block_threads, max_rounds_per_hop=max_rounds_per_hop,
                   device=device, use_graph=use_graph, stream=stream,
                   hop_timeout_ms=hop_timeout_ms, cluster_size=cluster_size,
                   time_mode=time_mode, pair_rmax=pair_rmax, pair_frac=pair_frac)


# ---- the C entry points, one to one ----

def cg_last_error() -> str:
    return load().cg_last_error().decode()


def cg_version() -> str:
    return load().cg_version().decode()


def cg_create(L, nu, W, xi, r_max, T, E, seed):
    h = load().cg_create(L, nu, W, xi, r_max, T, E, seed)
    if not h:
        raise CgError(CG_EINVAL, cg_last_error())
    return h


def _descs(reps):
    arr = (cg_replica_desc * len(reps))()
    for k, r in enumerate(reps):
        arr[k] = r if isinstance(r, cg_replica_desc) else desc(**r)
    return arr


def cg_create_batch(reps, o=None):
    arr = _descs(reps)
    h = load().cg_create_batch(len(reps), arr, ctypes.byref(o) if o is not None else None)
    if not h:
        raise CgError(CG_EINVAL, cg_last_error())
    return h


def cg_workspace_bytes(reps, o=None) -> int:
    arr = _descs(reps)
    return load().cg_workspace_bytes(len(reps), arr, ctypes.byref(o) if o is not None else None)


def cg_create_batch_ws(reps, o, workspace_ptr: int, ws_bytes: int):
    arr = _descs(reps)
    h = load().cg_create_batch_ws(len(reps), arr, ctypes.byref(o) if o is not None else None,
                                  ctypes.c_void_p(workspace_ptr), ws_bytes)
    if not h:
        raise CgError(CG_EINVAL, cg_last_error())
    return h


def cg_destroy(h):
    if h:
        load().cg_destroy(h)


def cg_num_replicas(h) -> int:
    return load().cg_num_replicas(h)


def cg_num_sites(h, replica=0) -> int:
    return load().cg_num_sites(h, replica)


def cg_site_positions(h, replica=0, n_sites=None):
    """(x, y) of a random-site replica's sites (float64 arrays)."""
    N = cg_num_sites(h, replica) if n_sites is None else int(n_sites)
    x = np.zeros(max(N, 1), dtype=np.float64)
    y = np.zeros(max(N, 1), dtype=np.float64)
    _check(load().cg_site_positions(h, replica, _ptr(x, ctypes.c_double),
                                    _ptr(y, ctypes.c_double)))
    return x[:N], y[:N]


def cg_run(h, n_hops, M):
    return _check(load().cg_run(h, n_hops, M), allow=(CG_ESTUCK,))


def cg_run_async(h, n_hops, M):
    return _check(load().cg_run_async(h, n_hops, M))


def cg_sync(h):
    return _check(load().cg_sync(h), allow=(CG_ESTUCK,))


def cg_run_logged(h, n_hops, M):
    R = cg_num_replicas(h)
    log = np.zeros(R * int(n_hops), HOP_DTYPE)
    rc = load().cg_run_logged(h, n_hops, M, log.ctypes.data_as(ctypes.POINTER(cg_hop)))
    _check(rc, allow=(CG_ESTUCK,))
    return rc, log.reshape(R, int(n_hops))


def _out(spec, N, dtype):
    """True -> a new array, False/None -> skipped, an array -> used as is."""
    if isinstance(spec, np.ndarray):
        assert spec.dtype == dtype and spec.size == N and spec.flags.c_contiguous
        return spec
    return np.zeros(N, dtype) if spec else None


def cg_read_state(h, replica=0, n=True, eps=True, phi=True, counters=True):
    """Each of n / eps / phi is True (new array), False (skip) or a caller array."""
    N = cg_num_sites(h, replica)
    n_a = _out(n, N, np.uint8)
    e_a = _out(eps, N, np.float64)
    p_a = _out(phi, N, np.float64)
    c = cg_counters() if counters else None
    _check(load().cg_read_state(h, replica, _ptr(n_a, ctypes.c_uint8), _ptr(e_a, ctypes.c_double),
                                _ptr(p_a, ctypes.c_double),
                                ctypes.byref(c) if c is not None else None))
    return n_a, e_a, p_a, (c.as_dict() if c is not None else None)


def cg_write_state(h, replica, n, eps=None, phi=None, counters=None):
    n = np.ascontiguousarray(n, dtype=np.uint8)
    eps = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    phi = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    c = None if counters is None else cg_counters(
        **{f: counters.get(f, 0) for f, _ in cg_counters._fields_})
    return _check(load().cg_write_state(h, replica, _ptr(n, ctypes.c_uint8),
                                        _ptr(eps, ctypes.c_double), _ptr(phi, ctypes.c_double),
                                        ctypes.byref(c) if c is not None else None))


def cg_observables(h, replica=0) -> dict:
    o = cg_obs()
    _check(load().cg_observables(h, replica, ctypes.byref(o)))
    return o.as_dict()


def cg_refresh(h):
    return _check(load().cg_refresh(h))


def cg_refresh_async(h):
    return _check(load().cg_refresh_async(h))


def cg_microbench(kind, device=0) -> float:
    out = ctypes.c_double(0.0)
    _check(load().cg_microbench(kind, device, ctypes.byref(out)))
    return out.value


def cg_refresh_tc_noalloc(L, R, nu, occ_ptr, phi_ptr, eps_ptr, max_err_ptr=None, stream=None):
    """Device pointers (ints) in, CG status out; raises on error."""
    return _check(load().cg_refresh_tc_noalloc(
        L, R, nu, ctypes.c_void_p(occ_ptr), ctypes.c_void_p(phi_ptr), ctypes.c_void_p(eps_ptr),
        ctypes.c_void_p(max_err_ptr) if max_err_ptr else None,
        ctypes.c_void_p(stream) if stream else None))


def cg_set_trace(h, first_time, points_per_decade=8.0, capacity=256):
    return _check(load().cg_set_trace(h, first_time, points_per_decade, capacity))


def cg_read_trace(h, replica=0, capacity=256):
    out = np.zeros(capacity, TRACE_DTYPE)
    n = load().cg_read_trace(h, replica, out.ctypes.data_as(ctypes.POINTER(cg_trace_point)),
                             capacity)
    _check(n if n < 0 else CG_OK)
    return out[:n]


def cg_autotune(h, hops_per_trial=0):
    return _check(load().cg_autotune(h, hops_per_trial))


def cg_num_groups(h) -> int:
    return load().cg_num_groups(h)


def cg_group_shape(h, index):
    L, t, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    M = ctypes.c_uint()
    _check(load().cg_group_shape(h, index, ctypes.byref(L), ctypes.byref(t), ctypes.byref(M),
                                 ctypes.byref(c)))
    return {"L": L.value, "threads": t.value, "M": M.value, "cluster": c.value}


def cg_set_toy_acceptance(h, A0):
    return _check(load().cg_set_toy_acceptance(h, A0))


def cg_debug_philox(ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    _check(load().cg_debug_philox(_ptr(ctr, ctypes.c_uint32), _ptr(key, ctypes.c_uint32),
                                  _ptr(out, ctypes.c_uint32), len(ctr)))
    return out


def cg_debug_gauss(seed, replica, hops):
    seed = np.ascontiguousarray(seed, dtype=np.uint64)
    replica = np.ascontiguousarray(replica, dtype=np.uint32)
    hops = np.ascontiguousarray(hops, dtype=np.uint64)
    out = np.zeros(len(hops), np.float64)
    _check(load().cg_debug_gauss(_ptr(seed, ctypes.c_uint64), _ptr(replica, ctypes.c_uint32),
                                 _ptr(hops, ctypes.c_uint64), _ptr(out, ctypes.c_double), len(hops)))
    return out


def cg_debug_exp(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    _check(load().cg_debug_exp(_ptr(x, ctypes.c_double), _ptr(out, ctypes.c_double), len(x)))
    return out


def cg_group_replicas(h, group):
    """Replica indices of a group (the replicas with its L and dimension)."""
    out = np.zeros(max(cg_num_replicas(h), 1), np.int32)
    n = load().cg_group_replicas(h, group, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if n < 0:
        raise CgError(n, cg_last_error())
    return out[:n].copy()


def group_dims(h, group):
    """(replica indices, sites N, bitmask words per replica) of one group."""
    reps = cg_group_replicas(h, group)
    N = cg_num_sites(h, int(reps[0]))
    return reps, N, (N + 31) // 32


def _vp(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def cg_read_group_state(h, group, occ=True, eps=True, counters=True, precision=None, dims=None):
    """Whole-group state: occ (count, words) uint32, eps (count, N) in the
    handle's precision (pass `precision`; float64 is assumed otherwise) and
    the counters as a COUNTERS_DTYPE array.  Caller arrays (e.g. pinned) are
    filled in place; False skips an array; `dims` is group_dims(h, group)."""
    idx, N, words = dims if dims is not None else group_dims(h, group)
    cnt = len(idx)
    dt = np.float32 if precision == CG_FP32 else np.float64
    pick = lambda a, shape, d: a if isinstance(a, np.ndarray) else (np.zeros(shape, d) if a else None)
    o = pick(occ, (cnt, words), np.uint32)
    e = pick(eps, (cnt, N), dt)
    c = pick(counters, cnt, COUNTERS_DTYPE)
    for a, size in ((o, cnt * words), (e, cnt * N), (c, cnt)):
        assert a is None or (a.size == size and a.flags.c_contiguous)
    assert c is None or c.dtype == COUNTERS_DTYPE
    _check(load().cg_read_group_state(h, group, _ptr(o, ctypes.c_uint32), _vp(e), _vp(c)))
    return o, e, c


def cg_write_group_state(h, group, occ=None, eps=None, counters=None, dims=None):
    idx, N, words = dims if dims is not None else group_dims(h, group)
    cnt = len(idx)
    if occ is not None:
        assert occ.dtype == np.uint32 and occ.size == cnt * words and occ.flags.c_contiguous
    if eps is not None:
        assert eps.size == cnt * N and eps.flags.c_contiguous
    if counters is not None:
        counters = np.ascontiguousarray(counters, dtype=COUNTERS_DTYPE)
        assert counters.size == cnt
    return _check(load().cg_write_group_state(h, group, _ptr(occ, ctypes.c_uint32), _vp(eps),
                                              _vp(counters)))


def cg_debug_tower(h, replica, x1):
    x1 = np.ascontiguousarray(x1, dtype=np.uint32)
    out = np.zeros(len(x1), dtype=np.int32)
    _check(load().cg_debug_tower(h, replica, _ptr(x1, ctypes.c_uint32),
                                 _ptr(out, ctypes.c_int32), len(x1)))
    return out


def cg_eps_histogram(h, first, count, nbins, lo, hi, counts_dev_ptr):
    """Add the g(eps) counts of replicas first..first+count-1 to the device
    array of nbins uint64 at counts_dev_ptr (enqueued; cg_sync to read)."""
    return _check(load().cg_eps_histogram(h, int(first), int(count), int(nbins), float(lo),
                                          float(hi), ctypes.c_void_p(int(counts_dev_ptr))))


class System:
    """Owns one libcg handle over R replicas, with device memory and the
    stream supplied by PyTorch."""

    def __init__(self, reps, precision=CG_FP64, refresh_every=0, refresh_kind=CG_REFRESH_AUTO,
                 block_threads=0, max_rounds_per_hop=0, device=0, torch_memory=True,
                 hop_timeout_ms=0, cluster_size=0, use_graph=0, time_mode=0, pair_frac=0.0,
                 pair_rmax=0):
        import torch
        self.reps = [r if isinstance(r, dict) else r for r in reps]
        torch.cuda.set_device(device)
        # a dedicated torch stream: libcg launches on it, callers can record
        # torch events on it
        self.stream = torch.cuda.Stream(device)
        self.opts = opts(precision=precision, refresh_every=refresh_every,
                         refresh_kind=refresh_kind, block_threads=block_threads,
                         max_rounds_per_hop=max_rounds_per_hop, device=device,
                         stream=self.stream.cuda_stream, hop_timeout_ms=hop_timeout_ms,
                         cluster_size=cluster_size, use_graph=use_graph, time_mode=time_mode,
                         pair_frac=pair_frac, pair_rmax=pair_rmax)
        self.workspace = None
        self.device = device
        if torch_memory:
            nbytes = cg_workspace_bytes(self.reps, self.opts)
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{device}")
            base = self.workspace.data_ptr()
            aligned = (base + 255) & ~255
            self.h = cg_create_batch_ws(self.reps, self.opts, aligned, nbytes + 256 - (aligned - base))
        else:
            self.h = cg_create_batch(self.reps, self.opts)
        self.R = cg_num_replicas(self.h)

    def close(self):
        if getattr(self, "h", None):
            cg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, n_hops, M):
        return cg_run(self.h, n_hops, M)

    def run_logged(self, n_hops, M):
        return cg_run_logged(self.h, n_hops, M)

    def state(self, replica=0):
        return cg_read_state(self.h, replica)

    def observables(self, replica=0):
        return cg_observables(self.h, replica)

    def eps_histogram(self, nbins, lo, hi, first=0, count=None, counts=None):
        """g(eps) counts of the replicas as a device int64 tensor (uint64
        bits); pass ``counts`` to keep adding snapshots into the same one."""
        import torch
        if count is None:
            count = len(self.reps) - first
        if counts is None:
            counts = torch.zeros(int(nbins), dtype=torch.int64, device=f"cuda:{self.device}")
        cg_eps_histogram(self.h, first, count, nbins, lo, hi, counts.data_ptr())
        cg_sync(self.h)
        return counts

    def group_dims(self, group):
        if not hasattr(self, "_dims"):
            self._dims = {}
        if group not in self._dims:
            self._dims[group] = group_dims(self.h, group)
        return self._dims[group]

    def read_group(self, group, occ=True, eps=True, counters=True):
        return cg_read_group_state(self.h, group, occ, eps, counters,
                                   precision=self.opts.precision, dims=self.group_dims(group))

    def write_group(self, group, occ=None, eps=None, counters=None):
        return cg_write_group_state(self.h, group, occ, eps, counters,
                                    dims=self.group_dims(group))
