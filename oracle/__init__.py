"""Serial CPU oracle of the mixed rejection KMC chain (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product library
never does.  The arithmetic lives in ``cg_oracle.c`` (plain C, binary64, no
FMA contraction); this module compiles it with gcc and exposes it through
ctypes.  Which passage of the paper each C function follows is stated in the
C file's header.

Parity status of each oracle function (what pins it, in ``tests/``):

* ``philox``            pinned: cuRAND's host-side Philox4_32_10 generator
                        (counter words 0-2, both key words) and its device
                        generator (all four counter words, on a GPU:
                        tests/test_gpu_philox_curand.py).
* ``cg_exp``            pinned: ``math.exp`` within 2 ulp over [-23, 0].
* tables / tower        pinned: closed forms (Gauss circle counts, 1/sqrt 2,
                        shell symmetry, sum of weights).
* ``eps_scratch``       pinned: a dense numpy contraction of Eq. 1's pair
                        term (a library matmul over an independently built
                        distance matrix).
* ``delta_e``           pinned: H(beta) - H(alpha) from a numpy evaluation
                        of Eq. 1.
* chain (``run``)       pinned: exact enumeration of detailed balance on an
                        N=8 ring and the L=4 torus; visit frequencies against
                        Boltzmann weights; the constant-acceptance closed
                        forms <p> = 1/[1-(1-A)^M], <m> = 1/A; the T -> infinity
                        acceptance p_theta computed by brute force.
* cubic lattice         pinned: the hop ball against a brute-force count and
  (``Chain(L, dim=3)``)  order, the 1/r table against closed forms, eps and
                        dH against numpy evaluations of Eq. 1 on the 3D
                        torus, incremental eps against scratch, detailed
                        balance over every state of two electrons on a 4^3
                        torus (tests/test_oracle_3d.py).
* stochastic time       pinned: ``log`` and ``cos2pi`` against libm,
  (``log``, ``cos2pi``,  ``gauss`` against the standard normal law (moments,
  ``gauss``,             tail mass, Kolmogorov-Smirnov distance, lag-1
  ``time_increment``)    correlation), ``time_increment`` against its closed
                        forms, a chain's time against the increments
                        recomputed from its hop log (tests/test_oracle_time.py).
* two-electron hops     pinned: ``delta_e_pair`` against numpy evaluations of
  (``set_pair``,         Eq. 1 before and after the pair move; detailed balance
  ``delta_e_pair``)      of the single + pair kernel by exact enumeration of
                        every state of three electrons on a 4 x 4 torus (and
                        its failure without the reverse-offset condition); the
                        oracle's own labels against that kernel's row
                        (chi-square); attempt-weighted Boltzmann visits;
                        incremental eps, energy and dipole against scratch;
                        p2 = 0 equal to the single-hop chain; on the cubic
                        lattice the pair dH against numpy Eq. 1, detailed
                        balance of two electrons on a 4^3 torus, and the
                        labels of a 16-electron state against its kernel row
                        (tests/test_oracle_pair.py).
* random sites          pinned: positions against the Philox definition;
  (``random_sites``)     partner lists, 1/r and dx against a numpy brute force;
                        symmetric integer weights; eps and dH against numpy
                        Eq. 1; exact detailed balance over every half-filled
                        state of 16 sites; labels against the kernel row;
                        eps and energy after a run (tests/test_oracle_random.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libcg_oracle.so")

_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_EINVAL = -1
ORC_ESTUCK = -5


def build(force: bool = False) -> str:
    """Compile ``cg_oracle.c`` into ``oracle/_build/libcg_oracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Counters(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint64), ("hops", ctypes.c_uint64),
                ("attempts", ctypes.c_uint64), ("evaluated", ctypes.c_uint64),
                ("P", ctypes.c_int64), ("energy", ctypes.c_double),
                ("time", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Hop(ctypes.Structure):
    _fields_ = [("i", ctypes.c_uint32), ("j", ctypes.c_uint32),
                ("q", ctypes.c_uint32), ("p", ctypes.c_uint32),
                ("round", ctypes.c_uint64), ("dx", ctypes.c_int32),
                ("dy", ctypes.c_int32), ("dE", ctypes.c_double),
                ("k", ctypes.c_uint32), ("l", ctypes.c_uint32),
                ("dx2", ctypes.c_int32), ("dy2", ctypes.c_int32)]


HOP_DTYPE = np.dtype([("i", "<u4"), ("j", "<u4"), ("q", "<u4"), ("p", "<u4"),
                      ("round", "<u8"), ("dx", "<i4"), ("dy", "<i4"),
                      ("dE", "<f8"), ("k", "<u4"), ("l", "<u4"),
                      ("dx2", "<i4"), ("dy2", "<i4")])
assert HOP_DTYPE.itemsize == ctypes.sizeof(Hop)


class Label(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int32), ("vec", ctypes.c_int32),
                ("i", ctypes.c_uint32), ("j", ctypes.c_uint32),
                ("dx", ctypes.c_int32), ("dy", ctypes.c_int32), ("dz", ctypes.c_int32),
                ("theta", ctypes.c_int32), ("dE", ctypes.c_double),
                ("u", ctypes.c_double), ("x", ctypes.c_uint32 * 4),
                ("pair", ctypes.c_int32), ("vec2", ctypes.c_int32),
                ("ex", ctypes.c_int32), ("ey", ctypes.c_int32), ("ez", ctypes.c_int32),
                ("k", ctypes.c_uint32), ("l", ctypes.c_uint32),
                ("dx2", ctypes.c_int32), ("dy2", ctypes.c_int32), ("dz2", ctypes.c_int32),
                ("y", ctypes.c_uint32 * 4)]


def lib():
    """Build (if needed) and load the oracle shared library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        u8p, u32p, u64p = P(ctypes.c_uint8), P(ctypes.c_uint32), P(ctypes.c_uint64)
        i32p, dp = P(ctypes.c_int32), P(ctypes.c_double)
        L.orc_philox.argtypes = [u32p, u32p, u32p]
        L.orc_philox.restype = None
        L.orc_cg_exp.argtypes = [ctypes.c_double]
        L.orc_cg_exp.restype = ctypes.c_double
        L.orc_exp_core.argtypes = [ctypes.c_double]
        L.orc_exp_core.restype = ctypes.c_double
        L.orc_new.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, ctypes.c_int,
                              ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                              ctypes.c_uint32]
        L.orc_new3.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                               ctypes.c_uint32]
        L.orc_new3.restype = ctypes.c_void_p
        L.orc_new_random.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32]
        L.orc_new_random.restype = ctypes.c_void_p
        L.orc_get_positions.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_get_positions.restype = None
        L.orc_num_pairs.argtypes = [ctypes.c_void_p]
        L.orc_num_pairs.restype = ctypes.c_int
        L.orc_get_pairs.argtypes = [ctypes.c_void_p, i32p, u32p, u64p, dp, dp]
        L.orc_get_pairs.restype = None
        L.orc_Zmax.argtypes = [ctypes.c_void_p]
        L.orc_Zmax.restype = ctypes.c_double
        L.orc_get_vectors_z.argtypes = [ctypes.c_void_p, i32p]
        L.orc_get_vectors_z.restype = None
        L.orc_tinv_of3.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_tinv_of3.restype = ctypes.c_double
        L.orc_new.restype = ctypes.c_void_p
        L.orc_free.argtypes = [ctypes.c_void_p]
        L.orc_free.restype = None
        for name in ("orc_num_vectors", "orc_num_sites"):
            getattr(L, name).argtypes = [ctypes.c_void_p]
            getattr(L, name).restype = ctypes.c_int
        for name in ("orc_Z", "orc_Gamma", "orc_energy_scratch"):
            getattr(L, name).argtypes = [ctypes.c_void_p]
            getattr(L, name).restype = ctypes.c_double
        L.orc_get_vectors.argtypes = [ctypes.c_void_p, i32p, i32p, u64p, dp]
        L.orc_get_vectors.restype = None
        L.orc_get_tinv.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_tinv.restype = None
        L.orc_tinv_of.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.orc_tinv_of.restype = ctypes.c_double
        L.orc_get_state.argtypes = [ctypes.c_void_p, u8p, dp, dp]
        L.orc_get_state.restype = None
        L.orc_set_state.argtypes = [ctypes.c_void_p, u8p, dp]
        L.orc_set_state.restype = ctypes.c_int
        L.orc_set_eps.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_eps.restype = None
        L.orc_get_counters.argtypes = [ctypes.c_void_p, P(Counters)]
        L.orc_get_counters.restype = None
        L.orc_set_counters.argtypes = [ctypes.c_void_p, P(Counters)]
        L.orc_set_counters.restype = None
        L.orc_set_toy.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
        L.orc_set_toy.restype = None
        L.orc_log.argtypes = [ctypes.c_double]
        L.orc_log.restype = ctypes.c_double
        L.orc_cos2pi.argtypes = [ctypes.c_double]
        L.orc_cos2pi.restype = ctypes.c_double
        L.orc_gauss.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
        L.orc_gauss.restype = ctypes.c_double
        L.orc_time_increment.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_double]
        L.orc_time_increment.restype = ctypes.c_double
        L.orc_set_time_mode.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_time_mode.restype = None
        L.orc_tower_many.argtypes = [ctypes.c_void_p, u32p, i32p, ctypes.c_int]
        L.orc_tower_many.restype = None
        L.orc_delta_e.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int]
        L.orc_delta_e.restype = ctypes.c_double
        L.orc_delta_e_pair.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 6
        L.orc_delta_e_pair.restype = ctypes.c_double
        L.orc_set_pair.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        L.orc_set_pair.restype = ctypes.c_int
        L.orc_pair_threshold.argtypes = [ctypes.c_void_p]
        L.orc_pair_threshold.restype = ctypes.c_uint32
        L.orc_eps_scratch.argtypes = [ctypes.c_void_p, dp]
        L.orc_eps_scratch.restype = None
        L.orc_eval_label.argtypes = [ctypes.c_void_p, ctypes.c_uint64,
                                     ctypes.c_uint32, P(Label)]
        L.orc_eval_label.restype = None
        L.orc_run.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                              ctypes.c_uint64, P(Hop)]
        L.orc_run.restype = ctypes.c_int
        _lib = L
        return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox(ctr, key):
    """Philox-4x32-10 block: ``ctr`` four uint32 words, ``key`` two."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                     _ptr(out, ctypes.c_uint32))
    return out


def cg_exp(x: float) -> float:
    """The acceptance exponential (0 below -23)."""
    return lib().orc_cg_exp(float(x))


def exp_core(x: float) -> float:
    """Cody-Waite + Taylor exp for -745 < x <= 0."""
    return lib().orc_exp_core(float(x))


def log(x: float) -> float:
    """Project natural logarithm (atanh series) of a normal x > 0."""
    return lib().orc_log(float(x))


def cos2pi(u: float) -> float:
    """cos(2 pi u) for u in [0, 1) (exact quarter reduction + Taylor)."""
    return lib().orc_cos2pi(float(u))


def gauss(seed: int, replica: int, hop: int) -> float:
    """Standard normal deviate of executed hop ``hop`` (reading R13)."""
    return lib().orc_gauss(int(seed), int(replica), int(hop))


def time_increment(Gamma: float, m: int, z: float) -> float:
    """max(0, (m + sqrt(m) z) / Gamma) (reading R13)."""
    return lib().orc_time_increment(float(Gamma), int(m), float(z))


class Chain:
    """One replica of the serial mixed-rejection chain on an Lx x Ly torus."""

    def __init__(self, Lx, Ly=None, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05,
                 E=0.0, seed=0, replica=0, Lz=1, dim=None, pair_frac=0.0, pair_rmax=0,
                 random_sites=False):
        """Lx x Ly x Lz torus; dim=3 makes the cubic lattice Lx = Ly = Lz;
        pair_frac > 0 adds two-electron hops (reading R15); random_sites puts
        N = Lx^2 sites at random positions in the Lx x Lx box (reading R16)."""
        Ly = Lx if Ly is None else Ly
        if dim == 3:
            Ly = Lz = Lx
        self._lib = lib()
        if random_sites:
            self._h = self._lib.orc_new_random(int(Lx), float(nu), float(W), float(xi),
                                               int(r_max), float(T), float(E), int(seed),
                                               int(replica))
        else:
            self._h = self._lib.orc_new3(int(Lx), int(Ly), int(Lz), float(nu), float(W),
                                         float(xi), int(r_max), float(T), float(E),
                                         int(seed), int(replica))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        if pair_frac:
            self.set_pair(pair_frac, pair_rmax)
        self.Lx, self.Ly, self.Lz = int(Lx), int(Ly), int(Lz)
        self.N = self.Lx * self.Ly * self.Lz
        self.nu, self.W, self.xi, self.r_max = nu, W, xi, r_max
        self.T, self.E, self.seed, self.replica = T, E, seed, replica

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None

    # ---- tables ----
    @property
    def V(self):
        return self._lib.orc_num_vectors(self._h)

    @property
    def Z(self):
        return self._lib.orc_Z(self._h)

    @property
    def Gamma(self):
        return self._lib.orc_Gamma(self._h)

    def vectors(self):
        V = self.V
        dx = np.zeros(V, np.int32)
        dy = np.zeros(V, np.int32)
        Wi = np.zeros(V, np.uint64)
        w = np.zeros(V, np.float64)
        self._lib.orc_get_vectors(self._h, _ptr(dx, ctypes.c_int32),
                                  _ptr(dy, ctypes.c_int32),
                                  _ptr(Wi, ctypes.c_uint64),
                                  _ptr(w, ctypes.c_double))
        return dx, dy, Wi, w

    def tower(self, x1):
        """Tower sampling (vector index, -1 for a null proposal) for words x1."""
        x1 = np.ascontiguousarray(x1, dtype=np.uint32)
        out = np.zeros(len(x1), np.int32)
        self._lib.orc_tower_many(self._h, _ptr(x1, ctypes.c_uint32), _ptr(out, ctypes.c_int32),
                                 len(x1))
        return out

    def tinv_table(self):
        """Folded 1/r table: (Ly/2+1, Lx/2+1), or (Lz/2+1, Ly/2+1, Lx/2+1) in 3D."""
        shape = (self.Ly // 2 + 1, self.Lx // 2 + 1)
        if self.Lz > 1:
            shape = (self.Lz // 2 + 1,) + shape
        t = np.zeros(shape, np.float64)
        self._lib.orc_get_tinv(self._h, _ptr(t, ctypes.c_double))
        return t

    def tinv(self, dx, dy, dz=0):
        return self._lib.orc_tinv_of3(self._h, int(dx), int(dy), int(dz))

    def positions(self):
        """Random sites (R16): the x and y positions."""
        x = np.zeros(self.N, np.float64)
        y = np.zeros(self.N, np.float64)
        self._lib.orc_get_positions(self._h, _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double))
        return x, y

    def pairs(self):
        """Random sites (R16): partner-list offsets (N + 1), partners, running
        integer weights, 1/r and the minimum-image dx of every pair."""
        M = self._lib.orc_num_pairs(self._h)
        off = np.zeros(self.N + 1, np.int32)
        j = np.zeros(max(M, 1), np.uint32)
        C = np.zeros(max(M, 1), np.uint64)
        g = np.zeros(max(M, 1), np.float64)
        dx = np.zeros(max(M, 1), np.float64)
        self._lib.orc_get_pairs(self._h, _ptr(off, ctypes.c_int32), _ptr(j, ctypes.c_uint32),
                                _ptr(C, ctypes.c_uint64), _ptr(g, ctypes.c_double),
                                _ptr(dx, ctypes.c_double))
        return off, j[:M], C[:M], g[:M], dx[:M]

    @property
    def Zmax(self):
        return self._lib.orc_Zmax(self._h)

    def vectors_z(self):
        dz = np.zeros(self.V, np.int32)
        self._lib.orc_get_vectors_z(self._h, _ptr(dz, ctypes.c_int32))
        return dz

    # ---- state ----
    def state(self):
        n = np.zeros(self.N, np.uint8)
        eps = np.zeros(self.N, np.float64)
        phi = np.zeros(self.N, np.float64)
        self._lib.orc_get_state(self._h, _ptr(n, ctypes.c_uint8),
                                _ptr(eps, ctypes.c_double),
                                _ptr(phi, ctypes.c_double))
        return n, eps, phi

    def set_state(self, n, phi=None):
        n = np.ascontiguousarray(n, dtype=np.uint8)
        if phi is not None:
            phi = np.ascontiguousarray(phi, dtype=np.float64)
            rc = self._lib.orc_set_state(self._h, _ptr(n, ctypes.c_uint8),
                                         _ptr(phi, ctypes.c_double))
        else:
            rc = self._lib.orc_set_state(self._h, _ptr(n, ctypes.c_uint8), None)
        if rc != ORC_OK:
            raise ValueError("bad occupation")

    def set_eps(self, eps):
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        self._lib.orc_set_eps(self._h, _ptr(eps, ctypes.c_double))

    def eps_scratch(self):
        out = np.zeros(self.N, np.float64)
        self._lib.orc_eps_scratch(self._h, _ptr(out, ctypes.c_double))
        return out

    def energy_scratch(self):
        return self._lib.orc_energy_scratch(self._h)

    def counters(self):
        c = Counters()
        self._lib.orc_get_counters(self._h, ctypes.byref(c))
        return c.as_dict()

    def set_counters(self, d):
        c = Counters(**d)
        self._lib.orc_set_counters(self._h, ctypes.byref(c))

    def set_time_mode(self, mode):
        """0: t = attempts / Gamma (R4, default); 1: Gaussian dt per hop (R13)."""
        self._lib.orc_set_time_mode(self._h, int(mode))

    def set_pair(self, p2, R):
        """Two-electron hops (reading R15): a fraction p2 of the labels
        proposes a pair move with offsets inside the disk of radius R."""
        if self._lib.orc_set_pair(self._h, float(p2), int(R)) != ORC_OK:
            raise ValueError("bad pair parameters")

    @property
    def pair_threshold(self):
        """T_p: a label is a pair proposal iff its word x3 < T_p."""
        return self._lib.orc_pair_threshold(self._h)

    def set_toy(self, A0=None):
        self._lib.orc_set_toy(self._h, 0 if A0 is None else 1,
                              0.0 if A0 is None else float(A0))

    # ---- physics ----
    def delta_e(self, i, j, dx):
        return self._lib.orc_delta_e(self._h, int(i), int(j), int(dx))

    def delta_e_pair(self, i, j, k, l, dx1, dx2):
        """dH of the pair hop i -> j, k -> l (reading R15)."""
        return self._lib.orc_delta_e_pair(self._h, int(i), int(j), int(k), int(l),
                                          int(dx1), int(dx2))

    def eval_label(self, rnd, k):
        lab = Label()
        self._lib.orc_eval_label(self._h, int(rnd), int(k), ctypes.byref(lab))
        return lab

    def run(self, n_hops, M, max_rounds=1 << 62, log=False):
        """Execute ``n_hops`` hops; returns (status, hop log or None)."""
        if log:
            arr = np.zeros(int(n_hops), HOP_DTYPE)
            rc = self._lib.orc_run(self._h, int(n_hops), int(M), int(max_rounds),
                                   arr.ctypes.data_as(ctypes.POINTER(Hop)))
            return rc, arr
        rc = self._lib.orc_run(self._h, int(n_hops), int(M), int(max_rounds), None)
        return rc, None
