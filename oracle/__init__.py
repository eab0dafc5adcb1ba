"""Python view of the CPU oracle (plain C, FP64 / integer) for the checkerboard
single-spin-flip Metropolis method (Weigel & Yavors'kii 2011, Section 2).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously correct
restatement of the method that the CUDA library is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library under test never does.

All spin arrays are in natural order (index x + L*y (+ L*L*z)); see
``oracle/oracle.h`` for the conventions and the random-number counter layout.
"""
import ctypes
import numpy as np

from .build import build as _build

_lib = None

_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_vp = ctypes.c_void_p
_int, _u32, _u64, _i64, _dbl = (ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                ctypes.c_int64, ctypes.c_double)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build())
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_ising_init.argtypes = [_int, _int, _u64, _u32, _i8p]
        L.orc_ea_couplings.argtypes = [_int, _int, _u64, _u32, _i8p]
        L.orc_ising_measure.argtypes = [_int, _int, _dbl, _vp, _i8p,
                                        ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]
        L.orc_ising_sweeps.argtypes = [_int, _int, _dbl, _vp, _dbl, _u64, _u32, _i64, _i64,
                                       _i8p, _vp, _vp]
        L.orc_ising_heatbath_sweeps.argtypes = L.orc_ising_sweeps.argtypes
        L.orc_ising_site_update.argtypes = [_int, _int, _dbl, _vp, _dbl, _u64, _u32, _i64, _int,
                                            _i8p, _i64]
        L.orc_ising_site_update.restype = _int
        L.orc_ising_multihit_sweeps.argtypes = [_int, _int, _int, _int, _dbl, _vp, _dbl, _u64,
                                                _u32, _i64, _i64, _i8p, _vp, _vp]
        L.orc_ising_sw_sweeps.argtypes = [_int, _int, _dbl, _dbl, _u64, _u32, _i64, _i64, _i8p,
                                          _vp, _vp, _vp, _vp]
        L.orc_ising_sw_sweeps.restype = _int
        L.orc_walker_init.argtypes = [_int, _int, _int, _u64, _u32, _i8p, ctypes.POINTER(_int)]
        L.orc_walker_init.restype = _int
        L.orc_wl_sweeps.argtypes = [_int, _int, _int, _u64, _u32, _i64, _i64, _int, _int, _i8p,
                                    ctypes.POINTER(_int), _i64p, _u32p,
                                    ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_int), _dbl]
        L.orc_wl_sweeps.restype = _i64
        L.orc_muca_sweeps.argtypes = [_int, _int, _int, _f64p, _u64, _u32, _i64, _i64, _i8p,
                                      ctypes.POINTER(_int),
                                      np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")]
        L.orc_dos_glue.argtypes = [_int, _int, _i32p, _i32p, _f64p, _int,
                                   np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS"), _f64p]
        L.orc_dos_glue.restype = _int
        L.orc_xy_init.argtypes = [_int, _int, _u64, _u32, _f64p]
        L.orc_heis_init.argtypes = [_int, _int, _u64, _u32, _f64p]
        L.orc_xy_measure.argtypes = [_int, _int, _dbl, _vp, _f64p, ctypes.POINTER(_dbl), _f64p]
        L.orc_heis_measure.argtypes = [_int, _int, _dbl, _vp, _f64p, ctypes.POINTER(_dbl), _f64p]
        L.orc_xy_sweeps.argtypes = [_int, _int, _dbl, _vp, _dbl, _u64, _u32, _i64, _i64,
                                    _f64p, _vp, _vp, _dbl, _vp, _vp, _i64]
        L.orc_xy_sweeps.restype = _i64
        L.orc_heis_sweeps.argtypes = [_int, _int, _dbl, _vp, _dbl, _u64, _u32, _i64, _i64,
                                      _int, _f64p, _vp, _vp, _dbl, _vp, _vp, _i64]
        L.orc_heis_sweeps.restype = _i64
        L.orc_xy_heatbath_sweeps.argtypes = [_int, _int, _dbl, _vp, _dbl, _u64, _u32, _i64,
                                             _i64, _int, _f64p, _vp, _vp, _dbl, _vp, _i64]
        L.orc_xy_heatbath_sweeps.restype = _i64
        L.orc_heis_heatbath_sweeps.argtypes = [_int, _int, _dbl, _vp, _dbl, _u64, _u32, _i64,
                                               _i64, _int, _int, _f64p, _vp, _vp, _dbl, _vp,
                                               _i64]
        L.orc_heis_heatbath_sweeps.restype = _i64
        L.orc_ea_pt_sweeps.argtypes = [_int, _int, _i8p, _int, _f64p, _u64, _u32, _i64, _i64,
                                       _i8p, _i32p, _f64p]
        _lib = L
    return _lib


def nsites(d, L):
    return L ** d


def _ptr(a):
    return None if a is None else a.ctypes.data


def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32),
                            np.ascontiguousarray(key, np.uint32), out)
    return out


# ------------------------------------------------------------------ Ising --

def ising_init(d, L, seed, replica=0):
    s = np.empty(nsites(d, L), np.int8)
    lib().orc_ising_init(d, L, seed, replica, s)
    return s


def ea_couplings(d, L, seed, sample):
    """+-1 forward-bond couplings, shape (d, N)."""
    jb = np.empty((d, nsites(d, L)), np.int8)
    lib().orc_ea_couplings(d, L, seed, sample, jb.reshape(-1))
    return jb


def _bonds_i8(Jb, d, L):
    if Jb is None:
        return None
    jb = np.ascontiguousarray(Jb, np.int8)
    assert jb.size == d * nsites(d, L)
    return jb


def _bonds_f32(Jb, d, L):
    if Jb is None:
        return None
    jb = np.ascontiguousarray(Jb, np.float32)
    assert jb.size == d * nsites(d, L)
    return jb


def ising_measure(d, L, s, J=1.0, Jb=None):
    """(E, M) of an Ising configuration (Eq. 1)."""
    jb = _bonds_i8(Jb, d, L)
    E, M = _dbl(), _dbl()
    lib().orc_ising_measure(d, L, J, _ptr(jb), np.ascontiguousarray(s, np.int8),
                            ctypes.byref(E), ctypes.byref(M))
    return E.value, M.value


def ising_sweeps(d, L, s, beta, seed, t0, nsweeps, J=1.0, Jb=None, replica=0, series=True):
    """Run nsweeps sweeps in place on s; return (E[nsweeps], |m|[nsweeps])."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    jb = _bonds_i8(Jb, d, L)
    E = np.empty(nsweeps) if series else None
    m = np.empty(nsweeps) if series else None
    lib().orc_ising_sweeps(d, L, J, _ptr(jb), beta, seed, replica, t0, nsweeps, s,
                           _ptr(E), _ptr(m))
    return E, m


def ising_heatbath_sweeps(d, L, s, beta, seed, t0, nsweeps, J=1.0, Jb=None, replica=0,
                          series=True):
    """Heat-bath sweeps in place on s; return (E[nsweeps], |m|[nsweeps])."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    jb = _bonds_i8(Jb, d, L)
    E = np.empty(nsweeps) if series else None
    m = np.empty(nsweeps) if series else None
    lib().orc_ising_heatbath_sweeps(d, L, J, _ptr(jb), beta, seed, replica, t0, nsweeps, s,
                                    _ptr(E), _ptr(m))
    return E, m


def ising_site_updates(d, L, s, sites, beta, seed, t, J=1.0, Jb=None, replica=0,
                       heatbath=False):
    """New spins of the given sites in sweep t, each from the configuration s
    (natural order, the neighbour values its colour's update sees)."""
    jb = _bonds_i8(Jb, d, L)
    assert s.dtype == np.int8 and s.flags.c_contiguous
    f = lib().orc_ising_site_update
    return np.array([f(d, L, J, _ptr(jb), beta, seed, replica, t, int(heatbath), s, int(i))
                     for i in sites], np.int8)


def ising_multihit_sweeps(d, L, T, k, s, beta, seed, t0, nsweeps, J=1.0, Jb=None, replica=0,
                          series=True):
    """k-fold multi-hit sweeps in tiles of side T, in place on s."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    assert T % 2 == 0 and L % (2 * T) == 0
    jb = _bonds_i8(Jb, d, L)
    E = np.empty(nsweeps) if series else None
    m = np.empty(nsweeps) if series else None
    lib().orc_ising_multihit_sweeps(d, L, T, k, J, _ptr(jb), beta, seed, replica, t0, nsweeps,
                                    s, _ptr(E), _ptr(m))
    return E, m


def ising_sw_sweeps(d, L, s, beta, seed, t0, nsweeps, J=1.0, replica=0, series=True,
                    clusters=False):
    """Swendsen-Wang updates in place on s; return (E, |m|), plus, with
    clusters=True, the last update's active bonds (d, N) and cluster labels
    (smallest site of each site's cluster, N)."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    N = nsites(d, L)
    E = np.empty(nsweeps) if series else None
    m = np.empty(nsweeps) if series else None
    act = np.zeros((d, N), np.uint8) if clusters else None
    lab = np.zeros(N, np.int64) if clusters else None
    rc = lib().orc_ising_sw_sweeps(d, L, J, beta, seed, replica, t0, nsweeps, s, _ptr(E),
                                   _ptr(m), _ptr(act), _ptr(lab))
    if rc != 0:
        raise MemoryError("oracle Swendsen-Wang update: out of memory")
    if clusters:
        return E, m, act, lab
    return E, m


class Walker:
    """One windowed MUCA / Wang-Landau walker of the 2D Ising model (oracle
    state: natural-order +-1 spins, level, and the per-window arrays)."""

    def __init__(self, L, klo, khi, seed, walker):
        assert L >= 4 and L & (L - 1) == 0, "L must be a power of two"
        self.L, self.klo, self.khi, self.seed, self.walker = L, klo, khi, seed, walker
        self.K = khi - klo + 1
        self.s = np.empty(L * L, np.int8)
        lev = _int()
        rc = lib().orc_walker_init(L, klo, khi, seed, walker, self.s, ctypes.byref(lev))
        if rc != 0:
            raise RuntimeError("walker %d did not reach levels [%d, %d]" % (walker, klo, khi))
        self.level = lev.value
        self.S = np.zeros(self.K, np.int64)
        self.H = np.zeros(self.K, np.uint32)
        self.visited = 0
        self.stage = 0
        self.t = 0

    def wl(self, nsweeps, final_stage, flat_percent=80, tie_tol=0.0, seed=None):
        lev, vis, st = _int(self.level), ctypes.c_uint64(self.visited), _int(self.stage)
        ties = lib().orc_wl_sweeps(self.L, self.klo, self.khi,
                                   self.seed if seed is None else seed, self.walker, self.t,
                                   nsweeps, final_stage, flat_percent, self.s, ctypes.byref(lev),
                                   self.S, self.H, ctypes.byref(vis), ctypes.byref(st), tie_tol)
        self.level, self.visited, self.stage = lev.value, vis.value, st.value
        self.t += nsweeps
        return ties

    def muca(self, Sw, nsweeps, seed=None):
        """Multicanonical sweeps with weights Sw (ln W over the window levels);
        returns the histogram of this run."""
        Sw = np.ascontiguousarray(Sw, np.float64)
        assert Sw.size == self.K
        H = np.zeros(self.K, np.uint64)
        lev = _int(self.level)
        lib().orc_muca_sweeps(self.L, self.klo, self.khi, Sw, self.seed if seed is None else seed,
                              self.walker, self.t, nsweeps, self.s, ctypes.byref(lev), H)
        self.level = lev.value
        self.t += nsweeps
        return H


def dos_glue(N, klo, khi, S, visited):
    """Glue window estimates S[w, :] into ln g over levels 0..N (NaN where
    no window visited)."""
    klo = np.ascontiguousarray(klo, np.int32)
    khi = np.ascontiguousarray(khi, np.int32)
    S = np.ascontiguousarray(S, np.float64)
    out = np.empty(N + 1)
    rc = lib().orc_dos_glue(N, len(klo), klo, khi, S, S.shape[1],
                            np.ascontiguousarray(visited, np.uint64), out)
    if rc != 0:
        raise ValueError("windows do not share their edge levels")
    return out


# --------------------------------------------------------------- O(n) -----

def xy_init(d, L, seed, replica=0):
    th = np.empty(nsites(d, L))
    lib().orc_xy_init(d, L, seed, replica, th)
    return th


def heis_init(d, L, seed, replica=0):
    s = np.empty((nsites(d, L), 3))
    lib().orc_heis_init(d, L, seed, replica, s.reshape(-1))
    return s


def xy_measure(d, L, theta, J=1.0, Jb=None):
    jb = _bonds_f32(Jb, d, L)
    E, M = _dbl(), np.zeros(2)
    lib().orc_xy_measure(d, L, J, _ptr(jb), np.ascontiguousarray(theta, np.float64),
                         ctypes.byref(E), M)
    return E.value, M


def heis_measure(d, L, s, J=1.0, Jb=None):
    jb = _bonds_f32(Jb, d, L)
    E, M = _dbl(), np.zeros(3)
    lib().orc_heis_measure(d, L, J, _ptr(jb), np.ascontiguousarray(s, np.float64).reshape(-1),
                           ctypes.byref(E), M)
    return E.value, M


def xy_sweeps(d, L, theta, beta, seed, t0, nsweeps, J=1.0, Jb=None, replica=0,
              tie_tol=0.0, ties_cap=0, series=True, heatbath=False, colours=3, tie_info=False):
    """Sweeps (Metropolis, or heat-bath if heatbath) in place on theta; return
    (E, |m|, near-ties (k,2) array, count), and with tie_info=True (Metropolis)
    also the (k,2) array of (margin, condition factor K) of each near-tie.
    Heat-bath only: colours = 1 or 2 runs just the pass of colour 0 or 1."""
    assert theta.dtype == np.float64 and theta.flags.c_contiguous
    assert colours == 3 or heatbath
    assert not (tie_info and heatbath)
    jb = _bonds_f32(Jb, d, L)
    E = np.empty(nsweeps) if series else None
    m = np.empty(nsweeps) if series else None
    ties = np.zeros((max(ties_cap, 1), 2), np.int64)
    info = np.zeros((max(ties_cap, 1), 2)) if tie_info else None
    if heatbath:
        n = lib().orc_xy_heatbath_sweeps(d, L, J, _ptr(jb), beta, seed, replica, t0, nsweeps,
                                         colours, theta, _ptr(E), _ptr(m), tie_tol, _ptr(ties),
                                         ties_cap)
    else:
        n = lib().orc_xy_sweeps(d, L, J, _ptr(jb), beta, seed, replica, t0, nsweeps, theta,
                                _ptr(E), _ptr(m), tie_tol, _ptr(ties), _ptr(info), ties_cap)
    k = min(n, ties_cap)
    if tie_info:
        return E, m, ties[:k], n, info[:k]
    return E, m, ties[:k], n


def heis_sweeps(d, L, s, beta, seed, t0, nsweeps, J=1.0, Jb=None, replica=0,
                renorm_every=16, tie_tol=0.0, ties_cap=0, series=True, heatbath=False,
                colours=3, tie_info=False):
    """Sweeps (Metropolis, or heat-bath if heatbath) in place on s (N,3);
    return (E, |m|, near-ties (k,2) array, count), and with tie_info=True
    (Metropolis) also the (k,2) array of (margin, condition factor K) of each
    near-tie.  Heat-bath only: colours = 1 or 2 runs just the pass of colour 0
    or 1."""
    assert s.dtype == np.float64 and s.flags.c_contiguous
    assert colours == 3 or heatbath
    assert not (tie_info and heatbath)
    jb = _bonds_f32(Jb, d, L)
    E = np.empty(nsweeps) if series else None
    m = np.empty(nsweeps) if series else None
    ties = np.zeros((max(ties_cap, 1), 2), np.int64)
    info = np.zeros((max(ties_cap, 1), 2)) if tie_info else None
    if heatbath:
        n = lib().orc_heis_heatbath_sweeps(d, L, J, _ptr(jb), beta, seed, replica, t0, nsweeps,
                                           colours, renorm_every, s.reshape(-1), _ptr(E),
                                           _ptr(m), tie_tol, _ptr(ties), ties_cap)
    else:
        n = lib().orc_heis_sweeps(d, L, J, _ptr(jb), beta, seed, replica, t0, nsweeps,
                                  renorm_every, s.reshape(-1), _ptr(E), _ptr(m), tie_tol,
                                  _ptr(ties), _ptr(info), ties_cap)
    k = min(n, ties_cap)
    if tie_info:
        return E, m, ties[:k], n, info[:k]
    return E, m, ties[:k], n


# ------------------------------------------------------------ EA + PT -----

def ea_pt_sweeps(d, L, Jb, betas, seed, sample, t0, nsweeps, spins, slot_of_temp):
    """Replica-exchange sweeps of one EA sample, in place on spins (ntemps, N)
    and slot_of_temp (ntemps,); return E[nsweeps, ntemps] by temperature."""
    betas = np.ascontiguousarray(betas, np.float64)
    nt = betas.size
    assert spins.dtype == np.int8 and spins.shape == (nt, nsites(d, L))
    assert slot_of_temp.dtype == np.int32 and slot_of_temp.flags.c_contiguous
    E = np.empty((nsweeps, nt))
    lib().orc_ea_pt_sweeps(d, L, np.ascontiguousarray(Jb, np.int8).reshape(-1), nt, betas,
                           seed, sample, t0, nsweeps, spins.reshape(-1), slot_of_temp,
                           E.reshape(-1))
    return E
